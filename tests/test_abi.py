"""The C-ABI library builds for sm_103a, loads, and exports every entry point of
include/lqcd.h; argument validation happens before any device call (CPU only)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0911_2285_gb300.build import build
    return build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lqcd_eigbicg_init", "lqcd_solve", "lqcd_deflate", "lqcd_eigs", "lqcd_apply", "lqcd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lqcd_[a-z_0-9]+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    lib = C.CDLL(libpath)
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_status_strings(libpath):
    from paper_0911_2285_gb300 import lqcd as L
    assert L.status_str(L.OK) == "ok"
    assert "argument" in L.status_str(L.ERR_ARG)


@pytest.mark.parametrize("bad", [dict(m=16, nev=8), dict(dims=(1, 4, 4, 4)), dict(tol=0.0), dict(k_max=9),
                                 dict(kappa=-1.0), dict(m=80), dict(n_def_max=200),
                                 dict(dims=(4, 4, 3, 4), evenodd=True), dict(evenodd=True, gamma5=True),
                                 dict(gamma5=True, bicgstab=True)])
def test_init_rejects_bad_parameters_without_touching_the_device(libpath, bad):
    import numpy as np
    from paper_0911_2285_gb300 import lqcd as L
    args = dict(dims=(4, 4, 4, 4), kappa=0.12, nev=8, m=24, tol=1e-10)
    args.update(bad)
    dims = args.pop("dims")
    v = int(np.prod(dims))
    links = np.zeros(max(v, 1) * 36, dtype=np.complex128)
    with pytest.raises(L.LQCDError) as e:
        L.Solver(links if v > 0 else links, dims, **args)
    assert e.value.status == L.ERR_ARG


def test_init_refuses_a_plan_above_the_hbm_budget_without_touching_the_device(libpath):
    """The memory plan is checked against hbm_budget_bytes before any device call."""
    import numpy as np
    from paper_0911_2285_gb300 import lqcd as L
    dims = (8, 8, 8, 8)
    links = np.zeros(int(np.prod(dims)) * 36, dtype=np.complex128)
    with pytest.raises(L.LQCDError) as e:
        L.Solver(links, dims, 0.12, nev=8, m=24, tol=1e-10, precision="mixed", k_max=8,
                 hbm_budget_bytes=8 << 20)
    assert e.value.status == L.ERR_OOM
    assert "budget" in L.last_error()


def test_binding_pairs_fields_of_one_kind():
    """The binding hands the library two fields of one call only when both are host
    memory or both device memory of the context's GPU (host logic, no context)."""
    np = pytest.importorskip("numpy")
    from paper_0911_2285_gb300.lqcd import Solver
    s = Solver.__new__(Solver)
    s._own_stream, s._device = True, None
    a = np.zeros((2, 24), dtype=np.complex128)
    c = np.ones((2, 24), dtype=np.complex128)
    pa, pc, dev = s._fields(a, c, 48, 48)
    assert dev == 0 and pa.value == a.ctypes.data and pc.value == c.ctypes.data
    with pytest.raises(ValueError):
        s._fields(a, c, 48, 24)
    with pytest.raises(TypeError):
        s._fields(a, c.astype(np.complex64))
    torch = pytest.importorskip("torch")
    pa, pc, dev = s._fields(a, torch.zeros(2, 24, dtype=torch.complex128))
    assert dev == 0
