"""Failure detection on the GPU, in forms that fault, trap or hang nothing:

* a genuine BiCG breakdown (sigma = (phat, A p) = 0 on a constructed source)
  returns LQCD_ERR_BREAKDOWN with the solve info filled, as the oracle's BiCG
  raises Breakdown on the same input;
* host-side fault injection (LQCD_FAULT=alloc:N): every device allocation of
  the context's set-up, made to fail in turn, gives LQCD_ERR_OOM and a clean
  tear-down, and a context created afterwards works;
* a bounded device wait on a flag that nothing sets gives up after the
  run-time limit and returns LQCD_ERR_TIMEOUT promptly; the device stays usable.
"""
import ctypes as C
import os
import time

import numpy as np
import pytest

from oracle.bicg import Breakdown, bicg
from oracle.wilson import WilsonOperator
from seeded_inputs import workload_source
from tests.gpu_util import true_resid, workload

pytestmark = pytest.mark.gpu


def free_links(dims):
    lx, ly, lz, lt = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    for a in range(3):
        u[..., a, a] = 1.0
    return u


def breakdown_source(dims):
    """b = 2 on spin 0, colour 0 of the even-x sites, 0 elsewhere. On the free
    field, sigma_0 = b^H A b = V (2 - 12 kappa), which vanishes at kappa = 1/6:
    the hops in y, z, t see the same value on both sides (the gamma terms cancel),
    the x hops see zeros, so (D b) = 12 on b's support."""
    lx, ly, lz, lt = dims
    b = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    b[:, :, :, 0::2, 0, 0] = 2.0
    return b.reshape(-1)


def test_bicg_breakdown_is_reported_not_hidden():
    from paper_0911_2285_gb300 import Solver, lqcd
    dims = (4, 4, 4, 4)
    kappa = 1.0 / 6.0
    links = free_links(dims)
    b = breakdown_source(dims)
    op = WilsonOperator(links, kappa, dims)
    with pytest.raises(Breakdown):
        bicg(op, b, tol=1e-10)
    with Solver(links, dims, kappa, nev=4, m=12, tol=1e-10, precision="fp64", k_max=2) as s:
        x, info, st = s.solve(b, mode="plain", raise_on_fail=False)
        assert st == lqcd.ERR_BREAKDOWN
        assert info[0]["iters"] == 0
        assert abs(info[0]["true_resid"] - 1.0) <= 1e-12      # x = x0 = 0
        assert np.all(x[0] == 0)
        # the context stays usable
        b2 = workload_source("4^4", 0)
        x2, i2, st2 = s.solve(b2, mode="plain")
        assert st2 == lqcd.OK and true_resid(op, b2, x2[0]) <= 1e-10


def test_injected_allocation_failures_tear_down_cleanly(monkeypatch):
    from paper_0911_2285_gb300 import Solver, lqcd
    w, links, op = workload("4^4")
    args = dict(nev=w["nev"], m=w["m"], n1=1, tol=1e-10, precision="mixed", k_max=2)
    n_fail = 0
    for n in range(1, 64):
        monkeypatch.setenv("LQCD_FAULT", f"alloc:{n}")
        try:
            s = Solver(links, w["dims"], w["kappa"], **args)
        except lqcd.LQCDError as e:
            assert e.status == lqcd.ERR_OOM, str(e)
            n_fail += 1
            continue
        s.close()          # n is past the last allocation: set-up succeeded
        break
    else:
        pytest.fail("set-up never succeeded")
    assert n_fail >= 20
    monkeypatch.delenv("LQCD_FAULT")
    with Solver(links, w["dims"], w["kappa"], **args) as s:
        b = workload_source("4^4", 0)
        x, info, _ = s.solve(b, mode="plain")
    assert true_resid(op, b, x[0]) <= 1e-10


def test_bounded_wait_times_out_and_device_stays_usable():
    torch = pytest.importorskip("torch")
    from paper_0911_2285_gb300 import lqcd
    L = lqcd.lib()
    flag = torch.zeros(4, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    try:
        assert L.lqcd_set_wait_limit(2_000_000) == lqcd.OK        # about 1 ms
        t0 = time.perf_counter()
        st = L.lqcd_wait_flag(C.c_void_p(flag.data_ptr()), stream)
        dt = time.perf_counter() - t0
        assert st == lqcd.ERR_TIMEOUT
        assert dt < 1.0, dt
        flag.fill_(1)
        torch.cuda.synchronize()
        assert L.lqcd_wait_flag(C.c_void_p(flag.data_ptr()), stream) == lqcd.OK
    finally:
        assert L.lqcd_set_wait_limit(0) == lqcd.OK
    w, links, op = workload("4^4")
    from paper_0911_2285_gb300 import Solver
    with Solver(links, w["dims"], w["kappa"], nev=w["nev"], m=w["m"], tol=1e-10, precision="mixed", k_max=1) as s:
        b = workload_source("4^4", 0)
        x, info, _ = s.solve(b, mode="eigbicg")
    assert true_resid(op, b, x[0]) <= 1e-10
