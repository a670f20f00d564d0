"""The allocation-free eigen-solver entry point against the allocating one.

``lqcd_small_eig_noalloc`` is for callers that cannot allocate device memory at
the moment they need a small eigen-solve (their device memory is all handed to
their own pool or budget, or an allocation's implicit synchronisation would stall
other streams). It takes device pointers and keeps its scratch in a static device
array shared by every call. These tests call it through the C ABI twice in a row
on different matrices and compare each result with ``lqcd_small_eig`` (which
allocates), so the second call also shows that stale scratch from the first does
not leak into its output. They also interleave it with the allocating solver on
a smaller matrix (which must not lower the kernel's shared-memory limit below
what a later, larger allocation-free call needs) and cover the eigenvalues-only
form (Y = Z = NULL). This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(torch, L, c, vectors=True):
    n = c.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    dc = torch.from_numpy(c).to("cuda")
    dl = torch.zeros(n, dtype=torch.complex128, device="cuda")
    dy = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    dz = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    py = C.c_void_p(dy.data_ptr()) if vectors else None
    pz = C.c_void_p(dz.data_ptr()) if vectors else None
    st = L.lqcd_small_eig_noalloc(n, C.c_void_p(dc.data_ptr()), C.c_void_p(dl.data_ptr()), py, pz,
                                  C.c_void_p(stream))
    return st, dl.cpu().numpy(), dy.cpu().numpy(), dz.cpu().numpy()


def _check(c, lam, y, z, lam_ref, y_ref, z_ref, vectors=True):
    n = c.shape[0]
    scale = np.abs(lam_ref).max()
    assert np.abs(lam - lam_ref).max() <= 1e-12 * scale
    if not vectors:
        return
    assert np.abs(y - y_ref).max() <= 1e-10
    assert np.abs(z - z_ref).max() <= 1e-10 * max(1.0, np.abs(z_ref).max())
    for i in range(n):
        assert np.linalg.norm(c @ y[:, i] - lam[i] * y[:, i]) <= 1e-10 * scale


def test_noalloc_small_eig_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_0911_2285_gb300 import lqcd
    L = lqcd.lib()
    rng = np.random.default_rng(2024)
    for n in (40, 17):
        c = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        lam_ref, y_ref, z_ref = lqcd.small_eig(c)
        st, lam, y, z = _noalloc(torch, L, c)
        assert st == lqcd.OK, lqcd.status_str(st)
        _check(c, lam, y, z, lam_ref, y_ref, z_ref)


def test_noalloc_after_smaller_allocating_call_and_eigenvalues_only():
    """Largest size, then the allocating solver on n = 40 (a size whose shared
    memory needs the opt-in, but less than n = 80 does), then the largest size
    again: the second allocation-free call must still launch. Then the
    eigenvalues-only form."""
    torch = pytest.importorskip("torch")
    from paper_0911_2285_gb300 import lqcd
    L = lqcd.lib()
    rng = np.random.default_rng(77)
    c80 = rng.standard_normal((80, 80)) + 1j * rng.standard_normal((80, 80))
    c40 = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    ref80 = lqcd.small_eig(c80)
    st, lam, y, z = _noalloc(torch, L, c80)
    assert st == lqcd.OK, lqcd.status_str(st)
    _check(c80, lam, y, z, *ref80)
    ref40 = lqcd.small_eig(c40)
    st, lam, y, z = _noalloc(torch, L, c80)
    assert st == lqcd.OK, (lqcd.status_str(st), lqcd.last_error())
    _check(c80, lam, y, z, *ref80)
    st, lam, _, _ = _noalloc(torch, L, c40, vectors=False)
    assert st == lqcd.OK, lqcd.status_str(st)
    _check(c40, lam, None, None, *ref40, vectors=False)


def test_noalloc_small_eig_rejects_sizes_beyond_its_scratch():
    from paper_0911_2285_gb300 import lqcd
    L = lqcd.lib()
    dummy = C.c_void_p(16)
    assert L.lqcd_small_eig_noalloc(81, dummy, dummy, dummy, dummy, None) == lqcd.ERR_ARG
    assert L.lqcd_small_eig_noalloc(8, dummy, dummy, dummy, None, None) == lqcd.ERR_ARG
