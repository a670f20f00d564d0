"""The allocation-free eigen-solver entry point against the allocating one.

``lqcd_small_eig_noalloc`` is for callers that cannot allocate device memory at
the moment they need a small eigen-solve (their device memory is all handed to
their own pool or budget, or an allocation's implicit synchronisation would stall
other streams). It takes device pointers and keeps its scratch in a static device
array shared by every call. This test calls it through the C ABI twice in a row
on different matrices and compares each result with ``lqcd_small_eig`` (which
allocates), so the second call also shows that stale scratch from the first does
not leak into its output. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_small_eig_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_0911_2285_gb300 import lqcd
    L = lqcd.lib()
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream().cuda_stream
    for n in (40, 17):
        c = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        lam_ref, y_ref, z_ref = lqcd.small_eig(c)
        dc = torch.from_numpy(c).to("cuda")
        dl = torch.zeros(n, dtype=torch.complex128, device="cuda")
        dy = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
        dz = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        st = L.lqcd_small_eig_noalloc(n, C.c_void_p(dc.data_ptr()), C.c_void_p(dl.data_ptr()),
                                      C.c_void_p(dy.data_ptr()), C.c_void_p(dz.data_ptr()), C.c_void_p(stream))
        assert st == lqcd.OK, lqcd.status_str(st)
        lam, y, z = dl.cpu().numpy(), dy.cpu().numpy(), dz.cpu().numpy()
        scale = np.abs(lam_ref).max()
        assert np.abs(lam - lam_ref).max() <= 1e-12 * scale
        assert np.abs(y - y_ref).max() <= 1e-10
        assert np.abs(z - z_ref).max() <= 1e-10 * max(1.0, np.abs(z_ref).max())
        for i in range(n):
            assert np.linalg.norm(c @ y[:, i] - lam[i] * y[:, i]) <= 1e-10 * scale


def test_noalloc_small_eig_rejects_sizes_beyond_its_scratch():
    from paper_0911_2285_gb300 import lqcd
    L = lqcd.lib()
    dummy = C.c_void_p(16)
    assert L.lqcd_small_eig_noalloc(81, dummy, dummy, dummy, dummy, None) == lqcd.ERR_ARG
