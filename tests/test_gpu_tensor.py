"""GPU tests of the tensor-core (tcgen05, 3xTF32) inner-product matrices of FP32
fields, C = X^H Y, used by the deflation and eigenspace-growth projections, and
of the CUDA-core path they replace: exact on integer-valued fields, FP32-level
accuracy on random fields (relative to the Cauchy-Schwarz bound |x_i| |y_j|),
both paths agreeing, over one and several row tiles (a > 128), column groups
(b > 8), split-K over many K-tiles, and the ragged shapes of the solver."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def fields(a, n, seed, kind="normal"):
    import torch
    rng = np.random.default_rng(seed)
    if kind == "int":
        z = rng.integers(-3, 4, size=(a, n)) + 1j * rng.integers(-3, 4, size=(a, n))
    else:
        z = rng.standard_normal((a, n)) + 1j * rng.standard_normal((a, n))
    z = z.astype(np.complex64)
    return z, torch.from_numpy(z).cuda()


def ref_dots(x, y):
    return np.conj(x.astype(np.complex128)) @ y.astype(np.complex128).T


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("a,b,n", [(1, 1, 3072), (5, 3, 3072), (80, 8, 49152), (130, 12, 3072), (8, 16, 65536)])
def test_integer_fields_exact(path, a, b, n):
    """Small integers are exact in TF32 and their sums exact in FP32: any mix-up of
    rows, columns, real/imaginary parts or K-tiles shows as a nonzero difference."""
    from paper_0911_2285_gb300.lqcd import field_dots
    x, X = fields(a, n, 1 + a, "int")
    y, Y = fields(b, n, 2 + b, "int")
    c, _ = field_dots(X, Y, path=path)
    assert np.array_equal(c, ref_dots(x, y))


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("a,b,n", [(10, 8, 884736), (80, 20, 393216), (33, 1, 12 * 4 ** 4)])
def test_random_fields_fp32_accuracy(path, a, b, n):
    from paper_0911_2285_gb300.lqcd import field_dots
    x, X = fields(a, n, 10 + a)
    y, Y = fields(b, n, 20 + b)
    c, _ = field_dots(X, Y, path=path)
    ref = ref_dots(x, y)
    bound = np.outer(np.linalg.norm(x, axis=1), np.linalg.norm(y, axis=1))
    assert np.max(np.abs(c - ref) / bound) <= 2e-6


@pytest.mark.parametrize("path", [0, 1])
def test_norms_without_cancellation(path):
    """C_ii = |x_i|^2 sums positive terms only: the relative error shows the
    accumulation itself (the tensor core truncates as it accumulates; short
    separate runs keep it at FP32 level)."""
    from paper_0911_2285_gb300.lqcd import field_dots
    x, X = fields(16, 884736, 77)
    c, _ = field_dots(X, X, path=path)
    nrm = np.linalg.norm(x.astype(np.complex128), axis=1) ** 2
    assert np.max(np.abs(np.diag(c) - nrm) / nrm) <= 1e-6
    assert np.max(np.abs(np.diag(c).imag)) <= 1e-6 * nrm.max()


def test_paths_agree_and_tensor_path_is_faster_at_solver_shape():
    """The growth projection shape of the 24^3x64 solver (80 eigenspace columns
    against 8 fields of 10.6M complex numbers): both paths agree to FP32 level; the
    tensor-core one is timed against the CUDA-core one."""
    import torch
    from paper_0911_2285_gb300.lqcd import field_dots
    n = 12 * 24 ** 3 * 64
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(80, n, dtype=torch.complex64, device="cuda", generator=g)
    Y = torch.randn(8, n, dtype=torch.complex64, device="cuda", generator=g)
    c1, t1 = field_dots(X, Y, path=1, reps=3)
    c0, t0 = field_dots(X, Y, path=0, reps=3)
    bound = np.outer(torch.linalg.vector_norm(X, dim=1).double().cpu().numpy(),
                     torch.linalg.vector_norm(Y, dim=1).double().cpu().numpy())
    assert np.max(np.abs(c1 - c0) / bound) <= 4e-6
    gb = (80 + 8) * n * 8 / 1e9
    print(f"\nX^H Y 80x8, n={n}: tensor {t1:.3f} ms ({gb / t1 * 1e3:.0f} GB/s), CUDA cores {t0:.3f} ms")
    assert t1 < t0


def test_rejects_unsupported_shape():
    from paper_0911_2285_gb300 import lqcd
    x, X = fields(4, 3080, 1)      # 2n not a multiple of 32
    y, Y = fields(2, 3080, 2)
    with pytest.raises(lqcd.LQCDError):
        lqcd.field_dots(X, Y, path=1)
    c, _ = lqcd.field_dots(X, Y, path=0)
    bound = np.outer(np.linalg.norm(x, axis=1), np.linalg.norm(y, axis=1))
    assert np.max(np.abs(c - ref_dots(x, y)) / bound) <= 2e-6


def test_restart_product_tensor_cores_match_cuda_cores():
    """eigBiCG with restarts in mixed precision (8^4, m = 40, nev = 10): the window
    product never feeds back into the BiCG iterates of the window leg, so both paths
    restart equally often; the correction leg deflates with the Ritz vectors each path
    built, so the total iteration counts agree to a few and both meet the FP64 true
    residual with the oracle's A. Stopped just after the first restart, the projected
    window matrix H (restart Ritz values plus the coupling row and column formed from
    the new basis vectors) agrees between the paths to FP32 rounding."""
    from paper_0911_2285_gb300 import Solver
    from seeded_inputs import z2_source
    from tests.gpu_util import true_resid, workload
    w, links, op = workload("8^4")
    b = z2_source(w["dims"], 4321)
    full, early = {}, {}
    with Solver(links, w["dims"], w["kappa"], nev=w["nev"], m=w["m"], n1=1, tol=1e-10, maxiter=4000,
                precision="mixed", k_max=2) as s:
        for tc in (True, False):
            s.set_tensor_cores(tc)
            s.reset_eigenspace()
            x, info, _ = s.solve(b, mode="eigbicg")
            full[tc] = (x[0], info[0], s.last_window()[2])
    with Solver(links, w["dims"], w["kappa"], nev=w["nev"], m=w["m"], n1=1, tol=1e-10, maxiter=w["m"] + 6,
                precision="mixed", k_max=2) as s:
        for tc in (True, False):
            s.set_tensor_cores(tc)
            s.solve(b, mode="eigbicg", raise_on_fail=False)   # the second solve starts from a fresh window
            early[tc] = s.last_window()
    (x1, i1, n1), (x0, i0, n0) = full[True], full[False]
    assert i1["restarts"] == i0["restarts"] and i1["restarts"] >= 3
    assert n1 == n0
    assert abs(i1["iters"] - i0["iters"]) <= 3 and i1["outer_steps"] == i0["outer_steps"] == 1
    assert true_resid(op, b, x1) <= 1e-10 and true_resid(op, b, x0) <= 1e-10
    (H1, _, r1), (H0, _, r0) = early[True], early[False]
    assert r1 == r0 == 1 and H1.shape == H0.shape
    assert np.max(np.abs(H1 - H0)) <= 1e-4 * np.max(np.abs(H0))
