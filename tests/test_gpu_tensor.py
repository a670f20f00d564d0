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
