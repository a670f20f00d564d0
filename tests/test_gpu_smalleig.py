"""GPU parity of the device small-matrix kernels: the eigen-solver with left and right
vectors (against LAPACK through the oracle) and the BiCG-eigen restart coefficients
(against the oracle's Algorithm BiCG-eigen)."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle.bicg import eigbicg, restart_coefficients
from oracle.smalleig import eig_lr
from tests.gpu_util import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 3, 7, 24, 40, 64, 80])
def test_small_eig_matches_lapack(n):
    from paper_0911_2285_gb300 import small_eig
    rng = np.random.default_rng(100 + n)
    c = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lam, y, z = small_eig(c)
    y_o, z_o, lam_o = eig_lr(c)
    scale = np.abs(lam_o).max()
    assert np.abs(lam - lam_o).max() <= 1e-12 * scale
    for i in range(n):
        assert np.linalg.norm(c @ y[:, i] - lam[i] * y[:, i]) <= 1e-12 * scale
        assert abs(np.vdot(z[:, i], y[:, i]) - 1) <= 1e-10
        # same normalisation as the oracle: vectors agree up to rounding
        assert np.linalg.norm(y[:, i] - y_o[:, i]) <= 1e-8


def test_small_eig_tridiagonal_bicg_matrix():
    """The projected matrix of a real BiCG window (non-normal tridiagonal)."""
    from paper_0911_2285_gb300 import small_eig
    w, links, op = workload("4^4")
    from seeded_inputs import workload_source
    res = eigbicg(op, workload_source("4^4", 0), nev=8, m=24)
    H = res.first_window[2]
    lam, y, z = small_eig(H)
    y_o, z_o, lam_o = eig_lr(H)
    assert np.abs(lam - lam_o).max() <= 1e-12 * np.abs(lam_o).max()
    for i in range(8):
        assert np.linalg.norm(y[:, i] - y_o[:, i]) <= 1e-9


def _same_set(a, b, tol):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return len(a) == len(b) and cost[r, c].max() <= tol


@pytest.mark.parametrize("m,nev", [(24, 8), (40, 10), (20, 6)])
def test_restart_coefficients_match_oracle(m, nev):
    from paper_0911_2285_gb300 import restart_coefficients as dev_restart
    from seeded_inputs import workload_source
    w, links, op = workload("4^4")
    res = eigbicg(op, workload_source("4^4", 0), nev=nev, m=m)
    H = res.first_window[2]
    yc_o, zc_o, lam_o = restart_coefficients(H, nev)
    yc, zc, lam = dev_restart(H, nev)
    assert len(lam) == len(lam_o)
    # the nev smallest (the ones kept by later restarts and the final Ritz step)
    # agree tightly; eigenvalues of T along nearly dependent pairs amplify rounding
    assert np.abs(lam[:nev] - lam_o[:nev]).max() <= 1e-9 * np.abs(lam_o).max()
    assert _same_set(lam, lam_o, 1e-5 * np.abs(lam_o).max())
    # the restarted pair is biorthonormal and diagonalises H on the device as well
    assert np.abs(np.conj(zc.T) @ yc - np.eye(len(lam))).max() <= 1e-5
    assert np.abs(np.conj(zc.T) @ H @ yc - np.diag(lam)).max() <= 1e-5 * np.abs(lam).max()


def test_restart_coefficients_random_matrix():
    from paper_0911_2285_gb300 import restart_coefficients as dev_restart
    rng = np.random.default_rng(7)
    m, nev = 30, 6
    H = np.diag(np.linspace(0.1, 2.0, m)) + 0.3 * (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    yc_o, zc_o, lam_o = restart_coefficients(H, nev)
    yc, zc, lam = dev_restart(H, nev)
    assert _same_set(lam, lam_o, 1e-10 * np.abs(lam_o).max())
    # coefficient vectors agree column by column (same ordering and normalisation)
    for i in range(len(lam)):
        j = int(np.argmin(np.abs(lam_o - lam[i])))
        ph = np.vdot(yc_o[:, j], yc[:, i])
        ph /= abs(ph)
        assert np.linalg.norm(yc[:, i] - ph * yc_o[:, j]) <= 1e-8 * np.linalg.norm(yc_o[:, j])
