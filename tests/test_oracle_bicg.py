"""Pins for the oracle's BiCG and eigBiCG (paper Sec. 2, Algorithms eigBiCG and BiCG-eigen).

Fixed points used: a dense LU solve; the reduction of BiCG to CG (scipy) for a
Hermitian positive definite matrix; the biorthogonality of BiCG residuals;
the real BiCG scalars of the gamma5 shadow residual (Sec. 4); the Lanczos
relations ``W^H V = I`` and ``W^H A V = H`` that the paper's H formulas must
satisfy; matrices with a known spectrum (free field, designed similarity
transform) whose smallest eigenvalues the Ritz values must reach; and the
4^4 dense spectrum stored in ``tests/golden``.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.bicg import Breakdown, bicg, eigbicg, restart_coefficients
from oracle.smalleig import biorthogonalize, eig_lr
from oracle.wilson import DenseOperator, WilsonOperator
from seeded_inputs import WORKLOADS, gauge_links, gaussian_source, workload_links, workload_source

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def wilson(dims=(2, 2, 2, 2), eps=0.5, seed=1, kappa=0.12):
    return WilsonOperator(gauge_links(dims, eps, seed), kappa, dims)


def unit_links(dims):
    lx, ly, lz, lt = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    for a in range(3):
        u[..., a, a] = 1.0
    return u


def designed(n=200, seed=3):
    """A = S diag(lam) S^-1 with four isolated small eigenvalues."""
    rng = np.random.default_rng(seed)
    small = np.array([0.01, 0.02 + 0.01j, 0.02 - 0.01j, 0.05])
    lam = np.concatenate([small, 1 + 0.5 * rng.random(n - 4) + 0.3j * (rng.random(n - 4) - 0.5)])
    s = np.eye(n) + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    return DenseOperator(s @ np.diag(lam) @ np.linalg.inv(s)), small, rng


def test_bicg_matches_dense_solve():
    op = wilson((2, 2, 2, 4))
    b = gaussian_source(op.dims, 3)
    res = bicg(op, b, tol=1e-12)
    xd = np.linalg.solve(op.dense(), b)
    assert np.linalg.norm(res.x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert res.true_resid <= 1e-12


def test_bicg_reduces_to_cg_for_hpd(rng):
    """HPD A with rhat0 = r0: BiCG produces the CG iterates (library CG as reference)."""
    n = 60
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = g @ np.conj(g.T) / n + 0.5 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ours = []
    bicg(DenseOperator(a), b, tol=1e-13, callback=lambda j, x, r, rh: ours.append(x.copy()))
    theirs = []
    spla.cg(a, b, rtol=1e-13, maxiter=len(ours), callback=lambda xk: theirs.append(xk.copy()))
    k = min(12, len(ours), len(theirs))
    assert k >= 8
    for j in range(k):
        assert np.linalg.norm(ours[j] - theirs[j]) <= 1e-9 * np.linalg.norm(theirs[j])


def test_bicg_residuals_biorthogonal(rng):
    """(rhat_i, r_j) = 0 for i != j (two-sided Lanczos, Sec. 2)."""
    n = 80
    a = np.eye(n) + 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    rs, rhs = [], []
    bicg(DenseOperator(a), b, tol=1e-14,
         callback=lambda j, x, r, rh: (rs.append(r.copy()), rhs.append(rh.copy())))
    k = 8
    for i in range(k):
        for j in range(k):
            if i != j:
                val = abs(np.vdot(rhs[i], rs[j]))
                assert val <= 1e-9 * np.linalg.norm(rhs[i]) * np.linalg.norm(rs[j])


def test_gamma5_shadow_gives_real_scalars():
    """Sec. 4: with rhat0 = gamma5 r0, rhat_j = gamma5 r_j and alpha, beta are real."""
    op = WilsonOperator(workload_links("4^4"), 0.12, (4, 4, 4, 4))
    b = workload_source("4^4", 0)
    res = bicg(op, b, rhat0=op.gamma5(b), history=True, tol=1e-10)
    for alpha, beta in res.snapshots:
        assert abs(alpha.imag) <= 1e-9 * abs(alpha)
        assert abs(beta.imag) <= 1e-9 * abs(beta)
    assert res.true_resid <= 1e-10


def test_bicg_breakdown_detected(rng):
    n = 20
    a = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    b = np.zeros(n, dtype=np.complex128)
    b[0] = 1
    rhat0 = np.zeros(n, dtype=np.complex128)
    rhat0[1] = 1   # (rhat0, r0) = 0
    with pytest.raises(Breakdown):
        bicg(DenseOperator(a), b, rhat0=rhat0)


def test_bicg_plain_iteration_count_4x4x4x4():
    """4^4 workload: BiCG converges to 1e-10 (58 iterations with these inputs)."""
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    res = bicg(op, workload_source("4^4", 0), tol=1e-10)
    assert res.true_resid <= 1e-10
    assert 40 <= res.iters <= 80


# ----------------------------------------------------------------- eig_lr

@pytest.mark.parametrize("n", [1, 2, 7, 24])
def test_eig_lr_conventions(n, rng):
    c = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y, z, lam = eig_lr(c)
    assert np.all(np.diff(np.abs(lam)) >= 0)
    ref = np.linalg.eigvals(c)
    assert np.abs(np.sort_complex(ref) - np.sort_complex(lam)).max() < 1e-10 * max(1, np.abs(ref).max())
    for i in range(n):
        assert np.linalg.norm(c @ y[:, i] - lam[i] * y[:, i]) < 1e-10 * np.abs(lam).max()
        assert np.linalg.norm(np.conj(z[:, i]) @ c - lam[i] * np.conj(z[:, i])) < 1e-8 * np.abs(lam).max() * np.linalg.norm(z[:, i])
        assert abs(np.linalg.norm(y[:, i]) - 1) < 1e-13
        assert abs(np.vdot(z[:, i], y[:, i]) - 1) < 1e-12
        k = np.argmax(np.abs(y[:, i]))
        assert abs(y[k, i].imag) < 1e-14 and y[k, i].real > 0


def test_biorthogonalize_identity_and_span(rng):
    m, k = 12, 3
    c = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    y, z, _ = eig_lr(c)
    y2 = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    z2 = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    Y, Z = biorthogonalize(y[:, :k], z[:, :k], y2, z2)
    assert np.abs(np.conj(Z.T) @ Y - np.eye(2 * k)).max() < 1e-10
    # span preserved: [y1 y2] and Y span the same space
    basis = np.hstack([y[:, :k], y2])
    proj = basis @ np.linalg.lstsq(basis, Y, rcond=None)[0]
    assert np.abs(proj - Y).max() < 1e-10
    assert np.allclose(Y[:, :k], y[:, :k])


def test_biorthogonalize_drops_dependent_pair(rng):
    m, k = 10, 2
    c = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    y, z, _ = eig_lr(c)
    y2 = y[:, :k].copy()
    z2 = z[:, :k].copy()
    Y, Z = biorthogonalize(y[:, :k], z[:, :k], y2, z2)
    assert Y.shape[1] == k and Z.shape[1] == k


# ------------------------------------------------------------ eigBiCG

def _window_identities(op, V, W, H):
    AV = np.stack([op.apply(V[:, i]) for i in range(V.shape[1])], axis=1)
    bi = np.abs(np.conj(W.T) @ V - np.eye(V.shape[1])).max()
    proj = np.abs(np.conj(W.T) @ AV - H).max() / np.abs(H).max()
    return bi, proj


def test_eigbicg_first_window_lanczos_identities():
    """The H entries built from BiCG scalars equal W^H A V; W^H V = I."""
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    res = eigbicg(op, workload_source("4^4", 0), nev=8, m=24)
    V, W, H = res.first_window
    bi, proj = _window_identities(op, V, W, H)
    assert bi < 1e-10
    assert proj < 1e-10


def test_eigbicg_restart_keeps_projection():
    """After every restart (coupling row/column included) W^H A V = H to 1e-8."""
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    res = eigbicg(op, workload_source("4^4", 0), nev=8, m=24, snapshot_every=1)
    assert res.restarts >= 2
    checked = 0
    for V, W, H in res.snapshots[24:]:
        _, proj = _window_identities(op, V, W, H)
        assert proj < 1e-8
        checked += 1
    assert checked > 10
    assert res.true_resid <= 1e-10


def test_eigbicg_solution_matches_bicg():
    """The window does not change the BiCG iteration (same x, same count)."""
    op = wilson((2, 2, 2, 4))
    b = gaussian_source(op.dims, 8)
    r1 = bicg(op, b)
    r2 = eigbicg(op, b, nev=4, m=12)
    assert r1.iters == r2.iters
    assert np.linalg.norm(r1.x - r2.x) <= 1e-12 * np.linalg.norm(r1.x)


def _petrov_galerkin_eigs(H, Ys, Zs, rng):
    """Eigenvalues of H restricted obliquely to span(Ys) along span(Zs), via QR bases."""
    k = Ys.shape[1]
    mix = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    qy, _ = np.linalg.qr(Ys @ mix)
    qz, _ = np.linalg.qr(Zs)
    return np.linalg.eigvals(np.linalg.solve(np.conj(qz.T) @ qy, np.conj(qz.T) @ H @ qy))


def _assert_same_set(a, b, tol):
    from scipy.optimize import linear_sum_assignment
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    assert len(a) == len(b)
    assert cost[r, c].max() < tol


def test_restart_lambda_invariant_under_basis_choice(rng):
    """T7: Lambda of BiCG-eigen depends only on the spans of the 2nev vectors, not on
    the LU route: a QR-based oblique projection onto the same spans gives the same set."""
    m, nev = 20, 5
    H = np.diag(np.linspace(0.1, 2.0, m)) + 0.3 * (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    yc, zc, lam = restart_coefficients(H, nev)
    assert len(lam) == 2 * nev
    y_m, z_m, _ = eig_lr(H)
    y_m1, z_m1, _ = eig_lr(H[: m - 1, : m - 1])
    pad = np.zeros((1, nev))
    Ys = np.hstack([y_m[:, :nev], np.vstack([y_m1[:, :nev], pad])])
    Zs = np.hstack([z_m[:, :nev], np.vstack([z_m1[:, :nev], pad])])
    _assert_same_set(lam, _petrov_galerkin_eigs(H, Ys, Zs, rng), 1e-9 * np.abs(lam).max())
    # limited by the conditioning of T's eigenvectors
    assert np.abs(np.conj(zc.T) @ yc - np.eye(len(lam))).max() < 1e-6
    assert np.abs(np.conj(zc.T) @ H @ yc - np.diag(lam)).max() < 1e-6 * np.abs(lam).max()


def test_restart_on_bicg_window_drops_dependent_pairs(rng):
    """On a real BiCG H the m and m-1 Ritz vectors can be nearly dependent; the kept
    spans still give the Petrov-Galerkin eigenvalues and a biorthonormal pair."""
    op = WilsonOperator(workload_links("4^4"), 0.12, (4, 4, 4, 4))
    res = eigbicg(op, workload_source("4^4", 0), nev=6, m=20)
    H = res.first_window[2]
    yc, zc, lam = restart_coefficients(H, 6)
    assert 6 <= len(lam) <= 12
    _assert_same_set(lam, _petrov_galerkin_eigs(H, yc, zc, rng), 1e-8 * np.abs(lam).max())
    assert np.abs(np.conj(zc.T) @ yc - np.eye(len(lam))).max() < 1e-5


def test_eigbicg_free_field_ritz_closed_form():
    """U = 1, kappa = 0.12 on 4^4: lowest eigenvalue 1 - 8 kappa, next shell 1 - 6k +- 2ik."""
    dims = (4, 4, 4, 4)
    kappa = 0.12
    op = WilsonOperator(unit_links(dims), kappa, dims)
    res = eigbicg(op, gaussian_source(dims, 7), nev=4, m=16, tol=1e-12)
    lam = res.evals
    assert abs(lam[0] - (1 - 8 * kappa)) < 1e-8 * abs(1 - 8 * kappa)
    shell = 1 - 6 * kappa
    assert min(abs(lam[1:3] - (shell - 2j * kappa))) < 1e-8
    assert min(abs(lam[1:3] - (shell + 2j * kappa))) < 1e-8


def test_eigbicg_designed_spectrum():
    """Known spectrum: the four isolated eigenvalues are found to 1e-8 relative."""
    op, small, rng = designed()
    b = rng.standard_normal(op.n) + 0j
    res = eigbicg(op, b, nev=4, m=16, tol=1e-12)
    for s in small:
        assert np.min(np.abs(res.evals - s)) < 1e-8 * abs(s)
    assert res.restarts >= 1


def test_eigbicg_converged_ritz_match_dense_4x4x4x4():
    """Table-1 analogue on the 4^4 workload: every Ritz pair that the two-sided
    estimate calls converged lies on the stored dense spectrum."""
    g = np.loadtxt(os.path.join(GOLDEN, "wilson_4x4x4x4_lowest_eigs.txt"), comments="#")
    dense = g[:, 0] + 1j * g[:, 1]
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    res = eigbicg(op, workload_source("4^4", 0), nev=8, m=24, tol=1e-10)
    for i, lam in enumerate(res.evals):
        u, z = res.U[:, i], res.Q[:, i]
        ru = np.linalg.norm(op.apply(u) - lam * u)
        rz = np.linalg.norm(op.apply_dag(z) - np.conj(lam) * z)
        est = ru * rz / abs(np.vdot(z, u))
        d = np.min(np.abs(dense - lam))
        # The two-sided estimate bounds the eigenvalue error to first order.
        assert d <= 10 * est + 1e-12
