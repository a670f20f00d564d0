"""Pins for the oracle's Incremental eigBiCG, deflation and Rayleigh-Ritz (paper Sec. 2).

Fixed points: the Galerkin condition ``U_l^H r = 0`` after oblique deflation;
independence of the deflated guess from the bases chosen for the two spaces;
deflation with the whole space (``U_r = U_l = I``) is the exact solve; the
block growth of ``H`` equals ``U_l^H A U_r`` formed densely; Rayleigh-Ritz on
exact eigenvectors (dense LAPACK) returns their eigenvalues; solutions of
the incremental run meet the true-residual tolerance.
"""
import numpy as np
import scipy.linalg as sla

from oracle.incremental import (Eigenspace, deflate, deflated_bicg, grow, incremental_eigbicg,
                                rayleigh_ritz)
from oracle.wilson import WilsonOperator
from seeded_inputs import WORKLOADS, gauge_links, gaussian_source, workload_links, workload_source, z2_source


def small_op(dims=(2, 2, 2, 2), kappa=0.12, eps=0.5, seed=1):
    return WilsonOperator(gauge_links(dims, eps, seed), kappa, dims)


def random_space(op, k, rng):
    ur = rng.standard_normal((op.n, k)) + 1j * rng.standard_normal((op.n, k))
    ul = rng.standard_normal((op.n, k)) + 1j * rng.standard_normal((op.n, k))
    aur = np.stack([op.apply(ur[:, i]) for i in range(k)], axis=1)
    return Eigenspace(op.n, ur, ul, np.conj(ul.T) @ aur)


def test_deflation_galerkin_condition(rng):
    op = small_op((2, 2, 2, 4))
    sp = random_space(op, 12, rng)
    b = gaussian_source(op.dims, 1)
    x0 = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    x = deflate(op, sp, b, x0)
    r = b - op.apply(x)
    assert np.abs(np.conj(sp.Ul.T) @ r).max() <= 1e-12 * np.linalg.norm(b) * np.sqrt(op.n)


def test_deflation_basis_invariance(rng):
    op = small_op((2, 2, 2, 4))
    sp = random_space(op, 10, rng)
    g = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    k = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    ur2, ul2 = sp.Ur @ g, sp.Ul @ k
    aur2 = np.stack([op.apply(ur2[:, i]) for i in range(10)], axis=1)
    sp2 = Eigenspace(op.n, ur2, ul2, np.conj(ul2.T) @ aur2)
    b = gaussian_source(op.dims, 2)
    x1 = deflate(op, sp, b, np.zeros(op.n, complex))
    x2 = deflate(op, sp2, b, np.zeros(op.n, complex))
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)


def test_deflation_with_whole_space_is_exact_solve():
    op = small_op()
    eye = np.eye(op.n, dtype=np.complex128)
    sp = Eigenspace(op.n, eye, eye.copy(), op.dense())
    b = gaussian_source(op.dims, 3)
    x = deflate(op, sp, b, np.zeros(op.n, complex))
    assert np.linalg.norm(op.apply(x) - b) <= 1e-12 * np.linalg.norm(b)


def test_grow_matches_dense_projection(rng):
    op = small_op((2, 2, 2, 4))
    sp = Eigenspace(op.n)
    for _ in range(3):
        vn = rng.standard_normal((op.n, 4)) + 1j * rng.standard_normal((op.n, 4))
        wn = rng.standard_normal((op.n, 4)) + 1j * rng.standard_normal((op.n, 4))
        old = sp.size
        sp = grow(op, sp, vn, wn)
        a = op.dense()
        assert np.abs(sp.H - np.conj(sp.Ul.T) @ a @ sp.Ur).max() <= 1e-12 * np.abs(sp.H).max()
        if old:
            # the new blocks are oblique-orthogonal to the old ones
            assert np.abs(np.conj(sp.Ul[:, :old].T) @ sp.Ur[:, old:]).max() < 1e-10
            assert np.abs(np.conj(sp.Ur[:, :old].T) @ sp.Ul[:, old:]).max() < 1e-10
        assert np.allclose(np.linalg.norm(sp.Ur[:, old:], axis=0), 1)


def test_grow_drops_vectors_already_in_space(rng):
    op = small_op()
    sp = random_space(op, 6, rng)
    sp2 = grow(op, sp, sp.Ur[:, :2] @ np.array([[1.0], [2.0]]), sp.Ul[:, :1])
    assert sp2.size == sp.size


def test_rayleigh_ritz_on_exact_eigenvectors():
    op = small_op((2, 2, 2, 2), kappa=0.124)
    a = op.dense()
    lam, zl, zr = sla.eig(a, left=True, right=True)
    idx = np.argsort(np.abs(lam))[:8]
    ur, ul = zr[:, idx], zl[:, idx]
    sp = Eigenspace(op.n, ur, ul, np.conj(ul.T) @ a @ ur)
    rl, u, w, res = rayleigh_ritz(op, sp)
    cost = np.abs(rl[:, None] - lam[idx][None, :])
    assert np.all(cost.min(axis=1) < 1e-12)
    assert np.all(res < 1e-12)


def test_incremental_solves_workload_4x4x4x4():
    """Algorithm Incremental eigBiCG on the 4^4 workload links, 5 Z2 sources:
    every solution meets the true-residual tolerance and H = U_l^H A U_r."""
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    srcs = [z2_source(w["dims"], 5000 + i) for i in range(5)]
    out = incremental_eigbicg(op, srcs, nev=8, m=24, n1=3, tol=1e-10)
    assert out.modes == ["eigbicg"] * 3 + ["deflated"] * 2
    for x, b in zip(out.x, srcs):
        assert np.linalg.norm(b - op.apply(x)) <= 1e-10 * np.linalg.norm(b)
    assert out.space.size > 8
    aur = np.stack([op.apply(out.space.Ur[:, i]) for i in range(out.space.size)], axis=1)
    assert np.abs(out.space.H - np.conj(out.space.Ul.T) @ aur).max() < 1e-10 * np.abs(out.space.H).max()


def test_deflation_reduces_iterations_weak_links():
    """Near-free links (eps = 0.05) have an isolated low mode group that eigBiCG
    resolves; deflating it must cut the BiCG iteration count (paper Fig. 1 effect)."""
    dims = (4, 4, 4, 4)
    op = WilsonOperator(gauge_links(dims, 0.05, 21), 0.122, dims)
    srcs = [z2_source(dims, 7000 + i) for i in range(4)]
    out = incremental_eigbicg(op, srcs, nev=6, m=20, n1=2, tol=1e-10)
    assert max(out.iters[2:]) < out.iters[0]


def test_deftol_restart_converges():
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    rng = np.random.default_rng(0)
    sp = random_space(op, 6, rng)
    b = workload_source("4^4", 0)
    x, it, mv, tr = deflated_bicg(op, sp, b, tol=1e-10, deftol=1e-4)
    assert tr <= 1e-10
    assert np.linalg.norm(b - op.apply(x)) <= 1e-10 * np.linalg.norm(b)


def test_incremental_rayleigh_ritz_converged_pairs_match_dense_weak_field():
    """Eight eigBiCG sources (nev = 10, m = 30) on a weakly disordered 4^4 field
    whose lowest twelve eigenvalues are isolated: every Rayleigh-Ritz pair whose
    two-sided estimate is below 1e-8 |lambda| lies on the dense LAPACK spectrum
    (stored under tests/golden/) to 1e-8 relative, and there are at least eight."""
    import os
    g = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "wilson_4x4x4x4_eps0.1_lowest_eigs.txt"),
                   comments="#")
    dense = g[:, 0] + 1j * g[:, 1]
    dims = (4, 4, 4, 4)
    op = WilsonOperator(gauge_links(dims, 0.1, 21), 0.122, dims)
    out = incremental_eigbicg(op, [z2_source(dims, 7000 + i) for i in range(8)], nev=10, m=30, n1=8, tol=1e-10)
    lam, u, w, res = rayleigh_ritz(op, out.space)
    conv = 0
    for i in range(len(lam)):
        ru = np.linalg.norm(op.apply(u[:, i]) - lam[i] * u[:, i])
        rz = np.linalg.norm(op.apply_dag(w[:, i]) - np.conj(lam[i]) * w[:, i])
        est = ru * rz / abs(np.vdot(w[:, i], u[:, i]))
        if est <= 1e-8 * abs(lam[i]):
            conv += 1
            assert np.min(np.abs(dense - lam[i])) <= 1e-8 * abs(lam[i])
    assert conv >= 8
