"""Pins for the oracle's Wilson-Dirac operator (paper Sec. 3 test matrices, Sec. 4 symmetry).

Each check is fixed by mathematics outside the oracle's own code:
the Clifford algebra, the free-field (U = 1) plane-wave solution, the
gamma5-Hermiticity of Wilson fermions (Sec. 4), gauge covariance, and the
matrix adjoint computed by transposing a dense build.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle.wilson import GAMMA, GAMMA5, WilsonOperator
from seeded_inputs import gauge_links, gaussian_source, random_su3, volume


def unit_links(dims):
    lx, ly, lz, lt = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    for a in range(3):
        u[..., a, a] = 1.0
    return u


def test_gamma_clifford_algebra():
    for mu in range(4):
        assert np.allclose(GAMMA[mu], np.conj(GAMMA[mu].T))
        for nu in range(4):
            anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def test_links_are_su3():
    u = gauge_links((2, 2, 2, 4), 0.5, 1).reshape(-1, 3, 3)
    eye = np.einsum("nab,ncb->nac", u, np.conj(u))
    assert np.abs(eye - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-13


def _plane_wave(dims, n_mom, chi):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    p = [2 * np.pi * n_mom[mu] / dims[mu] for mu in range(4)]
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return (phase[..., None, None] * chi[None, None, None, None]).reshape(-1), p, phase


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_free_field_plane_waves(dims, rng):
    """U = 1: A e^{ipx} chi = e^{ipx} [(1 - 2 kappa sum cos p) + 2 i kappa sum sin p_mu gamma_mu] chi."""
    kappa = 0.13
    op = WilsonOperator(unit_links(dims), kappa, dims)
    for _ in range(5):
        n_mom = [rng.integers(0, dims[mu]) for mu in range(4)]
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        v, p, phase = _plane_wave(dims, n_mom, chi)
        m = (1 - 2 * kappa * sum(np.cos(p))) * np.eye(4) + 2j * kappa * sum(
            np.sin(p[mu]) * GAMMA[mu] for mu in range(4))
        expect = (phase[..., None, None] * (m @ chi)[None, None, None, None]).reshape(-1)
        assert np.abs(op.apply(v) - expect).max() < 1e-12
        mdag = np.conj(m.T)
        expect_dag = (phase[..., None, None] * (mdag @ chi)[None, None, None, None]).reshape(-1)
        assert np.abs(op.apply_dag(v) - expect_dag).max() < 1e-12


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_free_field_spectrum_dense(dims):
    """Eigenvalues 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p), multiplicity 6 each.

    L = 2 directions make the forward and backward neighbour the same site,
    so both hops must accumulate into the same entry.
    """
    kappa = 0.11
    op = WilsonOperator(unit_links(dims), kappa, dims)
    ev = np.linalg.eigvals(op.dense())
    expect = []
    for nt in range(dims[3]):
        for nz in range(dims[2]):
            for ny in range(dims[1]):
                for nx in range(dims[0]):
                    p = [2 * np.pi * n / d for n, d in zip((nx, ny, nz, nt), dims)]
                    re = 1 - 2 * kappa * sum(np.cos(p))
                    im = 2 * kappa * np.sqrt(sum(np.sin(q) ** 2 for q in p))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.array(expect)
    assert len(ev) == 12 * volume(dims)
    cost = np.abs(ev[:, None] - expect[None, :])
    rows, cols = linear_sum_assignment(cost)
    assert cost[rows, cols].max() < 1e-12


def test_gamma5_hermiticity_and_adjoint_dense():
    """Sec. 4: gamma5 A gamma5 = A^dagger; the oracle's A^dagger equals conj(A)^T."""
    dims = (2, 2, 2, 2)
    op = WilsonOperator(gauge_links(dims, 0.7, 5), 0.12, dims)
    a = op.dense()
    adag = np.empty_like(a)
    e = np.zeros(op.n, dtype=np.complex128)
    for j in range(op.n):
        e[j] = 1
        adag[:, j] = op.apply_dag(e)
        e[j] = 0
    g5 = np.kron(np.eye(volume(dims)), np.kron(GAMMA5, np.eye(3)))
    assert np.abs(adag - np.conj(a.T)).max() < 1e-14
    assert np.abs(g5 @ a @ g5 - np.conj(a.T)).max() < 1e-14


def test_adjoint_identity_random_vectors(rng):
    dims = (4, 4, 4, 4)
    op = WilsonOperator(gauge_links(dims, 0.5, 1), 0.12, dims)
    u = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    v = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    lhs = np.vdot(u, op.apply(v))
    rhs = np.vdot(op.apply_dag(u), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # gamma5 A gamma5 v == A^dagger v
    g5av = op.gamma5(op.apply(op.gamma5(v)))
    assert np.abs(g5av - op.apply_dag(v)).max() < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_gauge_covariance(dims, rng):
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^+, psi -> G psi  =>  A psi -> G A psi."""
    lx, ly, lz, lt = dims
    links = gauge_links(dims, 0.5, 3)
    g = random_su3(np.random.default_rng(99), volume(dims), 2.0).reshape(lt, lz, ly, lx, 3, 3)
    lg = np.empty_like(links)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=3 - mu)
        lg[mu] = np.einsum("...ab,...bc,...dc->...ad", g, links[mu], np.conj(g_fwd))
    psi = gaussian_source(dims, 4).reshape(lt, lz, ly, lx, 4, 3)
    gpsi = np.einsum("...ab,...sb->...sa", g, psi).reshape(-1)
    a = WilsonOperator(links, 0.125, dims)
    ag = WilsonOperator(lg, 0.125, dims)
    lhs = ag.apply(gpsi)
    rhs = np.einsum("...ab,...sb->...sa", g, a.apply(psi.reshape(-1)).reshape(psi.shape)).reshape(-1)
    assert np.abs(lhs - rhs).max() < 1e-13
    lhs = ag.apply_dag(gpsi)
    rhs = np.einsum("...ab,...sb->...sa", g, a.apply_dag(psi.reshape(-1)).reshape(psi.shape)).reshape(-1)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_kappa_zero_is_identity(rng):
    dims = (2, 2, 2, 4)
    op = WilsonOperator(gauge_links(dims, 0.5, 2), 0.0, dims)
    v = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    assert np.array_equal(op.apply(v), v)
