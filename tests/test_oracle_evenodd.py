"""Pins of the even-odd (Schur complement) Wilson oracle: the reconstructed
solution solves the full system, det A = det A_hat on a 2^4 lattice, the
gamma5 symmetry survives, the Schur system needs fewer BiCG iterations, and
the free field's Schur spectrum follows from the hopping spectrum."""
import numpy as np

from oracle.bicg import bicg
from oracle.evenodd import EvenOddOperator
from oracle.wilson import WilsonOperator
from seeded_inputs import WORKLOADS, gauge_links, gaussian_source, workload_links


def test_schur_solve_reconstructs_the_full_solution():
    w = WORKLOADS["4^4"]
    links = workload_links("4^4")
    full = WilsonOperator(links, w["kappa"], w["dims"])
    eo = EvenOddOperator(links, w["kappa"], w["dims"])
    b = gaussian_source(w["dims"], 21)
    res = bicg(eo, eo.prepare(b), tol=1e-12)
    x = eo.reconstruct(b, res.x)
    assert np.linalg.norm(b - full.apply(x)) <= 1e-10 * np.linalg.norm(b)
    ref = bicg(full, b, tol=1e-12)
    assert res.iters < ref.iters


def test_determinant_and_gamma5_symmetry_2x4():
    dims, kappa = (2, 2, 2, 2), 0.13
    links = gauge_links(dims, 0.5, 4)
    a = WilsonOperator(links, kappa, dims).dense()
    eo = EvenOddOperator(links, kappa, dims)
    ah = eo.dense()
    s_full, l_full = np.linalg.slogdet(a)
    s_eo, l_eo = np.linalg.slogdet(ah)
    assert abs(l_full - l_eo) <= 1e-10 * abs(l_full) + 1e-12
    assert abs(s_full - s_eo) <= 1e-10
    g5 = np.stack([eo.gamma5(e) for e in np.eye(eo.n)], axis=1)
    assert np.abs(g5 @ ah @ g5 - np.conj(ah.T)).max() <= 1e-13


def test_free_field_schur_spectrum():
    """U = 1: D_hop has eigenvalues d with -d also an eigenvalue (the parity
    sign flip), so A_hat's eigenvalues are 1 - kappa^2 d^2 over the hopping spectrum."""
    dims, kappa = (4, 4, 2, 2), 0.1
    lx, ly, lz, lt = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    for c in range(3):
        u[..., c, c] = 1.0
    full = WilsonOperator(u, kappa, dims).dense()
    d = (np.eye(full.shape[0]) - full) / kappa          # D_hop
    dev = np.linalg.eigvals(d)
    expect = np.sort_complex(1 - kappa ** 2 * dev ** 2)
    got = np.linalg.eigvals(EvenOddOperator(u, kappa, dims).dense())
    # every Schur eigenvalue is one of the predicted values (each appears twice there)
    for g in got:
        assert np.min(np.abs(expect - g)) <= 1e-10
