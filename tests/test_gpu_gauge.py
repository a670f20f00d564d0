"""Gauge covariance of the GPU path (Sec. 3's operator): under
U_mu(x) -> G(x) U_mu(x) G(x+mu)^+ with G(x) in SU(3), the Wilson matrix becomes
G A G^+, so A' (G v) = G (A v), the solution of A' x' = G b is x' = G x, and the
BiCG recursion -- whose scalars are inner products, invariant under the unitary
G -- builds the same eigBiCG window matrix H. The GPU never sees G: each context
is built from its own links, and the oracle supplies only the check of x.
"""
import numpy as np
import pytest

from oracle.wilson import WilsonOperator
from seeded_inputs import gauge_links, gaussian_source, random_su3, volume

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 8)
KAPPA = 0.12


def transformed():
    lx, ly, lz, lt = DIMS
    links = gauge_links(DIMS, 0.5, 3)
    g = random_su3(np.random.default_rng(99), volume(DIMS), 2.0).reshape(lt, lz, ly, lx, 3, 3)
    lg = np.empty_like(links)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=3 - mu)
        lg[mu] = np.einsum("...ab,...bc,...dc->...ad", g, links[mu], np.conj(g_fwd))

    def rot(v):
        psi = np.asarray(v).reshape(lt, lz, ly, lx, 4, 3)
        return np.einsum("...ab,...sb->...sa", g, psi).reshape(-1)

    return links, lg, rot


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_operator_and_solution_are_gauge_covariant(prec):
    from paper_0911_2285_gb300 import Solver
    links, lg, rot = transformed()
    b = gaussian_source(DIMS, 4)
    gb = rot(b)
    tol_op = 1e-13 if prec == "fp64" else 5e-6   # FP32: both sides round their own links
    with Solver(links, DIMS, KAPPA, nev=4, m=16, precision=prec, k_max=1) as s, \
            Solver(lg, DIMS, KAPPA, nev=4, m=16, precision=prec, k_max=1) as sg:
        for p in ("fp64", prec):
            lhs = sg.apply(gb, precision=p)[0]
            rhs = rot(s.apply(b, precision=p)[0])
            assert np.abs(lhs - rhs).max() <= (1e-13 if p == "fp64" else tol_op) * np.abs(rhs).max()
        x, _, _ = s.solve(b, mode="plain")
        xg, _, _ = sg.solve(gb, mode="plain")
    opg = WilsonOperator(lg, KAPPA, DIMS)
    assert np.linalg.norm(gb - opg.apply(xg[0])) <= 1e-10 * np.linalg.norm(gb)
    gx = rot(x[0])
    assert np.linalg.norm(xg[0] - gx) <= 1e-8 * np.linalg.norm(gx)


def test_eigbicg_window_is_gauge_invariant():
    """FP64 eigBiCG without a restart (kappa = 0.11: the oracle's BiCG needs 49
    iterations, below m = 64): the window matrix H of the transformed problem
    equals the original one to rounding."""
    from paper_0911_2285_gb300 import Solver
    links, lg, rot = transformed()
    b = gaussian_source(DIMS, 5)
    with Solver(links, DIMS, 0.11, nev=8, m=64, precision="fp64", k_max=1) as s, \
            Solver(lg, DIMS, 0.11, nev=8, m=64, precision="fp64", k_max=1) as sg:
        s.solve(b, mode="eigbicg")
        H, ritz, restarts = s.last_window(0)
        sg.solve(rot(b), mode="eigbicg")
        Hg, ritzg, restartsg = sg.last_window(0)
    assert restarts == 0 and restartsg == 0
    n = min(H.shape[0], Hg.shape[0])
    assert abs(H.shape[0] - Hg.shape[0]) <= 1
    assert np.abs(H[:n, :n] - Hg[:n, :n]).max() <= 1e-10 * np.abs(H).max()
