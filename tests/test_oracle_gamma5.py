"""Pins of the gamma5-Hermitian BiCG oracle (Sec. 4): its iterates equal the
general BiCG with the shadow start gamma5 r_0 (which needs A^H), its scalars
are real, it uses one product with A per iteration, and with the same shadow
start the eigBiCG window's left vectors are gamma5 images of the right ones
and the projected matrix is real."""
import numpy as np
import pytest

from oracle.bicg import bicg, bicg_g5, eigbicg
from seeded_inputs import WORKLOADS, gaussian_source, workload_links
from oracle.wilson import WilsonOperator


@pytest.fixture(scope="module")
def problem():
    w = WORKLOADS["4^4"]
    links = workload_links("4^4")
    return WilsonOperator(links, w["kappa"], w["dims"]), gaussian_source(w["dims"], 11)


def test_g5_bicg_equals_bicg_with_gamma5_shadow(problem):
    op, b = problem
    ref = bicg(op, b, tol=1e-10, rhat0=op.gamma5(b), history=True)
    g5 = bicg_g5(op, b, tol=1e-10, history=True)
    assert g5.iters == ref.iters
    # the two recursions round differently and BiCG amplifies rounding as it goes:
    # tight agreement early, FP64-recurrence agreement throughout
    for j, ((a1, b1), (a0, b0)) in enumerate(zip(g5.snapshots, ref.snapshots)):
        tol = 1e-11 if j < 10 else 1e-6
        assert abs(a1 - a0) <= tol * abs(a0) and abs(b1 - b0) <= tol * abs(b0), j
    assert np.linalg.norm(g5.x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    assert np.linalg.norm(b - op.apply(g5.x)) <= 1e-10 * np.linalg.norm(b)


def test_g5_bicg_real_scalars_and_one_product(problem):
    op, b = problem
    ref = bicg(op, b, tol=1e-10, rhat0=op.gamma5(b), history=True)
    # the general recursion's alpha and beta come out real with this shadow start
    assert max(abs(np.imag(a)) / abs(a) for a, _ in ref.snapshots[:10]) <= 1e-12
    assert max(abs(np.imag(a)) / abs(a) for a, _ in ref.snapshots) <= 1e-8
    assert max(abs(np.imag(c)) / abs(c) for _, c in ref.snapshots) <= 1e-8
    mv0 = op.matvecs
    g5 = bicg_g5(op, b, tol=1e-10)
    # one A product per iteration, plus the start residual and the true-residual checks
    assert op.matvecs - mv0 <= g5.iters + 3
    assert ref.matvecs >= 2 * ref.iters


def test_g5_window_left_vectors_and_real_H(problem):
    op, b = problem
    res = eigbicg(op, b, nev=4, m=16, tol=1e-10, rhat0=op.gamma5(b))
    V, W, H = res.first_window
    for k in range(V.shape[1]):
        g = op.gamma5(V[:, k])
        c = np.vdot(g, W[:, k]) / np.vdot(g, g)
        assert np.linalg.norm(W[:, k] - c * g) <= 1e-10 * np.linalg.norm(W[:, k])
        assert abs(np.imag(c)) <= 1e-10 * abs(c)
    assert np.max(np.abs(np.imag(H))) <= 1e-10 * np.max(np.abs(H))
    # Ritz values of a real H: real or in conjugate pairs
    lam = np.linalg.eigvals(np.real(H))
    for l in lam:
        if abs(l.imag) > 1e-9:
            assert np.min(np.abs(lam - np.conj(l))) <= 1e-8 * abs(l)


def test_g5_incremental_solves_weak_links():
    """Incremental eigBiCG with the gamma5 shadow start in every BiCG run (Sec. 4)
    on a near-free field: every solution meets the tolerance and the phases run
    as the algorithm says. (The restarts keep nev pairs by modulus and may split a
    conjugate pair at the cut, so after a restart the window's Ritz values are no
    longer exactly paired; the first window's are, see above.) Gaussian sources:
    a complex Z2 source has entries of modulus one, so
    rho_0 = r_0^H gamma5 r_0 = |upper spins|^2 - |lower spins|^2 = 0 and the gamma5
    shadow start breaks down at once (pinned below)."""
    from oracle.incremental import incremental_eigbicg
    from seeded_inputs import gauge_links
    dims = (4, 4, 4, 4)
    op = WilsonOperator(gauge_links(dims, 0.05, 21), 0.122, dims)
    srcs = [gaussian_source(dims, 7000 + i) for i in range(4)]
    out = incremental_eigbicg(op, srcs, nev=6, m=20, n1=2, tol=1e-10, gamma5=True)
    for x, b in zip(out.x, srcs):
        assert np.linalg.norm(b - op.apply(x)) <= 1e-10 * np.linalg.norm(b)
    assert out.modes == ["eigbicg", "eigbicg", "deflated", "deflated"]
    assert out.space.size >= 6


def test_g5_shadow_start_breaks_down_on_z2_sources(problem):
    """Entries of modulus one give r_0^H gamma5 r_0 = 0 exactly: BiCG with the
    gamma5 shadow start reports a rho breakdown before its first step."""
    from oracle.bicg import Breakdown
    from seeded_inputs import z2_source
    op, _ = problem
    b = z2_source(op.dims, 5)
    assert abs(np.vdot(op.gamma5(b), b)) <= 1e-14 * np.vdot(b, b).real
    with pytest.raises(Breakdown):
        bicg_g5(op, b, tol=1e-10)
