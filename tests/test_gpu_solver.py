"""GPU parity of the solve path: BiCG (FP64 and mixed precision), the eigBiCG window
(projected matrix H and Ritz values against the oracle's Algorithm eigBiCG),
oblique deflation and the eigenspace growth of Algorithm Incremental eigBiCG,
Rayleigh-Ritz, batching (alone vs in a batch) and error reporting."""
import numpy as np
import pytest

from oracle.bicg import bicg, eigbicg
from oracle.incremental import Eigenspace, deflate, rayleigh_ritz
from seeded_inputs import gauge_links, gaussian_source, workload_source, z2_source
from tests.gpu_util import rel, small_problem, true_resid, workload

pytestmark = pytest.mark.gpu


def solver(name, **kw):
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload(name)
    args = dict(nev=w["nev"], m=w["m"], n1=w["n1"], tol=1e-10, maxiter=2000, precision="fp64", k_max=4)
    args.update(kw)
    return Solver(links, w["dims"], w["kappa"], **args), op, w


def test_plain_bicg_fp64_matches_oracle_iterations():
    s, op, w = solver("4^4")
    b = workload_source("4^4", 0)
    with s:
        x, info, _ = s.solve(b, mode="plain")
    ref = bicg(op, b, tol=1e-10)
    assert abs(info[0]["iters"] - ref.iters) <= 1
    assert true_resid(op, b, x[0]) <= 1e-10
    assert rel(x[0], ref.x) <= 1e-8
    assert info[0]["true_resid"] <= 1e-10


@pytest.mark.parametrize("name", ["4^4", "8^4"])
def test_mixed_precision_reaches_fp64_residual(name):
    s, op, w = solver(name, precision="mixed")
    b = workload_source(name, 0)
    with s:
        x, info, _ = s.solve(b, mode="plain")
    assert true_resid(op, b, x[0]) <= 1e-10
    assert info[0]["reliable_updates"] >= 1
    ref = bicg(op, b, tol=1e-10)
    assert info[0]["iters"] <= 1.5 * ref.iters + 10


def test_eigbicg_first_window_H_matches_oracle():
    """No restart (m larger than the iteration count): the projected matrix built
    from the GPU BiCG scalars equals the oracle's to 1e-11 (FP64)."""
    s, op, w = solver("4^4", m=64, nev=8)
    b = workload_source("4^4", 0)
    with s:
        x, info, _ = s.solve(b, mode="eigbicg")
        H, ritz, restarts = s.last_window(0)
    ref = eigbicg(op, b, nev=8, m=64)
    assert restarts == 0 and ref.restarts == 0
    assert H.shape == ref.H.shape
    assert np.abs(H - ref.H).max() <= 1e-11 * np.abs(ref.H).max()
    assert np.abs(np.sort_complex(ritz) - np.sort_complex(ref.evals)).max() <= 1e-9
    assert true_resid(op, b, x[0]) <= 1e-10


def test_eigbicg_restarts_match_oracle_ritz_values():
    s, op, w = solver("4^4", m=24, nev=8)
    b = workload_source("4^4", 0)
    with s:
        x, info, _ = s.solve(b, mode="eigbicg")
        H, ritz, restarts = s.last_window(0)
    ref = eigbicg(op, b, nev=8, m=24)
    assert restarts == ref.restarts and restarts >= 2
    assert info[0]["iters"] == ref.iters
    assert np.abs(np.sort_complex(ritz) - np.sort_complex(ref.evals)).max() <= 1e-6 * np.abs(ref.evals).max()
    assert true_resid(op, b, x[0]) <= 1e-10


def test_eigbicg_ritz_vectors_match_oracle_after_restarts():
    """FP64 eigBiCG with restarts: the stored right/left Ritz vectors (first eigBiCG
    source, empty eigenspace: normalised Ritz vectors) span the oracle's ones."""
    s, op, w = solver("4^4", m=24, nev=8, n1=1)
    b = workload_source("4^4", 0)
    with s:
        s.solve(b, mode="eigbicg")
        ur, ul, H = s.eigspace_get()
        _, ritz, restarts = s.last_window(0)
    ref = eigbicg(op, b, nev=8, m=24)
    assert restarts >= 2
    for i in range(len(ritz)):
        j = int(np.argmin(np.abs(ref.evals - ritz[i])))
        u = ref.U[:, j] / np.linalg.norm(ref.U[:, j])
        q = ref.Q[:, j] / np.linalg.norm(ref.Q[:, j])
        assert abs(abs(np.vdot(u, ur[i])) - 1) <= 1e-6
        assert abs(abs(np.vdot(q, ul[i])) - 1) <= 1e-6


def test_eigbicg_free_field_ritz_closed_form_on_gpu():
    from paper_0911_2285_gb300 import Solver
    dims = (4, 4, 4, 4)
    lx, ly, lz, lt = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    for a in range(3):
        u[..., a, a] = 1.0
    kappa = 0.12
    exact = 1 - 8 * kappa
    b = gaussian_source(dims, 7)
    for prec in ("fp64", "mixed"):
        with Solver(u, dims, kappa, nev=4, m=16, n1=1, tol=1e-12 if prec == "fp64" else 1e-10,
                    precision=prec, k_max=1) as s:
            s.solve(b, mode="eigbicg")
            _, ritz, _ = s.last_window(0)
            lam0 = ritz[np.argmin(np.abs(ritz - exact))]
            # window Ritz value: FP64 to 1e-8; FP32 Krylov vectors with reliable updates to 1e-2
            tol = 1e-8 if prec == "fp64" else 1e-2
            assert abs(lam0 - exact) <= tol * exact, ritz
            # FP64 Rayleigh-Ritz on the stored eigenspace (Sec. 2): two-sided accuracy
            ev, res, _, _ = s.eigs()
            best = ev[np.argmin(np.abs(ev - exact))]
            # MIXED: the lowest free-field eigenvalue is 12-fold degenerate and a
            # single source's Krylov space holds one vector of it; FP32 rounding
            # excites the other eleven directions, which the window (nev = 4) cannot
            # hold apart, so the error depends on the rounding of the operator shape
            # the autotuner picks (1.2e-6 .. 3.6e-4 measured). The fixed 1e-6 bound
            # on a non-degenerate spectrum is in test_gpu_eigenspace.py.
            if prec == "fp64":
                assert abs(best - exact) <= 1e-10 * exact, ev
            else:
                assert abs(best - exact) <= 1e-3 * exact, (ev, res)


def test_deflate_matches_oracle():
    """Oblique deflation on a given eigenspace (FP64): x0 + U_r H^{-1} U_l^H (b - A x0)."""
    s, op, w = solver("4^4", n_def_max=16)
    rng = np.random.default_rng(3)
    k = 12
    ur = rng.standard_normal((k, op.n)) + 1j * rng.standard_normal((k, op.n))
    ul = rng.standard_normal((k, op.n)) + 1j * rng.standard_normal((k, op.n))
    aur = np.stack([op.apply(ur[i]) for i in range(k)], axis=1)
    sp = Eigenspace(op.n, ur.T.copy(), ul.T.copy(), np.conj(ul) @ aur)
    b = np.stack([workload_source("4^4", 0), z2_source(w["dims"], 5)])
    x0 = np.stack([np.zeros(op.n, complex), rng.standard_normal(op.n) + 0j])
    with s:
        s.eigspace_set(ur, ul)
        ur2, ul2, H = s.eigspace_get()
        assert np.abs(H - sp.H).max() <= 1e-12 * np.abs(sp.H).max()
        xd = s.deflate(b, x0)
    for i in range(2):
        ref = deflate(op, sp, b[i], x0[i])
        assert rel(xd[i], ref) <= 1e-10
        r = b[i] - op.apply(xd[i])
        assert np.abs(np.conj(ul) @ r).max() <= 1e-9 * np.linalg.norm(b[i])


def test_rayleigh_ritz_exact_eigenvectors():
    from paper_0911_2285_gb300 import Solver
    import scipy.linalg as sla
    dims = (2, 2, 2, 2)
    links, op = small_problem(dims, kappa=0.124)
    a = op.dense()
    lam, zl, zr = sla.eig(a, left=True, right=True)
    idx = np.argsort(np.abs(lam))[:8]
    with Solver(links, dims, 0.124, nev=4, m=12, precision="fp64", k_max=2, n_def_max=16) as s:
        s.eigspace_set(zr[:, idx].T.copy(), zl[:, idx].T.copy())
        ev, res, u, wv = s.eigs(vectors=True)
    cost = np.abs(ev[:, None] - lam[idx][None, :])
    assert cost.min(axis=1).max() <= 1e-11
    assert res.max() <= 1e-11
    for i in range(len(ev)):
        assert np.linalg.norm(op.apply(u[i]) - ev[i] * u[i]) <= 1e-10 * np.linalg.norm(u[i])
        assert np.linalg.norm(op.apply_dag(wv[i]) - np.conj(ev[i]) * wv[i]) <= 1e-10 * np.linalg.norm(wv[i])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_incremental_auto_mode(prec):
    """Algorithm Incremental eigBiCG: n1 eigBiCG solves grow the eigenspace, the rest
    are deflated; every solution meets the FP64 true residual with the oracle's A;
    the grown H equals U_l^H A U_r formed by the oracle."""
    s, op, w = solver("4^4", precision=prec, n1=2, k_max=2)
    srcs = np.stack([z2_source(w["dims"], 5000 + i) for i in range(5)])
    with s:
        x1, i1, _ = s.solve(srcs[:2], mode="auto")
        assert [i["mode_used"] for i in i1] == [1, 1]
        n_def = s.eigspace_size()
        assert 8 < n_def <= 16
        x2, i2, _ = s.solve(srcs[2:], mode="auto")
        assert [i["mode_used"] for i in i2] == [2, 2, 2]
        ur, ul, H = s.eigspace_get()
    for xi, bi in zip(np.concatenate([x1, x2]), srcs):
        assert true_resid(op, bi, xi) <= 1e-10
    aur = np.stack([op.apply(ur[i]) for i in range(n_def)], axis=1)
    href = np.conj(ul) @ aur
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert np.abs(H - href).max() <= tol * np.abs(href).max()
    # new blocks are oblique-orthogonal to the earlier ones
    n1 = min(8, n_def)
    assert np.abs(np.conj(ul[:n1]) @ ur[n1:].T).max() <= (1e-9 if prec == "fp64" else 1e-4)


def test_batch_equals_alone_bitwise():
    """Deterministic per-slot reductions: a source solved alone and inside a batch of
    four gives the same x bit for bit (same eigenspace snapshot)."""
    s, op, w = solver("4^4", precision="mixed", k_max=4)
    srcs = np.stack([z2_source(w["dims"], 6000 + i) for i in range(4)])
    with s:
        xb, ib, _ = s.solve(srcs, mode="plain")
        xa, ia, _ = s.solve(srcs[2], mode="plain")
    assert np.array_equal(xa[0], xb[2])
    assert ia[0]["iters"] == ib[2]["iters"]


def test_noconv_and_zero_source():
    from paper_0911_2285_gb300 import Solver, lqcd
    w, links, op = workload("4^4")
    with Solver(links, w["dims"], w["kappa"], nev=4, m=12, tol=1e-10, maxiter=5, precision="mixed", k_max=2) as s:
        b = workload_source("4^4", 0)
        x, info, st = s.solve(b, mode="plain", raise_on_fail=False)
        assert st == lqcd.ERR_NOCONV
        assert info[0]["iters"] == 5
        assert info[0]["true_resid"] > 1e-10
        z = np.zeros_like(b)
        x, info, st = s.solve(z, mode="plain", raise_on_fail=False)
        assert st == lqcd.OK and np.all(x == 0)


def test_deflated_with_deftol_restart():
    s, op, w = solver("4^4", precision="mixed", n1=1, deftol=1e-4)
    srcs = np.stack([z2_source(w["dims"], 7000 + i) for i in range(2)])
    with s:
        s.solve(srcs[0], mode="eigbicg")
        x, info, _ = s.solve(srcs[1], mode="deflated")
    assert info[0]["outer_steps"] == 1
    assert true_resid(op, srcs[1], x[0]) <= 1e-10


def test_second_eigbicg_solve_starts_a_fresh_window():
    """A windowed solve on slots that already restarted in an earlier solve sees a
    fresh projected matrix: the same source gives the same window H, Ritz values
    and restart count as the first time, bit for bit (mixed precision, 8^4)."""
    s, op, w = solver("8^4", precision="mixed", n1=1, k_max=2)
    b = z2_source(w["dims"], 777)
    with s:
        s.solve(b, mode="eigbicg")
        h1, l1, r1 = s.last_window()
        s.reset_eigenspace()
        s.solve(b, mode="eigbicg")
        h2, l2, r2 = s.last_window()
    assert r1 == r2 and r1 >= 3
    assert np.array_equal(h1, h2) and np.array_equal(l1, l2)


def test_eigenspace_checkpoint_resume(tmp_path):
    """Checkpoint/resume of the accumulated eigenspace: a new context on the same
    gauge field loads the saved U_r, U_l (H recomputed on its operator) and deflates
    like the original; a context with another kappa refuses the file."""
    from paper_0911_2285_gb300 import Solver
    s, op, w = solver("4^4", precision="mixed", n1=1, k_max=2)
    b1, b2 = z2_source(w["dims"], 8800), z2_source(w["dims"], 8801)
    path = tmp_path / "space.npz"
    with s:
        s.solve(b1, mode="eigbicg")
        ur, ul, H = s.eigspace_get()
        s.save_eigenspace(path)
        _, i1, _ = s.solve(b2, mode="deflated")
    s2, _, _ = solver("4^4", precision="mixed", n1=1, k_max=2)
    with s2:
        s2.load_eigenspace(path)
        ur2, ul2, H2 = s2.eigspace_get()
        x2, i2, _ = s2.solve(b2, mode="deflated")
    assert ur.shape[0] > 0 and np.array_equal(ur, ur2) and np.array_equal(ul, ul2)
    assert np.abs(H2 - H).max() <= 1e-5 * np.abs(H).max()
    assert abs(i1[0]["iters"] - i2[0]["iters"]) <= 2
    assert true_resid(op, b2, x2[0]) <= 1e-10
    _, links, _ = workload("4^4")
    with Solver(links, w["dims"], 0.11, nev=w["nev"], m=w["m"], precision="mixed", k_max=1) as s3:
        with pytest.raises(ValueError):
            s3.load_eigenspace(path)


def test_batch_size_autotuner_picks_the_fastest_rate_and_is_used():
    """k_max = 0: init times one BiCG iteration on 1, 2, 4, 8 slots and keeps the
    batch size with the most right-hand sides per second; lqcd_solve then runs the
    sources in batches of that size (sources of one batch share its wall time)."""
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload("8^4")
    with Solver(links, w["dims"], w["kappa"], nev=w["nev"], m=w["m"], tol=1e-10, precision="mixed",
                k_max=0) as s:
        k = s.batch_size()
        ms = s.batch_timings()
        rates = {kk: kk / ms[kk] for kk in (1, 2, 4, 8)}
        assert all(ms[kk] > 0 for kk in rates)
        assert k in rates and rates[k] >= 0.99 * max(rates.values()), (k, rates)
        srcs = np.stack([z2_source(w["dims"], 9100 + i) for i in range(k + 1)])
        x, info, _ = s.solve(srcs, mode="plain")
    secs = [i["seconds"] for i in info]
    assert len(set(secs[:k])) == 1 and secs[k] != secs[0]
    for i in range(k + 1):
        assert true_resid(op, srcs[i], x[i]) <= 1e-10
