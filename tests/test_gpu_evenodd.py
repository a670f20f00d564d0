"""GPU parity of the even-odd (Schur complement) operator, the form of the paper's
test matrices (Sec. 3): A_hat = 1 - kappa^2 D_oe D_eo on the odd half lattice,
b_hat = b_o + kappa D_oe b_e, x_e = b_e + kappa D_eo x_o. Checked against
``oracle/evenodd.py``: A_hat and A_hat^+ element-wise (FP64 and FP32), the
BiCG operator pair, plain BiCG on the Schur system (iterations, reconstructed
full solution, full-system residual), fewer iterations than the full system,
mixed precision, Incremental eigBiCG in AUTO mode (the grown H against the
oracle's U_l^H A_hat U_r), and the serving session with full fields."""
import numpy as np
import pytest

from oracle.bicg import bicg
from oracle.evenodd import EvenOddOperator
from seeded_inputs import workload_source, z2_source
from tests.gpu_util import rel, true_resid, workload

pytestmark = pytest.mark.gpu


def eo_problem(name):
    w, links, op = workload(name)
    return w, links, op, EvenOddOperator(links, w["kappa"], w["dims"])


def eo_solver(name, **kw):
    from paper_0911_2285_gb300 import Solver
    w, links, op, eo = eo_problem(name)
    args = dict(nev=w["nev"], m=w["m"], n1=w["n1"], tol=1e-10, maxiter=2000, precision="fp64", k_max=4,
                evenodd=True)
    args.update(kw)
    return Solver(links, w["dims"], w["kappa"], **args), op, eo, w


def rnd(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("mixed", 2e-6)])
def test_schur_operator_matches_oracle(prec, tol):
    s, op, eo, w = eo_solver("8^4", precision="mixed")
    v = np.stack([rnd(eo.n, 3), rnd(eo.n, 4)])
    with s:
        a = s.apply(v, precision=prec)
        ad = s.apply(v, dagger=True, precision=prec)
    for i in range(2):
        assert rel(a[i], eo.apply(v[i])) <= tol
        assert rel(ad[i], eo.apply_dag(v[i])) <= tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_schur_operator_pair_hook(prec, tol):
    s, op, eo, w = eo_solver("8^4", precision=prec, k_max=2)
    p = np.stack([rnd(eo.n, 5), rnd(eo.n, 6)])
    ph = np.stack([rnd(eo.n, 7), rnd(eo.n, 8)])
    with s:
        ap, ahp, sig = s.apply_pair(p, ph, 0)
    for i in range(2):
        ref = eo.apply(p[i])
        assert rel(ap[i], ref) <= tol
        assert rel(ahp[i], eo.apply_dag(ph[i])) <= tol
        assert abs(sig[i] - np.vdot(ph[i], ref)) <= 10 * tol * np.linalg.norm(ph[i]) * np.linalg.norm(ref)


def test_schur_pair_full_size_batch():
    """The launch configuration of the benchmark's even-odd arm: 24^3x64, a batch
    of 8 slots. Slots 0 and 7 hold independent random half fields, compared with
    the oracle's A_hat and A_hat^+ element by element (FP32: 2e-6) with sigma;
    slots 1..6 hold complex multiples of slot 0's fields, whose outputs must be
    the same multiples."""
    w, links, op, eo = eo_problem("24^3x64")
    from paper_0911_2285_gb300 import Solver
    p0, p7, h0, h7 = rnd(eo.n, 31), rnd(eo.n, 37), rnd(eo.n, 51), rnd(eo.n, 57)
    c = np.exp(1j * np.arange(1, 7)) * np.arange(2, 8) / 4.0
    p = np.stack([p0] + [ci * p0 for ci in c] + [p7])
    ph = np.stack([h0] + [ci * h0 for ci in c] + [h7])
    with Solver(links, w["dims"], w["kappa"], nev=2, m=8, n1=1, tol=1e-10, precision="mixed", k_max=8,
                evenodd=True) as s:
        ap, ahp, sig = s.apply_pair(p, ph, 0)
    del p, ph
    for i, (pi, hi) in ((0, (p0, h0)), (7, (p7, h7))):
        ref = eo.apply(pi)
        assert rel(ap[i], ref) <= 2e-6, i
        assert rel(ahp[i], eo.apply_dag(hi)) <= 2e-6, i
        sref = np.vdot(hi, ref)
        assert abs(sig[i] - sref) <= 1e-5 * abs(sref), i
    for j, ci in enumerate(c, start=1):
        assert rel(ap[j], ci * ap[0]) <= 1e-6, j
        assert rel(ahp[j], ci * ahp[0]) <= 1e-6, j
        assert abs(sig[j] - abs(ci) ** 2 * sig[0]) <= 1e-5 * abs(ci) ** 2 * abs(sig[0]), j


def test_schur_bicg_fp64_matches_oracle_and_beats_the_full_system():
    s, op, eo, w = eo_solver("4^4")
    b = workload_source("4^4", 0)
    ref = bicg(eo, eo.prepare(b), tol=1e-10 * np.linalg.norm(b) / np.linalg.norm(eo.prepare(b)))
    xref = eo.reconstruct(b, ref.x)
    with s:
        x, info, _ = s.solve(b, mode="plain")
    assert abs(info[0]["iters"] - ref.iters) <= 1, (info[0]["iters"], ref.iters)
    assert rel(x[0], xref) <= 1e-8
    assert true_resid(op, b, x[0]) <= 1e-10
    assert abs(info[0]["true_resid"] - true_resid(op, b, x[0])) <= 1e-3 * info[0]["true_resid"]
    full = bicg(op, b, tol=1e-10)
    assert info[0]["iters"] < full.iters


@pytest.mark.parametrize("name", ["4^4", "8^4"])
def test_schur_mixed_precision_reaches_fp64_residual(name):
    s, op, eo, w = eo_solver(name, precision="mixed")
    b = workload_source(name, 2)
    with s:
        x, info, _ = s.solve(b, mode="plain")
    assert true_resid(op, b, x[0]) <= 1e-10
    assert info[0]["true_resid"] <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_schur_incremental_auto_mode(prec):
    """Incremental eigBiCG on the Schur system: eigBiCG grows the eigenspace of
    A_hat, deflated BiCG follows; every full solution meets the FP64 residual with
    the oracle's A, and the grown H equals U_l^H A_hat U_r formed by the oracle."""
    s, op, eo, w = eo_solver("4^4", precision=prec, n1=2, k_max=2)
    srcs = np.stack([z2_source(w["dims"], 5100 + i) for i in range(5)])
    with s:
        x1, i1, _ = s.solve(srcs[:2], mode="auto")
        x2, i2, _ = s.solve(srcs[2:], mode="auto")
        ur, ul, H = s.eigspace_get()
    assert [i["mode_used"] for i in i1 + i2] == [1, 1, 2, 2, 2]
    for xi, bi in zip(np.concatenate([x1, x2]), srcs):
        assert true_resid(op, bi, xi) <= 1e-10
    n = ur.shape[0]
    assert n > 0 and ur.shape[1] == eo.n
    href = np.conj(ul) @ np.stack([eo.apply(ur[i]) for i in range(n)], axis=1)
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert np.abs(H - href).max() <= tol * np.abs(href).max()


def test_schur_serving_session_with_full_fields():
    s, op, eo, w = eo_solver("4^4", precision="mixed", n1=1)
    srcs = [z2_source(w["dims"], 5200 + i) for i in range(3)]
    xs = [np.zeros_like(b) for b in srcs]
    with s:
        tickets = [s.submit(srcs[i], xs[i], mode="auto") for i in range(3)]
        done = {}
        for _ in range(100000):
            pending = s.progress()
            for t in tickets:
                if t not in done:
                    d, info, st = s.poll(t)
                    if d:
                        done[t] = (info, st)
            if len(done) == 3 and pending == 0:
                break
    for i, t in enumerate(tickets):
        assert done[t][1] == 0 and done[t][0]["true_resid"] <= 1e-10
        assert true_resid(op, srcs[i], xs[i]) <= 1e-10
