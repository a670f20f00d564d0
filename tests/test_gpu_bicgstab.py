"""GPU parity of BiCGStab, the paper's phase-2 solver (Alg. Incremental eigBiCG,
step 3: "solve the system using BiCGStab", with the DefTol re-deflation), against
the oracle's ``bicgstab`` and ``deflated_bicgstab``: iterations and solution of
plain BiCGStab (FP64), mixed precision reaching the FP64 residual, deflated
BiCGStab with and without the DefTol restart on an eigenspace grown by eigBiCG,
two products with A per step, batch vs alone, and a mixed serving session."""
import numpy as np
import pytest

from oracle.bicg import bicgstab
from oracle.incremental import Eigenspace, deflated_bicgstab
from oracle.wilson import WilsonOperator
from seeded_inputs import gauge_links, workload_source, z2_source
from tests.gpu_util import rel, true_resid, workload

pytestmark = pytest.mark.gpu


def stab_solver(name, **kw):
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload(name)
    args = dict(nev=w["nev"], m=w["m"], n1=w["n1"], tol=1e-10, maxiter=2000, precision="fp64", k_max=4,
                bicgstab=True)
    args.update(kw)
    return Solver(links, w["dims"], w["kappa"], **args), op, w


def test_plain_bicgstab_fp64_matches_oracle():
    s, op, w = stab_solver("4^4")
    b = workload_source("4^4", 0)
    ref = bicgstab(op, b, tol=1e-10)
    with s:
        x, info, _ = s.solve(b, mode="plain")
    assert abs(info[0]["iters"] - ref.iters) <= 1, (info[0]["iters"], ref.iters)
    assert rel(x[0], ref.x) <= 1e-8
    assert true_resid(op, b, x[0]) <= 1e-10
    # two products with A per step (+ the start residual and the final check)
    assert 2 * info[0]["iters"] <= info[0]["matvecs"] <= 2 * info[0]["iters"] + 3


@pytest.mark.parametrize("name", ["4^4", "8^4"])
def test_bicgstab_mixed_precision_reaches_fp64_residual(name):
    s, op, w = stab_solver(name, precision="mixed")
    b = workload_source(name, 1)
    ref = bicgstab(op, b, tol=1e-10)
    with s:
        x, info, _ = s.solve(b, mode="plain")
    assert true_resid(op, b, x[0]) <= 1e-10
    assert info[0]["reliable_updates"] >= 1
    assert info[0]["iters"] <= 1.5 * ref.iters + 10


@pytest.mark.parametrize("deftol", [0.0, 1e-4])
def test_deflated_bicgstab_matches_oracle(deftol):
    """An eigenspace set from FP64 vectors (the same on both sides), then deflated
    BiCGStab with and without the DefTol restart: iteration count within 2 of the
    oracle's deflated_bicgstab, solution to the FP64 tolerance."""
    dims = (4, 4, 4, 4)
    links = gauge_links(dims, 0.05, 21)
    op = WilsonOperator(links, 0.122, dims)
    from oracle.incremental import incremental_eigbicg
    ref_space = incremental_eigbicg(op, [z2_source(dims, 7000 + i) for i in range(2)], nev=6, m=20, n1=2,
                                    tol=1e-10).space
    b = z2_source(dims, 7100)
    ref = deflated_bicgstab(op, ref_space, b, tol=1e-10, deftol=deftol)
    from paper_0911_2285_gb300 import Solver
    with Solver(links, dims, 0.122, nev=6, m=20, n1=2, tol=1e-10, deftol=deftol, precision="fp64", k_max=2,
                bicgstab=True) as s:
        s.eigspace_set(ref_space.Ur.T.copy(), ref_space.Ul.T.copy())
        x, info, _ = s.solve(b, mode="deflated")
    assert abs(info[0]["iters"] - ref.iters) <= 2, (info[0]["iters"], ref.iters)
    assert info[0]["outer_steps"] == (1 if deftol > 0 else 0) == ref.restarts
    assert true_resid(op, b, x[0]) <= 1e-10


def test_bicgstab_batch_equals_alone_bitwise():
    s, op, w = stab_solver("4^4", precision="mixed")
    srcs = np.stack([z2_source(w["dims"], 6300 + i) for i in range(4)])
    with s:
        xb, ib, _ = s.solve(srcs, mode="plain")
        xa, ia, _ = s.solve(srcs[2], mode="plain")
    assert np.array_equal(xa[0], xb[2]) and ia[0]["iters"] == ib[2]["iters"]


def test_incremental_with_bicgstab_phase2_in_a_session():
    """AUTO requests in a serving session of a BiCGStab context: the first n1 run
    eigBiCG (BiCG with the window, then the correction leg in mixed precision), the
    rest deflated BiCGStab, in the same chunks of iterations; every request meets
    the FP64 residual with the oracle's A."""
    s, op, w = stab_solver("4^4", precision="mixed", n1=2, k_max=4)
    srcs = [z2_source(w["dims"], 6400 + i) for i in range(6)]
    xs = [np.zeros_like(b) for b in srcs]
    with s:
        tickets = [s.submit(srcs[i], xs[i], mode="auto") for i in range(6)]
        done = {}
        for _ in range(100000):
            pending = s.progress()
            for t in tickets:
                if t not in done:
                    d, info, st = s.poll(t)
                    if d:
                        done[t] = (info, st)
            if len(done) == 6 and pending == 0:
                break
    modes = [done[t][0]["mode_used"] for t in tickets]
    assert modes[:2] == [1, 1] and all(m == 2 for m in modes[2:])
    for i, t in enumerate(tickets):
        assert done[t][1] == 0
        assert true_resid(op, srcs[i], xs[i]) <= 1e-10
