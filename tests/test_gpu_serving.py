"""GPU tests of the serving session (continuous batching through lqcd_submit /
lqcd_progress / lqcd_poll): every request meets the FP64 true residual with the
oracle's operator, a request gives the same solution bit for bit alone and in a
mix that joins and leaves the batch around it, the incremental eigenspace grows
from the first n1 requests, and several resident operators serve one trace."""
import numpy as np
import pytest

from seeded_inputs import workload_source, z2_source
from tests.gpu_util import true_resid, workload

pytestmark = pytest.mark.gpu


def solver(name, **kw):
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload(name)
    args = dict(nev=w["nev"], m=w["m"], n1=w["n1"], tol=1e-10, maxiter=2000, precision="mixed", k_max=4)
    args.update(kw)
    return Solver(links, w["dims"], w["kappa"], **args), op, w


def drain(s, tickets, limit=100000):
    out = {}
    for _ in range(limit):
        pending = s.progress()
        for t in list(tickets):
            done, info, status = s.poll(t)
            if done:
                out[t] = (info, status)
                tickets.remove(t)
        if not tickets and pending == 0:
            return out
    raise AssertionError("session did not drain")


@pytest.mark.parametrize("mode", ["plain", "deflated"])
def test_alone_equals_in_mix_bitwise(mode):
    """Same eigenspace, same slot-independent reductions: a request solved alone and
    one that shares the batch with requests admitted before, with and after it gives
    the same x bit for bit and the same iteration count."""
    s, op, w = solver("4^4", n1=1, deftol=1e-4 if mode == "deflated" else 0.0)
    srcs = [z2_source(w["dims"], 8000 + i) for i in range(7)]
    with s:
        if mode == "deflated":
            s.solve(z2_source(w["dims"], 8100), mode="eigbicg")
            assert s.eigspace_size() > 0
        xa = np.zeros_like(srcs[3])
        ta = s.submit(srcs[3], xa, mode=mode)
        ra = drain(s, [ta])
        xs = [np.zeros_like(b) for b in srcs]
        tickets = [s.submit(srcs[i], xs[i], mode=mode) for i in range(3)]
        for _ in range(3):                      # the first three run a few chunks alone
            s.progress()
        tickets += [s.submit(srcs[i], xs[i], mode=mode) for i in range(3, 7)]   # 7 > 4 slots: queueing
        res = drain(s, list(tickets))
    assert np.array_equal(xa, xs[3])
    assert ra[ta][0]["iters"] == res[tickets[3]][0]["iters"]
    assert ra[ta][0]["outer_steps"] == (1 if mode == "deflated" else 0)
    for b, x, t in zip(srcs, xs, tickets):
        info, status = res[t]
        assert status == 0
        assert true_resid(op, b, x) <= 1e-10


def test_session_matches_lqcd_solve_iterations():
    """The session runs the same BiCG as lqcd_solve: same iteration counts (FP64)."""
    s, op, w = solver("4^4", precision="fp64", k_max=2)
    srcs = np.stack([workload_source("4^4", i) for i in range(3)])
    with s:
        xr, ir, _ = s.solve(srcs, mode="plain")
        xs = [np.zeros_like(b) for b in srcs]
        ts = [s.submit(srcs[i], xs[i], mode="plain") for i in range(3)]
        res = drain(s, list(ts))
    for i in range(3):
        assert res[ts[i]][0]["iters"] == ir[i]["iters"]
        assert np.abs(xs[i] - xr[i]).max() <= 1e-9 * np.abs(xr[i]).max()


def test_session_incremental_auto():
    """AUTO in the session: the first n1 requests run eigBiCG (both in flight at once)
    and grow the eigenspace as they retire; the rest wait for a slot and are deflated."""
    s, op, w = solver("4^4", n1=2, k_max=2)
    srcs = [z2_source(w["dims"], 8200 + i) for i in range(6)]
    xs = [np.zeros_like(b) for b in srcs]
    with s:
        ts = [s.submit(b, x) for b, x in zip(srcs, xs)]
        res = drain(s, list(ts))
        n_def = s.eigspace_size()
    assert [res[t][0]["mode_used"] for t in ts] == [1, 1, 2, 2, 2, 2]
    assert 0 < n_def <= 2 * w["nev"]
    for b, x, t in zip(srcs, xs, ts):
        assert res[t][1] == 0
        assert true_resid(op, b, x) <= 1e-10


def test_solve_refused_while_session_busy():
    from paper_0911_2285_gb300 import lqcd
    s, op, w = solver("4^4", k_max=2)
    b = workload_source("4^4", 0)
    x = np.zeros_like(b)
    with s:
        t = s.submit(b, x, mode="plain")
        s.progress()
        with pytest.raises(lqcd.LQCDError) as e:
            s.solve(b, mode="plain")
        assert e.value.status == lqcd.ERR_STATE
        drain(s, [t])
        x2, info, _ = s.solve(b, mode="plain")       # free again
    assert true_resid(op, b, x) <= 1e-10 and true_resid(op, b, x2[0]) <= 1e-10


def test_serving_loop_two_operators():
    """The request loop over two resident operators (two gauge fields) on a Poisson
    trace: every request completes, meets the true residual of its own operator, and the
    report's latency percentiles are ordered."""
    from paper_0911_2285_gb300.serving import Server, poisson_trace
    sa, opa, wa = solver("4^4", n1=1, k_max=3)
    sb, opb, wb = solver("8^4", n1=1, k_max=3, maxiter=4000)
    ops = {"4^4": opa, "8^4": opb}
    dims = {"4^4": wa["dims"], "8^4": wb["dims"]}
    trace = poisson_trace(10, rate_hz=200.0, mix={"4^4": 2, "8^4": 1}, seed=3,
                          make_source=lambda name, i: z2_source(dims[name], 9000 + i))
    with sa, sb:
        rep, reqs = Server({"4^4": sa, "8^4": sb}).run(trace, realtime=True)
    summ = rep.summary()
    assert summ["requests"] == 10 and summ["failed"] == 0
    assert 0 < summ["latency_p50_s"] <= summ["latency_p99_s"]
    for r in reqs:
        assert r.status == 0
        assert true_resid(ops[r.op], r.b, r.x) <= 1e-10


def test_session_edge_cases():
    """A zero source completes with x = 0; a request that hits maxiter reports
    LQCD_ERR_NOCONV without disturbing the request beside it; unknown tickets and
    switching the tensor-core path while requests are in flight are refused."""
    from paper_0911_2285_gb300 import lqcd
    s, op, w = solver("4^4", k_max=2, maxiter=6)
    b = workload_source("4^4", 0)
    z = np.zeros_like(b)
    xz, xb = np.zeros_like(b), np.zeros_like(b)
    with s:
        tz = s.submit(z, xz, mode="plain")
        tb = s.submit(b, xb, mode="plain")
        with pytest.raises(lqcd.LQCDError) as e:
            s.set_tensor_cores(False)
        assert e.value.status == lqcd.ERR_STATE
        res = drain(s, [tz, tb])
        with pytest.raises(lqcd.LQCDError):
            s.poll(10 ** 9)
        s.set_tensor_cores(True)   # free again
    assert res[tz][1] == lqcd.OK and np.all(xz == 0)
    assert res[tb][1] == lqcd.ERR_NOCONV and res[tb][0]["iters"] == 6


def test_admission_by_device_memory_queues_and_admits_as_windows_free():
    """hbm_budget_bytes with room for the fixed plan and one eigBiCG window: of three
    eigBiCG requests only one holds a window at a time, the others wait in the queue
    (no error) while a plain request submitted after them is admitted past them;
    each waiting request is admitted when the window before it is released, and
    every request finishes with the FP64 residual."""
    from paper_0911_2285_gb300 import lqcd
    s0, op, w = solver("8^4", n1=3)
    with s0:
        plan, win, att = s0.memory_info()
    assert att == 0 and win > 0
    s, op, w = solver("8^4", n1=3, hbm_budget_bytes=plan + win + win // 2)
    srcs = [z2_source(w["dims"], 8500 + i) for i in range(4)]
    xs = [np.zeros_like(b) for b in srcs]
    with s:
        tickets = [s.submit(srcs[i], xs[i], mode="eigbicg") for i in range(3)]
        tickets.append(s.submit(srcs[3], xs[3], mode="plain"))
        s.progress()
        assert s.memory_info()[2] == 1
        done, seen, max_att = {}, 0, 0
        for _ in range(100000):
            pending = s.progress()
            max_att = max(max_att, s.memory_info()[2])
            for t in tickets:
                if t not in done:
                    d, info, st = s.poll(t)
                    if d:
                        done[t] = (info, st)
            if len(done) == 4 and pending == 0:
                break
        else:
            raise AssertionError("session did not drain")
        assert s.memory_info()[2] == 0
    assert max_att == 1
    # the plain request, submitted last, finished before the last eigBiCG one
    order = list(done)
    assert order.index(tickets[3]) < order.index(tickets[2])
    for i, t in enumerate(tickets):
        info, st = done[t]
        assert st == lqcd.OK
        assert info["mode_used"] == (1 if i < 3 else 3)
        assert true_resid(op, srcs[i], xs[i]) <= 1e-10


def test_budget_without_room_for_a_window():
    """A budget that holds the fixed plan but no eigBiCG window: an explicit eigBiCG
    request finishes with LQCD_ERR_OOM, an AUTO request runs deflated BiCG instead,
    and a batched eigBiCG solve returns LQCD_ERR_OOM."""
    from paper_0911_2285_gb300 import lqcd
    s0, op, w = solver("8^4")
    with s0:
        plan, win, _ = s0.memory_info()
    s, op, w = solver("8^4", hbm_budget_bytes=plan + win // 2)
    b = z2_source(w["dims"], 8600)
    with s:
        x1, x2 = np.zeros_like(b), np.zeros_like(b)
        t1 = s.submit(b, x1, mode="eigbicg")
        t2 = s.submit(b, x2, mode="auto")
        res = drain(s, [t1, t2])
        assert res[t1][1] == lqcd.ERR_OOM
        assert res[t2][1] == lqcd.OK and res[t2][0]["mode_used"] == 2
        assert true_resid(op, b, x2) <= 1e-10
        _, _, st = s.solve(b, mode="eigbicg", raise_on_fail=False)
        assert st == lqcd.ERR_OOM
