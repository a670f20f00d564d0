"""Host logic of the serving loop, with a stand-in solver: trace statistics,
admission order, completion and latency bookkeeping."""
import numpy as np

from paper_0911_2285_gb300.serving import Request, ServeReport, Server, poisson_trace


class FakeSolver:
    """Runs each request for a fixed number of progress() calls on k slots; x = 2 b."""

    def __init__(self, k, steps):
        self.k, self.steps = k, steps
        self.queue, self.slots, self.done, self.next = [], {}, {}, 1
        self.admitted = []
        self.max_busy = 0

    def submit(self, b, x, mode="auto"):
        t = self.next
        self.next += 1
        self.queue.append((t, b, x))
        return t

    def progress(self, wait=True):
        for t in list(self.slots):
            self.slots[t][0] -= 1
            if self.slots[t][0] == 0:
                _, b, x = self.slots.pop(t)
                x[:] = 2 * b
                self.done[t] = {"iters": self.steps}
        while self.queue and len(self.slots) < self.k:
            t, b, x = self.queue.pop(0)
            self.slots[t] = [self.steps, b, x]
            self.admitted.append(t)
        self.max_busy = max(self.max_busy, len(self.slots))
        return len(self.slots) + len(self.queue)

    def poll(self, t):
        if t in self.done:
            return True, self.done.pop(t), 0
        return False, None, 0


def test_poisson_trace_statistics_and_determinism():
    mk = lambda name, i: np.full(4, i, dtype=np.complex128)
    tr = poisson_trace(4000, rate_hz=50.0, mix={"a": 3, "b": 1}, seed=11, make_source=mk)
    t = np.array([r.t_arrival for r in tr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0          # exponential mean 1/rate
    assert abs(gaps.std() - 1 / 50.0) < 0.1 / 50.0           # and std 1/rate
    frac_a = np.mean([r.op == "a" for r in tr])
    assert abs(frac_a - 0.75) < 0.03
    # per-operator source index counts up
    ia = [int(r.b[0].real) for r in tr if r.op == "a"]
    assert ia == list(range(len(ia)))
    tr2 = poisson_trace(4000, rate_hz=50.0, mix={"a": 3, "b": 1}, seed=11, make_source=mk)
    assert [r.t_arrival for r in tr2] == list(t) and [r.op for r in tr2] == [r.op for r in tr]


def test_server_completes_everything_in_order_of_admission():
    mk = lambda name, i: np.arange(3, dtype=np.complex128) + i
    tr = poisson_trace(25, rate_hz=1e6, mix={"a": 1, "b": 1}, seed=2, make_source=mk)
    fa, fb = FakeSolver(k=3, steps=4), FakeSolver(k=2, steps=2)
    rep, reqs = Server({"a": fa, "b": fb}).run(tr, realtime=False)
    s = rep.summary()
    assert s["requests"] == 25 and s["failed"] == 0
    assert len(rep.latencies) == 25 and min(rep.latencies) >= 0
    assert s["latency_p50_s"] <= s["latency_p99_s"]
    for r in reqs:
        assert np.array_equal(r.x, 2 * r.b)
        assert r.info == {"iters": 4 if r.op == "a" else 2}
    # FIFO admission per operator and slot limits respected
    assert fa.admitted == sorted(fa.admitted) and fb.admitted == sorted(fb.admitted)
    assert fa.max_busy == 3 and fb.max_busy == 2


def test_report_summary_percentiles():
    rep = ServeReport(latencies=list(np.linspace(0.0, 1.0, 101)), makespan=2.0, completed=101)
    s = rep.summary()
    assert abs(s["latency_p50_s"] - 0.5) < 1e-12 and abs(s["latency_p99_s"] - 0.99) < 1e-12
    assert abs(s["rhs_per_s"] - 50.5) < 1e-12
    assert isinstance(Request(0, "a", np.zeros(1), 0.0).ticket, int)
