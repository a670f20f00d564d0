"""Request loop serving Wilson-Dirac solves on one GPU (continuous batching).

Host-side scheduling only: every solve runs in ``liblqcd.so`` through the
session calls of the C ABI (``lqcd_submit`` / ``lqcd_progress`` /
``lqcd_poll``). One :class:`~paper_0911_2285_gb300.lqcd.Solver` per gauge
field keeps its links and its growing eigenspace resident on the device; the
first requests of each field run eigBiCG and feed the eigenspace, later ones
run deflated BiCG (Algorithm Incremental eigBiCG). Each context has a fixed
number of batch slots; an eigBiCG request also needs a window, which the
library allocates only when the device-memory plan has room (admission by
memory). Requests that arrive while the slots (or the memory) are taken wait
in the context's queue and are admitted as they free up, while the other slots
keep iterating, so the work of different requests overlaps inside the same
operator launches, and contexts on different gauge fields run on their own
CUDA streams.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from .lqcd import Solver

POLL_S = 20e-6   # default host pause between non-blocking polls when nothing finished


@dataclass
class Request:
    rid: int
    op: str                 # name of the gauge field / operator
    b: np.ndarray           # source (host)
    t_arrival: float        # seconds after the start of the trace
    x: np.ndarray | None = None
    ticket: int = -1
    t_submit: float = 0.0
    t_done: float = 0.0
    info: dict | None = None
    status: int = -1


@dataclass
class ServeReport:
    latencies: list = field(default_factory=list)
    makespan: float = 0.0
    completed: int = 0
    failed: int = 0

    def summary(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {
            "requests": self.completed,
            "failed": self.failed,
            "rhs_per_s": self.completed / self.makespan if self.makespan > 0 else 0.0,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_mean_s": float(lat.mean()),
            "makespan_s": self.makespan,
        }


def poisson_trace(n_requests, rate_hz, mix, seed, make_source):
    """Poisson arrivals at ``rate_hz``; operator chosen from ``mix`` ({name: weight}).

    ``make_source(op_name, index)`` returns the host source of the i-th request of an operator.
    """
    rng = np.random.default_rng(seed)
    names = list(mix)
    w = np.array([mix[k] for k in names], dtype=np.float64)
    w /= w.sum()
    t = 0.0
    counts = {k: 0 for k in names}
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        op = names[int(rng.choice(len(names), p=w))]
        out.append(Request(rid, op, make_source(op, counts[op]), t))
        counts[op] += 1
    return out


class Server:
    """Continuous-batching request loop over several resident operators."""

    def __init__(self, operators: dict[str, Solver], poll_s: float = POLL_S):
        """``poll_s``: seconds to yield the host core between non-blocking polls that
        found nothing finished (0 = spin)."""
        self.ops = operators
        self.poll_s = poll_s

    def run(self, requests, realtime=True, mode="auto"):
        """Serve ``requests`` (sorted by arrival). With ``realtime`` the arrivals
        follow the trace clock; otherwise everything arrives at once."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        rep = ServeReport()
        pending = {name: {} for name in self.ops}   # ticket -> request
        t0 = time.perf_counter()
        i = 0
        active = {name: 0 for name in self.ops}
        while i < len(reqs) or any(active.values()) or any(pending.values()):
            now = time.perf_counter() - t0
            # admit every request that has arrived
            while i < len(reqs) and (not realtime or reqs[i].t_arrival <= now):
                r = reqs[i]
                r.x = np.zeros_like(r.b)
                r.t_submit = time.perf_counter() - t0
                if not realtime:
                    r.t_arrival = r.t_submit
                r.ticket = self.ops[r.op].submit(r.b, r.x, mode=mode)
                pending[r.op][r.ticket] = r
                i += 1
            # advance every operator that has work (each on its own stream); block on
            # one only when nothing else can happen meanwhile
            busy = [n for n in self.ops if pending[n] or active[n]]
            wait = len(busy) == 1 and (not realtime or i == len(reqs))
            finished = 0
            for name in busy:
                solver = self.ops[name]
                active[name] = solver.progress(wait=wait)
                for ticket in list(pending[name]):
                    done, info, status = solver.poll(ticket)
                    if done:
                        finished += 1
                        r = pending[name].pop(ticket)
                        r.t_done = time.perf_counter() - t0
                        r.info, r.status = info, status
                        rep.latencies.append(r.t_done - r.t_arrival)
                        if status == 0:
                            rep.completed += 1
                        else:
                            rep.failed += 1
            if realtime and i < len(reqs) and not any(active.values()) and not any(pending.values()):
                wait_s = reqs[i].t_arrival - (time.perf_counter() - t0)
                if wait_s > 0:
                    time.sleep(wait_s)
            elif not wait and busy and not finished and self.poll_s > 0:
                time.sleep(self.poll_s)   # nothing finished: yield the core briefly instead of spinning
        rep.makespan = time.perf_counter() - t0
        return rep, reqs
