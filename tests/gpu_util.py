"""Shared helpers for the GPU parity tests (seeded inputs, oracle operators)."""
import numpy as np

from oracle.wilson import WilsonOperator
from seeded_inputs import WORKLOADS, gauge_links, workload_links


def workload(name):
    w = WORKLOADS[name]
    links = workload_links(name)
    return w, links, WilsonOperator(links, w["kappa"], w["dims"])


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def true_resid(op, b, x):
    return float(np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b))


def random_field(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2)


def small_problem(dims, eps=0.5, seed=1, kappa=0.12):
    links = gauge_links(dims, eps, seed)
    return links, WilsonOperator(links, kappa, dims)
