"""Pins of the BiCGStab oracle (the paper's phase-2 solver, Sec. 2) and of
deflated BiCGStab: the exact solution of dense systems, finite termination on
a matrix with few distinct eigenvalues, the recursive residual tracking the
true one, two products with A per step on the Wilson operator, and zero
iterations after deflation with a complete eigenspace."""
import numpy as np
import scipy.linalg as sla

from oracle.bicg import bicgstab
from oracle.incremental import Eigenspace, deflated_bicgstab
from oracle.wilson import DenseOperator, WilsonOperator
from seeded_inputs import WORKLOADS, gaussian_source, workload_links


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))


def test_dense_solution():
    n = 40
    a = 4 * np.eye(n) + _rand(n, 1) / np.sqrt(n)
    b = np.random.default_rng(2).standard_normal(n) + 0j
    res = bicgstab(DenseOperator(a), b, tol=1e-12)
    ref = np.linalg.solve(a, b)
    assert np.linalg.norm(res.x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_finite_termination_few_distinct_eigenvalues():
    n, lam = 40, np.array([1.0, 2.0 + 1j, 3.0, 0.5 - 0.5j, 5.0])
    s = _rand(n, 3) + 6 * np.eye(n)
    a = s @ np.diag(np.resize(lam, n)) @ np.linalg.inv(s)
    b = np.random.default_rng(4).standard_normal(n) + 0j
    res = bicgstab(DenseOperator(a), b, tol=1e-10)
    assert res.iters <= len(lam) + 1
    assert np.linalg.norm(b - a @ res.x) <= 1e-10 * np.linalg.norm(b)


def test_recursive_residual_tracks_true_residual():
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    b = gaussian_source(w["dims"], 3)
    gaps, orth = [], []

    def cb(j, x, r, t):
        gaps.append(np.linalg.norm(b - op.apply(x) - r))
        orth.append(abs(np.vdot(t, r)) / (np.linalg.norm(t) * np.linalg.norm(r)))

    bicgstab(op, b, tol=1e-10, callback=cb)
    assert max(gaps) <= 1e-9 * np.linalg.norm(b)
    # the minimal-residual step leaves the residual orthogonal to t = A s
    assert max(orth) <= 1e-10


def test_wilson_two_products_per_step():
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    b = gaussian_source(w["dims"], 5)
    mv0 = op.matvecs
    res = bicgstab(op, b, tol=1e-10)
    assert res.true_resid <= 1e-10
    assert 2 * res.iters + 1 <= op.matvecs - mv0 <= 2 * res.iters + 3


def test_deflation_with_complete_eigenspace_needs_no_iteration():
    n = 30
    a = 3 * np.eye(n) + _rand(n, 6) / np.sqrt(n)
    lam, vl, vr = sla.eig(a, left=True, right=True)
    space = Eigenspace(n, Ur=vr, Ul=vl, H=np.conj(vl.T) @ a @ vr)
    b = np.random.default_rng(7).standard_normal(n) + 1j
    res = deflated_bicgstab(DenseOperator(a), space, b, tol=1e-10)
    assert res.iters == 0
    assert np.linalg.norm(b - a @ res.x) <= 1e-10 * np.linalg.norm(b)
