"""BiCG, Algorithm eigBiCG and Algorithm BiCG-eigen, FP64, numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2 of the paper step by step, in its notation, on vectors of
length ``N``; ``op`` supplies ``apply`` (``A v``) and ``apply_dag``
(``A^dagger v``). Inner products are ``(w, v) = w^H v``.

Readings where the printed algorithm is garbled or silent (also used by the
GPU library):

* index typos in Algorithm eigBiCG are read as ``x_j = x_{j-1} + alpha_{j-1} p_{j-1}``,
  ``rhat_j = rhat_{j-1} - conj(alpha_{j-1}) A^H phat_{j-1}``, ``beta_{j-2}/alpha_{j-2}``
  in the diagonal of H, and ``Q = W^(vs) z^(nev)`` for the final Ritz vectors;
* the shadow residual is ``rhat_0 = r_0`` (Sec. 2: normally ``bhat = b``, ``xhat_0 = x_0``);
* the stored products ``q = A p``, ``s = A^H phat`` are taken in the iteration
  where ``vs = m-1`` before ``vs`` is incremented, so at the restart one
  iteration later they are ``A p_{j-2}`` and ``A^H phat_{j-2}``;
* the restart coupling ``H_{2nev+1,k} = (||r_{j-1}||/rho_{j-1}) (A^H phat - conj(beta) s)^H v_k``
  keeps the scalar unconjugated, as printed;
* after the restart the window holds as many vectors as survive the
  biorthogonalization (``2 nev`` unless pairs are dropped as dependent);
* breakdown: ``|rho| < 1e-14 ||rhat|| ||r||`` or ``|sigma| < 1e-14 ||phat|| ||A p||``;
* convergence: the recursive ``||r_j|| <= tol ||b||`` of the algorithm, then
  confirmed with the true residual ``||b - A x||``; if the confirmation fails the
  recursive residual is replaced by the true one (``rho`` recomputed) and the
  iteration continues.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .smalleig import biorthogonalize, eig_lr

BREAKDOWN_TOL = 1e-14


class Breakdown(RuntimeError):
    pass


class NoConvergence(RuntimeError):
    pass


def _dot(w, v):
    return np.vdot(w, v)


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    matvecs: int
    true_resid: float
    resnorms: list = field(default_factory=list)
    # eigBiCG only
    evals: np.ndarray | None = None
    U: np.ndarray | None = None          # right Ritz vectors (N x nev)
    Q: np.ndarray | None = None          # left Ritz vectors (N x nev)
    restarts: int = 0
    vs: int = 0
    H: np.ndarray | None = None          # final projection matrix H^(vs)
    V: np.ndarray | None = None          # final window (N x vs)
    W: np.ndarray | None = None
    first_window: tuple | None = None    # (V, W, H) when vs first reaches m
    snapshots: list = field(default_factory=list)


def bicg(op, b, x0=None, tol=1e-10, maxiter=10000, rhat0=None, history=False, callback=None):
    """Plain BiCG (the iteration of Algorithm eigBiCG without the window).

    ``callback(j, x, r, rhat)`` (optional) sees every iterate; ``history``
    keeps the ``(alpha, beta)`` pairs in ``SolveResult.snapshots``.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    mv0 = op.matvecs
    r = b - op.apply(x)
    rhat = r.copy() if rhat0 is None else np.array(rhat0, dtype=np.complex128)
    p = r.copy()
    phat = rhat.copy()
    rho = _dot(rhat, r)
    bnorm = np.linalg.norm(b)
    rnorm = np.linalg.norm(r)
    hist = [rnorm]
    scal = []
    j = 0
    if rnorm <= tol * bnorm:
        return SolveResult(x, 0, op.matvecs - mv0, rnorm / bnorm, hist)
    while j < maxiter:
        j += 1
        if abs(rho) < BREAKDOWN_TOL * np.linalg.norm(rhat) * rnorm:
            raise Breakdown(f"rho breakdown at iteration {j}")
        ap = op.apply(p)
        ahp = op.apply_dag(phat)
        sigma = _dot(phat, ap)
        if abs(sigma) < BREAKDOWN_TOL * np.linalg.norm(phat) * np.linalg.norm(ap):
            raise Breakdown(f"sigma breakdown at iteration {j}")
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * ap
        rhat = rhat - np.conj(alpha) * ahp
        rho_new = _dot(rhat, r)
        beta = rho_new / rho
        p = r + beta * p
        phat = rhat + np.conj(beta) * phat
        rho = rho_new
        rnorm = np.linalg.norm(r)
        hist.append(rnorm)
        if history:
            scal.append((alpha, beta))
        if callback is not None:
            callback(j, x, r, rhat)
        if rnorm <= tol * bnorm:
            true_r = b - op.apply(x)
            tn = np.linalg.norm(true_r)
            if tn <= tol * bnorm:
                res = SolveResult(x, j, op.matvecs - mv0, tn / bnorm, hist)
                if history:
                    res.snapshots = scal
                return res
            r = true_r
            rho = _dot(rhat, r)
            rnorm = tn
    raise NoConvergence(f"BiCG: no convergence in {maxiter} iterations")


def restart_coefficients(H, nev):
    """Coefficient-space part of Algorithm BiCG-eigen.

    Given ``H = H^(m)`` (m x m), returns ``(Yc, Zc, lam)`` such that the
    restarted window is ``V <- V Yc``, ``W <- W Zc`` and ``H <- diag(lam)``:

    1. ``[y, z, E] = eig(H^(m))`` and ``eig(H^(m-1))`` (leading principal
       submatrix), nev smallest of each; pad the latter with a zero row;
    2. bi-orthogonalize the ``2 nev`` right vectors against the left ones;
    3. ``T = zt^H H yt``, ``[u, q, lam] = eig(T)``;
    4. ``Yc = yt u``, ``Zc = zt q``.
    """
    m = H.shape[0]
    y_m, z_m, _ = eig_lr(H)
    y_m1, z_m1, _ = eig_lr(H[: m - 1, : m - 1])
    k1 = min(nev, m)
    k2 = min(nev, m - 1)
    y1, z1 = y_m[:, :k1], z_m[:, :k1]
    y2 = np.vstack([y_m1[:, :k2], np.zeros((1, k2), dtype=np.complex128)])
    z2 = np.vstack([z_m1[:, :k2], np.zeros((1, k2), dtype=np.complex128)])
    yt, zt = biorthogonalize(y1, z1, y2, z2)
    t = np.conj(zt.T) @ H @ yt
    u, q, lam = eig_lr(t)
    return yt @ u, zt @ q, lam


def eigbicg(op, b, nev, m, x0=None, tol=1e-10, maxiter=10000, snapshot_every=0, rhat0=None):
    """Algorithm eigBiCG(nev, m): BiCG plus a window of m residuals.

    Returns a :class:`SolveResult` carrying x, the final nev Ritz values and
    right/left Ritz vectors, and the final window (for identity checks).
    ``snapshot_every > 0`` stores ``(V, W, H)`` copies of the active window at
    the end of every ``snapshot_every``-th iteration. ``rhat0`` replaces the
    shadow start ``r_0`` (Sec. 4: ``gamma5 r_0`` for gamma5-Hermitian A).
    """
    if m <= 2 * nev:
        raise ValueError("eigBiCG needs m > 2 nev")
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    mv0 = op.matvecs
    # Steps 1-2: initial residuals, directions, rho_0, vs = 0.
    r = b - op.apply(x)
    rhat = r.copy() if rhat0 is None else np.array(rhat0, dtype=np.complex128)
    p = r.copy()
    phat = rhat.copy()
    rho = _dot(rhat, r)
    vs = 0
    V = np.zeros((n, m), dtype=np.complex128)
    W = np.zeros((n, m), dtype=np.complex128)
    H = np.zeros((m, m), dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    rnorm = np.linalg.norm(r)
    hist = [rnorm]
    res = SolveResult(x, 0, 0, rnorm / bnorm, hist)
    alpha_prev = beta_prev = None
    q = s = None
    restarts = 0
    j = 0
    converged = rnorm <= tol * bnorm
    while not converged:
        if j >= maxiter:
            raise NoConvergence(f"eigBiCG: no convergence in {maxiter} iterations")
        j += 1
        if abs(rho) < BREAKDOWN_TOL * np.linalg.norm(rhat) * rnorm:
            raise Breakdown(f"rho breakdown at iteration {j}")
        # Step 3a: A p_{j-1}, A^H phat_{j-1}, sigma, alpha, x update.
        ap = op.apply(p)
        ahp = op.apply_dag(phat)
        sigma = _dot(phat, ap)
        if abs(sigma) < BREAKDOWN_TOL * np.linalg.norm(phat) * np.linalg.norm(ap):
            raise Breakdown(f"sigma breakdown at iteration {j}")
        alpha = rho / sigma
        x = x + alpha * p
        # Step 3b: keep A p and A^H phat one iteration before the window fills.
        if vs == m - 1:
            q = ap.copy()
            s = ahp.copy()
        # Step 3c: restart with BiCG-eigen, then the coupling row/column.
        if vs == m:
            if res.first_window is None and restarts == 0:
                res.first_window = (V.copy(), W.copy(), H.copy())
            yc, zc, lam = restart_coefficients(H, nev)
            kk = len(lam)
            V_new = V @ yc
            W_new = W @ zc
            V[:] = 0
            W[:] = 0
            V[:, :kk] = V_new
            W[:, :kk] = W_new
            H[:] = 0
            H[np.arange(kk), np.arange(kk)] = lam
            vs = kk
            restarts += 1
            a_vec = ap - beta_prev * q                 # = ||r_{j-1}|| A v_{kk+1}
            c_vec = ahp - np.conj(beta_prev) * s       # = A^H rhat_{j-1}
            for k in range(kk):
                H[kk, k] = (rnorm / rho) * _dot(c_vec, V[:, k])
                H[k, kk] = (1.0 / rnorm) * _dot(W[:, k], a_vec)
        # Step 3d: append v_vs, w_vs.
        vs += 1
        V[:, vs - 1] = r / rnorm
        W[:, vs - 1] = (rnorm / np.conj(rho)) * rhat
        # Step 3e-g: residual update, rho_j, beta_{j-1}, directions.
        r_new = r - alpha * ap
        rhat_new = rhat - np.conj(alpha) * ahp
        rho_new = _dot(rhat_new, r_new)
        beta = rho_new / rho
        p = r_new + beta * p
        phat = rhat_new + np.conj(beta) * phat
        rnorm_new = np.linalg.norm(r_new)
        # Step 3h-i: tridiagonal entries of H.
        if j == 1:
            H[vs - 1, vs - 1] = 1.0 / alpha
        else:
            H[vs - 1, vs - 1] = 1.0 / alpha + beta_prev / alpha_prev
        if vs < m:
            H[vs - 1, vs] = -(rnorm / rnorm_new) * beta / alpha
            H[vs, vs - 1] = -(rnorm_new / rnorm) / alpha
        alpha_prev, beta_prev = alpha, beta
        r, rhat, rho, rnorm = r_new, rhat_new, rho_new, rnorm_new
        hist.append(rnorm)
        if snapshot_every and j % snapshot_every == 0:
            res.snapshots.append((V[:, :vs].copy(), W[:, :vs].copy(), H[:vs, :vs].copy()))
        # Step 3j: convergence, confirmed with the true residual.
        if rnorm <= tol * bnorm:
            true_r = b - op.apply(x)
            tn = np.linalg.norm(true_r)
            if tn <= tol * bnorm:
                converged = True
                rnorm_true = tn
            else:
                r = true_r
                rho = _dot(rhat, r)
                rnorm = tn
    # Step 4: final nev Ritz pairs from H^(vs).
    res.x = x
    res.iters = j
    res.matvecs = op.matvecs - mv0
    res.true_resid = (rnorm_true if j else rnorm) / bnorm
    res.restarts = restarts
    res.vs = vs
    res.H = H[:vs, :vs].copy()
    res.V = V[:, :vs].copy()
    res.W = W[:, :vs].copy()
    if vs > 0:
        y, z, lam = eig_lr(H[:vs, :vs])
        k = min(nev, vs)
        res.evals = lam[:k]
        res.U = V[:, :vs] @ y[:, :k]
        res.Q = W[:, :vs] @ z[:, :k]
    else:
        res.evals = np.zeros(0, dtype=np.complex128)
        res.U = np.zeros((n, 0), dtype=np.complex128)
        res.Q = np.zeros((n, 0), dtype=np.complex128)
    return res


def bicg_g5(op, b, x0=None, tol=1e-10, maxiter=10000, history=False):
    """BiCG for gamma5-Hermitian A (Sec. 4): with the shadow start
    ``rhat_0 = gamma5 r_0`` the shadow sequences are ``rhat_j = gamma5 r_j`` and
    ``phat_j = gamma5 p_j``, so ``A^H phat = gamma5 (A p)``: one product with A
    per iteration, no shadow vectors. ``rho = r^H gamma5 r`` and
    ``sigma = p^H gamma5 A p`` are real (gamma5 A is Hermitian), hence real
    alpha and beta. ``op`` supplies ``apply`` and ``gamma5``.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    mv0 = op.matvecs
    r = b - op.apply(x)
    p = r.copy()
    rho = float(np.real(_dot(op.gamma5(r), r)))
    bnorm = np.linalg.norm(b)
    rnorm = np.linalg.norm(r)
    hist = [rnorm]
    scal = []
    if rnorm <= tol * bnorm:
        return SolveResult(x, 0, op.matvecs - mv0, rnorm / bnorm, hist)
    j = 0
    while j < maxiter:
        j += 1
        if abs(rho) < BREAKDOWN_TOL * rnorm * rnorm:
            raise Breakdown(f"rho breakdown at iteration {j}")
        ap = op.apply(p)
        g5ap = op.gamma5(ap)            # = A^H phat with phat = gamma5 p
        sigma = float(np.real(_dot(p, g5ap)))
        if abs(sigma) < BREAKDOWN_TOL * np.linalg.norm(p) * np.linalg.norm(ap):
            raise Breakdown(f"sigma breakdown at iteration {j}")
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * ap
        rho_new = float(np.real(_dot(op.gamma5(r), r)))
        beta = rho_new / rho
        p = r + beta * p
        rho = rho_new
        rnorm = np.linalg.norm(r)
        hist.append(rnorm)
        if history:
            scal.append((alpha, beta))
        if rnorm <= tol * bnorm:
            true_r = b - op.apply(x)
            tn = np.linalg.norm(true_r)
            if tn <= tol * bnorm:
                res = SolveResult(x, j, op.matvecs - mv0, tn / bnorm, hist)
                if history:
                    res.snapshots = scal
                return res
            r = true_r
            rho = float(np.real(_dot(op.gamma5(r), r)))
            rnorm = tn
    raise NoConvergence(f"gamma5 BiCG: no convergence in {maxiter} iterations")


def bicgstab(op, b, x0=None, tol=1e-10, maxiter=10000, callback=None):
    """BiCGStab (van der Vorst 1992), the paper's phase-2 solver (Sec. 2), with
    the shadow start ``rhat = r_0``: each step is a BiCG step followed by a
    one-dimensional minimal-residual step, two products with A and none with
    A^H. Convergence on the recursive residual is confirmed with the true one
    (replaced and continued if it fails, as for BiCG above).
    ``callback(j, x, r, t)`` sees every iterate and ``t = A s`` of the step
    (the minimal-residual step makes the new ``r`` orthogonal to ``t``).
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    mv0 = op.matvecs
    r = b - op.apply(x)
    rhat = r.copy()
    bnorm = np.linalg.norm(b)
    rnorm = np.linalg.norm(r)
    hist = [rnorm]
    if rnorm <= tol * bnorm:
        return SolveResult(x, 0, op.matvecs - mv0, rnorm / bnorm, hist)
    rho_old = alpha = omega = 1.0 + 0j
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    j = 0
    while j < maxiter:
        j += 1
        rho = _dot(rhat, r)
        if abs(rho) < BREAKDOWN_TOL * np.linalg.norm(rhat) * rnorm:
            raise Breakdown(f"rho breakdown at iteration {j}")
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = op.apply(p)
        den = _dot(rhat, v)
        if abs(den) < BREAKDOWN_TOL * np.linalg.norm(rhat) * np.linalg.norm(v):
            raise Breakdown(f"(rhat, A p) breakdown at iteration {j}")
        alpha = rho / den
        s = r - alpha * v
        t = op.apply(s)
        tt = _dot(t, t).real
        omega = _dot(t, s) / tt if tt > 0 else 0.0 + 0j
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        rnorm = np.linalg.norm(r)
        hist.append(rnorm)
        if callback is not None:
            callback(j, x, r, t)
        if rnorm <= tol * bnorm:
            true_r = b - op.apply(x)
            tn = np.linalg.norm(true_r)
            if tn <= tol * bnorm:
                return SolveResult(x, j, op.matvecs - mv0, tn / bnorm, hist)
            r = true_r
            rnorm = tn
        if omega == 0:
            raise Breakdown(f"omega breakdown at iteration {j}")
    raise NoConvergence(f"BiCGStab: no convergence in {maxiter} iterations")
