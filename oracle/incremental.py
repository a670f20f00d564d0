"""Algorithm Incremental eigBiCG, oblique deflation and Rayleigh-Ritz (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2 of the paper, Algorithm Incremental eigBiCG:

1. start with empty ``U_l, U_r, H``;
2. for the first ``n1`` right-hand sides: deflate the initial guess
   (``x0 <- x0 + U_r d`` with ``H d = U_l^H (b - A x0)``), solve with eigBiCG,
   bi-orthogonalize the new Ritz vectors against ``[U_r, U_l]``, grow ``H`` by
   the block formula and append the vectors;
3. for the remaining right-hand sides: deflate the initial guess and solve.
   The paper's phase-2 solver is BiCGStab; the library solves phase 2 with
   BiCG (same iteration as eigBiCG without the window), and so does this
   oracle. ``DefTol`` re-deflation (restart when ``||r|| < DefTol ||b||``) is
   supported; ``DefTol = 0`` (the paper's Fig. 1 setting) never restarts.

Readings:

* "bi-orthogonalize [V, W] against [U_r, U_l]" is the oblique projection
  ``V' = V - U_r (U_l^H U_r)^{-1} U_l^H V``, ``W' = W - U_l (U_r^H U_l)^{-1} U_r^H W``;
  every new column is then scaled to unit 2-norm, and a pair is dropped when
  either projected column keeps less than ``1e-8`` of its norm;
* ``H`` is ``U_l^H A U_r``; its new blocks ``U_l^H A V'``, ``W'^H A U_r`` and
  ``W'^H A V'`` cost ``2 nev`` extra products (``A V'`` and ``A^H W'``);
* the small systems with ``H`` are solved by LU with partial pivoting.
* Rayleigh-Ritz on the accumulated spaces: the pencil ``(U_l^H A U_r, U_l^H U_r)``;
  its eigenvalues, right vectors ``U_r y`` and left vectors ``U_l z``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .bicg import bicg, bicgstab, eigbicg
from .smalleig import order_smallest

DROP_TOL = 1e-8


@dataclass
class Eigenspace:
    n: int
    Ur: np.ndarray = None
    Ul: np.ndarray = None
    H: np.ndarray = None

    def __post_init__(self):
        if self.Ur is None:
            self.Ur = np.zeros((self.n, 0), dtype=np.complex128)
            self.Ul = np.zeros((self.n, 0), dtype=np.complex128)
            self.H = np.zeros((0, 0), dtype=np.complex128)

    @property
    def size(self):
        return self.Ur.shape[1]


def deflate(op, space: Eigenspace, b, x0):
    """``x0 + U_r d`` with ``H d = U_l^H (b - A x0)`` (Incremental eigBiCG, steps 2-3)."""
    x0 = np.asarray(x0, dtype=np.complex128)
    if space.size == 0:
        return x0.copy()
    r = b - op.apply(x0)
    c = np.conj(space.Ul.T) @ r
    d = sla.lu_solve(sla.lu_factor(space.H), c)
    return x0 + space.Ur @ d


def grow(op, space: Eigenspace, Vn, Wn, drop_tol=DROP_TOL):
    """Add new right/left vectors to the eigenspace (Incremental eigBiCG, step 2)."""
    Vn = np.asarray(Vn, dtype=np.complex128)
    Wn = np.asarray(Wn, dtype=np.complex128)
    if space.size:
        Ur, Ul = space.Ur, space.Ul
        M = np.conj(Ul.T) @ Ur
        Vp = Vn - Ur @ sla.solve(M, np.conj(Ul.T) @ Vn)
        Wp = Wn - Ul @ sla.solve(np.conj(M.T), np.conj(Ur.T) @ Wn)
    else:
        Vp, Wp = Vn.copy(), Wn.copy()
    keep = []
    for i in range(Vp.shape[1]):
        nv0, nw0 = np.linalg.norm(Vn[:, i]), np.linalg.norm(Wn[:, i])
        nv, nw = np.linalg.norm(Vp[:, i]), np.linalg.norm(Wp[:, i])
        if nv > drop_tol * nv0 and nw > drop_tol * nw0:
            Vp[:, i] /= nv
            Wp[:, i] /= nw
            keep.append(i)
    Vp = Vp[:, keep]
    Wp = Wp[:, keep]
    if not keep:
        return space
    AVp = np.stack([op.apply(Vp[:, i]) for i in range(Vp.shape[1])], axis=1)
    AhWp = np.stack([op.apply_dag(Wp[:, i]) for i in range(Wp.shape[1])], axis=1)
    top_right = np.conj(space.Ul.T) @ AVp           # U_l^H A V'
    bottom_left = np.conj(AhWp.T) @ space.Ur         # W'^H A U_r = (A^H W')^H U_r
    bottom_right = np.conj(Wp.T) @ AVp               # W'^H A V'
    H = np.block([[space.H, top_right], [bottom_left, bottom_right]])
    return Eigenspace(space.n, np.hstack([space.Ur, Vp]), np.hstack([space.Ul, Wp]), H)


@dataclass
class IncrementalResult:
    x: list = field(default_factory=list)
    iters: list = field(default_factory=list)
    matvecs: list = field(default_factory=list)
    true_resid: list = field(default_factory=list)
    modes: list = field(default_factory=list)
    space: Eigenspace | None = None
    ritz: list = field(default_factory=list)


def _shadow(op, b, x, gamma5):
    """Shadow start of a BiCG run from x: ``r_0`` (general) or ``gamma5 r_0`` (Sec. 4)."""
    return op.gamma5(b - op.apply(x)) if gamma5 else None


def deflated_bicg(op, space, b, x0=None, tol=1e-10, deftol=0.0, maxiter=10000, gamma5=False):
    """Phase-2 solve: deflate the initial guess and run BiCG.

    With ``tol < deftol`` the solve stops once at ``deftol ||b||``, re-deflates
    the current iterate and restarts BiCG to ``tol`` (the paper's DefTol
    restart read as one restart at the ``DefTol`` crossing). ``gamma5``: the
    shadow start of each BiCG run is ``gamma5 r_0`` (Sec. 4).
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    x = deflate(op, space, b, x)
    iters = 0
    mv = 0
    if deftol > tol:
        res = bicg(op, b, x, tol=deftol, maxiter=maxiter, rhat0=_shadow(op, b, x, gamma5))
        iters += res.iters
        mv += res.matvecs
        x = deflate(op, space, b, res.x)
    res = bicg(op, b, x, tol=tol, maxiter=maxiter - iters, rhat0=_shadow(op, b, x, gamma5))
    return res.x, iters + res.iters, mv + res.matvecs, res.true_resid


def deflated_bicgstab(op, space, b, x0=None, tol=1e-10, deftol=0.0, maxiter=10000):
    """Phase 2 as the paper runs it (Sec. 2): deflate the initial guess, solve
    with BiCGStab; with ``deftol > tol`` stop at ``deftol``, deflate the current
    iterate again and continue to ``tol`` (one restart)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    x = deflate(op, space, b, x)
    outer = 0
    iters = 0
    if deftol > tol and space.size > 0:
        first = bicgstab(op, b, x, tol=deftol, maxiter=maxiter)
        iters += first.iters
        x = deflate(op, space, b, first.x)
        outer = 1
    res = bicgstab(op, b, x, tol=tol, maxiter=maxiter)
    res.iters += iters
    res.restarts = outer
    return res


def incremental_eigbicg(op, sources, nev, m, n1, tol=1e-10, deftol=0.0, maxiter=10000,
                        x0s=None, gamma5=False):
    """Algorithm Incremental eigBiCG over a list of right-hand sides (sequential).
    ``gamma5``: every BiCG run starts its shadow sequence at ``gamma5 r_0`` (the
    gamma5-Hermitian variant of Sec. 4)."""
    space = Eigenspace(op.n)
    out = IncrementalResult()
    for k, b in enumerate(sources):
        b = np.asarray(b, dtype=np.complex128)
        x0 = np.zeros_like(b) if x0s is None else np.asarray(x0s[k], dtype=np.complex128)
        mv0 = op.matvecs
        if k < n1:
            x0 = deflate(op, space, b, x0)
            res = eigbicg(op, b, nev, m, x0=x0, tol=tol, maxiter=maxiter, rhat0=_shadow(op, b, x0, gamma5))
            space = grow(op, space, res.U, res.Q)
            out.x.append(res.x)
            out.iters.append(res.iters)
            out.true_resid.append(res.true_resid)
            out.modes.append("eigbicg")
            out.ritz.append(res.evals)
        else:
            x, it, _, tr = deflated_bicg(op, space, b, x0, tol=tol, deftol=deftol, maxiter=maxiter, gamma5=gamma5)
            out.x.append(x)
            out.iters.append(it)
            out.true_resid.append(tr)
            out.modes.append("deflated")
        out.matvecs.append(op.matvecs - mv0)
    out.space = space
    return out


def rayleigh_ritz(op, space: Eigenspace, nmax=None):
    """Final eigenpairs from Rayleigh-Ritz with ``U_l``, ``U_r`` as search spaces.

    Solves ``(U_l^H A U_r) y = lam (U_l^H U_r) y`` and ``z^H (U_l^H A U_r) = lam z^H (U_l^H U_r)``;
    returns ``lam`` (smallest |lam| first), ``U_r y``, ``U_l z`` and the
    residuals ``||A u - lam u|| / ||u||``.
    """
    Ur, Ul = space.Ur, space.Ul
    M = np.conj(Ul.T) @ Ur
    lam, zl, zr = sla.eig(space.H, M, left=True, right=True)
    order = order_smallest(lam)
    if nmax is not None:
        order = order[:nmax]
    lam = lam[order]
    u = Ur @ zr[:, order]
    w = Ul @ zl[:, order]
    res = []
    for i in range(len(lam)):
        ui = u[:, i]
        res.append(np.linalg.norm(op.apply(ui) - lam[i] * ui) / np.linalg.norm(ui))
    return lam, u, w, np.array(res)
