"""Small dense eigenproblems of the projected matrices (FP64, LAPACK via scipy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's notation (Sec. 1): ``[zr, zl, D] = eig(C)`` returns right
eigenvectors ``zr``, left eigenvectors ``zl`` and eigenvalues ``D`` sorted by a
user criterion; eigBiCG uses "smallest absolute value" (Sec. 2). The paper
fixes neither the order of ties nor the scaling of the vectors; the readings
used here (and by the GPU library) are:

* order: ascending ``|lambda|``, exact ties broken by ascending ``Im(lambda)``;
* right vectors ``y`` have unit 2-norm, with the phase fixed so that the
  entry of largest modulus (first such index) is real and positive;
* left vectors are scaled so that ``z^H y = 1`` (the paper's biorthogonality
  ``(w_j, v_j) = 1`` carried over to the coefficient space).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def order_smallest(lam):
    """Indices of ``lam`` in the paper's order (smallest |lambda| first, then Im)."""
    lam = np.asarray(lam)
    return np.array(sorted(range(len(lam)), key=lambda i: (abs(lam[i]), lam[i].imag)),
                    dtype=np.int64)


def normalise_pair(y, z):
    """Apply the vector conventions to one right/left pair."""
    y = y / np.linalg.norm(y)
    k = int(np.argmax(np.abs(y)))
    y = y * (np.conj(y[k]) / abs(y[k]))
    d = np.vdot(z, y)          # z^H y
    z = z / np.conj(d)
    return y, z


def eig_lr(c):
    """``[y, z, lam] = eig(C)`` with right and left vectors, sorted smallest |lambda| first."""
    c = np.asarray(c, dtype=np.complex128)
    lam, zl, zr = sla.eig(c, left=True, right=True)
    order = order_smallest(lam)
    lam = lam[order]
    zr = zr[:, order]
    zl = zl[:, order]
    y = np.empty_like(zr)
    z = np.empty_like(zl)
    for i in range(len(lam)):
        y[:, i], z[:, i] = normalise_pair(zr[:, i], zl[:, i])
    return y, z, lam


# Pivots below this (absolute; the coefficient vectors are unit-scaled) are
# treated as linear dependence and the pair is dropped.
PIVOT_TOL = 1e-10


def biorthogonalize(y1, z1, y2, z2, tol=PIVOT_TOL):
    """Bi-orthogonalize ``[y1; y2]`` against ``[z1; z2]`` (Algorithm BiCG-eigen).

    ``y1, z1`` (the eigenvectors of ``H^(m)``) are already biorthogonal
    (``z1^H y1 = I``) and are kept unchanged, as the paper notes. ``y2, z2``
    (those of ``H^(m-1)``, zero-padded) are first made oblique-orthogonal to
    the first block (``y2 -= y1 (z1^H y2)``, ``z2 -= z1 (y1^H z2)``), then
    biorthogonalized among themselves through an LU factorisation with
    complete pivoting of ``M = z2^H y2 = P L U Q^T``: ``y2 <- y2 Q U^{-1}``,
    ``z2 <- z2 P L^{-H}``. The factorisation stops at the first pivot below
    ``tol``; the remaining (nearly dependent) pairs are dropped.
    Returns ``(Y, Z)`` with ``Z^H Y = I``.
    """
    y2 = y2 - y1 @ (np.conj(z1.T) @ y2)
    z2 = z2 - z1 @ (np.conj(y1.T) @ z2)
    mat = np.conj(z2.T) @ y2
    k = mat.shape[0]
    a = mat.copy()
    row_perm = list(range(k))
    col_perm = list(range(k))
    rank = 0
    for i in range(k):
        sub = np.abs(a[i:, i:])
        piv = np.unravel_index(int(np.argmax(sub)), sub.shape)
        pr, pc = piv[0] + i, piv[1] + i
        if sub[piv] < tol:
            break
        a[[i, pr], :] = a[[pr, i], :]
        row_perm[i], row_perm[pr] = row_perm[pr], row_perm[i]
        a[:, [i, pc]] = a[:, [pc, i]]
        col_perm[i], col_perm[pc] = col_perm[pc], col_perm[i]
        a[i + 1:, i] /= a[i, i]
        a[i + 1:, i + 1:] -= np.outer(a[i + 1:, i], a[i, i + 1:])
        rank += 1
    lower = np.tril(a[:rank, :rank], -1) + np.eye(rank)
    upper = np.triu(a[:rank, :rank])
    yp = y2[:, col_perm[:rank]]
    zp = z2[:, row_perm[:rank]]
    y2t = sla.solve_triangular(upper.T, yp.T, lower=True).T if rank else yp
    # z2t = zp L^{-H}:  z2t^H = L^{-1} zp^H
    z2t = np.conj(sla.solve_triangular(lower, np.conj(zp.T), lower=True, unit_diagonal=True).T) if rank else zp
    return np.hstack([y1, y2t]), np.hstack([z1, z2t])
