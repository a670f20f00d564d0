"""Even-odd (Schur complement) form of the Wilson operator, FP64, numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's test matrices are even-odd preconditioned (Sec. 3). ``D_hop``
connects only sites of opposite parity ``(x + y + z + t) mod 2`` (all extents
even), so with ``A = 1 - kappa D_hop`` split into even and odd blocks,

    A = [[1, -kappa D_eo], [-kappa D_oe, 1]],

the odd unknowns solve ``A_hat x_o = b_hat`` with the Schur complement
``A_hat = 1 - kappa^2 D_oe D_eo`` and ``b_hat = b_o + kappa D_oe b_e``, and
``x_e = b_e + kappa D_eo x_o``. ``det A = det A_hat``, and ``A_hat`` keeps the
gamma5 symmetry ``gamma5 A_hat gamma5 = A_hat^dagger``. Vectors of the odd
sublattice are flat complex128 arrays of ``12 V / 2`` entries in site order.
"""
from __future__ import annotations

import numpy as np

from .wilson import GAMMA5, _spin, field_shape, hop, to_field


class EvenOddOperator:
    """``A_hat`` on the odd sublattice, same interface as ``WilsonOperator``."""

    def __init__(self, links, kappa, dims):
        self.links = np.asarray(links, dtype=np.complex128)
        self.kappa = float(kappa)
        self.dims = tuple(int(d) for d in dims)
        if any(d % 2 for d in self.dims):
            raise ValueError("even-odd splitting needs even extents")
        lx, ly, lz, lt = self.dims
        t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
        self.odd = ((x + y + z + t) % 2) == 1          # [lt, lz, ly, lx]
        self.n = 12 * int(self.odd.sum())
        self.matvecs = 0

    # odd-sublattice vector <-> full field (zero on the other parity)
    def embed(self, v, odd=True):
        f = np.zeros(field_shape(self.dims), dtype=np.complex128)
        f[self.odd if odd else ~self.odd] = np.asarray(v, dtype=np.complex128).reshape(-1, 4, 3)
        return f

    def extract(self, f, odd=True):
        return f[self.odd if odd else ~self.odd].reshape(-1)

    def _schur(self, v, dagger):
        psi = self.embed(v)
        tmp = hop(self.links, psi, dagger)               # odd -> even sites
        tmp[self.odd] = 0.0
        out = hop(self.links, tmp, dagger)               # even -> odd sites
        return np.asarray(v, dtype=np.complex128) - self.kappa ** 2 * self.extract(out)

    def apply(self, v):
        self.matvecs += 1
        return self._schur(v, False)

    def apply_dag(self, v):
        self.matvecs += 1
        return self._schur(v, True)

    def gamma5(self, v):
        return _spin(GAMMA5, np.asarray(v, dtype=np.complex128).reshape(-1, 4, 3)).reshape(-1)

    def prepare(self, b):
        """``b_hat = b_o + kappa D_oe b_e`` from a full source ``b``."""
        f = to_field(b, self.dims)
        be = f.copy()
        be[self.odd] = 0.0
        return self.extract(f) + self.kappa * self.extract(hop(self.links, be, False))

    def reconstruct(self, b, x_odd):
        """Full solution: ``x_e = b_e + kappa D_eo x_o`` and ``x_o``."""
        f = to_field(b, self.dims)
        xo = self.embed(x_odd)
        xe = f + self.kappa * hop(self.links, xo, False)
        xe[self.odd] = 0.0
        return (xe + xo).reshape(-1)

    def dense(self):
        a = np.empty((self.n, self.n), dtype=np.complex128)
        e = np.zeros(self.n, dtype=np.complex128)
        for j in range(self.n):
            e[j] = 1.0
            a[:, j] = self.apply(e)
            e[j] = 0.0
        return a
