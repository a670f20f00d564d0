"""Wilson-Dirac operator of the paper's test problems (Sec. 3), FP64, numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper solves ``A x = b`` for quenched Wilson matrices with
``kappa = 1/(8 + 2 m_q)`` (Sec. 3) and uses gamma5-Hermiticity
``gamma5 A = A^dagger gamma5`` (Sec. 4). It does not print the operator; this
module uses the textbook unpreconditioned Wilson form

    A psi(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                                        + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]

with periodic boundaries in all four directions. The adjoint is written out
from the matrix elements (not through gamma5), so that the gamma5-Hermiticity
check in the tests is a real check:

    A^dagger psi(x) = psi(x) - kappa * sum_mu [ (1 + gamma_mu) U_mu(x) psi(x+mu)
                                               + (1 - gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]

Gamma matrices: Euclidean, Hermitian, chiral basis
``gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]``, ``gamma_4 = [[0, 1], [1, 0]]``,
so ``gamma5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1)``.

Field layout: ``[Lt][Lz][Ly][Lx][spin 4][colour 3]``; links ``[mu][Lt][Lz][Ly][Lx][3][3]``
with ``mu = 0..3 = x, y, z, t``; direction ``mu`` runs along array axis ``3 - mu``.
"""
from __future__ import annotations

import numpy as np

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.stack([
    _block(_Z2, -1j * _S1, 1j * _S1, _Z2),
    _block(_Z2, -1j * _S2, 1j * _S2, _Z2),
    _block(_Z2, -1j * _S3, 1j * _S3, _Z2),
    _block(_Z2, _I2, _I2, _Z2),
])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
I4 = np.eye(4, dtype=np.complex128)


def field_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx, 4, 3)


def to_field(v, dims):
    return np.asarray(v, dtype=np.complex128).reshape(field_shape(dims))


def _spin(mat, psi):
    """Apply a 4x4 spin matrix to every site of a field."""
    return np.einsum("st,...tc->...sc", mat, psi)


def _colour(u, psi):
    """Apply per-site 3x3 colour matrices ``u[...,a,b]`` to ``psi[...,s,b]``."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def _colour_dag(u, psi):
    """Apply ``u^dagger`` per site."""
    return np.einsum("...ba,...sb->...sa", np.conj(u), psi)


def hop(links, psi, dagger=False):
    """``D_hop psi`` (or ``D_hop^dagger psi`` when ``dagger``) on a field array."""
    out = np.zeros_like(psi)
    sign = 1.0 if dagger else -1.0
    for mu in range(4):
        ax = 3 - mu
        u = links[mu]
        fwd = _colour(u, np.roll(psi, -1, axis=ax))               # U_mu(x) psi(x+mu)
        u_back = np.roll(u, 1, axis=ax)                             # U_mu(x-mu)
        bwd = _colour_dag(u_back, np.roll(psi, 1, axis=ax))        # U_mu(x-mu)^+ psi(x-mu)
        out += _spin(I4 + sign * GAMMA[mu], fwd)
        out += _spin(I4 - sign * GAMMA[mu], bwd)
    return out


class WilsonOperator:
    """``A = 1 - kappa D_hop`` on flat complex128 vectors of length ``12 V``."""

    def __init__(self, links, kappa, dims):
        self.links = np.asarray(links, dtype=np.complex128)
        self.kappa = float(kappa)
        self.dims = tuple(int(d) for d in dims)
        lx, ly, lz, lt = self.dims
        self.volume = lx * ly * lz * lt
        self.n = 12 * self.volume
        assert self.links.shape == (4, lt, lz, ly, lx, 3, 3)
        self.matvecs = 0

    def apply(self, v):
        """``A v``."""
        self.matvecs += 1
        psi = to_field(v, self.dims)
        return (psi - self.kappa * hop(self.links, psi, False)).reshape(-1)

    def apply_dag(self, v):
        """``A^dagger v``."""
        self.matvecs += 1
        psi = to_field(v, self.dims)
        return (psi - self.kappa * hop(self.links, psi, True)).reshape(-1)

    def gamma5(self, v):
        psi = to_field(v, self.dims)
        return _spin(GAMMA5, psi).reshape(-1)

    def dense(self):
        """Dense ``N x N`` matrix, column by column (small lattices only)."""
        a = np.empty((self.n, self.n), dtype=np.complex128)
        e = np.zeros(self.n, dtype=np.complex128)
        for j in range(self.n):
            e[j] = 1.0
            a[:, j] = self.apply(e)
            e[j] = 0.0
        return a


class DenseOperator:
    """Same interface as :class:`WilsonOperator` for an explicit matrix."""

    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.complex128)
        self.n = self.a.shape[0]
        self.matvecs = 0

    def apply(self, v):
        self.matvecs += 1
        return self.a @ v

    def apply_dag(self, v):
        self.matvecs += 1
        return np.conj(self.a.T) @ v

    def dense(self):
        return self.a.copy()
