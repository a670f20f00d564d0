"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and shapes them into gauge links and
sources. It holds none of the solver's arithmetic: no Dirac operator, no
Krylov recurrence, no eigen-solve of the projected matrices. Both the CPU
oracle and the CUDA path consume its outputs, which is the only thing the two
share.

Conventions (shared by every consumer):

* lattice ``dims = (Lx, Ly, Lz, Lt)``; site index ``s = x + Lx*(y + Ly*(z + Lz*t))``;
  a field is stored C-order as ``[Lt][Lz][Ly][Lx][spin 4][colour 3]`` complex128;
* links ``[mu 4][Lt][Lz][Ly][Lx][3][3]`` complex128, ``mu = 0,1,2,3 = x,y,z,t``;
* the paper's test matrices (quenched Wilson configurations, Sec. 3) are not
  available, so random near-identity SU(3) fields ``U = exp(i*eps*H)`` with
  ``H`` Hermitian traceless Gaussian stand in for them;
* random generator: numpy ``default_rng`` (PCG64); link seeds 1, 2, 3, 4 for
  4^4, 8^4, 16^3x32, 24^3x64; source ``i`` of workload ``c`` uses seed
  ``1000*c + i``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "gauge_links",
    "gaussian_source",
    "z2_source",
    "random_su3",
    "WORKLOADS",
    "workload_links",
    "workload_source",
]


def volume(dims) -> int:
    lx, ly, lz, lt = dims
    return int(lx) * int(ly) * int(lz) * int(lt)


def _hermitian_traceless(rng: np.random.Generator, count: int) -> np.ndarray:
    """Draw ``count`` Hermitian traceless 3x3 matrices.

    Draw order: all real parts of a ``[count][3][3]`` array first, then all
    imaginary parts. ``G = (N(0,1) + i N(0,1))/sqrt(2)``, ``H = (G+G^H)/2 - tr/3``.
    """
    re = rng.standard_normal((count, 3, 3))
    im = rng.standard_normal((count, 3, 3))
    g = (re + 1j * im) / np.sqrt(2.0)
    h = 0.5 * (g + np.conj(np.swapaxes(g, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None, :, :]
    return h


def random_su3(rng: np.random.Generator, count: int, eps: float) -> np.ndarray:
    """``count`` SU(3) matrices ``exp(i*eps*H)`` via the eigen-decomposition of H."""
    h = _hermitian_traceless(rng, count)
    w, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    u = np.einsum("nab,nb,ncb->nac", q, ph, np.conj(q))
    return u


def gauge_links(dims, eps: float, seed: int) -> np.ndarray:
    """Random gauge field, shape ``[4][Lt][Lz][Ly][Lx][3][3]`` complex128.

    The underlying draw is one ``[4][V][3][3]`` array, directions outermost,
    sites in lexicographic order.
    """
    lx, ly, lz, lt = dims
    v = volume(dims)
    rng = np.random.default_rng(seed)
    u = random_su3(rng, 4 * v, eps)
    return np.ascontiguousarray(u.reshape(4, lt, lz, ly, lx, 3, 3))


def gaussian_source(dims, seed: int) -> np.ndarray:
    """Gaussian complex source ``(N(0,1)+iN(0,1))/sqrt(2)``, flat length ``12V``."""
    n = 12 * volume(dims)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    return (re + 1j * im) / np.sqrt(2.0)


def z2_source(dims, seed: int) -> np.ndarray:
    """Complex Z2 noise ``(eta1 + i eta2)/sqrt(2)``, ``eta in {+1,-1}``, flat length ``12V``."""
    n = 12 * volume(dims)
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(2, n), dtype=np.int8)
    eta = 1.0 - 2.0 * bits.astype(np.float64)
    return (eta[0] + 1j * eta[1]) / np.sqrt(2.0)


# The five synthetic workloads: the paper's multi-RHS problem (Eq. main-problem)
# on random-link stand-ins for its Wilson matrices (Sec. 3). Keys are the
# lattice shapes; values give the link smearing, hopping parameter, solver
# window, sources and the seed family used above.
WORKLOADS = {
    "4^4": dict(dims=(4, 4, 4, 4), eps=0.5, kappa=0.12, link_seed=1, cfg=1,
                nev=8, m=24, n1=1, n_rhs=1, source="gaussian"),
    "8^4": dict(dims=(8, 8, 8, 8), eps=0.3, kappa=0.124, link_seed=2, cfg=2,
                nev=10, m=40, n1=4, n_rhs=12, source="z2"),
    "16^3x32": dict(dims=(16, 16, 16, 32), eps=0.3, kappa=0.124, link_seed=3, cfg=3,
                    nev=10, m=60, n1=4, n_rhs=24, source="z2"),
    "24^3x64": dict(dims=(24, 24, 24, 64), eps=0.3, kappa=0.1245, link_seed=4, cfg=4,
                    nev=10, m=60, n1=8, n_rhs=64, source="z2"),
}


def workload_source(name: str, i: int) -> np.ndarray:
    """Source ``i`` (0-based) of a named workload."""
    w = WORKLOADS[name]
    seed = 1000 * w["cfg"] + i
    if w["source"] == "gaussian":
        return gaussian_source(w["dims"], seed)
    return z2_source(w["dims"], seed)


def workload_links(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return gauge_links(w["dims"], w["eps"], w["link_seed"])
