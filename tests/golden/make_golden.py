"""Write the stored expected values under ``tests/golden/``.

Calls only the oracle (``oracle/``), the seeded input generators and
LAPACK (scipy). Run from the repository root:

    python tests/golden/make_golden.py

``wilson_4x4x4x4_lowest_eigs.txt``: the 64 eigenvalues of smallest modulus of
the dense 3072 x 3072 Wilson matrix ``A = 1 - kappa D_hop`` of the 4^4
workload (random links eps = 0.5, seed 1, kappa = 0.12), from a dense
LAPACK eigensolve. They are the reference against which converged eigBiCG
Ritz values are checked (the paper's Table 1 compares eigBiCG with
un-restarted BiCG in the same way, Sec. 3).

``wilson_4x4x4x4_eps0.1_lowest_eigs.txt``: the same for a weakly disordered
4^4 field (links eps = 0.1, seed 21, kappa = 0.122). Its lowest twelve
eigenvalues form an isolated group (|lambda| ~ 0.03, the next ones ~ 0.35),
which Incremental eigBiCG resolves to full FP64 accuracy; the GPU's converged
Rayleigh-Ritz pairs are checked against it.
"""
import os
import sys

import numpy as np
import scipy.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.wilson import WilsonOperator  # noqa: E402
from seeded_inputs import WORKLOADS, gauge_links, workload_links  # noqa: E402


def write_lowest(op, path, header):
    lam = sla.eigvals(op.dense())
    lam = lam[np.argsort(np.abs(lam), kind="stable")][:64]
    with open(path, "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for z in lam:
            f.write(f"{z.real:.17e} {z.imag:.17e}\n")
    print("wrote", path)


def weak_field():
    dims = (4, 4, 4, 4)
    return WilsonOperator(gauge_links(dims, 0.1, 21), 0.122, dims)


def main():
    w = WORKLOADS["4^4"]
    op = WilsonOperator(workload_links("4^4"), w["kappa"], w["dims"])
    a = op.dense()
    lam = sla.eigvals(a)
    lam = lam[np.argsort(np.abs(lam), kind="stable")][:64]
    path = os.path.join(HERE, "wilson_4x4x4x4_lowest_eigs.txt")
    with open(path, "w") as f:
        f.write("# 64 smallest-|lambda| eigenvalues of A = 1 - kappa D_hop, 4^4 workload\n")
        f.write("# (links eps=0.5 seed=1, kappa=0.12), dense LAPACK eigvals of the oracle's matrix.\n")
        f.write("# Written by tests/golden/make_golden.py. Columns: Re Im\n")
        for z in lam:
            f.write(f"{z.real:.17e} {z.imag:.17e}\n")
    print("wrote", path)
    write_lowest(weak_field(), os.path.join(HERE, "wilson_4x4x4x4_eps0.1_lowest_eigs.txt"),
                 ["64 smallest-|lambda| eigenvalues of A = 1 - kappa D_hop on 4^4",
                  "(links eps=0.1 seed=21, kappa=0.122), dense LAPACK eigvals of the oracle's matrix.",
                  "Written by tests/golden/make_golden.py. Columns: Re Im"])


if __name__ == "__main__":
    main()
