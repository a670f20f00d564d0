"""CPU FP64 oracle for Incremental eigBiCG (Abdel-Rehim, Orginos, Stathopoulos,
"Extending the eigCG algorithm to non-symmetric linear systems with multiple
right-hand sides", Lattice 2009).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
statement of what the GPU library computes. Only the test-suite, the
``__graft_entry__.smoke`` check and the CPU-baseline leg of ``bench.py`` may
import it. The product library never calls into it and shares no code with it
(the seeded input generators in ``seeded_inputs`` are the only common module).

Modules:

* :mod:`oracle.wilson`   -- Wilson-Dirac operator ``A = 1 - kappa*D_hop`` and its
  adjoint (the paper's test matrices, Sec. 3; gamma5-Hermiticity, Sec. 4);
* :mod:`oracle.smalleig` -- ``[zr, zl, D] = eig(C)`` with the paper's selection
  by smallest absolute value (Sec. 1 notation, Algorithm BiCG-eigen);
* :mod:`oracle.bicg`     -- BiCG, Algorithm eigBiCG and Algorithm BiCG-eigen;
* :mod:`oracle.incremental` -- Algorithm Incremental eigBiCG, the oblique
  deflation of the initial guess and the final Rayleigh-Ritz step (Sec. 2).

Everything is complex128 (FP64). Parity pins: see ``tests/test_oracle_*.py``.
"""
