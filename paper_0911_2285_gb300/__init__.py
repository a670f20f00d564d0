"""GB300 (sm_103a) Incremental eigBiCG for Wilson-Dirac systems with many right-hand sides.

The numerical work is in ``liblqcd.so`` (CUDA kernels behind the C ABI of
``include/lqcd.h``); :mod:`paper_0911_2285_gb300.lqcd` is its ctypes binding
and :mod:`paper_0911_2285_gb300.serving` the request loop.
"""
from .lqcd import (FP64, MIXED, MODE_AUTO, MODE_DEFLATED, MODE_EIGBICG, MODE_PLAIN, LQCDError, Solver,
                   restart_coefficients, small_eig)

__all__ = ["Solver", "LQCDError", "small_eig", "restart_coefficients", "FP64", "MIXED", "MODE_AUTO",
           "MODE_EIGBICG", "MODE_DEFLATED", "MODE_PLAIN"]
