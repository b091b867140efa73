"""GB300 (sm_103a) Runge–Kutta DG solver with the jump filter of arXiv 2407.19169.

The compute path is the CUDA library libdgjf.so behind the C ABI of include/dg.h; this package is
its thin Python binding (``Solver``) plus the seeded input generators (``inputs``).
"""
from ._native import (BASIS_P, BASIS_Q, BC_OUTFLOW, BC_PERIODIC, EQ_ADVECTION, EQ_BURGERS, EQ_EULER,
                      IC_ENTROPY1D, IC_QUADRANT2D, IC_RIEMANN1D, IC_SINE, IC_VORTEX2D, PREC_FP32_MIXED,
                      PREC_FP64, DGError, Solver, load)

__all__ = ["Solver", "DGError", "load", "BASIS_P", "BASIS_Q", "BC_OUTFLOW", "BC_PERIODIC", "EQ_ADVECTION",
           "EQ_BURGERS", "EQ_EULER", "IC_ENTROPY1D", "IC_QUADRANT2D", "IC_RIEMANN1D", "IC_SINE",
           "IC_VORTEX2D", "PREC_FP32_MIXED", "PREC_FP64"]
