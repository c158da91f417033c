"""dd_nls: optimized Schwarz time stepping for the 2D NLS / GPE on one GB300 (sm_103a).

Besse & Xing, "Domain decomposition algorithms for the two dimensional nonlinear
Schroedinger equation and simulation of Bose-Einstein condensates" (arXiv:1603.05110).

The method runs in the CUDA library ``libddnls.so`` behind the C-ABI of
``include/dd_nls.h``; ``binding`` is its ctypes binding and ``workloads`` the seeded inputs.
"""
from . import workloads  # noqa: F401
from .binding import (BC_NEUMANN, BC_SAME, CLASSICAL, FP32_DW, FP32_INNER, FP64, GUESS_PREVIOUS,  # noqa: F401
                      GUESS_ZERO, PRECONDITIONED, PSOLVE_GMRES, PSOLVE_MODAL, TC_PADE, TC_ROBIN,
                      CNN, Batch, DDNLSError, Solver,
                      default_params, load)
