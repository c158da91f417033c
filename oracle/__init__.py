"""Plain FP64 CPU oracle for the optimized Schwarz method of Besse & Xing (arXiv:1603.05110).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or execute
anything in this package.  The product path (the CUDA library and its Python binding) never
imports it and shares no code with it.

Modules:
* ``fem``  -- Q1 element assembly on a uniform mesh (Sec. 2.2).
* ``nls``  -- the time step (eq. CNS), strip problems with Robin (eq. NproblemRobinNL) or
  S_pade^m (eq. NproblemSPNL) data, the classical (eq. algo_d) and preconditioned
  (eq. algo_pd) Schwarz algorithms, L_h (eq. Lmpi) by unit solves and on the cosine modes,
  mass and energy diagnostics.
* ``gpe``  -- the rotating frame of Sec. 5.2 (eq. x1Ax, GPE_Trans, u1u): time-dependent trap,
  angular momentum and the energy of eq. (GPE), lab-frame reconstruction on the valid zone.
* ``cnn``  -- the learned interface guess (no counterpart in the paper).

Parity status: every function is pinned by a ``-m "not gpu"`` test against values fixed by
the mathematics (brute force, closed forms, invariants, textbook special cases); the
paper's printed iteration counts (Table Influence_p_NL_2_32) are a soft pin only.
"""
from . import fem, gpe, nls  # noqa: F401
