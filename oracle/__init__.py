"""ORACLE (test infrastructure only).

A plain, slow, FP64 CPU implementation of the nodal discontinuous Galerkin
semi-discretisation of the 2D TM Maxwell equations (upwind flux, PEC walls)
and of the LSRK(5,4) time integrator, written from the chapter's description
of the method.  It exists to check the CUDA library.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
(and its ``--impl reference`` arm) may import it.  It shares no code with the
CUDA library (``paper_1304_5546_gb300``) and imports nothing from it.
"""
from .dg2d import *  # noqa: F401,F403
