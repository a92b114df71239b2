"""Oracle: a plain, slow, FP64 CPU implementation of one semi-implicit BDF step of the paper's
P1-P1 VMS-LES Navier-Stokes discretisation (Section 2.3) and of the aSIMPLE-preconditioned
GMRES solve (Section 2.4); also the outlet conditions of Section 2.2 (backflow stabilisation,
resistance), the moving-domain parts (lifting, mesh velocity, u* = u^EXT - u_ALE) and the fully
implicit formulation solved by Newton's method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library (no kernels, no
headers, no helpers, no constants) and neither imports the other; the two meet only through
the seeded inputs of the ``synthetic`` package.

Element integrals are plain C (``lfx_oracle.c``); global assembly, boundary conditions and the
linear solve are numpy/scipy (``core.py``, ``krylov.py``).  Parity status of each function is
in its docstring; every function is pinned by ``tests/test_oracle_*.py``.
"""
from .core import *  # noqa: F401,F403
from .krylov import *  # noqa: F401,F403
