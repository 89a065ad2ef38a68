"""FP64 CPU oracle for the AsyFLEXA fixed-stepsize block update.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use it.  It shares no code with the CUDA library (no kernels, headers, helpers or
constants); the only thing both sides consume is the problem data produced by the
seeded generators in ``inputs/``.

``oracle.cores`` (imported on demand) is the multi-core C form of the method for LASSO
(``cores.c``), for the core-count study of Section 4.2.
"""

from .asyflexa import *  # noqa: F401,F403
