"""GB300-native (sm_103a) AsyFLEXA block-update library: C ABI + thin Python binding.

The compute path is the CUDA library ``_lib/libasyflexa.so`` (see ``include/asyflexa.h``);
``native`` marshals arguments to it.  There is no CPU implementation in this package.
"""

from .native import (  # noqa: F401
    ASYNC, SYNC, F32, F64, BF16, FP8E4M3, LOSS_LASSO, LOSS_NCQUAD,
    AsyflexaError, Problem, Opts, Stats, Solver, default_opts, lib, EXPORTS, LIB_PATH,
)

__version__ = "0.1.0"
