"""GB300-native star-forest communication (PetscSF's Bcast / Reduce / FetchAndOp hot path).

The compute path is libsfgb.so (hand-written sm_103a kernels behind the C ABI of
include/sf.h); this package only marshals arguments.  Importing it loads the library and
raises ImportError when it has not been built: there is no CPU fallback.
"""
from . import _abi
from ._abi import SFError, SF_FOLD_BLOCK

_abi.load()

from .sf import StarForest, Batch, launch_count, OPS, MODES, PATHS  # noqa: E402

__all__ = ["StarForest", "Batch", "SFError", "launch_count", "OPS", "MODES", "PATHS", "SF_FOLD_BLOCK"]
