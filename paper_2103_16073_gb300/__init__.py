"""GB300 (sm_103a) FMM-accelerated Helmholtz BEM for room acoustics.

The C-ABI library libfmmbem.so (include/fmmbem.h) does every computation;
``binding`` marshals arguments to it.  The binding, and with it the shared
library, is loaded on the first use of one of its names (``fb_*``, ``FB_*``,
``lib``, ``FBError``, ...), so that the input generators (``workloads``) can
be imported without mapping the library.  When the library cannot be built
or loaded that first use raises: there is no CPU fallback.
"""
from __future__ import annotations

import importlib

_BINDING_NAMES = {"lib", "FBError", "SolverOpts", "SolveInfo", "PHASES", "STATUS_NAMES"}


def _is_binding_name(name: str) -> bool:
    return name.startswith(("fb_", "FB_")) or name in _BINDING_NAMES


def __getattr__(name):
    # submodules (workloads, training, ...) never reach the binding here
    if not _is_binding_name(name):
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
    binding = importlib.import_module(".binding", __name__)
    return getattr(binding, name)
