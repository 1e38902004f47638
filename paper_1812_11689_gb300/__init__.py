"""rpForests kNN search (arXiv 1812.11689) on one GB300 (sm_103a).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/rpforest.h``); this package only marshals arguments to it.
"""
from ._lib import RpfError  # noqa: F401


def __getattr__(name):
    if name in ("Forest", "directions", "FORM_PLAIN", "FORM_CHOSEN", "GROWTH_DEFAULT",
                "GROWTH_FP64", "GROWTH_CERTIFIED"):
        from . import forest
        return getattr(forest, name)
    raise AttributeError(name)
