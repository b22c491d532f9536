"""GB300-native 4D generalized subjective-surface segmentation (arXiv 2111.11866).

The computation lives in ``_build/libseg4d.so`` (CUDA, sm_103a; C ABI in
``include/seg4d.h``); ``_lib`` is its ctypes binding and ``synth`` holds the
seeded synthetic inputs.  Build with ``build.build()``.
"""

__all__ = ["Seg4D", "Params", "Seg4DError", "build"]


def __getattr__(name):
    if name in ("Seg4D", "Params", "Seg4DError"):
        from . import _lib
        return getattr(_lib, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
