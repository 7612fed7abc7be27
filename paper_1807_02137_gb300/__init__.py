"""GB300 (sm_103a) multigrid solver for level-set selective segmentation (arXiv 1807.02137).

The solver is a CUDA library behind the C ABI of include/segmg.h; ``segmg`` is its thin Python
binding and ``synth`` holds the seeded synthetic inputs.  ``build()`` compiles the library.
"""
from .buildlib import build, LIB  # noqa: F401

__all__ = ["build", "LIB"]
