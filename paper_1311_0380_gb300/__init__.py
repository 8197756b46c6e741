"""GB300 (sm_103a) implementation of the SVT linearised track fit hot path.

Submodules:
  synth   -- seeded synthetic inputs (event words, constant tables, tracks)
  api     -- Python face of the C ABI in include/svt.h (libsvt.so)
  build   -- in-tree nvcc build of libsvt.so
Importing the package loads nothing; ``api`` loads the CUDA library on first
use and raises if it is missing.
"""
__version__ = "1.0.0"
