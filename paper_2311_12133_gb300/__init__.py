"""HPEZ (arXiv 2311.12133) interpolation predict-and-quantize path for GB300.

The compute runs in hand-written sm_103a CUDA kernels behind the C-ABI
library ``libhpez.so`` (declared in ``include/hpez.h``); ``hpez`` is its thin
ctypes binding.  ``fields`` draws the seeded synthetic inputs.
"""
