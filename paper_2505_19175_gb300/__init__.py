"""GB300-native differentiable triangle-splat rasterizer (arXiv 2505.19175).

The compute path is a C-ABI CUDA library (``include/trisplat.h``); this package is its
thin Python binding plus an autograd wrapper and the serving front end. The native
library is loaded on first use and its absence is an error: there is no CPU fallback.
"""
