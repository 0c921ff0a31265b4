"""GB300-native (sm_103a) per-frame non-rigid deformation solve.

libdefsolve.so (CUDA kernels behind a C ABI, include/defsolve.h) does all the work; defsolve.py
is its ctypes binding, build.py compiles it in-tree and serve.py is the multi-stream serving loop.
"""
