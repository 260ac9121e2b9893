"""GB300-native GPAIR hot path: the direct windowed forward operator of a sum of isotropic 3-D
Gaussians, its exact adjoint with amplitude/centre/width gradients, voxelisation and the
reconstruction step (arXiv 2602.03893, Methods).

The compute lives in libgpair.so (hand-written sm_103a CUDA behind the C ABI of
include/gpair.h); `_lib` is its ctypes binding.  Importing this package does not load the
library; the first call does, and raises if it cannot.
"""
__all__ = ["synth"]
