"""GB300 (sm_103a) rasterizer for native 4D Gaussians -- the optimisation hot path of Instant4D
(arXiv 2510.01119): Eq. 7-8 slicing, temporal opacity, EWA projection, tile binning with a device
radix sort, compositing, the analytic backward, fused Adam, and voxel-grid pruning.

All compute is in libi4d.so (hand-written CUDA, C ABI in include/i4d.h); this package only
marshals arguments.  Submodules: ``build`` (nvcc build), ``_lib`` (ctypes binding, same names as
the C ABI), ``rasterizer`` (buffers + torch.autograd.Function), ``prune``, ``train``.
"""
__all__ = ["build", "_lib", "rasterizer", "prune", "train"]
