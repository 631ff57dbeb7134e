"""GB300-native (sm_103a) Modified Virtual Grid Difference discretisation of the
Laplace-Beltrami operator on point clouds, with device-resident solves of
(sigma I - L) u = f.

Submodules:
  api      PyTorch-facing calls over the C ABI (knn, assemble, spmv, solve)
  batch    uneven clouds through shared persistent launches
  serve    continuous-batching request loop
  inputs   seeded synthetic clouds and exact solutions (no method arithmetic)
  build    nvcc build of the in-tree libmvgd.so
"""
__all__ = ["api", "inputs", "build"]
