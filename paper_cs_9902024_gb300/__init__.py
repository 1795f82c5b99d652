"""GB300-native ensemble DSMC for unsteady rarefied gas flows.

Submodules (imported explicitly, so that importing the package loads no
native code):
  workloads  synthetic workload descriptions (inputs only)
  build      in-tree nvcc build of libdsmc.so for sm_103a
  dsmc       ctypes binding of the C ABI in include/dsmc.h
"""
