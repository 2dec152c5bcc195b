"""GB300-native diffuse-interface finite-volume step (arXiv 2009.14555).

  workloads   seeded synthetic inputs shaped like the paper's problems
  solver      Solver: the C ABI of libdis.so over torch device memory
  autograd    torch.autograd.Function over the library's adjoint
  _lib        ctypes binding of include/dis.h
  build       nvcc build of libdis.so for sm_103a
"""
