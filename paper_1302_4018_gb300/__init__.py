"""GB300 library for hierarchical probing of Tr(A^-1) on 4-D toroidal lattices.

Submodules:
  hprobe    ctypes binding of libhprobe.so (the C ABI of include/hprobe.h)
  autograd  torch.autograd.Function over hp_trace_inv_grad
  synth     seeded synthetic inputs (gauge links, mass fields, batch configs)
  build     nvcc build of libhprobe.so for sm_103a
Importing the package loads nothing; ``hprobe`` loads the CUDA library and
fails loudly if it has not been built.
"""
