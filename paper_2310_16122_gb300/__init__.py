"""GB300-native (sm_103a) CRK-HACC short-range pair kernels behind a C ABI (libcrk.so).

Modules: ``native`` (ctypes binding of include/crk.h), ``api`` (PyTorch
device memory and streams), ``autograd`` (adjoint-backed autograd
functions), ``workloads`` (seeded synthetic inputs), ``build`` (nvcc build).
Importing the package loads nothing; the binding raises if libcrk.so is
missing.
"""
