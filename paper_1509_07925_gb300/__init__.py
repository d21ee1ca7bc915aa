"""GB300-native apply of the multidimensional butterfly factorization.

Package layout:
  csrc/        C++ host builder (FP64), packer, C ABI, sm_103a CUDA kernels
  buildlib.py  compiles csrc/ into _lib/libmbf.so for sm_103a
  binding.py   ctypes binding with the names of include/mbf.h
"""
from .binding import (  # noqa: F401
    MBF_PREC_AUTO, MBF_PREC_BF16X3, MBF_PREC_FP32_SIMT, MBF_PREC_TF32, MBF_TREE_POLAR,
    MBF_TREE_SQUARE, MBF_TREE_UNIFORM, HostFactors, MbfError, Operator, lib)
