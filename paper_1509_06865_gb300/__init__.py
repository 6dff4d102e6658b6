"""GB300-native multigrid Rayleigh quotient eigensolver for the Hermitian
clover-improved Wilson operator Q = gamma5 D (arXiv:1509.06865).

The compute path is libmgeig.so (hand-written CUDA for sm_103a behind the C ABI
in include/mgeig.h); ``Context`` is its ctypes binding.
"""
from ._lib import (EBREAKDOWN, EINVAL, ENOCONV, ENOTSETUP, ETIMEOUT, FP64, GMRES, LEARNED, LINKS_BF16, LINKS_F16,
                   LINKS_LEVEL, MIXED, NET_SHAPE, OP_D, OP_Q, PREC_F32, PREC_F64, PREC_F64_DS, PREC_F32_F64_DS, SAP, Context, MgeigError, check_params,
                   load, solve_batch)

__all__ = ["Context", "MgeigError", "check_params", "load", "solve_batch", "FP64", "MIXED", "SAP", "GMRES", "LEARNED", "NET_SHAPE", "OP_Q", "OP_D", "PREC_F64", "PREC_F64_DS", "PREC_F32_F64_DS",
           "PREC_F32", "LINKS_LEVEL", "LINKS_BF16", "LINKS_F16", "EINVAL", "ENOTSETUP", "ENOCONV", "EBREAKDOWN",
           "ETIMEOUT"]
