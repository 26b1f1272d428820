"""Randomized bilinear computation for matrix products on GB300 (sm_103a).

The compute path is the C-ABI library librbc.so (include/rbc.h, csrc/); this package is
its build script and a thin ctypes binding.
"""
from .rbc import (  # noqa: F401
    RBC_EBUSY, RBC_ECUDA, RBC_EINVAL, RBC_EKAPPA, RBC_ENOMEM, RBC_ETIMEOUT, RBC_EUNSUPPORTED, RBC_OK,
    DRAW_PER_LEVEL, DRAW_PER_NODE, ERR_AVERAGE, ERR_EACH, IO_F32, IO_F64, LEAF_3XBF16, LEAF_3XTF32, LEAF_BF16,
    LEAF_BF16X6, LEAF_F16, LEAF_F16X3, LEAF_F32, LEAF_F64, LEAF_NAMES, LEAF_TF32, RAND_FULL, RAND_NONE, RAND_PERM, RAND_SIGN,
    SIGNATURES, Group, Plan, Queue, RbcError, lib, matmul, norms, realization_errors, realizations,
)
