"""GB300-native filtered block-sparse matrix multiply.

    C = beta * C + alpha * A . B      (block products filtered on block norms)

The computation is the local block multiplication of Sec. 2 of "Increasing
the Efficiency of Sparse Matrix-Matrix Multiplication with a 2.5D Algorithm
and One-Sided MPI" (blocked CSR matrices, result pattern determined by the
multiplication, on-the-fly filtering on the product of block norms), as called
by every tick of Algorithms 1 and 2. Every step runs in the CUDA kernels of
``libbsm.so`` behind the C ABI of ``include/bsm.h``; this package only
marshals arguments (see :mod:`paper_1705_10218_gb300.bsm`).
"""
from .bsm import (  # noqa: F401
    BSM_FP64_G8,
    BSM_FP64_NUM_KERNELS,
    BSM_FP64_PK12,
    BSM_FP64_PK16,
    BSM_FP64_T16_B2,
    BSM_FP64_T16_B3,
    BSM_FP64_T32,
    BSM_LAUNCH_PER_STACK,
    BSM_LAUNCH_PERSISTENT,
    BSM_PREC_FP64,
    BSM_PREC_SPLIT_BF16X3,
    BSM_PREC_SPLIT_TF32X2,
    BSM_SPLIT_BLOCKS,
    BSM_SPLIT_CHUNKS,
    BSM_SPLIT_PANEL,
    BsmError,
    Context,
    Matrix,
    Server,
    Stats,
    lib,
    lib_path,
)
