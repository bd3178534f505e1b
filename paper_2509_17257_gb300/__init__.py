"""GB300-native H²-matrix × dense-block product and block CG (arXiv 2509.17257).

The compute path is the CUDA library ``_build/libh2.so`` (sources in
``csrc/``, C ABI in ``include/h2.h``); this package is its binding.
"""
from .h2 import (  # noqa: F401
    DTYPES,
    EXPORTS,
    H2_BF16,
    H2_CG_COLUMNWISE,
    H2_E_BADARG,
    H2_E_BREAKDOWN,
    H2_E_CUDA,
    H2_E_NOCONVERGE,
    H2_E_OOM,
    H2_E_TIMEOUT,
    H2_E_UNSUPPORTED,
    H2_F32,
    H2_F64,
    H2_OK,
    H2Error,
    H2Batch,
    H2Matrix,
    h2_autotune,
    LIB_PATH,
    SolveResult,
    h2_adjoint_grads,
    h2_block_cg,
    h2_coupling_get,
    h2_coupling_set,
    h2_shift_set,
    h2_build,
    h2_free,
    h2_info,
    h2_matmul,
    h2_matmul_noalloc,
    h2_matmul_transposed,
    h2_timing_enable,
    h2_timing_query,
    PHASES,
    h2_tree_build,
    lib,
)
from .autograd import H2Solve, h2_solve  # noqa: E402,F401
