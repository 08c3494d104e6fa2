"""GB300 (sm_103a) implementation of the FTK pose-scoring path of arXiv 1905.12317.

The computation lives in ``_build/libftk.so`` (hand-written CUDA kernels behind the
C ABI of ``include/ftk.h``). This package is its thin Python binding.
"""

from .binding import (  # noqa: F401
    BF16,
    BF16X3,
    FP16,
    FP32,
    PRECISIONS,
    FtkError,
    Plan,
    align_best_groups,
    groups_workspace_size,
    header_functions,
    load_library,
    rank_profile,
)
