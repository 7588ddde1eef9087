"""FP64 CPU oracle for LSLU / Hybrid LSLU (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked
against.  Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does.  It shares no code with
the CUDA library: it reads only the seeded inputs from the tomography module.
"""
from .lslu_oracle import (  # noqa: F401
    OracleResult,
    hessenberg_rect_pivoted,
    projected_svd,
    tikhonov_y,
    projected_residual,
    gcv_value,
    gcv_slope,
    select_lambda,
    lambda_grid,
    hybrid_lslu,
)
