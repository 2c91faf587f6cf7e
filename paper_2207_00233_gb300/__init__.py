"""GB300 (sm_103a) Frequency Selective Extrapolation block-loss concealment.

Python access to the C-ABI of ``libfse_gb300.so`` (see ``include/fse.h``).
The library is required: importing this package does not build it, and the
functions raise when it is missing.
"""
from ._native import (  # noqa: F401
    EXPORTED, FSE_EXEC_GROUPS, FSE_OPT_AUTOTUNE, FSE_OPT_GROUP_LAUNCHES, FSE_OPT_INPUTS_READY, FSE_OPT_PERSISTENT_CTAS, FSE_OPT_SERVE_LATENCY_MS, FSE_OPT_SERVE_MAX_BATCH, FSE_OPT_W_TABLES, FSE_OPT_CLAIM_ORDER, FSE_OPT_PHASE_CLOCKS, FSE_CLAIM_DELAYED, FSE_CLAIM_HEIGHT, FSE_CLAIM_LIST,
    FSE_OPT_SERVE_SLOTS, FSE_OPT_SPIN_LIMIT, FSE_OPT_TEST_STUCK_DEP, FSE_OPT_KEEP_TRACE, FSE_EXEC_PERSISTENT, FSE_MAX_ITERS, FSE_ORDER_LINESCAN,
    FSE_ORDER_OPTIMIZED, FSE_PREC_BF16, FSE_PREC_BF16X3, FSE_PREC_FP16, FSE_PREC_FP32,
    FSE_PREC_TF32, FSE_PREC_TF32X3, Context, FseError, fse_frame, fse_loop_microbench, fse_measure_peaks, fse_params, fse_plan_claims, fse_plan_order, fse_stats, lib,
    make_params, strerror,
)
