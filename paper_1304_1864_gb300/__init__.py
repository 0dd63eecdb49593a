"""GB300-native mixed-precision MRRR eigensolver for symmetric tridiagonal matrices.

The solver is the CUDA library libmrrr.so (C ABI in include/mrrr.h); this
package holds its sources (csrc/), the build step (build.py), the ctypes
binding (_binding.py) and the seeded synthetic test matrices (inputs.py).
"""
from ._binding import (  # noqa: F401
    MRRR_ALL, MRRR_INDEX, MRRR_VALUE, MRRR_PLAIN, MRRR_MIXED, MRRR_OK, MRRR_ERR_ARG, MRRR_ERR_NONFINITE,
    MRRR_ERR_NOCONV, MRRR_ERR_NOMEM, MRRR_ERR_CUDA, MRRR_FLAG_TIMING, MRRR_FLAG_STRICT_GROWTH, MRRR_FLAG_NO_TUNE,
    MRRR_FLAG_NO_LOWPREC_BISECT, MRRR_FLAG_TEST_REJECT_CHILD, MRRR_FLAG_E_REP, MRRR_FLAG_RRR_TEST, MRRR_FLAG_TEST_NO_REP, MRRR_ERR_CANCELLED, mrrr_serve_cancel, MrrrError, MrrrParams, MrrrStats, lib, make_params, mrrr_eigvecs_noalloc_s,
    mrrr_solve_batch_d,
    mrrr_solve_batch_s, mrrr_solve_d, mrrr_solve_s, mrrr_strerror, mrrr_version, solve, solve_batch, strerror,
    MRRR_PENDING, MrrrRequest, MrrrServeConfig, MrrrServeInfo, MrrrServeStats, Server, mrrr_serve_close,
    mrrr_serve_open, mrrr_serve_poll, mrrr_serve_stats_get, mrrr_serve_submit, mrrr_probe_fp64_fma, probe_fp64,
    mrrr_partition_s, mrrr_partition_d, partition, mrrr_syev_s, mrrr_syev_d, solve_dense,
)
