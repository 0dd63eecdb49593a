// Per-precision entry points of the solver (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "mrrr.h"
#include "mrrr_types.cuh"

namespace mrrr {
// binary32 input/output: working precision binary64 (mixed) or binary32 (plain)
int solve_batch_s_mixed(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats);
int solve_batch_s_plain(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats);
// binary64 input/output: working precision double-double (mixed) or binary64 (plain)
int solve_batch_d_mixed(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats);
int solve_batch_d_plain(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats);
}  // namespace mrrr
