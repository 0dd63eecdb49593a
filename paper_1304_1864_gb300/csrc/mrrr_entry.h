// Per-precision entry points of the solver (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "mrrr.h"
#include "mrrr_types.cuh"

namespace mrrr {
// Stream-ordered device memory of the library: one memory pool per device,
// created on first use, that keeps freed blocks cached for the next solve
// (release threshold: no limit) instead of returning them to the driver at
// every synchronisation, and never reuses a block across streams by
// inserting a wait between them.  alloc returns nullptr on failure.
void* dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
// Pinned host memory for small copies between host and device (a copy from
// or to pageable memory goes through a synchronous staging path of the
// driver).  *got receives the block's size, to pass back to host_free.
void* host_alloc(size_t bytes, size_t* got);
void host_free(void* p, size_t got);

// Online autotuner of the persistent RQI grid (resident one-warp CTAs per
// SM).  Workloads are grouped into classes by `key` (working precision, and
// the magnitudes of the list length and of the largest n).  The first runs
// of a class try the candidates kRqiTuneWarps in turn and report their time;
// afterwards the fastest is used.  The choice only changes scheduling: each
// eigenpair's arithmetic, and so every result, is the same for every grid.
constexpr int kRqiTuneCandidates = 3;
constexpr int kRqiTuneWarps[kRqiTuneCandidates] = {16, 8, 4};
// returns the warps per SM to use; *trial = the candidate to time in this
// run, or -1 once the class is decided
int rqi_tune_pick(unsigned key, int* trial);
void rqi_tune_report(unsigned key, int trial, float ms);

// The root-level classification of a batch (Algorithm 1, line 7, at the
// root representation), for partitioning index ranges: a solve given a
// RootSep stops after classifying the root level and returns, for every
// eigenvalue item of every matrix in item order, the item's 1-based index j
// within its block, its matrix and block, and the relative separation
// reldist from the next item of the same block (+inf at the end of a block;
// the classification separates the two where it is >= gaptol).  W and Z are
// not touched.
struct RootSep {
    std::vector<int> j, matrix, block;
    std::vector<double> rel;
};

// binary32 input/output: working precision binary64 (mixed) or binary32 (plain)
int solve_batch_s_mixed(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats, RootSep* root_sep = nullptr);
int solve_batch_s_plain(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats, RootSep* root_sep = nullptr);
// binary64 input/output: working precision double-double (mixed) or binary64 (plain)
int solve_batch_d_mixed(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats, RootSep* root_sep = nullptr);
int solve_batch_d_plain(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats, RootSep* root_sep = nullptr);
}  // namespace mrrr
