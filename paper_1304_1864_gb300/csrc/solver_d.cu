// binary64 input/output instantiations of the solver.
#include "mrrr_entry.h"
#include "mrrr_solver.cuh"

namespace mrrr {
int solve_batch_d_mixed(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats, RootSep* root_sep) {
    return solve_batch<double, dd>(P, mats, cfg, max_depth, st, stats, root_sep);
}
int solve_batch_d_plain(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                        mrrr_stats* stats, RootSep* root_sep) {
    return solve_batch<double, double>(P, mats, cfg, max_depth, st, stats, root_sep);
}
}  // namespace mrrr
