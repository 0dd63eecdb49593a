// Kernels and host driver of the solver.  Every step of Algorithm 1 runs in
// a kernel below; the host only sizes allocations and launches from the
// counts the kernels report (one small device-to-host read per tree level).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mrrr.h"
#include "mrrr_phases.cuh"

namespace mrrr {

constexpr int kThreads = 128;

inline int grid_for(long long n, int threads = kThreads) { return (int)((n + threads - 1) / threads); }

// ------------------------------------------------------------------ kernels

template <class X>
__global__ void k_prep(MatrixDesc* mats, BlockDesc* blocks, double* wd, double* we, SolveCfg cfg) {
    int p = blockIdx.x;
    if (threadIdx.x != 0) return;
    MatrixDesc& M = mats[p];
    prep_matrix<X>(M, blocks, wd, we, cfg);
    for (int b = 0; b < M.nblocks; ++b) blocks[M.row0 + b].matrix = p;
}

template <class Y>
__global__ void k_root(const int* blist, int nb, BlockDesc* blocks, const MatrixDesc* mats, const double* wd,
                       const double* we, Y* reps, SolveCfg cfg) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    BlockDesc& B = blocks[blist[t]];
    root_block<Y>(B, mats[B.matrix], wd, we, reps, cfg);
}

// Exclusive scan of the item counts over the block list (one CTA), plus the
// per-matrix totals: item range, number of returned eigenpairs.
static __global__ void k_scan_items(const int* blist, int nb, BlockDesc* blocks, MatrixDesc* mats, int nmat,
                             int* total_out) {
    __shared__ int part[1024];
    const int T = blockDim.x;
    int per = (nb + T - 1) / T;
    int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += blocks[blist[b]].nitems;
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < T; ++i) {
            int v = part[i];
            part[i] = acc;
            acc += v;
        }
        *total_out = acc;
    }
    __syncthreads();
    int off = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        BlockDesc& B = blocks[blist[b]];
        B.item0 = off;
        off += B.nitems;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nmat; p += T) {
        MatrixDesc& M = mats[p];
        int item0 = -1, nit = 0, kout = 0;
        for (int b = 0; b < M.nblocks; ++b) {
            const BlockDesc& B = blocks[M.row0 + b];
            if (item0 < 0 && B.nitems > 0) item0 = B.item0;
            nit += B.nitems;
            if (B.w_hi >= B.w_lo) kout += B.w_hi - B.w_lo + 1;
        }
        if (M.range == RANGE_INDEX && M.nblocks > 0) kout = M.iu - M.il + 1;
        M.item0 = item0 < 0 ? 0 : item0;
        M.nitems = nit;
        M.kout = M.nblocks > 0 ? kout : 0;
    }
}

template <class Y>
__global__ void k_init_items(const int* blist, int nb, const BlockDesc* blocks, Item* items, const Y* reps) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    init_block_items<Y>(blocks[blist[t]], blist[t], items, reps);
}

template <class Y>
__global__ void k_bisect(Item* items, const int* list, int count, const BlockDesc* blocks, double rtol,
                         int verify, unsigned long long* step_counter) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int it = list ? list[t] : t;
    Item& I = items[it];
    unsigned long long steps = 0;
    bisect_item<Y>(I, blocks[I.block].pivmin, rtol, verify, 200, &steps);
    atomicAdd(step_counter, steps);
}

static __global__ void k_assign_cols(Item* items, int count, const MatrixDesc* mats, const BlockDesc* blocks) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    assign_col(t, items, mats, blocks);
}

static __global__ void k_classify_blocks(const int* blist, int nb, const BlockDesc* blocks, Item* items, double gaptol,
                                  int* single_list, Cluster* clusters, int* member_list, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const BlockDesc& B = blocks[blist[t]];
    if (B.nitems == 0) return;
    classify_group(B.item0, B.item0 + B.nitems, items, gaptol, single_list, clusters, member_list, C);
}

static __global__ void k_classify_clusters(const Cluster* groups, int ng, Item* items, double gaptol, int* single_list,
                                    Cluster* clusters, int* member_list, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ng) return;
    classify_group(groups[t].a, groups[t].b, items, gaptol, single_list, clusters, member_list, C);
}

template <class Y>
__global__ void k_shift(const Cluster* clusters, int nc, Item* items, const BlockDesc* blocks, Y* pool,
                        SolveCfg cfg, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    shift_cluster<Y>(clusters[t], items, blocks, pool, cfg, C);
}

template <class X, class Y>
__global__ void k_rqi(Item* items, const int* list, int count, MatrixDesc* mats, const BlockDesc* blocks,
                      SolveCfg cfg, Y* scratch, int nmax, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    Item& I = items[list[t]];
    Scratch<Y> Wk;
    Y* base = scratch + (size_t)(t >> 5) * (size_t)(2 * nmax) * 32 + (t & 31);
    Wk.a = base;
    Wk.b = base + (size_t)nmax * 32;
    Wk.stride = 32;
    rqi_item<X, Y>(I, mats, blocks, cfg, Wk, C);
}

template <class X>
__global__ void k_sort_fix(MatrixDesc* mats, int nmat) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nmat) return;
    if (mats[p].nblocks > 1) sort_fix_matrix<X>(mats[p]);
}

// ------------------------------------------------------------------ host driver

// Stream-ordered allocations released together at the end of a solve.
struct Arena {
    cudaStream_t st;
    std::vector<void*> ptrs;
    bool failed = false;
    explicit Arena(cudaStream_t s) : st(s) {}
    template <class T> T* alloc(size_t count) {
        void* p = nullptr;
        size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            failed = true;
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return (T*)p;
    }
    ~Arena() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

#define MRRR_CK(call)                                  \
    do {                                               \
        cudaError_t err__ = (call);                    \
        if (err__ != cudaSuccess) return MRRR_ERR_CUDA; \
    } while (0)

#define MRRR_ALLOC(var, T, count)                       \
    T* var = arena.alloc<T>(count);                     \
    if (!var) return MRRR_ERR_NOMEM

// Optional per-phase device timing with CUDA events on the solve's stream.
struct Timeline {
    bool on;
    cudaStream_t st;
    struct Rec {
        int phase, launches;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    cudaEvent_t cur_a = nullptr;
    int cur = -1;
    Timeline(bool enabled, cudaStream_t s) : on(enabled), st(s) {}
    void begin(int phase) {
        if (!on) return;
        cudaEventCreate(&cur_a);
        cudaEventRecord(cur_a, st);
        cur = phase;
    }
    void end(int launches = 1) {
        if (!on) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, st);
        recs.push_back({cur, launches, cur_a, b});
    }
    void collect(mrrr_stats* s) {
        for (Rec& r : recs) {
            float ms = 0.f;
            if (s && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                s->phase_ms[r.phase] += ms;
                s->phase_launches[r.phase] += r.launches;
            }
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        recs.clear();
        if (s) s->timed = on ? 1 : 0;
    }
    ~Timeline() { collect(nullptr); }
};

template <class Y> struct ScratchBudget {
    static size_t bytes() { return (size_t)4 << 30; }  // 4 GiB of RQI scratch per wave
};

// Solve a batch of independent tridiagonals (a single solve is a batch of
// one).  mats[p] carries the input/output device pointers, n, ldz and range;
// the remaining fields are filled in.  Returns 0 or a negative status; the
// per-matrix status and count are left in mats[p].status / mats[p].kout.
template <class X, class Y>
int solve_batch(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                mrrr_stats* stats) {
    long long N = 0;
    int nmax = 1;
    for (int p = 0; p < P; ++p) {
        mats[p].row0 = (int)N;
        mats[p].status = ST_OK;
        mats[p].nblocks = 0;
        mats[p].kout = 0;
        N += mats[p].n;
        nmax = std::max(nmax, mats[p].n);
    }
    if (N > (1LL << 30) / 4) return MRRR_ERR_ARG;
    Arena arena(st);
    Timeline tl(stats && (cfg.flags & MRRR_FLAG_TIMING), st);
    MRRR_ALLOC(d_mats, MatrixDesc, P);
    MRRR_ALLOC(d_blocks, BlockDesc, N);
    MRRR_ALLOC(wd, double, N);
    MRRR_ALLOC(we, double, N);
    MRRR_ALLOC(reps, Y, 4 * N);
    MRRR_ALLOC(d_C, DevCounters, 1);
    MRRR_ALLOC(d_total, int, 1);
    MRRR_CK(cudaMemsetAsync(d_C, 0, sizeof(DevCounters), st));
    MRRR_CK(cudaMemcpyAsync(d_mats, mats, sizeof(MatrixDesc) * P, cudaMemcpyHostToDevice, st));

    // a1: scale + split
    tl.begin(MRRR_PHASE_PREP);
    k_prep<X><<<P, 32, 0, st>>>(d_mats, d_blocks, wd, we, cfg);
    tl.end();
    MRRR_CK(cudaGetLastError());
    MRRR_CK(cudaMemcpyAsync(mats, d_mats, sizeof(MatrixDesc) * P, cudaMemcpyDeviceToHost, st));
    MRRR_CK(cudaStreamSynchronize(st));
    std::vector<int> blist;
    for (int p = 0; p < P; ++p)
        for (int b = 0; b < mats[p].nblocks; ++b) blist.push_back(mats[p].row0 + b);
    const int NB = (int)blist.size();
    DevCounters C{};
    if (NB > 0) {
        MRRR_ALLOC(d_blist, int, NB);
        MRRR_CK(cudaMemcpyAsync(d_blist, blist.data(), sizeof(int) * NB, cudaMemcpyHostToDevice, st));
        // a2: root representations
        tl.begin(MRRR_PHASE_ROOT);
        k_root<Y><<<grid_for(NB), kThreads, 0, st>>>(d_blist, NB, d_blocks, d_mats, wd, we, reps, cfg);
        k_scan_items<<<1, 1024, 0, st>>>(d_blist, NB, d_blocks, d_mats, P, d_total);
        tl.end(2);
        MRRR_CK(cudaGetLastError());
        int K = 0;
        MRRR_CK(cudaMemcpyAsync(&K, d_total, sizeof(int), cudaMemcpyDeviceToHost, st));
        MRRR_CK(cudaMemcpyAsync(mats, d_mats, sizeof(MatrixDesc) * P, cudaMemcpyDeviceToHost, st));
        MRRR_CK(cudaStreamSynchronize(st));
        if (K > 0) {
            MRRR_ALLOC(items, Item, K);
            MRRR_ALLOC(single_list, int, K);
            MRRR_ALLOC(member_list, int, K);
            MRRR_ALLOC(clus_a, Cluster, K / 2 + 1);
            MRRR_ALLOC(clus_b, Cluster, K / 2 + 1);
            tl.begin(MRRR_PHASE_ROOT);
            k_init_items<Y><<<grid_for(NB), kThreads, 0, st>>>(d_blist, NB, d_blocks, items, reps);
            tl.end();
            // eigenvector columns of a split matrix are zero outside their block
            tl.begin(MRRR_PHASE_FINISH);
            int nz = 0;
            for (int p = 0; p < P; ++p) {
                if (mats[p].nblocks > 1 && mats[p].kout > 0) {
                    MRRR_CK(cudaMemset2DAsync(mats[p].Z, sizeof(X) * (size_t)mats[p].ldz, 0,
                                              sizeof(X) * (size_t)mats[p].n, mats[p].kout, st));
                    ++nz;
                }
            }
            tl.end(nz);
            // a3: initial eigenvalues by bisection on the root reps
            tl.begin(MRRR_PHASE_BISECT);
            k_bisect<Y><<<grid_for(K), kThreads, 0, st>>>(items, nullptr, K, d_blocks, cfg.rtol_class, 0,
                                                          &d_C->qd_bisect);
            tl.end();
            tl.begin(MRRR_PHASE_CLASSIFY);
            k_assign_cols<<<grid_for(K), kThreads, 0, st>>>(items, K, d_mats, d_blocks);
            tl.end();
            MRRR_CK(cudaGetLastError());
            // a4/a5: classification and the representation tree, level by level
            Cluster* groups = nullptr;
            int ngroups = 0;
            for (int level = 0;; ++level) {
                Cluster* out = (level % 2 == 0) ? clus_a : clus_b;
                MRRR_CK(cudaMemsetAsync(&d_C->pool_need, 0, sizeof(unsigned long long), st));
                MRRR_CK(cudaMemsetAsync(&d_C->ncluster, 0, 2 * sizeof(int), st));  // ncluster, nmember
                bool force = level >= max_depth;
                double gt = force ? -INFINITY : cfg.gaptol;
                tl.begin(MRRR_PHASE_CLASSIFY);
                if (level == 0)
                    k_classify_blocks<<<grid_for(NB), kThreads, 0, st>>>(d_blist, NB, d_blocks, items, gt,
                                                                         single_list, out, member_list, d_C);
                else
                    k_classify_clusters<<<grid_for(ngroups), kThreads, 0, st>>>(groups, ngroups, items, gt,
                                                                                single_list, out, member_list, d_C);
                tl.end();
                MRRR_CK(cudaGetLastError());
                MRRR_CK(cudaMemcpyAsync(&C, d_C, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
                MRRR_CK(cudaStreamSynchronize(st));
                if (C.ncluster == 0) break;
                MRRR_ALLOC(pool, Y, (size_t)C.pool_need);
                tl.begin(MRRR_PHASE_SHIFT);
                k_shift<Y><<<grid_for(C.ncluster), kThreads, 0, st>>>(out, C.ncluster, items, d_blocks, pool, cfg, d_C);
                tl.end();
                tl.begin(MRRR_PHASE_REFINE);
                k_bisect<Y><<<grid_for(C.nmember), kThreads, 0, st>>>(items, member_list, C.nmember, d_blocks,
                                                                      cfg.rtol_class, 1, &d_C->qd_refine);
                tl.end();
                MRRR_CK(cudaGetLastError());
                groups = out;
                ngroups = C.ncluster;
            }
            // a6/a7: RQI for every singleton, in waves bounded by the scratch budget
            const int S = C.nsingle;
            if (S > 0) {
                size_t per = 2 * (size_t)nmax * sizeof(Y);
                long long wave = (long long)(ScratchBudget<Y>::bytes() / per);
                wave = std::max<long long>(32, wave / 32 * 32);
                wave = std::min<long long>(wave, ((long long)S + 31) / 32 * 32);
                MRRR_ALLOC(scratch, Y, (size_t)wave * 2 * nmax);
                for (long long s0 = 0; s0 < S; s0 += wave) {
                    int cnt = (int)std::min<long long>(wave, S - s0);
                    tl.begin(MRRR_PHASE_RQI);
                    k_rqi<X, Y><<<grid_for(cnt), kThreads, 0, st>>>(items, single_list + s0, cnt, d_mats, d_blocks,
                                                                    cfg, scratch, nmax, d_C);
                    tl.end();
                    MRRR_CK(cudaGetLastError());
                }
            }
            tl.begin(MRRR_PHASE_FINISH);
            k_sort_fix<X><<<grid_for(P, 32), 32, 0, st>>>(d_mats, P);
            tl.end();
            MRRR_CK(cudaGetLastError());
        }
    }
    MRRR_CK(cudaMemcpyAsync(&C, d_C, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    MRRR_CK(cudaMemcpyAsync(mats, d_mats, sizeof(MatrixDesc) * P, cudaMemcpyDeviceToHost, st));
    MRRR_CK(cudaStreamSynchronize(st));
    int rc = 0;
    for (int p = 0; p < P && rc == 0; ++p) {
        if (mats[p].status == ST_ERR_NONFINITE) rc = MRRR_ERR_NONFINITE;
    }
    if (rc == 0 && C.noconv > 0) rc = MRRR_ERR_NOCONV;
    if (stats) {
        stats->nblocks = NB;
        stats->d_max = C.d_max;
        stats->nclusters = C.nclusters_total;
        stats->largest_cluster = C.largest_cluster;
        stats->reps_failed = C.reps_failed;
        stats->rqi_iters = C.rqi_iters;
        stats->fallbacks = C.fallbacks;
        stats->noconv = C.noconv;
        stats->qd_bisect = (long long)C.qd_bisect;
        stats->qd_refine = (long long)C.qd_refine;
        stats->qd_rqi = (long long)C.qd_rqi;
        stats->qd_shift = (long long)C.qd_shift;
        stats->qd_low = (long long)C.qd_steps_low;
        tl.collect(stats);
    }
    if (arena.failed) return MRRR_ERR_NOMEM;
    return rc;
}

}  // namespace mrrr
