// C ABI (include/mrrr.h): argument checks, host/device staging, parameter
// defaults, dispatch to the per-precision solvers.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "mrrr.h"
#include "mrrr_entry.h"
#include "mrrr_host.h"

namespace {

using mrrr::MatrixDesc;
using mrrr::SolveCfg;

// ---------------------------------------------------------------- memory pool

}  // namespace

namespace mrrr {

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
bool g_pool_ok[64];

cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ok[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        // a block freed on one stream is not handed to another stream by
        // making that stream wait for the first one: independent solves on
        // different streams must not be chained through the allocator
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        g_pool[dev] = pool;
        g_pool_ok[dev] = true;
    }
    return g_pool[dev];
}
}  // namespace

void* dev_alloc(size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = pool_for_current_device();
    void* p = nullptr;
    if (!pool || cudaMallocFromPoolAsync(&p, bytes ? bytes : 1, pool, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// Pinned host blocks for the solver's small readbacks and uploads, by
// power-of-two size class (>= 4 KiB), kept for reuse.
namespace {
std::mutex g_host_mu;
std::vector<std::pair<size_t, void*>> g_host_free;
size_t host_class(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
}
}  // namespace

void* host_alloc(size_t bytes, size_t* got) {
    const size_t c = host_class(bytes);
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        for (size_t i = 0; i < g_host_free.size(); ++i) {
            if (g_host_free[i].first == c) {
                void* p = g_host_free[i].second;
                g_host_free.erase(g_host_free.begin() + (long)i);
                *got = c;
                return p;
            }
        }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *got = c;
    return p;
}

void host_free(void* p, size_t got) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_host_mu);
    g_host_free.emplace_back(got, p);
}

namespace {
struct TuneState {
    int next = 0;                            // next candidate to try
    float ms[kRqiTuneCandidates] = {0, 0, 0};
    int reported = 0;                        // candidates with a time
    int chosen = -1;
};
std::mutex g_tune_mu;
std::unordered_map<unsigned, TuneState> g_tune;
}  // namespace

int rqi_tune_pick(unsigned key, int* trial) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneState& t = g_tune[key];
    if (t.chosen >= 0) {
        *trial = -1;
        return kRqiTuneWarps[t.chosen];
    }
    if (t.next < kRqiTuneCandidates) {
        *trial = t.next++;
        return kRqiTuneWarps[*trial];
    }
    // every candidate handed out, some still running: use the first meanwhile
    *trial = -1;
    return kRqiTuneWarps[0];
}

void rqi_tune_report(unsigned key, int trial, float ms) {
    if (trial < 0 || trial >= kRqiTuneCandidates) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneState& t = g_tune[key];
    t.ms[trial] = ms;
    if (++t.reported == kRqiTuneCandidates) {
        int best = 0;
        for (int c = 1; c < kRqiTuneCandidates; ++c)
            if (t.ms[c] < t.ms[best]) best = c;
        t.chosen = best;
    }
}

}  // namespace mrrr

namespace {

using mrrr::classify_ptr;
using mrrr::make_cfg;
using mrrr::PTR_DEVICE;
using mrrr::PTR_HOST;
using mrrr::PTR_OTHER_DEVICE;

struct DevBuf {
    void* p = nullptr;
    cudaStream_t st;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    bool alloc(size_t bytes) { return (p = mrrr::dev_alloc(bytes, st)) != nullptr; }
    ~DevBuf() {
        mrrr::dev_free(p, st);
    }
};

template <class X>
int solve_one(int n, const X* d, const X* e, mrrr_range range, X vl, X vu, int il, int iu, mrrr_mode mode,
              const mrrr_params* prm, int* m_out, X* W, X* Z, int ldz, void* stream) {
    const bool xs = std::is_same<X, float>::value;
    if (m_out) *m_out = 0;
    if (n < 0 || (mode != MRRR_PLAIN && mode != MRRR_MIXED)) return MRRR_ERR_ARG;
    if (range != MRRR_ALL && range != MRRR_INDEX && range != MRRR_VALUE) return MRRR_ERR_ARG;
    if (n == 0) return MRRR_OK;
    if (!d || (n > 1 && !e) || !W || !Z || ldz < n) return MRRR_ERR_ARG;
    if (range == MRRR_INDEX && (il < 1 || iu > n || il > iu)) return MRRR_ERR_ARG;
    if (range == MRRR_VALUE && !(vl < vu)) return MRRR_ERR_ARG;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int kmax = range == MRRR_INDEX ? iu - il + 1 : n;
    // stage host buffers through device memory
    DevBuf bd(st), be(st), bw(st), bz(st);
    const X* dd_ = d;
    const X* de_ = e;
    X* dW = W;
    X* dZ = Z;
    int dldz = ldz;
    static const X zero1[1] = {X(0)};
    if (n == 1) e = zero1;
    const mrrr::PtrKind kd = classify_ptr(d), ke = n > 1 ? classify_ptr(e) : PTR_HOST;
    const mrrr::PtrKind kw = classify_ptr(W), kz = classify_ptr(Z);
    if (kd == PTR_OTHER_DEVICE || ke == PTR_OTHER_DEVICE || kw == PTR_OTHER_DEVICE || kz == PTR_OTHER_DEVICE)
        return MRRR_ERR_ARG;
    if (kd == PTR_HOST) {
        if (!bd.alloc(sizeof(X) * n)) return MRRR_ERR_NOMEM;
        if (cudaMemcpyAsync(bd.p, d, sizeof(X) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) return MRRR_ERR_CUDA;
        dd_ = (const X*)bd.p;
    }
    if (ke == PTR_HOST) {
        size_t ne = n > 1 ? (size_t)(n - 1) : 1;
        if (!be.alloc(sizeof(X) * ne)) return MRRR_ERR_NOMEM;
        if (cudaMemcpyAsync(be.p, e, sizeof(X) * ne, cudaMemcpyHostToDevice, st) != cudaSuccess) return MRRR_ERR_CUDA;
        de_ = (const X*)be.p;
    }
    const bool hostW = kw == PTR_HOST, hostZ = kz == PTR_HOST;
    if (hostW) {
        if (!bw.alloc(sizeof(X) * kmax)) return MRRR_ERR_NOMEM;
        dW = (X*)bw.p;
    }
    if (hostZ) {
        if (!bz.alloc(sizeof(X) * (size_t)n * kmax)) return MRRR_ERR_NOMEM;
        dZ = (X*)bz.p;
        dldz = n;
    }
    MatrixDesc M;
    memset(&M, 0, sizeof(M));
    M.d = dd_;
    M.e = de_;
    M.W = dW;
    M.Z = dZ;
    M.ldz = dldz;
    M.n = n;
    M.range = (int)range;
    M.vl = (double)vl;
    M.vu = (double)vu;
    M.il = il;
    M.iu = iu;
    SolveCfg cfg = make_cfg(xs, mode == MRRR_MIXED, prm);
    int max_depth = (prm && prm->max_depth > 0) ? prm->max_depth : 16;
    mrrr_stats* stats = prm ? prm->stats : nullptr;
    if (stats) memset(stats, 0, sizeof(*stats));
    int rc;
    if (xs) {
        rc = mode == MRRR_MIXED ? mrrr::solve_batch_s_mixed(1, &M, cfg, max_depth, st, stats)
                                : mrrr::solve_batch_s_plain(1, &M, cfg, max_depth, st, stats);
    } else {
        rc = mode == MRRR_MIXED ? mrrr::solve_batch_d_mixed(1, &M, cfg, max_depth, st, stats)
                                : mrrr::solve_batch_d_plain(1, &M, cfg, max_depth, st, stats);
    }
    if (rc != MRRR_OK && rc != MRRR_ERR_NOCONV) return rc;
    const int k = M.kout;
    if (k > 0 && hostW) {
        if (cudaMemcpyAsync(W, dW, sizeof(X) * k, cudaMemcpyDeviceToHost, st) != cudaSuccess) return MRRR_ERR_CUDA;
    }
    if (k > 0 && hostZ) {
        if (cudaMemcpy2DAsync(Z, sizeof(X) * (size_t)ldz, dZ, sizeof(X) * (size_t)n, sizeof(X) * (size_t)n, k,
                              cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return MRRR_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return MRRR_ERR_CUDA;
    if (m_out) *m_out = k;
    return rc;
}

// Byte offsets of the host-side buffers of a batch inside one staging block
// of device memory (each 256-byte aligned).
struct Staged {
    size_t d = SIZE_MAX, e = SIZE_MAX, W = SIZE_MAX, Z = SIZE_MAX;
};

template <class X>
int solve_many(int nb, const int* n, const X* const* d, const X* const* e, const int* il, const int* iu,
               mrrr_mode mode, const mrrr_params* prm, int* m_out, X* const* W, X* const* Z, const int* ldz,
               int* status, void* stream) {
    const bool xs = std::is_same<X, float>::value;
    if (nb < 0 || (nb > 0 && (!n || !d || !W || !Z || !ldz || !status))) return MRRR_ERR_ARG;
    if (mode != MRRR_PLAIN && mode != MRRR_MIXED) return MRRR_ERR_ARG;
    if ((il == nullptr) != (iu == nullptr)) return MRRR_ERR_ARG;
    if (nb == 0) return MRRR_OK;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    std::vector<MatrixDesc> mats;
    std::vector<int> map;  // mats index -> batch index
    std::vector<Staged> staged;
    static const X zero1[1] = {X(0)};
    X* dzero = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    size_t stage_bytes = 0;
    auto take = [&](size_t bytes) {
        size_t off = stage_bytes;
        stage_bytes += (bytes + 255) / 256 * 256;
        return off;
    };
    for (int p = 0; p < nb; ++p) {
        status[p] = MRRR_OK;
        if (m_out) m_out[p] = 0;
        if (n[p] < 0 || (n[p] > 0 && (ldz[p] < n[p] || !d[p] || !W[p] || !Z[p] || (n[p] > 1 && (!e || !e[p]))))) {
            status[p] = MRRR_ERR_ARG;
            continue;
        }
        if (il && (il[p] < 1 || iu[p] > n[p] || il[p] > iu[p])) {
            status[p] = MRRR_ERR_ARG;
            continue;
        }
        if (n[p] == 0) continue;
        // host buffers are staged through one block of device memory; device
        // buffers of another device are an argument error
        const mrrr::PtrKind kd = classify_ptr(d[p]), ke = n[p] > 1 ? classify_ptr(e[p]) : PTR_DEVICE;
        const mrrr::PtrKind kw = classify_ptr(W[p]), kz = classify_ptr(Z[p]);
        if (kd == PTR_OTHER_DEVICE || ke == PTR_OTHER_DEVICE || kw == PTR_OTHER_DEVICE || kz == PTR_OTHER_DEVICE) {
            status[p] = MRRR_ERR_ARG;
            continue;
        }
        const size_t np = (size_t)n[p];
        const size_t kp = il ? (size_t)(iu[p] - il[p] + 1) : np;
        Staged sg;
        if (kd == PTR_HOST) sg.d = take(sizeof(X) * np);
        if (ke == PTR_HOST) sg.e = take(sizeof(X) * (np - 1));
        if (kw == PTR_HOST) sg.W = take(sizeof(X) * kp);
        if (kz == PTR_HOST) sg.Z = take(sizeof(X) * np * kp);
        MatrixDesc M;
        memset(&M, 0, sizeof(M));
        M.d = d[p];
        M.e = (e && n[p] > 1) ? (const void*)e[p] : nullptr;
        M.W = W[p];
        M.Z = Z[p];
        M.ldz = ldz[p];
        M.n = n[p];
        M.range = il ? MRRR_INDEX : MRRR_ALL;
        M.il = il ? il[p] : 1;
        M.iu = il ? iu[p] : n[p];
        mats.push_back(M);
        map.push_back(p);
        staged.push_back(sg);
    }
    int rc = MRRR_OK;
    DevBuf stage(st);
    if (stage_bytes > 0 && !stage.alloc(stage_bytes)) return MRRR_ERR_NOMEM;
    char* sbase = (char*)stage.p;
    for (size_t q = 0; q < mats.size(); ++q) {
        MatrixDesc& M = mats[q];
        const Staged& sg = staged[q];
        const size_t np = (size_t)M.n;
        if (sg.d != SIZE_MAX) {
            if (cudaMemcpyAsync(sbase + sg.d, M.d, sizeof(X) * np, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return MRRR_ERR_CUDA;
            M.d = sbase + sg.d;
        }
        if (sg.e != SIZE_MAX) {
            if (cudaMemcpyAsync(sbase + sg.e, M.e, sizeof(X) * (np - 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return MRRR_ERR_CUDA;
            M.e = sbase + sg.e;
        }
        if (sg.W != SIZE_MAX) M.W = sbase + sg.W;
        if (sg.Z != SIZE_MAX) {
            M.Z = sbase + sg.Z;
            M.ldz = M.n;
        }
        if (M.n == 1 || !M.e) {
            if (!dzero) {
                if (!(dzero = (X*)mrrr::dev_alloc(sizeof(X), st))) return MRRR_ERR_NOMEM;
                if (cudaMemcpyAsync(dzero, zero1, sizeof(X), cudaMemcpyHostToDevice, st) != cudaSuccess)
                    return MRRR_ERR_CUDA;
            }
            M.e = dzero;
        }
    }
    if (!mats.empty()) {
        SolveCfg cfg = make_cfg(xs, mode == MRRR_MIXED, prm);
        int max_depth = (prm && prm->max_depth > 0) ? prm->max_depth : 16;
        mrrr_stats* stats = prm ? prm->stats : nullptr;
        if (stats) memset(stats, 0, sizeof(*stats));
        int P = (int)mats.size();
        if (xs)
            rc = mode == MRRR_MIXED ? mrrr::solve_batch_s_mixed(P, mats.data(), cfg, max_depth, st, stats)
                                    : mrrr::solve_batch_s_plain(P, mats.data(), cfg, max_depth, st, stats);
        else
            rc = mode == MRRR_MIXED ? mrrr::solve_batch_d_mixed(P, mats.data(), cfg, max_depth, st, stats)
                                    : mrrr::solve_batch_d_plain(P, mats.data(), cfg, max_depth, st, stats);
        for (int q = 0; q < P; ++q) {
            int p = map[q];
            int sp = mats[q].status;
            status[p] = sp == mrrr::ST_ERR_NONFINITE ? MRRR_ERR_NONFINITE
                        : sp == mrrr::ST_ERR_NOCONV  ? MRRR_ERR_NOCONV
                                                     : (rc == MRRR_OK || rc == MRRR_ERR_NOCONV ? MRRR_OK : rc);
            if (m_out) m_out[p] = mats[q].kout;
        }
        // results of host outputs back from the staging block
        if (rc == MRRR_OK || rc == MRRR_ERR_NOCONV) {
            for (int q = 0; q < P; ++q) {
                const MatrixDesc& M = mats[q];
                const Staged& sg = staged[q];
                const int p = map[q];
                const int k = M.kout;
                if (k <= 0) continue;
                if (sg.W != SIZE_MAX &&
                    cudaMemcpyAsync(W[p], M.W, sizeof(X) * (size_t)k, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    return MRRR_ERR_CUDA;
                if (sg.Z != SIZE_MAX &&
                    cudaMemcpy2DAsync(Z[p], sizeof(X) * (size_t)ldz[p], M.Z, sizeof(X) * (size_t)M.n,
                                      sizeof(X) * (size_t)M.n, k, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    return MRRR_ERR_CUDA;
            }
        }
    }
    mrrr::dev_free(dzero, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MRRR_ERR_CUDA;
    if (rc != MRRR_OK && rc != MRRR_ERR_NOCONV) return rc;
    for (int p = 0; p < nb; ++p)
        if (status[p] != MRRR_OK) return status[p];
    return MRRR_OK;
}

// Index partition of one tridiagonal for nparts independent solves (Sec. 2,
// classification; the multi-GPU split of the wanted index range): parts are
// contiguous index ranges whose boundaries lie where the root classification
// separates consecutive eigenvalues, so that no cluster -- and no child
// representation -- is shared by two parts.  For each interior target
// t_p = round(p n / nparts) the root classification of a window of indices
// around t_p is computed (one batched solve stopped after the root level,
// each window an index range of the same matrix), and the boundary is put
// after the index j nearest to t_p whose separation from j + 1 is at least
// kCutMargin gaptol, considering only pairs whose own neighbours lie in the
// window (their brackets are then those of a full solve).  Windows without
// such a pair grow fourfold until they cover the matrix; a matrix that
// splits into blocks is cut evenly (its blocks are independent).
constexpr double kCutMargin = 4.0;

template <class X>
int partition_one(int n, const X* d, const X* e, mrrr_mode mode, const mrrr_params* prm, int nparts, int* il,
                  int* iu, void* stream) {
    const bool xs = std::is_same<X, float>::value;
    if (n < 0 || nparts < 1 || !il || !iu || (mode != MRRR_PLAIN && mode != MRRR_MIXED)) return MRRR_ERR_ARG;
    if (n > 0 && (!d || (n > 1 && !e))) return MRRR_ERR_ARG;
    // even split first: the answer for small or split matrices
    std::vector<int> cut(nparts + 1);
    for (int p = 0; p <= nparts; ++p) cut[p] = (int)(((long long)n * p + nparts / 2) / nparts);
    auto emit = [&]() {
        for (int p = 0; p < nparts; ++p) {
            il[p] = cut[p] + 1;
            iu[p] = cut[p + 1];
        }
        return MRRR_OK;
    };
    if (nparts == 1 || n <= 2) return emit();
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const mrrr::PtrKind kd = classify_ptr(d), ke = classify_ptr(e);
    if (kd == PTR_OTHER_DEVICE || ke == PTR_OTHER_DEVICE) return MRRR_ERR_ARG;
    DevBuf bd(st), be(st), bdummy(st);
    const X* dd_ = d;
    const X* de_ = e;
    if (kd == PTR_HOST) {
        if (!bd.alloc(sizeof(X) * n)) return MRRR_ERR_NOMEM;
        if (cudaMemcpyAsync(bd.p, d, sizeof(X) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) return MRRR_ERR_CUDA;
        dd_ = (const X*)bd.p;
    }
    if (ke == PTR_HOST) {
        if (!be.alloc(sizeof(X) * (n - 1))) return MRRR_ERR_NOMEM;
        if (cudaMemcpyAsync(be.p, e, sizeof(X) * (n - 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return MRRR_ERR_CUDA;
        de_ = (const X*)be.p;
    }
    if (!bdummy.alloc(256)) return MRRR_ERR_NOMEM;  // W and Z are never written by a root-only solve
    SolveCfg cfg = make_cfg(xs, mode == MRRR_MIXED, prm);
    const double need = kCutMargin * cfg.gaptol;
    std::vector<int> todo;  // interior targets still without a cut
    for (int p = 1; p < nparts; ++p) todo.push_back(p);
    std::vector<int> half(nparts, 32);
    while (!todo.empty()) {
        std::vector<MatrixDesc> mats;
        for (int p : todo) {
            MatrixDesc M;
            memset(&M, 0, sizeof(M));
            M.d = dd_;
            M.e = de_;
            M.W = bdummy.p;
            M.Z = bdummy.p;
            M.ldz = n;
            M.n = n;
            M.range = MRRR_INDEX;
            M.il = std::max(1, cut[p] - half[p]);
            M.iu = std::min(n, cut[p] + half[p]);
            mats.push_back(M);
        }
        mrrr::RootSep rs;
        const int P = (int)mats.size();
        int rc;
        if (xs)
            rc = mode == MRRR_MIXED ? mrrr::solve_batch_s_mixed(P, mats.data(), cfg, 16, st, nullptr, &rs)
                                    : mrrr::solve_batch_s_plain(P, mats.data(), cfg, 16, st, nullptr, &rs);
        else
            rc = mode == MRRR_MIXED ? mrrr::solve_batch_d_mixed(P, mats.data(), cfg, 16, st, nullptr, &rs)
                                    : mrrr::solve_batch_d_plain(P, mats.data(), cfg, 16, st, nullptr, &rs);
        if (rc != MRRR_OK) return rc;
        for (int q = 0; q < P; ++q)
            if (mats[q].status == mrrr::ST_ERR_NONFINITE) return MRRR_ERR_NONFINITE;
        if (mats[0].nblocks > 1) break;  // blocks are independent: the even split stands
        std::vector<int> next;
        for (int q = 0; q < P; ++q) {
            const int p = todo[q];
            // items of window q, in index order (one block)
            int best = -1;
            long long bestd = 0;
            const int K = (int)rs.j.size();
            for (int t = 1; t + 2 < K; ++t) {
                if (rs.matrix[t] != q || rs.matrix[t - 1] != q || rs.matrix[t + 2] != q) continue;
                if (!(rs.rel[t] >= need)) continue;
                const long long dist = std::llabs((long long)rs.j[t] - cut[p]);
                if (best < 0 || dist < bestd) {
                    best = rs.j[t];
                    bestd = dist;
                }
            }
            if (best >= 0) {
                cut[p] = best;
            } else if (2 * half[p] < n) {
                half[p] *= 4;
                next.push_back(p);
            } else {
                cut[p] = -1;  // no separated pair anywhere: this boundary merges with a neighbour
            }
        }
        todo.swap(next);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return MRRR_ERR_CUDA;
    // boundaries without a cut, or out of order, collapse onto the previous one
    cut[0] = 0;
    cut[nparts] = n;
    for (int p = 1; p < nparts; ++p)
        if (cut[p] < cut[p - 1]) cut[p] = cut[p - 1];
    for (int p = nparts - 1; p >= 1; --p)
        if (cut[p] > cut[p + 1]) cut[p] = cut[p + 1];
    return emit();
}

}  // namespace

extern "C" {

int mrrr_partition_s(int n, const float* d, const float* e, mrrr_mode mode, const mrrr_params* params, int nparts,
                     int* il, int* iu, void* stream) {
    return partition_one<float>(n, d, e, mode, params, nparts, il, iu, stream);
}

int mrrr_partition_d(int n, const double* d, const double* e, mrrr_mode mode, const mrrr_params* params,
                     int nparts, int* il, int* iu, void* stream) {
    return partition_one<double>(n, d, e, mode, params, nparts, il, iu, stream);
}


int mrrr_solve_batch_s(int nb, const int* n, const float* const* d, const float* const* e, const int* il,
                       const int* iu, mrrr_mode mode, const mrrr_params* params, int* m_out, float* const* W,
                       float* const* Z, const int* ldz, int* status, void* stream) {
    return solve_many<float>(nb, n, d, e, il, iu, mode, params, m_out, W, Z, ldz, status, stream);
}

int mrrr_solve_batch_d(int nb, const int* n, const double* const* d, const double* const* e, const int* il,
                       const int* iu, mrrr_mode mode, const mrrr_params* params, int* m_out, double* const* W,
                       double* const* Z, const int* ldz, int* status, void* stream) {
    return solve_many<double>(nb, n, d, e, il, iu, mode, params, m_out, W, Z, ldz, status, stream);
}


int mrrr_solve_s(int n, const float* d, const float* e, mrrr_range range, float vl, float vu, int il, int iu,
                 mrrr_mode mode, const mrrr_params* params, int* m_out, float* W, float* Z, int ldz, void* stream) {
    return solve_one<float>(n, d, e, range, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream);
}

int mrrr_solve_d(int n, const double* d, const double* e, mrrr_range range, double vl, double vu, int il, int iu,
                 mrrr_mode mode, const mrrr_params* params, int* m_out, double* W, double* Z, int ldz,
                 void* stream) {
    return solve_one<double>(n, d, e, range, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream);
}

const char* mrrr_strerror(int status) {
    switch (status) {
        case MRRR_OK: return "success";
        case MRRR_ERR_ARG: return "invalid argument";
        case MRRR_ERR_NONFINITE: return "non-finite value in the input";
        case MRRR_ERR_NOCONV: return "an eigenpair did not meet its stopping criterion";
        case MRRR_ERR_NOMEM: return "device memory allocation failed";
        case MRRR_ERR_CUDA: return "CUDA runtime error or no CUDA device";
        case MRRR_ERR_TIMEOUT: return "a bounded device-side wait ran out";
        case MRRR_ERR_NOREP: return "no candidate representation passed the acceptance test";
        case MRRR_ERR_CANCELLED: return "the request was cancelled before it ran";
        default: return "unknown status";
    }
}

const char* mrrr_version(void) { return "mrrr-gb300 0.1 (sm_103a)"; }

}  // extern "C"
