// Eigenvectors for given eigenvalues with no device allocation at all: a
// variant of the RQI kernel whose scratch lives in one file-scope device array
// (see mrrr_eigvecs_noalloc_s in include/mrrr.h).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "mrrr.h"
#include "mrrr_host.h"
#include "mrrr_phases.cuh"

namespace {

using namespace mrrr;

constexpr int kMaxN = MRRR_NOALLOC_MAX_N;
constexpr int kMaxK = MRRR_NOALLOC_MAX_K;

// Layout of the static scratch (byte offsets, each 256-aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffMat = 0;
constexpr size_t kOffBlk = align256(kOffMat + sizeof(MatrixDesc));
constexpr size_t kOffCnt = align256(kOffBlk + sizeof(BlockDesc));
constexpr size_t kOffStatus = align256(kOffCnt + sizeof(DevCounters));
constexpr size_t kOffWd = align256(kOffStatus + sizeof(int));
constexpr size_t kOffWe = align256(kOffWd + sizeof(double) * kMaxN);
constexpr size_t kOffRep = align256(kOffWe + sizeof(double) * kMaxN);
constexpr size_t kOffRepLo = align256(kOffRep + sizeof(double) * 4 * kMaxN);
constexpr size_t kOffWout = align256(kOffRepLo + sizeof(float) * 2 * kMaxN);
constexpr size_t kOffWork = align256(kOffWout + sizeof(float) * kMaxK);
constexpr size_t kBytes = align256(kOffWork + sizeof(double) * 2 * (size_t)kMaxN * kMaxK);
static_assert(kBytes == MRRR_NOALLOC_SCRATCH_BYTES, "header constant must match the layout");

// The scratch array.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

enum : int { NA_OK = 0, NA_NONFINITE = 1, NA_REDUCIBLE = 2 };

// The status slot (256 bytes) holds the status word and, after it, the
// brackets of the two eigenvalues just outside the given range in the root
// representation: [lo, hi] of lambda_{il-1} and of lambda_{il+k} (an absent
// neighbour has lo = hi = NaN).
constexpr size_t kOffNbr = kOffStatus + 8;
static_assert(kOffNbr + 4 * sizeof(double) <= kOffWd, "neighbour brackets must fit in the status slot");

// Bracket of eigenvalue j of the root rep by multisection on the 32 lanes of
// one warp: each sweep counts at 32 equispaced interior points (count_at,
// the tuned binary64 Sturm count) and keeps the sub-interval where the count
// reaches j, down to relative width rtol.  Invariant count(lo) < j <=
// count(hi); the first point whose count reaches j is the new upper end and
// the point before it the new lower end, which stays well defined where
// rounding makes the counts non-monotone.
__device__ void warp_bracket(const double* rep, int n, int j, double pivmin, double rtol, double lo, double hi,
                             double* out) {
    const int q = threadIdx.x & 31;
    for (int it = 0; it < 64; ++it) {
        const double tol = fmax(rtol * fmax(fabs(lo), fabs(hi)), 2.0 * pivmin);
        if (!(tol < hi - lo)) break;
        const double x = lo + (hi - lo) * (double)(q + 1) / 33.0;
        const bool inside = x > lo && x < hi;
        const int c = inside ? count_at<double, true>(rep, rep + 3 * n, n, x, pivmin) : 0;
        const unsigned reach = __ballot_sync(0xffffffffu, inside && c >= j);
        const unsigned in = __ballot_sync(0xffffffffu, inside);
        if (!in) break;  // no representable interior point left
        const int f = reach ? __ffs(reach) - 1 : 32;
        // new ends from the lanes' points (points outside the bracket are skipped)
        double nhi = hi, nlo = lo;
        for (int k = 0; k < 32; ++k) {
            const double xk = __shfl_sync(0xffffffffu, x, k);
            if (!((in >> k) & 1u)) continue;
            if (k < f) nlo = xk;
            else if (k == f) nhi = xk;
        }
        lo = nlo;
        hi = nhi;
    }
    if (q == 0) {
        out[0] = lo;
        out[1] = hi;
    }
}

// Kernel 1 (one CTA of 64 threads): scale, check irreducibility, root
// representation, then (one warp each) the brackets of the eigenvalues just
// below and just above the given range, which bound the gaps of the first
// and last given eigenvalue as the outer neighbours do in the solver.
__global__ void k_noalloc_root(unsigned char* base, const float* d, const float* e, int n, int il, int k,
                               SolveCfg cfg) {
    MatrixDesc& M = *(MatrixDesc*)(base + kOffMat);
    BlockDesc& B = *(BlockDesc*)(base + kOffBlk);
    int* status = (int*)(base + kOffStatus);
    double* wd = (double*)(base + kOffWd);
    double* we = (double*)(base + kOffWe);
    double* rep = (double*)(base + kOffRep);
    float* rep_lo = (float*)(base + kOffRepLo);
    __shared__ double s_gl, s_gu, s_g[2], s_mu[2];
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        double tn = 0.0;
        int bad = NA_OK;
        for (int i = 0; i < n; ++i) {
            double s = fabs((double)d[i]);
            if (!isfinite((double)d[i])) bad = NA_NONFINITE;
            if (i > 0) s += fabs((double)e[i - 1]);
            if (i < n - 1) {
                if (!isfinite((double)e[i])) bad = NA_NONFINITE;
                s += fabs((double)e[i]);
            }
            tn = fmax(tn, s);
        }
        double scale = 1.0;
        if (tn > 0.0) {
            int ex;
            frexp(tn, &ex);
            scale = ldexp(1.0, -ex);
        }
        for (int i = 0; i < n; ++i) {
            wd[i] = (double)d[i] * scale;
            we[i] = i < n - 1 ? (double)e[i] * scale : 0.0;
            if (bad == NA_OK && i < n - 1 && fabs((double)e[i]) <= cfg.eps_x * tn) bad = NA_REDUCIBLE;
        }
        memset(&M, 0, sizeof(M));
        M.n = n;
        M.nblocks = 1;
        M.scale = scale;
        M.tnorm = tn;
        M.range = RANGE_ALL;
        memset(&B, 0, sizeof(B));
        B.matrix = 0;
        B.row0 = 0;
        B.mrow = 0;
        B.n = n;
        *status = bad;
        s_bad = bad;
        if (bad == NA_OK) root_bounds<double>(B, wd, we, &s_gl, &s_gu);
    }
    double* nbr = (double*)(base + kOffNbr);
    if (threadIdx.x < 4) nbr[threadIdx.x] = NAN;
    __syncthreads();
    if (s_bad != NA_OK) return;
    if (n == 1) {
        if (threadIdx.x == 0) root_trivial<double, float>(B, wd, rep, rep_lo);
        return;
    }
    if (threadIdx.x == 0 || threadIdx.x == 32) {
        int side = threadIdx.x == 32;
        s_g[side] = root_candidate<double>(B, wd, we, rep, s_gl, s_gu, side, &s_mu[side]);
    }
    __syncthreads();
    if (threadIdx.x == 0) root_choose(B, M, s_gl, s_gu, s_g[0], s_mu[0], s_g[1], s_mu[1], cfg);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) root_move<double>(B, rep, i);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) root_element<double, float>(B, M, rep, rep_lo, i, cfg, we);
    __syncthreads();
    const int w = threadIdx.x >> 5;  // warp 0: lambda_{il-1}, warp 1: lambda_{il+k}
    const int j = w == 0 ? il - 1 : il + k;
    if (j >= 1 && j <= n) warp_bracket(rep, n, j, B.pivmin, cfg.rtol_class, B.gl, B.gu, nbr + 2 * w);
}

// Kernel 2 (one thread per eigenvalue): bracket the given eigenvalue
// lambda_{il+t} in the root rep, then the RQI of the solver (twisted
// factorizations, guarded by bisection) with its scratch in the static array.
__global__ void k_noalloc_rqi(unsigned char* base, const float* W, int il, int k, float* Z, int ldz, SolveCfg cfg) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k) return;
    if (*(const int*)(base + kOffStatus) != NA_OK) return;
    MatrixDesc* mats = (MatrixDesc*)(base + kOffMat);
    const BlockDesc* blocks = (const BlockDesc*)(base + kOffBlk);
    DevCounters* C = (DevCounters*)(base + kOffCnt);
    const BlockDesc& B = blocks[0];
    MatrixDesc M = mats[0];  // private copy: outputs of this call
    M.W = base + kOffWout;
    M.Z = Z;
    M.ldz = ldz;
    const int n = M.n;
    double lam = (double)W[t] * M.scale - B.mu;
    double w = 4.0 * cfg.eps_x * (fabs((double)W[t]) * M.scale + fabs(B.mu)) + 4.0 * B.pivmin;
    Item I;
    memset(&I, 0, sizeof(I));
    I.lo = lam - w;
    I.hi = lam + w;
    I.rep = base + kOffRep;
    I.rep_lo = base + kOffRepLo;
    I.n = n;
    I.j = il + t;
    I.block = 0;
    I.matrix = 0;
    I.outcol = t;
    I.sig_hi = B.mu;
    I.wanted = 1;
    I.rhint = -1;
    int fails = 0;
    verify_endpoint<double>(I, B, 0, &fails);
    verify_endpoint<double>(I, B, 1, &fails);
    // gaps from the neighbouring given eigenvalues; at the ends of the range,
    // from the bracket of the eigenvalue just outside it (none beyond
    // lambda_1 or lambda_n)
    const double* nbr = (const double*)(base + kOffNbr);
    if (t > 0) I.gapL = fmax(lam - ((double)W[t - 1] * M.scale - B.mu) - w, 0.5 * w);
    else I.gapL = il > 1 ? fmax(lam - nbr[1] - w, 0.5 * w) : INFINITY;
    if (t + 1 < k) I.gapR = fmax(((double)W[t + 1] * M.scale - B.mu) - lam - w, 0.5 * w);
    else I.gapR = il + k <= n ? fmax(nbr[2] - lam - w, 0.5 * w) : INFINITY;
    Scratch<double> Wk;
    Wk.a = (double*)(base + kOffWork) + (size_t)t * 2 * kMaxN;
    Wk.b = Wk.a + kMaxN;
    Wk.stride = 1;
    rqi_item<float, double>(I, &M, blocks, cfg, Wk, C, cfg.max_rqi, true);
}

// Device address of the scratch array, looked up once per device with that
// device current.
std::mutex g_mu;
void* g_addr[64];
bool g_done[64];

int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_done[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MRRR_ERR_CUDA;
        }
        g_addr[dev] = p;
        g_done[dev] = true;
    }
    *out = (unsigned char*)g_addr[dev];
    return MRRR_OK;
}

}  // namespace

extern "C" int mrrr_eigvecs_noalloc_s(int n, const float* d, const float* e, int il, int k, const float* W,
                                      float* Z, int ldz, void* stream) {
    if (n < 1 || n > MRRR_NOALLOC_MAX_N || k < 1 || k > MRRR_NOALLOC_MAX_K) return MRRR_ERR_ARG;
    if (il < 1 || il + k - 1 > n || ldz < n) return MRRR_ERR_ARG;
    if (!d || (n > 1 && !e) || !W || !Z) return MRRR_ERR_ARG;
    int devs = 0;
    if (cudaGetDeviceCount(&devs) != cudaSuccess || devs == 0) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    // every buffer must be device memory of the current device
    if (classify_ptr(d) != PTR_DEVICE || (n > 1 && classify_ptr(e) != PTR_DEVICE) || classify_ptr(W) != PTR_DEVICE ||
        classify_ptr(Z) != PTR_DEVICE)
        return MRRR_ERR_ARG;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != MRRR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the defaults of mrrr_solve_s in MRRR_MIXED mode
    const SolveCfg cfg = make_cfg(true, true, nullptr);
    // the counters of the previous call must not leak into this one
    if (cudaMemsetAsync(base + kOffCnt, 0, sizeof(DevCounters), st) != cudaSuccess) return MRRR_ERR_CUDA;
    k_noalloc_root<<<1, 64, 0, st>>>(base, d, n > 1 ? e : d, n, il, k, cfg);
    k_noalloc_rqi<<<(k + 63) / 64, 64, 0, st>>>(base, W, il, k, Z, ldz, cfg);
    if (cudaGetLastError() != cudaSuccess) return MRRR_ERR_CUDA;
    int status = 0;
    DevCounters C;
    if (cudaMemcpyAsync(&status, base + kOffStatus, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&C, base + kOffCnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MRRR_ERR_CUDA;
    if (status == NA_NONFINITE) return MRRR_ERR_NONFINITE;
    if (status == NA_REDUCIBLE) return MRRR_ERR_ARG;
    return C.noconv > 0 ? MRRR_ERR_NOCONV : MRRR_OK;
}
