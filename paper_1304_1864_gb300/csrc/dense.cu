// Dense symmetric eigenproblem A z = lambda z by reduction to tridiagonal
// form, the tridiagonal MRRR solver, and back-transformation (the dense
// experiment of Sec. 5, Fig. 3: A = Q T Q^T, whose reduction dominates the
// time while the tridiagonal stage sets the accuracy).  See mrrr_syev_s /
// mrrr_syev_d in include/mrrr.h.
//
// The reduction is the classical Householder tridiagonalisation in the I/O
// precision x, one reflector per column: for column k of the trailing
// matrix, with x = A[k+1:n, k],
//     beta = -sign(x_0) ||x||,  tau = (beta - x_0) / beta,
//     v = x / (x_0 - beta), v_0 = 1,   so that (I - tau v v^T) x = beta e_1,
// and the trailing block A22 = A[k+1:n, k+1:n] becomes H A22 H by the
// symmetric rank-2 update
//     p = tau A22 v,  w = p - (tau / 2)(p^T v) v,  A22 -= v w^T + w v^T.
// Then d_k = A[k, k], e_k = beta.  The eigenvectors of A are Q z with
// Q = H_0 H_1 ... H_{n-3}, applied to the tridiagonal eigenvectors in reverse
// order: Z[k+1:n, :] -= tau_k v_k (v_k^T Z[k+1:n, :]); each column is then
// signed so that its entry of largest magnitude is positive.
//
// Reductions (norms, the columns of A22 v, the dot products of the
// back-transformation) are fixed-order trees in x, so a result does not
// depend on scheduling.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>

#include "mrrr.h"
#include "mrrr_entry.h"
#include "mrrr_host.h"

namespace {

constexpr int kT = 256;       // threads of the row-parallel kernels
constexpr int kColChunk = 64; // columns of A22 per block of the matrix-vector product

// sum over a CTA of kT threads (fixed tree order); all threads get the result
template <class X>
__device__ X cta_sum(X v, X* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    X r = sh[0];
    __syncthreads();
    return r;
}

template <class X>
__device__ X cta_max(X v, X* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + h]);
        __syncthreads();
    }
    X r = sh[0];
    __syncthreads();
    return r;
}

// Reflector of column k (one CTA): x = A[k+1:n, k] (m = n-k-1 values).
// Writes d_k, e_k = beta, tau_k, v (v_0 = 1) to vbuf and v_1.. below the
// subdiagonal of column k (kept for the back-transformation).
template <class X>
__global__ void k_house(X* A, int n, int k, X* d, X* e, X* tau, X* vbuf) {
    __shared__ X sh[kT];
    const int m = n - k - 1;
    X* x = A + (size_t)k * n + (k + 1);
    X amax = 0;
    for (int i = 1 + threadIdx.x; i < m; i += kT) amax = fmax(amax, fabs(x[i]));
    amax = cta_max(amax, sh);
    const X alpha = x[0];
    X ss = 0;
    if (amax > 0) {
        const X inv = X(1) / amax;
        for (int i = 1 + threadIdx.x; i < m; i += kT) {
            const X t = x[i] * inv;
            ss += t * t;
        }
    }
    ss = cta_sum(ss, sh);
    X beta, t, sc;
    if (amax == 0) {
        beta = alpha;  // already reduced: H = I
        t = 0;
        sc = 0;
    } else {
        // ||x|| = hypot(alpha, amax sqrt(ss)) without overflow
        const X tail = amax * sqrt(ss);
        const X big = fmax(fabs(alpha), tail), small = fmin(fabs(alpha), tail);
        const X r = small / big;
        const X nrm = big * sqrt(X(1) + r * r);
        beta = alpha >= 0 ? -nrm : nrm;
        t = (beta - alpha) / beta;
        sc = X(1) / (alpha - beta);
    }
    for (int i = threadIdx.x; i < m; i += kT) {
        const X vi = i == 0 ? X(1) : x[i] * sc;
        vbuf[i] = vi;
        if (i > 0) x[i] = vi;
    }
    if (threadIdx.x == 0) {
        d[k] = A[(size_t)k * n + k];
        e[k] = beta;
        tau[k] = t;
        x[0] = beta;
    }
}

// Partial products of p = A22 v: block (rb, c) sums the columns
// [c kColChunk, (c+1) kColChunk) of the rows of its row block.
template <class X>
__global__ void k_symv(const X* A, int n, int k, const X* v, X* part) {
    const int m = n - k - 1;
    const int i = blockIdx.x * kT + threadIdx.x;
    const int c = blockIdx.y;
    const int j0 = c * kColChunk, j1 = min(m, j0 + kColChunk);
    if (i >= m) return;
    const X* col = A + (size_t)(k + 1) * n + (k + 1);
    X acc = 0;
    for (int j = j0; j < j1; ++j) acc += col[(size_t)j * n + i] * v[j];
    part[(size_t)c * m + i] = acc;
}

// w = p - (tau/2)(p^T v) v with p = tau * (sum of the partial products), one CTA.
template <class X>
__global__ void k_w(const X* part, int nchunk, int n, int k, const X* tau, const X* v, X* w) {
    __shared__ X sh[kT];
    const int m = n - k - 1;
    const X t = tau[k];
    X dot = 0;
    for (int i = threadIdx.x; i < m; i += kT) {
        X p = 0;
        for (int c = 0; c < nchunk; ++c) p += part[(size_t)c * m + i];
        p *= t;
        w[i] = p;
        dot += p * v[i];
    }
    dot = cta_sum(dot, sh);
    const X h = X(0.5) * t * dot;
    for (int i = threadIdx.x; i < m; i += kT) w[i] -= h * v[i];
}

// A22 -= v w^T + w v^T (column-major, threads along the rows).
template <class X>
__global__ void k_syr2(X* A, int n, int k, const X* v, const X* w) {
    const int m = n - k - 1;
    const int i = blockIdx.x * kT + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= m || j >= m) return;
    X* col = A + (size_t)(k + 1 + j) * n + (k + 1);
    col[i] -= v[i] * w[j] + w[i] * v[j];
}

// The last 2 x 2 block (or the 1 x 1 matrix).
template <class X>
__global__ void k_tail(const X* A, int n, X* d, X* e, X* tau) {
    if (threadIdx.x != 0) return;
    if (n >= 2) {
        d[n - 2] = A[(size_t)(n - 2) * n + (n - 2)];
        e[n - 2] = A[(size_t)(n - 2) * n + (n - 1)];
        tau[n - 2] = 0;
    }
    d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
}

// s_j = v_k^T Z[k+1:n, j] (one CTA per column j).
template <class X>
__global__ void k_dotv(const X* A, int n, int k, const X* Z, int ldz, X* s) {
    __shared__ X sh[kT];
    const int m = n - k - 1;
    const int j = blockIdx.x;
    const X* v = A + (size_t)k * n + (k + 1);  // v_0 = 1 implicit, v_i below
    const X* z = Z + (size_t)j * ldz + (k + 1);
    X acc = 0;
    for (int i = threadIdx.x; i < m; i += kT) acc += (i == 0 ? X(1) : v[i]) * z[i];
    acc = cta_sum(acc, sh);
    if (threadIdx.x == 0) s[j] = acc;
}

// Z[k+1:n, j] -= tau_k v_k s_j.
template <class X>
__global__ void k_ger(const X* A, int n, int k, const X* tau, X* Z, int ldz, const X* s) {
    const int m = n - k - 1;
    const int i = blockIdx.x * kT + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= m) return;
    const X* v = A + (size_t)k * n + (k + 1);
    const X vi = i == 0 ? X(1) : v[i];
    Z[(size_t)j * ldz + (k + 1) + i] -= tau[k] * vi * s[j];
}

// Sign convention of the back-transformed vectors (one CTA per column): the
// entry of largest magnitude (the first on ties) is made positive.
template <class X>
__global__ void k_sign(X* Z, int n, int ldz) {
    __shared__ X sv[kT];
    __shared__ int si[kT];
    X* z = Z + (size_t)blockIdx.x * ldz;
    X best = -1;
    int bi = 0;
    for (int i = threadIdx.x; i < n; i += kT) {
        const X a = fabs(z[i]);
        if (a > best) {
            best = a;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const X b = sv[threadIdx.x + h];
            const int j = si[threadIdx.x + h];
            if (b > sv[threadIdx.x] || (b == sv[threadIdx.x] && j < si[threadIdx.x])) {
                sv[threadIdx.x] = b;
                si[threadIdx.x] = j;
            }
        }
        __syncthreads();
    }
    __shared__ int flip;
    if (threadIdx.x == 0) flip = z[si[0]] < 0;
    __syncthreads();
    if (flip)
        for (int i = threadIdx.x; i < n; i += kT) z[i] = -z[i];
}

struct Buf {
    void* p = nullptr;
    cudaStream_t st;
    explicit Buf(cudaStream_t s) : st(s) {}
    bool alloc(size_t bytes) { return (p = mrrr::dev_alloc(bytes ? bytes : 1, st)) != nullptr; }
    ~Buf() { mrrr::dev_free(p, st); }
};

inline int grid1(int m) { return (m + kT - 1) / kT; }

template <class X>
int syev_one(int n, const X* A, int lda, mrrr_range range, X vl, X vu, int il, int iu, mrrr_mode mode,
             const mrrr_params* prm, int* m_out, X* W, X* Z, int ldz, void* stream) {
    if (m_out) *m_out = 0;
    if (n < 0 || lda < n || (n > 0 && (!A || !W || !Z || ldz < n))) return MRRR_ERR_ARG;
    if (range != MRRR_ALL && range != MRRR_INDEX && range != MRRR_VALUE) return MRRR_ERR_ARG;
    if (range == MRRR_INDEX && n > 0 && (il < 1 || iu > n || il > iu)) return MRRR_ERR_ARG;
    if (range == MRRR_VALUE && !(vl < vu)) return MRRR_ERR_ARG;
    if (mode != MRRR_PLAIN && mode != MRRR_MIXED) return MRRR_ERR_ARG;
    if (n == 0) return MRRR_OK;
    if (n > 46340) return MRRR_ERR_ARG;  // n * n must index an int-sized grid dimension product
    int devs = 0;
    if (cudaGetDeviceCount(&devs) != cudaSuccess || devs == 0) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    const mrrr::PtrKind ka = mrrr::classify_ptr(A), kw = mrrr::classify_ptr(W), kz = mrrr::classify_ptr(Z);
    if (ka == mrrr::PTR_OTHER_DEVICE || kw == mrrr::PTR_OTHER_DEVICE || kz == mrrr::PTR_OTHER_DEVICE)
        return MRRR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int kmax = range == MRRR_INDEX ? iu - il + 1 : n;
    const int nchunk = (n + kColChunk - 1) / kColChunk;
    Buf bA(st), bd(st), be(st), btau(st), bv(st), bw(st), bpart(st), bs(st), bW(st), bZ(st);
    if (!bA.alloc(sizeof(X) * (size_t)n * n) || !bd.alloc(sizeof(X) * n) || !be.alloc(sizeof(X) * n) ||
        !btau.alloc(sizeof(X) * n) || !bv.alloc(sizeof(X) * n) || !bw.alloc(sizeof(X) * n) ||
        !bpart.alloc(sizeof(X) * (size_t)nchunk * n) || !bs.alloc(sizeof(X) * kmax) || !bW.alloc(sizeof(X) * kmax) ||
        !bZ.alloc(sizeof(X) * (size_t)n * kmax))
        return MRRR_ERR_NOMEM;
    X* Aw = (X*)bA.p;
    X* d = (X*)bd.p;
    X* e = (X*)be.p;
    X* tau = (X*)btau.p;
    X* v = (X*)bv.p;
    X* w = (X*)bw.p;
    X* part = (X*)bpart.p;
    X* s = (X*)bs.p;
    X* Wt = (X*)bW.p;
    X* Zt = (X*)bZ.p;
    if (cudaMemcpy2DAsync(Aw, sizeof(X) * n, A, sizeof(X) * (size_t)lda, sizeof(X) * n, n,
                          ka == mrrr::PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MRRR_ERR_CUDA;
    // reduction to tridiagonal form, one reflector per column
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        k_house<X><<<1, kT, 0, st>>>(Aw, n, k, d, e, tau, v);
        k_symv<X><<<dim3(grid1(m), (m + kColChunk - 1) / kColChunk), kT, 0, st>>>(Aw, n, k, v, part);
        k_w<X><<<1, kT, 0, st>>>(part, (m + kColChunk - 1) / kColChunk, n, k, tau, v, w);
        k_syr2<X><<<dim3(grid1(m), m), kT, 0, st>>>(Aw, n, k, v, w);
    }
    k_tail<X><<<1, 32, 0, st>>>(Aw, n, d, e, tau);
    if (cudaGetLastError() != cudaSuccess) return MRRR_ERR_CUDA;
    // the tridiagonal eigenproblem
    int mfound = 0;
    int rc;
    if (std::is_same<X, float>::value)
        rc = mrrr_solve_s(n, (const float*)d, (const float*)e, range, (float)vl, (float)vu, il, iu, mode, prm,
                          &mfound, (float*)Wt, (float*)Zt, n, st);
    else
        rc = mrrr_solve_d(n, (const double*)d, (const double*)e, range, (double)vl, (double)vu, il, iu, mode, prm,
                          &mfound, (double*)Wt, (double*)Zt, n, st);
    if (rc != MRRR_OK && rc != MRRR_ERR_NOCONV) return rc;
    // back-transformation Z = H_0 H_1 ... H_{n-3} Z_T
    if (mfound > 0) {
        for (int k = n - 3; k >= 0; --k) {
            const int m = n - k - 1;
            k_dotv<X><<<mfound, kT, 0, st>>>(Aw, n, k, Zt, n, s);
            k_ger<X><<<dim3(grid1(m), mfound), kT, 0, st>>>(Aw, n, k, tau, Zt, n, s);
        }
        k_sign<X><<<mfound, kT, 0, st>>>(Zt, n, n);
        if (cudaGetLastError() != cudaSuccess) return MRRR_ERR_CUDA;
        const cudaMemcpyKind kW = kw == mrrr::PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        const cudaMemcpyKind kZ = kz == mrrr::PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (cudaMemcpyAsync(W, Wt, sizeof(X) * mfound, kW, st) != cudaSuccess ||
            cudaMemcpy2DAsync(Z, sizeof(X) * (size_t)ldz, Zt, sizeof(X) * n, sizeof(X) * n, mfound, kZ, st) !=
                cudaSuccess)
            return MRRR_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return MRRR_ERR_CUDA;
    if (m_out) *m_out = mfound;
    return rc;
}

}  // namespace

extern "C" {

int mrrr_syev_s(int n, const float* A, int lda, mrrr_range range, float vl, float vu, int il, int iu,
                mrrr_mode mode, const mrrr_params* params, int* m_out, float* W, float* Z, int ldz, void* stream) {
    return syev_one<float>(n, A, lda, range, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream);
}

int mrrr_syev_d(int n, const double* A, int lda, mrrr_range range, double vl, double vu, int il, int iu,
                mrrr_mode mode, const mrrr_params* params, int* m_out, double* W, double* Z, int ldz, void* stream) {
    return syev_one<double>(n, A, lda, range, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream);
}

}  // extern "C"
