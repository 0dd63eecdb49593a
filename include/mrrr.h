/*
 * mrrr.h -- C ABI of the GB300 mixed-precision MRRR tridiagonal eigensolver.
 *
 * Problem (paper Sec. 1): given a real symmetric tridiagonal T with diagonal
 * d[0..n-1] and off-diagonal e[0..n-2], compute eigenpairs (lambda_i, z_i),
 * T z_i = lambda_i z_i, ||z_i||_2 = 1, for an index set
 * I subset {1..n} with lambda_1 <= ... <= lambda_n.  The method is MRRR
 * (Algorithm 1) with the mixed-precision scheme of Sec. 3: input/output in
 * precision x, all sensitive work in a working precision y > x:
 *
 *   mrrr_solve_s, MRRR_MIXED : x = binary32, y = binary64  ("single/double")
 *   mrrr_solve_d, MRRR_MIXED : x = binary64, y = double-double (~106 bits),
 *                              standing in for the paper's "double/quadruple"
 *   MRRR_PLAIN               : y = x (the conventional single-precision solver
 *                              the paper compares against)
 *
 * Conventions shared by every entry point:
 *  - Indices il..iu are 1-based and inclusive.  A value range is the
 *    half-open interval (vl, vu].
 *  - d, e, W, Z may be device pointers or host pointers (pageable or
 *    pinned); host buffers are staged through device memory by the call.
 *    Device buffers must be memory of the device that is current at the
 *    call (or managed memory); another device's memory is MRRR_ERR_ARG.
 *    The caller owns every buffer.  W must hold k entries and Z n x k
 *    entries, column-major with leading dimension ldz >= n, where
 *    k = iu - il + 1 (MRRR_INDEX), n (MRRR_ALL) or, for MRRR_VALUE, n
 *    (the count found is returned in *m_out).
 *  - W is returned in ascending order and column j of Z belongs to W[j].
 *    Each column has unit 2-norm and is signed so that an entry of largest
 *    magnitude is positive.
 *  - All work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream).  The call returns after the results are complete on that
 *    stream.  There is no host (CPU) fallback: without a usable CUDA device
 *    the call fails with MRRR_ERR_CUDA.
 *  - Return value: 0 on success or a negative mrrr_status code.  On
 *    MRRR_ERR_NOCONV the outputs are filled but at least one eigenpair did
 *    not meet its stopping criterion.
 */
#ifndef MRRR_H
#define MRRR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { MRRR_ALL = 0, MRRR_INDEX = 1, MRRR_VALUE = 2 } mrrr_range;

/* MRRR_PLAIN: working precision = I/O precision.  MRRR_MIXED: the next
 * higher precision (Sec. 3.1). */
typedef enum { MRRR_PLAIN = 0, MRRR_MIXED = 1 } mrrr_mode;

typedef enum {
    MRRR_OK = 0,
    MRRR_ERR_ARG = -1,        /* invalid argument (sizes, ranges, ldz, NULL) */
    MRRR_ERR_NONFINITE = -2,  /* NaN or Inf in d or e */
    MRRR_ERR_NOCONV = -3,     /* an eigenpair missed its stopping test; outputs filled */
    MRRR_ERR_NOMEM = -4,      /* device allocation failed */
    MRRR_ERR_CUDA = -5,       /* CUDA runtime error / no device */
    MRRR_ERR_TIMEOUT = -6,    /* a bounded device-side wait ran out */
    MRRR_ERR_NOREP = -7,      /* informational: no candidate passed the representation test */
    MRRR_ERR_CANCELLED = -8   /* serving: the request was cancelled before it ran */
} mrrr_status;

/* Phases of a solve, indexing mrrr_stats.phase_ms. */
enum {
    MRRR_PHASE_PREP = 0,     /* scaling and splitting (a1) */
    MRRR_PHASE_ROOT = 1,     /* root representations and eigenvalue items (a2) */
    MRRR_PHASE_BISECT = 2,   /* initial eigenvalues by bisection (a3) */
    MRRR_PHASE_CLASSIFY = 3, /* classification into singletons and clusters (a4) */
    MRRR_PHASE_SHIFT = 4,    /* child representations of clusters (a5) */
    MRRR_PHASE_REFINE = 5,   /* refinement of cluster eigenvalues (a5) */
    MRRR_PHASE_RQI = 6,      /* Rayleigh quotient iteration, vectors, stores (a6, a7) */
    MRRR_PHASE_FINISH = 7,   /* output ordering and zero fill */
    MRRR_NPHASES = 8
};

/* Per-solve statistics (optional output). */
typedef struct {
    int nblocks;          /* blocks after splitting (Sec. 3.2, Preprocessing) */
    int d_max;            /* depth of the representation tree (Sec. 2) */
    int nclusters;        /* clusters processed (Algorithm 1, lines 14-17) */
    int largest_cluster;  /* size of the largest cluster; rho = largest_cluster / n */
    int reps_failed;      /* clusters whose chosen representation failed both growth tests */
    int rqi_iters;        /* Rayleigh quotient iterations (twisted solves), all eigenpairs */
    int fallbacks;        /* eigenpairs that needed the bisection fallback */
    int noconv;           /* eigenpairs that missed the stopping criterion */
    long long qd_bisect;  /* qd steps (one row of one transform) in the initial bisection */
    long long qd_refine;  /* qd steps in the refinement bisection of cluster eigenvalues */
    long long qd_rqi;     /* qd steps in the Rayleigh quotient iterations */
    long long qd_shift;   /* qd steps in building child representations */
    long long qd_low;     /* qd steps of the pre-bisection in a precision below the working one */
    int verify_fail;      /* pre-bisection brackets widened by the working-precision check */
    int reps_relaxed;     /* child reps accepted only under the relaxed growth bound of Eq. (3.6) */
    int rqi_warps_per_sm; /* resident warps per SM of the persistent RQI grid (largest RQI list) */
    int timed;            /* 1 if phase_ms / phase_launches were measured (MRRR_FLAG_TIMING) */
    int phase_launches[MRRR_NPHASES]; /* kernel launches per phase */
    double phase_ms[MRRR_NPHASES];    /* device time per phase (CUDA events on the solve's stream) */
    long long rqi_rows;   /* sum over all RQI steps of the order n of the step's block: each step is one
                             twisted factorization and solve of n rows (Sec. 2) */
    int reps_backtracked; /* clusters processed again from the representation one level up because no
                             candidate built from their parent passed (Sec. 3.2, "The representation tree") */
    int reps_krr_relaxed; /* (MRRR_FLAG_RRR_TEST) children accepted with a relative condition estimate above
                             10, i.e. only under the relaxed k_rr bound of Eq. (3.7) */
    double krr_max;       /* (MRRR_FLAG_RRR_TEST) largest relative condition estimate of an accepted child */
} mrrr_stats;

/* Tuning parameters; a zero field selects the default given in brackets. */
typedef struct {
    double gaptol;     /* classification tolerance, Eq. (3.3) [PLAIN 1e-3 (x=d) / 3e-3 (x=s);
                          MIXED 1e-5 (s/d), 1e-10 (d/dd)] */
    double xi;         /* bound of the random relative perturbation of the root
                          representation, Algorithm 1 line 2 [PLAIN 8 eps_x; MIXED 4 eps_x] */
    double krs;        /* RQI stopping constant k_rs, Eq. (2.2) and (3.8) [1] */
    int max_depth;     /* depth cap of the representation tree [16] */
    int max_rqi;       /* RQI steps before the bisection fallback [10] */
    uint64_t seed;     /* seed of the perturbation sequence [0] */
    int flags;         /* MRRR_FLAG_* variant bits [0] */
    mrrr_stats* stats; /* if non-NULL, receives the statistics of the call (host memory) */
} mrrr_params;

/* Variant bits for mrrr_params.flags. */
#define MRRR_FLAG_NO_LOWPREC_BISECT 1 /* never pre-bracket eigenvalues in a lower precision */
#define MRRR_FLAG_TIMING 4            /* time every phase with CUDA events (fills stats->phase_ms) */
#define MRRR_FLAG_STRICT_GROWTH 8     /* MIXED: accept child reps only under the y = x growth bound,
                                         not the relaxed bound of Sec. 3.2, Eq. (3.6) */
#define MRRR_FLAG_NO_TUNE 16          /* use the default RQI grid instead of the autotuned one */
#define MRRR_FLAG_E_REP 64            /* e-representation (Sec. 3.2, "Choice of representations"): the root
                                         keeps the input's off-diagonal e_i as data and every child keeps its
                                         parent's LD_i = e_i exactly (stored once), instead of forming
                                         LD = d l from its own pivots */
#define MRRR_FLAG_RRR_TEST 128        /* accept a child representation only if the relative condition number
                                         of the cluster's eigenvalues along an approximate cluster vector is
                                         within the k_rr bound: 10, or with y > x the relaxed bound
                                         max{10, eps_x gaptol / (eps_y sqrt(n))} of Sec. 3.2, Eq. (3.7) */
#define MRRR_FLAG_TEST_NO_REP 256     /* testing only: turn down every candidate representation, in the
                                         first search and in backtracking, so that every cluster takes its
                                         best failed candidate (the branch of Algorithm 1, lines 15-17, for
                                         "no suitable representation"; counted in reps_failed) */
#define MRRR_FLAG_TEST_REJECT_CHILD 32 /* testing only: turn down every child representation built from a
                                          parent that is itself a child, which forces the backtracking
                                          branch of the representation tree (Sec. 3.2) */

/*
 * Single-precision input/output (x = binary32).  MRRR_MIXED computes in
 * binary64 (paper "single/double", Sec. 4.1); MRRR_PLAIN in binary32.
 * range/vl/vu/il/iu select the eigenpairs as described above.  params may be
 * NULL (all defaults).  On success *m_out (may be NULL for ALL/INDEX) holds
 * the number of eigenpairs returned.
 */
int mrrr_solve_s(int n, const float* d, const float* e, mrrr_range range, float vl, float vu,
                 int il, int iu, mrrr_mode mode, const mrrr_params* params, int* m_out,
                 float* W, float* Z, int ldz, void* stream);

/*
 * Double-precision input/output (x = binary64).  MRRR_MIXED computes the
 * representation-tree shifts, the qd transforms and the twisted
 * factorizations in double-double (the role binary128 plays in the paper's
 * "double/quadruple" solver, Sec. 4.1); MRRR_PLAIN in binary64.
 */
int mrrr_solve_d(int n, const double* d, const double* e, mrrr_range range, double vl, double vu,
                 int il, int iu, mrrr_mode mode, const mrrr_params* params, int* m_out,
                 double* W, double* Z, int ldz, void* stream);

/*
 * Batched solve (all eigenpairs of each matrix, or the index range
 * il[p]..iu[p] when il and iu are non-NULL): nb independent tridiagonals,
 * each solved on its own (Algorithm 1 per matrix), in one sequence of
 * launches over all matrices.  The arrays n, d, e, W, Z, ldz, il, iu,
 * m_out and status are host arrays of length nb; each d[p], e[p], W[p],
 * Z[p] may be a device pointer or a host pointer, as for mrrr_solve_s (host
 * inputs are copied to one staging block of device memory before the solve,
 * host outputs copied back from it after; n[p] = 1 needs no e[p]).  status[p]
 * receives the matrix's own status and m_out[p] (may be NULL) its count.
 * Returns 0 if every matrix succeeded, else the first failing status.
 */
int mrrr_solve_batch_s(int nb, const int* n, const float* const* d, const float* const* e, const int* il,
                       const int* iu, mrrr_mode mode, const mrrr_params* params, int* m_out, float* const* W,
                       float* const* Z, const int* ldz, int* status, void* stream);
int mrrr_solve_batch_d(int nb, const int* n, const double* const* d, const double* const* e, const int* il,
                       const int* iu, mrrr_mode mode, const mrrr_params* params, int* m_out, double* const* W,
                       double* const* Z, const int* ldz, int* status, void* stream);

/*
 * Dense symmetric eigenproblem A z = lambda z (the dense experiment of
 * Sec. 5, Fig. 3): Householder reduction of A to tridiagonal form
 * T = Q^T A Q in the I/O precision, the tridiagonal solve of
 * mrrr_solve_s / _d (mode MRRR_MIXED or MRRR_PLAIN, params, range as
 * there), and back-transformation Z = Q Z_T.  A is n x n, column-major with
 * leading dimension lda >= n, symmetric (both triangles are read, neither
 * is written); W and Z as for mrrr_solve_s.  A, W, Z may be host or device
 * pointers.  The reduction costs O(n^3) and dominates the time for large
 * n; the tridiagonal stage sets the accuracy of the eigenvectors.  n is at
 * most 46340.  Returns as mrrr_solve_s.
 */
int mrrr_syev_s(int n, const float* A, int lda, mrrr_range range, float vl, float vu, int il, int iu,
                mrrr_mode mode, const mrrr_params* params, int* m_out, float* W, float* Z, int ldz, void* stream);
int mrrr_syev_d(int n, const double* A, int lda, mrrr_range range, double vl, double vu, int il, int iu,
                mrrr_mode mode, const mrrr_params* params, int* m_out, double* W, double* Z, int ldz,
                void* stream);

/*
 * Index partition for independent solves of one matrix, e.g. one part per
 * GPU (the eigenpairs of an index range need no data from the other
 * ranges).  Splits 1..n into nparts contiguous ranges il[p]..iu[p]
 * (1-based, inclusive; il[p] = iu[p] + 1 for an empty part; il[0] = 1,
 * iu[nparts-1] = n) whose boundaries lie where the classification of the
 * root representation separates consecutive eigenvalues (Sec. 2,
 * "Classification of the eigenvalues", with a margin of 4 gaptol), so that
 * no cluster and no child representation is shared by two parts; each
 * boundary is the separated pair nearest to the even split p n / nparts.
 * Solving part p with mrrr_solve_s / _d (MRRR_INDEX, il[p]..iu[p], the same
 * mode and params) gives eigenpairs that are mutually orthogonal with those
 * of the other parts to the method's accuracy.  A matrix that splits into
 * blocks is cut evenly.  d, e may be host or device pointers; il and iu are
 * host arrays of nparts entries.  The work (root representation and
 * bisection of the eigenvalues near the candidate boundaries) is enqueued on
 * `stream` and the call returns when it is complete.
 */
int mrrr_partition_s(int n, const float* d, const float* e, mrrr_mode mode, const mrrr_params* params, int nparts,
                     int* il, int* iu, void* stream);
int mrrr_partition_d(int n, const double* d, const double* e, mrrr_mode mode, const mrrr_params* params,
                     int nparts, int* il, int* iu, void* stream);

/*
 * Eigenvectors for given eigenvalues without any device allocation.
 *
 * The paper has no counterpart of this entry point.  It is for callers that
 * must not allocate device memory when they call the solver: real-time or
 * embedded hosts that reserve all their memory at start-up and treat any
 * later allocation as a failure, and libraries whose device memory belongs
 * to another framework's allocator, where a cudaMalloc of its own would
 * bypass that allocator's accounting and limits.  It runs the solver's
 * Rayleigh-quotient / twisted-factorization kernel on one fixed scratch
 * array instead of allocated buffers, and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * Input: T (d[0..n-1], e[0..n-2], binary32, device pointers) and k of its
 * eigenvalues W[0..k-1] = lambda_il .. lambda_{il+k-1} in ascending order
 * (for instance as returned by mrrr_solve_s).  Output: Z (device, n x k,
 * column-major, leading dimension ldz >= n), column t the unit eigenvector of
 * lambda_{il+t}, largest entry positive.  Work: the root representation with
 * binary64 internals as in mrrr_solve_s (MRRR_MIXED, the same parameter
 * defaults), each given eigenvalue bracketed by binary64 Sturm counts, the
 * eigenvalues just below and just above the range bracketed by bisection
 * (they bound the gaps of the first and last given eigenvalue, as in the
 * solver), then Rayleigh quotient iteration with twisted factorizations on
 * that one representation.  There is no representation tree, so the given
 * eigenvalues must be separated relative to each other by more than 1e-5
 * (the mixed gaptol); within tighter clusters use mrrr_solve_s.  The matrix
 * must not split (no |e_i| <= 2^-24 ||T||_1).
 *
 * Errors: sizes beyond the limits below, other invalid sizes, NULL or host
 * pointers, and device memory of a device other than the current one return
 * MRRR_ERR_ARG before anything is launched.  A reducible matrix is detected
 * on the device: the call then returns MRRR_ERR_ARG after its kernels ran,
 * with Z not written; non-finite input likewise returns MRRR_ERR_NONFINITE.
 *
 * Limits: n <= MRRR_NOALLOC_MAX_N and k <= MRRR_NOALLOC_MAX_K.  The scratch
 * is one file-scope device array of MRRR_NOALLOC_SCRATCH_BYTES bytes that
 * every GPU loading the library holds until the process exits.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture begins.  All calls share the array and it keeps
 * the previous call's contents (each call clears what must start at zero);
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  The call reads its status
 * back and synchronises `stream` before it returns.
 */
#define MRRR_NOALLOC_MAX_N 1024
#define MRRR_NOALLOC_MAX_K 1024
#define MRRR_NOALLOC_SCRATCH_BYTES 16839680
int mrrr_eigvecs_noalloc_s(int n, const float* d, const float* e, int il, int k, const float* W, float* Z,
                           int ldz, void* stream);

/*
 * Serving loop: continuous batching of independent solve requests.
 *
 * The paper solves one matrix at a time; this is the request loop around the
 * same solver for many clients.  A server owns `workers` host threads, each
 * with its own CUDA stream.  Submitted requests wait in arrival order; a free
 * worker admits the oldest pending request and every later pending request
 * of the same precision and mode, as long as the device bytes charged to the
 * admitted requests stay within `hbm_budget` (a request is charged its
 * device inputs, device copies of host outputs and the solver's own
 * representation, item and RQI scratch; a request larger than the whole
 * budget runs alone once nothing else is admitted), and runs them as one
 * batched solve (mrrr_solve_batch_s / _d semantics, each matrix solved on its
 * own, so a result does not depend on what it was batched with).  Requests
 * that arrive while batches run are admitted by the next worker that frees
 * up, so work from different batches overlaps on the device.
 *
 * Ownership: the caller owns the output buffers named in the request (host
 * or device; host outputs are written by a device-to-host copy when the
 * batch completes) and must keep them, and device inputs, alive until the
 * request is polled complete.  Host inputs are copied at submit.  Device
 * buffers are used only after the work the caller queued on the request's
 * stream before submit (an event recorded at submit).  Every call
 * is thread-safe.  A server is bound to the device current at open.
 */
typedef struct mrrr_server mrrr_server;

typedef struct {
    int workers;          /* concurrent batches (host threads + streams) [2] */
    int max_batch;        /* requests per batch [512] */
    long long hbm_budget; /* device bytes for admitted requests; 0: half the free memory at open */
    int alloc_failures;   /* testing only: the first alloc_failures batches fail as if their device
                             allocation had failed (every request in them completes with
                             MRRR_ERR_NOMEM; the server goes on) [0] */
} mrrr_serve_config;

typedef struct {
    int precision;   /* 0: binary32 I/O (as mrrr_solve_s), 1: binary64 I/O (as mrrr_solve_d) */
    mrrr_mode mode;  /* MRRR_MIXED or MRRR_PLAIN */
    int n;           /* order, >= 1 */
    const void* d;   /* diagonal, n values of the request's precision (host or device) */
    const void* e;   /* off-diagonal, n - 1 values (may be NULL when n = 1) */
    int il, iu;      /* 1-based index range; il = 0 selects all eigenpairs */
    void* W;         /* output eigenvalues, >= iu - il + 1 (or n) values (host or device) */
    void* Z;         /* output eigenvectors, column-major, leading dimension ldz >= n */
    int ldz;
    void* stream;    /* device buffers are ready once the work queued on this cudaStream_t before
                        submit has run (NULL: the legacy default stream); completion is reported by
                        mrrr_serve_poll, not ordered on this stream */
} mrrr_request;

typedef struct {
    int status;        /* the request's own status (0 or a negative MRRR_ERR_*) */
    int m;             /* eigenpairs returned */
    int batch;         /* requests in the batch it ran in */
    double queue_ms;   /* submit to admission */
    double latency_ms; /* submit to completion (outputs written) */
} mrrr_serve_info;

typedef struct {
    long long completed;  /* requests completed since open */
    long long eigenpairs; /* eigenpairs returned by them */
    long long batches;    /* batched solves run */
    double p50_ms, p99_ms, max_ms; /* latency percentiles over the completed requests */
    double busy_s;        /* wall time from the first admission to the last completion */
} mrrr_serve_stats;

#define MRRR_PENDING 1  /* mrrr_serve_poll: not complete yet */

/* Start a server (cfg may be NULL for the defaults). */
int mrrr_serve_open(const mrrr_serve_config* cfg, mrrr_server** out);
/* Queue a request; *ticket identifies it for mrrr_serve_poll.  Argument
   errors are reported here, before anything is queued. */
int mrrr_serve_submit(mrrr_server* s, const mrrr_request* req, long long* ticket);
/* Wait up to wait_ms (< 0: no limit) for the request.  Returns MRRR_PENDING
   if it is not complete, else its status, fills *info (may be NULL) and
   retires the ticket.  An unknown ticket returns MRRR_ERR_ARG. */
int mrrr_serve_poll(mrrr_server* s, long long ticket, int wait_ms, mrrr_serve_info* info);
/* Withdraw a request that has not been admitted yet: returns MRRR_OK, and its
   poll then returns MRRR_ERR_CANCELLED with the output buffers untouched.  A
   request already admitted or completed is not withdrawn: MRRR_PENDING (poll
   it for its result).  An unknown or retired ticket returns MRRR_ERR_ARG. */
int mrrr_serve_cancel(mrrr_server* s, long long ticket);
/* Latency and throughput counters since open (cancelled requests are not
   counted). */
int mrrr_serve_stats_get(mrrr_server* s, mrrr_serve_stats* out);
/* Finish every queued request, stop the workers and free the server. */
int mrrr_serve_close(mrrr_server* s);

/* Human-readable text for a status code (static storage). */
const char* mrrr_strerror(int status);

/* Library version string (static storage). */
const char* mrrr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MRRR_H */
