// Device-side descriptors shared by the solver kernels and the host driver.
#pragma once

#include <cstdint>

namespace mrrr {

// Parameters of one solve (Sec. 3.2 and Sec. 4.1 defaults are filled in by
// the host driver from mrrr_params).
struct SolveCfg {
    double eps_x;       // unit roundoff of the input/output precision (Table 1)
    double eps_y;       // unit roundoff of the working precision
    double gaptol;      // classification tolerance (Sec. 2, Eq. 3.3)
    double rtol_class;  // relative bracket width for classification: 1e-2 gaptol (Sec. 4.1)
    double xi;          // perturbation bound of the root representation
    double krs;         // RQI stopping constant
    double growth_k;    // element-growth acceptance factor (max |d+| <= growth_k spdiam)
    int max_rqi;        // RQI steps before the bisection fallback
    int mixed;          // 1: mixed precision stopping rules (Sec. 3.2), 0: plain (Sec. 2)
    uint64_t seed;      // perturbation seed
    int flags;
};

enum : int { RANGE_ALL = 0, RANGE_INDEX = 1, RANGE_VALUE = 2 };

enum : int {
    ST_OK = 0,
    ST_ERR_NONFINITE = -2,
    ST_ERR_NOCONV = -3,
};

struct MatrixDesc {
    const void* d;      // input diagonal (precision x, device)
    const void* e;      // input off-diagonal (precision x, device)
    void* W;            // output eigenvalues (x, device)
    void* Z;            // output eigenvectors (x, device), column-major
    int ldz;
    int n;
    int row0;           // first row in the concatenated working arrays
    int range;
    double vl, vu;
    int il, iu;
    // filled by the solver
    int nblocks;        // blocks after splitting; block descriptors at [row0, row0 + nblocks)
    int item0, nitems;  // eigenvalue items of this matrix
    int kout;           // number of eigenpairs returned
    double scale;       // T was multiplied by this power of two
    double tnorm;       // ||T||_1 before scaling
    int status;
};

struct BlockDesc {
    int matrix;
    int row0;           // first global row of the block
    int mrow;           // first row of the block within its matrix
    int n;              // block size
    double mu;          // root shift (scaled coordinates): M_root = T_block - mu I
    double gl, gu;      // bracket of the root rep's spectrum
    double spdiam;      // spectral diameter bound (Gershgorin width)
    double pivmin;      // pivot guard
    int side;           // +1: root shift at the left end (positive definite), -1: right end
    double growth;      // max |d_i| of the root factorization
    int w_lo, w_hi;     // wanted local indices (1-based, inclusive; w_lo > w_hi: none)
    int f_lo, f_hi;     // computed local indices (wanted plus one neighbour each side)
    int item0, nitems;
    int rep_off;        // offset of the root rep in the root-rep array (4 * row0)
};

// One eigenvalue of one block, carried through the representation tree.
struct Item {
    double lo, hi;      // bracket in the coordinates of the current rep
    double gapL, gapR;  // absolute distance to the neighbouring eigenvalues (left/right)
    double sig_hi, sig_lo;  // accumulated shift sigma of the current rep (hi + lo)
    const void* rep;    // current rep [D | L | LD | LLD], working precision
    const void* rep_lo; // rounded copy [D | LLD] of the rep in the low precision (pre-bisection)
    int n;              // rep (block) size
    int j;              // 1-based index within the block
    int block;
    int matrix;
    int outcol;         // output column, -1 if the item is only a neighbour
    int depth;          // depth of the current rep in the representation tree
    int kind;           // KIND_*
    int wanted;         // 1 if the eigenpair is returned, 0 if only a neighbour
    // the representation one level up (the parent of `rep`; nullptr at the
    // root), its accumulated shift, and the span [span_lo, span_hi] (in its
    // coordinates) of the cluster `rep` was made for, with that cluster's
    // gaps to the rest of the spectrum -- for backtracking
    const void* rep_up;
    double sig_up_hi, sig_up_lo;
    double span_lo, span_hi;
    double span_gapL, span_gapR;
    // Rayleigh quotient iteration state carried between passes
    double lam_hi, lam_lo;  // current shift (hi + lo)
    int rqi_done;       // iterations done so far
    int rhint;          // twist index for the next iteration (-1: full factorization)
};

enum : int { KIND_OPEN = 0, KIND_SINGLETON = 1, KIND_CLUSTER = 2, KIND_DROPPED = 3 };

// A cluster of consecutive items sharing one rep (Algorithm 1, line 14).
struct Cluster {
    int a, b;           // item range [a, b)
    int n;              // rep size
    long long pool_off; // offset of the child rep in this level's pool (elements)
    double gapL, gapR;  // distance to the eigenvalues outside the cluster
    int depth;          // depth of the parent rep
    int pad;
};

struct DevCounters {
    unsigned long long qd_bisect;  // qd steps (one row of one transform) in the initial bisection
    unsigned long long qd_refine;  // ... in the refinement bisection of cluster eigenvalues
    unsigned long long qd_rqi;     // ... in the Rayleigh quotient iterations (incl. fallbacks)
    unsigned long long qd_shift;   // ... in building child representations
    unsigned long long qd_steps_low;
    unsigned long long rqi_rows;   // sum over RQI steps of the block order n
    unsigned long long pool_need;  // pool elements requested at the current level
    int nsingle;        // singletons appended to the singleton list
    int ncluster;       // clusters appended at the current level
    int nmember;        // cluster members appended at the current level
    int rqi_iters;
    int fallbacks;
    int noconv;
    int reps_failed;
    int nclusters_total;
    int largest_cluster;
    int d_max;
    int forced;
    int verify_fail;    // low-precision brackets that failed verification and were widened
    int reps_relaxed;   // child reps accepted only under the relaxed growth bound of Eq. (3.6)
    int reps_backtracked;  // clusters processed again from the representation one level up
    int reps_krr_relaxed;  // children accepted with a relative condition estimate above 10 (Eq. (3.7))
    unsigned long long krr_max_bits;  // largest relative condition estimate of an accepted child (bits)
    int nrefine;        // items needing working-precision refinement at the current step
    int npark;          // eigenpairs parked for the next RQI pass
    int nvfix;          // items with a bracket end that failed its first check
};

}  // namespace mrrr
