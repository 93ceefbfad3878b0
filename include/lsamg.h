/*
 * lsamg.h -- C ABI of the B300 LS-AMG-DD library (liblsamg.so, sm_103a).
 *
 * LS-AMG-DD (least-squares AMG domain decomposition) preconditioner for SPD
 * systems assembled from element blocks, A = sum_T R_T^T A_T R_T with A_T >= 0
 * (Section 4, eq. 4.1).  The library factors each element block into a local
 * Gram factor so that A = G^T G (Prop. 5.1), builds the aggregates, overlaps and
 * the exact SPSD splitting of Section 2 (eqs. 2.2-2.7), solves the local reduced
 * eigenproblems (eq. 2.9) with the adaptive cutoff tau_cut = c max mult (eq. 2.10)
 * to form the interpolation P, recurses with G_c = G P, and applies a V-cycle with
 * multiplicative Schwarz smoothing and a dense coarsest solve (Section 6 preamble).
 *
 * Conventions for every entry point:
 *  - all sizes are counts of elements (not bytes) unless named *_bytes;
 *  - "device" pointers must be CUDA device (or managed) memory of the current device,
 *    "host" pointers ordinary host memory;
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream); work is
 *    ordered on it and entry points return after the results are complete on the host
 *    side they report (setup and solve synchronise the stream before returning);
 *  - the caller owns every input and output buffer; the handle owns everything the
 *    library derives (hierarchy, workspaces) and lsamg_destroy frees it;
 *  - every call returns an lsamg_status; no C++ exception crosses the ABI; on error a
 *    thread-local message is available from lsamg_last_error().
 */
#ifndef LSAMG_H
#define LSAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSAMG_OK = 0,
    LSAMG_INVALID_ARG = 1,     /* bad size, DOF index out of range, duplicate DOF in an element */
    LSAMG_NOT_SPSD = 2,        /* an element block is not symmetric positive semidefinite */
    LSAMG_SINGULAR = 3,        /* a zero/negative pivot in A_ww, A_Omega or the coarsest matrix */
    LSAMG_NO_CONVERGENCE = 4,  /* maxit reached; x holds the last iterate */
    LSAMG_CUDA = 5,            /* a CUDA runtime call failed */
    LSAMG_OOM = 6,             /* device allocation failed */
    LSAMG_DEVICE_TIMEOUT = 7,  /* a bounded device-side loop gave up */
    LSAMG_NAN = 8,             /* NaN/Inf met in a residual or right-hand side */
    LSAMG_LIMIT = 9            /* a size exceeds a documented implementation limit */
} lsamg_status;

typedef struct lsamg_handle lsamg_handle;

/* Problem description (Section 4 eq. 4.1): n_elems element blocks of uniform size n_T.
 * elem_dofs : [n_elems][n_T] int32, 0-based global DOF ids, distinct within a row.
 * elem_mats : [n_elems][n_T][n_T] float64 row-major, symmetric positive semidefinite.
 * elem_coef : [n_elems] float64 or NULL; if given, A_T = elem_coef[e] * elem_mats[e].
 * on_host   : 0 = the three arrays are device pointers, 1 = host pointers (copied in). */
typedef struct {
    int64_t n_dofs;
    int64_t n_elems;
    int32_t n_T;
    int32_t on_host;
    const int32_t *elem_dofs;
    const double *elem_mats;
    const double *elem_coef;
} lsamg_problem;

/* Options.  Defaults (lsamg_options_default) are the paper's Section 6 choices:
 * tau_c = 0.75 (tau_cut = tau_c * max_j mult(j), eq. 2.10), two aggregation passes on
 * every level, at most 3 levels, stop below min_coarse = 10 DOFs or above
 * max_density = 0.25 structural density; plus the outer-solver choices. */
typedef struct {
    double tau_c;
    int32_t agg_passes;          /* aggregation passes on level 0 */
    int32_t agg_passes_coarse;   /* aggregation passes on levels >= 1 */
    int32_t max_levels;
    int32_t min_coarse;
    double max_density;
    int32_t vcycle_fp32;         /* 1: FP32 V-cycle inside FP64 flexible CG; 0: all-FP64 PCG */
    int32_t maxit;
    double rtol;                 /* stop when ||b - A x||_2 <= rtol ||b||_2 */
    int64_t chunk_bytes;         /* device workspace budget for batched local problems (0 = auto) */
    int32_t use_graph;           /* 1: the V-cycle inside apply / solve runs as a CUDA graph, captured
                                    at first use (per precision and right-hand-side count) and
                                    replayed; off while profiling */
    int32_t verbose;
    int32_t profile;             /* 1: time every kernel class with CUDA events on the stream */
    int32_t large_dense;         /* local problems above this order use multi-CTA kernels (0 = 2048) */
    int32_t split_sweep;         /* Schwarz colours whose largest overlap exceeds this use the blocked
                                    many-CTA sweep, smaller ones one CTA per subdomain (0 = 128) */
    int32_t sweep_block;         /* rows per diagonal block of the blocked triangular solves of the
                                    Schwarz and coarsest factors, 1..64 (0 = 64); fixed at setup */
    int32_t smoother;            /* 0: multiplicative Schwarz, colour-ordered (the paper's tests);
                                    1: additive Schwarz over all subdomains at once, damped by
                                    1 / #colours (the parallel block smoother Section 2 allows) */
    int32_t closure;             /* overlaps Omega_i: 0: G-row closure (Def. 5.3; eq. 2.4, the paper's
                                    method); 1: algebraic A-closure (Def. 5.2): omega_i and every p
                                    with an assembled entry A(q, p) != 0 for some q in omega_i,
                                    entries summed over the elements in ascending element order and
                                    compared with exact zero.  Element DOFs outside Omega_i^A are
                                    left out of the local matrices, so the splitting of Thm 5.6 need
                                    not hold (the Table 2 comparison) */
} lsamg_options;

lsamg_options lsamg_options_default(void);

/* Build the hierarchy.  Inputs may be freed once the call returns.  On success *out
 * receives a new handle (destroy with lsamg_destroy). */
int lsamg_setup(const lsamg_problem *prob, const lsamg_options *opts, void *stream,
                lsamg_handle **out);

/* One V-cycle z = B^{-1} r (Section 2 error propagator E_TG).  r, z: device float64
 * [nrhs][n_dofs] contiguous; precision of the cycle follows opts.vcycle_fp32 unless
 * `fp32` is 0/1 (-1 = follow options). */
int lsamg_apply(lsamg_handle *h, const double *r, double *z, int32_t nrhs, int32_t fp32,
                void *stream);

/* Preconditioned solve of A x = b to ||r|| <= rtol ||b||, x0 = the incoming x if
 * use_x0 != 0 else 0.  b, x: device float64 [nrhs][n_dofs].  iters, relres: host arrays
 * [nrhs] (may be NULL).  mode: 0 = FP64 PCG with the FP64 V-cycle, 1 = FP64 flexible
 * CG(1) with the FP32 V-cycle, 2 = the stationary iteration x <- x + B^{-1}(b - A x) with the
 * FP64 V-cycle, stopped at ||r|| <= rtol ||r_0|| (Section 6 standalone cycles; relres is then
 * ||r|| / ||r_0||), -1 = from options.  Returns LSAMG_NO_CONVERGENCE if any right-hand side
 * missed the tolerance within maxit. */
int lsamg_solve(lsamg_handle *h, const double *b, double *x, int32_t nrhs, int32_t mode,
                int32_t use_x0, void *stream, int32_t *iters, double *relres);

/* Same as lsamg_solve with HOST b and x (copied in and out inside the call). */
int lsamg_solve_host(lsamg_handle *h, const double *b_host, double *x_host, int32_t nrhs,
                     int32_t mode, void *stream, int32_t *iters, double *relres);

/* Gram SpMV y = G_l^T (G_l x) on level l (Section 2 eq. 2.1, Prop. 5.1).  x, y: device
 * arrays of the level's size; fp32 selects the float32 copy of G (x, y then float32). */
int lsamg_gram_spmv(lsamg_handle *h, int32_t level, const void *x, void *y, int32_t fp32,
                    void *stream);

/* Adjoint element gradient g_e = -lambda_e^T K_e x_e for A(theta) = sum_e theta_e K_e,
 * computed as -(G_T lambda_e).(G_T x_e)/theta_e on level 0.  lam, x: device float64
 * [n_dofs]; g: device float64 [n_elems].  Requires elem_coef at setup. */
int lsamg_elem_grad(lsamg_handle *h, const double *lam, const double *x, double *g,
                    void *stream);

/* Hierarchy statistics (Section 6: level sizes, operator and grid complexity). */
typedef struct {
    int32_t n_levels;
    int64_t n[8];
    int64_t nnz[8];
    int64_t n_elems[8];
    int32_t n_agg[8];
    int32_t n_colours[8];
    double tau[8];
    double min_gap[8];           /* min over aggregates of |mu tau_cut - 1| */
    double op_complexity;
    double grid_complexity;
    double setup_seconds;
    double stage_seconds[16];    /* see lsamg_stage_name */
    double setup_flops;          /* counted FP64 flops of the dense local work */
} lsamg_stats;

int lsamg_get_stats(lsamg_handle *h, lsamg_stats *out);
const char *lsamg_stage_name(int32_t i);

/* Copy one derived array of level `level` to host memory (for verification).
 * what: see LSAMG_Q_* below.  If out == NULL or cap_bytes is too small, only
 * *bytes_needed is set and LSAMG_OK returned. */
enum {
    LSAMG_Q_AGG = 0,          /* int32 [n]        aggregate of each DOF                      */
    LSAMG_Q_MULT = 1,         /* int32 [ne]       mult(T) (eq. 2.5)                          */
    LSAMG_Q_OMEGA_PTR = 2,    /* int64 [nagg+1]   Omega_i CSR offsets (eq. 2.4)              */
    LSAMG_Q_OMEGA_IDX = 3,    /* int32 [..]       Omega_i sorted DOF ids                     */
    LSAMG_Q_K = 4,            /* int32 [nagg]     retained modes per aggregate               */
    LSAMG_Q_ZOFF = 5,         /* int64 [nagg+1]   offsets of Z_i blocks                      */
    LSAMG_Q_Z = 6,            /* float64 [..]     Z_i row-major |omega_i| x k_i, rows in
                                                   ascending DOF order of omega_i             */
    LSAMG_Q_CELEM_PTR = 7,    /* int64 [ne_c+1]   next level's element map offsets           */
    LSAMG_Q_CELEM_IDX = 8,    /* int32 [..]       next level's element maps                  */
    LSAMG_Q_GOFF = 9,         /* int64 [ne+1]     this level's G value offsets               */
    LSAMG_Q_GROWS = 10,       /* int32 [ne]       rows m_T of each element's G               */
    LSAMG_Q_G = 11,           /* float64 [..]     this level's G_T row-major m_T x n_T       */
    LSAMG_Q_COLOUR = 12,      /* int32 [nagg]     smoother colour of each subdomain          */
    LSAMG_Q_EPTR = 13,        /* int64 [ne+1]     this level's element map offsets           */
    LSAMG_Q_EIDX = 14,        /* int32 [..]       this level's element maps                  */
    LSAMG_Q_MU = 15,          /* float64 [nagg]   gap |mu tau - 1| per aggregate             */
    LSAMG_Q_CGROUP = 16       /* int32 [ne]       coarse element (merged group) of each element, -1 if none */
};
int lsamg_query(lsamg_handle *h, int32_t level, int32_t what, void *out, int64_t cap_bytes,
                int64_t *bytes_needed);

/* Per-kernel-class device time since the last call (profile option on): out[0] = milliseconds,
 * out[1] = launches, out[2] = algorithmic FLOPs, out[3] = algorithmic bytes.  Collecting
 * synchronises the stream the kernels ran on and resets the counters of every class.
 * lsamg_kernel_stats_all fills out[4 * n_classes]. */
int32_t lsamg_kernel_classes(void);
const char *lsamg_kernel_name(int32_t cls);
int lsamg_kernel_stats_all(double *out);

/* Number of CUDA kernel launches the library has issued in this process. */
int64_t lsamg_launch_count(void);

/* FP64 matrix product on the FP16 tensor cores (no paper counterpart: the dense kernel behind
 * the set-up's Cholesky, triangular-solve, Gram and reduction updates, exposed for verification
 * and for callers with their own dense work).
 *   C = alpha A B^T + beta C,  A: M x K, B: N x K, C: M x N, all column-major FP64 on the device
 *   (A[i + k lda], B[j + k ldb], C[i + j ldc]; lda >= M, ldb >= N, ldc >= M).
 * Each row of A and of B is scaled by a power of two and cut into seven 8-bit integer slices held
 * exactly in FP16; the 28 slice products that carry FP64 precision are accumulated exactly in
 * FP32 by tcgen05.mma (accumulators in tensor memory) over K pieces of 128 and in 64-bit
 * integers across pieces, then rounded once to FP64 and combined with C.  The
 * error of C_ij is a few units of 2^-53 K max_k|A_ik| max_k|B_jk| (the normwise bound of an FP64
 * dot product).  beta == 0 does not read C.  Allocates workspace (about 14 (M + N) K bytes).
 * Returns LSAMG_INVALID_ARG for bad sizes or leading dimensions, LSAMG_DEVICE_TIMEOUT if a staging
 * wait gave up; synchronises `stream`. */
int lsamg_dgemm_nt(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                   const double *B, int64_t ldb, double beta, double *C, int64_t ldc, void *stream);

/* Allocation-free Gram SpMV (the paper has no counterpart: this is a library convenience).
 * It computes the element Gram SpMV
 *   y = sum_T R_T^T G_T^T (G_T x_T)
 * from element factors the caller holds, with no handle.  It is meant for callers that cannot
 * allocate device memory: an application whose device memory is owned by another allocator
 * (a framework's caching pool that has reserved the GPU, so a cudaMalloc from here would fail
 * or fragment it), and code in latency-critical loops, where cudaMalloc / cudaFree would
 * synchronise the device.  The call makes no cudaMalloc, cudaFree or allocating library call.
 * The intermediate G_T x_T lives instead in a file-scope static device array of
 * LSAMG_STATIC_SCRATCH_WORDS doubles (8 MiB, held on every GPU that loads the library until
 * the process exits; the first 32 words are a header).
 *   elem_dofs : device int32 [n_elems][n_T], 0-based DOF ids
 *   G         : device float64 [n_elems][m][n_T] row-major, m rows per element (zero rows allowed)
 *   x, y      : device float64 [n_dofs]; y is overwritten
 * Returns LSAMG_LIMIT, launching nothing, if n_elems * m > LSAMG_STATIC_SCRATCH_WORDS - 32, and
 * LSAMG_INVALID_ARG for bad sizes or a DOF id outside [0, n_dofs) (out-of-range entries are
 * skipped, not read).  The caller must pass buffers of exactly these types and sizes: the
 * library cannot see the extent of a raw pointer.
 * The call reads the error flag back to the host and synchronises `stream` before returning,
 * so it cannot be recorded into a CUDA graph: called while `stream` is capturing, it returns
 * LSAMG_INVALID_ARG without enqueuing anything.  The first call on each device also looks up
 * the array's device address (cudaGetSymbolAddress, with that device current).  The array
 * keeps the last call's contents; each call clears the part that must start at zero (the
 * error flag) and overwrites the rest it reads.  Every call on a device shares the one array,
 * so calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. */
#define LSAMG_STATIC_SCRATCH_WORDS (1 << 20)
int lsamg_gram_spmv_static(int64_t n_dofs, int64_t n_elems, int32_t n_T, int32_t m,
                           const int32_t *elem_dofs, const double *G, const double *x, double *y,
                           void *stream);

void lsamg_destroy(lsamg_handle *h);
const char *lsamg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LSAMG_H */
