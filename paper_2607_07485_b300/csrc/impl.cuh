// Internal data model of liblsamg.  Every level is kept in element-block form:
// a list of (element DOF map, dense Gram block G_T) pairs (Prop. 5.1), plus the
// aggregation, closure, interpolation and smoother data built on it (Section 2).
#pragma once
#include "common.cuh"

namespace lsamg {

// Warp 0 lists, in ascending order, the element columns c < n with keep(c) into own[]; returns
// the count through *cnt (visible after the caller's __syncthreads).
template <class F>
__device__ __forceinline__ void warp_compact(int n, int32_t *own, int *cnt, F keep) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int q = 0;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int c = c0 + lane;
        const bool k = c < n && keep(c);
        const unsigned m = __ballot_sync(0xffffffffu, k);
        if (k) own[q + __popc(m & ((1u << lane) - 1u))] = c;
        q += __popc(m);
    }
    if (lane == 0) *cnt = q;
}

struct Level {
    int64_t n = 0;   // DOFs
    int64_t ne = 0;  // elements (level 0) or merged coarse elements (levels >= 1)
    // element maps (CSR) and Gram blocks G_T (row-major m_T x n_T)
    DBuf<int64_t> eptr;
    DBuf<int32_t> eidx;
    DBuf<int64_t> goff;
    DBuf<int32_t> grows;
    DBuf<double> G64;
    DBuf<float> G32;
    // element blocks A_T = G_T^T G_T (row-major n_T x n_T), kept during set-up only
    DBuf<int64_t> aoff;
    DBuf<double> AT;
    // DOF -> elements
    DBuf<int64_t> dptr;
    DBuf<int32_t> didx;
    int64_t nnz = 0;        // structural nnz of the assembled operator
    int64_t nnz_e = 0;      // sum of element map lengths
    int32_t max_nT = 0;     // largest element map
    // aggregation and closure (Section 2 eqs. 2.2-2.5)
    int32_t nagg = 0;
    int32_t maxmult = 0;
    double tau = 0.0;
    DBuf<int32_t> agg;      // [n]
    DBuf<int64_t> eaptr;    // element -> touching aggregates (sorted)
    DBuf<int32_t> eaidx;
    DBuf<int32_t> mult;     // [ne]
    DBuf<int64_t> aeptr;    // aggregate -> elements touching omega_i
    DBuf<int32_t> aeidx;
    DBuf<int64_t> wptr;     // omega_i CSR (sorted DOFs)
    DBuf<int32_t> widx;
    DBuf<int32_t> posw;     // [n] rank of a DOF inside its aggregate
    DBuf<int64_t> Optr;     // Omega_i CSR (sorted DOFs)
    DBuf<int32_t> Oidx;
    DBuf<int32_t> Olpos;    // omega-first local index of each Omega_i entry
    DBuf<int64_t> oeptr;    // aggregate -> elements meeting Omega_i
    DBuf<int32_t> oeidx;
    DBuf<int64_t> oelocoff; // per (aggregate, element) entry: offset of its local positions
    DBuf<int32_t> oeloc;    // sorted-Omega local index of each element DOF, -1 if outside
    std::vector<int32_t> h_nw, h_nO;  // host copies of |omega_i| and |Omega_i|
    // interpolation P = [R_w^T Z_i]
    int64_t nc = 0;
    DBuf<int32_t> k;        // [nagg]
    DBuf<int64_t> off;      // [nagg+1] coarse DOF offsets
    DBuf<int64_t> zoff;     // [nagg+1] offsets of Z_i (row-major |omega_i| x k_i)
    DBuf<double> Z64;
    DBuf<float> Z32;
    std::vector<int32_t> h_k;
    int32_t max_k = 0;                 // largest k_i (shared-memory staging of the interpolation)
    int32_t max_nw = 0;                // largest |omega_i|
    double transfer_bytes[2] = {0.0, 0.0};   // bytes of one restriction (or interpolation), FP32 / FP64
    std::vector<double> h_gap;
    DBuf<int32_t> cgroup;   // [ne] coarse element of each element (-1 if none)
    // multiplicative Schwarz smoother
    int32_t ncol = 0;
    std::vector<int64_t> colptr;  // host: colour c holds colagg[colptr[c]..colptr[c+1])
    DBuf<int32_t> colagg;
    DBuf<int32_t> colour;
    DBuf<int64_t> Loff;     // packed lower-triangular Cholesky factor of A_Omega (row-major)
    DBuf<double> L64;
    DBuf<float> L32;
    // coarsest level: packed lower Cholesky factor of the dense operator
    bool coarsest = false;
    DBuf<double> Ld64;
    DBuf<float> Ld32;
    DBuf<int64_t> cs_ptr, cs_off;   // {0, n} and {0}: the coarsest matrix as one blocked system
    // inverted diagonal blocks of the Schwarz (or coarsest) factors for the blocked triangular
    // solves: block b of system a at Doff[a] + b tri_cb(tri_cb+1)/2, packed lower row-major
    int32_t tri_cb = 64;
    DBuf<int64_t> Doff;
    DBuf<double> Di64;
    // cycle workspaces (allocated for nrhs_ws right-hand sides)
    int32_t nrhs_ws = 0;
    int32_t max_grows_cached = 0;   // largest G_T row count (shared-memory staging size)
    int64_t Omega_total = 0;        // sum of |Omega_i| (Schwarz workspace per right-hand side)
    // algorithmic bytes per application (index 0: FP32, 1: FP64): Gram SpMV, one colour of the
    // Schwarz sweep (per colour), the coarsest triangular solves
    double spmv_bytes[2] = {0, 0};
    double spmv_fmas = 0;               // multiply-adds of one Gram SpMV (two per stored G_T entry)
    std::vector<double> sweep_bytes[2];
    std::vector<int32_t> colmax;        // largest |Omega_i| of each colour
    std::vector<int64_t> colpairs;      // colour c owns pairs [colpairs[c], colpairs[c+1])
    DBuf<int32_t> pair_agg;             // (subdomain, element meeting Omega) pairs by colour
    DBuf<int64_t> pair_ent;             // ... the entry index into oeidx / oelocoff
    double coarse_bytes[2] = {0, 0};
    // wavefront triangular solves: per solve group (the colours, then all subdomains; the
    // coarsest level has one group) the forward and backward task lists (system index within the
    // group's system list, block) at wf_tasks[fwd], [bwd]; per-system flag offsets; the flags
    // (forward, backward) and, after them, an error record (code, item)
    struct WaveGroup {
        int64_t fwd = 0, bwd = 0, ntask = 0;
    };
    std::vector<WaveGroup> wf_groups;
    DBuf<int32_t> wf_tasks;
    DBuf<int64_t> wf_foff;
    DBuf<uint32_t> wf_flags;
    int64_t wf_nflags = 0;
    DBuf<double> b64, x64, r64, ws64;
    DBuf<float> b32, x32, r32, ws32;
};

struct Options {
    lsamg_options o;
};

struct Handle {
    cudaStream_t stream = nullptr;
    lsamg_options opt{};
    std::vector<Level> levels;
    DBuf<int> err;              // device error flag (code, info)
    DBuf<double> coef;          // level-0 element coefficients (for the adjoint gradient)
    int64_t n0 = 0, ne0 = 0;
    int32_t nT0 = 0;
    lsamg_stats stats{};
    // solve workspaces (FP64 outer Krylov vectors)
    int32_t nrhs_ws = 0;
    DBuf<double> kr, kz, kp, kq, kro, kx, dots;
    // V-cycle captured as a CUDA graph (option use_graph), one per precision; re-captured when
    // the right-hand-side count or the cycle workspaces (generation ws_gen) change
    struct CycleGraph {
        cudaGraphExec_t exec = nullptr;
        int32_t nrhs = 0;
        int64_t gen = -1;
    } graphs[2];
    int64_t ws_gen = 0;
    cudaStream_t cap_stream = nullptr;
    Handle() = default;
    Handle(const Handle &) = delete;
    Handle &operator=(const Handle &) = delete;
    ~Handle() {
        for (auto &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

// ------------------------------------------------------------------- graph.cu
void check_input(const Level &L, int *err, cudaStream_t s);
void build_dof_elem(Level &L, int *err, cudaStream_t s);
void aggregate_level(Level &L, int passes, int *err, cudaStream_t s);
void closure_level(Level &L, double tau_c, int closure, int *err, cudaStream_t s);
void colour_level(Level &L, int *err, cudaStream_t s);
int64_t structural_nnz_level0(Level &L, int *err, cudaStream_t s);
int64_t structural_nnz_coarse(const Level &fine, int *err, cudaStream_t s);
void check_err(const int *err, cudaStream_t s, const char *where);

// ------------------------------------------------------------------- setup.cu
void factor_elements(Level &L, int *err, cudaStream_t s);
void local_spectral(Level &L, const lsamg_options &o, int *err, cudaStream_t s, double *flops);
void build_coarse(Level &fine, Level &coarse, int *err, cudaStream_t s, double *flops);
void smoother_setup(Level &L, const lsamg_options &o, int *err, cudaStream_t s, double *flops);
void coarsest_setup(Level &L, int *err, cudaStream_t s, double *flops);
// thread-local message returned by lsamg_last_error
void set_last_error(const std::string &msg);
// invert the diagonal blocks (tri_cb rows) of nsys packed factors; h_n: host orders of the systems
void tri_inverse_setup(int64_t nsys, const int64_t *Optr, const std::vector<int32_t> &h_n, const double *L64,
                       const int64_t *Loff, int cb, DBuf<int64_t> &Doff, DBuf<double> &D64, cudaStream_t s);
// task lists of the wavefront triangular solves: groups[g] lists its systems' orders (in the
// order of the group's system array); nsys_total systems on the level, sysid[g][i] their ids
void wave_setup(Level &L, const std::vector<std::vector<int32_t>> &group_sizes,
                const std::vector<std::vector<int32_t>> &group_ids, const std::vector<int32_t> &all_sizes, int cb,
                cudaStream_t s);
// device error record of the wavefront solves of a level (LSAMG_DEVICE_TIMEOUT if a wait gave up)
void wave_check(const Level &L, cudaStream_t s);

// ------------------------------------------------------------------- cycle.cu
void ensure_cycle_ws(Level &L, int nrhs, cudaStream_t s);
template <class T>
void vcycle(Handle &H, int l, int nrhs, cudaStream_t s);
template <class T>
void gram_spmv(const Level &L, const T *x, T *y, const T *b, int nrhs, cudaStream_t s);
void elem_grad(const Level &L, const double *coef, const double *lam, const double *x, double *g,
               cudaStream_t s);
// FP64 vector helpers used by the Krylov drivers
void vec_dots(const double *a, const double *b, int64_t n, int nrhs, double *out, cudaStream_t s);
void vec_axpy(double *y, const double *x, const double *alpha, int64_t n, int nrhs, double sign,
              cudaStream_t s);
void vec_xpby(double *p, const double *z, const double *beta, int64_t n, int nrhs, cudaStream_t s);
template <class A, class B>
void vec_convert(B *dst, const A *src, int64_t count, cudaStream_t s);

}  // namespace lsamg
