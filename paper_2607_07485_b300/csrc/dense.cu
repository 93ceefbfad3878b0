// Batched variable-size FP64 dense kernels (see dense.cuh).  FP64 arithmetic throughout:
// these serve the local eigenproblems whose small eigenvalues select the coarse space.
#include "dense.cuh"
#include "ozaki.cuh"

namespace lsamg {

namespace {

constexpr int NB = 32;          // panel width of the pivoted Cholesky
constexpr double DEPS = 2.220446049250313e-16;

// ------------------------------------------------------------------------- potrf
__global__ void k_maxdiag(const double *base, const int64_t *off, const int32_t *ld,
                          const int32_t *nn, int64_t count, double *md) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const double *A = base + off[b];
    int n = nn[b], L = ld[b];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(A[i + (int64_t)i * L]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; i++) r = fmax(r, w[i]);
        md[b] = r;
    }
}

// diagonal block (PB x PB) of step j0 in shared memory, one CTA per matrix
template <int PB>
__global__ void k_potf2(double *base, const int64_t *off, const int32_t *ld, const int32_t *nn,
                        int64_t count, int j0, int mode, const double *md, int *err) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    int n = nn[b];
    if (j0 >= n) return;
    int bs = min(PB, n - j0);
    int L = ld[b];
    double *A = base + off[b] + (int64_t)j0 + (int64_t)j0 * L;
    __shared__ double s[PB][PB + 1];
    __shared__ double piv;
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        int i = t % bs, j = t / bs;
        s[i][j] = (i >= j) ? A[i + (int64_t)j * L] : 0.0;
    }
    __syncthreads();
    const double tol = (mode == POTRF_PSD) ? (double)n * DEPS * md[b] : 0.0;
    for (int k = 0; k < bs; k++) {
        if (threadIdx.x == 0) {
            double d = s[k][k];
            double p;
            if (mode == POTRF_SPD) {
                if (!(d > 0.0) || !isfinite(d)) {
                    flag_error(err, LSAMG_SINGULAR, (int)b);
                    d = 1.0;
                }
                p = sqrt(d);
            } else {
                p = (d > tol) ? sqrt(d) : 0.0;
            }
            s[k][k] = p;
            piv = (p > 0.0) ? 1.0 / p : 0.0;   // one division per column (the FP64 pipe is scarce)
        }
        __syncthreads();
        const double rp = piv;
        for (int i = k + 1 + threadIdx.x; i < bs; i += blockDim.x) s[i][k] *= rp;
        __syncthreads();
        int m = bs - k - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            int i = k + 1 + t % m, j = k + 1 + t / m;
            if (i >= j) s[i][j] -= s[i][k] * s[j][k];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        int i = t % bs, j = t / bs;
        if (i >= j) A[i + (int64_t)j * L] = s[i][j];
    }
}

// rows below the diagonal block: A21 <- A21 L11^{-T} (one thread per row, the row in registers)
template <int PB>
__global__ void __launch_bounds__(128) k_potrf_panel(double *base, const int64_t *off, const int32_t *ld,
                                                     const int32_t *nn, int64_t count, int j0) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    int n = nn[b];
    if (j0 >= n) return;
    int bs = min(PB, n - j0);
    int L = ld[b];
    double *A = base + off[b];
    __shared__ double l[PB][PB + 1];
    __shared__ double rdiag[PB];
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        int i = t % bs, j = t / bs;
        l[i][j] = (i >= j) ? A[(j0 + i) + (int64_t)(j0 + j) * L] : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < bs; c += blockDim.x) rdiag[c] = (l[c][c] != 0.0) ? 1.0 / l[c][c] : 0.0;
    __syncthreads();
    int r = j0 + bs + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double x[PB];
#pragma unroll
    for (int c = 0; c < PB; c++)
        if (c < bs) x[c] = A[r + (int64_t)(j0 + c) * L];
#pragma unroll
    for (int c = 0; c < PB; c++) {
        if (c < bs) {
            double v = x[c];
#pragma unroll
            for (int k = 0; k < PB; k++)
                if (k < c) v -= x[k] * l[c][k];
            x[c] = v * rdiag[c];
        }
    }
#pragma unroll
    for (int c = 0; c < PB; c++)
        if (c < bs) A[r + (int64_t)(j0 + c) * L] = x[c];
}

// one panel of the pivoted Cholesky (one CTA per matrix); columns j0 .. j0+NB-1 of the block
__global__ void __launch_bounds__(256) k_pstf_panel(double *base, const int64_t *off,
                                                    const int32_t *ld, const int32_t *nfull,
                                                    const int32_t *b0s, const int32_t *bns,
                                                    int64_t count, int j0, int32_t *perm,
                                                    const int64_t *permoff, int32_t *rank,
                                                    double *work, const int64_t *workoff,
                                                    const double *md) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = bns[b];
    if (j0 >= n || rank[b] >= 0) return;  // finished or stopped earlier
    const int L = ld[b], N = nfull[b], g0 = b0s[b];
    double *M = base + off[b];                        // whole view
    double *A = M + (int64_t)g0 + (int64_t)g0 * L;    // the pivoted block
    int32_t *pv = perm + permoff[b];
    double *w = work + workoff[b];
    const double tol = 10.0 * DEPS * md[b];
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ int piv;
    __shared__ double pval;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int i = j0 + threadIdx.x; i < n; i += blockDim.x) w[i] = A[i + (int64_t)i * L];
    __syncthreads();
    const int jend = min(n, j0 + NB);
    for (int j = j0; j < jend; j++) {
        // pivot: largest updated diagonal among rows j..n-1 (first index on ties)
        double bv = -1e300;
        int bi = n;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x)
            if (w[i] > bv || (w[i] == bv && i < bi)) {
                bv = w[i];
                bi = i;
            }
        for (int o = 16; o; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = red_v[0];
            int id = red_i[0];
            for (int q = 1; q < nwarp; q++)
                if (red_v[q] > v || (red_v[q] == v && red_i[q] < id)) {
                    v = red_v[q];
                    id = red_i[q];
                }
            piv = id;
            pval = v;
        }
        __syncthreads();
        const int p = piv;
        if (!(pval > tol)) {
            // numerically zero trailing block: rank j, zero pivots from here on
            for (int i = j + threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)i * L] = 0.0;
            if (threadIdx.x == 0) rank[b] = j;
            return;
        }
        if (p != j) {
            // symmetric interchange of P = g0+j and Q = g0+p inside the stored lower triangle of
            // the whole view (LAPACK pstrf order): row segments left of P, the diagonal, column P
            // against row Q between them, and the columns below Q
            const int P = g0 + j, Q = g0 + p;
            for (int c = threadIdx.x; c < P; c += blockDim.x) {
                double t = M[P + (int64_t)c * L];
                M[P + (int64_t)c * L] = M[Q + (int64_t)c * L];
                M[Q + (int64_t)c * L] = t;
            }
            for (int r = P + 1 + threadIdx.x; r < Q; r += blockDim.x) {
                double t = M[r + (int64_t)P * L];
                M[r + (int64_t)P * L] = M[Q + (int64_t)r * L];
                M[Q + (int64_t)r * L] = t;
            }
            for (int r = Q + 1 + threadIdx.x; r < N; r += blockDim.x) {
                double t = M[r + (int64_t)P * L];
                M[r + (int64_t)P * L] = M[r + (int64_t)Q * L];
                M[r + (int64_t)Q * L] = t;
            }
            if (threadIdx.x == 0) {
                double t = M[P + (int64_t)P * L];
                M[P + (int64_t)P * L] = M[Q + (int64_t)Q * L];
                M[Q + (int64_t)Q * L] = t;
                t = w[j];
                w[j] = w[p];
                w[p] = t;
                int u = pv[j];
                pv[j] = pv[p];
                pv[p] = u;
            }
            __syncthreads();
        }
        const double ljj = sqrt(w[j]), rjj = 1.0 / ljj;
        // column j: l_ij = (a_ij - sum_{k in panel, k<j} l_ik l_jk) / l_jj
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double v = A[i + (int64_t)j * L];
            for (int k = j0; k < j; k++) v -= A[i + (int64_t)k * L] * A[j + (int64_t)k * L];
            v *= rjj;
            A[i + (int64_t)j * L] = v;
            w[i] -= v * v;
        }
        __syncthreads();
        if (threadIdx.x == 0) A[j + (int64_t)j * L] = ljj;
        __syncthreads();
    }
    (void)lane;
}

// ------------------------------------------------------------------------- trsm
constexpr int TB = 64;   // block rows of the blocked triangular solves (the product K)
constexpr int SW = 16;   // right-hand-side columns per CTA of the diagonal-block solve

// X_r = L_rr^{-1} B_r (trans: L_rr^{-T} B_r) for the diagonal block of rows [r0, r0 + TB): a CTA
// per 16 right-hand-side columns, both blocks in shared memory, right-looking substitution.
// Zero diagonal entries (semidefinite factors) give zero solution rows.
__global__ void __launch_bounds__(256) k_trsm_diag(const double *baseL, const int64_t *loff,
                                                   const int32_t *lld, const int32_t *nn,
                                                   double *baseB, const int64_t *boff,
                                                   const int32_t *bld, const int32_t *bcols,
                                                   int64_t count, int r0, int trans) {
    __shared__ double Ls[TB][TB + 1];
    __shared__ double X[TB][SW + 1];
    int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b], ncol = bcols[b];
    const int c0 = blockIdx.x * SW;
    if (r0 >= n || c0 >= ncol) return;
    const int bs = min(TB, n - r0), cs = min(SW, ncol - c0);
    const double *Lm = baseL + loff[b];
    const int LL = lld[b], LB = bld[b];
    double *B = baseB + boff[b] + (int64_t)c0 * LB;
    for (int t = threadIdx.x; t < TB * TB; t += blockDim.x) {
        const int i = t % TB, k = t / TB;
        Ls[i][k] = (i < bs && k < bs && i >= k) ? Lm[(r0 + i) + (int64_t)(r0 + k) * LL] : 0.0;
    }
    for (int t = threadIdx.x; t < TB * SW; t += blockDim.x) {
        const int i = t % TB, c = t / TB;
        X[i][c] = (i < bs && c < cs) ? B[(r0 + i) + (int64_t)c * LB] : 0.0;
    }
    __syncthreads();
    __shared__ double rdiag[TB];
    for (int c = threadIdx.x; c < bs; c += blockDim.x) rdiag[c] = (Ls[c][c] != 0.0) ? 1.0 / Ls[c][c] : 0.0;
    __syncthreads();
    for (int step = 0; step < bs; step++) {
        const int k = trans ? bs - 1 - step : step;
        if (threadIdx.x < SW) X[k][threadIdx.x] *= rdiag[k];
        __syncthreads();
        if (!trans) {
            const int m = bs - k - 1;
            for (int t = threadIdx.x; t < m * SW; t += blockDim.x) {
                const int i = k + 1 + t % m, c = t / m;
                X[i][c] -= Ls[i][k] * X[k][c];
            }
        } else {
            for (int t = threadIdx.x; t < k * SW; t += blockDim.x) {
                const int i = t % k, c = t / k;
                X[i][c] -= Ls[k][i] * X[k][c];
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < TB * SW; t += blockDim.x) {
        const int i = t % TB, c = t / TB;
        if (i < bs && c < cs) B[(r0 + i) + (int64_t)c * LB] = X[i][c];
    }
}

// ------------------------------------------------------------------------- transpose
__global__ void k_transpose(const double *baseS, const int64_t *soff, const int32_t *sld,
                            const int32_t *sn, double *baseD, const int64_t *doff,
                            const int32_t *dld, int64_t count) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    int n = sn[b];
    int T = (n + 31) / 32;
    if ((int)blockIdx.x >= T * T) return;
    int ti = blockIdx.x / T, tj = blockIdx.x % T;
    const double *S = baseS + soff[b];
    double *D = baseD + doff[b];
    int LS = sld[b], LD = dld[b];
    __shared__ double t[32][33];
    for (int u = threadIdx.x; u < 1024; u += blockDim.x) {
        int i = u % 32, j = u / 32;
        int gi = ti * 32 + i, gj = tj * 32 + j;
        t[i][j] = (gi < n && gj < n) ? S[gi + (int64_t)gj * LS] : 0.0;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < 1024; u += blockDim.x) {
        int i = u % 32, j = u / 32;
        int gi = tj * 32 + i, gj = ti * 32 + j;  // D[gi, gj] = S[gj, gi]
        if (gi < n && gj < n) D[gi + (int64_t)gj * LD] = t[j][i];
    }
}


// ------------------------------------------------------------------------- stebz
__device__ int sturm_count(const double *d, const double *e, int n, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
    for (int i = 1; i < n; i++) {
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

// The same count with the division replaced by an approximate reciprocal refined by one Newton
// step (relative error about 2^-40, a few FP64 operations instead of a full division on this
// GPU's slow FP64 pipe).  Used by the bisection only: it perturbs the recurrence like a relative
// change of about 2^-40 in T, far below the 1e-12 ||T|| width the eigenvalues are bisected to.
// |q| >= pivmin keeps e^2 / q finite.
__device__ __forceinline__ double rcp_newton(double q) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
    return fma(r, fma(-q, r, 1.0), r);
}
__device__ int sturm_count_fast(const double *d, const double *e, int n, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
    for (int i = 1; i < n; i++) {
        const double ei = e[i - 1];
        q = fma(-ei * ei, rcp_newton(q), d[i] - x);
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

__device__ double bisect_index(const double *d, const double *e, int n, int j, double lo, double hi,
                               double pivmin, double atol) {
    // smallest x with count(x) >= j + 1, to absolute width atol (= 2 eps ||T||: the accuracy the
    // inverse-iteration shifts need)
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (hi - lo <= atol + pivmin || mid == lo || mid == hi) break;
        if (sturm_count_fast(d, e, n, mid, pivmin) >= j + 1)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

// per matrix: Gershgorin interval (block reduction), pivmin, and k = #eigenvalues below sigma
__global__ void __launch_bounds__(256) k_stebz_count(const double *dd, const double *ee, const int64_t *toff,
                                                     const int32_t *nn, int64_t count, double sigma, int32_t *kout,
                                                     double *bnd) {
    __shared__ double rlo[256], rhi[256], rem[256];
    const int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b];
    const double *d = dd + toff[b], *e = ee + toff[b];
    double lo = 1e300, hi = -1e300, emax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i < n - 1) emax = fmax(emax, e[i] * e[i]);
    }
    rlo[threadIdx.x] = lo;
    rhi[threadIdx.x] = hi;
    rem[threadIdx.x] = emax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            rlo[threadIdx.x] = fmin(rlo[threadIdx.x], rlo[threadIdx.x + o]);
            rhi[threadIdx.x] = fmax(rhi[threadIdx.x], rhi[threadIdx.x + o]);
            rem[threadIdx.x] = fmax(rem[threadIdx.x], rem[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double l = rlo[0], h = rhi[0];
        const double tn = fmax(fabs(l), fabs(h));
        const double pivmin = 2.2250738585072014e-308 * fmax(1.0, rem[0]);
        bnd[3 * b + 0] = l - 2.0 * DEPS * tn * n - pivmin;
        bnd[3 * b + 1] = h + 2.0 * DEPS * tn * n + pivmin;
        bnd[3 * b + 2] = pivmin;
        kout[b] = (n > 0) ? sturm_count(d, e, n, sigma, pivmin) : 0;
    }
}

// one thread per wanted eigenvalue: indices 0 .. k-1 (kept) and k (the first discarded, for the
// gap) of every matrix, spread over the whole GPU
__global__ void __launch_bounds__(128) k_stebz_bisect(const double *dd, const double *ee, const int64_t *toff,
                                                      const int32_t *nn, int64_t count, const int32_t *kk,
                                                      const double *bnd, const int64_t *pre, double *w,
                                                      double *edge) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pre[count]) return;
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int64_t b = lo;
    const int j = (int)(t - pre[b]);
    const int n = nn[b], k = kk[b];
    const double glo = bnd[3 * b], ghi = bnd[3 * b + 1], pivmin = bnd[3 * b + 2];
    // shifts to 1e-12 ||T||: the retained vectors are orthonormalised together afterwards, so
    // eigenvalues closer than that only need to land in their cluster's subspace
    const double lam = bisect_index(dd + toff[b], ee + toff[b], n, j, glo, ghi, pivmin,
                                    1e-12 * fmax(fabs(glo), fabs(ghi)));
    if (j < k) w[toff[b] + j] = lam;
    if (j == k - 1) edge[2 * b] = lam;
    if (j == k) edge[2 * b + 1] = lam;
}

// gap = min |lambda / sigma - 1| over the last kept and the first discarded eigenvalue
__global__ void k_stebz_gap(const int32_t *nn, int64_t count, const int32_t *kk, const double *edge, double sigma,
                            double *gap) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const int n = nn[b], k = kk[b];
    double g = 1e300;
    if (k > 0) g = fmin(g, fabs(edge[2 * b] / sigma - 1.0));
    if (k < n) g = fmin(g, fabs(edge[2 * b + 1] / sigma - 1.0));
    gap[b] = g;
}

// ------------------------------------------------------------------------- stein
__device__ __forceinline__ double urand(uint32_t a, uint32_t b) {
    uint32_t x = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return (double)x * (2.0 / 4294967296.0) - 1.0;
}

// Inverse iteration, one thread per wanted eigenvalue over the whole batch (thread t -> matrix b,
// index j through the prefix `pre` of the counts k).  Three steps of (T - lambda I) x <- x with
// partially pivoted tridiagonal LU from a seeded random start; numerically equal eigenvalues are
// separated by multiples of 10 eps ||T||.  The retained vectors are orthonormalised together
// afterwards (CholeskyQR2): the span matters, not the individual vectors.  Work arrays of matrix b
// at work[woff[b] + (a n + i) k + j] (a = 0..2: the LU factors), coalesced over j.
__global__ void __launch_bounds__(128) k_stein(const double *dd, const double *ee, const int64_t *toff,
                                               const int32_t *nn, int64_t count, const double *wv,
                                               const int32_t *kk, const int64_t *pre, const double *tnorm,
                                               double *baseV, const int64_t *voff, const int32_t *vld,
                                               double *work, const int64_t *woff) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pre[count]) return;
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int64_t b = lo;
    const int j = (int)(t - pre[b]);
    const int n = nn[b], k = kk[b];
    const double *d = dd + toff[b], *e = ee + toff[b], *w = wv + toff[b];
    const double pertol = 10.0 * DEPS * tnorm[b];
    double *dg = work + woff[b], *su = dg + (int64_t)n * k, *su2 = su + (int64_t)n * k;
    double *x = baseV + voff[b] + (int64_t)j * vld[b];     // the vector itself is the work vector
    int q = j;
    while (q > 0 && w[q] - w[q - 1] < pertol) q--;
    const double lam = w[j] + (double)(j - q) * pertol;
    for (int i = 0; i < n; i++) x[i] = urand((uint32_t)j, (uint32_t)i);
    for (int it = 0; it < 3; it++) {
        double mx = 0.0;
        for (int i = 0; i < n; i++) mx = fmax(mx, fabs(x[i]));
        const double sc = (mx > 0.0) ? 1.0 / mx : 1.0;
        double diag = d[0] - lam, sup = (n > 1) ? e[0] : 0.0, rhs = x[0] * sc;
        for (int i = 0; i < n - 1; i++) {
            const double sub = e[i], nd = d[i + 1] - lam, ns = (i + 1 < n - 1) ? e[i + 1] : 0.0;
            const double nrhs = x[i + 1] * sc;
            const int64_t ii = (int64_t)i * k + j;
            if (fabs(diag) >= fabs(sub)) {
                if (diag == 0.0) diag = pertol;
                const double m = sub / diag;
                dg[ii] = diag;
                su[ii] = sup;
                su2[ii] = 0.0;
                x[i] = rhs;
                diag = nd - m * sup;
                sup = ns;
                rhs = nrhs - m * rhs;
            } else {
                const double m = diag / sub;
                dg[ii] = sub;
                su[ii] = nd;
                su2[ii] = ns;
                x[i] = nrhs;
                diag = sup - m * nd;
                sup = -m * ns;
                rhs = rhs - m * nrhs;
            }
        }
        if (diag == 0.0) diag = pertol;
        double x1 = rhs / diag, x2 = 0.0;           // x[i+1], x[i+2] of the back substitution
        x[n - 1] = x1;
        for (int i = n - 2; i >= 0; i--) {
            const int64_t ii = (int64_t)i * k + j;
            const double v = (x[i] - su[ii] * x1 - su2[ii] * x2) / dg[ii];
            x[i] = v;
            x2 = x1;
            x1 = v;
        }
    }
    double nr = 0.0;
    for (int i = 0; i < n; i++) nr += x[i] * x[i];
    const double inv = (nr > 0.0) ? 1.0 / sqrt(nr) : 0.0;
    for (int i = 0; i < n; i++) x[i] *= inv;
}

// ||T||_inf per matrix (the scale of the eigenvalue separation)
__global__ void __launch_bounds__(256) k_tnorm(const double *dd, const double *ee, const int64_t *toff,
                                               const int32_t *nn, int64_t count, double *out) {
    __shared__ double red[256];
    const int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b];
    const double *d = dd + toff[b], *e = ee + toff[b];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        t = fmax(t, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0));
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = fmax(red[0], 1e-300);
}

// ------------------------------------------------------------------------- ormtr (blocked)
constexpr int QB = 64;   // reflectors per block of the back-transformation

// explicit Y of reflector block [j0, j0 + QB): column i = reflector j0 + i (unit at row j0+i+1,
// A's entries below it, zeros above; a zero column past the last reflector), rows j0+1 .. n-1,
// stored at Y[yoff + r + i n] with r the absolute row
__global__ void __launch_bounds__(256) k_ormtr_y(const double *baseA, const int64_t *aoff, const int32_t *ald,
                                                 const int32_t *nn, int64_t count, int j0, double *Y,
                                                 const int64_t *yoff) {
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b];
    if (j0 > n - 2) return;
    const double *A = baseA + aoff[b];
    const int LA = ald[b];
    double *Yb = Y + yoff[b];
    const int R = n - j0 - 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)R * QB;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / R), r = j0 + 1 + (int)(t % R);
        const int j = j0 + i;
        double y = 0.0;
        if (j <= n - 2) {
            if (r == j + 1) y = 1.0;
            else if (r > j + 1) y = A[r + (int64_t)j * LA];
        }
        Yb[r + (int64_t)i * n] = y;
    }
}

// T of the block (forward, columnwise): T(i,i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i)
// with G = Y^T Y; one CTA per matrix, T upper triangular at Tb[b QB^2] column-major
__global__ void __launch_bounds__(64) k_ormtr_t(const int32_t *nn, int64_t count, int j0, const double *tt,
                                                const int64_t *toff, const double *G, double *Tb) {
    __shared__ double T[QB][QB + 1];
    __shared__ double g[QB];
    const int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b];
    if (j0 > n - 2) return;
    const double *Gb = G + b * QB * QB;
    const int c = threadIdx.x;
    for (int i = 0; i < QB; i++) {
        const int j = j0 + i;
        const double ti = (j <= n - 2) ? tt[toff[b] + j] : 0.0;
        if (c < i) g[c] = Gb[c + i * QB];
        __syncthreads();
        // row c of column i: -tau_i sum_{p=c..i-1} T(c, p) g(p)
        if (c < i) {
            double acc = 0.0;
            for (int p2 = c; p2 < i; p2++) acc += T[c][p2] * g[p2];
            T[c][i] = -ti * acc;
        }
        if (c == i) T[i][i] = ti;
        if (c > i) T[c][i] = 0.0;
        __syncthreads();
    }
    double *out = Tb + b * QB * QB;
    for (int i = 0; i < QB; i++) out[c + i * QB] = T[c][i];
}

// Z = T Z for the block (Z: QB x k column-major at Z[zoff])
__global__ void __launch_bounds__(256) k_ormtr_tz(const int32_t *nn, const int32_t *kk, int64_t count, int j0,
                                                  const double *Tb, double *Z, const int64_t *zoff) {
    __shared__ double T[QB][QB + 1];
    __shared__ double zc[4][QB];
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b], k = kk[b];
    if (j0 > n - 2) return;
    const double *Tm = Tb + b * QB * QB;
    for (int t = threadIdx.x; t < QB * QB; t += blockDim.x) T[t % QB][t / QB] = Tm[t];
    __syncthreads();
    const int sub = threadIdx.x >> 6, r = threadIdx.x & 63;
    for (int c0 = blockIdx.x * 4; c0 < k; c0 += gridDim.x * 4) {
        const int c = c0 + sub;
        double *z = Z + zoff[b] + (int64_t)c * QB;
        if (c < k) zc[sub][r] = z[r];
        __syncthreads();
        if (c < k) {
            double acc = 0.0;
            for (int p2 = r; p2 < QB; p2++) acc += T[r][p2] * zc[sub][p2];
            z[r] = acc;
        }
        __syncthreads();
    }
}

}  // namespace

// ============================================================================= host wrappers
namespace {
// A22 -= L21 L21^T (lower triangle) after panel [j0, j0 + w) of every view: L21 = rows
// [j0 + w, n_b) of those columns, all on the tensor cores.  g0[b] offsets the factored block
// inside view b (pivoted Cholesky); skip[b] >= 0 skips a view (factorisation already stopped).
void lower_update(double *base, const MatBatch &A, const std::vector<int32_t> &nb_of,
                  const std::vector<int32_t> *g0, int j0, int w, oz::Workspace &ws, const int32_t *skip,
                  int *err, cudaStream_t s) {
    std::vector<oz::SplitJob> sj;
    std::vector<oz::GemmJob> gj;
    int64_t h = 0, e = 0;
    for (int64_t b = 0; b < A.count; b++) {
        const int n = nb_of[b];
        const int r0 = j0 + w;
        const int m = n - r0;
        if (m <= 0 || j0 >= n) continue;
        const int64_t L = A.h_ld[b], g = g0 ? (*g0)[b] : 0;
        const int64_t base_off = A.h_off[b] + g + g * L;
        oz::SplitJob J{base_off + r0 + (int64_t)j0 * L, 1, L, h, e, m, w};
        sj.push_back(J);
        oz::GemmJob G{h, h, e, e, base_off + r0 + (int64_t)r0 * L, 1, L, m, m, w, 1, (int32_t)b, 0};
        gj.push_back(G);
        h += oz::slice_halves(m, w);
        e += oz::exp_ints(m);
    }
    if (gj.empty()) return;
    ws.reserve(h, e, s);
    oz::split(base, sj, ws.sl.p, ws.ex.p, s);
    oz::gemm(ws.sl.p, ws.ex.p, base, gj, -1.0, 1.0, err, s, skip);
}
// Inside a super panel [s0, s1): after panel [j0, j0 + w), the columns [j0 + w, s1) of the rows
// below are brought up to date: A[j0+w : n, j0+w : s1) -= L[j0+w : n, j0 : j0+w) L[j0+w : s1,
// j0 : j0+w)^T, as a lower-triangular product on the square [j0 + w, s1) and a full one on the
// rows [s1, n) below it.
void panel_update(double *base, const MatBatch &A, int j0, int w, int s1, oz::Workspace &ws, int *err,
                  cudaStream_t s) {
    std::vector<oz::SplitJob> sj;
    std::vector<oz::GemmJob> gj;
    int64_t h = 0, e = 0;
    for (int64_t b = 0; b < A.count; b++) {
        const int n = A.h_n[b];
        const int c0 = j0 + w, c1 = std::min(n, s1);
        if (c0 >= c1) continue;
        const int64_t L = A.h_ld[b], o = A.h_off[b];
        // rows [c0, c1) of the panel: both operands of the square part, B of the rectangle
        const int ms = c1 - c0;
        sj.push_back(oz::SplitJob{o + c0 + (int64_t)j0 * L, 1, L, h, e, ms, w});
        const int64_t hs = h, es = e;
        h += oz::slice_halves(ms, w);
        e += oz::exp_ints(ms);
        gj.push_back(oz::GemmJob{hs, hs, es, es, o + c0 + (int64_t)c0 * L, 1, L, ms, ms, w, 1, 0, 0});
        const int mr = n - c1;
        if (mr > 0) {
            sj.push_back(oz::SplitJob{o + c1 + (int64_t)j0 * L, 1, L, h, e, mr, w});
            gj.push_back(oz::GemmJob{h, hs, e, es, o + c1 + (int64_t)c0 * L, 1, L, mr, ms, w, 0, 0, 0});
            h += oz::slice_halves(mr, w);
            e += oz::exp_ints(mr);
        }
    }
    if (gj.empty()) return;
    ws.reserve(h, e, s);
    oz::split(base, sj, ws.sl.p, ws.ex.p, s);
    oz::gemm(ws.sl.p, ws.ex.p, base, gj, -1.0, 1.0, err, s);
}
}  // namespace

// Two-level blocking: 64-column panels (FP64) inside super panels of SUPER columns.  Within a
// super panel the updates after each panel touch only the super panel's columns (K = 64); the
// trailing matrix beyond it is updated once per super panel with K = SUPER, where the
// tensor-core products run several times faster than at K = 64.
constexpr int SUPER = 256;

void potrf_batched(double *base, const MatBatch &A, PotrfMode mode, int *err, cudaStream_t s) {
    if (A.count == 0 || A.maxn == 0) return;
    constexpr int PB = 64;
    DBuf<double> md;
    md.alloc(A.count, s);
    k_maxdiag<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, md.p);
    CK_LAUNCH();
    oz::Workspace ws;
    for (int j0 = 0; j0 < A.maxn; j0 += PB) {
        int rem = A.maxn - j0 - PB;
        {
            // the FP64 panel: diagonal block and the rows below it (the trailing update is a
            // tensor-core product, timed as its own class)
            double fl = 0.0;
            for (auto v : A.h_n) {
                const double bs = std::min(PB, v - j0), m = std::max(0, v - j0 - PB);
                if (bs > 0) fl += bs * bs * bs / 3.0 + m * bs * bs;
            }
            KTime kt(KC_POTRF, s, fl);
            k_potf2<PB><<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, j0, mode, md.p,
                                                         err);
            CK_LAUNCH();
            if (rem > 0) {
                dim3 gp((unsigned)cdiv(rem, 128), (unsigned)A.count);
                k_potrf_panel<PB><<<gp, 128, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, j0);
                CK_LAUNCH();
            }
        }
        if (rem <= 0) break;
        const int s0 = j0 - j0 % SUPER, s1 = s0 + SUPER;
        if (j0 + PB < s1) {
            panel_update(base, A, j0, PB, s1, ws, err, s);        // inside the super panel
        } else {
            lower_update(base, A, A.h_n, nullptr, s0, SUPER, ws, nullptr, err, s);   // beyond it
        }
    }
}

namespace {
__global__ void k_maxdiag_block(const double *base, const int64_t *off, const int32_t *ld,
                                const int32_t *b0, const int32_t *bn, int64_t count, double *md,
                                int32_t *perm, const int64_t *permoff, int32_t *rank) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int L = ld[b], g0 = b0[b], n = bn[b];
    const double *A = base + off[b] + (int64_t)g0 + (int64_t)g0 * L;
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        m = fmax(m, A[i + (int64_t)i * L]);
        perm[permoff[b] + i] = i;
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; i++) r = fmax(r, w[i]);
        md[b] = r;
        rank[b] = (n == 0) ? 0 : -1;
    }
}
}  // namespace

namespace {
__global__ void k_rank_finish(int32_t *rank, const int32_t *bn, int64_t count) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < count && rank[b] < 0) rank[b] = bn[b];
}
}  // namespace

void pstrf_batched(double *base, const MatBatch &A, const int32_t *b0, const int32_t *bn,
                   const std::vector<int32_t> &h_b0, const std::vector<int32_t> &h_bn,
                   int32_t max_bn, int32_t *perm, const int64_t *permoff, int32_t *rank,
                   int *err, cudaStream_t s) {
    if (A.count == 0 || max_bn == 0) return;
    DBuf<double> md, work;
    DBuf<int64_t> woff;
    md.alloc(A.count, s);
    // work shares the permutation layout (one double per block row)
    int64_t tot = read1(permoff + A.count, s);
    work.alloc(std::max<int64_t>(tot, 1), s);
    k_maxdiag_block<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, b0, bn, A.count, md.p,
                                                       perm, permoff, rank);
    CK_LAUNCH();
    oz::Workspace ws;
    for (int j0 = 0; j0 < max_bn; j0 += NB) {
        {
            KTime kt(KC_PSTRF, s);
            k_pstf_panel<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, b0, bn,
                                                          A.count, j0, perm, permoff, rank, work.p,
                                                          permoff, md.p);
            CK_LAUNCH();
        }
        if (max_bn - j0 - NB <= 0) break;
        lower_update(base, A, h_bn, &h_b0, j0, NB, ws, rank, err, s);
    }
    k_rank_finish<<<(unsigned)cdiv(A.count, 256), 256, 0, s>>>(rank, bn, A.count);
    CK_LAUNCH();
}

void trsm_batched(const double *base_L, const MatBatch &Lb, double *base_B, const MatBatch &Bb,
                  bool trans, cudaStream_t s, int *err) {
    if (Bb.count == 0 || Bb.maxm == 0 || Lb.maxn == 0) return;
    const int nblk = (int)cdiv(Bb.maxn, TB);
    dim3 g((unsigned)cdiv(Bb.maxm, SW), (unsigned)Bb.count);
    oz::Workspace ws;
    // B rows [r0, r1) -= op(L) X over the solved rows [k0, k1) (two-level blocking as in potrf:
    // the rows of the current super block after every 64-row block, the rest once per super
    // block).  Forward: C rows below, A-op = L[r0:r1, k0:k1]; backward (trans): C rows above,
    // A-op = L[k0:k1, r0:r1]^T.  B-op = X[k0:k1, :]^T.
    auto update = [&](int r0, int r1, int k0, int k1) {
        std::vector<oz::SplitJob> sa, sb;
        std::vector<oz::GemmJob> gj;
        int64_t h = 0, e = 0;
        for (int64_t b = 0; b < Bb.count; b++) {
            const int n = Bb.h_n[b], m = Bb.h_m[b];
            const int kk1 = std::min(n, k1), rr1 = std::min(n, r1);
            const int M = rr1 - r0, K = kk1 - k0;
            if (M <= 0 || K <= 0 || m <= 0) continue;
            const int64_t LL = Lb.h_ld[b], LB = Bb.h_ld[b];
            sa.push_back(trans ? oz::SplitJob{Lb.h_off[b] + k0 + (int64_t)r0 * LL, LL, 1, h, e, M, K}
                               : oz::SplitJob{Lb.h_off[b] + r0 + (int64_t)k0 * LL, 1, LL, h, e, M, K});
            const int64_t ha = h, ea = e;
            h += oz::slice_halves(M, K);
            e += oz::exp_ints(M);
            sb.push_back(oz::SplitJob{Bb.h_off[b] + k0, LB, 1, h, e, m, K});
            const int64_t hb = h, eb = e;
            h += oz::slice_halves(m, K);
            e += oz::exp_ints(m);
            gj.push_back(oz::GemmJob{ha, hb, ea, eb, Bb.h_off[b] + r0, 1, LB, M, m, K, 0, 0, 0});
        }
        if (gj.empty()) return;
        ws.reserve(h, e, s);
        oz::split(base_L, sa, ws.sl.p, ws.ex.p, s);
        oz::split(base_B, sb, ws.sl.p, ws.ex.p, s);
        oz::gemm(ws.sl.p, ws.ex.p, base_B, gj, -1.0, 1.0, err, s);
    };
    for (int step = 0; step < nblk; step++) {
        const int kb = trans ? nblk - 1 - step : step;
        const int r0 = kb * TB;
        {
            // the FP64 diagonal-block solves (the rest of B is a tensor-core product)
            double fl = 0.0;
            for (size_t i = 0; i < Bb.h_n.size(); i++) {
                const double bs = std::min(TB, Bb.h_n[i] - r0);
                if (bs > 0) fl += bs * bs * Bb.h_m[i];
            }
            KTime kt(KC_TRSM, s, fl);
            k_trsm_diag<<<g, 256, 0, s>>>(base_L, Lb.off.p, Lb.ld.p, Lb.n.p, base_B, Bb.off.p, Bb.ld.p, Bb.m.p,
                                          Bb.count, r0, trans ? 1 : 0);
            CK_LAUNCH();
        }
        const int s0 = r0 - r0 % SUPER, s1 = s0 + SUPER;
        if (!trans) {
            update(r0 + TB, s1, r0, r0 + TB);                   // rows of this super block
            if (r0 + TB >= s1) update(s1, Bb.maxn, s0, s1);     // below it, K = SUPER
        } else {
            update(s0, r0, r0, r0 + TB);                        // rows of this super block
            if (r0 == s0) update(0, s0, s0, s1);                // above it, K = SUPER
        }
    }
}

void syrk_tn_batched(double *base_C, const MatBatch &Cb, const double *base_W, const MatBatch &Wb,
                     double alpha, bool w_rowmajor, cudaStream_t s, int *err) {
    if (Cb.count == 0 || Cb.maxn == 0) return;
    // C (n x n, full) += alpha W^T W, W: K x n; the split operand is W^T (n rows of length K)
    std::vector<oz::SplitJob> sj;
    std::vector<oz::GemmJob> gj;
    int64_t h = 0, e = 0;
    for (int64_t b = 0; b < Cb.count; b++) {
        const int n = Cb.h_n[b], K = Wb.h_n[b];
        if (n <= 0 || K <= 0) continue;
        const int64_t ld = Wb.h_ld[b];
        const int64_t rs = w_rowmajor ? 1 : ld, ks = w_rowmajor ? ld : 1;   // W(k, i) at k*ks + i*rs
        sj.push_back(oz::SplitJob{Wb.h_off[b], rs, ks, h, e, n, K});
        gj.push_back(oz::GemmJob{h, h, e, e, Cb.h_off[b], 1, Cb.h_ld[b], n, n, K, 0, 0, 0});
        h += oz::slice_halves(n, K);
        e += oz::exp_ints(n);
    }
    if (gj.empty()) return;
    oz::Workspace ws;
    ws.reserve(h, e, s);
    oz::split(base_W, sj, ws.sl.p, ws.ex.p, s);
    oz::gemm(ws.sl.p, ws.ex.p, base_C, gj, alpha, 1.0, err, s);
}

void transpose_batched(const double *base_S, const MatBatch &Sb, double *base_D, const MatBatch &Db,
                       cudaStream_t s) {
    if (Sb.count == 0 || Sb.maxn == 0) return;
    int64_t T = cdiv(Sb.maxn, 32);
    dim3 g((unsigned)(T * T), (unsigned)Sb.count);
    k_transpose<<<g, 256, 0, s>>>(base_S, Sb.off.p, Sb.ld.p, Sb.n.p, base_D, Db.off.p, Db.ld.p,
                                  Sb.count);
    CK_LAUNCH();
}

void stebz_batched(const double *d, const double *e, const int64_t *toff, const int32_t *n,
                   int64_t count, double sigma, int32_t *k, double *w, double *gap,
                   cudaStream_t s) {
    if (count == 0) return;
    KTime kt(KC_STEBZ, s);
    DBuf<double> bnd, edge;
    bnd.alloc(3 * count, s);
    edge.alloc(2 * count, s);
    k_stebz_count<<<(unsigned)count, 256, 0, s>>>(d, e, toff, n, count, sigma, k, bnd.p);
    CK_LAUNCH();
    auto hk = to_host(k, count, s);
    auto hn = to_host(n, count, s);
    std::vector<int64_t> pre(count + 1, 0);
    for (int64_t b = 0; b < count; b++) pre[b + 1] = pre[b] + std::min(hk[b] + 1, hn[b]);
    DBuf<int64_t> dpre;
    upload(dpre, pre, s);
    if (pre[count] > 0) {
        k_stebz_bisect<<<(unsigned)cdiv(pre[count], 128), 128, 0, s>>>(d, e, toff, n, count, k, bnd.p, dpre.p, w,
                                                                      edge.p);
        CK_LAUNCH();
    }
    k_stebz_gap<<<(unsigned)cdiv(count, 256), 256, 0, s>>>(n, count, k, edge.p, sigma, gap);
    CK_LAUNCH();
}

namespace {
__global__ void k_transpose_rect(const double *baseS, const int64_t *soff, const int32_t *sld,
                                 const int32_t *sn, const int32_t *sm, double *baseD, const int64_t *doff,
                                 const int32_t *dld, int64_t count) {
    int64_t b = blockIdx.z;
    if (b >= count) return;
    const int n = sn[b], m = sm[b];
    const int ti = blockIdx.x, tj = blockIdx.y;  // tile rows (of S) / tile cols
    if (ti * 32 >= n || tj * 32 >= m) return;
    const double *S = baseS + soff[b];
    double *D = baseD + doff[b];
    const int LS = sld[b], LD = dld[b];
    __shared__ double t[32][33];
    for (int u = threadIdx.x; u < 1024; u += blockDim.x) {
        const int i = u % 32, j = u / 32;
        const int gi = ti * 32 + i, gj = tj * 32 + j;
        t[i][j] = (gi < n && gj < m) ? S[gi + (int64_t)gj * LS] : 0.0;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < 1024; u += blockDim.x) {
        const int j = u % 32, i = u / 32;        // D[gj, gi] = S[gi, gj]
        const int gi = ti * 32 + i, gj = tj * 32 + j;
        if (gi < n && gj < m) D[gj + (int64_t)gi * LD] = t[i][j];
    }
}

__global__ void k_shift_diag(double *base, const int64_t *off, const int32_t *ld, const int32_t *nn,
                             int64_t count, double rel) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b], L = ld[b];
    double *A = base + off[b];
    __shared__ double tr;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; i++) t = fmax(t, A[i + (int64_t)i * L]);
        tr = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)i * L] += rel * tr;
}
}  // namespace

void transpose_rect_batched(const double *base_S, const MatBatch &Sb, double *base_D, const MatBatch &Db,
                            cudaStream_t s) {
    if (Sb.count == 0 || Sb.maxn == 0 || Sb.maxm == 0) return;
    dim3 g((unsigned)cdiv(Sb.maxn, 32), (unsigned)cdiv(Sb.maxm, 32), (unsigned)Sb.count);
    k_transpose_rect<<<g, 256, 0, s>>>(base_S, Sb.off.p, Sb.ld.p, Sb.n.p, Sb.m.p, base_D, Db.off.p, Db.ld.p,
                                       Sb.count);
    CK_LAUNCH();
}

void cholqr2_batched(double *base_V, const MatBatch &Vb, int *err, cudaStream_t s) {
    if (Vb.count == 0 || Vb.maxm == 0) return;
    const int64_t cnt = Vb.count;
    std::vector<int64_t> goff(cnt + 1, 0), toff(cnt + 1, 0);
    std::vector<int32_t> kk(cnt), nn(cnt);
    for (int64_t i = 0; i < cnt; i++) {
        kk[i] = Vb.h_m[i];
        nn[i] = Vb.h_n[i];
        goff[i + 1] = goff[i] + (int64_t)kk[i] * kk[i];
        toff[i + 1] = toff[i] + (int64_t)kk[i] * nn[i];
    }
    DBuf<double> G, T;
    G.alloc(std::max<int64_t>(goff[cnt], 1), s);
    T.alloc(std::max<int64_t>(toff[cnt], 1), s);
    MatBatch bG, bT, bTt;
    std::vector<int64_t> go(goff.begin(), goff.end() - 1), to(toff.begin(), toff.end() - 1);
    bG.set(go, kk, kk, kk, s);          // k x k Gram / Cholesky factor
    bTt.set(to, kk, kk, nn, s);         // V^T: k rows x n columns, ld k (trsm right-hand side)
    bT.set(to, kk, kk, {}, s);          // destination views for the transposes (ld k)
    MatBatch bV2;                        // V as the source of the transposes: n rows, k columns
    std::vector<int64_t> vo(Vb.h_n.size());
    {
        auto ho = to_host(Vb.off.p, cnt, s);
        auto hl = to_host(Vb.ld.p, cnt, s);
        for (int64_t i = 0; i < cnt; i++) vo[i] = ho[i];
        bV2.set(vo, hl, nn, kk, s);
    }
    MatBatch bTsrc;                      // V^T as the source of the back-transpose: k rows, n cols
    bTsrc.set(to, kk, kk, nn, s);
    for (int pass = 0; pass < 2; pass++) {
        G.zero(s);
        MatBatch bW;                     // W = V as K x k with K = n rows (column-major)
        {
            auto hl = to_host(Vb.ld.p, cnt, s);
            bW.set(vo, hl, nn, kk, s);
        }
        syrk_tn_batched(G.p, bG, base_V, bW, 1.0, false, s);                       // G = V^T V
        if (pass == 0) {
            k_shift_diag<<<(unsigned)cnt, 256, 0, s>>>(G.p, bG.off.p, bG.ld.p, bG.n.p, cnt, 1e-13);
            CK_LAUNCH();
        }
        potrf_batched(G.p, bG, POTRF_SPD, err, s);                                   // G = L L^T
        transpose_rect_batched(base_V, bV2, T.p, bT, s);                             // T = V^T
        trsm_batched(G.p, bG, T.p, bTt, false, s);                                   // T = L^{-1} V^T
        transpose_rect_batched(T.p, bTsrc, base_V, bV2, s);                          // V = T^T
    }
}

void stein_batched(const double *d, const double *e, const int64_t *toff, const int32_t *n,
                   const double *w, const int32_t *k, double *base_V, const MatBatch &Vb, cudaStream_t s) {
    if (Vb.count == 0) return;
    KTime kt(KC_STEIN, s);
    const int64_t cnt = Vb.count;
    std::vector<int64_t> pre(cnt + 1, 0), woff(cnt + 1, 0);
    for (int64_t b = 0; b < cnt; b++) {
        pre[b + 1] = pre[b] + Vb.h_m[b];
        woff[b + 1] = woff[b] + 3 * (int64_t)Vb.h_n[b] * Vb.h_m[b];
    }
    if (pre[cnt] == 0) return;
    DBuf<int64_t> dpre, dwo;
    DBuf<double> work, tn;
    upload(dpre, pre, s);
    upload(dwo, std::vector<int64_t>(woff.begin(), woff.end() - 1), s);
    work.alloc(std::max<int64_t>(woff[cnt], 1), s);
    tn.alloc(cnt, s);
    k_tnorm<<<(unsigned)cnt, 256, 0, s>>>(d, e, toff, n, cnt, tn.p);
    CK_LAUNCH();
    k_stein<<<(unsigned)cdiv(pre[cnt], 128), 128, 0, s>>>(d, e, toff, n, cnt, w, k, dpre.p, tn.p, base_V, Vb.off.p,
                                                          Vb.ld.p, work.p, dwo.p);
    CK_LAUNCH();
}

void ormtr_batched(const double *base_A, const MatBatch &Ab, const double *tau, const int64_t *toff,
                   double *base_V, const MatBatch &Vb, cudaStream_t s, int *err) {
    if (Vb.count == 0 || Vb.maxm == 0) return;
    // V = Q V, Q = H_0 ... H_{n-2} in blocks of QB reflectors, last block first; each block is
    // I - Y T Y^T (compact WY), applied as V -= Y (T (Y^T V)) with the two large products on the
    // tensor cores
    const int64_t cnt = Vb.count;
    std::vector<int64_t> yoff(cnt + 1, 0), zoff(cnt + 1, 0);
    for (int64_t b = 0; b < cnt; b++) {
        yoff[b + 1] = yoff[b] + (int64_t)Vb.h_n[b] * QB;
        zoff[b + 1] = zoff[b] + (int64_t)QB * std::max(Vb.h_m[b], 1);
    }
    DBuf<double> Y, Z, G, T;
    DBuf<int64_t> dyo, dzo;
    Y.alloc(std::max<int64_t>(yoff[cnt], 1), s);
    Z.alloc(std::max<int64_t>(zoff[cnt], 1), s);
    G.alloc(cnt * QB * QB, s);
    T.alloc(cnt * QB * QB, s);
    upload(dyo, std::vector<int64_t>(yoff.begin(), yoff.end() - 1), s);
    upload(dzo, std::vector<int64_t>(zoff.begin(), zoff.end() - 1), s);
    oz::Workspace ws;
    const int nblk = (int)cdiv(std::max(Vb.maxn - 1, 1), QB);
    for (int p = nblk - 1; p >= 0; p--) {
        const int j0 = p * QB;
        dim3 gy((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv((int64_t)Vb.maxn * QB, 256), 64)),
                (unsigned)cnt);
        {
            KTime kt(KC_ORMTR, s);
            k_ormtr_y<<<gy, 256, 0, s>>>(base_A, Ab.off.p, Ab.ld.p, Ab.n.p, cnt, j0, Y.p, dyo.p);
            CK_LAUNCH();
        }
        // operands: Y^T (QB rows of length R), V^T (k rows of length R), Y (R rows of length QB)
        std::vector<oz::SplitJob> sy, sv;
        std::vector<oz::GemmJob> gg, gz, gv;
        int64_t h = 0, e = 0;
        for (int64_t b = 0; b < cnt; b++) {
            const int n = Vb.h_n[b], k = Vb.h_m[b];
            if (j0 > n - 2 || k <= 0) continue;
            const int R = n - j0 - 1;
            sy.push_back(oz::SplitJob{yoff[b] + j0 + 1, n, 1, h, e, QB, R});
            const int64_t hy = h, ey = e;
            h += oz::slice_halves(QB, R);
            e += oz::exp_ints(QB);
            sv.push_back(oz::SplitJob{Vb.h_off[b] + j0 + 1, Vb.h_ld[b], 1, h, e, k, R});
            const int64_t hv = h, ev = e;
            h += oz::slice_halves(k, R);
            e += oz::exp_ints(k);
            gg.push_back(oz::GemmJob{hy, hy, ey, ey, b * QB * QB, 1, QB, QB, QB, R, 0, 0, 0});
            gz.push_back(oz::GemmJob{hy, hv, ey, ev, zoff[b], 1, QB, QB, k, R, 0, 0, 0});
        }
        if (gg.empty()) continue;
        ws.reserve(h, e, s);
        oz::split(Y.p, sy, ws.sl.p, ws.ex.p, s);
        oz::split(base_V, sv, ws.sl.p, ws.ex.p, s);
        oz::gemm(ws.sl.p, ws.ex.p, G.p, gg, 1.0, 0.0, err, s);
        oz::gemm(ws.sl.p, ws.ex.p, Z.p, gz, 1.0, 0.0, err, s);
        {
            KTime kt(KC_ORMTR, s);
            k_ormtr_t<<<(unsigned)cnt, QB, 0, s>>>(Vb.n.p, cnt, j0, tau, toff, G.p, T.p);
            CK_LAUNCH();
            dim3 gt((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(Vb.maxm, 4), 32)), (unsigned)cnt);
            k_ormtr_tz<<<gt, 256, 0, s>>>(Vb.n.p, Vb.m.p, cnt, j0, T.p, Z.p, dzo.p);
            CK_LAUNCH();
        }
        // V(j0+1:, :) -= Y Z
        std::vector<oz::SplitJob> s1, s2;
        h = 0;
        e = 0;
        for (int64_t b = 0; b < cnt; b++) {
            const int n = Vb.h_n[b], k = Vb.h_m[b];
            if (j0 > n - 2 || k <= 0) continue;
            const int R = n - j0 - 1;
            s1.push_back(oz::SplitJob{yoff[b] + j0 + 1, 1, n, h, e, R, QB});
            const int64_t ha = h, ea = e;
            h += oz::slice_halves(R, QB);
            e += oz::exp_ints(R);
            s2.push_back(oz::SplitJob{zoff[b], QB, 1, h, e, k, QB});
            const int64_t hb = h, eb = e;
            h += oz::slice_halves(k, QB);
            e += oz::exp_ints(k);
            gv.push_back(oz::GemmJob{ha, hb, ea, eb, Vb.h_off[b] + j0 + 1, 1, Vb.h_ld[b], R, k, QB, 0, 0, 0});
        }
        ws.reserve(h, e, s);
        oz::split(Y.p, s1, ws.sl.p, ws.ex.p, s);
        oz::split(Z.p, s2, ws.sl.p, ws.ex.p, s);
        oz::gemm(ws.sl.p, ws.ex.p, base_V, gv, -1.0, 1.0, err, s);
    }
}

}  // namespace lsamg
