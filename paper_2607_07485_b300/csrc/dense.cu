// Batched variable-size FP64 dense kernels (see dense.cuh).  FP64 arithmetic throughout:
// these serve the local eigenproblems whose small eigenvalues select the coarse space.
#include "dense.cuh"

namespace lsamg {

namespace {

constexpr int NB = 32;          // panel width of the blocked Cholesky / TRSM
constexpr int TT = 64;          // output tile of the update kernels
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

__global__ void k_potf2(double *base, const int64_t *off, const int32_t *ld, const int32_t *nn,
                        int64_t count, int j0, int mode, const double *md, int *err) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    int n = nn[b];
    if (j0 >= n) return;
    int bs = min(NB, n - j0);
    int L = ld[b];
    double *A = base + off[b] + (int64_t)j0 + (int64_t)j0 * L;
    __shared__ double s[NB][NB + 1];
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
            piv = p;
        }
        __syncthreads();
        double p = piv;
        for (int i = k + 1 + threadIdx.x; i < bs; i += blockDim.x) s[i][k] = (p > 0.0) ? s[i][k] / p : 0.0;
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

// rows below the diagonal block: A21 <- A21 L11^{-T}
__global__ void k_potrf_panel(double *base, const int64_t *off, const int32_t *ld,
                              const int32_t *nn, int64_t count, int j0) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    int n = nn[b];
    if (j0 >= n) return;
    int bs = min(NB, n - j0);
    int L = ld[b];
    double *A = base + off[b];
    __shared__ double l[NB][NB + 1];
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        int i = t % bs, j = t / bs;
        l[i][j] = (i >= j) ? A[(j0 + i) + (int64_t)(j0 + j) * L] : 0.0;
    }
    __syncthreads();
    int r = j0 + bs + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double x[NB];
#pragma unroll
    for (int c = 0; c < NB; c++)
        if (c < bs) x[c] = A[r + (int64_t)(j0 + c) * L];
#pragma unroll
    for (int c = 0; c < NB; c++) {
        if (c < bs) {
            double v = x[c];
#pragma unroll
            for (int k = 0; k < NB; k++)
                if (k < c) v -= x[k] * l[c][k];
            x[c] = (l[c][c] != 0.0) ? v / l[c][c] : 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < NB; c++)
        if (c < bs) A[r + (int64_t)(j0 + c) * L] = x[c];
}

__device__ __forceinline__ void tri_index(int t, int &ti, int &tj) {
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) i++;
    while (i * (i + 1) / 2 > t) i--;
    ti = i;
    tj = t - i * (i + 1) / 2;
}

// trailing update A22 -= L21 L21^T on lower tiles
__global__ void __launch_bounds__(256) k_potrf_update(double *base, const int64_t *off,
                                                      const int32_t *ld, const int32_t *nn,
                                                      int64_t count, int j0, const int32_t *b0,
                                                      const int32_t *stop, int full) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    if (stop && stop[b] >= 0) return;  // pivoted factorisation already truncated
    int n = nn[b];
    int bs = min(NB, n - j0);
    int r0 = j0 + min(NB, n - j0);
    int m = n - r0;
    if (m <= 0 || bs <= 0) return;
    int T = (m + TT - 1) / TT;
    int ti, tj;
    if (full) {
        if ((int64_t)blockIdx.x >= (int64_t)T * T) return;
        ti = blockIdx.x / T;
        tj = blockIdx.x % T;
    } else {
        if ((int64_t)blockIdx.x >= (int64_t)T * (T + 1) / 2) return;
        tri_index(blockIdx.x, ti, tj);
    }
    int L = ld[b];
    const int o0 = b0 ? b0[b] : 0;
    double *A = base + off[b] + (int64_t)o0 + (int64_t)o0 * L;
    __shared__ double As[NB][TT + 1];
    __shared__ double Bs[NB][TT + 1];
    int ib = r0 + ti * TT, jb = r0 + tj * TT;
    for (int t = threadIdx.x; t < NB * TT; t += blockDim.x) {
        int rr = t % TT, k = t / TT;
        int gi = ib + rr, gj = jb + rr;
        As[k][rr] = (k < bs && gi < n) ? A[gi + (int64_t)(j0 + k) * L] : 0.0;
        Bs[k][rr] = (k < bs && gj < n) ? A[gj + (int64_t)(j0 + k) * L] : 0.0;
    }
    __syncthreads();
    int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[4][4] = {};
#pragma unroll 8
    for (int k = 0; k < NB; k++) {
        double a[4], c[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            a[u] = As[k][ty * 4 + u];
            c[u] = Bs[k][tx * 4 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], c[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            int gi = ib + ty * 4 + u, gj = jb + tx * 4 + v;
            if (gi < n && gj < n && (full || gi >= gj)) A[gi + (int64_t)gj * L] -= acc[u][v];
        }
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
        const double ljj = sqrt(w[j]);
        // column j: l_ij = (a_ij - sum_{k in panel, k<j} l_ik l_jk) / l_jj
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double v = A[i + (int64_t)j * L];
            for (int k = j0; k < j; k++) v -= A[i + (int64_t)k * L] * A[j + (int64_t)k * L];
            v /= ljj;
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
constexpr int SW = 32;  // right-hand-side strip width

__global__ void __launch_bounds__(256) k_trsm(const double *baseL, const int64_t *loff,
                                              const int32_t *lld, const int32_t *nn,
                                              double *baseB, const int64_t *boff,
                                              const int32_t *bld, const int32_t *bcols,
                                              int64_t count, int trans) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    int n = nn[b];
    int ncol = bcols[b];
    int c0 = blockIdx.x * SW;
    if (c0 >= ncol || n <= 0) return;
    int cs = min(SW, ncol - c0);
    const double *Lm = baseL + loff[b];
    int LL = lld[b];
    double *B = baseB + boff[b] + (int64_t)c0 * bld[b];
    int LB = bld[b];
    __shared__ double Ls[NB][NB + 1];
    __shared__ double Xs[NB][SW + 1];
    __shared__ double acc[NB][SW + 1];
    int nrb = (n + NB - 1) / NB;
    for (int step = 0; step < nrb; step++) {
        int rb = trans ? (nrb - 1 - step) : step;
        int r0 = rb * NB, rs = min(NB, n - r0);
        for (int t = threadIdx.x; t < NB * SW; t += blockDim.x) {
            int i = t % NB, c = t / NB;
            acc[i][c] = (i < rs && c < cs) ? B[(r0 + i) + (int64_t)c * LB] : 0.0;
        }
        __syncthreads();
        int kb0 = trans ? rb + 1 : 0, kb1 = trans ? nrb : rb;
        for (int kb = kb0; kb < kb1; kb++) {
            int k0 = kb * NB, ks = min(NB, n - k0);
            for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
                int i = t % NB, k = t / NB;
                double v = 0.0;
                if (!trans) {
                    if (i < rs && k < ks) v = Lm[(r0 + i) + (int64_t)(k0 + k) * LL];  // L[r0+i, k0+k]
                } else {
                    if (i < rs && k < ks) v = Lm[(k0 + k) + (int64_t)(r0 + i) * LL];  // L[k0+k, r0+i]
                }
                Ls[i][k] = v;
            }
            for (int t = threadIdx.x; t < NB * SW; t += blockDim.x) {
                int k = t % NB, c = t / NB;
                Xs[k][c] = (k < ks && c < cs) ? B[(k0 + k) + (int64_t)c * LB] : 0.0;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < NB * SW; t += blockDim.x) {
                int i = t % NB, c = t / NB;
                double v = acc[i][c];
#pragma unroll 8
                for (int k = 0; k < NB; k++) v -= Ls[i][k] * Xs[k][c];
                acc[i][c] = v;
            }
            __syncthreads();
        }
        // diagonal block
        for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
            int i = t % NB, k = t / NB;
            Ls[i][k] = (i < rs && k < rs && i >= k) ? Lm[(r0 + i) + (int64_t)(r0 + k) * LL] : 0.0;
        }
        __syncthreads();
        if (threadIdx.x < cs) {
            int c = threadIdx.x;
            if (!trans) {
                for (int i = 0; i < rs; i++) {
                    double v = acc[i][c];
                    for (int k = 0; k < i; k++) v -= Ls[i][k] * acc[k][c];
                    acc[i][c] = (Ls[i][i] != 0.0) ? v / Ls[i][i] : 0.0;
                }
            } else {
                for (int i = rs - 1; i >= 0; i--) {
                    double v = acc[i][c];
                    for (int k = i + 1; k < rs; k++) v -= Ls[k][i] * acc[k][c];
                    acc[i][c] = (Ls[i][i] != 0.0) ? v / Ls[i][i] : 0.0;
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NB * SW; t += blockDim.x) {
            int i = t % NB, c = t / NB;
            if (i < rs && c < cs) B[(r0 + i) + (int64_t)c * LB] = acc[i][c];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------- syrk (C -= W^T W)
__global__ void __launch_bounds__(256) k_syrk_tn(double *baseC, const int64_t *coff,
                                                 const int32_t *cld, const int32_t *cn,
                                                 const double *baseW, const int64_t *woff,
                                                 const int32_t *wld, const int32_t *wk,
                                                 int64_t count, double alpha, int wrow) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    int n = cn[b], K = wk[b];
    int T = (n + TT - 1) / TT;
    if ((int)blockIdx.x >= T * T || K <= 0) return;
    int ti = blockIdx.x / T, tj = blockIdx.x % T;
    double *C = baseC + coff[b];
    int LC = cld[b];
    const double *W = baseW + woff[b];
    const int64_t rs = wrow ? (int64_t)wld[b] : 1, cs = wrow ? 1 : (int64_t)wld[b];
    __shared__ double As[NB][TT + 1];
    __shared__ double Bs[NB][TT + 1];
    int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[4][4] = {};
    int ib = ti * TT, jb = tj * TT;
    for (int k0 = 0; k0 < K; k0 += NB) {
        for (int t = threadIdx.x; t < NB * TT; t += blockDim.x) {
            int k = t % NB, rr = t / NB;
            int gk = k0 + k;
            As[k][rr] = (gk < K && ib + rr < n) ? W[gk * rs + (int64_t)(ib + rr) * cs] : 0.0;
            Bs[k][rr] = (gk < K && jb + rr < n) ? W[gk * rs + (int64_t)(jb + rr) * cs] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < NB; k++) {
            double a[4], c[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                a[u] = As[k][ty * 4 + u];
                c[u] = Bs[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], c[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            int gi = ib + ty * 4 + u, gj = jb + tx * 4 + v;
            if (gi < n && gj < n) C[gi + (int64_t)gj * LC] += alpha * acc[u][v];
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

// ------------------------------------------------------------------------- sytd2
__device__ double block_sum(double v, double *red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; i++) r += red[i];
    return r;
}

// One CTA per matrix.  Per column j: Householder vector v (staged in shared memory), the
// symmetric product p = tau A22 v in ONE sweep over the stored lower triangle (each warp owns
// columns: column sums reduce in registers, the transposed contributions accumulate in shared
// memory with atomics), then the rank-2 update A22 -= v w^T + w v^T.
constexpr int SYTD2_THREADS = 512;

__global__ void __launch_bounds__(512) k_sytd2(double *base, const int64_t *off, const int32_t *ld,
                                               const int32_t *nn, int64_t count, double *dd,
                                               double *ee, double *tt, const int64_t *toff,
                                               double *pwork, const int64_t *pwoff, int use_smem) {
    extern __shared__ double smv[];
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b];
    const int L = ld[b];
    double *A = base + off[b];
    double *d = dd + toff[b], *e = ee + toff[b], *tau = tt + toff[b];
    double *tbuf = smv;                                   // one 32 x 33 tile buffer per warp
    double *p = use_smem ? smv + (blockDim.x / 32) * 32 * 33 : pwork + 2 * pwoff[b];
    double *v = use_smem ? p + n : pwork + 2 * pwoff[b] + n;
    __shared__ double red[32];
    __shared__ double sh_tau, sh_scale;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int j = 0; j < n - 1; j++) {
        const int m = n - j - 1;
        double *x = A + (j + 1) + (int64_t)j * L;
        double sig = 0.0;
        for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) sig += x[i] * x[i];
        sig = block_sum(sig, red);
        if (threadIdx.x == 0) {
            const double alpha = x[0];
            d[j] = A[j + (int64_t)j * L];
            if (sig == 0.0) {
                sh_tau = 0.0;
                e[j] = alpha;
                sh_scale = 0.0;
            } else {
                const double beta = -copysign(sqrt(alpha * alpha + sig), alpha);
                sh_tau = (beta - alpha) / beta;
                sh_scale = 1.0 / (alpha - beta);
                e[j] = beta;
            }
            tau[j] = sh_tau;
        }
        __syncthreads();
        const double tj = sh_tau, sc = sh_scale;
        if (tj == 0.0) continue;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double vi = (i == 0) ? 1.0 : x[i] * sc;
            v[i] = vi;
            if (i > 0) x[i] = vi;
            p[i] = 0.0;
        }
        __syncthreads();
        double *A22 = A + (j + 1) + (int64_t)(j + 1) * L;
        // p = A22 v, tiled: each warp owns row blocks; a 32 x 32 tile is loaded coalesced into
        // the warp's shared buffer, row sums stay in registers, column sums (the transposed
        // half) go out with 32 shared atomics per tile
        {
            double(*tile)[33] = reinterpret_cast<double(*)[33]>(tbuf + (int64_t)warp * 32 * 33);
            const int nbk = (m + 31) / 32;
            for (int rb = warp; rb < nbk; rb += nwarp) {
                const int r0 = rb * 32;
                double rsum = 0.0;
                for (int cb = 0; cb <= rb; cb++) {
                    const int c0 = cb * 32;
                    for (int c = 0; c < 32; c++) {
                        const int gr = r0 + lane, gc = c0 + c;
                        double a = 0.0;
                        if (gr < m && gc < m && gr >= gc) a = A22[gr + (int64_t)gc * L];
                        tile[lane][c] = a;
                    }
                    __syncwarp();
                    // row sums: lane = row (diagonal tile: its stored lower part, diagonal included)
                    for (int c = 0; c < 32; c++) {
                        const int gc = c0 + c;
                        if (gc < m) rsum += tile[lane][c] * v[gc];
                    }
                    // column sums: lane = column, strictly below the diagonal
                    double csum = 0.0;
                    for (int i = 0; i < 32; i++) {
                        const int gr = r0 + i;
                        if (gr < m && (cb != rb || i > lane)) csum += tile[i][lane] * v[gr];
                    }
                    if (c0 + lane < m && csum != 0.0) atomicAdd(&p[c0 + lane], csum);
                    __syncwarp();
                }
                if (r0 + lane < m) atomicAdd(&p[r0 + lane], rsum);
            }
        }
        __syncthreads();
        double pv = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            p[i] *= tj;
            pv += p[i] * v[i];
        }
        pv = block_sum(pv, red);
        const double kk = -0.5 * tj * pv;
        for (int i = threadIdx.x; i < m; i += blockDim.x) p[i] += kk * v[i];  // w
        __syncthreads();
        for (int c = warp; c < m; c += nwarp) {
            const double vc = v[c], wc = p[c];
            double *col = A22 + (int64_t)c * L;
            for (int r = c + lane; r < m; r += 32) col[r] -= v[r] * wc + p[r] * vc;
        }
        __syncthreads();
        if (threadIdx.x == 0) x[0] = e[j];
        __syncthreads();
    }
    if (threadIdx.x == 0 && n > 0) d[n - 1] = A[(n - 1) + (int64_t)(n - 1) * L];
}

// ---- multi-CTA tridiagonalisation for large matrices (one column per group of launches)
constexpr int TRT = 64;          // tile of the symmetric product / rank-2 update

// Householder vector of column j for every large matrix; restores the previous subdiagonal
__global__ void __launch_bounds__(256) k_tr_house(double *base, const int64_t *off, const int32_t *ld,
                                                  const int32_t *nn, int64_t count, int j, double *dd,
                                                  double *ee, double *tt, const int64_t *toff,
                                                  double *vbuf, double *pbuf, const int64_t *voff) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b], L = ld[b];
    double *A = base + off[b];
    double *d = dd + toff[b], *e = ee + toff[b], *tau = tt + toff[b];
    if (j > 0 && j <= n - 1 && threadIdx.x == 0) A[j + (int64_t)(j - 1) * L] = e[j - 1];
    if (j >= n - 1) {
        if (j == n - 1 && threadIdx.x == 0) d[n - 1] = A[(n - 1) + (int64_t)(n - 1) * L];
        return;
    }
    const int m = n - j - 1;
    double *x = A + (j + 1) + (int64_t)j * L;
    double *v = vbuf + voff[b], *p = pbuf + voff[b];
    __shared__ double red[32];
    __shared__ double sh_tau, sh_scale;
    double sig = 0.0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) sig += x[i] * x[i];
    sig = block_sum(sig, red);
    if (threadIdx.x == 0) {
        const double alpha = x[0];
        d[j] = A[j + (int64_t)j * L];
        if (sig == 0.0) {
            sh_tau = 0.0;
            sh_scale = 0.0;
            e[j] = alpha;
        } else {
            const double beta = -copysign(sqrt(alpha * alpha + sig), alpha);
            sh_tau = (beta - alpha) / beta;
            sh_scale = 1.0 / (alpha - beta);
            e[j] = beta;
        }
        tau[j] = sh_tau;
    }
    __syncthreads();
    const double sc = sh_scale, tj = sh_tau;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double vi = (i == 0) ? 1.0 : x[i] * sc;
        if (i > 0) x[i] = vi;
        v[i] = (tj == 0.0) ? 0.0 : vi;
        p[i] = 0.0;
    }
}

// p += A22 v over the stored lower triangle, one 64 x 64 tile per CTA (atomics into p)
__global__ void __launch_bounds__(128) k_tr_symv(const double *base, const int64_t *off,
                                                 const int32_t *ld, const int32_t *nn, int64_t count,
                                                 int j, const double *vbuf, double *pbuf,
                                                 const int64_t *voff, const double *tt,
                                                 const int64_t *toff) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b];
    const int m = n - j - 1;
    if (m <= 0 || tt[toff[b] + j] == 0.0) return;
    const int T = (m + TRT - 1) / TRT;
    if ((int64_t)blockIdx.x >= (int64_t)T * (T + 1) / 2) return;
    int ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int L = ld[b];
    const double *A22 = base + off[b] + (j + 1) + (int64_t)(j + 1) * L;
    const double *v = vbuf + voff[b];
    double *p = pbuf + voff[b];
    __shared__ double T_[TRT][TRT + 1];
    __shared__ double vr[TRT], vc[TRT];
    const int r0 = ti * TRT, c0 = tj * TRT;
    for (int t = threadIdx.x; t < TRT * TRT; t += blockDim.x) {
        const int rr = t % TRT, cc = t / TRT;
        const int gr = r0 + rr, gc = c0 + cc;
        double a = 0.0;
        if (gr < m && gc < m && gr >= gc) a = A22[gr + (int64_t)gc * L];
        T_[rr][cc] = a;
    }
    for (int t = threadIdx.x; t < TRT; t += blockDim.x) {
        vr[t] = (r0 + t < m) ? v[r0 + t] : 0.0;
        vc[t] = (c0 + t < m) ? v[c0 + t] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < TRT) {
        const int rr = threadIdx.x;
        double sacc = 0.0;
        for (int cc = 0; cc < TRT; cc++) sacc += T_[rr][cc] * vc[cc];
        if (r0 + rr < m) atomicAdd(&p[r0 + rr], sacc);
    } else {
        const int cc = threadIdx.x - TRT;
        double sacc = 0.0;
        for (int rr = 0; rr < TRT; rr++)
            if (ti != tj || rr > cc) sacc += T_[rr][cc] * vr[rr];
        if (c0 + cc < m) atomicAdd(&p[c0 + cc], sacc);
    }
}

// p <- w = tau p - (tau^2/2)(p^T v) v
__global__ void __launch_bounds__(256) k_tr_w(const int32_t *nn, int64_t count, int j, const double *vbuf,
                                              double *pbuf, const int64_t *voff, const double *tt,
                                              const int64_t *toff) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int m = nn[b] - j - 1;
    if (m <= 0) return;
    const double tj = tt[toff[b] + j];
    if (tj == 0.0) return;
    const double *v = vbuf + voff[b];
    double *p = pbuf + voff[b];
    __shared__ double red[32];
    double pv = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) pv += p[i] * v[i];
    pv = block_sum(pv, red) * tj;
    const double kk = -0.5 * tj * pv;
    for (int i = threadIdx.x; i < m; i += blockDim.x) p[i] = tj * p[i] + kk * v[i];
}

// A22 -= v w^T + w v^T on the stored lower triangle, one 64 x 64 tile per CTA
__global__ void __launch_bounds__(256) k_tr_update(double *base, const int64_t *off, const int32_t *ld,
                                                   const int32_t *nn, int64_t count, int j,
                                                   const double *vbuf, const double *pbuf,
                                                   const int64_t *voff, const double *tt,
                                                   const int64_t *toff) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    const int m = nn[b] - j - 1;
    if (m <= 0 || tt[toff[b] + j] == 0.0) return;
    const int T = (m + TRT - 1) / TRT;
    if ((int64_t)blockIdx.x >= (int64_t)T * (T + 1) / 2) return;
    int ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int L = ld[b];
    double *A22 = base + off[b] + (j + 1) + (int64_t)(j + 1) * L;
    const double *v = vbuf + voff[b], *w = pbuf + voff[b];
    const int r0 = ti * TRT, c0 = tj * TRT;
    for (int t = threadIdx.x; t < TRT * TRT; t += blockDim.x) {
        const int rr = t % TRT, cc = t / TRT;
        const int gr = r0 + rr, gc = c0 + cc;
        if (gr < m && gc < m && gr >= gc) A22[gr + (int64_t)gc * L] -= v[gr] * w[gc] + w[gr] * v[gc];
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

__device__ double bisect_index(const double *d, const double *e, int n, int j, double lo, double hi,
                               double pivmin, double atol) {
    // smallest x with count(x) >= j + 1, to absolute width atol (= 2 eps ||T||: the accuracy the
    // inverse-iteration shifts need)
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (hi - lo <= atol + pivmin || mid == lo || mid == hi) break;
        if (sturm_count(d, e, n, mid, pivmin) >= j + 1)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

__global__ void k_stebz(const double *dd, const double *ee, const int64_t *toff, const int32_t *nn,
                        int64_t count, double sigma, int32_t *kout, double *w, double *gap) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    int n = nn[b];
    const double *d = dd + toff[b], *e = ee + toff[b];
    __shared__ double glo, ghi, pivmin;
    __shared__ int kk;
    __shared__ double lam_lo, lam_hi;
    if (threadIdx.x == 0) {
        double lo = 1e300, hi = -1e300, emax = 0.0;
        for (int i = 0; i < n; i++) {
            double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
            lo = fmin(lo, d[i] - r);
            hi = fmax(hi, d[i] + r);
            if (i < n - 1) emax = fmax(emax, e[i] * e[i]);
        }
        double tn = fmax(fabs(lo), fabs(hi));
        pivmin = 2.2250738585072014e-308 * fmax(1.0, emax);
        glo = lo - 2.0 * DEPS * tn * n - pivmin;
        ghi = hi + 2.0 * DEPS * tn * n + pivmin;
        kk = (n > 0) ? sturm_count(d, e, n, sigma, pivmin) : 0;
        kout[b] = kk;
        lam_lo = -1.0;
        lam_hi = -1.0;
    }
    __syncthreads();
    int k = kk;
    // eigenvalues 0..k-1 (kept) and k (first discarded) for the gap
    for (int j = threadIdx.x; j <= k && j < n; j += blockDim.x) {
        // shifts to 1e-12 ||T||: the retained vectors are orthonormalised together afterwards, so
        // eigenvalues closer than that only need to land in their cluster's subspace
        double lam = bisect_index(d, e, n, j, glo, ghi, pivmin, 1e-12 * fmax(fabs(glo), fabs(ghi)));
        if (j < k) w[toff[b] + j] = lam;
        if (j == k - 1) lam_lo = lam;
        if (j == k) lam_hi = lam;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double g = 1e300;
        if (k > 0) g = fmin(g, fabs(lam_lo / sigma - 1.0));
        if (k < n) g = fmin(g, fabs(lam_hi / sigma - 1.0));
        gap[b] = g;
    }
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

constexpr int STEIN_SLOTS = 64;  // eigenvalues iterated concurrently per matrix (one per thread)

__global__ void __launch_bounds__(256) k_stein(const double *dd, const double *ee,
                                               const int64_t *toff, const int32_t *nn,
                                               int64_t count, const double *wv, const int32_t *kk,
                                               double *baseV, const int64_t *voff,
                                               const int32_t *vld, double *work,
                                               const int64_t *workoff, int cluster_orth) {
    int64_t b = blockIdx.x;
    if (b >= count) return;
    const int n = nn[b], k = kk[b];
    if (k <= 0 || n <= 0) return;
    const double *d = dd + toff[b], *e = ee + toff[b], *w = wv + toff[b];
    double *V = baseV + voff[b];
    const int LV = vld[b];
    double *W = work + workoff[b];  // 4 n STEIN_SLOTS doubles, element i of slot s at [i*S + s]
    constexpr int S = STEIN_SLOTS;
    __shared__ double red[32];
    __shared__ double tnorm;
    __shared__ double hsh[1024];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    {
        double t = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            t = fmax(t, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0));
        for (int o = 16; o; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) red[warp] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int q = 0; q < nwarp; q++) r = fmax(r, red[q]);
            tnorm = fmax(r, 1e-300);
        }
        __syncthreads();
    }
    // eigenvectors of eigenvalues closer than ortol are re-orthogonalised; farther apart, exact-shift
    // inverse iteration already gives orthogonality ~eps*||T||/gap <= 1e-10
    const double ortol = 1e-6 * tnorm, pertol = 10.0 * DEPS * tnorm;
    // ---- phase 1: independent inverse iteration, one eigenvalue per thread at a time
    if (threadIdx.x < S) {
        const int sl = threadIdx.x;
        double *dg = W, *su = W + (int64_t)n * S, *su2 = W + 2 * (int64_t)n * S,
               *x = W + 3 * (int64_t)n * S;
        for (int j = sl; j < k; j += S) {
            // separate numerically equal eigenvalues by multiples of pertol
            int q = j;
            while (q > 0 && w[q] - w[q - 1] < pertol) q--;
            const double lam = w[j] + (double)(j - q) * pertol;
            for (int i = 0; i < n; i++) x[(int64_t)i * S + sl] = urand((uint32_t)j, (uint32_t)i);
            for (int it = 0; it < 3; it++) {
                double mx = 0.0;
                for (int i = 0; i < n; i++) mx = fmax(mx, fabs(x[(int64_t)i * S + sl]));
                const double sc = (mx > 0.0) ? 1.0 / mx : 1.0;
                // factor T - lam I with partial pivoting while eliminating the right-hand side
                double diag = d[0] - lam, sup = (n > 1) ? e[0] : 0.0, rhs = x[sl] * sc;
                for (int i = 0; i < n - 1; i++) {
                    const double sub = e[i], nd = d[i + 1] - lam, ns = (i + 1 < n - 1) ? e[i + 1] : 0.0;
                    const double nrhs = x[(int64_t)(i + 1) * S + sl] * sc;
                    const int64_t ii = (int64_t)i * S + sl;
                    if (fabs(diag) >= fabs(sub)) {
                        if (diag == 0.0) diag = pertol;
                        const double m = sub / diag;
                        dg[ii] = diag;
                        su[ii] = sup;
                        su2[ii] = 0.0;
                        x[ii] = rhs;
                        diag = nd - m * sup;
                        sup = ns;
                        rhs = nrhs - m * rhs;
                    } else {
                        const double m = diag / sub;
                        dg[ii] = sub;
                        su[ii] = nd;
                        su2[ii] = ns;
                        x[ii] = nrhs;
                        diag = sup - m * nd;
                        sup = -m * ns;
                        rhs = rhs - m * nrhs;
                    }
                }
                if (diag == 0.0) diag = pertol;
                const int64_t il = (int64_t)(n - 1) * S + sl;
                dg[il] = diag;
                x[il] = rhs / diag;
                for (int i = n - 2; i >= 0; i--) {
                    const int64_t ii = (int64_t)i * S + sl;
                    double v = x[ii] - su[ii] * x[ii + S];
                    if (i + 2 < n) v -= su2[ii] * x[ii + 2 * S];
                    x[ii] = v / dg[ii];
                }
            }
            double nr = 0.0;
            for (int i = 0; i < n; i++) nr += x[(int64_t)i * S + sl] * x[(int64_t)i * S + sl];
            const double inv = (nr > 0.0) ? 1.0 / sqrt(nr) : 0.0;
            double *vj = V + (int64_t)j * LV;
            for (int i = 0; i < n; i++) vj[i] = x[(int64_t)i * S + sl] * inv;
        }
    }
    __syncthreads();
    if (!cluster_orth) return;
    // ---- phase 2: orthonormalise every cluster (gaps <= ortol) by classical Gram-Schmidt twice
    int c0 = 0;
    while (c0 < k) {
        int c1 = c0 + 1;
        while (c1 < k && w[c1] - w[c1 - 1] <= ortol) c1++;
        for (int j = c0 + 1; j < c1; j++) {
            double *vj = V + (int64_t)j * LV;
            for (int pass = 0; pass < 2; pass++) {
                for (int i0 = c0; i0 < j; i0 += 1024) {
                    const int i1 = min(j, i0 + 1024);
                    for (int i = i0 + warp; i < i1; i += nwarp) {
                        const double *vi = V + (int64_t)i * LV;
                        double sd = 0.0;
                        for (int r = lane; r < n; r += 32) sd += vi[r] * vj[r];
                        for (int o = 16; o; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
                        if (lane == 0) hsh[i - i0] = sd;
                    }
                    __syncthreads();
                    for (int r = threadIdx.x; r < n; r += blockDim.x) {
                        double acc = 0.0;
                        for (int i = i0; i < i1; i++) acc += hsh[i - i0] * V[(int64_t)i * LV + r];
                        vj[r] -= acc;
                    }
                    __syncthreads();
                }
            }
            double nr = 0.0;
            for (int r = threadIdx.x; r < n; r += blockDim.x) nr += vj[r] * vj[r];
            nr = block_sum(nr, red);
            const double inv = (nr > 0.0) ? 1.0 / sqrt(nr) : 0.0;
            for (int r = threadIdx.x; r < n; r += blockDim.x) vj[r] *= inv;
            __syncthreads();
        }
        c0 = c1;
    }
}

// ------------------------------------------------------------------------- ormtr
__global__ void __launch_bounds__(256) k_ormtr(const double *baseA, const int64_t *aoff,
                                               const int32_t *ald, const int32_t *nn,
                                               const double *tt, const int64_t *toff,
                                               double *baseV, const int64_t *voff,
                                               const int32_t *vld, const int32_t *vcols,
                                               int64_t count) {
    int64_t b = blockIdx.y;
    if (b >= count) return;
    int n = nn[b], k = vcols[b];
    const int lane = threadIdx.x & 31;
    int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= k) return;
    const double *A = baseA + aoff[b];
    int LA = ald[b];
    const double *tau = tt + toff[b];
    double *v = baseV + voff[b] + (int64_t)c * vld[b];
    for (int j = n - 2; j >= 0; j--) {
        double t = tau[j];
        if (t == 0.0) continue;
        int m = n - j - 1;
        const double *h = A + (j + 1) + (int64_t)j * LA;  // h[0] implicit 1
        double s = 0.0;
        for (int r = lane; r < m; r += 32) s += (r == 0 ? 1.0 : h[r]) * v[j + 1 + r];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        s *= t;
        for (int r = lane; r < m; r += 32) v[j + 1 + r] -= s * (r == 0 ? 1.0 : h[r]);
        __syncwarp();
    }
}

}  // namespace

// ============================================================================= host wrappers
void potrf_batched(double *base, const MatBatch &A, PotrfMode mode, int *err, cudaStream_t s) {
    if (A.count == 0 || A.maxn == 0) return;
    double fl = 0.0;
    for (auto v : A.h_n) fl += (double)v * v * v / 3.0;
    KTime kt(KC_POTRF, s, fl);
    DBuf<double> md;
    md.alloc(A.count, s);
    k_maxdiag<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, md.p);
    CK_LAUNCH();
    for (int j0 = 0; j0 < A.maxn; j0 += NB) {
        k_potf2<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, j0, mode,
                                                 md.p, err);
        CK_LAUNCH();
        int rem = A.maxn - j0 - NB;
        if (rem <= 0) break;
        dim3 gp((unsigned)cdiv(rem, 128), (unsigned)A.count);
        k_potrf_panel<<<gp, 128, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, j0);
        CK_LAUNCH();
        int64_t T = cdiv(rem, TT);
        dim3 gu((unsigned)(T * (T + 1) / 2), (unsigned)A.count);
        k_potrf_update<<<gu, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, A.count, j0, nullptr,
                                          nullptr, 0);
        CK_LAUNCH();
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
                   int32_t max_bn, int32_t *perm, const int64_t *permoff, int32_t *rank,
                   cudaStream_t s) {
    if (A.count == 0 || max_bn == 0) return;
    KTime kt(KC_PSTRF, s);
    DBuf<double> md, work;
    DBuf<int64_t> woff;
    md.alloc(A.count, s);
    // work shares the permutation layout (one double per block row)
    int64_t tot = read1(permoff + A.count, s);
    work.alloc(std::max<int64_t>(tot, 1), s);
    k_maxdiag_block<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, b0, bn, A.count, md.p,
                                                       perm, permoff, rank);
    CK_LAUNCH();
    for (int j0 = 0; j0 < max_bn; j0 += NB) {
        k_pstf_panel<<<(unsigned)A.count, 256, 0, s>>>(base, A.off.p, A.ld.p, A.n.p, b0, bn,
                                                      A.count, j0, perm, permoff, rank, work.p,
                                                      permoff, md.p);
        CK_LAUNCH();
        int rem = max_bn - j0 - NB;
        if (rem <= 0) break;
        int64_t T = cdiv(rem, TT);
        dim3 gu((unsigned)(T * (T + 1) / 2), (unsigned)A.count);
        k_potrf_update<<<gu, 256, 0, s>>>(base, A.off.p, A.ld.p, bn, A.count, j0, b0, rank, 0);
        CK_LAUNCH();
    }
    k_rank_finish<<<(unsigned)cdiv(A.count, 256), 256, 0, s>>>(rank, bn, A.count);
    CK_LAUNCH();
}

void trsm_batched(const double *base_L, const MatBatch &Lb, double *base_B, const MatBatch &Bb,
                  bool trans, cudaStream_t s) {
    if (Bb.count == 0 || Bb.maxm == 0 || Lb.maxn == 0) return;
    double fl = 0.0;
    for (size_t i = 0; i < Bb.h_n.size(); i++) fl += (double)Bb.h_n[i] * Bb.h_n[i] * Bb.h_m[i];
    KTime kt(KC_TRSM, s, fl);
    dim3 g((unsigned)cdiv(Bb.maxm, SW), (unsigned)Bb.count);
    k_trsm<<<g, 256, 0, s>>>(base_L, Lb.off.p, Lb.ld.p, Lb.n.p, base_B, Bb.off.p, Bb.ld.p, Bb.m.p,
                             Bb.count, trans ? 1 : 0);
    CK_LAUNCH();
}

void syrk_tn_batched(double *base_C, const MatBatch &Cb, const double *base_W, const MatBatch &Wb,
                     double alpha, bool w_rowmajor, cudaStream_t s) {
    if (Cb.count == 0 || Cb.maxn == 0) return;
    double fl = 0.0;
    for (size_t i = 0; i < Cb.h_n.size(); i++) fl += 2.0 * Cb.h_n[i] * Cb.h_n[i] * Wb.h_n[i];
    KTime kt(KC_SYRK, s, fl);
    int64_t T = cdiv(Cb.maxn, TT);
    dim3 g((unsigned)(T * T), (unsigned)Cb.count);
    k_syrk_tn<<<g, 256, 0, s>>>(base_C, Cb.off.p, Cb.ld.p, Cb.n.p, base_W, Wb.off.p, Wb.ld.p, Wb.n.p,
                                Cb.count, alpha, w_rowmajor ? 1 : 0);
    CK_LAUNCH();
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

namespace {
void sytd2_large(double *base, const MatBatch &Ab, double *d, double *e, double *tau,
                 const int64_t *toff, cudaStream_t s) {
    // v / p workspaces: reuse the toff layout (n entries per matrix)
    int64_t tot = read1(toff + Ab.count, s);
    DBuf<double> vb, pb;
    vb.alloc(std::max<int64_t>(tot, 1), s);
    pb.alloc(std::max<int64_t>(tot, 1), s);
    for (int j = 0; j < Ab.maxn; j++) {
        k_tr_house<<<(unsigned)Ab.count, 256, 0, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, Ab.count, j, d, e,
                                                      tau, toff, vb.p, pb.p, toff);
        CK_LAUNCH();
        const int m = Ab.maxn - j - 1;
        if (m <= 0) break;
        const int64_t T = cdiv(m, TRT);
        dim3 g((unsigned)(T * (T + 1) / 2), (unsigned)Ab.count);
        k_tr_symv<<<g, 128, 0, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, Ab.count, j, vb.p, pb.p, toff, tau, toff);
        CK_LAUNCH();
        k_tr_w<<<(unsigned)Ab.count, 256, 0, s>>>(Ab.n.p, Ab.count, j, vb.p, pb.p, toff, tau, toff);
        CK_LAUNCH();
        k_tr_update<<<g, 256, 0, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, Ab.count, j, vb.p, pb.p, toff, tau, toff);
        CK_LAUNCH();
    }
}
}  // namespace

void sytd2_batched(double *base, const MatBatch &Ab, double *d, double *e, double *tau,
                   const int64_t *toff, cudaStream_t s) {
    if (Ab.count == 0) return;
    double fl = 0.0;
    for (auto v : Ab.h_n) fl += 4.0 / 3.0 * v * v * v;
    KTime kt(KC_SYTD2, s, fl);
    if (Ab.maxn > g_large_dense) {
        // large matrices get many CTAs per column; all matrices of this batch go this way
        sytd2_large(base, Ab, d, e, tau, toff, s);
        return;
    }
    const size_t tiles = (SYTD2_THREADS / 32) * 32 * 33 * sizeof(double);
    const size_t need = tiles + 2 * (size_t)std::max(Ab.maxn, 1) * sizeof(double);
    const bool smem = need <= 220 * 1024;
    DBuf<double> pw;
    if (!smem) {
        int64_t tot = read1(toff + Ab.count, s);
        pw.alloc(std::max<int64_t>(2 * tot, 1), s);
    }
    const size_t dyn = smem ? need : tiles;
    CK(cudaFuncSetAttribute(k_sytd2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    k_sytd2<<<(unsigned)Ab.count, SYTD2_THREADS, dyn, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, Ab.count,
                                                 d, e, tau, toff, pw.p, toff, smem ? 1 : 0);
    CK_LAUNCH();
}

void stebz_batched(const double *d, const double *e, const int64_t *toff, const int32_t *n,
                   int64_t count, double sigma, int32_t *k, double *w, double *gap,
                   cudaStream_t s) {
    if (count == 0) return;
    KTime kt(KC_STEBZ, s);
    k_stebz<<<(unsigned)count, 128, 0, s>>>(d, e, toff, n, count, sigma, k, w, gap);
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
                   const double *w, const int32_t *k, double *base_V, const MatBatch &Vb,
                   double *work, const int64_t *workoff, cudaStream_t s, bool cluster_orth) {
    if (Vb.count == 0) return;
    KTime kt(KC_STEIN, s);
    k_stein<<<(unsigned)Vb.count, 256, 0, s>>>(d, e, toff, n, Vb.count, w, k, base_V, Vb.off.p,
                                              Vb.ld.p, work, workoff, cluster_orth ? 1 : 0);
    CK_LAUNCH();
}

void ormtr_batched(const double *base_A, const MatBatch &Ab, const double *tau, const int64_t *toff,
                   double *base_V, const MatBatch &Vb, cudaStream_t s) {
    if (Vb.count == 0 || Vb.maxm == 0) return;
    double fl = 0.0;
    // n - 1 reflectors of lengths n-1 ... 1, each applied to m vectors at 4 flops per entry
    for (size_t i = 0; i < Vb.h_n.size(); i++) fl += 2.0 * Vb.h_n[i] * Vb.h_n[i] * Vb.h_m[i];
    KTime kt(KC_ORMTR, s, fl);
    dim3 g((unsigned)cdiv(Vb.maxm, 8), (unsigned)Vb.count);
    k_ormtr<<<g, 256, 0, s>>>(base_A, Ab.off.p, Ab.ld.p, Ab.n.p, tau, toff, base_V, Vb.off.p,
                              Vb.ld.p, Vb.m.p, Vb.count);
    CK_LAUNCH();
}

}  // namespace lsamg
