// Solve-phase kernels: Gram SpMV y = G^T (G x) (Section 2 eq. 2.1, Prop. 5.1), the
// multiplicative Schwarz sweep on the overlaps, restriction / interpolation with
// P = [R_w^T Z_i], the dense coarsest solve (Section 2 E_TG; Section 6 preamble), and
// the FP64 vector kernels of the outer Krylov loop.  Templated on float / double.
#include <type_traits>

#include "impl.cuh"

namespace lsamg {

namespace {

inline unsigned gridv(int64_t items, int per = 256, int64_t cap = 148 * 32) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(items, per), cap));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- Gram SpMV
// y[rhs] (+)= sign * G_T^T (G_T x_T) for every element, scattered with atomics.
// One CTA per element; t = G_T x_T is staged in shared memory.
template <class T>
__global__ void __launch_bounds__(128) k_spmv(const int64_t *eptr, const int32_t *eidx, int64_t ne,
                                              const T *G, const int64_t *goff,
                                              const int32_t *grows, const T *x, T *y, int64_t n,
                                              int nrhs, T sign) {
    extern __shared__ unsigned char smraw[];
    T *t = reinterpret_cast<T *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
        const int64_t b = eptr[e];
        const int nT = (int)(eptr[e + 1] - b);
        const int m = grows[e];
        const T *g = G + goff[e];
        for (int r = 0; r < nrhs; r++) {
            const T *xr = x + (int64_t)r * n;
            for (int row = warp; row < m; row += nwarp) {
                const T *gr = g + (int64_t)row * nT;
                T s = 0;
                for (int c = lane; c < nT; c += 32) s += gr[c] * xr[eidx[b + c]];
                s = warp_sum(s);
                if (lane == 0) t[row] = s;
            }
            __syncthreads();
            T *yr = y + (int64_t)r * n;
            for (int c = threadIdx.x; c < nT; c += blockDim.x) {
                T s = 0;
                for (int row = 0; row < m; row++) s += g[(int64_t)row * nT + c] * t[row];
                atomicAdd(&yr[eidx[b + c]], sign * s);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- packed triangular solves
// In-place solve of L L^T v = v for a packed lower row-major factor (row i at i(i+1)/2),
// vector v in global memory (one right-hand side).  Called by a whole CTA.
template <class T>
__device__ void chol_solve_packed(const T *L, int n, T *v, T *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // forward: L y = v
    for (int r0 = 0; r0 < n; r0 += 32) {
        const int rs = min(32, n - r0);
        // off-block GEMV: red[i] = v[r0+i] - sum_{j<r0} L[r0+i, j] y[j]
        for (int i = warp; i < rs; i += nwarp) {
            const T *row = L + (int64_t)(r0 + i) * (r0 + i + 1) / 2;
            T s = 0;
            for (int j = lane; j < r0; j += 32) s += row[j] * v[j];
            s = warp_sum(s);
            if (lane == 0) red[i] = v[r0 + i] - s;
        }
        __syncthreads();
        if (warp == 0) {
            T yl = 0;  // lane i holds y[r0+i]
            for (int i = 0; i < rs; i++) {
                const T *row = L + (int64_t)(r0 + i) * (r0 + i + 1) / 2 + r0;
                T c = (lane < i) ? row[lane] * yl : (T)0;
                c = warp_sum(c);
                T yi = (red[i] - c) / row[i];
                if (lane == i) yl = yi;
            }
            if (lane < rs) v[r0 + lane] = yl;
        }
        __syncthreads();
    }
    // backward: L^T x = y
    const int nb = (n + 31) / 32;
    for (int bi = nb - 1; bi >= 0; bi--) {
        const int r0 = bi * 32, rs = min(32, n - r0);
        if (warp == 0) {
            T xl = (lane < rs) ? v[r0 + lane] : (T)0;  // lane i holds x[r0+i] (running)
            for (int i = rs - 1; i >= 0; i--) {
                const T *row = L + (int64_t)(r0 + i) * (r0 + i + 1) / 2 + r0;
                T xi = __shfl_sync(0xffffffffu, xl, i) / row[i];
                if (lane == i) xl = xi;
                if (lane < i) xl -= row[lane] * xi;
            }
            if (lane < rs) v[r0 + lane] = xl;
        }
        __syncthreads();
        // update the rows above: v[j] -= sum_{i in block} L[r0+i, j] x[r0+i], j < r0
        for (int j = threadIdx.x; j < r0; j += blockDim.x) {
            T s = 0;
            for (int i = 0; i < rs; i++) s += L[(int64_t)(r0 + i) * (r0 + i + 1) / 2 + j] * v[r0 + i];
            v[j] -= s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- Schwarz sweep (one colour)
template <class T>
__global__ void __launch_bounds__(256) k_schwarz(const int32_t *aggs, int64_t na,
                                                 const int64_t *Optr, const int32_t *Oidx,
                                                 const T *Lp, const int64_t *Loff,
                                                 const int64_t *oeptr, const int32_t *oeidx,
                                                 const int64_t *locoff, const int32_t *loc,
                                                 const int64_t *eptr, const int32_t *eidx,
                                                 const T *G, const int64_t *goff,
                                                 const int32_t *grows, T *x, T *res, T *ws,
                                                 int64_t n, int64_t wsn, int nrhs) {
    extern __shared__ unsigned char smraw[];
    T *t = reinterpret_cast<T *>(smraw);  // element G_T delta staging (max rows)
    __shared__ T red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int64_t ia = blockIdx.x; ia < na; ia += gridDim.x) {
        const int32_t a = aggs[ia];
        const int64_t ob = Optr[a];
        const int nO = (int)(Optr[a + 1] - ob);
        const T *L = Lp + Loff[a];
        for (int r = 0; r < nrhs; r++) {
            T *v = ws + (int64_t)r * wsn + ob;
            T *xr = x + (int64_t)r * n;
            T *rr = res + (int64_t)r * n;
            for (int i = threadIdx.x; i < nO; i += blockDim.x) v[i] = rr[Oidx[ob + i]];
            __syncthreads();
            chol_solve_packed<T>(L, nO, v, red);
            // x_Omega += delta  (overlaps of one colour are disjoint)
            for (int i = threadIdx.x; i < nO; i += blockDim.x) xr[Oidx[ob + i]] += v[i];
            __syncthreads();
            // res -= A R_Omega^T delta = sum over elements meeting Omega of G_T^T G_T delta_T
            for (int64_t j = oeptr[a]; j < oeptr[a + 1]; j++) {
                const int32_t e = oeidx[j];
                const int64_t b = eptr[e];
                const int nT = (int)(eptr[e + 1] - b);
                const int m = grows[e];
                const T *g = G + goff[e];
                const int32_t *lc = loc + locoff[j];
                for (int row = warp; row < m; row += nwarp) {
                    const T *gr = g + (int64_t)row * nT;
                    T s = 0;
                    for (int c = lane; c < nT; c += 32) {
                        int p = lc[c];
                        if (p >= 0) s += gr[c] * v[p];
                    }
                    s = warp_sum(s);
                    if (lane == 0) t[row] = s;
                }
                __syncthreads();
                for (int c = threadIdx.x; c < nT; c += blockDim.x) {
                    T s = 0;
                    for (int row = 0; row < m; row++) s += g[(int64_t)row * nT + c] * t[row];
                    atomicAdd(&rr[eidx[b + c]], -s);
                }
                __syncthreads();
            }
        }
    }
}

// ---------------------------------------------------------------- transfers
// rc[off_a + j] = sum_p Z_a[p, j] res[omega_a[p]] (P^T r, P = blockdiag R_omega^T Z_a).  One CTA
// per aggregate: the 8 warps take interleaved rows of Z_a (coalesced, 4 rows in flight), lanes
// take columns in chunks of 128, and the warps' partial sums are added in shared memory.
template <class T>
__global__ void __launch_bounds__(256) k_restrict(const int64_t *wptr, const int32_t *widx, const int32_t *k,
                                                  const int64_t *off, const T *Z, const int64_t *zoff,
                                                  int64_t nagg, const T *res, int64_t n, T *rc, int64_t nc,
                                                  int nrhs) {
    __shared__ T red[8][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t a = blockIdx.x; a < nagg; a += gridDim.x) {
        const int ka = k[a];
        const int64_t wb = wptr[a];
        const int nw = (int)(wptr[a + 1] - wb);
        const T *z = Z + zoff[a];
        for (int r = 0; r < nrhs; r++) {
            const T *rr = res + (int64_t)r * n;
            for (int j0 = 0; j0 < ka; j0 += 128) {
                T acc[4] = {0, 0, 0, 0};
#pragma unroll 4
                for (int p = warp; p < nw; p += 8) {
                    const T rp = rr[widx[wb + p]];
                    const T *zr = z + (int64_t)p * ka + j0;
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int j = lane + 32 * u;
                        if (j0 + j < ka) acc[u] += zr[j] * rp;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) red[warp][lane + 32 * u] = acc[u];
                __syncthreads();
                if (threadIdx.x < 128 && j0 + (int)threadIdx.x < ka) {
                    T sum = 0;
#pragma unroll
                    for (int w = 0; w < 8; w++) sum += red[w][threadIdx.x];
                    rc[(int64_t)r * nc + off[a] + j0 + threadIdx.x] = sum;
                }
                __syncthreads();
            }
        }
    }
}

// x[omega_a[p]] += sum_j Z_a[p, j] ec[off_a + j] (x += P e_c).  One CTA per aggregate, the coarse
// values staged in shared memory, a warp per row of Z_a (4 rows in flight).
template <class T>
__global__ void __launch_bounds__(256) k_interp(const int64_t *wptr, const int32_t *widx, const int32_t *k,
                                                const int64_t *off, const T *Z, const int64_t *zoff,
                                                int64_t nagg, const T *ec, int64_t nc, T *x, int64_t n,
                                                int nrhs) {
    extern __shared__ unsigned char smraw[];
    T *e = reinterpret_cast<T *>(smraw);   // [max k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t a = blockIdx.x; a < nagg; a += gridDim.x) {
        const int ka = k[a];
        const int64_t wb = wptr[a];
        const int nw = (int)(wptr[a + 1] - wb);
        const T *z = Z + zoff[a];
        for (int r = 0; r < nrhs; r++) {
            __syncthreads();
            for (int j = threadIdx.x; j < ka; j += blockDim.x) e[j] = ec[(int64_t)r * nc + off[a] + j];
            __syncthreads();
            T *xr = x + (int64_t)r * n;
#pragma unroll 4
            for (int p = warp; p < nw; p += 8) {
                const T *zr = z + (int64_t)p * ka;
                T sum = 0;
                for (int j = lane; j < ka; j += 32) sum += zr[j] * e[j];
                sum = warp_sum(sum);
                if (lane == 0) xr[widx[wb + p]] += sum;
            }
        }
    }
}

// ---------------------------------------------------------------- blocked triangular solves
// In-place solve of L L^T v = v for several independent packed lower row-major factors (row i
// at offset i(i+1)/2): the subdomains of one Schwarz colour, or the coarsest matrix.  Rows are
// cut into blocks of cb <= TRI_CB rows whose diagonal blocks are inverted once at set-up
// (Dinv, FP64 packed lower row-major, block b of system a at Doff[a] + b cb(cb+1)/2; the
// product with it is formed in FP64 in the FP32 cycle too, since an explicit inverse of an
// ill-conditioned block rounded to FP32 loses its small components to cancellation).  Every launch
// advances all systems by one block: CTA 0 of a system finishes the next diagonal block (its
// update by the block just solved, then the product with the inverted diagonal block; all of
// its loads are issued on entry), CTAs 1.. apply the block just solved to the rest of the
// system with coalesced loads, many in flight per thread.
constexpr int TRI_CB = 64;      // largest block
constexpr int TRI_RG = 8;       // right-hand sides per pass through shared memory
constexpr int TRI_RPW = TRI_CB / 8;   // block rows per warp in CTA 0
constexpr int TRI_NU = TRI_CB / 32;   // block columns per lane
constexpr int TRI_ROWS = 64;    // rows per forward update CTA (8 per warp)
constexpr int TRI_COLS = 128;   // columns per backward update CTA (2 row halves per column)

__host__ __device__ inline int64_t tri_block_words(int cb) { return (int64_t)cb * (cb + 1) / 2; }

// Forward substitution L y = v.  Block k = rows [k cb, (k+1) cb) already holds y_k; finish block
// k+1.  k = -1 starts every system (solves block 0).
template <class T>
__global__ void __launch_bounds__(256) k_tri_fwd(const int32_t *sys, const int64_t *Optr, const T *Lp,
                                                 const int64_t *Loff, const double *Dp, const int64_t *Doff,
                                                 int k, int cb, T *ws, int64_t wsn, int nrhs) {
    __shared__ T sm[2 * TRI_RG * TRI_CB];
    const int32_t a = sys ? sys[blockIdx.y] : (int32_t)blockIdx.y;
    const int64_t ob = Optr[a];
    const int n = (int)(Optr[a + 1] - ob);
    const int r0 = k * cb, r1 = r0 + cb;
    if (r1 >= n) return;
    const int r2 = min(n, r1 + cb);
    const T *L = Lp + Loff[a];
    T *v = ws + ob;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *y = sm;                       // [TRI_RG][cb]  y_k
    T *tv = sm + TRI_RG * TRI_CB;    // [TRI_RG][cb]  block k+1 right-hand sides
    if (blockIdx.x > 0) {
        // rows i in [i0, i0 + TRI_ROWS) beyond block k+1: v_i -= L[i, r0:r1] y_k
        if (k < 0) return;
        const int64_t i0 = (int64_t)r2 + (int64_t)(blockIdx.x - 1) * TRI_ROWS;
        if (i0 >= n) return;
        constexpr int NQ = TRI_ROWS / 8;
        T lv[NQ][TRI_NU];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int64_t i = i0 + warp + 8 * q;
#pragma unroll
            for (int u = 0; u < TRI_NU; u++) {
                const int j = lane + 32 * u;
                lv[q][u] = (i < n && j < cb) ? L[i * (i + 1) / 2 + r0 + j] : (T)0;
            }
        }
        for (int g0 = 0; g0 < nrhs; g0 += TRI_RG) {
            const int nr = min(TRI_RG, nrhs - g0);
            __syncthreads();
            for (int q = threadIdx.x; q < nr * cb; q += blockDim.x) {
                const int r = q / cb;
                y[r * TRI_CB + q - r * cb] = v[(int64_t)(g0 + r) * wsn + r0 + (q - r * cb)];
            }
            __syncthreads();
            for (int r = 0; r < nr; r++) {
                T *vr = v + (int64_t)(g0 + r) * wsn;
                T old[NQ];
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    const int64_t i = i0 + warp + 8 * q;
                    old[q] = (lane == 0 && i < n) ? vr[i] : (T)0;
                }
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    T acc = 0;
#pragma unroll
                    for (int u = 0; u < TRI_NU; u++) {
                        const int j = lane + 32 * u;
                        if (j < cb) acc += lv[q][u] * y[r * TRI_CB + j];
                    }
                    acc = warp_sum(acc);
                    const int64_t i = i0 + warp + 8 * q;
                    if (lane == 0 && i < n) vr[i] = old[q] - acc;
                }
            }
        }
        return;
    }
    // CTA 0: block k+1 = rows [r1, r2); t = v - L[r1:r2, r0:r1] y_k, then y_{k+1} = Dinv t
    const int nb = r2 - r1;
    const double *Di = Dp + Doff[a] + (int64_t)(k + 1) * tri_block_words(cb);
    T pv[TRI_RPW][TRI_NU];
    double dv[TRI_RPW][TRI_NU];
#pragma unroll
    for (int q = 0; q < TRI_RPW; q++) {
        const int i = warp + 8 * q;
        const int64_t gi = (int64_t)r1 + i;
#pragma unroll
        for (int u = 0; u < TRI_NU; u++) {
            const int j = lane + 32 * u;
            pv[q][u] = (k >= 0 && i < nb && j < cb) ? L[gi * (gi + 1) / 2 + r0 + j] : (T)0;
            dv[q][u] = (i < nb && j <= i) ? Di[i * (i + 1) / 2 + j] : 0.0;
        }
    }
    for (int g0 = 0; g0 < nrhs; g0 += TRI_RG) {
        const int nr = min(TRI_RG, nrhs - g0);
        __syncthreads();
        for (int q = threadIdx.x; q < nr * TRI_CB; q += blockDim.x) {
            const int r = q / TRI_CB, j = q - r * TRI_CB;
            const T *vr = v + (int64_t)(g0 + r) * wsn;
            y[q] = (k >= 0 && j < cb) ? vr[r0 + j] : (T)0;
            tv[q] = (j < nb) ? vr[r1 + j] : (T)0;
        }
        __syncthreads();
        if (k >= 0) {
            for (int r = 0; r < nr; r++) {
#pragma unroll
                for (int q = 0; q < TRI_RPW; q++) {
                    const int i = warp + 8 * q;
                    T acc = 0;
#pragma unroll
                    for (int u = 0; u < TRI_NU; u++) acc += pv[q][u] * y[r * TRI_CB + lane + 32 * u];
                    acc = warp_sum(acc);
                    if (lane == 0 && i < nb) tv[r * TRI_CB + i] -= acc;
                }
            }
            __syncthreads();
        }
        for (int r = 0; r < nr; r++) {
            T *vr = v + (int64_t)(g0 + r) * wsn;
#pragma unroll
            for (int q = 0; q < TRI_RPW; q++) {
                const int i = warp + 8 * q;
                double acc = 0;
#pragma unroll
                for (int u = 0; u < TRI_NU; u++) acc += dv[q][u] * (double)tv[r * TRI_CB + lane + 32 * u];
                acc = warp_sum(acc);
                if (lane == 0 && i < nb) vr[r1 + i] = (T)acc;
            }
        }
    }
}

// Backward substitution L^T x = y.  Block k holds x_k (k < K = ceil(n / cb)); finish block k-1.
// k = K starts a system (solves its last block).
template <class T>
__global__ void __launch_bounds__(256) k_tri_bwd(const int32_t *sys, const int64_t *Optr, const T *Lp,
                                                 const int64_t *Loff, const double *Dp, const int64_t *Doff,
                                                 int k, int cb, T *ws, int64_t wsn, int nrhs) {
    __shared__ T sm[2 * TRI_RG * TRI_CB + TRI_RG * TRI_COLS];
    __shared__ double red[4 * TRI_RG * TRI_CB];   // CTA 0: partial sums of the 4 row parts
    const int32_t a = sys ? sys[blockIdx.y] : (int32_t)blockIdx.y;
    const int64_t ob = Optr[a];
    const int n = (int)(Optr[a + 1] - ob);
    const int K = (n + cb - 1) / cb;
    if (k > K || k < 1) return;
    const bool first = (k == K);
    const int r0 = k * cb, r1 = min(n, r0 + cb);        // block k (unless first)
    const int b0 = (k - 1) * cb, b1 = first ? n : r0;   // block k-1
    const T *L = Lp + Loff[a];
    T *v = ws + ob;
    const int tid = threadIdx.x;
    T *xk = sm;                                 // [TRI_RG][TRI_CB]  x_k
    if (blockIdx.x > 0) {
        // columns j in [c0, c0 + TRI_COLS) before block k-1: v_j -= sum_{i in block k} L[i, j] x_i
        if (first) return;
        const int c0 = (int)(blockIdx.x - 1) * TRI_COLS;
        if (c0 >= b0) return;
        const int col = tid & (TRI_COLS - 1), half = tid >> 7;
        const int j = c0 + col;
        T *part = sm + TRI_RG * TRI_CB;         // [TRI_RG][TRI_COLS]
        constexpr int NL = TRI_CB / 2;
        T lv[NL];
#pragma unroll
        for (int m = 0; m < NL; m++) {
            const int i = r0 + half + 2 * m;
            lv[m] = (j < b0 && i < r1) ? L[(int64_t)i * (i + 1) / 2 + j] : (T)0;
        }
        for (int g0 = 0; g0 < nrhs; g0 += TRI_RG) {
            const int nr = min(TRI_RG, nrhs - g0);
            __syncthreads();
            for (int q = tid; q < nr * TRI_CB; q += blockDim.x) {
                const int r = q / TRI_CB, i = q - r * TRI_CB;
                xk[q] = (r0 + i < r1) ? v[(int64_t)(g0 + r) * wsn + r0 + i] : (T)0;
            }
            __syncthreads();
            T acc[TRI_RG];
#pragma unroll
            for (int r = 0; r < TRI_RG; r++) {
                acc[r] = 0;
                if (r < nr) {
#pragma unroll
                    for (int m = 0; m < NL; m++) acc[r] += lv[m] * xk[r * TRI_CB + half + 2 * m];
                }
            }
            if (half == 1)
                for (int r = 0; r < nr; r++) part[r * TRI_COLS + col] = acc[r];
            __syncthreads();
            if (half == 0 && j < b0)
                for (int r = 0; r < nr; r++) v[(int64_t)(g0 + r) * wsn + j] -= acc[r] + part[r * TRI_COLS + col];
        }
        return;
    }
    // CTA 0: block k-1 = rows [b0, b1); t = v - L[r0:r1, b0:b1]^T x_k, then x_{k-1} = Dinv^T t.
    // Thread (col, part): column col of the block, rows part, part + 4, ...
    const int nb = b1 - b0;
    const int col = tid & (TRI_CB - 1), part = tid / TRI_CB;   // 4 parts
    constexpr int NP = TRI_CB / 4;
    const double *Di = Dp + Doff[a] + (int64_t)(k - 1) * tri_block_words(cb);
    T pv[NP];
    double dv[NP];
#pragma unroll
    for (int m = 0; m < NP; m++) {
        const int ii = part + 4 * m;              // row within block k / within block k-1
        const int gi = r0 + ii;
        pv[m] = (!first && col < nb && gi < r1) ? L[(int64_t)gi * (gi + 1) / 2 + b0 + col] : (T)0;
        dv[m] = (col < nb && ii < nb && ii >= col) ? Di[ii * (ii + 1) / 2 + col] : 0.0;
    }
    T *tv = sm + TRI_RG * TRI_CB;               // [TRI_RG][TRI_CB]
    for (int g0 = 0; g0 < nrhs; g0 += TRI_RG) {
        const int nr = min(TRI_RG, nrhs - g0);
        __syncthreads();
        for (int q = tid; q < nr * TRI_CB; q += blockDim.x) {
            const int r = q / TRI_CB, i = q - r * TRI_CB;
            const T *vr = v + (int64_t)(g0 + r) * wsn;
            xk[q] = (!first && r0 + i < r1) ? vr[r0 + i] : (T)0;
            tv[q] = (i < nb) ? vr[b0 + i] : (T)0;
        }
        __syncthreads();
        if (!first) {
            for (int r = 0; r < nr; r++) {
                T acc = 0;
#pragma unroll
                for (int m = 0; m < NP; m++) acc += pv[m] * xk[r * TRI_CB + part + 4 * m];
                red[(part * TRI_RG + r) * TRI_CB + col] = (double)acc;
            }
            __syncthreads();
            for (int q = tid; q < nr * TRI_CB; q += blockDim.x) {
                const int r = q / TRI_CB, c = q - r * TRI_CB;
                tv[q] -= (T)(red[(0 * TRI_RG + r) * TRI_CB + c] + red[(1 * TRI_RG + r) * TRI_CB + c] +
                             red[(2 * TRI_RG + r) * TRI_CB + c] + red[(3 * TRI_RG + r) * TRI_CB + c]);
            }
            __syncthreads();
        }
        for (int r = 0; r < nr; r++) {
            double acc = 0;
#pragma unroll
            for (int m = 0; m < NP; m++) acc += dv[m] * (double)tv[r * TRI_CB + part + 4 * m];
            red[(part * TRI_RG + r) * TRI_CB + col] = acc;
        }
        __syncthreads();
        for (int q = tid; q < nr * TRI_CB; q += blockDim.x) {
            const int r = q / TRI_CB, c = q - r * TRI_CB;
            if (c < nb)
                v[(int64_t)(g0 + r) * wsn + b0 + c] =
                    (T)(red[(0 * TRI_RG + r) * TRI_CB + c] + red[(1 * TRI_RG + r) * TRI_CB + c] +
                        red[(2 * TRI_RG + r) * TRI_CB + c] + red[(3 * TRI_RG + r) * TRI_CB + c]);
        }
    }
}

// Set-up: invert the diagonal blocks of the factors (FP64, column-parallel substitution in
// shared memory; thread j computes column j of L_bb^{-1}).  One CTA per (block, system).
__global__ void __launch_bounds__(TRI_CB) k_tri_inv(const int64_t *Optr, const double *Lp, const int64_t *Loff,
                                                    const int64_t *Doff, int cb, double *Dinv, int64_t y0) {
    __shared__ double Ls[TRI_CB * (TRI_CB + 1) / 2];   // L_bb, packed lower row-major
    __shared__ double X[TRI_CB * (TRI_CB + 1) / 2];    // L_bb^{-1}, packed lower column-major
    __shared__ double rd[TRI_CB];
    const int64_t a = y0 + blockIdx.y;
    const int n = (int)(Optr[a + 1] - Optr[a]);
    const int b0 = (int)blockIdx.x * cb;
    if (b0 >= n) return;
    const int nb = min(cb, n - b0);
    const double *L = Lp + Loff[a];
    const int tot = nb * (nb + 1) / 2;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        int i = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
        while ((i + 1) * (i + 2) / 2 <= q) i++;
        while (i * (i + 1) / 2 > q) i--;
        const int j = q - i * (i + 1) / 2;
        const int64_t gi = (int64_t)b0 + i;
        Ls[q] = L[gi * (gi + 1) / 2 + b0 + j];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < nb) rd[j] = 1.0 / Ls[j * (j + 1) / 2 + j];
    __syncthreads();
    if (j < nb) {
        double *xj = X + j * nb - j * (j - 1) / 2 - j;   // xj[i] = X(i, j), i >= j
        for (int i = j; i < nb; i++) {
            const double *li = Ls + i * (i + 1) / 2;
            double s = (i == j) ? 1.0 : 0.0;
            for (int m = j; m < i; m++) s -= li[m] * xj[m];
            xj[i] = s * rd[i];
        }
    }
    __syncthreads();
    double *D = Dinv + Doff[a] + (int64_t)blockIdx.x * tri_block_words(cb);
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        int i = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
        while ((i + 1) * (i + 2) / 2 <= q) i++;
        while (i * (i + 1) / 2 > q) i--;
        const int jj = q - i * (i + 1) / 2;
        D[q] = X[jj * nb - jj * (jj - 1) / 2 + (i - jj)];
    }
}

// ---------------------------------------------------------------- split Schwarz sweep (large subdomains)
// gather: ws[sub] = res[Omega_a]
template <class T>
__global__ void k_sw_gather(const int32_t *aggs, const int64_t *Optr, const int32_t *Oidx, const T *res,
                            T *ws, int64_t n, int64_t wsn, int nrhs) {
    const int32_t a = aggs[blockIdx.y];
    const int64_t ob = Optr[a], nO = Optr[a + 1] - ob;
    for (int r = 0; r < nrhs; r++)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nO; i += (int64_t)gridDim.x * blockDim.x)
            ws[(int64_t)r * wsn + ob + i] = res[(int64_t)r * n + Oidx[ob + i]];
}

// x[Omega_a] += ws[sub]
template <class T>
__global__ void k_sw_addx(const int32_t *aggs, const int64_t *Optr, const int32_t *Oidx, const T *ws, T *x,
                          int64_t n, int64_t wsn, int nrhs) {
    const int32_t a = aggs[blockIdx.y];
    const int64_t ob = Optr[a], nO = Optr[a + 1] - ob;
    for (int r = 0; r < nrhs; r++)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nO; i += (int64_t)gridDim.x * blockDim.x)
            x[(int64_t)r * n + Oidx[ob + i]] += ws[(int64_t)r * wsn + ob + i];
}

// x[Omega_a] += theta ws[sub] for subdomains that may overlap (additive smoother): atomic adds
template <class T>
__global__ void k_sw_addx_scaled(const int32_t *aggs, const int64_t *Optr, const int32_t *Oidx, const T *ws, T *x,
                                 T theta, int64_t n, int64_t wsn, int nrhs) {
    const int32_t a = aggs[blockIdx.y];
    const int64_t ob = Optr[a], nO = Optr[a + 1] - ob;
    for (int r = 0; r < nrhs; r++)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nO; i += (int64_t)gridDim.x * blockDim.x)
            atomicAdd(&x[(int64_t)r * n + Oidx[ob + i]], theta * ws[(int64_t)r * wsn + ob + i]);
}

// residual update res -= G_T^T G_T delta_T, one CTA per (subdomain, element meeting Omega) pair
template <class T>
__global__ void __launch_bounds__(128) k_sw_scatter(const int32_t *pa, const int64_t *pj, int64_t npairs,
                                                    const int64_t *Optr, const int64_t *locoff,
                                                    const int32_t *loc, const int32_t *oeidx,
                                                    const int64_t *eptr, const int32_t *eidx, const T *G,
                                                    const int64_t *goff, const int32_t *grows, const T *ws,
                                                    T *res, int64_t n, int64_t wsn, int nrhs) {
    extern __shared__ unsigned char smraw[];
    T *t = reinterpret_cast<T *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int64_t q = blockIdx.x; q < npairs; q += gridDim.x) {
        const int32_t a = pa[q];
        const int64_t j = pj[q];
        const int32_t e = oeidx[j];
        const int64_t b = eptr[e];
        const int nT = (int)(eptr[e + 1] - b);
        const int m = grows[e];
        const T *g = G + goff[e];
        const int32_t *lc = loc + locoff[j];
        for (int r = 0; r < nrhs; r++) {
            const T *v = ws + (int64_t)r * wsn + Optr[a];
            T *rr = res + (int64_t)r * n;
            for (int row = warp; row < m; row += nwarp) {
                const T *gr = g + (int64_t)row * nT;
                T sacc = 0;
                for (int c = lane; c < nT; c += 32) {
                    const int p = lc[c];
                    if (p >= 0) sacc += gr[c] * v[p];
                }
                sacc = warp_sum(sacc);
                if (lane == 0) t[row] = sacc;
            }
            __syncthreads();
            for (int c = threadIdx.x; c < nT; c += blockDim.x) {
                T sacc = 0;
                for (int row = 0; row < m; row++) sacc += g[(int64_t)row * nT + c] * t[row];
                atomicAdd(&rr[eidx[b + c]], -sacc);
            }
            __syncthreads();
        }
    }
}

template <class T>
__global__ void k_fill(T *a, int64_t n, T v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

template <class A, class B>
__global__ void k_convert(B *dst, const A *src, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}

// ---------------------------------------------------------------- FP64 vector kernels
__global__ void k_dots(const double *a, const double *b, int64_t n, int nrhs, double *out) {
    __shared__ double sh[32];
    for (int r = 0; r < nrhs; r++) {
        double s = 0.0;
        const double *ar = a + (int64_t)r * n, *br = b + (int64_t)r * n;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            s += ar[i] * br[i];
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            double u = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
            u = warp_sum(u);
            if (threadIdx.x == 0) atomicAdd(&out[r], u);
        }
        __syncthreads();
    }
}

__global__ void k_axpy(double *y, const double *x, const double *alpha, int64_t n, int nrhs,
                       double sign) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * nrhs;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] += sign * alpha[i / n] * x[i];
}

__global__ void k_xpby(double *p, const double *z, const double *beta, int64_t n, int nrhs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * nrhs;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta[i / n] * p[i];
}

__global__ void k_elem_grad(const int64_t *eptr, const int32_t *eidx, int64_t ne, const double *G,
                            const int64_t *goff, const int32_t *grows, const double *coef,
                            const double *lam, const double *x, double *g) {
    const int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w; e < ne; e += nw) {
        const int64_t b = eptr[e];
        const int nT = (int)(eptr[e + 1] - b);
        const int m = grows[e];
        const double *ge = G + goff[e];
        double acc = 0.0;
        for (int row = 0; row < m; row++) {
            double sl = 0.0, sx = 0.0;
            for (int c = lane; c < nT; c += 32) {
                double gv = ge[(int64_t)row * nT + c];
                int32_t d = eidx[b + c];
                sl += gv * lam[d];
                sx += gv * x[d];
            }
            sl = warp_sum(sl);
            sx = warp_sum(sx);
            acc += sl * sx;
        }
        if (lane == 0) g[e] = -acc / coef[e];
    }
}

}  // namespace

// =============================================================================== host side
template <class T>
void gram_spmv(const Level &L, const T *x, T *y, const T *b, int nrhs, cudaStream_t s) {
    // y = b - G^T G x  (b != nullptr), else y = G^T G x
    const int64_t tot = L.n * nrhs;
    if (b) {
        if (b != y) CK(cudaMemcpyAsync(y, b, tot * sizeof(T), cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemsetAsync(y, 0, tot * sizeof(T), s));
    }
    if (L.ne == 0) return;
    KTime kt(KC_SPMV, s, 0.0, L.spmv_bytes[std::is_same<T, double>::value ? 1 : 0] * (nrhs > 1 ? 1.0 : 1.0));
    const T *G = std::is_same<T, float>::value ? (const T *)L.G32.p : (const T *)L.G64.p;
    int32_t maxm = 0;
    // rows per element never exceed the element-map length on level 0; coarse groups can
    // have more rows (stacked members), bounded by their G size.  Shared memory holds one
    // row vector t of the largest element.
    maxm = L.max_grows_cached;
    size_t sm = (size_t)std::max(1, maxm) * sizeof(T);
    k_spmv<T><<<gridv(L.ne, 1, 148 * 24), 128, sm, s>>>(L.eptr.p, L.eidx.p, L.ne, G, L.goff.p,
                                                      L.grows.p, x, y, L.n, nrhs,
                                                      b ? (T)-1 : (T)1);
    CK_LAUNCH();
}

void ensure_cycle_ws(Level &L, int nrhs, cudaStream_t s) {
    if (L.nrhs_ws >= nrhs) return;
    const int64_t n = L.n * nrhs;
    L.b64.alloc(n, s);
    L.x64.alloc(n, s);
    L.r64.alloc(n, s);
    L.b32.alloc(n, s);
    L.x32.alloc(n, s);
    L.r32.alloc(n, s);
    int64_t wsn = L.coarsest ? 0 : L.Omega_total;
    L.ws64.alloc(std::max<int64_t>(wsn * nrhs, 1), s);
    L.ws32.alloc(std::max<int64_t>(wsn * nrhs, 1), s);
    L.nrhs_ws = nrhs;
}

template <class T>
static T *bvec(Level &L) {
    if constexpr (std::is_same<T, float>::value) return L.b32.p; else return L.b64.p;
}
template <class T>
static T *xvec(Level &L) {
    if constexpr (std::is_same<T, float>::value) return L.x32.p; else return L.x64.p;
}
template <class T>
static T *rvec(Level &L) {
    if constexpr (std::is_same<T, float>::value) return L.r32.p; else return L.r64.p;
}
template <class T>
static T *wsvec(Level &L) {
    if constexpr (std::is_same<T, float>::value) return L.ws32.p; else return L.ws64.p;
}

// L L^T v = v for systems sys[0..nsys) (sys == nullptr: systems 0..nsys-1) whose vectors sit at
// ws + Optr[a] (stride wsn per right-hand side), factors at Lp + Loff[a] and inverted diagonal
// blocks at Dp + Doff[a]; maxn bounds the systems' orders, cb is the block size of Dp.
template <class T>
static void tri_solve(const int32_t *sys, int64_t nsys, const int64_t *Optr, const T *Lp,
                      const int64_t *Loff, const double *Dp, const int64_t *Doff, int cb, int maxn, T *ws,
                      int64_t wsn, int nrhs, cudaStream_t s) {
    const int K = (maxn + cb - 1) / cb;
    for (int64_t y0 = 0; y0 < nsys; y0 += 65535) {
        const unsigned ny = (unsigned)std::min<int64_t>(65535, nsys - y0);
        if (!sys && y0 > 0) fail(LSAMG_LIMIT, "more than 65535 systems without an index list");
        const int32_t *sy = sys ? sys + y0 : nullptr;
        for (int k = -1; k <= K - 2; k++) {
            const int64_t rest = (int64_t)maxn - (int64_t)(k + 2) * cb;
            const unsigned gx = 1 + (unsigned)(k >= 0 && rest > 0 ? cdiv(rest, TRI_ROWS) : 0);
            k_tri_fwd<T><<<dim3(gx, ny), 256, 0, s>>>(sy, Optr, Lp, Loff, Dp, Doff, k, cb, ws, wsn, nrhs);
            CK_LAUNCH();
        }
        for (int k = K; k >= 1; k--) {
            const int64_t cols = (int64_t)(k - 1) * cb;
            const unsigned gx = 1 + (unsigned)(k < K && cols > 0 ? cdiv(cols, TRI_COLS) : 0);
            k_tri_bwd<T><<<dim3(gx, ny), 256, 0, s>>>(sy, Optr, Lp, Loff, Dp, Doff, k, cb, ws, wsn, nrhs);
            CK_LAUNCH();
        }
    }
}

void tri_inverse_setup(int64_t nsys, const int64_t *Optr, const std::vector<int32_t> &h_n, const double *L64,
                       const int64_t *Loff, int cb, DBuf<int64_t> &Doff, DBuf<double> &D64, cudaStream_t s) {
    if (cb < 1 || cb > TRI_CB) fail(LSAMG_INVALID_ARG, "triangular block size out of range");
    std::vector<int64_t> off(nsys + 1, 0);
    int maxn = 0;
    for (int64_t a = 0; a < nsys; a++) {
        off[a + 1] = off[a] + (int64_t)((h_n[a] + cb - 1) / cb) * tri_block_words(cb);
        maxn = std::max(maxn, h_n[a]);
    }
    upload(Doff, off, s);
    D64.alloc(std::max<int64_t>(off[nsys], 1), s);
    const int K = (maxn + cb - 1) / cb;
    for (int64_t y0 = 0; y0 < nsys && K > 0; y0 += 65535) {
        const unsigned ny = (unsigned)std::min<int64_t>(65535, nsys - y0);
        k_tri_inv<<<dim3((unsigned)K, ny), TRI_CB, 0, s>>>(Optr, L64, Loff, Doff.p, cb, D64.p, y0);
        CK_LAUNCH();
    }
}

// one colour of the sweep with many CTAs per subdomain: gather r_Omega, blocked solves with the
// Cholesky factor of A_Omega, x_Omega += delta, residual update through the element factors
template <class T>
static void sweep_split(Level &L, int c, int nrhs, cudaStream_t s) {
    const int64_t na = L.colptr[c + 1] - L.colptr[c];
    const int32_t *aggs = L.colagg.p + L.colptr[c];
    const T *Lp;
    const T *G;
    if constexpr (std::is_same<T, float>::value) {
        Lp = L.L32.p;
        G = L.G32.p;
    } else {
        Lp = L.L64.p;
        G = L.G64.p;
    }
    T *ws = wsvec<T>(L);
    const int maxn = L.colmax[c];
    dim3 gg((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(maxn, 256), 64)), (unsigned)na);
    k_sw_gather<T><<<gg, 256, 0, s>>>(aggs, L.Optr.p, L.Oidx.p, rvec<T>(L), ws, L.n, L.Omega_total, nrhs);
    CK_LAUNCH();
    tri_solve<T>(aggs, na, L.Optr.p, Lp, L.Loff.p, L.Di64.p, L.Doff.p, L.tri_cb, maxn, ws, L.Omega_total, nrhs, s);
    k_sw_addx<T><<<gg, 256, 0, s>>>(aggs, L.Optr.p, L.Oidx.p, ws, xvec<T>(L), L.n, L.Omega_total, nrhs);
    CK_LAUNCH();
    const int64_t np = L.colpairs[c + 1] - L.colpairs[c];
    if (np > 0) {
        size_t sm = (size_t)std::max(1, L.max_grows_cached) * sizeof(T);
        k_sw_scatter<T><<<(unsigned)std::min<int64_t>(np, 148 * 16), 128, sm, s>>>(
            L.pair_agg.p + L.colpairs[c], L.pair_ent.p + L.colpairs[c], np, L.Optr.p, L.oelocoff.p, L.oeloc.p,
            L.oeidx.p, L.eptr.p, L.eidx.p, G, L.goff.p, L.grows.p, ws, rvec<T>(L), L.n, L.Omega_total, nrhs);
        CK_LAUNCH();
    }
}

template <class T>
static void sweep(Level &L, int c, int nrhs, cudaStream_t s) {
    const int64_t na = L.colptr[c + 1] - L.colptr[c];
    if (na == 0) return;
    if (L.colmax[c] > g_split_sweep) {
        KTime kt(KC_SCHWARZ, s, 0.0, L.sweep_bytes[std::is_same<T, double>::value ? 1 : 0][c]);
        sweep_split<T>(L, c, nrhs, s);
        return;
    }
    const T *Lp;
    const T *G;
    if constexpr (std::is_same<T, float>::value) {
        Lp = L.L32.p;
        G = L.G32.p;
    } else {
        Lp = L.L64.p;
        G = L.G64.p;
    }
    size_t sm = (size_t)std::max(1, L.max_grows_cached) * sizeof(T);
    KTime kt(KC_SCHWARZ, s, 0.0, L.sweep_bytes[std::is_same<T, double>::value ? 1 : 0].empty() ? 0.0
                                     : L.sweep_bytes[std::is_same<T, double>::value ? 1 : 0][c]);
    k_schwarz<T><<<(unsigned)std::min<int64_t>(na, 148 * 8), 256, sm, s>>>(
        L.colagg.p + L.colptr[c], na, L.Optr.p, L.Oidx.p, Lp, L.Loff.p, L.oeptr.p, L.oeidx.p,
        L.oelocoff.p, L.oeloc.p, L.eptr.p, L.eidx.p, G, L.goff.p, L.grows.p, xvec<T>(L), rvec<T>(L),
        wsvec<T>(L), L.n, L.Omega_total, nrhs);
    CK_LAUNCH();
}

// Additive block Schwarz on the overlaps (the parallel smoother Section 2 allows):
// x += theta sum_i R_Omega_i^T A_Omega_i^{-1} R_Omega_i r over every subdomain at once, with
// theta = 1 / #colours (same-colour subdomains share no element, so each colour's projections
// sum to a projection and the damped smoother is A-non-expansive); then r = b - A x if asked.
template <class T>
static void additive_smooth(Level &L, int nrhs, bool update_residual, cudaStream_t s) {
    const int64_t na = L.ncol > 0 ? L.colptr[L.ncol] : 0;   // every subdomain, in colour order
    if (na == 0) return;
    const T *Lp;
    if constexpr (std::is_same<T, float>::value) Lp = L.L32.p; else Lp = L.L64.p;
    T *ws = wsvec<T>(L);
    int maxn = 0;
    double bytes = 0.0;
    for (int c = 0; c < L.ncol; c++) {
        maxn = std::max(maxn, L.colmax[c]);
        bytes += L.sweep_bytes[std::is_same<T, double>::value ? 1 : 0][c];
    }
    const T theta = (T)(1.0 / (double)L.ncol);
    {
        KTime kt(KC_SCHWARZ, s, 0.0, bytes);
        for (int64_t y0 = 0; y0 < na; y0 += 65535) {
            dim3 gg((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(maxn, 256), 64)),
                    (unsigned)std::min<int64_t>(65535, na - y0));
            k_sw_gather<T><<<gg, 256, 0, s>>>(L.colagg.p + y0, L.Optr.p, L.Oidx.p, rvec<T>(L), ws, L.n,
                                              L.Omega_total, nrhs);
            CK_LAUNCH();
        }
        tri_solve<T>(L.colagg.p, na, L.Optr.p, Lp, L.Loff.p, L.Di64.p, L.Doff.p, L.tri_cb, maxn, ws,
                     L.Omega_total, nrhs, s);
        for (int64_t y0 = 0; y0 < na; y0 += 65535) {
            dim3 gg((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(maxn, 256), 64)),
                    (unsigned)std::min<int64_t>(65535, na - y0));
            k_sw_addx_scaled<T><<<gg, 256, 0, s>>>(L.colagg.p + y0, L.Optr.p, L.Oidx.p, ws, xvec<T>(L), theta,
                                                   L.n, L.Omega_total, nrhs);
            CK_LAUNCH();
        }
    }
    if (update_residual) gram_spmv<T>(L, xvec<T>(L), rvec<T>(L), bvec<T>(L), nrhs, s);
}

template <class T>
void vcycle(Handle &H, int l, int nrhs, cudaStream_t s) {
    Level &L = H.levels[l];
    const int64_t tot = L.n * nrhs;
    T *b = bvec<T>(L), *x = xvec<T>(L), *r = rvec<T>(L);
    if (L.coarsest) {
        LSAMG_PROF("vc: coarsest solve", s);
        CK(cudaMemcpyAsync(x, b, tot * sizeof(T), cudaMemcpyDeviceToDevice, s));
        const T *Ld;
        if constexpr (std::is_same<T, float>::value) Ld = L.Ld32.p; else Ld = L.Ld64.p;
        KTime kt(KC_COARSE_SOLVE, s, 0.0, L.coarse_bytes[std::is_same<T, double>::value ? 1 : 0] * nrhs);
        tri_solve<T>(nullptr, 1, L.cs_ptr.p, Ld, L.cs_off.p, L.Di64.p, L.Doff.p, L.tri_cb, (int)L.n, x, L.n, nrhs, s);
        return;
    }
    Level &C = H.levels[l + 1];
    CK(cudaMemsetAsync(x, 0, tot * sizeof(T), s));
    CK(cudaMemcpyAsync(r, b, tot * sizeof(T), cudaMemcpyDeviceToDevice, s));
    {
        LSAMG_PROF(l == 0 ? "vc: L0 pre-smooth" : "vc: Lc pre-smooth", s);
        if (H.opt.smoother == 1)
            additive_smooth<T>(L, nrhs, true, s);
        else
            for (int c = 0; c < L.ncol; c++) sweep<T>(L, c, nrhs, s);
    }
    const T *Z;
    if constexpr (std::is_same<T, float>::value) Z = L.Z32.p; else Z = L.Z64.p;
    {
    KTime kt(KC_TRANSFER, s);
    k_restrict<T><<<gridv(L.nagg, 1, 148 * 16), 256, 0, s>>>(L.wptr.p, L.widx.p, L.k.p, L.off.p, Z,
                                                            L.zoff.p, L.nagg, r, L.n, bvec<T>(C),
                                                            C.n, nrhs);
    CK_LAUNCH();
    }
    vcycle<T>(H, l + 1, nrhs, s);
    {
    KTime kt(KC_TRANSFER, s);
    const size_t ism = (size_t)std::max(1, L.max_k) * sizeof(T);
    if (ism > 48 * 1024) {
        if (ism > 227 * 1024) fail(LSAMG_LIMIT, "coarse block too large for the interpolation kernel");
        CK(cudaFuncSetAttribute(k_interp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism));
    }
    k_interp<T><<<gridv(L.nagg, 1, 148 * 16), 256, ism, s>>>(L.wptr.p, L.widx.p, L.k.p, L.off.p, Z,
                                                          L.zoff.p, L.nagg, xvec<T>(C), C.n, x,
                                                          L.n, nrhs);
    CK_LAUNCH();
    }
    // residual after the coarse correction: r = b - A x
    CK(cudaMemcpyAsync(r, b, tot * sizeof(T), cudaMemcpyDeviceToDevice, s));
    {
        LSAMG_PROF(l == 0 ? "vc: L0 residual spmv" : "vc: Lc residual spmv", s);
        KTime kt(KC_SPMV, s, 0.0, L.spmv_bytes[std::is_same<T, double>::value ? 1 : 0]);
        const T *G;
        if constexpr (std::is_same<T, float>::value) G = L.G32.p; else G = L.G64.p;
        size_t sm = (size_t)std::max(1, L.max_grows_cached) * sizeof(T);
        k_spmv<T><<<gridv(L.ne, 1, 148 * 24), 128, sm, s>>>(L.eptr.p, L.eidx.p, L.ne, G, L.goff.p,
                                                          L.grows.p, x, r, L.n, nrhs, (T)-1);
        CK_LAUNCH();
    }
    {
        LSAMG_PROF(l == 0 ? "vc: L0 post-smooth" : "vc: Lc post-smooth", s);
        if (H.opt.smoother == 1)
            additive_smooth<T>(L, nrhs, false, s);
        else
            for (int c = L.ncol - 1; c >= 0; c--) sweep<T>(L, c, nrhs, s);
    }
}

template void vcycle<float>(Handle &, int, int, cudaStream_t);
template void vcycle<double>(Handle &, int, int, cudaStream_t);
template void gram_spmv<float>(const Level &, const float *, float *, const float *, int, cudaStream_t);
template void gram_spmv<double>(const Level &, const double *, double *, const double *, int,
                                cudaStream_t);

void elem_grad(const Level &L, const double *coef, const double *lam, const double *x, double *g,
               cudaStream_t s) {
    if (L.ne == 0) return;
    k_elem_grad<<<gridv(L.ne * 32), 256, 0, s>>>(L.eptr.p, L.eidx.p, L.ne, L.G64.p, L.goff.p,
                                                 L.grows.p, coef, lam, x, g);
    CK_LAUNCH();
}

void vec_dots(const double *a, const double *b, int64_t n, int nrhs, double *out, cudaStream_t s) {
    CK(cudaMemsetAsync(out, 0, nrhs * sizeof(double), s));
    k_dots<<<gridv(n, 256, 148 * 4), 256, 0, s>>>(a, b, n, nrhs, out);
    CK_LAUNCH();
}

void vec_axpy(double *y, const double *x, const double *alpha, int64_t n, int nrhs, double sign,
              cudaStream_t s) {
    k_axpy<<<gridv(n * nrhs), 256, 0, s>>>(y, x, alpha, n, nrhs, sign);
    CK_LAUNCH();
}

void vec_xpby(double *p, const double *z, const double *beta, int64_t n, int nrhs, cudaStream_t s) {
    k_xpby<<<gridv(n * nrhs), 256, 0, s>>>(p, z, beta, n, nrhs);
    CK_LAUNCH();
}

template <class A, class B>
void vec_convert(B *dst, const A *src, int64_t count, cudaStream_t s) {
    if (count <= 0) return;
    k_convert<A, B><<<gridv(count), 256, 0, s>>>(dst, src, count);
    CK_LAUNCH();
}
template void vec_convert<double, float>(float *, const double *, int64_t, cudaStream_t);
template void vec_convert<float, double>(double *, const float *, int64_t, cudaStream_t);
template void vec_convert<double, double>(double *, const double *, int64_t, cudaStream_t);

}  // namespace lsamg
