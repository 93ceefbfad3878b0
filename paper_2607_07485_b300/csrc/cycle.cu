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

// The same for levels whose element blocks fit 64 x 64 (the fine level: 40 x 40): a warp per
// element, eight per CTA.  G_T is loaded once, coalesced, into the warp's shared tile (rows padded
// to nT + 1: conflict-free row and column reads); t = G_T x_T with lanes on rows, then
// G_T^T t with lanes on columns, x_T gathered once per right-hand side and broadcast by shuffles.
constexpr int SPMV_WARPS = 8;
constexpr int SPMV_LOADS = 8;
template <class T>
__global__ void __launch_bounds__(256) k_spmv_warp(const int64_t *eptr, const int32_t *eidx, int64_t ne,
                                                   const T *G, const int64_t *goff, const int32_t *grows,
                                                   const T *x, T *y, int64_t n, int nrhs, T sign, int ldt,
                                                   int rows) {
    extern __shared__ unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *Gs = reinterpret_cast<T *>(smraw) + (int64_t)warp * rows * ldt;
    for (int64_t e = (int64_t)blockIdx.x * SPMV_WARPS + warp; e < ne; e += (int64_t)gridDim.x * SPMV_WARPS) {
        const int64_t b = eptr[e];
        const int nT = (int)(eptr[e + 1] - b);
        const int m = grows[e];
        const T *g = G + goff[e];
        // SPMV_LOADS loads per lane in flight before their stores (a load-store loop would wait
        // for each load in turn)
        const int tot = m * nT;
        for (int t0 = 0; t0 < tot; t0 += 32 * SPMV_LOADS) {
            T v[SPMV_LOADS];
#pragma unroll
            for (int u = 0; u < SPMV_LOADS; u++) {
                const int t = t0 + 32 * u + lane;
                v[u] = t < tot ? g[t] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < SPMV_LOADS; u++) {
                const int t = t0 + 32 * u + lane;
                if (t < tot) {
                    const int i = t / nT, c = t - i * nT;
                    Gs[i * ldt + c] = v[u];
                }
            }
        }
        const int d0 = lane < nT ? eidx[b + lane] : 0, d1 = lane + 32 < nT ? eidx[b + 32 + lane] : 0;
        __syncwarp();
        for (int r = 0; r < nrhs; r++) {
            const T *xr = x + (int64_t)r * n;
            const T x0 = lane < nT ? xr[d0] : (T)0, x1 = lane + 32 < nT ? xr[d1] : (T)0;
            T t0 = 0, t1 = 0;
            for (int c = 0; c < nT; c++) {
                const T xc = __shfl_sync(0xffffffffu, c < 32 ? x0 : x1, c & 31);
                if (lane < m) t0 += Gs[lane * ldt + c] * xc;
                if (lane + 32 < m) t1 += Gs[(lane + 32) * ldt + c] * xc;
            }
            T y0 = 0, y1 = 0;
            for (int i = 0; i < m; i++) {
                const T ti = __shfl_sync(0xffffffffu, i < 32 ? t0 : t1, i & 31);
                if (lane < nT) y0 += Gs[i * ldt + lane] * ti;
                if (lane + 32 < nT) y1 += Gs[i * ldt + lane + 32] * ti;
            }
            T *yr = y + (int64_t)r * n;
            if (lane < nT) atomicAdd(&yr[d0], sign * y0);
            if (lane + 32 < nT) atomicAdd(&yr[d1], sign * y1);
        }
        __syncwarp();
    }
}

// Larger elements (the Galerkin levels): a CTA per element.  x_T is gathered once into shared
// memory; the rows go by chunks of SPMV_RC: first t_i = G_T(i,:) x_T for the chunk's rows (a warp
// per two rows, lanes along the rows, eight loads per lane in flight), then the chunk's share
// G_T(chunk,:)^T t of the column sums, which stay in shared memory (each column owned by one
// thread).  The second pass re-reads a chunk read just before (16 rows, from L1/L2), so G_T
// crosses HBM once.  The arithmetic order is that of k_spmv: row sums lane-strided then
// shuffle-reduced, column sums row by row.
constexpr int SPMV_RC = 16;
template <class T>
__global__ void __launch_bounds__(256) k_spmv_rows(const int64_t *eptr, const int32_t *eidx, int64_t ne,
                                                   const T *G, const int64_t *goff, const int32_t *grows,
                                                   const T *x, T *y, int64_t n, int nrhs, T sign, int ldx) {
    extern __shared__ unsigned char smraw[];
    T *xs = reinterpret_cast<T *>(smraw);
    T *ys = xs + ldx;
    T *ts = ys + ldx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = 8;   // warps per CTA (launch bounds 256)
    for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
        const int64_t b = eptr[e];
        const int nT = (int)(eptr[e + 1] - b);
        const int m = grows[e];
        const T *g = G + goff[e];
        for (int r = 0; r < nrhs; r++) {
            const T *xr = x + (int64_t)r * n;
            for (int c = threadIdx.x; c < nT; c += blockDim.x) {
                xs[c] = xr[eidx[b + c]];
                ys[c] = (T)0;
            }
            __syncthreads();
            for (int i0 = 0; i0 < m; i0 += SPMV_RC) {
                const int rc = min(SPMV_RC, m - i0);
                if (warp < rc) {
                    const int i2 = warp + NW;
                    const bool two = i2 < rc;
                    const T *g1 = g + (int64_t)(i0 + warp) * nT;
                    const T *g2 = g + (int64_t)(i0 + (two ? i2 : warp)) * nT;
                    T s1 = 0, s2 = 0;
#pragma unroll 4
                    for (int c = lane; c < nT; c += 32) {
                        const T xc = xs[c];
                        s1 += g1[c] * xc;
                        if (two) s2 += g2[c] * xc;
                    }
                    s1 = warp_sum(s1);
                    s2 = warp_sum(s2);
                    if (lane == 0) {
                        ts[warp] = s1;
                        if (two) ts[i2] = s2;
                    }
                }
                __syncthreads();
                for (int c = threadIdx.x; c < nT; c += blockDim.x) {
                    const T *gc = g + (int64_t)i0 * nT + c;
                    T acc = ys[c];
#pragma unroll 4
                    for (int i = 0; i < rc; i++) acc += gc[(int64_t)i * nT] * ts[i];
                    ys[c] = acc;
                }
                __syncthreads();
            }
            T *yr = y + (int64_t)r * n;
            for (int c = threadIdx.x; c < nT; c += blockDim.x) atomicAdd(&yr[eidx[b + c]], sign * ys[c]);
            __syncthreads();
        }
    }
}

// shared memory of the warp-per-element kernels (eight padded G_T tiles), 0 when the level's
// element blocks exceed 64 x 64 or the tiles exceed 200 KB
template <class T>
size_t spmv_warp_smem(const Level &L) {
    if (L.max_nT > 64 || L.max_grows_cached > 64) return 0;
    const size_t sm = (size_t)SPMV_WARPS * std::max(1, L.max_grows_cached) * (L.max_nT + 1) * sizeof(T);
    return sm <= 200 * 1024 ? sm : 0;
}

// launches the Gram SpMV of level L: y (+)= sign G^T G x
template <class T>
void launch_spmv(const Level &L, const T *G, const T *x, T *y, int nrhs, T sign, cudaStream_t s) {
    const size_t rows_sm = (2 * (size_t)std::max(1, L.max_nT) + SPMV_RC) * sizeof(T);
    if (const size_t sm = spmv_warp_smem<T>(L)) {
        const int ldt = L.max_nT + 1, rows = std::max(1, L.max_grows_cached);
        CK(cudaFuncSetAttribute(k_spmv_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const unsigned grid = gridv(L.ne, SPMV_WARPS, 148 * 8);
        k_spmv_warp<T><<<grid, 32 * SPMV_WARPS, sm, s>>>(L.eptr.p, L.eidx.p, L.ne, G, L.goff.p, L.grows.p, x, y,
                                                        L.n, nrhs, sign, ldt, rows);
    } else if (rows_sm <= 160 * 1024) {
        CK(cudaFuncSetAttribute(k_spmv_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_sm));
        k_spmv_rows<T><<<gridv(L.ne, 1, 148 * 8), 256, rows_sm, s>>>(L.eptr.p, L.eidx.p, L.ne, G, L.goff.p,
                                                                     L.grows.p, x, y, L.n, nrhs, sign,
                                                                     std::max(1, L.max_nT));
    } else {
        const size_t sm = (size_t)std::max(1, L.max_grows_cached) * sizeof(T);
        k_spmv<T><<<gridv(L.ne, 1, 148 * 24), 128, sm, s>>>(L.eptr.p, L.eidx.p, L.ne, G, L.goff.p, L.grows.p, x,
                                                          y, L.n, nrhs, sign);
    }
    CK_LAUNCH();
}

template <class T>
double spmv_flops(const Level &L, int nrhs) {
    return std::is_same<T, double>::value ? 2.0 * L.spmv_fmas * nrhs : 0.0;   // FP64 work only
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
// rc[off_a + j] = sum_p Z_a[p, j] res[omega_a[p]] (P^T r, P = blockdiag R_omega^T Z_a).  CTA
// (x, a) takes the 128 columns 128 x .. of Z_a over all its rows: the 8 warps take interleaved
// rows (coalesced, 4 rows in flight), lanes 4 x 32 columns, and the warps' partial sums are added
// in shared memory in a fixed order.  Large coarse blocks are spread over several CTAs.
template <class T>
__global__ void __launch_bounds__(256) k_restrict(const int64_t *wptr, const int32_t *widx, const int32_t *k,
                                                  const int64_t *off, const T *Z, const int64_t *zoff,
                                                  int64_t nagg, const T *res, int64_t n, T *rc, int64_t nc,
                                                  int nrhs) {
    __shared__ T red[8][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = (int)blockIdx.x * 128;
    for (int64_t a = blockIdx.y; a < nagg; a += gridDim.y) {
        const int ka = k[a];
        if (j0 >= ka) continue;
        const int64_t wb = wptr[a];
        const int nw = (int)(wptr[a + 1] - wb);
        const T *z = Z + zoff[a];
        for (int r = 0; r < nrhs; r++) {
            const T *rr = res + (int64_t)r * n;
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

// x[omega_a[p]] += sum_j Z_a[p, j] ec[off_a + j] (x += P e_c).  CTA (x, a) takes rows
// TR_ROWS x .. of aggregate a: the coarse values staged in shared memory, a warp per row of Z_a
// (4 rows in flight).
constexpr int TR_ROWS = 64;
template <class T>
__global__ void __launch_bounds__(256) k_interp(const int64_t *wptr, const int32_t *widx, const int32_t *k,
                                                const int64_t *off, const T *Z, const int64_t *zoff,
                                                int64_t nagg, const T *ec, int64_t nc, T *x, int64_t n,
                                                int nrhs) {
    extern __shared__ unsigned char smraw[];
    T *e = reinterpret_cast<T *>(smraw);   // [max k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p0 = (int)blockIdx.x * TR_ROWS;
    for (int64_t a = blockIdx.y; a < nagg; a += gridDim.y) {
        const int ka = k[a];
        const int64_t wb = wptr[a];
        const int nw = (int)(wptr[a + 1] - wb);
        if (p0 >= nw || ka == 0) continue;
        const int p1 = min(nw, p0 + TR_ROWS);
        const T *z = Z + zoff[a];
        for (int r = 0; r < nrhs; r++) {
            __syncthreads();
            for (int j = threadIdx.x; j < ka; j += blockDim.x) e[j] = ec[(int64_t)r * nc + off[a] + j];
            __syncthreads();
            T *xr = x + (int64_t)r * n;
#pragma unroll 4
            for (int p = p0 + warp; p < p1; p += 8) {
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
// The Schwarz (and coarsest) factors are packed lower row-major (row i at offset i(i+1)/2).  Rows
// are cut into blocks of cb <= TRI_CB rows whose diagonal blocks are inverted once at set-up
// (Dinv, FP64 packed lower row-major, block b of system a at Doff[a] + b cb(cb+1)/2; the product
// with it is formed in FP64 in the FP32 cycle too, since an explicit inverse of an
// ill-conditioned block rounded to FP32 loses its small components to cancellation).
constexpr int TRI_CB = 64;      // largest block

__host__ __device__ inline int64_t tri_block_words(int cb) { return (int64_t)cb * (cb + 1) / 2; }

// ---------------------------------------------------------------- wavefront triangular solves
// L L^T v = v for the systems of one solve group (a Schwarz colour, all subdomains, or the
// coarsest matrix) in two persistent cooperative launches, one per substitution.  A task is one
// block row (forward) or block column (backward) of cb <= 64 rows of one system; the tasks are
// listed in dependency order (forward: by block index, backward: by distance from the last
// block) and CTA c takes tasks c, c + grid, ...  A task streams its part of the packed factor once,
// consuming finished blocks of the same system as their flags come up (epoch-stamped, acquire /
// release), applies the FP64 inverted diagonal block and publishes its own block.  Since every
// CTA is resident (cooperative launch) and a task waits only on tasks listed before it, the
// smallest unfinished task can always proceed.  Every wait is bounded (2 s on the global timer):
// on expiry the kernel records LSAMG_DEVICE_TIMEOUT and returns.
constexpr int WF_RG = 4;            // right-hand sides per pass over the factor

__device__ __forceinline__ uint32_t wf_load_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void wf_store_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t wf_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// thread 0 waits until flag >= epoch (wrap-safe); the CTA then proceeds together.  Returns false
// (for every thread) when the wait gave up.
__device__ __forceinline__ bool wf_wait(const uint32_t *flag, uint32_t epoch, int *err, int *s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if ((int32_t)(wf_load_acquire(flag) - epoch) < 0) {
            const uint64_t t0 = wf_timer();
            while ((int32_t)(wf_load_acquire(flag) - epoch) < 0) {
                if (wf_timer() - t0 > 2000000000ull) {
                    ok = 0;
                    if (err && atomicCAS(err, 0, LSAMG_DEVICE_TIMEOUT) == 0) err[1] = (int)blockIdx.x;
                    break;
                }
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <class T, bool FWD, int RG>
__global__ void __launch_bounds__(256, FWD ? (RG > 1 ? 2 : 3) : 4) k_tri_wave(const int32_t *tasks, int64_t ntask, const int32_t *sys,
                                                  const int64_t *Optr, const T *Lp, const int64_t *Loff,
                                                  const double *Dp, const int64_t *Doff, const int64_t *Foff,
                                                  uint32_t *flags, uint32_t epoch, int cb, T *ws, int64_t wsn,
                                                  int nrhs, int *err) {
    __shared__ T yj[RG][TRI_CB];
    __shared__ double tv[RG][TRI_CB];
    __shared__ double vo[RG][TRI_CB];                    // this block of the right-hand sides
    __shared__ double red[8][RG][TRI_CB];
    __shared__ double sDi[TRI_CB * (TRI_CB + 1) / 2];       // inverted diagonal block
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t q = blockIdx.x; q < ntask; q += gridDim.x) {
        const int si = tasks[2 * q], k = tasks[2 * q + 1];
        const int32_t a = sys ? sys[si] : si;
        const int64_t ob = Optr[a];
        const int n = (int)(Optr[a + 1] - ob);
        const int K = (n + cb - 1) / cb;
        const int r0 = k * cb, nb = min(cb, n - r0);
        const T *L = Lp + Loff[a];
        T *v = ws + ob;
        uint32_t *fl = flags + Foff[a];
        {
            // the inverted diagonal block is staged while the dependencies are consumed (it is
            // needed only at the end of the task, on the critical path of the wavefront)
            const double *Di = Dp + Doff[a] + (int64_t)k * tri_block_words(cb);
            const int nw = nb * (nb + 1) / 2;
            for (int t = threadIdx.x; t < nw; t += blockDim.x) sDi[t] = __ldg(Di + t);
        }
        for (int g0 = 0; g0 < nrhs; g0 += RG) {
            const int nr = min(RG, nrhs - g0);
            // own block of the right-hand sides: written only by this task
            for (int t = threadIdx.x; t < nr * TRI_CB; t += blockDim.x) {
                const int r = t / TRI_CB, c = t - r * TRI_CB;
                vo[r][c] = (c < nb) ? (double)__ldcg(v + (int64_t)(g0 + r) * wsn + r0 + c) : 0.0;
            }
            // per-warp partial sums over every dependency block: forward, rows warp + 8 i of the
            // block (each lane over two columns); backward, columns lane / lane + 32 (each warp
            // over rows warp + 8 i of the dependency block)
            T part[RG][8];
#pragma unroll
            for (int r = 0; r < RG; r++)
#pragma unroll
                for (int i = 0; i < 8; i++) part[r][i] = 0;
            const int jn = FWD ? k : K - 1 - k;          // dependency blocks
            for (int jj = 0; jj < jn; jj++) {
                const int j = FWD ? jj : K - 1 - jj;
                const int c0 = j * cb, nc = min(cb, n - c0);
                // the factor block does not depend on the wavefront: its loads are in flight
                // before the wait for block j
                T lv[8][2];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int ii = warp + 8 * i;
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int c = lane + 32 * u;
                        if (FWD) {   // L[r0 + i, c0 + c]: rows of this block, columns of block j
                            const int64_t gi = (int64_t)r0 + ii;
                            lv[i][u] = (ii < nb && c < nc) ? L[gi * (gi + 1) / 2 + c0 + c] : (T)0;
                        } else {     // L[c0 + i, r0 + c]: rows of block j, columns of this block
                            const int64_t gi = (int64_t)c0 + ii;
                            lv[i][u] = (ii < nc && c < nb) ? L[gi * (gi + 1) / 2 + r0 + c] : (T)0;
                        }
                    }
                }
                if (!wf_wait(fl + j, epoch, err, &s_ok)) return;
                for (int t = threadIdx.x; t < nr * TRI_CB; t += blockDim.x) {
                    const int r = t / TRI_CB, c = t - r * TRI_CB;
                    yj[r][c] = (c < nc) ? __ldcg(v + (int64_t)(g0 + r) * wsn + c0 + c) : (T)0;
                }
                __syncthreads();
                if (FWD) {
#pragma unroll
                    for (int r = 0; r < RG; r++)
                        if (r < nr)
#pragma unroll
                            for (int i = 0; i < 8; i++) part[r][i] += lv[i][0] * yj[r][lane] + lv[i][1] * yj[r][lane + 32];
                } else {
#pragma unroll
                    for (int r = 0; r < RG; r++)
                        if (r < nr)
#pragma unroll
                            for (int i = 0; i < 8; i++) {
                                const T y = yj[r][warp + 8 * i];
                                part[r][0] += lv[i][0] * y;
                                part[r][1] += lv[i][1] * y;
                            }
                }
                __syncthreads();
            }
            // combine the partial sums: t = v_block - (L_block,deps . y_deps)
            if (FWD) {
                // butterfly over the warp: the RG * 8 sums (r, i) end one per group of 32 / (8 RG)
                // lanes (index 8 r + i = lane / (32 / (8 RG))), which then finish the sum
                constexpr int NV = RG * 8, SPAN = 32 / NV;
                static_assert(NV <= 32 && 32 % NV == 0, "partial sums per lane");
                double x[NV];
#pragma unroll
                for (int r = 0; r < RG; r++)
#pragma unroll
                    for (int i = 0; i < 8; i++) x[8 * r + i] = (double)part[r][i];
#pragma unroll
                for (int o = 16, c = NV; c > 1; o >>= 1, c >>= 1) {
                    const bool up = (lane & o) != 0;
#pragma unroll
                    for (int t = 0; t < c / 2; t++) {
                        const double send = up ? x[t] : x[t + c / 2];
                        const double keep = up ? x[t + c / 2] : x[t];
                        x[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
#pragma unroll
                for (int o = SPAN / 2; o >= 1; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
                if (lane % SPAN == 0) {
                    const int idx = lane / SPAN;
                    red[0][idx >> 3][warp + 8 * (idx & 7)] = x[0];
                }
                __syncthreads();
                for (int t = threadIdx.x; t < nr * TRI_CB; t += blockDim.x) {
                    const int r = t / TRI_CB, i = t - r * TRI_CB;
                    tv[r][i] = (i < nb) ? vo[r][i] - red[0][r][i] : 0.0;
                }
            } else {
#pragma unroll
                for (int r = 0; r < RG; r++) {   // columns lane and lane + 32, summed over this warp's rows
                    red[warp][r][lane] = (double)part[r][0];
                    red[warp][r][lane + 32] = (double)part[r][1];
                }
                __syncthreads();
                for (int t = threadIdx.x; t < nr * TRI_CB; t += blockDim.x) {
                    const int r = t / TRI_CB, c = t - r * TRI_CB;
                    double sacc = 0.0;
#pragma unroll
                    for (int w = 0; w < 8; w++) sacc += red[w][r][c];
                    tv[r][c] = (c < nb) ? vo[r][c] - sacc : 0.0;
                }
            }
            __syncthreads();
            // this block: y = Dinv t (forward) or x = Dinv^T t (backward), FP64; 4 threads per entry
            {
                const int e = threadIdx.x >> 2, p = threadIdx.x & 3;
                double acc[RG];
#pragma unroll
                for (int r = 0; r < RG; r++) acc[r] = 0.0;
                if (e < nb) {
                    if (FWD) {
                        for (int c = p; c <= e; c += 4) {
                            const double d = sDi[e * (e + 1) / 2 + c];
#pragma unroll
                            for (int r = 0; r < RG; r++)
                                if (r < nr) acc[r] += d * tv[r][c];
                        }
                    } else {
                        for (int i = e + p; i < nb; i += 4) {
                            const double d = sDi[i * (i + 1) / 2 + e];
#pragma unroll
                            for (int r = 0; r < RG; r++)
                                if (r < nr) acc[r] += d * tv[r][i];
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < RG; r++) {
                    acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], 1);
                    acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], 2);
                }
                __syncthreads();
                if (p == 0 && e < nb)
                    for (int r = 0; r < nr; r++) v[(int64_t)(g0 + r) * wsn + r0 + e] = (T)acc[r];
            }
            __syncthreads();
        }
        // publish the block
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) wf_store_release(fl + k, epoch);
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

// The same for levels whose element blocks fit 64 x 64 (the fine level): a warp per pair, eight
// per CTA, G_T staged in the warp's shared tile as in k_spmv_warp (rows padded to nT + 1), the
// subdomain correction gathered once per right-hand side and broadcast by shuffles.
template <class T>
__global__ void __launch_bounds__(256) k_sw_scatter_warp(const int32_t *pa, const int64_t *pj, int64_t npairs,
                                                         const int64_t *Optr, const int64_t *locoff,
                                                         const int32_t *loc, const int32_t *oeidx,
                                                         const int64_t *eptr, const int32_t *eidx, const T *G,
                                                         const int64_t *goff, const int32_t *grows, const T *ws,
                                                         T *res, int64_t n, int64_t wsn, int nrhs, int ldt,
                                                         int rows) {
    extern __shared__ unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *Gs = reinterpret_cast<T *>(smraw) + (int64_t)warp * rows * ldt;
    for (int64_t q = (int64_t)blockIdx.x * SPMV_WARPS + warp; q < npairs; q += (int64_t)gridDim.x * SPMV_WARPS) {
        const int32_t a = pa[q];
        const int64_t j = pj[q];
        const int32_t e = oeidx[j];
        const int64_t b = eptr[e];
        const int nT = (int)(eptr[e + 1] - b);
        const int m = grows[e];
        const T *g = G + goff[e];
        const int32_t *lc = loc + locoff[j];
        const int tot = m * nT;
        for (int t0 = 0; t0 < tot; t0 += 32 * SPMV_LOADS) {
            T v[SPMV_LOADS];
#pragma unroll
            for (int u = 0; u < SPMV_LOADS; u++) {
                const int t = t0 + 32 * u + lane;
                v[u] = t < tot ? g[t] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < SPMV_LOADS; u++) {
                const int t = t0 + 32 * u + lane;
                if (t < tot) {
                    const int i = t / nT, c = t - i * nT;
                    Gs[i * ldt + c] = v[u];
                }
            }
        }
        const int p0 = lane < nT ? lc[lane] : -1, p1 = lane + 32 < nT ? lc[lane + 32] : -1;
        const int d0 = lane < nT ? eidx[b + lane] : 0, d1 = lane + 32 < nT ? eidx[b + 32 + lane] : 0;
        __syncwarp();
        for (int r = 0; r < nrhs; r++) {
            const T *v = ws + (int64_t)r * wsn + Optr[a];
            const T x0 = p0 >= 0 ? v[p0] : (T)0, x1 = p1 >= 0 ? v[p1] : (T)0;
            T t0 = 0, t1 = 0;
            for (int c = 0; c < nT; c++) {
                const T xc = __shfl_sync(0xffffffffu, c < 32 ? x0 : x1, c & 31);
                if (lane < m) t0 += Gs[lane * ldt + c] * xc;
                if (lane + 32 < m) t1 += Gs[(lane + 32) * ldt + c] * xc;
            }
            T y0 = 0, y1 = 0;
            for (int i = 0; i < m; i++) {
                const T ti = __shfl_sync(0xffffffffu, i < 32 ? t0 : t1, i & 31);
                if (lane < nT) y0 += Gs[i * ldt + lane] * ti;
                if (lane + 32 < nT) y1 += Gs[i * ldt + lane + 32] * ti;
            }
            T *rr = res + (int64_t)r * n;
            if (lane < nT) atomicAdd(&rr[d0], -y0);
            if (lane + 32 < nT) atomicAdd(&rr[d1], -y1);
        }
        __syncwarp();
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
    KTime kt(KC_SPMV, s, spmv_flops<T>(L, nrhs), L.spmv_bytes[std::is_same<T, double>::value ? 1 : 0]);
    const T *G = std::is_same<T, float>::value ? (const T *)L.G32.p : (const T *)L.G64.p;
    launch_spmv<T>(L, G, x, y, nrhs, b ? (T)-1 : (T)1, s);
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

// L L^T v = v for the systems of solve group `grp` of level L (system array sys, or systems
// 0..nsys-1 when sys == nullptr) whose vectors sit at ws + Optr[a] (stride wsn per right-hand side),
// factors at Lp + Loff[a] and inverted diagonal blocks at Dp + Doff[a] (block size cb): the
// forward and the backward wavefront launches.
template <class T>
static void tri_solve(Level &L, int grp, const int32_t *sys, const int64_t *Optr, const T *Lp,
                      const int64_t *Loff, const double *Dp, const int64_t *Doff, int cb, T *ws, int64_t wsn,
                      int nrhs, cudaStream_t s) {
    const Level::WaveGroup &g = L.wf_groups[grp];
    if (g.ntask == 0) return;
    uint32_t *flags = L.wf_flags.p;
    int *err = reinterpret_cast<int *>(L.wf_flags.p + 2 * L.wf_nflags);
    CK(cudaMemsetAsync(flags, 0, 2 * L.wf_nflags * sizeof(uint32_t), s));
    // one right-hand side: the kernels specialised for it hold a quarter of the partial sums
    static int occ[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
    const int ti = std::is_same<T, double>::value ? 1 : 0;
    const int single = nrhs == 1 ? 1 : 0;
    // right-hand sides in groups of WF_RG, one forward and one backward wavefront per group (epoch
    // = group + 1 on the same flags): a task publishes its block after all the right-hand sides
    // it carries, so carrying more of them in one launch would lengthen the critical path with
    // every group
    for (int g0 = 0, gi = 0; g0 < nrhs; g0 += WF_RG, gi++)
    for (int dir = 0; dir < 2; dir++) {
        const bool fwd = dir == 0;
        void *fn = single ? (fwd ? (void *)k_tri_wave<T, true, 1> : (void *)k_tri_wave<T, false, 1>)
                          : (fwd ? (void *)k_tri_wave<T, true, WF_RG> : (void *)k_tri_wave<T, false, WF_RG>);
        int &oc = occ[single][ti][dir];
        if (!oc) {
            int o = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, 256, 0));
            int dev = 0, sms = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            oc = std::max(1, o) * sms;
        }
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(g.ntask, oc));
        const int32_t *tasks = L.wf_tasks.p + 2 * (fwd ? g.fwd : g.bwd);
        int64_t ntask = g.ntask;
        uint32_t *fl = flags + (fwd ? 0 : L.wf_nflags);
        uint32_t epoch = (uint32_t)gi + 1;
        const int64_t *foff = L.wf_foff.p;
        T *wsg = ws + (int64_t)g0 * wsn;
        int nr = std::min(WF_RG, nrhs - g0);
        void *args[] = {(void *)&tasks, (void *)&ntask, (void *)&sys, (void *)&Optr, (void *)&Lp, (void *)&Loff,
                        (void *)&Dp, (void *)&Doff, (void *)&foff, (void *)&fl, (void *)&epoch, (void *)&cb,
                        (void *)&wsg, (void *)&wsn, (void *)&nr, (void *)&err};
        CK(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, s));
        count_launch();
    }
}

void wave_setup(Level &L, const std::vector<std::vector<int32_t>> &group_sizes,
                const std::vector<std::vector<int32_t>> &group_ids, const std::vector<int32_t> &all_sizes, int cb,
                cudaStream_t s) {
    std::vector<int64_t> foff(all_sizes.size() + 1, 0);
    for (size_t a = 0; a < all_sizes.size(); a++) foff[a + 1] = foff[a] + cdiv(all_sizes[a], cb);
    std::vector<int32_t> tasks;
    L.wf_groups.clear();
    for (size_t gi = 0; gi < group_sizes.size(); gi++) {
        const auto &sz = group_sizes[gi];
        Level::WaveGroup g;
        int Kmax = 0;
        for (auto n : sz) Kmax = std::max<int>(Kmax, (int)cdiv(n, cb));
        g.fwd = (int64_t)tasks.size() / 2;
        for (int k = 0; k < Kmax; k++)            // forward: by block index, then system
            for (size_t i = 0; i < sz.size(); i++)
                if (k < cdiv(sz[i], cb)) {
                    tasks.push_back((int32_t)i);
                    tasks.push_back(k);
                }
        g.ntask = (int64_t)tasks.size() / 2 - g.fwd;
        g.bwd = (int64_t)tasks.size() / 2;
        for (int d = 0; d < Kmax; d++)            // backward: by distance from the last block
            for (size_t i = 0; i < sz.size(); i++) {
                const int K = (int)cdiv(sz[i], cb);
                if (d < K) {
                    tasks.push_back((int32_t)i);
                    tasks.push_back(K - 1 - d);
                }
            }
        (void)group_ids;
        L.wf_groups.push_back(g);
    }
    upload(L.wf_tasks, tasks, s);
    upload(L.wf_foff, std::vector<int64_t>(foff.begin(), foff.end() - 1), s);
    L.wf_nflags = foff.back();
    L.wf_flags.alloc(2 * L.wf_nflags + 2, s);
    L.wf_flags.zero(s);
}

void wave_check(const Level &L, cudaStream_t s) {
    if (!L.wf_flags.p) return;
    int h[2];
    CK(cudaMemcpyAsync(h, L.wf_flags.p + 2 * L.wf_nflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[0] != 0) {
        char buf[200];
        snprintf(buf, sizeof buf, "triangular solve: a dependency wait gave up (code %d, CTA %d)", h[0], h[1]);
        fail(h[0], buf);
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
    tri_solve<T>(L, c, aggs, L.Optr.p, Lp, L.Loff.p, L.Di64.p, L.Doff.p, L.tri_cb, ws, L.Omega_total, nrhs, s);
    k_sw_addx<T><<<gg, 256, 0, s>>>(aggs, L.Optr.p, L.Oidx.p, ws, xvec<T>(L), L.n, L.Omega_total, nrhs);
    CK_LAUNCH();
    const int64_t np = L.colpairs[c + 1] - L.colpairs[c];
    const size_t wsm = spmv_warp_smem<T>(L);
    if (np > 0 && wsm > 0) {
        const int ldt = L.max_nT + 1, rows = std::max(1, L.max_grows_cached);
        const size_t sm = wsm;
        CK(cudaFuncSetAttribute(k_sw_scatter_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_sw_scatter_warp<T><<<gridv(np, SPMV_WARPS, 148 * 8), 32 * SPMV_WARPS, sm, s>>>(
            L.pair_agg.p + L.colpairs[c], L.pair_ent.p + L.colpairs[c], np, L.Optr.p, L.oelocoff.p, L.oeloc.p,
            L.oeidx.p, L.eptr.p, L.eidx.p, G, L.goff.p, L.grows.p, ws, rvec<T>(L), L.n, L.Omega_total, nrhs, ldt,
            rows);
        CK_LAUNCH();
    } else if (np > 0) {
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
        tri_solve<T>(L, L.ncol, L.colagg.p, L.Optr.p, Lp, L.Loff.p, L.Di64.p, L.Doff.p, L.tri_cb, ws,
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
        tri_solve<T>(L, 0, nullptr, L.cs_ptr.p, Ld, L.cs_off.p, L.Di64.p, L.Doff.p, L.tri_cb, x, L.n, nrhs, s);
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
    KTime kt(KC_TRANSFER, s, 0.0, L.transfer_bytes[std::is_same<T, double>::value ? 1 : 0] * nrhs);
    const dim3 gr((unsigned)std::max<int64_t>(1, cdiv(L.max_k, 128)),
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>(L.nagg, 65535)));
    k_restrict<T><<<gr, 256, 0, s>>>(L.wptr.p, L.widx.p, L.k.p, L.off.p, Z, L.zoff.p, L.nagg, r, L.n, bvec<T>(C),
                                     C.n, nrhs);
    CK_LAUNCH();
    }
    vcycle<T>(H, l + 1, nrhs, s);
    {
    KTime kt(KC_TRANSFER, s, 0.0, L.transfer_bytes[std::is_same<T, double>::value ? 1 : 0] * nrhs);
    const size_t ism = (size_t)std::max(1, L.max_k) * sizeof(T);
    if (ism > 48 * 1024) {
        if (ism > 227 * 1024) fail(LSAMG_LIMIT, "coarse block too large for the interpolation kernel");
        CK(cudaFuncSetAttribute(k_interp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism));
    }
    const dim3 gi((unsigned)std::max<int64_t>(1, cdiv(L.max_nw, TR_ROWS)),
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>(L.nagg, 65535)));
    k_interp<T><<<gi, 256, ism, s>>>(L.wptr.p, L.widx.p, L.k.p, L.off.p, Z, L.zoff.p, L.nagg, xvec<T>(C), C.n, x,
                                     L.n, nrhs);
    CK_LAUNCH();
    }
    // residual after the coarse correction: r = b - A x
    CK(cudaMemcpyAsync(r, b, tot * sizeof(T), cudaMemcpyDeviceToDevice, s));
    {
        LSAMG_PROF(l == 0 ? "vc: L0 residual spmv" : "vc: Lc residual spmv", s);
        KTime kt(KC_SPMV, s, spmv_flops<T>(L, nrhs), L.spmv_bytes[std::is_same<T, double>::value ? 1 : 0]);
        const T *G;
        if constexpr (std::is_same<T, float>::value) G = L.G32.p; else G = L.G64.p;
        launch_spmv<T>(L, G, x, r, nrhs, (T)-1, s);
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
