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
template <class T>
__global__ void k_restrict(const int64_t *wptr, const int32_t *widx, const int32_t *k,
                           const int64_t *off, const T *Z, const int64_t *zoff, int64_t nagg,
                           const T *res, int64_t n, T *rc, int64_t nc, int nrhs) {
    for (int64_t a = blockIdx.x; a < nagg; a += gridDim.x) {
        const int ka = k[a];
        const int64_t wb = wptr[a];
        const int nw = (int)(wptr[a + 1] - wb);
        const T *z = Z + zoff[a];
        for (int r = 0; r < nrhs; r++)
            for (int j = threadIdx.x; j < ka; j += blockDim.x) {
                T s = 0;
                for (int p = 0; p < nw; p++) s += z[(int64_t)p * ka + j] * res[(int64_t)r * n + widx[wb + p]];
                rc[(int64_t)r * nc + off[a] + j] = s;
            }
    }
}

template <class T>
__global__ void k_interp(const int64_t *wptr, const int32_t *widx, const int32_t *k,
                         const int64_t *off, const T *Z, const int64_t *zoff, int64_t nagg,
                         const T *ec, int64_t nc, T *x, int64_t n, int nrhs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int64_t a = blockIdx.x; a < nagg; a += gridDim.x) {
        const int ka = k[a];
        const int64_t wb = wptr[a];
        const int nw = (int)(wptr[a + 1] - wb);
        const T *z = Z + zoff[a];
        for (int r = 0; r < nrhs; r++)
            for (int p = warp; p < nw; p += nwarp) {
                T s = 0;
                for (int j = lane; j < ka; j += 32) s += z[(int64_t)p * ka + j] * ec[(int64_t)r * nc + off[a] + j];
                s = warp_sum(s);
                if (lane == 0) x[(int64_t)r * n + widx[wb + p]] += s;
            }
    }
}

// ---------------------------------------------------------------- blocked coarsest solve
constexpr int CB = 256;            // rows per block of the multi-CTA triangular solves

// forward solve of the diagonal block rows [r0, r1) of L y = v (columns < r0 already applied)
template <class T>
__global__ void __launch_bounds__(256) k_cs_fwd_diag(const T *L, int r0, int r1, T *v, int64_t stride) {
    __shared__ T red[32];
    T *vr = v + (int64_t)blockIdx.x * stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int b0 = r0; b0 < r1; b0 += 32) {
        const int rs = min(32, r1 - b0);
        for (int i = warp; i < rs; i += nwarp) {
            const T *row = L + (int64_t)(b0 + i) * (b0 + i + 1) / 2;
            T sacc = 0;
            for (int j = r0 + lane; j < b0; j += 32) sacc += row[j] * vr[j];
            sacc = warp_sum(sacc);
            if (lane == 0) red[i] = vr[b0 + i] - sacc;
        }
        __syncthreads();
        if (warp == 0) {
            T yl = 0;
            for (int i = 0; i < rs; i++) {
                const T *row = L + (int64_t)(b0 + i) * (b0 + i + 1) / 2 + b0;
                T c = (lane < i) ? row[lane] * yl : (T)0;
                c = warp_sum(c);
                T yi = (red[i] - c) / row[i];
                if (lane == i) yl = yi;
            }
            if (lane < rs) vr[b0 + lane] = yl;
        }
        __syncthreads();
    }
}

// v[r] -= sum_{j in [r0, r1)} L[r, j] y[j] for rows r >= r1 (warp per row)
template <class T>
__global__ void __launch_bounds__(256) k_cs_fwd_update(const T *L, int r0, int r1, int n, T *v,
                                                       int64_t stride) {
    T *vr = v + (int64_t)blockIdx.y * stride;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = r1 + wid; r < n; r += nw) {
        const T *row = L + r * (r + 1) / 2;
        T sacc = 0;
        for (int j = r0 + lane; j < r1; j += 32) sacc += row[j] * vr[j];
        sacc = warp_sum(sacc);
        if (lane == 0) vr[r] -= sacc;
    }
}

// backward solve of the diagonal block [r0, r1) of L^T x = y (rows >= r1 already applied)
template <class T>
__global__ void __launch_bounds__(256) k_cs_bwd_diag(const T *L, int r0, int r1, T *v, int64_t stride) {
    T *vr = v + (int64_t)blockIdx.x * stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = (r1 - r0 + 31) / 32;
    for (int bi = nb - 1; bi >= 0; bi--) {
        const int b0 = r0 + bi * 32, rs = min(32, r1 - b0);
        if (warp == 0) {
            T xl = (lane < rs) ? vr[b0 + lane] : (T)0;
            for (int i = rs - 1; i >= 0; i--) {
                const T *row = L + (int64_t)(b0 + i) * (b0 + i + 1) / 2 + b0;
                T xi = __shfl_sync(0xffffffffu, xl, i) / row[i];
                if (lane == i) xl = xi;
                if (lane < i) xl -= row[lane] * xi;
            }
            if (lane < rs) vr[b0 + lane] = xl;
        }
        __syncthreads();
        for (int j = r0 + threadIdx.x; j < b0; j += blockDim.x) {
            T sacc = 0;
            for (int i = 0; i < rs; i++) sacc += L[(int64_t)(b0 + i) * (b0 + i + 1) / 2 + j] * vr[b0 + i];
            vr[j] -= sacc;
        }
        __syncthreads();
    }
}

// v[j] -= sum_{i in [r0, r1)} L[i, j] x[i] for columns j < r0 (thread per column)
template <class T>
__global__ void __launch_bounds__(256) k_cs_bwd_update(const T *L, int r0, int r1, T *v, int64_t stride) {
    T *vr = v + (int64_t)blockIdx.y * stride;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < r0;
         j += (int64_t)gridDim.x * blockDim.x) {
        T sacc = 0;
        for (int i = r0; i < r1; i++) sacc += L[(int64_t)i * (i + 1) / 2 + j] * vr[i];
        vr[j] -= sacc;
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

template <class T>
__global__ void __launch_bounds__(256) k_sw_fwd_diag(const int32_t *aggs, const int64_t *Optr, const T *Lp,
                                                     const int64_t *Loff, int r0, T *ws, int64_t wsn, int nrhs) {
    __shared__ T red[32];
    const int32_t a = aggs[blockIdx.x];
    const int n = (int)(Optr[a + 1] - Optr[a]);
    if (r0 >= n) return;
    const int r1 = min(n, r0 + CB);
    const T *L = Lp + Loff[a];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = 0; r < nrhs; r++) {
        T *vr = ws + (int64_t)r * wsn + Optr[a];
        for (int b0 = r0; b0 < r1; b0 += 32) {
            const int rs = min(32, r1 - b0);
            for (int i = warp; i < rs; i += nwarp) {
                const T *row = L + (int64_t)(b0 + i) * (b0 + i + 1) / 2;
                T sacc = 0;
                for (int j = r0 + lane; j < b0; j += 32) sacc += row[j] * vr[j];
                sacc = warp_sum(sacc);
                if (lane == 0) red[i] = vr[b0 + i] - sacc;
            }
            __syncthreads();
            if (warp == 0) {
                T yl = 0;
                for (int i = 0; i < rs; i++) {
                    const T *row = L + (int64_t)(b0 + i) * (b0 + i + 1) / 2 + b0;
                    T c = (lane < i) ? row[lane] * yl : (T)0;
                    c = warp_sum(c);
                    T yi = (red[i] - c) / row[i];
                    if (lane == i) yl = yi;
                }
                if (lane < rs) vr[b0 + lane] = yl;
            }
            __syncthreads();
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_sw_fwd_update(const int32_t *aggs, const int64_t *Optr, const T *Lp,
                                                       const int64_t *Loff, int r0, T *ws, int64_t wsn, int nrhs) {
    const int32_t a = aggs[blockIdx.y];
    const int n = (int)(Optr[a + 1] - Optr[a]);
    const int r1 = min(n, r0 + CB);
    if (r1 >= n) return;
    const T *L = Lp + Loff[a];
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int r = 0; r < nrhs; r++) {
        T *vr = ws + (int64_t)r * wsn + Optr[a];
        for (int64_t i = r1 + wid; i < n; i += nw) {
            const T *row = L + i * (i + 1) / 2;
            T sacc = 0;
            for (int j = r0 + lane; j < r1; j += 32) sacc += row[j] * vr[j];
            sacc = warp_sum(sacc);
            if (lane == 0) vr[i] -= sacc;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_sw_bwd_diag(const int32_t *aggs, const int64_t *Optr, const T *Lp,
                                                     const int64_t *Loff, int r1g, T *ws, int64_t wsn, int nrhs) {
    const int32_t a = aggs[blockIdx.x];
    const int n = (int)(Optr[a + 1] - Optr[a]);
    // aligned block [r1g - CB, r1g) clipped to this subdomain
    const int r0 = max(0, r1g - CB);
    if (r0 >= n) return;
    const int r1 = min(r1g, n);
    const T *L = Lp + Loff[a];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < nrhs; r++) {
        T *vr = ws + (int64_t)r * wsn + Optr[a];
        const int nb = (r1 - r0 + 31) / 32;
        for (int bi = nb - 1; bi >= 0; bi--) {
            const int b0 = r0 + bi * 32, rs = min(32, r1 - b0);
            if (warp == 0) {
                T xl = (lane < rs) ? vr[b0 + lane] : (T)0;
                for (int i = rs - 1; i >= 0; i--) {
                    const T *row = L + (int64_t)(b0 + i) * (b0 + i + 1) / 2 + b0;
                    T xi = __shfl_sync(0xffffffffu, xl, i) / row[i];
                    if (lane == i) xl = xi;
                    if (lane < i) xl -= row[lane] * xi;
                }
                if (lane < rs) vr[b0 + lane] = xl;
            }
            __syncthreads();
            for (int j = r0 + threadIdx.x; j < b0; j += blockDim.x) {
                T sacc = 0;
                for (int i = 0; i < rs; i++) sacc += L[(int64_t)(b0 + i) * (b0 + i + 1) / 2 + j] * vr[b0 + i];
                vr[j] -= sacc;
            }
            __syncthreads();
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_sw_bwd_update(const int32_t *aggs, const int64_t *Optr, const T *Lp,
                                                       const int64_t *Loff, int r1g, T *ws, int64_t wsn, int nrhs) {
    const int32_t a = aggs[blockIdx.y];
    const int n = (int)(Optr[a + 1] - Optr[a]);
    const int r0 = max(0, r1g - CB);
    if (r0 >= n) return;
    const int r1 = min(r1g, n);
    const T *L = Lp + Loff[a];
    for (int r = 0; r < nrhs; r++) {
        T *vr = ws + (int64_t)r * wsn + Optr[a];
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < r0; j += (int64_t)gridDim.x * blockDim.x) {
            T sacc = 0;
            for (int i = r0; i < r1; i++) sacc += L[(int64_t)i * (i + 1) / 2 + j] * vr[i];
            vr[j] -= sacc;
        }
    }
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
__global__ void __launch_bounds__(1024) k_coarse_solve(const T *L, int n, T *v, int64_t stride,
                                                       int nrhs) {
    __shared__ T red[32];
    for (int r = blockIdx.x; r < nrhs; r += gridDim.x) chol_solve_packed<T>(L, n, v + r * stride, red);
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
    for (int r0 = 0; r0 < maxn; r0 += CB) {
        k_sw_fwd_diag<T><<<(unsigned)na, 256, 0, s>>>(aggs, L.Optr.p, Lp, L.Loff.p, r0, ws, L.Omega_total, nrhs);
        CK_LAUNCH();
        if (r0 + CB < maxn) {
            dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv((int64_t)(maxn - r0 - CB) * 32, 256), 256)), (unsigned)na);
            k_sw_fwd_update<T><<<g, 256, 0, s>>>(aggs, L.Optr.p, Lp, L.Loff.p, r0, ws, L.Omega_total, nrhs);
            CK_LAUNCH();
        }
    }
    // backward: every subdomain walks its own blocks from its end; blocks are aligned to the
    // forward partition (multiples of CB from the start), so r1 runs over CB-multiples and the
    // subdomain's own n
    std::vector<int> ends;
    for (int r1 = ((maxn + CB - 1) / CB) * CB; r1 > 0; r1 -= CB) ends.push_back(r1);
    for (int r1 : ends) {
        // subdomains whose size is not a multiple of CB treat their last partial block when
        // r1 is the first CB-multiple >= n: pass r1 and let each use min(r1, n)
        k_sw_bwd_diag<T><<<(unsigned)na, 256, 0, s>>>(aggs, L.Optr.p, Lp, L.Loff.p, r1, ws, L.Omega_total, nrhs);
        CK_LAUNCH();
        dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(std::max(r1 - CB, 1), 256), 256)), (unsigned)na);
        k_sw_bwd_update<T><<<g, 256, 0, s>>>(aggs, L.Optr.p, Lp, L.Loff.p, r1, ws, L.Omega_total, nrhs);
        CK_LAUNCH();
    }
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
        const int n = (int)L.n;
        KTime kt(KC_COARSE_SOLVE, s, 0.0, L.coarse_bytes[std::is_same<T, double>::value ? 1 : 0] * nrhs);
        if (n <= 2 * CB) {
            k_coarse_solve<T><<<(unsigned)nrhs, 1024, 0, s>>>(Ld, n, x, L.n, nrhs);
            CK_LAUNCH();
            return;
        }
        for (int r0 = 0; r0 < n; r0 += CB) {
            const int r1 = std::min(n, r0 + CB);
            k_cs_fwd_diag<T><<<(unsigned)nrhs, 256, 0, s>>>(Ld, r0, r1, x, L.n);
            CK_LAUNCH();
            if (r1 < n) {
                dim3 g((unsigned)std::min<int64_t>(cdiv((int64_t)(n - r1) * 32, 256), 148 * 8), (unsigned)nrhs);
                k_cs_fwd_update<T><<<g, 256, 0, s>>>(Ld, r0, r1, n, x, L.n);
                CK_LAUNCH();
            }
        }
        for (int r1 = n; r1 > 0; r1 -= CB) {
            const int r0 = std::max(0, r1 - CB);
            k_cs_bwd_diag<T><<<(unsigned)nrhs, 256, 0, s>>>(Ld, r0, r1, x, L.n);
            CK_LAUNCH();
            if (r0 > 0) {
                dim3 g((unsigned)std::min<int64_t>(cdiv(r0, 256), 148 * 8), (unsigned)nrhs);
                k_cs_bwd_update<T><<<g, 256, 0, s>>>(Ld, r0, r1, x, L.n);
                CK_LAUNCH();
            }
        }
        return;
    }
    Level &C = H.levels[l + 1];
    CK(cudaMemsetAsync(x, 0, tot * sizeof(T), s));
    CK(cudaMemcpyAsync(r, b, tot * sizeof(T), cudaMemcpyDeviceToDevice, s));
    {
        LSAMG_PROF(l == 0 ? "vc: L0 pre-smooth" : "vc: Lc pre-smooth", s);
        for (int c = 0; c < L.ncol; c++) sweep<T>(L, c, nrhs, s);
    }
    const T *Z;
    if constexpr (std::is_same<T, float>::value) Z = L.Z32.p; else Z = L.Z64.p;
    {
    KTime kt(KC_TRANSFER, s);
    k_restrict<T><<<gridv(L.nagg, 1, 148 * 16), 128, 0, s>>>(L.wptr.p, L.widx.p, L.k.p, L.off.p, Z,
                                                            L.zoff.p, L.nagg, r, L.n, bvec<T>(C),
                                                            C.n, nrhs);
    CK_LAUNCH();
    }
    vcycle<T>(H, l + 1, nrhs, s);
    {
    KTime kt(KC_TRANSFER, s);
    k_interp<T><<<gridv(L.nagg, 1, 148 * 16), 256, 0, s>>>(L.wptr.p, L.widx.p, L.k.p, L.off.p, Z,
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
