// Numerical set-up of one level (FP64): element Gram factors (Section 5.2, Prop. 5.1),
// the local reduced eigenproblems that define P (Section 2 eqs. 2.6-2.10), the coarse
// Gram G_c = G P merged by coarse element map (Section 2 end, Remark 5.2), the Schwarz
// factors of the overlaps and the dense coarsest factor.
#include <algorithm>

#include "impl.cuh"
#include "dense.cuh"

namespace lsamg {

namespace {

constexpr double DEPS = 2.220446049250313e-16;

inline unsigned gridc(int64_t items, int per = 256, int64_t cap = 148 * 32) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(items, per), cap));
}

__device__ __forceinline__ int64_t lbound(const int32_t *a, int64_t n, int32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- element factor
// Pivoted Cholesky A_T = P L L^T P^T with rank truncation (Section 5.2); G_T = L^T P^T.
constexpr int FACT_MAX = 96;

__global__ void k_elem_factor(const double *AT, const int64_t *aoff, const int32_t *nT_of,
                              int64_t ne, double *G, const int64_t *goff, int32_t *grows, int *err) {
    extern __shared__ double a[];
    __shared__ int perm[FACT_MAX];
    __shared__ int piv_i;
    __shared__ double maxd;
    __shared__ int rank;
    for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
        int n = nT_of[e];
        const double *A = AT + aoff[e];
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = A[t];
        for (int t = threadIdx.x; t < n; t += blockDim.x) perm[t] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int i = 0; i < n; i++) m = fmax(m, a[i * n + i]);
            maxd = m;
            rank = n;
        }
        __syncthreads();
        const double tol = (double)n * DEPS * maxd;
        for (int j = 0; j < n; j++) {
            if (threadIdx.x == 0) {
                int p = j;
                double best = a[j * n + j];
                for (int i = j + 1; i < n; i++)
                    if (a[i * n + i] > best) {
                        best = a[i * n + i];
                        p = i;
                    }
                piv_i = (best > tol) ? p : -1;
                if (piv_i < 0) rank = j;
            }
            __syncthreads();
            int p = piv_i;
            if (p < 0) break;
            if (p != j) {
                for (int t = threadIdx.x; t < n; t += blockDim.x) {  // swap rows
                    double u = a[j * n + t];
                    a[j * n + t] = a[p * n + t];
                    a[p * n + t] = u;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += blockDim.x) {  // swap columns
                    double u = a[t * n + j];
                    a[t * n + j] = a[t * n + p];
                    a[t * n + p] = u;
                }
                if (threadIdx.x == 0) {
                    int u = perm[j];
                    perm[j] = perm[p];
                    perm[p] = u;
                }
                __syncthreads();
            }
            double ljj = sqrt(a[j * n + j]);
            __syncthreads();
            if (threadIdx.x == 0) a[j * n + j] = ljj;
            for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) a[i * n + j] /= ljj;
            __syncthreads();
            int m = n - j - 1;
            for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
                int i = j + 1 + t / m, k = j + 1 + t % m;
                if (k <= i) {
                    a[i * n + k] -= a[i * n + j] * a[k * n + j];
                    if (k < i) a[k * n + i] = a[i * n + k];
                }
            }
            __syncthreads();
        }
        int r = rank;
        // the truncated Schur complement must be negligible for an SPSD block
        for (int t = threadIdx.x; t < (n - r) * (n - r); t += blockDim.x) {
            int i = r + t / (n - r), k = r + t % (n - r);
            double v = a[i * n + k];
            if ((i == k && v < -1e-12 * maxd) || fabs(v) > 1e-9 * maxd)
                flag_error(err, LSAMG_NOT_SPSD, (int)e);
        }
        double *g = G + goff[e];
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            int row = t / n, c = t % n;  // G[row, perm[c]] = L[c, row] for c >= row
            if (row < r) g[row * n + perm[c]] = (c >= row) ? a[c * n + row] : 0.0;
            else g[row * n + c] = 0.0;
        }
        if (threadIdx.x == 0) grows[e] = r;
        __syncthreads();
    }
}


// CTAs per aggregate for the dense assemblies: one while the batch fills the GPU, more when it
// has few aggregates.  Each CTA of an aggregate owns the destination columns c with
// c % slices == slice, so every entry is summed by one CTA, in element order: the assembled
// blocks are the same bits on every run.
static int assembly_slices(int64_t na) {
    const int64_t want = (148 * 4 + na - 1) / std::max<int64_t>(na, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, 16));
}

// ---------------------------------------------------------------- local problem assembly
// At (omega-first, column-major |Omega| x |Omega|) += A_T / mult(T) and Aww += A_T on
// omega x omega, over the elements touching omega_i (eqs. 2.6-2.9).  A_T is symmetric, so
// entry (r, c) of the element is read as A_T[c][r] (consecutive threads, consecutive r).
__global__ void k_assemble_gep(const int32_t *alist, int64_t na, const int64_t *aeptr, const int32_t *aeidx,
                               const int64_t *eptr, const int32_t *eidx, const double *AT,
                               const int64_t *aoff, const int32_t *mult, const int64_t *Optr,
                               const int32_t *Oidx, const int32_t *Olpos, const int64_t *wptr,
                               double *At, const int64_t *atoff, double *Aww,
                               const int64_t *awoff, int es) {
    extern __shared__ int32_t pos[];   // [maxE] positions, then [maxE] owned element columns
    __shared__ int ncols;
    int64_t li = blockIdx.x;
    if (li >= na) return;
    int64_t a = alist[li];
    const int32_t *Om = Oidx + Optr[a];
    const int32_t *lp = Olpos + Optr[a];
    int64_t nO = Optr[a + 1] - Optr[a];
    int nw = (int)(wptr[a + 1] - wptr[a]);
    double *T1 = At + atoff[li];
    double *T2 = Aww + awoff[li];
    const int slice = blockIdx.y;
    for (int64_t j = aeptr[a]; j < aeptr[a + 1]; j++) {
        int32_t e = aeidx[j];
        int64_t b = eptr[e];
        int n = (int)(eptr[e + 1] - b);
        int32_t *own = pos + n;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            // -1: an element DOF outside Omega_i (only under the A-closure, whose local
            // matrices drop those rows and columns)
            const int32_t q = eidx[b + t];
            const int64_t k = lbound(Om, nO, q);
            pos[t] = (k < nO && Om[k] == q) ? lp[k] : -1;
        }
        __syncthreads();
        warp_compact(n, own, &ncols, [&](int c) { return pos[c] >= 0 && pos[c] % es == slice; });
        __syncthreads();
        const double *Ae = AT + aoff[e];
        const double w = 1.0 / (double)mult[e];
        const int nc = ncols;
        for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
            const int c = own[t / n], r = t % n;
            const double v = Ae[(int64_t)c * n + r];
            const int pr = pos[r], pc = pos[c];
            if (pr < 0) continue;
            T1[pr + (int64_t)pc * nO] += w * v;
            if (pr < nw && pc < nw) T2[pr + (int64_t)pc * nw] += v;
        }
        __syncthreads();
    }
}

// A_Omega (sorted-Omega order, column-major) += A_T over the elements meeting Omega_i; the CTAs
// of a subdomain own interleaved destination columns (deterministic, no atomics)
__global__ void k_assemble_smoother(int64_t a0, int64_t na, const int64_t *oeptr,
                                    const int32_t *oeidx, const int64_t *eptr, const double *AT,
                                    const int64_t *aoff, const int64_t *locoff, const int32_t *loc,
                                    const int64_t *Optr, double *AO, const int64_t *ooff, int es) {
    extern __shared__ int32_t own[];
    __shared__ int ncols;
    int64_t li = blockIdx.x;
    if (li >= na) return;
    int64_t a = a0 + li;
    int64_t nO = Optr[a + 1] - Optr[a];
    double *M = AO + ooff[li];
    const int slice = blockIdx.y;
    for (int64_t j = oeptr[a]; j < oeptr[a + 1]; j++) {
        int32_t e = oeidx[j];
        int n = (int)(eptr[e + 1] - eptr[e]);
        const int32_t *p = loc + locoff[j];
        warp_compact(n, own, &ncols, [&](int c) { return p[c] >= 0 && p[c] % es == slice; });
        __syncthreads();
        const double *Ae = AT + aoff[e];
        const int nc = ncols;
        for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
            const int c = own[t / n], r = t % n;
            const int pr = p[r];
            if (pr >= 0) M[pr + (int64_t)p[c] * nO] += Ae[(int64_t)c * n + r];
        }
        __syncthreads();
    }
}

// packed lower row-major copy of a column-major Cholesky factor (FP64 and FP32)
__global__ void k_pack_lower(const double *Lc, const int64_t *loff, const int32_t *nn, int64_t na,
                             double *P64, float *P32, const int64_t *poff) {
    int64_t li = blockIdx.y;
    if (li >= na) return;
    int n = nn[li];
    const double *L = Lc + loff[li];
    int64_t tot = (int64_t)n * (n + 1) / 2;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((int64_t)(r + 1) * (r + 2) / 2 <= t) r++;
        while ((int64_t)r * (r + 1) / 2 > t) r--;
        int c = (int)(t - (int64_t)r * (r + 1) / 2);
        double v = L[r + (int64_t)c * n];
        P64[poff[li] + t] = v;
        P32[poff[li] + t] = (float)v;
    }
}

// sign fix (largest |entry| positive, first on ties) and row-major store of Z_i
__global__ void k_store_z(const double *V, const int64_t *voff, const int32_t *nw_of,
                          const int32_t *k_of, int64_t na, double *Z64, float *Z32,
                          const int64_t *zoff) {
    int64_t li = blockIdx.x;
    if (li >= na) return;
    int nw = nw_of[li], k = k_of[li];
    const double *v = V + voff[li];
    int lane = threadIdx.x & 31;
    for (int c = threadIdx.x >> 5; c < k; c += blockDim.x >> 5) {
        const double *col = v + (int64_t)c * nw;
        double best = -1.0;
        int bi = 0;
        for (int i = lane; i < nw; i += 32) {
            double m = fabs(col[i]);
            if (m > best) {
                best = m;
                bi = i;
            }
        }
        for (int o = 16; o; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        double sg = (col[bi] < 0.0) ? -1.0 : 1.0;
        for (int i = lane; i < nw; i += 32) {
            double z = sg * col[i];
            Z64[zoff[li] + (int64_t)i * k + c] = z;
            Z32[zoff[li] + (int64_t)i * k + c] = (float)z;
        }
    }
}

// ---------------------------------------------------------------- coarse elements
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

__global__ void k_coarse_len(const int64_t *eaptr, const int32_t *eaidx, int64_t ne,
                             const int32_t *k, int64_t *len, uint64_t *keys) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        uint64_t h = 0x9e3779b97f4a7c15ull;
        for (int64_t j = eaptr[e]; j < eaptr[e + 1]; j++) {
            s += k[eaidx[j]];
            h = mix64(h ^ (uint64_t)(uint32_t)eaidx[j]) + 0x9e3779b97f4a7c15ull;
        }
        len[e] = s;
        // sort key: (hash of the element's aggregate set [40 bits], element id [24+ bits])
        keys[e] = (s > 0) ? (h & 0xffffffffff000000ull) : ~0ull;
    }
}

__global__ void k_make_keys(const uint64_t *h, int64_t ne, uint64_t *keys) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x)
        keys[e] = (h[e] == ~0ull) ? ~0ull : (h[e] | (uint64_t)e);
}

__global__ void k_extract_order(const uint64_t *keys, int64_t ne, int32_t *order) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ne;
         s += (int64_t)gridDim.x * blockDim.x)
        order[s] = (keys[s] == ~0ull) ? -1 : (int32_t)(keys[s] & 0xffffffull);
}

__global__ void k_same_set(const int32_t *order, int64_t ne, const int64_t *eaptr,
                           const int32_t *eaidx, const uint64_t *h, int32_t *leader_flag,
                           int32_t *run_start, int *err) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ne;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = order[s];
        if (e < 0) {
            run_start[s] = -1;
            continue;
        }
        bool same = false;
        if (s > 0) {
            int32_t f = order[s - 1];
            if (h[f] == h[e]) {
                int64_t b1 = eaptr[e], l1 = eaptr[e + 1] - b1, b2 = eaptr[f], l2 = eaptr[f + 1] - b2;
                if (l1 != l2) {
                    flag_error(err, LSAMG_LIMIT, (int)e);  // 64-bit hash collision
                } else {
                    same = true;
                    for (int64_t t = 0; t < l1; t++)
                        if (eaidx[b1 + t] != eaidx[b2 + t]) same = false;
                    if (!same) flag_error(err, LSAMG_LIMIT, (int)e);
                }
            }
        }
        leader_flag[e] = same ? 0 : 1;
        run_start[s] = same ? -2 : (int32_t)s;
    }
}

__global__ void k_assign_group(const int32_t *order, int64_t ne, const int32_t *run_start,
                               const int64_t *gid_of_leader, int32_t *cgroup) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ne;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (run_start[s] == -1) continue;
        int32_t e = order[s];
        int64_t t = s;
        while (run_start[t] == -2) t--;
        cgroup[e] = (int32_t)gid_of_leader[order[t]];
    }
}

__global__ void k_leader_of_group(const int32_t *leader_flag, const int64_t *gid, int64_t ne,
                                  int32_t *leader) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x)
        if (leader_flag[e]) leader[gid[e]] = (int32_t)e;
}

__global__ void k_group_sizes(const int32_t *leader, int64_t ng, const int64_t *clen,
                              const int64_t *mptr, const int32_t *midx, const int32_t *grows,
                              int64_t *gcols, int64_t *grow_tot) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        gcols[g] = clen[leader[g]];
        int64_t r = 0;
        for (int64_t j = mptr[g]; j < mptr[g + 1]; j++) r += grows[midx[j]];
        grow_tot[g] = r;
    }
}

__global__ void k_fill_cmap(const int32_t *leader, int64_t ng, const int64_t *eaptr,
                            const int32_t *eaidx, const int32_t *k, const int64_t *off,
                            const int64_t *cptr, int32_t *cidx) {
    int64_t g = blockIdx.x;
    if (g >= ng) return;
    int32_t e = leader[g];
    if (threadIdx.x == 0) {
        int64_t o = cptr[g];
        for (int64_t j = eaptr[e]; j < eaptr[e + 1]; j++) {
            int32_t a = eaidx[j];
            for (int32_t t = 0; t < k[a]; t++) cidx[o++] = (int32_t)(off[a] + t);
        }
    }
}

// G_c rows of one element: G_c,T = G_T (R_T P), tile of 32 rows x 64 coarse columns.
// work item = (element, row tile, column tile); RTP entries built from Z blocks on the fly.
__global__ void __launch_bounds__(256) k_gc(const int32_t *items, int64_t nitems,
                                            const int64_t *eptr, const int32_t *eidx,
                                            const double *G, const int64_t *goff,
                                            const int32_t *grows, const int64_t *eaptr,
                                            const int32_t *eaidx, const int32_t *agg,
                                            const int32_t *posw, const int32_t *k,
                                            const double *Z, const int64_t *zoff,
                                            const int32_t *cgroup, const int64_t *cgoff,
                                            const int64_t *cgcols, const int64_t *rowbase,
                                            double *Gc) {
    int64_t it = blockIdx.x;
    if (it >= nitems) return;
    int32_t e = items[3 * it], tr = items[3 * it + 1], tc = items[3 * it + 2];
    int64_t b = eptr[e];
    int n = (int)(eptr[e + 1] - b);
    int m = grows[e];
    int g = cgroup[e];
    int ncol = (int)cgcols[g];
    // column c of the coarse map -> (aggregate, mode): blocks in eagg(e) order
    __shared__ int32_t blk_a[64];
    __shared__ int32_t blk_start[65];
    __shared__ int nblk;
    if (threadIdx.x == 0) {
        int nb = 0, c = 0;
        for (int64_t j = eaptr[e]; j < eaptr[e + 1] && nb < 63; j++) {
            blk_a[nb] = eaidx[j];
            blk_start[nb] = c;
            c += k[eaidx[j]];
            nb++;
        }
        blk_start[nb] = c;
        nblk = nb;
    }
    // operands as double-float pairs (the product is FP64 multiply-add bound otherwise)
    __shared__ float2 Gs[32][33];
    __shared__ float2 Rs[32][65];
    const int r0 = tr * 32, c0 = tc * 64;
    int ty = threadIdx.x / 32, tx = threadIdx.x % 32;  // 8 x 32 threads: rows ty*4.., cols tx*2..
    float ah[4][2] = {}, al[4][2] = {};
    __syncthreads();
    for (int q0 = 0; q0 < n; q0 += 32) {
        for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
            int r = t / 32, q = t % 32;
            Gs[r][q] = df_split((r0 + r < m && q0 + q < n) ? G[goff[e] + (int64_t)(r0 + r) * n + q0 + q] : 0.0);
        }
        for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
            int q = t / 64, c = t % 64;
            double v = 0.0;
            int gq = q0 + q, gc = c0 + c;
            if (gq < n && gc < ncol) {
                int32_t dof = eidx[b + gq];
                int32_t a = agg[dof];
                int bi = 0;
                while (bi + 1 < nblk && blk_start[bi + 1] <= gc) bi++;
                if (blk_a[bi] == a) {
                    int mode = gc - blk_start[bi];
                    v = Z[zoff[a] + (int64_t)posw[dof] * k[a] + mode];
                }
            }
            Rs[q][c] = df_split(v);
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 32; q++) {
            float2 r0v[4], c0v[2];
#pragma unroll
            for (int u = 0; u < 4; u++) r0v[u] = Gs[ty * 4 + u][q];
#pragma unroll
            for (int v = 0; v < 2; v++) c0v[v] = Rs[q][tx * 2 + v];
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 2; v++) df_mac(ah[u][v], al[u][v], r0v[u], c0v[v]);
        }
        __syncthreads();
    }
    double *out = Gc + cgoff[g] + rowbase[e] * (int64_t)ncol;
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {
            int r = r0 + ty * 4 + u, c = c0 + tx * 2 + v;
            if (r < m && c < ncol) out[(int64_t)r * ncol + c] = (double)ah[u][v] + (double)al[u][v];
        }
}

// compressed coarse factor: G'[r, perm[c]] = L[c, r] (c >= r, r < rank) from a pivoted
// Cholesky P A_g P^T = L L^T stored column-major in W
__global__ void k_extract_factor(const double *W, const int64_t *woff, const int64_t *nn,
                                 const int32_t *perm, const int64_t *permoff, const int32_t *rank,
                                 const int64_t *goff, int64_t ng, double *G64, float *G32) {
    int64_t g = blockIdx.y;
    if (g >= ng) return;
    const int64_t n = nn[g];
    const int r = rank[g];
    const double *L = W + woff[g];
    const int32_t *pv = perm + permoff[g];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)r * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = t / n, c = t % n;
        double v = (c >= row) ? L[c + row * n] : 0.0;
        G64[goff[g] + row * n + pv[c]] = v;
        G32[goff[g] + row * n + pv[c]] = (float)v;
    }
}

__global__ void k_rowbase(const int64_t *mptr, const int32_t *midx, int64_t ng,
                          const int32_t *grows, int64_t *rowbase) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = 0;
        for (int64_t j = mptr[g]; j < mptr[g + 1]; j++) {
            rowbase[midx[j]] = r;
            r += grows[midx[j]];
        }
    }
}

__global__ void k_to_f32(const double *a, float *b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void k_symmetrize_sq(double *A, const int64_t *off, const int64_t *nn, int64_t ng) {
    int64_t g = blockIdx.y;
    if (g >= ng) return;
    int64_t n = nn[g];
    double *M = A + off[g];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / n, j = t % n;
        if (i < j) {
            double v = 0.5 * (M[i * n + j] + M[j * n + i]);
            M[i * n + j] = v;
            M[j * n + i] = v;
        }
    }
}

// dense coarsest matrix: D = sum_T R_T^T A_T R_T (column-major n x n).  A CTA owns column j and
// adds, in the ascending element order of the DOF -> element map, column loc(j, T) of every
// A_T containing j: each entry has one writer and a fixed summation order (no atomics).
__global__ void k_assemble_dense(const int64_t *eptr, const int32_t *eidx, const int64_t *dptr,
                                 const int32_t *didx, const double *AT, const int64_t *aoff, double *D,
                                 int64_t n) {
    __shared__ int cloc;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        double *col = D + j * n;
        for (int64_t q = dptr[j]; q < dptr[j + 1]; q++) {
            const int32_t e = didx[q];
            const int64_t b = eptr[e];
            const int m = (int)(eptr[e + 1] - b);
            for (int t = threadIdx.x; t < m; t += blockDim.x)
                if (eidx[b + t] == (int32_t)j) cloc = t;   // DOFs of an element are distinct
            __syncthreads();
            const double *A = AT + aoff[e] + (int64_t)cloc * m;
            for (int t = threadIdx.x; t < m; t += blockDim.x) col[eidx[b + t]] += A[t];
            __syncthreads();
        }
    }
}

}  // namespace

// =============================================================================== host
void factor_elements(Level &L, int *err, cudaStream_t s) {
    auto hptr = to_host(L.eptr.p, L.ne + 1, s);
    std::vector<int32_t> nT(L.ne);
    int32_t mx = 0;
    for (int64_t e = 0; e < L.ne; e++) {
        nT[e] = (int32_t)(hptr[e + 1] - hptr[e]);
        mx = std::max(mx, nT[e]);
    }
    if (mx > FACT_MAX) fail(LSAMG_LIMIT, "element size above the element-factor limit (96)");
    DBuf<int32_t> dnT;
    upload(dnT, nT, s);
    L.goff.alloc(L.ne + 1, s);
    CK(cudaMemcpyAsync(L.goff.p, L.aoff.p, (L.ne + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    int64_t tot = read1(L.aoff.p + L.ne, s);
    L.G64.alloc(std::max<int64_t>(tot, 1), s);
    L.grows.alloc(std::max<int64_t>(L.ne, 1), s);
    size_t sm = (size_t)mx * mx * sizeof(double);
    KTime kt(KC_ELEM_FACTOR, s, (double)L.ne * mx * mx * mx / 3.0);
    CK(cudaFuncSetAttribute(k_elem_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_elem_factor<<<gridc(L.ne, 1, 148 * 16), 128, sm, s>>>(L.AT.p, L.aoff.p, dnT.p, L.ne, L.G64.p,
                                                          L.goff.p, L.grows.p, err);
    CK_LAUNCH();
    L.G32.alloc(std::max<int64_t>(tot, 1), s);
    k_to_f32<<<gridc(tot), 256, 0, s>>>(L.G64.p, L.G32.p, tot);
    CK_LAUNCH();
    check_err(err, s, "element factorisation");
}

static const char *lvl_name(int level, const char *stage) {
    static std::vector<std::string> store;
    static std::vector<std::pair<std::pair<int, std::string>, size_t>> index;
    for (auto &q : index)
        if (q.first.first == level && q.first.second == stage) return store[q.second].c_str();
    store.reserve(256);
    store.push_back("L" + std::to_string(level) + " " + stage);
    index.push_back({{level, stage}, store.size() - 1});
    return store.back().c_str();
}

int g_prof_level = 0;

void local_spectral(Level &L, const lsamg_options &o, int *err, cudaStream_t s, double *flops) {
    const int64_t nagg = L.nagg;
    // keep mu * tau_cut < 1 - 1e-9 (lambda > tau_cut and the ker S modes); the relative margin
    // discards exact ties mu = 1/tau_cut deterministically
    const double sigma = (1.0 - 1e-9) / L.tau;
    int64_t budget = o.chunk_bytes > 0 ? o.chunk_bytes : (int64_t)48 << 30;
    L.h_k.assign(nagg, 0);
    L.h_gap.assign(nagg, 0.0);
    struct Chunk {
        std::vector<int32_t> ids;
        int64_t na;
        DBuf<double> V;
        std::vector<int64_t> voff;
    };
    std::vector<Chunk> chunks;
    int32_t maxE = 0;
    {
        auto ep = to_host(L.eptr.p, L.ne + 1, s);
        for (int64_t e = 0; e < L.ne; e++) maxE = std::max<int32_t>(maxE, (int32_t)(ep[e + 1] - ep[e]));
    }
    // batches: aggregates of order <= 2048 (one CTA per matrix in the tridiagonalisation) and
    // larger ones (many CTAs per matrix) are processed in separate chunks.  Within each class the
    // aggregates go largest first: chunks then hold problems of similar order, and inside a launch
    // the longest ones start first, so no launch waits on one large matrix while SMs idle (local
    // problem orders vary several-fold and their cost as the cube).  Results are placed by
    // aggregate id, so the order changes no value.
    std::vector<int32_t> order;
    for (int pass = 0; pass < 2; pass++) {
        const size_t first = order.size();
        for (int64_t a = 0; a < nagg; a++)
            if ((L.h_nw[a] > g_large_dense) == (pass == 1)) order.push_back((int32_t)a);
        std::stable_sort(order.begin() + first, order.end(),
                         [&](int32_t x, int32_t y) { return L.h_nw[x] > L.h_nw[y]; });
    }
    size_t q0 = 0;
    while (q0 < order.size()) {
        // pick a chunk that fits the budget (at least one aggregate), same size class
        int64_t bytes = 0;
        size_t q1 = q0;
        const bool large = L.h_nw[order[q0]] > g_large_dense;
        while (q1 < order.size() && (L.h_nw[order[q1]] > g_large_dense) == large) {
            const int64_t nw = L.h_nw[order[q1]], nO = L.h_nO[order[q1]];
            const int64_t b = (nO * nO + 3 * nw * nw + 300 * nw) * 8;
            if (q1 > q0 && bytes + b > budget) break;
            bytes += b;
            q1++;
        }
        std::vector<int32_t> ids(order.begin() + q0, order.begin() + q1);
        const int64_t na = (int64_t)ids.size();
        DBuf<int32_t> dids;
        upload(dids, ids, s);
        std::vector<int64_t> atoff(na + 1), awoff(na + 1), coff(na + 1), toff(na + 1);
        std::vector<int32_t> nwv(na), nGv(na), nOv(na);
        atoff[0] = awoff[0] = coff[0] = toff[0] = 0;
        for (int64_t i = 0; i < na; i++) {
            int64_t nw = L.h_nw[ids[i]], nO = L.h_nO[ids[i]];
            nwv[i] = (int32_t)nw;
            nOv[i] = (int32_t)nO;
            nGv[i] = (int32_t)(nO - nw);
            atoff[i + 1] = atoff[i] + nO * nO;
            awoff[i + 1] = awoff[i] + nw * nw;
            coff[i + 1] = coff[i] + nw * nw;
            toff[i + 1] = toff[i] + nw;
            double fw = (double)nw, fg = (double)(nO - nw);
            *flops += fg * fg * fg / 3 + fg * fg * fw + 2 * fw * fw * fg + fw * fw * fw / 3 +
                      2 * fw * fw * fw + 4.0 / 3.0 * fw * fw * fw;
        }
        DBuf<double> At, Aww, C, dv, ev, tv, wv, gp;
        DBuf<int64_t> datoff, dawoff, dtoff;
        DBuf<int32_t> dk;
        At.alloc(std::max<int64_t>(atoff[na], 1), s);
        Aww.alloc(std::max<int64_t>(awoff[na], 1), s);
        C.alloc(std::max<int64_t>(coff[na], 1), s);
        At.zero(s);
        Aww.zero(s);
        upload(datoff, atoff, s);
        upload(dawoff, awoff, s);
        upload(dtoff, toff, s);
        int64_t tn = std::max<int64_t>(toff[na], 1);
        dv.alloc(tn, s);
        ev.alloc(tn, s);
        tv.alloc(tn, s);
        wv.alloc(tn, s);
        gp.alloc(na, s);
        dk.alloc(na, s);
        // 1. assemble At (omega-first) and A_ww
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: assemble"), s);
        KTime kt(KC_ASSEMBLE, s);
        const int es = assembly_slices(na);
        const size_t asm_smem = 2 * (size_t)maxE * sizeof(int32_t);
        if (asm_smem > 200 * 1024) fail(LSAMG_LIMIT, "element map longer than the assembly staging (25,600)");
        CK(cudaFuncSetAttribute(k_assemble_gep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_smem));
        k_assemble_gep<<<dim3((unsigned)na, (unsigned)es), 256, asm_smem, s>>>(
            dids.p, na, L.aeptr.p, L.aeidx.p, L.eptr.p, L.eidx.p, L.AT.p, L.aoff.p, L.mult.p, L.Optr.p,
            L.Oidx.p, L.Olpos.p, L.wptr.p, At.p, datoff.p, Aww.p, dawoff.p, es);
        CK_LAUNCH(); }
        // 2. Schur complement S = At_ww - At_wG At_GG^+ At_Gw via a semidefinite Cholesky of At_GG
        MatBatch bGG, bGw, bww, bW, bAww, bV, bC, bY;
        {
            std::vector<int64_t> o1(na), o2(na), o3(na);
            std::vector<int32_t> l1(na), mm(na);
            for (int64_t i = 0; i < na; i++) {
                o1[i] = atoff[i] + (int64_t)nwv[i] + (int64_t)nwv[i] * nOv[i];  // Gamma x Gamma
                o2[i] = atoff[i] + nwv[i];                                      // Gamma x omega
                o3[i] = atoff[i];                                               // omega x omega
                l1[i] = nOv[i];
                mm[i] = nwv[i];
            }
            bGG.set(o1, l1, nGv, {}, s);
            bGw.set(o2, l1, nGv, mm, s);
            bww.set(o3, l1, nwv, {}, s);
            bW.set(o2, l1, nGv, mm, s);
            std::vector<int64_t> o4(na), o5(na);
            for (int64_t i = 0; i < na; i++) {
                o4[i] = awoff[i];
                o5[i] = coff[i];
            }
            bAww.set(o4, nwv, nwv, nwv, s);
            bY.set(o3, l1, nwv, nwv, s);
            bC.set(o5, nwv, nwv, nwv, s);
        }
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: schur"), s);
        {
            // rank-revealing pivoted Cholesky of At_GG (the pseudo-inverse in eq. 2.9); row and
            // column swaps run over the whole At so At_wG / At_Gw are permuted consistently
            MatBatch bAt;
            std::vector<int64_t> oall(na), poff(na + 1, 0);
            for (int64_t i = 0; i < na; i++) {
                oall[i] = atoff[i];
                poff[i + 1] = poff[i] + nGv[i];
            }
            bAt.set(oall, nOv, nOv, {}, s);
            DBuf<int32_t> db0, dbn, perm, rank;
            DBuf<int64_t> dpoff;
            upload(db0, nwv, s);
            upload(dbn, nGv, s);
            upload(dpoff, poff, s);
            perm.alloc(std::max<int64_t>(poff[na], 1), s);
            rank.alloc(na, s);
            int32_t maxG = 0;
            for (auto g : nGv) maxG = std::max(maxG, g);
            pstrf_batched(At.p, bAt, db0.p, dbn.p, nwv, nGv, maxG, perm.p, dpoff.p, rank.p, err, s);
        }
        trsm_batched(At.p, bGG, At.p, bGw, false, s, err);                 // W = L_G^{-1} At_Gw
        syrk_tn_batched(At.p, bww, At.p, bW, -1.0, false, s, err);          // S = At_ww - W^T W
        }
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: gep transform"), s);
        // 3. GEP S y = mu A_ww y -> C = L^{-1} S L^{-T}
        potrf_batched(Aww.p, bAww, POTRF_SPD, err, s);
        trsm_batched(Aww.p, bAww, At.p, bY, false, s, err);                // Y = L^{-1} S
        transpose_batched(At.p, bww, C.p, bC, s);                     // C = Y^T
        trsm_batched(Aww.p, bAww, C.p, bC, false, s, err);                 // C = L^{-1} S L^{-T}
        }
        // 4. tridiagonalise, count and bisect the eigenvalues below 1/tau_cut
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: sytd2"), s); sytd2_batched(C.p, bC, dv.p, ev.p, tv.p, dtoff.p, s); }
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: stebz"), s); stebz_batched(dv.p, ev.p, dtoff.p, bC.n.p, na, sigma, dk.p, wv.p, gp.p, s); }
        auto hk = to_host(dk.p, na, s);
        auto hg = to_host(gp.p, na, s);
        check_err(err, s, "local spectral problems (factorisations)");
        std::vector<int64_t> voff(na + 1);
        voff[0] = 0;
        for (int64_t i = 0; i < na; i++) {
            L.h_k[ids[i]] = hk[i];
            L.h_gap[ids[i]] = hg[i];
            voff[i + 1] = voff[i] + (int64_t)nwv[i] * hk[i];
            *flops += 4.0 * nwv[i] * (double)nwv[i] * hk[i] + (double)nwv[i] * nwv[i] * hk[i];
        }
        Chunk ch;
        ch.ids = ids;
        ch.na = na;
        ch.voff = voff;
        ch.V.alloc(std::max<int64_t>(voff[na], 1), s);
        {
            std::vector<int64_t> o(na);
            for (int64_t i = 0; i < na; i++) o[i] = voff[i];
            bV.set(o, nwv, nwv, hk, s);
        }
        // 5. eigenvectors: inverse iteration, back-transformation, Z = L^{-T} V
        {
            // inverse iteration per eigenvalue, then one CholeskyQR2 over all retained vectors:
            // P needs an orthonormal basis of the retained invariant subspace, not the eigenvectors
            LSAMG_PROF(lvl_name(g_prof_level, "ls: stein"), s);
            stein_batched(dv.p, ev.p, dtoff.p, bC.n.p, wv.p, dk.p, ch.V.p, bV, s);
            cholqr2_batched(ch.V.p, bV, err, s);
        }
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: ormtr"), s); ormtr_batched(C.p, bC, tv.p, dtoff.p, ch.V.p, bV, s, err); }
        { LSAMG_PROF(lvl_name(g_prof_level, "ls: trsm Z"), s); trsm_batched(Aww.p, bAww, ch.V.p, bV, true, s, err); }
        CK(cudaStreamSynchronize(s));
        check_err(err, s, "local spectral problems");
        chunks.push_back(std::move(ch));
        q0 = q1;
    }
    // P storage: Z_i row-major, sign-normalised
    std::vector<int64_t> zoff(nagg + 1), off(nagg + 1);
    zoff[0] = off[0] = 0;
    for (int64_t a = 0; a < nagg; a++) {
        zoff[a + 1] = zoff[a] + (int64_t)L.h_nw[a] * L.h_k[a];
        off[a + 1] = off[a] + L.h_k[a];
    }
    L.nc = off[nagg];
    upload(L.zoff, zoff, s);
    upload(L.off, off, s);
    upload(L.k, L.h_k, s);
    L.max_k = L.h_k.empty() ? 0 : *std::max_element(L.h_k.begin(), L.h_k.end());
    L.max_nw = L.h_nw.empty() ? 0 : *std::max_element(L.h_nw.begin(), L.h_nw.end());
    {
        // Z_i read once, omega-indexed fine vector and the coarse vector once each
        double zw = 0.0;
        for (int64_t a = 0; a < nagg; a++) zw += (double)L.h_nw[a] * L.h_k[a];
        for (int t = 0; t < 2; t++) {
            const double sz = t ? 8.0 : 4.0;
            L.transfer_bytes[t] = zw * sz + (double)L.n * (sz + 4.0) + (double)L.nc * sz;
        }
    }
    L.Z64.alloc(std::max<int64_t>(zoff[nagg], 1), s);
    L.Z32.alloc(std::max<int64_t>(zoff[nagg], 1), s);
    for (auto &ch : chunks) {
        DBuf<int64_t> dvo, dzo;
        DBuf<int32_t> dnw, dkk;
        std::vector<int64_t> zo(ch.na);
        std::vector<int32_t> nwv(ch.na), kv(ch.na);
        for (int64_t i = 0; i < ch.na; i++) {
            zo[i] = zoff[ch.ids[i]];
            nwv[i] = L.h_nw[ch.ids[i]];
            kv[i] = L.h_k[ch.ids[i]];
        }
        upload(dvo, ch.voff, s);
        upload(dzo, zo, s);
        upload(dnw, nwv, s);
        upload(dkk, kv, s);
        k_store_z<<<(unsigned)ch.na, 256, 0, s>>>(ch.V.p, dvo.p, dnw.p, dkk.p, ch.na, L.Z64.p, L.Z32.p,
                                                 dzo.p);
        CK_LAUNCH();
        CK(cudaStreamSynchronize(s));
    }
    check_err(err, s, "interpolation");
}

void build_coarse(Level &F, Level &C, int *err, cudaStream_t s, double *flops) {
    const int64_t ne = F.ne;
    // coarse map length of every element and a hash of its aggregate set
    DBuf<int64_t> clen;
    DBuf<uint64_t> h;
    clen.alloc(std::max<int64_t>(ne, 1), s);
    h.alloc(std::max<int64_t>(ne, 1), s);
    k_coarse_len<<<gridc(ne), 256, 0, s>>>(F.eaptr.p, F.eaidx.p, ne, F.k.p, clen.p, h.p);
    CK_LAUNCH();
    // sort elements by (hash of the aggregate set [high 40 bits], element id [low 24 bits]);
    // equal sets are then adjacent, each run led by its smallest element
    if (ne >= (1 << 24)) fail(LSAMG_LIMIT, "more than 2^24 elements on one level");
    DBuf<uint64_t> keys;
    DBuf<int32_t> dorder, lflag, rstart;
    keys.alloc(std::max<int64_t>(ne, 1), s);
    dorder.alloc(std::max<int64_t>(ne, 1), s);
    k_make_keys<<<gridc(ne), 256, 0, s>>>(h.p, ne, keys.p);
    CK_LAUNCH();
    sort_u64(keys.p, ne, s);
    k_extract_order<<<gridc(ne), 256, 0, s>>>(keys.p, ne, dorder.p);
    CK_LAUNCH();
    lflag.alloc(std::max<int64_t>(ne, 1), s);
    lflag.zero(s);
    rstart.alloc(std::max<int64_t>(ne, 1), s);
    k_same_set<<<gridc(ne), 256, 0, s>>>(dorder.p, ne, F.eaptr.p, F.eaidx.p, h.p, lflag.p, rstart.p,
                                         err);
    CK_LAUNCH();
    DBuf<int64_t> gid;
    gid.alloc(ne + 1, s);
    exclusive_scan_i32(lflag.p, gid.p, ne, s);
    const int64_t ng = read1(gid.p + ne, s);
    F.cgroup.alloc(std::max<int64_t>(ne, 1), s);
    CK(cudaMemsetAsync(F.cgroup.p, 0xff, std::max<int64_t>(ne, 1) * sizeof(int32_t), s));
    k_assign_group<<<gridc(ne), 256, 0, s>>>(dorder.p, ne, rstart.p, gid.p, F.cgroup.p);
    CK_LAUNCH();
    check_err(err, s, "coarse element grouping");
    DBuf<int32_t> leader;
    leader.alloc(std::max<int64_t>(ng, 1), s);
    k_leader_of_group<<<gridc(ne), 256, 0, s>>>(lflag.p, gid.p, ne, leader.p);
    CK_LAUNCH();
    // group -> member elements (ascending)
    DBuf<int64_t> mptr;
    DBuf<int32_t> midx;
    {
        // element -> group CSR (one or zero entries)
        auto cg = to_host(F.cgroup.p, ne, s);
        std::vector<int64_t> p(ne + 1, 0);
        std::vector<int32_t> idx;
        idx.reserve(ne);
        for (int64_t e = 0; e < ne; e++) {
            p[e + 1] = p[e] + (cg[e] >= 0);
            if (cg[e] >= 0) idx.push_back(cg[e]);
        }
        DBuf<int64_t> dp;
        DBuf<int32_t> di;
        upload(dp, p, s);
        upload(di, idx, s);
        csr_transpose(dp.p, di.p, ne, (int64_t)idx.size(), ng, mptr, midx, err, s);
    }
    DBuf<int64_t> gcols, growt;
    gcols.alloc(std::max<int64_t>(ng, 1), s);
    growt.alloc(std::max<int64_t>(ng, 1), s);
    k_group_sizes<<<gridc(ng), 256, 0, s>>>(leader.p, ng, clen.p, mptr.p, midx.p, F.grows.p, gcols.p,
                                           growt.p);
    CK_LAUNCH();
    auto hcols = to_host(gcols.p, ng, s);
    auto hrows = to_host(growt.p, ng, s);
    // coarse level element maps
    C.n = F.nc;
    C.ne = ng;
    C.eptr.alloc(ng + 1, s);
    exclusive_scan_i64(gcols.p, C.eptr.p, ng, s);
    C.nnz_e = read1(C.eptr.p + ng, s);
    C.eidx.alloc(std::max<int64_t>(C.nnz_e, 1), s);
    if (ng > 0) {
        k_fill_cmap<<<(unsigned)ng, 32, 0, s>>>(leader.p, ng, F.eaptr.p, F.eaidx.p, F.k.p, F.off.p,
                                                 C.eptr.p, C.eidx.p);
        CK_LAUNCH();
    }
    // coarse G: stacked G_c,T = G_T (R_T P) of the members (Section 2: G_c = G P)
    std::vector<int64_t> cgoff(ng + 1, 0), caoff(ng + 1, 0);
    std::vector<int32_t> crows(ng);
    int32_t maxc = 0;
    for (int64_t g = 0; g < ng; g++) {
        cgoff[g + 1] = cgoff[g] + hrows[g] * hcols[g];
        caoff[g + 1] = caoff[g] + hcols[g] * hcols[g];
        crows[g] = (int32_t)hrows[g];
        maxc = std::max<int32_t>(maxc, (int32_t)hcols[g]);
    }
    C.max_nT = maxc;
    DBuf<double> Gst;  // stacked G_c,T = G_T (R_T P) of the members (Section 2: G_c = G P)
    DBuf<int64_t> dgst;
    upload(dgst, cgoff, s);
    upload(C.aoff, caoff, s);
    Gst.alloc(std::max<int64_t>(cgoff[ng], 1), s);
    DBuf<int64_t> rowbase, dcgoff;
    rowbase.alloc(std::max<int64_t>(ne, 1), s);
    k_rowbase<<<gridc(ng), 256, 0, s>>>(mptr.p, midx.p, ng, F.grows.p, rowbase.p);
    CK_LAUNCH();
    {
        auto cg = to_host(F.cgroup.p, ne, s);
        auto fr = to_host(F.grows.p, ne, s);
        std::vector<int32_t> items;
        for (int64_t e = 0; e < ne; e++) {
            if (cg[e] < 0) continue;
            int64_t ncol = hcols[cg[e]];
            int64_t tr = cdiv(std::max<int32_t>(fr[e], 1), 32), tc = cdiv(ncol, 64);
            for (int64_t a = 0; a < tr; a++)
                for (int64_t b = 0; b < tc; b++) {
                    items.push_back((int32_t)e);
                    items.push_back((int32_t)a);
                    items.push_back((int32_t)b);
                }
            *flops += 2.0 * fr[e] * ncol * (double)(F.max_nT > 0 ? F.max_nT : 0);
        }
        DBuf<int32_t> ditems;
        upload(ditems, items, s);
        int64_t nit = (int64_t)items.size() / 3;
        if (nit > 0) {
            KTime kt(KC_COARSE_GRAM, s);
            k_gc<<<(unsigned)nit, 256, 0, s>>>(ditems.p, nit, F.eptr.p, F.eidx.p, F.G64.p, F.goff.p,
                                                F.grows.p, F.eaptr.p, F.eaidx.p, F.agg.p, F.posw.p,
                                                F.k.p, F.Z64.p, F.zoff.p, F.cgroup.p, dgst.p,
                                                gcols.p, rowbase.p, Gst.p);
            CK_LAUNCH();
        }
    }
    // A_g = G_g^T G_g (setup of the next level works on element blocks)
    C.AT.alloc(std::max<int64_t>(caoff[ng], 1), s);
    C.AT.zero(s);
    {
        MatBatch bA, bG;
        std::vector<int64_t> oa(ng), og(ng);
        std::vector<int32_t> nn(ng), kk(ng), ldg(ng);
        for (int64_t g = 0; g < ng; g++) {
            oa[g] = caoff[g];
            og[g] = cgoff[g];
            nn[g] = (int32_t)hcols[g];
            kk[g] = (int32_t)hrows[g];
            ldg[g] = (int32_t)hcols[g];
            *flops += 2.0 * hrows[g] * (double)hcols[g] * hcols[g];
        }
        bA.set(oa, nn, nn, {}, s);
        bG.set(og, ldg, kk, nn, s);
        syrk_tn_batched(C.AT.p, bA, Gst.p, bG, 1.0, true, s, err);
        DBuf<int64_t> dn;
        std::vector<int64_t> n64(hcols.begin(), hcols.end());
        upload(dn, n64, s);
        dim3 gsym(64, (unsigned)std::max<int64_t>(ng, 1));
        if (ng > 0) {
            k_symmetrize_sq<<<gsym, 256, 0, s>>>(C.AT.p, C.aoff.p, dn.p, ng);
            CK_LAUNCH();
        }
        // Remark 5.2: the coarse element's Gram rows are replaced by a rank-revealing factor of
        // A_g (rank <= min(stacked rows, columns)); G'^T G' = A_g up to the truncation of
        // numerically zero pivots, so the coarse operator is unchanged
        DBuf<double> Wf;
        Wf.alloc(std::max<int64_t>(caoff[ng], 1), s);
        CK(cudaMemcpyAsync(Wf.p, C.AT.p, caoff[ng] * sizeof(double), cudaMemcpyDeviceToDevice, s));
        MatBatch bW;
        std::vector<int32_t> zero(ng, 0);
        bW.set(oa, nn, nn, {}, s);
        std::vector<int64_t> poff(ng + 1, 0);
        int32_t maxn = 0;
        for (int64_t g = 0; g < ng; g++) {
            poff[g + 1] = poff[g] + hcols[g];
            maxn = std::max<int32_t>(maxn, (int32_t)hcols[g]);
            *flops += (double)hcols[g] * hcols[g] * hcols[g] / 3.0;
        }
        DBuf<int32_t> db0, dbn, perm, rank;
        DBuf<int64_t> dpoff;
        upload(db0, zero, s);
        upload(dbn, nn, s);
        upload(dpoff, poff, s);
        perm.alloc(std::max<int64_t>(poff[ng], 1), s);
        rank.alloc(std::max<int64_t>(ng, 1), s);
        pstrf_batched(Wf.p, bW, db0.p, dbn.p, zero, nn, maxn, perm.p, dpoff.p, rank.p, err, s);
        auto hr = to_host(rank.p, ng, s);
        std::vector<int64_t> ngoff(ng + 1, 0);
        std::vector<int32_t> nrows(ng);
        for (int64_t g = 0; g < ng; g++) {   // G_c of group g: its rank rows x its coarse columns
            ngoff[g + 1] = ngoff[g] + (int64_t)hr[g] * hcols[g];
            nrows[g] = hr[g];
        }
        upload(C.goff, ngoff, s);
        upload(C.grows, nrows, s);
        C.G64.alloc(std::max<int64_t>(ngoff[ng], 1), s);
        C.G32.alloc(std::max<int64_t>(ngoff[ng], 1), s);
        C.G64.zero(s);
        C.G32.zero(s);
        dim3 gx(64, (unsigned)std::max<int64_t>(ng, 1));
        if (ng > 0) {
            k_extract_factor<<<gx, 256, 0, s>>>(Wf.p, C.aoff.p, dn.p, perm.p, dpoff.p, rank.p, C.goff.p,
                                                 ng, C.G64.p, C.G32.p);
            CK_LAUNCH();
        }
    }
    CK(cudaStreamSynchronize(s));
    check_err(err, s, "coarse level");
}

void smoother_setup(Level &L, const lsamg_options &o, int *err, cudaStream_t s, double *flops) {
    const int64_t nagg = L.nagg;
    int32_t maxE = 1;
    {
        auto ep = to_host(L.eptr.p, L.ne + 1, s);
        for (int64_t e = 0; e < L.ne; e++) maxE = std::max<int32_t>(maxE, (int32_t)(ep[e + 1] - ep[e]));
    }
    if ((size_t)maxE * sizeof(int32_t) > 200 * 1024) fail(LSAMG_LIMIT, "element map longer than the assembly staging");
    std::vector<int64_t> loff(nagg + 1, 0);
    for (int64_t a = 0; a < nagg; a++) loff[a + 1] = loff[a] + (int64_t)L.h_nO[a] * (L.h_nO[a] + 1) / 2;
    upload(L.Loff, loff, s);
    L.L64.alloc(std::max<int64_t>(loff[nagg], 1), s);
    L.L32.alloc(std::max<int64_t>(loff[nagg], 1), s);
    int64_t budget = o.chunk_bytes > 0 ? o.chunk_bytes : (int64_t)48 << 30;
    int64_t a0 = 0;
    while (a0 < nagg) {
        int64_t bytes = 0, a1 = a0;
        while (a1 < nagg) {
            int64_t b = (int64_t)L.h_nO[a1] * L.h_nO[a1] * 8;
            if (a1 > a0 && bytes + b > budget) break;
            bytes += b;
            a1++;
        }
        const int64_t na = a1 - a0;
        std::vector<int64_t> mo(na + 1, 0), po(na);
        std::vector<int32_t> nn(na);
        for (int64_t i = 0; i < na; i++) {
            int64_t nO = L.h_nO[a0 + i];
            mo[i + 1] = mo[i] + nO * nO;
            nn[i] = (int32_t)nO;
            po[i] = loff[a0 + i];
            *flops += (double)nO * nO * nO / 3.0;
        }
        DBuf<double> AO;
        DBuf<int64_t> dmo, dpo;
        DBuf<int32_t> dnn;
        AO.alloc(std::max<int64_t>(mo[na], 1), s);
        AO.zero(s);
        upload(dmo, mo, s);
        upload(dpo, po, s);
        upload(dnn, nn, s);
        {
            KTime kta(KC_ASSEMBLE, s);
            const int es = assembly_slices(na);
            const size_t asm_smem = (size_t)maxE * sizeof(int32_t);
            CK(cudaFuncSetAttribute(k_assemble_smoother, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)asm_smem));
            k_assemble_smoother<<<dim3((unsigned)na, (unsigned)es), 256, asm_smem, s>>>(
                a0, na, L.oeptr.p, L.oeidx.p, L.eptr.p, L.AT.p, L.aoff.p, L.oelocoff.p, L.oeloc.p, L.Optr.p,
                AO.p, dmo.p, es);
            CK_LAUNCH();
        }
        MatBatch b;
        std::vector<int64_t> o1(mo.begin(), mo.end() - 1);
        b.set(o1, nn, nn, {}, s);
        potrf_batched(AO.p, b, POTRF_SPD, err, s);
        dim3 g(64, (unsigned)na);
        k_pack_lower<<<g, 256, 0, s>>>(AO.p, dmo.p, dnn.p, na, L.L64.p, L.L32.p, dpo.p);
        CK_LAUNCH();
        CK(cudaStreamSynchronize(s));
        check_err(err, s, "Schwarz factors");
        a0 = a1;
    }
    L.tri_cb = g_sweep_block > 0 ? std::min(g_sweep_block, 64) : 64;
    tri_inverse_setup(nagg, L.Optr.p, L.h_nO, L.L64.p, L.Loff.p, L.tri_cb, L.Doff, L.Di64, s);
    CK(cudaStreamSynchronize(s));
}

void coarsest_setup(Level &L, int *err, cudaStream_t s, double *flops) {
    const int64_t n = L.n;
    DBuf<double> D;
    D.alloc(std::max<int64_t>(n * n, 1), s);
    D.zero(s);
    if (L.ne > 0) {
        k_assemble_dense<<<gridc(n, 1, 148 * 16), 256, 0, s>>>(L.eptr.p, L.eidx.p, L.dptr.p, L.didx.p, L.AT.p,
                                                              L.aoff.p, D.p, n);
        CK_LAUNCH();
    }
    MatBatch b;
    b.set({0}, {(int32_t)n}, {(int32_t)n}, {}, s);
    potrf_batched(D.p, b, POTRF_SPD, err, s);
    *flops += (double)n * n * n / 3.0;
    int64_t tot = n * (n + 1) / 2;
    L.Ld64.alloc(std::max<int64_t>(tot, 1), s);
    L.Ld32.alloc(std::max<int64_t>(tot, 1), s);
    DBuf<int64_t> z;
    DBuf<int32_t> nn;
    upload(z, std::vector<int64_t>{0}, s);
    upload(nn, std::vector<int32_t>{(int32_t)n}, s);
    dim3 g((unsigned)std::min<int64_t>(cdiv(tot, 256), 148 * 8), 1);
    k_pack_lower<<<g, 256, 0, s>>>(D.p, z.p, nn.p, 1, L.Ld64.p, L.Ld32.p, z.p);
    CK_LAUNCH();
    upload(L.cs_ptr, std::vector<int64_t>{0, n}, s);
    upload(L.cs_off, std::vector<int64_t>{0}, s);
    L.tri_cb = g_sweep_block > 0 ? std::min(g_sweep_block, 64) : 64;
    tri_inverse_setup(1, L.cs_ptr.p, std::vector<int32_t>{(int32_t)n}, L.Ld64.p, L.cs_off.p, L.tri_cb, L.Doff,
                      L.Di64, s);
    CK(cudaStreamSynchronize(s));
    check_err(err, s, "coarsest factorisation");
}

}  // namespace lsamg
