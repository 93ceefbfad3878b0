// Integer set-up of one level: input validation, DOF->element maps, two-pass MIS(2)
// aggregation (Section 2 eq. 2.2; the Section 6 tests aggregate in two passes), element-form
// closure and multiplicity (eqs. 2.3-2.5, Thm 5.6),
// tau_cut (eq. 2.10), the element lists of each overlap and the smoother colouring.
//
// The structural graph (p ~ q iff p and q share an element) is never assembled: a
// max/min over the distance-1 neighbourhood of every node is computed as an element
// reduction followed by a scatter back to the element's nodes.
#include "impl.cuh"

namespace lsamg {

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t items, int per_block = TPB, int64_t cap = 148 * 32) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(items, per_block), cap));
}

// lowbias32 integer mix (C. Wellons, hash-prospector): priority of the MIS(2) rounds
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint64_t mis_key(int state, uint32_t v) {
    return ((uint64_t)(state + 1) << 62) | ((uint64_t)hash32(v) << 30) | (uint64_t)v;
}

// ---------------------------------------------------------------- validation
__global__ void k_check_input(const int64_t *eptr, const int32_t *eidx, int64_t ne, int64_t n,
                              int *err) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w; e < ne; e += nw) {
        int64_t b = eptr[e], en = eptr[e + 1];
        int len = (int)(en - b);
        for (int i = lane; i < len; i += 32) {
            int32_t d = eidx[b + i];
            if (d < 0 || d >= n) flag_error(err, LSAMG_INVALID_ARG, (int)e);
            for (int j = i + 1; j < len; j++)
                if (eidx[b + j] == d) flag_error(err, LSAMG_INVALID_ARG, (int)e);
        }
    }
}

// ---------------------------------------------------------------- neighbourhood reductions
// emax[e] = max/min over q in N(e) of key[map(q)]
template <bool MAX>
__global__ void k_elem_reduce(const int64_t *eptr, const int32_t *eidx, int64_t ne,
                              const int32_t *map, const uint64_t *key, uint64_t *eval) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w; e < ne; e += nw) {
        uint64_t acc = MAX ? 0ull : ~0ull;
        for (int64_t j = eptr[e] + lane; j < eptr[e + 1]; j += 32) {
            int32_t q = eidx[j];
            uint64_t v = key[map ? map[q] : q];
            acc = MAX ? max(acc, v) : min(acc, v);
        }
        for (int o = 16; o; o >>= 1) {
            uint64_t t = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = MAX ? max(acc, t) : min(acc, t);
        }
        if (lane == 0) eval[e] = acc;
    }
}

// out[map(q)] = max/min(out[map(q)], eval[e]) for q in N(e)
template <bool MAX>
__global__ void k_scatter_reduce(const int64_t *eptr, const int32_t *eidx, int64_t ne,
                                 const int32_t *map, const uint64_t *eval, uint64_t *out) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w; e < ne; e += nw) {
        uint64_t v = eval[e];
        for (int64_t j = eptr[e] + lane; j < eptr[e + 1]; j += 32) {
            int32_t q = eidx[j];
            unsigned long long *dst = (unsigned long long *)&out[map ? map[q] : q];
            if (MAX)
                atomicMax(dst, (unsigned long long)v);
            else
                atomicMin(dst, (unsigned long long)v);
        }
    }
}

struct Hop {
    const int64_t *eptr;
    const int32_t *eidx;
    int64_t ne;
    const int32_t *map;
    int64_t nn;
    uint64_t *eval;
};

// out = reduction of in over each node's distance-1 neighbourhood (the node included)
template <bool MAX>
void hop(const Hop &h, const uint64_t *in, uint64_t *out, cudaStream_t s) {
    CK(cudaMemcpyAsync(out, in, h.nn * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    unsigned g = grid_for(h.ne * 32);
    k_elem_reduce<MAX><<<g, TPB, 0, s>>>(h.eptr, h.eidx, h.ne, h.map, in, h.eval);
    CK_LAUNCH();
    k_scatter_reduce<MAX><<<g, TPB, 0, s>>>(h.eptr, h.eidx, h.ne, h.map, h.eval, out);
    CK_LAUNCH();
}

__global__ void k_mis_keys(const int8_t *state, int64_t nn, uint64_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x)
        key[v] = mis_key(state[v], (uint32_t)v);
}

__global__ void k_mis_decide(int8_t *state, const uint64_t *m2, int64_t nn, int *undecided) {
    int local = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (state[v] != 0) continue;
        uint64_t m = m2[v];
        if ((m & ((1ull << 30) - 1)) == (uint64_t)v)
            state[v] = 1;
        else if ((m >> 62) == 2ull)
            state[v] = -1;
        else
            local++;
    }
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(undecided, local);
}

__global__ void k_root_flags(const int8_t *state, int64_t nn, int32_t *flag) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = state[v] == 1;
}

__global__ void k_root_vals(const int8_t *state, const int64_t *rank, int64_t nn, uint64_t *val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x)
        val[v] = state[v] == 1 ? (uint64_t)(rank[v] + 1) : 0ull;
}

__global__ void k_agg_from_roots(const uint64_t *m, int64_t nn, int32_t *agg) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x)
        agg[v] = (int32_t)m[v] - 1;
}

__global__ void k_join_keys(const int32_t *agg, int64_t nn, uint64_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x)
        key[v] = agg[v] >= 0 ? (((uint64_t)hash32((uint32_t)v) << 32) | (uint64_t)v) : ~0ull;
}

__global__ void k_join(const int32_t *agg, const uint64_t *mn, int64_t nn, int32_t *agg_new,
                       int *remaining) {
    int local = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nn;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = agg[v];
        if (a < 0) {
            uint64_t m = mn[v];
            if (m != ~0ull)
                a = agg[(int64_t)(m & 0xffffffffull)];
            else
                local++;
        }
        agg_new[v] = a;
    }
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(remaining, local);
}

__global__ void k_compose(int32_t *agg, const int32_t *agg2, int64_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        agg[v] = agg2[agg[v]];
}

// One MIS(2) aggregation pass on nn nodes, nodes of element entries given by map (or the
// entries themselves).  Returns the number of aggregates; out[v] = aggregate of node v.
int32_t mis2_pass(const Level &L, const int32_t *map, int64_t nn, DBuf<int32_t> &out, int *err,
                  cudaStream_t s) {
    DBuf<int8_t> state;
    DBuf<uint64_t> key, m1, m2, eval;
    DBuf<int> cnt;
    state.alloc(nn, s);
    state.zero(s);
    key.alloc(nn, s);
    m1.alloc(nn, s);
    m2.alloc(nn, s);
    eval.alloc(std::max<int64_t>(L.ne, 1), s);
    cnt.alloc(1, s);
    Hop h{L.eptr.p, L.eidx.p, L.ne, map, nn, eval.p};
    unsigned gn = grid_for(nn);
    for (int round = 0;; round++) {
        if (round > 4096) fail(LSAMG_DEVICE_TIMEOUT, "MIS(2) did not terminate");
        k_mis_keys<<<gn, TPB, 0, s>>>(state.p, nn, key.p);
        CK_LAUNCH();
        hop<true>(h, key.p, m1.p, s);
        hop<true>(h, m1.p, m2.p, s);
        cnt.zero(s);
        k_mis_decide<<<gn, TPB, 0, s>>>(state.p, m2.p, nn, cnt.p);
        CK_LAUNCH();
        if (read1(cnt.p, s) == 0) break;
    }
    // aggregates: roots (ascending) with their distance-1 neighbourhoods
    DBuf<int32_t> flag;
    DBuf<int64_t> rank;
    flag.alloc(nn, s);
    rank.alloc(nn + 1, s);
    k_root_flags<<<gn, TPB, 0, s>>>(state.p, nn, flag.p);
    CK_LAUNCH();
    exclusive_scan_i32(flag.p, rank.p, nn, s);
    int64_t nroot = read1(rank.p + nn, s);
    k_root_vals<<<gn, TPB, 0, s>>>(state.p, rank.p, nn, key.p);
    CK_LAUNCH();
    hop<true>(h, key.p, m1.p, s);
    out.alloc(nn, s);
    k_agg_from_roots<<<gn, TPB, 0, s>>>(m1.p, nn, out.p);
    CK_LAUNCH();
    // remaining nodes join the aggregated neighbour with the smallest (hash, index)
    DBuf<int32_t> tmp;
    tmp.alloc(nn, s);
    for (int round = 0;; round++) {
        if (round > 1024) fail(LSAMG_DEVICE_TIMEOUT, "aggregation join did not terminate");
        k_join_keys<<<gn, TPB, 0, s>>>(out.p, nn, key.p);
        CK_LAUNCH();
        hop<false>(h, key.p, m1.p, s);
        cnt.zero(s);
        k_join<<<gn, TPB, 0, s>>>(out.p, m1.p, nn, tmp.p, cnt.p);
        CK_LAUNCH();
        std::swap(out, tmp);
        int rem = read1(cnt.p, s);
        if (rem == 0) break;
    }
    (void)err;
    return (int32_t)nroot;
}

// ---------------------------------------------------------------- closure helpers
__global__ void k_gather_agg(const int32_t *eidx, int64_t nnz, const int32_t *agg, int32_t *vals) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x)
        vals[j] = agg[eidx[j]];
}

__global__ void k_copy_i64_to_i32(const int64_t *a, int32_t *b, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        b[j] = (int32_t)a[j];
}

// count[r] = sum over c in rows(r) of len(c) where rows: CSR r -> c and len from ptr2
__global__ void k_count_union(const int64_t *ptr, const int32_t *idx, int64_t nr,
                              const int64_t *ptr2, int64_t *cnt) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int64_t j = ptr[r]; j < ptr[r + 1]; j++) c += ptr2[idx[j] + 1] - ptr2[idx[j]];
        cnt[r] = c;
    }
}

// vals[optr[r]..] = concatenation of idx2[ptr2[c]..ptr2[c+1]) over c in rows(r); warp per row
__global__ void k_fill_union(const int64_t *ptr, const int32_t *idx, int64_t nr, const int64_t *ptr2,
                             const int32_t *idx2, const int64_t *optr, int32_t *vals) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < nr; r += nw) {
        int64_t o = optr[r];
        for (int64_t j = ptr[r]; j < ptr[r + 1]; j++) {
            int32_t c = idx[j];
            int64_t b = ptr2[c], len = ptr2[c + 1] - b;
            for (int64_t t = lane; t < len; t += 32) vals[o + t] = idx2[b + t];
            o += len;
        }
    }
}

// out CSR = sorted unique union over c in rows(r) of list2(c).  (rows: ptr/idx, lists: ptr2/idx2)
void csr_union(const int64_t *ptr, const int32_t *idx, int64_t nr, const int64_t *ptr2,
               const int32_t *idx2, DBuf<int64_t> &optr, DBuf<int32_t> &oidx, int *err,
               cudaStream_t s) {
    DBuf<int64_t> cnt, cptr, ucnt;
    cnt.alloc(nr, s);
    cptr.alloc(nr + 1, s);
    if (nr > 0) {
        k_count_union<<<grid_for(nr), TPB, 0, s>>>(ptr, idx, nr, ptr2, cnt.p);
        CK_LAUNCH();
    }
    exclusive_scan_i64(cnt.p, cptr.p, nr, s);
    int64_t tot = read1(cptr.p + nr, s);
    DBuf<int32_t> vals;
    vals.alloc(std::max<int64_t>(tot, 1), s);
    if (nr > 0) {
        k_fill_union<<<grid_for(nr * 32), TPB, 0, s>>>(ptr, idx, nr, ptr2, idx2, cptr.p, vals.p);
        CK_LAUNCH();
    }
    ucnt.alloc(nr, s);
    seg_sort(vals.p, cptr.p, nr, ucnt.p, err, s);
    optr.alloc(nr + 1, s);
    exclusive_scan_i64(ucnt.p, optr.p, nr, s);
    int64_t utot = read1(optr.p + nr, s);
    oidx.alloc(std::max<int64_t>(utot, 1), s);
    seg_unique_compact(vals.p, cptr.p, nr, optr.p, oidx.p, s);
}

__global__ void k_posw(const int64_t *wptr, const int32_t *widx, int64_t nagg, int32_t *posw) {
    int64_t a = blockIdx.x;
    if (a >= nagg) return;
    for (int64_t j = wptr[a] + threadIdx.x; j < wptr[a + 1]; j += blockDim.x)
        posw[widx[j]] = (int32_t)(j - wptr[a]);
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t v) {
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

// omega-first local index of every Omega_i entry: omega DOFs by rank in omega_i, then the
// interface Gamma_i in ascending DOF order
__global__ void k_olpos(const int64_t *Optr, const int32_t *Oidx, const int64_t *wptr,
                        const int32_t *widx, const int32_t *agg, const int32_t *posw,
                        int64_t nagg, int32_t *lpos) {
    int64_t a = blockIdx.x;
    if (a >= nagg) return;
    int64_t b = Optr[a], e = Optr[a + 1];
    int64_t wb = wptr[a], nw = wptr[a + 1] - wb;
    for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
        int32_t q = Oidx[j];
        if (agg[q] == a)
            lpos[j] = posw[q];
        else
            lpos[j] = (int32_t)(nw + (j - b) - lower_bound_i32(widx + wb, nw, q));
    }
}

// Algebraic A-closure (Def. 5.2), decided on the G-row closure Omega^G_i, which contains it
// (an assembled entry A(q, p) needs an element holding both q and p).
// |A(r, r)| of every DOF, summed over its elements in ascending element order
__global__ void k_assembled_diag(const int64_t *dptr, const int32_t *didx, int64_t n, const int64_t *eptr,
                                 const int32_t *eidx, const double *AT, const int64_t *aoff, double *dg) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int64_t j = dptr[r]; j < dptr[r + 1]; j++) {
            const int32_t e = didx[j];
            const int64_t b = eptr[e];
            const int nT = (int)(eptr[e + 1] - b);
            int c = 0;
            while (c < nT && eidx[b + c] != (int32_t)r) c++;
            if (c < nT) v += AT[aoff[e] + (int64_t)c * nT + c];
        }
        dg[r] = fabs(v);
    }
}

// B_i = A(omega_i, Omega^G_i) stored column q-rank major: B[p_pos + q_rank * nO] = assembled A(q, p)
// over the elements touching omega_i, each entry summed in ascending element order by the one
// CTA owning its column (element matrices column-major: A_T(c, r) at Ae[r * nT + c])
__global__ void k_assemble_rect(const int32_t *ids, int64_t na, const int64_t *aeptr, const int32_t *aeidx,
                                const int64_t *eptr, const int32_t *eidx, const double *AT, const int64_t *aoff,
                                const int64_t *Optr, const int32_t *Oidx, const int32_t *agg,
                                const int32_t *posw, double *B, const int64_t *boff, int maxE, int es) {
    extern __shared__ int32_t sh[];   // [maxE] rows (position in Omega^G), [maxE] columns, [maxE] owned
    __shared__ int ncols;
    const int64_t li = blockIdx.x;
    if (li >= na) return;
    const int32_t a = ids[li];
    const int32_t *Om = Oidx + Optr[a];
    const int64_t nO = Optr[a + 1] - Optr[a];
    double *M = B + boff[li];
    int32_t *prow = sh, *pcol = sh + maxE, *own = sh + 2 * maxE;
    const int slice = blockIdx.y;
    for (int64_t j = aeptr[a]; j < aeptr[a + 1]; j++) {
        const int32_t e = aeidx[j];
        const int64_t b = eptr[e];
        const int n = (int)(eptr[e + 1] - b);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int32_t q = eidx[b + t];
            prow[t] = (int32_t)lower_bound_i32(Om, nO, q);   // N(T) is inside Omega^G_i
            pcol[t] = agg[q] == a ? posw[q] : -1;
        }
        __syncthreads();
        warp_compact(n, own, &ncols, [&](int c) { return pcol[c] >= 0 && pcol[c] % es == slice; });
        __syncthreads();
        const double *Ae = AT + aoff[e];
        const int nc = ncols;
        for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
            const int c = own[t / n], r = t % n;
            M[prow[r] + (int64_t)pcol[c] * nO] += Ae[(int64_t)r * n + c];
        }
        __syncthreads();
    }
}

// keep[j] for the entries of Omega^G_i: p in omega_i, or |A(q, p)| > cut sqrt(|A(q, q)| |A(p, p)|)
// for some q in omega_i (entries that cancel in exact arithmetic -- exact zeros on the finest
// level, rounding after coarse Galerkin products -- count as zero)
__global__ void k_a_keep(const int32_t *ids, int64_t na, const int64_t *Optr, const int32_t *Oidx,
                         const int32_t *agg, const int64_t *wptr, const int32_t *widx, const double *dg,
                         const double *B, const int64_t *boff, double cut, int32_t *keep) {
    const int64_t li = blockIdx.x;
    if (li >= na) return;
    const int32_t a = ids[li];
    const int64_t ob = Optr[a], nO = Optr[a + 1] - ob;
    const int64_t wb = wptr[a], nw = wptr[a + 1] - wb;
    const double *M = B + boff[li];
    for (int64_t rr = threadIdx.x; rr < nO; rr += blockDim.x) {
        const int32_t p = Oidx[ob + rr];
        bool k = agg[p] == a;
        for (int64_t c = 0; c < nw && !k; c++)
            k = fabs(M[rr + c * nO]) > cut * sqrt(dg[p] * dg[widx[wb + c]]);
        keep[ob + rr] = k ? 1 : 0;
    }
}

// per aggregate: number of kept entries; then the kept entries in order (one warp per aggregate)
__global__ void k_keep_count(const int64_t *Optr, const int32_t *keep, int64_t nagg, int64_t *cnt) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nagg;
         a += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int64_t j = Optr[a]; j < Optr[a + 1]; j++) c += keep[j];
        cnt[a] = c;
    }
}

__global__ void k_keep_fill(const int64_t *Optr, const int32_t *Oidx, const int32_t *keep, int64_t nagg,
                            const int64_t *optr, int32_t *oidx) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = w0; a < nagg; a += nwarp) {
        int64_t o = optr[a];
        for (int64_t j0 = Optr[a]; j0 < Optr[a + 1]; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool k = j < Optr[a + 1] && keep[j];
            const unsigned m = __ballot_sync(0xffffffffu, k);
            if (k) oidx[o + __popc(m & ((1u << lane) - 1u))] = Oidx[j];
            o += __popc(m);
        }
    }
}

// per (aggregate, element meeting Omega) entry: offset of its local-position block
__global__ void k_oeloc_count(const int64_t *oeptr, const int32_t *oeidx, int64_t nent,
                              const int64_t *eptr, int64_t *cnt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nent;
         j += (int64_t)gridDim.x * blockDim.x)
        cnt[j] = eptr[oeidx[j] + 1] - eptr[oeidx[j]];
}

__global__ void k_oeloc_fill(const int64_t *oeptr, const int32_t *oeidx, int64_t nagg,
                             const int64_t *eptr, const int32_t *eidx, const int64_t *Optr,
                             const int32_t *Oidx, const int64_t *locoff, int32_t *loc) {
    int64_t a = blockIdx.x;
    if (a >= nagg) return;
    const int32_t *Om = Oidx + Optr[a];
    int64_t nO = Optr[a + 1] - Optr[a];
    for (int64_t j = oeptr[a]; j < oeptr[a + 1]; j++) {
        int32_t e = oeidx[j];
        int64_t b = eptr[e], len = eptr[e + 1] - b;
        for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
            int32_t q = eidx[b + t];
            int64_t p = lower_bound_i32(Om, nO, q);
            loc[locoff[j] + t] = (p < nO && Om[p] == q) ? (int32_t)p : -1;
        }
    }
}

// ---------------------------------------------------------------- colouring
__global__ void k_remove_self(const int64_t *ptr, const int32_t *idx, int64_t nr, int32_t *cnt) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        for (int64_t j = ptr[r]; j < ptr[r + 1]; j++) c += idx[j] < r;
        cnt[r] = c;
    }
}

__global__ void k_fill_lower(const int64_t *ptr, const int32_t *idx, int64_t nr, const int64_t *optr,
                             int32_t *oidx) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = optr[r];
        for (int64_t j = ptr[r]; j < ptr[r + 1]; j++)
            if (idx[j] < r) oidx[o++] = idx[j];
    }
}

// Jones-Plassmann rounds with priority "lower index first": identical to the sequential
// greedy colouring in aggregate index order (each colour is the smallest one unused by the
// lower-index conflicting subdomains).
__global__ void k_jp_round(const int64_t *lptr, const int32_t *lidx, int64_t nagg, int32_t *colour,
                           int *uncoloured, int *err) {
    int local = 0;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nagg;
         a += (int64_t)gridDim.x * blockDim.x) {
        if (colour[a] >= 0) continue;
        bool ready = true;
        uint32_t used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t j = lptr[a]; j < lptr[a + 1]; j++) {
            int32_t c = colour[lidx[j]];
            if (c < 0) {
                ready = false;
                break;
            }
            if (c < 256) used[c >> 5] |= 1u << (c & 31);
        }
        if (!ready) {
            local++;
            continue;
        }
        int c = 0;
        while (c < 256 && (used[c >> 5] >> (c & 31)) & 1u) c++;
        if (c >= 256) flag_error(err, LSAMG_LIMIT, (int)a);
        colour[a] = c;
    }
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(uncoloured, local);
}

__global__ void k_colour_keys(const int32_t *colour, int64_t nagg, uint64_t *keys) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nagg;
         a += (int64_t)gridDim.x * blockDim.x)
        keys[a] = ((uint64_t)colour[a] << 32) | (uint64_t)a;
}

__global__ void k_colour_unpack(const uint64_t *keys, int64_t nagg, int32_t *colagg) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nagg;
         a += (int64_t)gridDim.x * blockDim.x)
        colagg[a] = (int32_t)(keys[a] & 0xffffffffull);
}

// ---------------------------------------------------------------- structural nnz
// (level 0: the row lengths of the DOF adjacency, computed by csr_union in
// structural_nnz_level0)
// coarse: nnz = sum_a k_a * sum_{b in nb(a)} k_b
__global__ void k_block_nnz(const int64_t *nptr, const int32_t *nidx, int64_t nagg,
                            const int32_t *k, int64_t *out) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nagg;
         a += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int64_t j = nptr[a]; j < nptr[a + 1]; j++) s += k[nidx[j]];
        out[a] = s * (int64_t)k[a];
    }
}

}  // namespace

void check_err(const int *err, cudaStream_t s, const char *where) {
    int h[2];
    CK(cudaMemcpyAsync(h, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[0] != 0) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s: device check failed (code %d, item %d)", where, h[0], h[1]);
        fail(h[0], buf);
    }
}

void check_input(const Level &L, int *err, cudaStream_t s) {
    if (L.ne > 0) {
        k_check_input<<<grid_for(L.ne * 32), TPB, 0, s>>>(L.eptr.p, L.eidx.p, L.ne, L.n, err);
        CK_LAUNCH();
    }
    check_err(err, s, "element DOF map validation");
}

void build_dof_elem(Level &L, int *err, cudaStream_t s) {
    csr_transpose(L.eptr.p, L.eidx.p, L.ne, L.nnz_e, L.n, L.dptr, L.didx, err, s);
}

void aggregate_level(Level &L, int passes, int *err, cudaStream_t s) {
    DBuf<int32_t> agg;
    int32_t nagg = mis2_pass(L, nullptr, L.n, agg, err, s);
    for (int p = 1; p < passes; p++) {
        DBuf<int32_t> agg2;
        int32_t n2 = mis2_pass(L, agg.p, nagg, agg2, err, s);
        k_compose<<<grid_for(L.n), TPB, 0, s>>>(agg.p, agg2.p, L.n);
        CK_LAUNCH();
        nagg = n2;
    }
    L.agg = std::move(agg);
    L.nagg = nagg;
    check_err(err, s, "aggregation");
}

// Relative size below which an assembled entry counts as zero in the A-closure.
constexpr double kACut = 1e-12;

__global__ void k_elem_len(const int64_t *eptr, int64_t ne, int32_t *len) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x)
        len[e] = (int32_t)(eptr[e + 1] - eptr[e]);
}

// Omega^A_i from Omega^G_i (OGptr / OGidx): the block A(omega_i, Omega^G_i) of every aggregate,
// assembled in chunks of at most 4 GB, decides which entries stay
static void a_closure(Level &L, const DBuf<int64_t> &OGptr, const DBuf<int32_t> &OGidx, DBuf<int64_t> &Optr,
                      DBuf<int32_t> &Oidx, int *err, cudaStream_t s) {
    const int64_t n = L.n, nagg = L.nagg, ne = L.ne;
    const int64_t nOG = read1(OGptr.p + nagg, s);
    DBuf<double> dg;
    dg.alloc(std::max<int64_t>(n, 1), s);
    if (n > 0) {
        k_assembled_diag<<<grid_for(n), TPB, 0, s>>>(L.dptr.p, L.didx.p, n, L.eptr.p, L.eidx.p, L.AT.p, L.aoff.p,
                                                     dg.p);
        CK_LAUNCH();
    }
    int32_t maxE = 1;
    if (ne > 0) {
        DBuf<int32_t> len;
        len.alloc(ne, s);
        k_elem_len<<<grid_for(ne), TPB, 0, s>>>(L.eptr.p, ne, len.p);
        CK_LAUNCH();
        maxE = std::max<int32_t>(1, max_i32(len.p, ne, s));
    }
    const size_t smem = 3 * (size_t)maxE * sizeof(int32_t);
    if (smem > 200 * 1024) fail(LSAMG_LIMIT, "element map longer than the A-closure staging (17,066)");
    CK(cudaFuncSetAttribute(k_assemble_rect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DBuf<int32_t> keep;
    keep.alloc(std::max<int64_t>(nOG, 1), s);
    auto og = to_host(OGptr.p, nagg + 1, s);
    auto wp = to_host(L.wptr.p, nagg + 1, s);
    const int64_t budget = (int64_t)4 << 30;
    for (int64_t a0 = 0; a0 < nagg;) {
        std::vector<int32_t> ids;
        std::vector<int64_t> boff(1, 0);
        int64_t a1 = a0;
        while (a1 < nagg) {
            const int64_t by = (og[a1 + 1] - og[a1]) * (wp[a1 + 1] - wp[a1]) * 8;
            if (a1 > a0 && (boff.back() * 8 + by) > budget) break;
            ids.push_back((int32_t)a1);
            boff.push_back(boff.back() + by / 8);
            a1++;
        }
        const int64_t na = (int64_t)ids.size();
        DBuf<int32_t> dids;
        DBuf<int64_t> dboff;
        upload(dids, ids, s);
        upload(dboff, boff, s);
        DBuf<double> B;
        B.alloc(std::max<int64_t>(boff.back(), 1), s);
        B.zero(s);
        const int es = (int)std::max<int64_t>(1, std::min<int64_t>((148 * 4 + na - 1) / na, 16));
        k_assemble_rect<<<dim3((unsigned)na, (unsigned)es), 256, smem, s>>>(
            dids.p, na, L.aeptr.p, L.aeidx.p, L.eptr.p, L.eidx.p, L.AT.p, L.aoff.p, OGptr.p, OGidx.p, L.agg.p,
            L.posw.p, B.p, dboff.p, maxE, es);
        CK_LAUNCH();
        k_a_keep<<<(unsigned)na, 256, 0, s>>>(dids.p, na, OGptr.p, OGidx.p, L.agg.p, L.wptr.p, L.widx.p, dg.p, B.p,
                                             dboff.p, kACut, keep.p);
        CK_LAUNCH();
        a0 = a1;
    }
    DBuf<int64_t> cnt;
    cnt.alloc(std::max<int64_t>(nagg, 1), s);
    if (nagg > 0) {
        k_keep_count<<<grid_for(nagg), TPB, 0, s>>>(OGptr.p, keep.p, nagg, cnt.p);
        CK_LAUNCH();
    }
    Optr.alloc(nagg + 1, s);
    exclusive_scan_i64(cnt.p, Optr.p, nagg, s);
    const int64_t tot = read1(Optr.p + nagg, s);
    Oidx.alloc(std::max<int64_t>(tot, 1), s);
    if (nagg > 0) {
        k_keep_fill<<<grid_for(nagg * 32), TPB, 0, s>>>(OGptr.p, OGidx.p, keep.p, nagg, Optr.p, Oidx.p);
        CK_LAUNCH();
    }
    trace("  A-closure: %lld of %lld G-row closure entries kept", (long long)tot, (long long)nOG);
}

void closure_level(Level &L, double tau_c, int closure, int *err, cudaStream_t s) {
    const int64_t ne = L.ne, n = L.n, nagg = L.nagg;
    // eagg(T): sorted distinct aggregates met by N(T); mult(T) = |eagg(T)|   (eq. 2.5)
    {
        DBuf<int32_t> vals;
        DBuf<int64_t> ucnt;
        vals.alloc(std::max<int64_t>(L.nnz_e, 1), s);
        ucnt.alloc(ne, s);
        k_gather_agg<<<grid_for(L.nnz_e), TPB, 0, s>>>(L.eidx.p, L.nnz_e, L.agg.p, vals.p);
        CK_LAUNCH();
        seg_sort(vals.p, L.eptr.p, ne, ucnt.p, err, s);
        L.eaptr.alloc(ne + 1, s);
        exclusive_scan_i64(ucnt.p, L.eaptr.p, ne, s);
        int64_t tot = read1(L.eaptr.p + ne, s);
        L.eaidx.alloc(std::max<int64_t>(tot, 1), s);
        seg_unique_compact(vals.p, L.eptr.p, ne, L.eaptr.p, L.eaidx.p, s);
        L.mult.alloc(ne, s);
        k_copy_i64_to_i32<<<grid_for(ne), TPB, 0, s>>>(ucnt.p, L.mult.p, ne);
        CK_LAUNCH();
        L.maxmult = max_i32(L.mult.p, ne, s);
        L.tau = tau_c * (double)L.maxmult;  // eq. 2.10: tau_cut = c max_j mult(j)
        // aggregate -> elements touching omega_i (rows of eq. 2.3)
        csr_transpose(L.eaptr.p, L.eaidx.p, ne, tot, nagg, L.aeptr, L.aeidx, err, s);
    }
    trace("  eagg/mult done (tau %.3f)", L.tau);
    // omega_i lists and ranks
    {
        DBuf<int64_t> ip;
        ip.alloc(n + 1, s);
        std::vector<int64_t> h(n + 1);
        for (int64_t i = 0; i <= n; i++) h[i] = i;
        CK(cudaMemcpyAsync(ip.p, h.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        csr_transpose(ip.p, L.agg.p, n, n, nagg, L.wptr, L.widx, err, s);
        L.posw.alloc(n, s);
        if (nagg > 0) {
            k_posw<<<(unsigned)nagg, 256, 0, s>>>(L.wptr.p, L.widx.p, nagg, L.posw.p);
            CK_LAUNCH();
        }
    }
    // G-row closure: Omega_i = union of N(T) over elements touching omega_i (eq. 2.4 = element
    // closure, Thm 5.6), built as per DOF q the aggregates whose overlap contains q, then
    // transposed.  A-closure: Omega_i^A per aggregate, and its transpose.
    {
        DBuf<int64_t> qptr;
        DBuf<int32_t> qidx;
        csr_union(L.dptr.p, L.didx.p, n, L.eaptr.p, L.eaidx.p, qptr, qidx, err, s);
        int64_t tot = read1(qptr.p + n, s);
        csr_transpose(qptr.p, qidx.p, n, tot, nagg, L.Optr, L.Oidx, err, s);
        if (closure != 0) {
            DBuf<int64_t> gptr = std::move(L.Optr);
            DBuf<int32_t> gidx = std::move(L.Oidx);
            a_closure(L, gptr, gidx, L.Optr, L.Oidx, err, s);
            tot = read1(L.Optr.p + nagg, s);
            csr_transpose(L.Optr.p, L.Oidx.p, nagg, tot, n, qptr, qidx, err, s);
        }
        int64_t nO = read1(L.Optr.p + nagg, s);
        trace("  Omega total %lld", (long long)nO);
        L.Olpos.alloc(std::max<int64_t>(nO, 1), s);
        if (nagg > 0) {
            k_olpos<<<(unsigned)nagg, 256, 0, s>>>(L.Optr.p, L.Oidx.p, L.wptr.p, L.widx.p, L.agg.p,
                                                   L.posw.p, nagg, L.Olpos.p);
            CK_LAUNCH();
        }
        // elements meeting Omega_i: per element the union over its DOFs, then transpose
        DBuf<int64_t> eoptr;
        DBuf<int32_t> eoidx;
        csr_union(L.eptr.p, L.eidx.p, ne, qptr.p, qidx.p, eoptr, eoidx, err, s);
        int64_t eot = read1(eoptr.p + ne, s);
        csr_transpose(eoptr.p, eoidx.p, ne, eot, nagg, L.oeptr, L.oeidx, err, s);
        int64_t nent = eot;
        DBuf<int64_t> cnt;
        cnt.alloc(std::max<int64_t>(nent, 1), s);
        if (nent > 0) {
            k_oeloc_count<<<grid_for(nent), TPB, 0, s>>>(L.oeptr.p, L.oeidx.p, nent, L.eptr.p, cnt.p);
            CK_LAUNCH();
        }
        L.oelocoff.alloc(nent + 1, s);
        exclusive_scan_i64(cnt.p, L.oelocoff.p, nent, s);
        int64_t tl = read1(L.oelocoff.p + nent, s);
        L.oeloc.alloc(std::max<int64_t>(tl, 1), s);
        if (nagg > 0) {
            k_oeloc_fill<<<(unsigned)nagg, 256, 0, s>>>(L.oeptr.p, L.oeidx.p, nagg, L.eptr.p,
                                                        L.eidx.p, L.Optr.p, L.Oidx.p,
                                                        L.oelocoff.p, L.oeloc.p);
            CK_LAUNCH();
        }
        trace("  element lists done");
        // colouring needs the conflict graph: a ~ b iff some element meets both overlaps
        DBuf<int64_t> aptr;
        DBuf<int32_t> aidx;
        csr_union(L.oeptr.p, L.oeidx.p, nagg, eoptr.p, eoidx.p, aptr, aidx, err, s);
        // keep lower-index neighbours only
        DBuf<int32_t> lc;
        DBuf<int64_t> lptr;
        lc.alloc(std::max<int64_t>(nagg, 1), s);
        if (nagg > 0) {
            k_remove_self<<<grid_for(nagg), TPB, 0, s>>>(aptr.p, aidx.p, nagg, lc.p);
            CK_LAUNCH();
        }
        lptr.alloc(nagg + 1, s);
        exclusive_scan_i32(lc.p, lptr.p, nagg, s);
        int64_t lt = read1(lptr.p + nagg, s);
        DBuf<int32_t> lidx;
        lidx.alloc(std::max<int64_t>(lt, 1), s);
        if (nagg > 0) {
            k_fill_lower<<<grid_for(nagg), TPB, 0, s>>>(aptr.p, aidx.p, nagg, lptr.p, lidx.p);
            CK_LAUNCH();
        }
        L.colour.alloc(std::max<int64_t>(nagg, 1), s);
        CK(cudaMemsetAsync(L.colour.p, 0xff, std::max<int64_t>(nagg, 1) * sizeof(int32_t), s));
        DBuf<int> cnt2;
        cnt2.alloc(1, s);
        for (int round = 0; nagg > 0; round++) {
            if (round > nagg + 1) fail(LSAMG_DEVICE_TIMEOUT, "colouring did not terminate");
            cnt2.zero(s);
            k_jp_round<<<grid_for(nagg), TPB, 0, s>>>(lptr.p, lidx.p, nagg, L.colour.p, cnt2.p, err);
            CK_LAUNCH();
            if (read1(cnt2.p, s) == 0) break;
        }
    }
    L.h_nw.resize(nagg);
    L.h_nO.resize(nagg);
    {
        auto wp = to_host(L.wptr.p, nagg + 1, s);
        auto op = to_host(L.Optr.p, nagg + 1, s);
        for (int64_t a = 0; a < nagg; a++) {
            L.h_nw[a] = (int32_t)(wp[a + 1] - wp[a]);
            L.h_nO[a] = (int32_t)(op[a + 1] - op[a]);
        }
    }
    check_err(err, s, "closure");
}

void colour_level(Level &L, int *err, cudaStream_t s) {
    const int64_t nagg = L.nagg;
    DBuf<uint64_t> keys;
    keys.alloc(std::max<int64_t>(nagg, 1), s);
    if (nagg > 0) {
        k_colour_keys<<<grid_for(nagg), TPB, 0, s>>>(L.colour.p, nagg, keys.p);
        CK_LAUNCH();
    }
    sort_u64(keys.p, nagg, s);
    L.colagg.alloc(std::max<int64_t>(nagg, 1), s);
    if (nagg > 0) {
        k_colour_unpack<<<grid_for(nagg), TPB, 0, s>>>(keys.p, nagg, L.colagg.p);
        CK_LAUNCH();
    }
    auto col = to_host(L.colour.p, nagg, s);
    int32_t nc = 0;
    for (auto c : col) nc = std::max(nc, c + 1);
    L.ncol = nc;
    L.colptr.assign(nc + 1, 0);
    for (auto c : col) L.colptr[c + 1]++;
    for (int c = 0; c < nc; c++) L.colptr[c + 1] += L.colptr[c];
    check_err(err, s, "colouring");
}

int64_t structural_nnz_level0(Level &L, int *err, cudaStream_t s) {
    // nnz = sum_p |U_{T contains p} N(T)|
    DBuf<int64_t> optr;
    DBuf<int32_t> oidx;
    csr_union(L.dptr.p, L.didx.p, L.n, L.eptr.p, L.eidx.p, optr, oidx, err, s);
    check_err(err, s, "structural nnz");
    return read1(optr.p + L.n, s);
}

int64_t structural_nnz_coarse(const Level &F, int *err, cudaStream_t s) {
    // coarse maps are unions of whole aggregate blocks: nnz = sum_a k_a sum_{b ~ a} k_b with
    // b ~ a iff some fine element touches both (nb(a) = union of eagg(T) over T touching a)
    DBuf<int64_t> nptr;
    DBuf<int32_t> nidx;
    csr_union(F.aeptr.p, F.aeidx.p, F.nagg, F.eaptr.p, F.eaidx.p, nptr, nidx, err, s);
    DBuf<int64_t> per;
    per.alloc(std::max<int64_t>(F.nagg, 1), s);
    if (F.nagg > 0) {
        k_block_nnz<<<grid_for(F.nagg), TPB, 0, s>>>(nptr.p, nidx.p, F.nagg, F.k.p, per.p);
        CK_LAUNCH();
    }
    check_err(err, s, "coarse structural nnz");
    return sum_i64(per.p, F.nagg, s);
}

}  // namespace lsamg
