// Blocked Householder tridiagonalisation of batches of symmetric matrices (lower storage), the
// reduction behind the local eigenproblems C y = mu y of eq. 2.9.
//
// Per panel of PNB columns (LAPACK's latrd/sytrd organisation):
//   * column j is brought up to date with the panel's earlier reflectors
//     (a -= V W(j,:)^T + W V(j,:)^T), its Householder reflector is formed (d_j, e_j, tau_j);
//   * y = A22 v, A22 the trailing matrix as it stood before the panel (split once per panel into
//     FP32 pairs, products in double-float arithmetic on the FP32 pipe), read once over its lower
//     triangle by 64 x 64 tiles spread over the whole GPU; every tile writes its two partial
//     products (the tile and its transpose) to its own slot and one CTA per matrix sums the
//     slots in a fixed order, so the result does not depend on scheduling;
//   * w = tau (y - V (W^T v) - W (V^T v)), w -= (tau/2)(w^T v) v;
//   * after the panel, A22 -= V W^T + W V^T over the lower triangle as one FP64 product of
//     K = 2 PNB on the tensor cores (ozaki.cuh).
// Conventions follow LAPACK's sytd2 (lower): H_j = I - tau_j v v^T with v = (1, A(j+2:n, j)),
// beta = -sign(alpha) ||(alpha, x)||, d_j = A(j, j), e_j = beta stored at A(j+1, j).
#include "dense.cuh"
#include "impl.cuh"
#include "ozaki.cuh"

namespace lsamg {
namespace {

constexpr int PNB = 32;   // reflectors per panel (the rank-2k update has K = 64)
constexpr int ST = 64;    // tile of the symmetric product

// The symmetric products y = A22 v carry two multiply-adds per stored entry, which would keep
// this GPU's FP64 pipe (1/64 of the FP32 rate) saturated below a third of the memory bandwidth.
// They run instead in double-float arithmetic on the FP32 pipe (common.cuh: df_split, df_mac,
// df_add): every entry of A22 and v is an FP32 pair holding its leading 48 bits, products keep
// their exact FP32 rounding error and the leading cross terms, sums are error-free.

__device__ double trd_block_sum(double v, double *red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; i++) r += red[i];
    return r;
}

// Per-matrix partial sums of one column step, one slot per row block of RB rows (fixed order
// of summation): [sigma, w^T v, s1[PNB], s2[PNB]].
constexpr int RB = 256;
constexpr int PSL = 2 + 2 * PNB;

// column j, rows j .. n-1 by blocks of RB: a -= V W(j,:)^T + W V(j,:)^T over the panel's earlier
// reflectors; partial sigma = sum a(r)^2 over rows r >= j+2
__global__ void __launch_bounds__(RB) k_trd_c1(double *base, const int64_t *off, const int32_t *ld, const int32_t *nn,
                                               int64_t count, int j, int j0, const double *VW, const int64_t *vwoff,
                                               double *part, const int64_t *partoff, double *dd,
                                               const int64_t *toff, double *alph) {
    __shared__ double red[32];
    __shared__ double wj[PNB], vj[PNB];
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b];
    const int r0 = j + blockIdx.x * RB;
    if (r0 >= n) return;
    const int jj = j - j0, L = ld[b];
    double *A = base + off[b];
    const double *V = VW + vwoff[b], *W = V + (int64_t)PNB * n;
    for (int q = threadIdx.x; q < jj; q += blockDim.x) {
        wj[q] = W[j + (int64_t)q * n];
        vj[q] = V[j + (int64_t)q * n];
    }
    __syncthreads();
    const int r = r0 + threadIdx.x;
    double sq = 0.0;
    if (r < n) {
        double a = A[r + (int64_t)j * L];
#pragma unroll 8
        for (int q = 0; q < jj; q++) a -= V[r + (int64_t)q * n] * wj[q] + W[r + (int64_t)q * n] * vj[q];
        A[r + (int64_t)j * L] = a;
        if (r >= j + 2) sq = a * a;
        if (r == j) dd[toff[b] + j] = a;          // d_j
        if (r == j + 1) alph[b] = a;              // alpha of the reflector
    }
    sq = trd_block_sum(sq, red);
    if (threadIdx.x == 0) part[partoff[b] + (int64_t)blockIdx.x * PSL] = sq;
}

// rows j+1 .. n-1 by blocks: v (unit first entry, the scaled column below it) into A, vbuf, V and
// WV; partial s1 = W^T v and s2 = V^T v over the panel's earlier columns
__global__ void __launch_bounds__(RB) k_trd_c3(double *base, const int64_t *off, const int32_t *ld, const int32_t *nn,
                                               int64_t count, int j, int j0, double *ee, double *tt,
                                               const int64_t *toff, const double *alph, double *VW, double *WV,
                                               const int64_t *vwoff, double *vbuf, double *part,
                                               const int64_t *partoff) {
    __shared__ double vs[RB];
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b];
    const int r0 = j + 1 + blockIdx.x * RB;
    if (r0 >= n) return;
    const int jj = j - j0, L = ld[b];
    double *A = base + off[b];
    double *V = VW + vwoff[b];
    const double *W = V + (int64_t)PNB * n;
    double *V2 = WV + vwoff[b] + (int64_t)PNB * n;
    // the Householder scalars of column j (LAPACK's larfg), from the row blocks' partial sums of
    // squares below the subdiagonal; every CTA of the matrix forms them, the first one stores them
    const int nrb = (n - j + RB - 1) / RB;
    double sig = 0.0;
    for (int q = 0; q < nrb; q++) sig += part[partoff[b] + (int64_t)q * PSL];
    const double alpha = alph[b];
    double t = 0.0, sc = 0.0, ej = alpha;
    if (sig != 0.0) {
        const double beta = -copysign(sqrt(alpha * alpha + sig), alpha);
        t = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
        ej = beta;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ee[toff[b] + j] = ej;
        tt[toff[b] + j] = t;
    }
    const int r = r0 + threadIdx.x;
    double v = 0.0;
    if (r < n) {
        if (r == j + 1) {
            v = 1.0;
            A[r + (int64_t)j * L] = ej;
        } else if (t != 0.0) {
            v = A[r + (int64_t)j * L] * sc;
            A[r + (int64_t)j * L] = v;
        }
        vbuf[toff[b] + r] = v;
        V[r + (int64_t)jj * n] = v;
        V2[r + (int64_t)jj * n] = v;
    }
    vs[threadIdx.x] = v;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double *pp = part + partoff[b] + (int64_t)blockIdx.x * PSL;
    for (int q = warp; q < jj; q += nwarp) {
        double a1 = 0.0, a2 = 0.0;
#pragma unroll 8
        for (int i = lane; i < RB; i += 32) {
            const int rr = r0 + i;
            if (rr < n) {
                a1 += W[rr + (int64_t)q * n] * vs[i];
                a2 += V[rr + (int64_t)q * n] * vs[i];
            }
        }
        for (int o = 16; o; o >>= 1) {
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            pp[2 + q] = a1;
            pp[2 + PNB + q] = a2;
        }
    }
}

__device__ __forceinline__ void trd_tri(int64_t t, int &ti, int &tj) {
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);   // corrected below
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) i++;
    while ((int64_t)i * (i + 1) / 2 > t) i--;
    ti = i;
    tj = (int)(t - (int64_t)i * (i + 1) / 2);
}

// (hi, lo) FP32 pairs of the trailing lower triangle (rows and columns >= j0) of every matrix,
// column-major with leading dimension n: the operand of the panel's symmetric products (the
// trailing matrix is the same for all column steps of a panel, so it is split once per panel)
__global__ void __launch_bounds__(256) k_trd_pairs(const double *base, const int64_t *off, const int32_t *ld,
                                                   const int32_t *nn, int64_t count, int j0, float2 *F,
                                                   const int64_t *foff) {
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b], L = ld[b];
    const int c = j0 + (int)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= n) return;
    const double *A = base + off[b] + (int64_t)c * L;
    float2 *Fc = F + foff[b] + (int64_t)c * n;
    for (int r = c + (threadIdx.x & 31); r < n; r += 32) Fc[r] = df_split(A[r]);
}

// partial products of the 64 x 64 tiles of the trailing lower triangle with v: slot (ti, tj)
// holds A22(ti, tj) v(tj) (the diagonal tile as the full symmetric block), slot (tj, ti) holds
// A22(ti, tj)^T v(ti).  CTA c takes the contiguous tile range [c total / grid, (c + 1) total /
// grid) of the batch (tiles of a matrix in row order, matrices in batch order): the matrix of
// its first tile is found once (32-way search by one warp), then tiles and matrices advance
// incrementally, and the loads of the next tile are in flight while the current one is used.
__global__ void __launch_bounds__(256, 4) k_trd_symv(const float2 *F, const int64_t *foff, const int32_t *nn,
                                                     int64_t count, int j, const int64_t *toff, const double *vbuf,
                                                     float2 *P, const int64_t *poff, const int64_t *pre) {
    // rows padded to 68 pairs: the 16 threads of a half-warp read 16 distinct 8-byte banks both
    // along rows and along columns
    __shared__ float2 tile[ST][ST + 4];
    __shared__ float2 vr[ST], vc[ST];
    __shared__ int s_b;
    constexpr int PER = ST * ST / 256;
    const int64_t total = pre[count];
    const int64_t w0 = total * blockIdx.x / gridDim.x, w1 = total * (blockIdx.x + 1) / gridDim.x;
    if (w0 >= w1) return;
    if (threadIdx.x < 32) {
        // largest b with pre[b] <= w0 (then pre[b + 1] > w0: the matrix holding tile w0)
        const int lane = threadIdx.x;
        int64_t lo = 0, hi = count - 1;
        while (hi > lo) {
            const int64_t step = (hi - lo + 32) / 32;
            const int64_t cand = lo + lane * step;
            const unsigned ok = __ballot_sync(0xffffffffu, cand <= hi && pre[cand] <= w0);
            lo += (int64_t)(31 - __clz((int)ok)) * step;
            hi = min(hi, lo + step - 1);
        }
        if (lane == 0) s_b = (int)lo;
    }
    __syncthreads();
    const int lane4 = threadIdx.x & 3, idx = threadIdx.x >> 2;   // 64 groups of 4 threads
    // state of the tile being loaded
    int b = s_b, ti, tj;
    trd_tri(w0 - pre[b], ti, tj);
    int L = nn[b], m = L - j - 1, T = (m + ST - 1) / ST;
    const float2 *A22 = F + foff[b] + (j + 1) + (int64_t)(j + 1) * L;
    const double *v = vbuf + toff[b] + (j + 1);
    float2 a[PER];
    double vx = 0.0;
    auto issue = [&]() {
        const int r0 = ti * ST, c0 = tj * ST;
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int t = threadIdx.x + 256 * u;
            const int rr = t % ST, cc = t / ST;
            const int gr = r0 + rr, gc = c0 + cc;
            a[u] = (gr < m && gc < m && gr >= gc) ? A22[gr + (int64_t)gc * L] : make_float2(0.f, 0.f);
        }
        if (threadIdx.x < 2 * ST) {
            const int k = (threadIdx.x < ST ? r0 : c0 - ST) + threadIdx.x;
            vx = k < m ? v[k] : 0.0;
        }
    };
    issue();
    for (int64_t w = w0; w < w1; w++) {
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int t = threadIdx.x + 256 * u;
            tile[t % ST][t / ST] = a[u];
        }
        if (threadIdx.x < ST) vr[threadIdx.x] = df_split(vx);
        else if (threadIdx.x < 2 * ST) vc[threadIdx.x - ST] = df_split(vx);
        __syncthreads();
        const int cti = ti, ctj = tj, cT = T;
        const int64_t cpo = poff[b];
        // next tile: advance within the matrix, else to the next non-empty matrix
        if (w + 1 < w1) {
            if (++tj > ti) {
                tj = 0;
                if (++ti >= T) {
                    do b++; while (pre[b + 1] <= w + 1);
                    ti = 0;
                    L = nn[b];
                    m = L - j - 1;
                    T = (m + ST - 1) / ST;
                    A22 = F + foff[b] + (j + 1) + (int64_t)(j + 1) * L;
                    v = vbuf + toff[b] + (j + 1);
                }
            }
            issue();
        }
        const bool diag = (cti == ctj);
        // row part: row idx, 16 columns per thread of the group
        float rh = 0.f, rl = 0.f, ch = 0.f, cl = 0.f;
        for (int c = lane4; c < ST; c += 4) {
            float2 x = tile[idx][c];
            if (diag && c > idx) x = tile[c][idx];       // upper half of the diagonal tile by symmetry
            df_mac(rh, rl, x, vc[c]);
        }
        if (!diag)
            for (int r = lane4; r < ST; r += 4) df_mac(ch, cl, tile[r][idx], vr[r]);
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            df_add(rh, rl, __shfl_xor_sync(0xffffffffu, rh, o), __shfl_xor_sync(0xffffffffu, rl, o));
            df_add(ch, cl, __shfl_xor_sync(0xffffffffu, ch, o), __shfl_xor_sync(0xffffffffu, cl, o));
        }
        if (lane4 == 0) {
            float2 *Pb = P + cpo;
            Pb[((int64_t)cti * cT + ctj) * ST + idx] = make_float2(rh, rl);
            if (!diag) Pb[((int64_t)ctj * cT + cti) * ST + idx] = make_float2(ch, cl);
        }
        __syncthreads();
    }
}

// w of column j, rows j+1 .. n-1 by blocks: y = the product slots summed in fixed order, then
// w' = tau (y - V s1 - W s2) into ybuf, partial w'^T v
__global__ void __launch_bounds__(RB) k_trd_w2(const int32_t *nn, int64_t count, int j, int j0, const double *tt,
                                               const int64_t *toff, const double *vbuf, const float2 *P,
                                               const int64_t *poff, double *VW, double *WV, const int64_t *vwoff,
                                               double *ybuf, double *part, const int64_t *partoff) {
    __shared__ double red[32];
    __shared__ double s1[PNB], s2[PNB];
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b];
    const int m = n - j - 1;
    const int r0 = j + 1 + blockIdx.x * RB;
    if (m <= 0 || r0 >= n) return;
    const int jj = j - j0;
    double *V = VW + vwoff[b], *W = V + (int64_t)PNB * n;
    double *W2 = WV + vwoff[b];
    const double tau = tt[toff[b] + j];
    const int r = r0 + threadIdx.x;
    if (tau == 0.0) {
        if (r < n) {
            W[r + (int64_t)jj * n] = 0.0;
            W2[r + (int64_t)jj * n] = 0.0;
        }
        return;
    }
    const int nrb = (m + RB - 1) / RB;
    const double *pb = part + partoff[b];
    for (int q = threadIdx.x; q < jj; q += blockDim.x) {
        double a1 = 0.0, a2 = 0.0;
        for (int k = 0; k < nrb; k++) {
            a1 += pb[(int64_t)k * PSL + 2 + q];
            a2 += pb[(int64_t)k * PSL + 2 + PNB + q];
        }
        s1[q] = a1;
        s2[q] = a2;
    }
    __syncthreads();
    const double *v = vbuf + toff[b];
    const int T = (m + ST - 1) / ST;
    const float2 *Pb = P + poff[b];
    double wv = 0.0;
    if (r < n) {
        const int i = r - j - 1, ti = i / ST, rr = i % ST;
        float yh = 0.f, yl = 0.f;   // the double-float slots, summed error-free
#pragma unroll 8
        for (int t = 0; t < T; t++) {
            const float2 q = Pb[((int64_t)ti * T + t) * ST + rr];
            df_add(yh, yl, q.x, q.y);
        }
        double y = (double)yh + (double)yl;
#pragma unroll 8
        for (int q = 0; q < jj; q++) y -= V[r + (int64_t)q * n] * s1[q] + W[r + (int64_t)q * n] * s2[q];
        y *= tau;
        ybuf[toff[b] + r] = y;
        wv = y * v[r];
    }
    wv = trd_block_sum(wv, red);
    if (threadIdx.x == 0) part[partoff[b] + (int64_t)blockIdx.x * PSL + 1] = wv;
}

// w = w' - (tau/2)(w'^T v) v into W and WV
__global__ void __launch_bounds__(RB) k_trd_w3(const int32_t *nn, int64_t count, int j, int j0, const double *tt,
                                               const int64_t *toff, const double *vbuf, double *VW, double *WV,
                                               const int64_t *vwoff, const double *ybuf, const double *part,
                                               const int64_t *partoff) {
    const int64_t b = blockIdx.y;
    if (b >= count) return;
    const int n = nn[b];
    const int m = n - j - 1;
    const int r0 = j + 1 + blockIdx.x * RB;
    if (m <= 0 || r0 >= n) return;
    const double tau = tt[toff[b] + j];
    if (tau == 0.0) return;
    const int jj = j - j0;
    const int nrb = (m + RB - 1) / RB;
    double wv = 0.0;
    for (int k = 0; k < nrb; k++) wv += part[partoff[b] + (int64_t)k * PSL + 1];
    const double alpha = -0.5 * tau * wv;
    const int r = r0 + threadIdx.x;
    if (r < n) {
        const double w = ybuf[toff[b] + r] + alpha * vbuf[toff[b] + r];
        VW[vwoff[b] + (int64_t)PNB * n + r + (int64_t)jj * n] = w;
        WV[vwoff[b] + r + (int64_t)jj * n] = w;
    }
}

}  // namespace

void sytd2_batched(double *base, const MatBatch &Ab, double *d, double *e, double *tau, const int64_t *toff,
                   cudaStream_t s) {
    if (Ab.count == 0 || Ab.maxn == 0) return;
    const int64_t cnt = Ab.count;
    std::vector<int64_t> vwoff(cnt + 1, 0), poff(cnt + 1, 0), fo(cnt + 1, 0);
    for (int64_t b = 0; b < cnt; b++) {
        const int64_t n = Ab.h_n[b];
        vwoff[b + 1] = vwoff[b] + 2 * PNB * n;
        fo[b + 1] = fo[b] + n * n;
        const int64_t T = cdiv(std::max<int64_t>(n - 1, 1), ST);
        poff[b + 1] = poff[b] + T * T * ST;
    }
    const int64_t tn = read1(toff + cnt, s);
    std::vector<int64_t> partoff(cnt + 1, 0);
    for (int64_t b = 0; b < cnt; b++) partoff[b + 1] = partoff[b] + cdiv(Ab.h_n[b], RB) * PSL;
    DBuf<double> VW, WV, vbuf, ybuf, part, alph;
    DBuf<float2> P;
    DBuf<int64_t> dvw, dpo, dpa, pre, dfo;
    DBuf<float2> F;
    F.alloc(std::max<int64_t>(fo[cnt], 1), s);
    upload(dfo, std::vector<int64_t>(fo.begin(), fo.end() - 1), s);
    VW.alloc(std::max<int64_t>(vwoff[cnt], 1), s);
    WV.alloc(std::max<int64_t>(vwoff[cnt], 1), s);
    P.alloc(std::max<int64_t>(poff[cnt], 1), s);
    vbuf.alloc(std::max<int64_t>(tn, 1), s);
    ybuf.alloc(std::max<int64_t>(tn, 1), s);
    part.alloc(std::max<int64_t>(partoff[cnt], 1), s);
    alph.alloc(cnt, s);
    // tile schedule of the symmetric products for every column step: tiles of the trailing lower
    // triangle per matrix and their exclusive prefix over the batch (a matrix whose reflector turns
    // out to be the identity is multiplied all the same; its w is zeroed)
    {
        std::vector<int64_t> h((int64_t)Ab.maxn * (cnt + 1), 0);
        for (int j = 0; j < Ab.maxn; j++) {
            int64_t *pj = h.data() + (int64_t)j * (cnt + 1), acc = 0;
            for (int64_t b = 0; b < cnt; b++) {
                pj[b] = acc;
                const int64_t m = Ab.h_n[b] - j - 1;
                if (m > 0) {
                    const int64_t T = cdiv(m, ST);
                    acc += T * (T + 1) / 2;
                }
            }
            pj[cnt] = acc;
        }
        upload(pre, h, s);
    }
    upload(dvw, std::vector<int64_t>(vwoff.begin(), vwoff.end() - 1), s);
    upload(dpo, std::vector<int64_t>(poff.begin(), poff.end() - 1), s);
    upload(dpa, std::vector<int64_t>(partoff.begin(), partoff.end() - 1), s);
    DBuf<int> err;
    err.alloc(2, s);
    err.zero(s);
    oz::Workspace ws;
    const unsigned symv_grid = 148 * 4;   // one resident wave (4 CTAs of 256 threads per SM)
    for (int j0 = 0; j0 < Ab.maxn; j0 += PNB) {
        const int j1 = std::min(Ab.maxn, j0 + PNB);
        {
            KTime kt(KC_SYTD2, s);
            const dim3 gp((unsigned)cdiv(Ab.maxn - j0, 8), (unsigned)cnt);
            k_trd_pairs<<<gp, 256, 0, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, cnt, j0, F.p, dfo.p);
            CK_LAUNCH();
        }
        for (int j = j0; j < j1; j++) {
            // the FP64 column steps (the panel's rank-2k update is a tensor-core product): the
            // trailing lower triangle is read once per column by the symmetric product
            double by = 0.0;
            for (auto v : Ab.h_n) {
                const double m = v - j - 1;
                if (m > 0) by += 4.0 * m * (m + 1);
            }
            const dim3 g3((unsigned)cdiv(std::max(Ab.maxn - j - 1, 1), RB), (unsigned)cnt);
            {
                KTime kt(KC_SYTD2, s);
                const dim3 g1((unsigned)cdiv(Ab.maxn - j, RB), (unsigned)cnt);
                k_trd_c1<<<g1, RB, 0, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, cnt, j, j0, VW.p, dvw.p, part.p, dpa.p, d,
                                           toff, alph.p);
                CK_LAUNCH();
                if (j >= Ab.maxn - 1) break;
                k_trd_c3<<<g3, RB, 0, s>>>(base, Ab.off.p, Ab.ld.p, Ab.n.p, cnt, j, j0, e, tau, toff, alph.p, VW.p,
                                           WV.p, dvw.p, vbuf.p, part.p, dpa.p);
                CK_LAUNCH();
            }
            {
                KTime ks(KC_SYMV, s, 0.0, by);
                k_trd_symv<<<symv_grid, 256, 0, s>>>(F.p, dfo.p, Ab.n.p, cnt, j, toff, vbuf.p, P.p, dpo.p,
                                                     pre.p + (int64_t)j * (cnt + 1));
                CK_LAUNCH();
            }
            {
                KTime kt(KC_SYTD2, s);
                k_trd_w2<<<g3, RB, 0, s>>>(Ab.n.p, cnt, j, j0, tau, toff, vbuf.p, P.p, dpo.p, VW.p, WV.p, dvw.p,
                                           ybuf.p, part.p, dpa.p);
                CK_LAUNCH();
                k_trd_w3<<<g3, RB, 0, s>>>(Ab.n.p, cnt, j, j0, tau, toff, vbuf.p, VW.p, WV.p, dvw.p, ybuf.p, part.p,
                                           dpa.p);
                CK_LAUNCH();
            }
        }
        // trailing update A22 -= V W^T + W V^T over rows / columns >= j1, K = 2 PNB
        std::vector<oz::SplitJob> sa, sb;
        std::vector<oz::GemmJob> gj;
        int64_t h = 0, ex = 0;
        for (int64_t b = 0; b < cnt; b++) {
            const int64_t n = Ab.h_n[b];
            const int m = (int)(n - j1);
            if (m <= 0) continue;
            const int64_t L = Ab.h_ld[b];
            sa.push_back(oz::SplitJob{vwoff[b] + j1, 1, n, h, ex, m, 2 * PNB});
            const int64_t ha = h, ea = ex;
            h += oz::slice_halves(m, 2 * PNB);
            ex += oz::exp_ints(m);
            sb.push_back(oz::SplitJob{vwoff[b] + j1, 1, n, h, ex, m, 2 * PNB});
            const int64_t hb = h, eb = ex;
            h += oz::slice_halves(m, 2 * PNB);
            ex += oz::exp_ints(m);
            gj.push_back(oz::GemmJob{ha, hb, ea, eb, Ab.h_off[b] + j1 + (int64_t)j1 * L, 1, L, m, m, 2 * PNB, 1, 0, 0});
        }
        if (gj.empty()) continue;
        ws.reserve(h, ex, s);
        oz::split(VW.p, sa, ws.sl.p, ws.ex.p, s);
        oz::split(WV.p, sb, ws.sl.p, ws.ex.p, s);
        oz::gemm(ws.sl.p, ws.ex.p, base, gj, -1.0, 1.0, err.p, s);
    }
    check_err(err.p, s, "tridiagonal reduction");
}

}  // namespace lsamg
