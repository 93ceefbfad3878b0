// FP64 products on FP16 tensor cores by exact splitting (see ozaki.cuh for the scheme).
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "ozaki.cuh"

namespace lsamg {
namespace oz {
namespace {

constexpr int NST = 3;                         // staging ring depth
constexpr int STAGE_BYTES = 2 * NS * BLK * 2;  // A and B slices of one K chunk
constexpr int GEMM_SMEM = NST * STAGE_BYTES + 64;

__device__ __forceinline__ int dcdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ int swz(int r, int k) {  // halves offset inside a 64 x 32 block
    return r * TK + ((((k >> 3) ^ (r >> 1)) & 3) << 3) + (k & 7);
}

// job index of CTA `blk` from an exclusive prefix of per-job CTA counts
__device__ __forceinline__ int find_job(const int64_t *pre, int njobs, int64_t blk) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------------- split
__global__ void __launch_bounds__(256) k_split(const double *src, const SplitJob *jobs, const int64_t *pre,
                                               int njobs, __half *dst, int32_t *exps) {
    __shared__ double rmax[TM][5];
    __shared__ int rexp[TM];
    const int j = find_job(pre, njobs, blockIdx.x);
    const SplitJob J = jobs[j];
    const int t = (int)(blockIdx.x - pre[j]);
    const int tiles = (int)stor_tiles(J.rows), nch = dcdiv(max(J.K, 1), TK);
    const int i0 = t * TM;
    const bool kfast = (J.ks == 1);
    const double *S = src + J.src_off;
    // row maxima over the whole K
    {
        double m = 0.0;
        int r, g, gs;
        if (kfast) { r = threadIdx.x >> 2; g = threadIdx.x & 3; gs = 4; }   // 4 threads per row
        else       { r = threadIdx.x & 63; g = threadIdx.x >> 6; gs = 4; }
        const int i = i0 + r;
        if (i < J.rows)
            for (int k = g; k < J.K; k += gs) m = fmax(m, fabs(S[(int64_t)i * J.rs + (int64_t)k * J.ks]));
        rmax[r][g] = m;
        __syncthreads();
        if (threadIdx.x < TM) {
            const double v = fmax(fmax(rmax[threadIdx.x][0], rmax[threadIdx.x][1]),
                                  fmax(rmax[threadIdx.x][2], rmax[threadIdx.x][3]));
            int e = 0;
            if (v > 0.0) frexp(v, &e);     // v < 2^e
            rexp[threadIdx.x] = e;
            exps[J.exp_off + i0 + threadIdx.x] = e;
        }
        __syncthreads();
    }
    // slices in integer arithmetic (the FP64 pipe is scarce): F = round(v 2^(55 - e_r)) exactly
    // from the bits of v (|F| < 2^55), then balanced base-256 digits a_p = round(F / 2^(48-8(p-1)))
    // with F -= a_p 2^(48-8(p-1)); the seven digits hold F exactly.  Two consecutive k per thread.
    const int64_t pstride = (int64_t)tiles * nch * BLK;
    for (int c = 0; c < nch; c++) {
        for (int idx = threadIdx.x; idx < BLK / 2; idx += blockDim.x) {
            int r, kk;
            if (kfast) { r = idx >> 4; kk = (idx & 15) * 2; } else { r = idx & 63; kk = (idx >> 6) * 2; }
            const int i = i0 + r;
            int dig[2][NS];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = c * TK + kk + h;
                double v = 0.0;
                if (i < J.rows && k < J.K) v = S[(int64_t)i * J.rs + (int64_t)k * J.ks];
                const uint64_t bits = (uint64_t)__double_as_longlong(v);
                int ef = (int)((bits >> 52) & 0x7ff);
                uint64_t mant = bits & ((1ull << 52) - 1);
                if (ef) mant |= 1ull << 52; else ef = 1;
                const int sh = ef - 1075 + 55 - rexp[r];      // v 2^(55 - e_r) = mant 2^sh
                int64_t F = 0;
                if (mant != 0 && sh > -64) {
                    if (sh >= 0) {
                        F = (int64_t)(mant << sh);
                    } else {
                        const int rs = -sh;
                        const uint64_t q = mant >> rs, rem = mant & ((1ull << rs) - 1), half = 1ull << (rs - 1);
                        F = (int64_t)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
                    }
                    if (bits >> 63) F = -F;
                }
#pragma unroll
                for (int p = 0; p < NS; p++) {
                    const int s2 = 48 - 8 * p;
                    const int64_t a = (s2 > 0) ? ((F + (1ll << (s2 - 1))) >> s2) : F;
                    F -= a << s2;
                    dig[h][p] = (int)a;
                }
            }
            const int o = swz(r, kk);
            __half2 *d = reinterpret_cast<__half2 *>(dst + J.dst_off + ((int64_t)t * nch + c) * BLK + o);
#pragma unroll
            for (int p = 0; p < NS; p++) {
                // |digit| <= 128: exact in FP32 through 1.5 * 2^23 and in FP16
                const float f0 = __int_as_float(0x4B400000 + dig[0][p]) - 12582912.0f;
                const float f1 = __int_as_float(0x4B400000 + dig[1][p]) - 12582912.0f;
                d[p * pstride / 2] = __floats2half2_rn(f0, f1);
            }
        }
    }
}

// ------------------------------------------------------------------------------- gemm
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of `bar`, giving up after `ns` nanoseconds
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > ns) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void tri_index(int64_t t, int &ti, int &tj) {
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) i++;
    while ((int64_t)i * (i + 1) / 2 > t) i--;
    ti = i;
    tj = (int)(t - (int64_t)i * (i + 1) / 2);
}

// v 2^e rounded to nearest (ties to even), negated if neg: integer instructions only while the
// result is a normal FP64 number (the FP64 pipe of this GPU is 1/64 of its FP32 rate)
__device__ __forceinline__ double i128_to_double(__int128 v, int e, bool neg) {
    if (v == 0) return 0.0;
    if (v < 0) { v = -v; neg = !neg; }
    const unsigned __int128 m = (unsigned __int128)v;
    const uint64_t h = (uint64_t)(m >> 64), l = (uint64_t)m;
    int p = h ? 127 - __clzll((long long)h) : 63 - __clzll((long long)l);   // top bit
    uint64_t mant;
    if (p <= 52) {
        mant = l << (52 - p);
    } else {
        const int sh = p - 52;
        const unsigned __int128 qq = m >> sh;
        const unsigned __int128 rem = m - (qq << sh);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        mant = (uint64_t)qq;
        if (rem > half || (rem == half && (mant & 1ull))) {
            mant++;
            if (mant == (1ull << 53)) { mant >>= 1; p++; }
        }
    }
    const int E = p + e;
    if (E > 1023 || E < -1022) {
        const double r = ldexp((double)mant, p - 52 + e);
        return neg ? -r : r;
    }
    const uint64_t bits = ((uint64_t)(E + 1023) << 52) | (mant & ((1ull << 52) - 1)) | (neg ? (1ull << 63) : 0ull);
    return __longlong_as_double((long long)bits);
}

// c + v 2^e for a 128-bit integer v (|v| < 2^100) rounded once: c's significand joins the integer
// sum at the common unit when both fit in 127 bits (otherwise one operand is below the other's
// rounding and an FP64 add of the rounded v is exact to the last bit's rounding)
__device__ __forceinline__ double i128_add_double(__int128 v, int e, double c) {
    const uint64_t cb = (uint64_t)__double_as_longlong(c);
    int ec = (int)((cb >> 52) & 0x7ff);
    if (ec == 0x7ff) return c + i128_to_double(v, e, false);          // inf / nan propagate
    int64_t mc = (int64_t)(cb & ((1ull << 52) - 1));
    if (ec) mc |= 1ll << 52; else ec = 1;
    if (mc == 0) return i128_to_double(v, e, false);
    if (v == 0) return c;
    if (cb >> 63) mc = -mc;
    const int E = ec - 1075;                                           // c = mc 2^E
    const unsigned __int128 av = (unsigned __int128)(v < 0 ? -v : v);
    const uint64_t vh = (uint64_t)(av >> 64), vl = (uint64_t)av;
    const int vb = vh ? 128 - __clzll((long long)vh) : 64 - __clzll((long long)vl);   // bits of |v|
    const int d = E - e;
    if (d >= 0 && d <= 126 - 53) return i128_to_double(v + ((__int128)mc << d), e, false);
    if (d < 0 && vb - d <= 126) return i128_to_double((v << (-d)) + (__int128)mc, E, false);
    return c + i128_to_double(v, e, false);
}

// epilogue of one output: C = beta C + alpha 2^e sum_d 2^-8(d-2) S_d (S_2..S_6 exact, tail = S_7 +
// S_8 / 256), the sum formed exactly as a 128-bit integer in units of 2^-48; with beta = 1 the old C
// joins the integer sum exactly and the result is rounded once.  FP64 instructions are scarce on
// this GPU: none in the common cases (alpha a power of two, beta 0 or 1).  Kept out of line: the
// product loop's registers are not needed here.
__device__ __forceinline__ double combine_out(__int128 v, int e, double alpha, double beta, double c);

__device__ __noinline__ void store_out(double *cp, int32_t s2, int32_t s3, int32_t s4, int32_t s5, int32_t s6,
                                       float tail, int e, double alpha, double beta) {
    const __int128 v = ((__int128)s2 << 48) + ((__int128)s3 << 40) + ((__int128)s4 << 32) + ((__int128)s5 << 24) +
                       ((__int128)s6 << 16) + (__int128)__float2ll_rn(tail * 256.0f);
    *cp = combine_out(v, e, alpha, beta, beta == 0.0 ? 0.0 : *cp);
}

// beta c + alpha v 2^e, rounded once when alpha is a power of two and beta is 0 or 1 (integer
// instructions only), else through FP64 arithmetic
__device__ __forceinline__ double combine_out(__int128 v, int e, double alpha, double beta, double c) {
    int e2;
    const double fr = frexp(fabs(alpha), &e2);
    if (fr != 0.5) {
        const double val = alpha * i128_to_double(v, e, false);
        return (beta == 0.0) ? val : (beta == 1.0) ? c + val : fma(beta, c, val);
    }
    if (alpha < 0.0) v = -v;
    e += e2 - 1;
    if (beta == 0.0) return i128_to_double(v, e, false);
    if (beta == 1.0) return i128_add_double(v, e, c);
    return fma(beta, c, i128_to_double(v, e, false));
}

// alpha and beta of a product, classified once on the host: the epilogue then runs on integer
// instructions only when alpha is a power of two (pow2, 2^(e2 - 1) with sign neg) and beta is 0
// or 1 (bmode 0 / 1; 2: general beta)
struct Scale {
    double alpha, beta;
    int32_t pow2, e2, neg, bmode;
};
inline Scale make_scale(double alpha, double beta) {
    Scale sc;
    sc.alpha = alpha;
    sc.beta = beta;
    int e2 = 0;
    const double fr = std::frexp(std::fabs(alpha), &e2);
    sc.pow2 = fr == 0.5 ? 1 : 0;
    sc.e2 = e2;
    sc.neg = alpha < 0.0 ? 1 : 0;
    sc.bmode = beta == 0.0 ? 0 : beta == 1.0 ? 1 : 2;
    return sc;
}
__device__ __forceinline__ double combine_scaled(__int128 v, int e, const Scale &sc, double c) {
    if (sc.pow2) {
        if (sc.neg) v = -v;
        e += sc.e2 - 1;
        if (sc.bmode == 0) return i128_to_double(v, e, false);
        if (sc.bmode == 1) return i128_add_double(v, e, c);
        return fma(sc.beta, c, i128_to_double(v, e, false));
    }
    const double val = sc.alpha * i128_to_double(v, e, false);
    return sc.bmode == 0 ? val : sc.bmode == 1 ? c + val : fma(sc.beta, c, val);
}

// v 2^e rounded to nearest (ties to even) for the 96-bit integer v = hi 2^32 + lo given as two
// 64-bit limbs (|hi| < 2^62).  Branch-free integer instructions while the result is a normal
// number, so that the compiler interleaves the conversions of a thread's outputs.
__device__ __forceinline__ double limbs_to_double(int64_t hi, int64_t lo, int e) {
    hi += lo >> 32;                                   // lo = (lo >> 32) 2^32 + low 32 bits
    uint32_t l = (uint32_t)lo;
    const bool neg = hi < 0;
    const uint64_t h = neg ? ~(uint64_t)hi + (l == 0u ? 1ull : 0ull) : (uint64_t)hi;   // |v| = h 2^32 + l
    l = neg ? 0u - l : l;
    // as a 96-bit number with its top limb nonzero when v != 0
    const bool hz = h == 0;
    const uint64_t H = hz ? (uint64_t)l : h;
    const uint32_t Lw = hz ? 0u : l;
    const int lz = __clzll((long long)H);             // 64 when v == 0 (result selected below)
    const int sh = lz & 63;
    const uint64_t top = (H << sh) | (sh ? (((uint64_t)Lw << 32) >> (64 - sh)) : 0ull);
    const uint32_t sticky = sh < 32 ? (Lw << sh) : 0u;   // bits of the low limb below the window
    uint64_t mant = top >> 11;
    const uint32_t rb = (uint32_t)(top & 0x7ffull);
    int E = 95 - lz + e - (hz ? 32 : 0);
    mant += (rb > 0x400u || (rb == 0x400u && (sticky != 0u || (mant & 1ull)))) ? 1ull : 0ull;
    const int ovf = (int)(mant >> 53);
    mant >>= ovf;
    E += ovf;
    if (H == 0) return 0.0;
    if (E > 1023 || E < -1022) {                       // overflow / subnormal range: FP64 scaling
        const double r = ldexp((double)mant, E - 52);
        return neg ? -r : r;
    }
    return __longlong_as_double(
        (long long)(((uint64_t)(E + 1023) << 52) | (mant & ((1ull << 52) - 1)) | (neg ? (1ull << 63) : 0ull)));
}

// 16 warps per CTA, warp tile 16 x 16 (one m16 tile, two n8 tiles): every slice's fragments
// of a 16-wide K step fit in registers (56), with per-diagonal exact int32 sums for the diagonals
// 2..6 and one FP32 sum for the two lowest-weight diagonals (S_7 + S_8 / 256, weights 2^-40 and
// 2^-48 of the leading one: with at most 256 K steps per product its rounding stays below
// 2^-75 of the leading unit times K, under the FP64 dot-product bound).
constexpr int GW = 16;               // warps per CTA
constexpr int GT = GW * 32;          // threads per CTA

// A product tile: its job, 64-row tiles of C and the operands' slice blocks
struct TileRef {
    int job, tm, tn, c0, nch;
    const __half *gA, *gB;
    int64_t pA, pB;
};

__device__ __forceinline__ TileRef decode_tile(const __half *sl, const GemmJob *jobs, const int64_t *pre, int njobs,
                                               int64_t t) {
    TileRef r;
    r.job = find_job(pre, njobs, t);
    const GemmJob &J = jobs[r.job];
    const int64_t local = t - pre[r.job];
    const int tilesN = dcdiv(J.N, TM);
    if (J.lower) tri_index(local, r.tm, r.tn);
    else { r.tm = (int)(local / tilesN); r.tn = (int)(local % tilesN); }
    const int ntot = dcdiv(max(J.ktot, 1), TK);          // chunks of the split operands
    r.c0 = J.k0 / TK;                                    // this pass's chunk range
    r.nch = dcdiv(max(J.K, 1), TK);
    r.gA = sl + J.a_off + (int64_t)r.tm * ntot * BLK;
    r.gB = sl + J.b_off + (int64_t)r.tn * ntot * BLK;
    r.pA = stor_tiles(J.M) * ntot * BLK;
    r.pB = stor_tiles(J.N) * ntot * BLK;
    return r;
}

// Persistent: CTA b takes tiles b, b + grid, ... (tiles of skipped jobs left out); thread 0 keeps
// the bulk-copy ring NST chunks ahead across tile boundaries, so the next tile's operands arrive
// while the current tile's epilogue runs.
__global__ void __launch_bounds__(GT, 1) k_gemm(const __half *sl, const int32_t *ex, double *C,
                                                const GemmJob *jobs, const int64_t *pre, int njobs, double alpha,
                                                double beta, int *err, const int32_t *skip) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NST * STAGE_BYTES);
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = pre[njobs];
    auto active = [&](int64_t t) {
        if (!skip) return true;
        return skip[jobs[find_job(pre, njobs, t)].skip_idx] < 0;
    };
    if (tid == 0) {
        for (int st = 0; st < NST; st++) mbar_init(&full[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_bad = 0;
    }
    __syncthreads();
    // producer state (thread 0, kept in shared memory to spare registers): the next (tile, chunk)
    // to stage and the number of chunks staged so far
    __shared__ int64_t s_ptile, s_issued;
    __shared__ int s_pchunk;
    __shared__ TileRef s_pref;
    auto prod_advance_tile = [&]() {
        int64_t t = s_ptile;
        while (t < total && !active(t)) t += gridDim.x;
        s_ptile = t;
        if (t < total) s_pref = decode_tile(sl, jobs, pre, njobs, t);
    };
    auto issue_next = [&]() {
        if (s_ptile >= total) return;
        const int st = (int)(s_issued % NST);
        unsigned char *sb = smem + st * STAGE_BYTES;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&full[st], STAGE_BYTES);
        const TileRef &P = s_pref;
        const int64_t cc = P.c0 + s_pchunk;
        for (int p = 0; p < NS; p++) {
            bulk_g2s(sb + p * BLK * 2, P.gA + p * P.pA + cc * BLK, BLK * 2, &full[st]);
            bulk_g2s(sb + (NS + p) * BLK * 2, P.gB + p * P.pB + cc * BLK, BLK * 2, &full[st]);
        }
        s_issued++;
        if (++s_pchunk == P.nch) {
            s_pchunk = 0;
            s_ptile += gridDim.x;
            prod_advance_tile();
        }
    };
    if (tid == 0) {
        s_ptile = blockIdx.x;
        s_issued = 0;
        s_pchunk = 0;
        prod_advance_tile();
        for (int k = 0; k < NST; k++) issue_next();
    }

    const int wm = warp >> 2, wn = warp & 3;     // warp tile: rows wm*16.., cols wn*16..
    // ldmatrix row / 16-byte chunk of this lane: the A tile (16 rows x 16 k), the B pair of n8 tiles
    const int arow = lane & 15, akc = lane >> 4;
    const int brow = ((lane >> 4) << 3) + (lane & 7), bkc = (lane >> 3) & 1;
    constexpr int NI = ND - 3;                   // exact int32 diagonals 2 .. 6
    int64_t consumed = 0;
    for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        if (!active(tile)) continue;
        const TileRef T = decode_tile(sl, jobs, pre, njobs, tile);
        const GemmJob &J = jobs[T.job];
        int32_t iacc[NI][2][4];
        float tail[2][4];
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                tail[b][q] = 0.f;
#pragma unroll
                for (int d = 0; d < NI; d++) iacc[d][b][q] = 0;
            }
        for (int c = 0; c < T.nch; c++, consumed++) {
            const int st = (int)(consumed % NST);
            const uint32_t parity = (uint32_t)((consumed / NST) & 1);
            if (tid == 0 && !mbar_wait_bounded(&full[st], parity, 2000000000ull)) s_bad = 1;
            __syncthreads();
            if (s_bad) {
                if (tid == 0) {
                    flag_error(err, LSAMG_DEVICE_TIMEOUT, (int)blockIdx.x);
                    // let the copies already in flight land before the CTA's shared memory is released
                    for (int64_t g2 = consumed; g2 < s_issued; g2++)
                        mbar_wait_bounded(&full[g2 % NST], (uint32_t)((g2 / NST) & 1), 1000000000ull);
                }
                return;
            }
            mbar_wait_bounded(&full[st], parity, 1000000000ull);   // completed: returns at once
            const uint32_t sA = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t sB = sA + NS * BLK * 2;
#pragma unroll 1
            for (int ks = 0; ks < 2; ks++) {
                // every A slice's fragment stays in registers for the step; a B fragment is read from
                // shared memory for each slice pair that uses it
                uint32_t af[NS][4];
#pragma unroll
                for (int p = 0; p < NS; p++) {
                    const int r = wm * 16 + arow, kc = ks * 2 + akc;
                    ldsm_x4(af[p], sA + p * BLK * 2 + r * 64 + ((((kc ^ (r >> 1)) & 3)) << 4));
                }
                const int br = wn * 16 + brow, bkk = ks * 2 + bkc;
                const uint32_t boff = br * 64 + ((((bkk ^ (br >> 1)) & 3)) << 4);
#pragma unroll
                for (int d = 2; d <= ND; d++) {
                    float acc[2][4];
#pragma unroll
                    for (int b = 0; b < 2; b++)
#pragma unroll
                        for (int q = 0; q < 4; q++) acc[b][q] = 0.f;
#pragma unroll
                    for (int p = 1; p <= NS; p++) {
                        const int q = d - p;
                        if (q < 1 || q > NS) continue;
                        uint32_t bf[4];
                        ldsm_x4(bf, sB + (q - 1) * BLK * 2 + boff);
#pragma unroll
                        for (int nt = 0; nt < 2; nt++) mma16816(acc[nt], af[p - 1], bf[2 * nt], bf[2 * nt + 1]);
                    }
                    // exact FP32 -> int32 (the sums are integers below 2^21 in magnitude), or the tail
#pragma unroll
                    for (int b = 0; b < 2; b++)
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            if (d - 2 < NI)
                                iacc[d - 2][b][q] += __float_as_int(acc[b][q] + 12582912.0f) - 0x4B400000;
                            else if (d == ND - 1)
                                tail[b][q] += acc[b][q];
                            else
                                tail[b][q] = fmaf(acc[b][q], 1.0f / 256.0f, tail[b][q]);
                        }
                }
            }
            __syncthreads();   // every warp is done with this stage
            if (tid == 0) issue_next();
        }
        const int g = lane >> 2, tg = lane & 3;
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = T.tm * TM + wm * 16 + g + ((q >> 1) << 3);
                const int jj = T.tn * TM + wn * 16 + nt * 8 + 2 * tg + (q & 1);
                if (i >= J.M || jj >= J.N || (J.lower && i < jj)) continue;
                store_out(C + J.c_off + (int64_t)i * J.crs + (int64_t)jj * J.ccs, iacc[0][nt][q], iacc[1][nt][q],
                          iacc[2][nt][q], iacc[3][nt][q], iacc[4][nt][q], tail[nt][q],
                          ex[J.a_exp + i] + ex[J.b_exp + jj] - 62, alpha, beta);
            }
    }
}

// ------------------------------------------------------------------------------- tcgen05 gemm
// The same products on the fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory).  A CTA computes a 128 x 32 tile of C.  In each 16-wide K step, A slice p multiplies
// the B slices 1 .. 8-p stacked along N in ONE instruction (N = 32 (8 - p)): the product of
// pair (p, q) lands in tensor-memory columns 32 (p + q - 2) .., i.e. in the accumulator of its
// diagonal d = p + q, so seven instructions per K step cover all 28 pairs.  Each diagonal sum
// of a K piece of 128 is an integer below 7 * 128 * 2^14 < 2^24, exact in FP32; the epilogue
// moves it into 64-bit integers (two per output, units 2^32 and 1 of the lowest weight) and
// forms the FP64 result once per tile.  The 7 x 32 FP32 accumulator columns are double
// buffered (2 x 256 of the 512 columns), so the epilogue of one piece overlaps the products of
// the next.  Warp 0 stages operands with bulk copies (three 70 KB stages), warp 1 owns the
// tensor memory and issues the products (one thread), warps 2..17 run the epilogue (four per
// 32-lane quarter of the tensor memory, 8 columns each).
namespace tcg {
constexpr int BM = 128, BN = 32;
constexpr int TST = 3;                         // staging ring depth
constexpr int A_BYTES = NS * BM * TK * 2;      // 7 slices x 128 rows x 64 B
constexpr int B_BYTES = NS * BN * TK * 2;      // 7 slices x 32 rows x 64 B
constexpr int STAGE = A_BYTES + B_BYTES;       // 70 KB
constexpr int PIECE = 4;                       // K chunks of 32 per accumulation piece
#ifndef TC_EPI_WARPS
#define TC_EPI_WARPS 16
#endif
constexpr int EPI_WARPS = TC_EPI_WARPS;        // epilogue warps: EPI_WARPS / 4 per lane quarter
constexpr int EC = BN / (EPI_WARPS / 4);       // columns per epilogue thread
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int SMEM = TST * STAGE + 1024;       // + alignment slack
constexpr uint32_t TMEM_COLS = 512;
constexpr uint64_t WAIT_NS = 2000000000ull;
}  // namespace tcg

__device__ __forceinline__ void tm_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D[tmem] (+)= A[smem] B[smem]^T, FP16 inputs, FP32 accumulation; acc = 0 overwrites D
__device__ __forceinline__ void umma_f16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive on `bar` once every product issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 32 lanes (this warp's quarter) x 8 consecutive 32-bit columns
__device__ __forceinline__ void tm_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// shared-memory matrix descriptor: K-major rows of 64 bytes in the 64-byte swizzle (16-byte
// chunk index XOR (row / 2) mod 4, the layout the operand blocks are stored in), 8-row groups
// 512 bytes apart
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// instruction descriptor of kind::f16: FP32 D, FP16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// tiles of a lower-triangular job before tile row tm: row t holds min(tilesN, 4 t + 4) tiles,
// those reaching the diagonal
__host__ __device__ inline int64_t tc_lower_prefix(int64_t tm, int64_t tilesN) {
    const int64_t t0 = tm < tilesN / 4 ? tm : tilesN / 4;
    return 2 * t0 * (t0 + 1) + (tm - t0) * tilesN;
}

struct TcTile {
    int job, tm, tn, nch;
};
__device__ __forceinline__ TcTile tc_decode(const GemmJob *jobs, const int64_t *pre, int njobs, int64_t t) {
    TcTile r;
    r.job = find_job(pre, njobs, t);
    const GemmJob &J = jobs[r.job];
    const int64_t local = t - pre[r.job];
    const int tilesN = dcdiv(J.N, tcg::BN);
    if (J.lower) {
        int lo = 0, hi = dcdiv(J.M, tcg::BM) - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tc_lower_prefix(mid, tilesN) <= local) lo = mid; else hi = mid - 1;
        }
        r.tm = lo;
        r.tn = (int)(local - tc_lower_prefix(lo, tilesN));
    } else {
        r.tm = (int)(local / tilesN);
        r.tn = (int)(local % tilesN);
    }
    r.nch = dcdiv(max(J.K, 1), TK);
    return r;
}

__global__ void __launch_bounds__(tcg::THREADS, 1)
    k_gemm_tc(const __half *sl, const int32_t *ex, double *C, const GemmJob *jobs, const int64_t *pre, int njobs,
              const Scale sc, int *err, const int32_t *skip) {
    using namespace tcg;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[TST], empty[TST], tfull[2], tempty[2], done;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t total = pre[njobs];
    auto active = [&](int64_t t) { return !skip || skip[jobs[find_job(pre, njobs, t)].skip_idx] < 0; };
    auto fail_wait = [&](int where) {
        if (!s_abort) flag_error(err, LSAMG_DEVICE_TIMEOUT, (int)blockIdx.x * 16 + where);
        s_abort = 1;
    };
    if (tid == 0) {
        for (int i = 0; i < TST; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
        mbar_init(&done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tm_alloc(&s_tmem, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_tmem;

    if (warp == 0) {
        // ---------------- producer: bulk copies of the slice blocks of every K chunk
        if (lane == 0) {
            int64_t it = 0;
            for (int64_t t = blockIdx.x; t < total && !s_abort; t += gridDim.x) {
                if (!active(t)) continue;
                const TcTile T = tc_decode(jobs, pre, njobs, t);
                const GemmJob &J = jobs[T.job];
                const int ntot = dcdiv(max(J.ktot, 1), TK), c0 = J.k0 / TK;
                const int64_t pA = stor_tiles(J.M) * ntot * BLK, pB = stor_tiles(J.N) * ntot * BLK;
                const __half *gA = sl + J.a_off + (int64_t)(2 * T.tm) * ntot * BLK;
                const __half *gB = sl + J.b_off + (int64_t)(T.tn >> 1) * ntot * BLK + (T.tn & 1) * (BN * TK);
                for (int c = 0; c < T.nch && !s_abort; c++, it++) {
                    const int st = (int)(it % TST);
                    if (it >= TST && !mbar_wait_bounded(&empty[st], (uint32_t)((it / TST - 1) & 1), WAIT_NS)) {
                        fail_wait(1);
                        break;
                    }
                    unsigned char *sb = smem + st * STAGE;
                    mbar_expect_tx(&full[st], STAGE);
                    const int64_t cc = c0 + c;
                    for (int p = 0; p < NS; p++) {
                        const __half *a = gA + p * pA + cc * BLK;
                        bulk_g2s(sb + p * (BM * TK * 2), a, BLK * 2, &full[st]);
                        bulk_g2s(sb + p * (BM * TK * 2) + BLK * 2, a + (int64_t)ntot * BLK, BLK * 2, &full[st]);
                        bulk_g2s(sb + A_BYTES + p * (BN * TK * 2), gB + p * pB + cc * BLK, BN * TK * 2, &full[st]);
                    }
                }
            }
            // copies still in flight land before the CTA's shared memory is released
            for (int64_t g = (it > TST ? it - TST : 0); g < it; g++)
                mbar_wait_bounded(&full[g % TST], (uint32_t)((g / TST) & 1), WAIT_NS);
        }
    } else if (warp == 1) {
        // ---------------- issuer: 7 products per 16-wide K step
        if (lane == 0) {
            int64_t it = 0, pc = 0;
            bool issued = false;
            for (int64_t t = blockIdx.x; t < total && !s_abort; t += gridDim.x) {
                if (!active(t)) continue;
                const TcTile T = tc_decode(jobs, pre, njobs, t);
                for (int c0 = 0; c0 < T.nch && !s_abort; c0 += PIECE, pc++) {
                    const int b = (int)(pc & 1);
                    if (pc >= 2 && !mbar_wait_bounded(&tempty[b], (uint32_t)(((pc >> 1) - 1) & 1), WAIT_NS)) {
                        fail_wait(2);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tbase + (uint32_t)b * 256u;
                    const int c1 = min(T.nch, c0 + PIECE);
                    for (int c = c0; c < c1; c++, it++) {
                        const int st = (int)(it % TST);
                        if (!mbar_wait_bounded(&full[st], (uint32_t)((it / TST) & 1), WAIT_NS)) {
                            fail_wait(3);
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(smem + st * STAGE), sbb = sa + A_BYTES;
#pragma unroll
                        for (int ks = 0; ks < 2; ks++)
#pragma unroll
                            for (int p = 1; p <= NS; p++)
                                umma_f16(dt + 32u * (p - 1), sdesc_sw64(sa + (p - 1) * (BM * TK * 2) + ks * 32),
                                         sdesc_sw64(sbb + ks * 32), idesc_f16(BM, BN * (8 - p)),
                                         (c > c0 || ks > 0 || p > 1) ? 1u : 0u);
                        umma_commit(&empty[st]);
                        issued = true;
                    }
                    if (s_abort) break;
                    umma_commit(&tfull[b]);
                }
            }
            if (issued) {
                // every product completed before the tensor memory is released
                umma_commit(&done);
                mbar_wait_bounded(&done, 0, WAIT_NS);
            }
        }
    } else {
        // ---------------- epilogue: rows 32 (warp % 4) + lane, EC columns per warp
        const int qd = warp & 3, cg = (warp - 2) >> 2;
        const int row = 32 * qd + lane;
        const uint32_t tq = tbase + ((uint32_t)(32 * qd) << 16);
        int64_t pc = 0;
        for (int64_t t = blockIdx.x; t < total && !s_abort; t += gridDim.x) {
            if (!active(t)) continue;
            const TcTile T = tc_decode(jobs, pre, njobs, t);
            const GemmJob &J = jobs[T.job];
            int64_t hi[EC], lo[EC];
#pragma unroll
            for (int j = 0; j < EC; j++) hi[j] = lo[j] = 0;
            bool ok = true;
            for (int c0 = 0; c0 < T.nch; c0 += PIECE, pc++) {
                const int b = (int)(pc & 1);
                if (!mbar_wait_bounded(&tfull[b], (uint32_t)((pc >> 1) & 1), WAIT_NS)) {
                    fail_wait(4);
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < EC / 8; h++) {
                    float v[NS][8];
#pragma unroll
                    for (int d = 0; d < NS; d++)
                        tm_ld8(tq + (uint32_t)b * 256u + 32u * d + (uint32_t)(EC * cg) + 8u * h, v[d]);
                    tm_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        // S_2..S_8: integers below 2^24, exact in FP32
                        hi[8 * h + j] += ((int64_t)__float2int_rn(v[0][j]) << 16) +
                                         ((int64_t)__float2int_rn(v[1][j]) << 8) + (int64_t)__float2int_rn(v[2][j]);
                        lo[8 * h + j] += ((int64_t)__float2int_rn(v[3][j]) << 24) +
                                         ((int64_t)__float2int_rn(v[4][j]) << 16) +
                                         ((int64_t)__float2int_rn(v[5][j]) << 8) + (int64_t)__float2int_rn(v[6][j]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
            }
            if (!ok) break;
            const int i = T.tm * BM + row;
            if (i >= J.M) continue;
            const int ea = ex[J.a_exp + i] - 62;
            double *crow = C + J.c_off + (int64_t)i * J.crs;
            const int j0 = T.tn * BN + EC * cg;
            double cv[EC];
            int eb[EC];
#pragma unroll
            for (int j = 0; j < EC; j++) {
                const int jj = j0 + j;
                const bool in = jj < J.N && !(J.lower && i < jj);
                cv[j] = (sc.bmode != 0 && in) ? crow[(int64_t)jj * J.ccs] : 0.0;
                eb[j] = jj < J.N ? ex[J.b_exp + jj] : 0;
            }
            // C = beta C + alpha v 2^e: v rounded once, then the (FP64) update of C
#pragma unroll
            for (int j = 0; j < EC; j++) {
                const int jj = j0 + j;
                if (jj >= J.N || (J.lower && i < jj)) continue;
                int e = ea + eb[j];
                if (sc.pow2) {
                    e += sc.e2 - 1;
                    if (sc.neg) {
                        hi[j] = -hi[j];
                        lo[j] = -lo[j];
                    }
                }
                double r = limbs_to_double(hi[j], lo[j], e);
                if (!sc.pow2) r *= sc.alpha;
                crow[(int64_t)jj * J.ccs] = sc.bmode == 0 ? r : sc.bmode == 1 ? cv[j] + r : fma(sc.beta, cv[j], r);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tm_dealloc(tbase, TMEM_COLS);
    }
}

// one device upload of a job array and the exclusive prefix of its CTA counts
template <class Job>
int64_t upload_jobs(const std::vector<Job> &jobs, const std::vector<int64_t> &cnt, DBuf<int64_t> &buf,
                    const Job *&djobs, const int64_t *&dpre, cudaStream_t s) {
    const size_t nj = jobs.size();
    const size_t jw = (sizeof(Job) + 7) / 8;
    std::vector<int64_t> h(nj * jw + nj + 1, 0);
    std::memcpy(h.data(), jobs.data(), nj * sizeof(Job));
    int64_t *pre = h.data() + nj * jw;
    pre[0] = 0;
    for (size_t i = 0; i < nj; i++) pre[i + 1] = pre[i] + cnt[i];
    const int64_t total = pre[nj];
    upload(buf, h, s);
    djobs = reinterpret_cast<const Job *>(buf.p);
    dpre = buf.p + nj * jw;
    return total;
}

}  // namespace

void split(const double *src, const std::vector<SplitJob> &jobs, __half *dst, int32_t *exps, cudaStream_t s) {
    if (jobs.empty()) return;
    static_assert(sizeof(SplitJob) % 8 == 0, "job layout");
    std::vector<int64_t> cnt(jobs.size());
    for (size_t i = 0; i < jobs.size(); i++) {
        cnt[i] = jobs[i].rows > 0 ? stor_tiles(jobs[i].rows) : 0;   // padding blocks are zero-filled
    }
    DBuf<int64_t> buf;
    const SplitJob *dj = nullptr;
    const int64_t *dp = nullptr;
    const int64_t total = upload_jobs(jobs, cnt, buf, dj, dp, s);
    if (total == 0) return;
    if (total > 0x7fffffff) fail(LSAMG_LIMIT, "split grid too large");
    double by = 0.0;   // FP64 operand read once, NS FP16 slices written
    for (const auto &J : jobs) by += (double)J.rows * J.K * (8.0 + 2.0 * NS);
    KTime kt(KC_TC_SPLIT, s, 0.0, by);
    k_split<<<(unsigned)total, 256, 0, s>>>(src, dj, dp, (int)jobs.size(), dst, exps);
    CK_LAUNCH();
}

static int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

// products on the tcgen05 tensor cores: one launch for every K (64-bit integer accumulation
// across K pieces in the epilogue)
static void gemm_tc(const __half *slices, const int32_t *exps, double *C, const std::vector<GemmJob> &jobs,
                    double alpha, double beta, int *err, cudaStream_t s, const int32_t *skip) {
    std::vector<GemmJob> js;
    std::vector<int64_t> cnt;
    double fl = 0.0;   // FP64-equivalent flops of the products (lower: the triangle only)
    for (const auto &J0 : jobs) {
        if (J0.M <= 0 || J0.N <= 0) continue;
        GemmJob J = J0;
        J.k0 = 0;
        J.ktot = J0.K;
        const int64_t tm = cdiv(J.M, tcg::BM), tn = cdiv(J.N, tcg::BN);
        if (J.lower && J.M != J.N) fail(LSAMG_INVALID_ARG, "lower-triangular product of a non-square block");
        js.push_back(J);
        cnt.push_back(J.lower ? tc_lower_prefix(tm, tn) : tm * tn);
        fl += (J.lower ? 1.0 : 2.0) * J.M * (double)J.N * J.K;
    }
    if (js.empty()) return;
    DBuf<int64_t> buf;
    const GemmJob *dj = nullptr;
    const int64_t *dp = nullptr;
    const int64_t total = upload_jobs(js, cnt, buf, dj, dp, s);
    if (total == 0) return;
    if (total > 0x7fffffff) fail(LSAMG_LIMIT, "product grid too large");
    KTime kt(KC_TC_GEMM, s, fl);
    CK(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg::SMEM));
    const unsigned grid = (unsigned)std::min<int64_t>(total, device_sms());
    k_gemm_tc<<<grid, tcg::THREADS, tcg::SMEM, s>>>(slices, exps, C, dj, dp, (int)js.size(), make_scale(alpha, beta),
                                                    err, skip);
    CK_LAUNCH();
}

void gemm(const __half *slices, const int32_t *exps, double *C, const std::vector<GemmJob> &jobs, double alpha,
          double beta, int *err, cudaStream_t s, const int32_t *skip) {
    if (jobs.empty()) return;
    static_assert(sizeof(GemmJob) % 8 == 0, "job layout");
    static const bool mma_sync = getenv("LSAMG_OZ_MMA") != nullptr;
    if (!mma_sync) {
        gemm_tc(slices, exps, C, jobs, alpha, beta, err, s, skip);
        return;
    }
    static_assert(KPIECE % TK == 0, "K pieces are whole chunks");
    int npieces = 1;
    for (const auto &J : jobs) npieces = std::max<int>(npieces, (int)cdiv(std::max(J.K, 1), KPIECE));
    CK(cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM));
    for (int pc = 0; pc < npieces; pc++) {
        // pass pc: the pc-th K piece of every job (C accumulates from the second pass on)
        std::vector<GemmJob> js;
        std::vector<int64_t> cnt;
        for (const auto &J0 : jobs) {
            if (J0.M <= 0 || J0.N <= 0) continue;
            const int64_t k0 = (int64_t)pc * KPIECE;
            if (pc > 0 && k0 >= J0.K) continue;
            GemmJob J = J0;
            J.ktot = J0.K;
            J.k0 = (int32_t)k0;
            J.K = (int32_t)std::min<int64_t>(KPIECE, std::max<int64_t>(J0.K - k0, 0));
            const int64_t tm = cdiv(J.M, TM), tn = cdiv(J.N, TM);
            if (J.lower && tm != tn) fail(LSAMG_INVALID_ARG, "lower-triangular product of a non-square block");
            js.push_back(J);
            cnt.push_back(J.lower ? tm * (tm + 1) / 2 : tm * tn);
        }
        if (js.empty()) continue;
        DBuf<int64_t> buf;
        const GemmJob *dj = nullptr;
        const int64_t *dp = nullptr;
        const int64_t total = upload_jobs(js, cnt, buf, dj, dp, s);
        if (total == 0) continue;
        if (total > 0x7fffffff) fail(LSAMG_LIMIT, "product grid too large");
        double fl = 0.0;   // FP64-equivalent flops of the products (lower: the triangle only)
        for (const auto &J : js) fl += (J.lower ? 1.0 : 2.0) * J.M * (double)J.N * J.K;
        KTime kt(KC_TC_GEMM, s, fl);
        const unsigned grid = (unsigned)std::min<int64_t>(total, device_sms());
        k_gemm<<<grid, GT, GEMM_SMEM, s>>>(slices, exps, C, dj, dp, (int)js.size(), alpha, pc == 0 ? beta : 1.0, err,
                                          skip);
        CK_LAUNCH();
    }
}

}  // namespace oz
}  // namespace lsamg
