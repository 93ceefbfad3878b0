// FP64 products on FP16 tensor cores by exact splitting (see ozaki.cuh for the scheme).
#include <cmath>
#include <cstring>

#include "ozaki.cuh"

namespace lsamg {
namespace oz {
namespace {

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
// Operands are split in three launches so that every (64-row tile, 32-wide K chunk) is its own
// CTA: the row exponents e_r are first cleared, then raised to the exponent of each chunk's row
// maximum (integer atomic maxima: the order does not matter), then each chunk is cut into
// slices.  Exponents are held as e + EXP_BIAS while the maxima are formed; 0 marks a row with no
// nonzero entry (exponent 0), and a stored value below EXP_BIAS / 2 is already final.
constexpr int EXP_BIAS = 1 << 20;
__device__ __forceinline__ int exp_decode(int v) { return v >= EXP_BIAS / 2 ? v - EXP_BIAS : v; }

constexpr int SPLIT_THREADS = 256;   // threads of k_split_max and k_split (a 64 x 32 chunk per CTA)
static_assert(BLK / 2 % SPLIT_THREADS == 0, "pairs of a chunk per thread");

__global__ void __launch_bounds__(256) k_split_clear(const SplitJob *jobs, const int64_t *pre, int njobs,
                                                     int32_t *exps) {
    const int j = find_job(pre, njobs, blockIdx.x);
    const int t = (int)(blockIdx.x - pre[j]);
    if (threadIdx.x < TM) exps[jobs[j].exp_off + t * TM + threadIdx.x] = 0;
}

// unit u of job j: tile u / nch, chunk u % nch
__global__ void __launch_bounds__(SPLIT_THREADS) k_split_max(const double *src, const SplitJob *jobs, const int64_t *pre,
                                                   int njobs, int32_t *exps) {
    __shared__ double rmax[TM][5];
    const int j = find_job(pre, njobs, blockIdx.x);
    const SplitJob J = jobs[j];
    const int nch = dcdiv(max(J.K, 1), TK);
    const int u = (int)(blockIdx.x - pre[j]), t = u / nch, c = u % nch;
    const int i0 = t * TM;
    const bool kfast = (J.ks == 1);
    const double *S = src + J.src_off;
    double m = 0.0;
    int r, g;
    if (kfast) { r = threadIdx.x >> 2; g = threadIdx.x & 3; }   // 4 threads per row
    else       { r = threadIdx.x & 63; g = threadIdx.x >> 6; }
    const int i = i0 + r;
    double v[TK / 4];   // this thread's entries of the chunk, all loads in flight at once
#pragma unroll
    for (int q = 0; q < TK / 4; q++) {
        const int k = c * TK + g + 4 * q;
        v[q] = (i < J.rows && k < J.K) ? S[(int64_t)i * J.rs + (int64_t)k * J.ks] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < TK / 4; q++) m = fmax(m, fabs(v[q]));
    rmax[r][g] = m;
    __syncthreads();
    if (threadIdx.x < TM) {
        const double v = fmax(fmax(rmax[threadIdx.x][0], rmax[threadIdx.x][1]),
                              fmax(rmax[threadIdx.x][2], rmax[threadIdx.x][3]));
        if (v > 0.0) {
            int e;
            frexp(v, &e);     // v < 2^e
            atomicMax(&exps[J.exp_off + i0 + threadIdx.x], e + EXP_BIAS);
        }
    }
}

__global__ void __launch_bounds__(SPLIT_THREADS) k_split(const double *src, const SplitJob *jobs, const int64_t *pre,
                                                         int njobs, __half *dst, int32_t *exps) {
    __shared__ int rexp[TM];
    const int j = find_job(pre, njobs, blockIdx.x);
    const SplitJob J = jobs[j];
    const int tiles = (int)stor_tiles(J.rows), nch = dcdiv(max(J.K, 1), TK);
    const int u = (int)(blockIdx.x - pre[j]), t = u / nch, c = u % nch;
    const int i0 = t * TM;
    const bool kfast = (J.ks == 1);
    const double *S = src + J.src_off;
    // the chunk's entries of this thread are loaded first, all in flight at once
    constexpr int IT = BLK / 2 / SPLIT_THREADS;
    double vin[IT][2];
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int idx = threadIdx.x + it * SPLIT_THREADS;
        int r, kk;
        if (kfast) { r = idx >> 4; kk = (idx & 15) * 2; } else { r = idx & 63; kk = (idx >> 6) * 2; }
        const int i = i0 + r;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int k = c * TK + kk + h;
            vin[it][h] = (i < J.rows && k < J.K) ? S[(int64_t)i * J.rs + (int64_t)k * J.ks] : 0.0;
        }
    }
    if (threadIdx.x < TM) rexp[threadIdx.x] = exp_decode(exps[J.exp_off + i0 + threadIdx.x]);
    __syncthreads();
    if (c == 0 && threadIdx.x < TM) exps[J.exp_off + i0 + threadIdx.x] = rexp[threadIdx.x];   // final form
    // slices in integer arithmetic (the FP64 pipe is scarce): F = round(v 2^(55 - e_r)) exactly
    // from the bits of v (|F| < 2^55), then its balanced base-256 digits, F = sum_p a_p 2^(48-8p)
    // with the low six a_p in [-128, 127] and |a_0| <= 128, which hold F exactly.  They are read
    // off G = F + 128 (1 + 2^8 + ... + 2^48) > 0: the low six digits are the bytes of G minus 128,
    // the top one G / 2^48 - 128.  Two consecutive k per thread.
    const int64_t pstride = (int64_t)tiles * nch * BLK;
    {
#pragma unroll
        for (int it = 0; it < IT; it++) {
            const int idx = threadIdx.x + it * SPLIT_THREADS;
            int r, kk;
            if (kfast) { r = idx >> 4; kk = (idx & 15) * 2; } else { r = idx & 63; kk = (idx >> 6) * 2; }
            int dig[2][NS];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const double v = vin[it][h];
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
                const uint64_t G = (uint64_t)(F + 0x80808080808080ll);   // > 0 since |F| < 2^55
                const uint32_t glo = (uint32_t)G, ghi = (uint32_t)(G >> 32);
                dig[h][0] = (int)(ghi >> 16) - 128;
#pragma unroll
                for (int p = 1; p < NS; p++) {
                    const int byte = 6 - p;                                // byte of G at 2^(48 - 8p)
                    const uint32_t w = byte >= 4 ? ghi : glo;
                    dig[h][p] = (int)((w >> (8 * (byte & 3))) & 255u) - 128;
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
            // C = beta C + alpha v 2^e: v rounded once, then the (FP64) update of C; the uniform
            // cases are separate loops so that no unused FP64 operation is issued
            double r[EC];
            const int es = sc.pow2 ? sc.e2 - 1 : 0;
            const bool flip = sc.pow2 && sc.neg;
#pragma unroll
            for (int j = 0; j < EC; j++)
                r[j] = limbs_to_double(flip ? -hi[j] : hi[j], flip ? -lo[j] : lo[j], ea + eb[j] + es);
            if (!sc.pow2) {
#pragma unroll
                for (int j = 0; j < EC; j++) r[j] *= sc.alpha;
            }
            if (sc.bmode == 1) {
#pragma unroll
                for (int j = 0; j < EC; j++) r[j] += cv[j];
            } else if (sc.bmode == 2) {
#pragma unroll
                for (int j = 0; j < EC; j++) r[j] = fma(sc.beta, cv[j], r[j]);
            }
#pragma unroll
            for (int j = 0; j < EC; j++) {
                const int jj = j0 + j;
                if (jj < J.N && !(J.lower && i < jj)) crow[(int64_t)jj * J.ccs] = r[j];
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
    // tiles (padding tiles included: they are zero-filled) and (tile, chunk) units per job
    std::vector<int64_t> ct(jobs.size()), cu(jobs.size());
    for (size_t i = 0; i < jobs.size(); i++) {
        ct[i] = jobs[i].rows > 0 ? stor_tiles(jobs[i].rows) : 0;
        cu[i] = ct[i] * cdiv(std::max(jobs[i].K, 1), TK);
    }
    DBuf<int64_t> bt, bu;
    const SplitJob *dj = nullptr, *dju = nullptr;
    const int64_t *dpt = nullptr, *dpu = nullptr;
    const int64_t tt = upload_jobs(jobs, ct, bt, dj, dpt, s);
    const int64_t tu = upload_jobs(jobs, cu, bu, dju, dpu, s);
    if (tt == 0) return;
    if (tu > 0x7fffffff) fail(LSAMG_LIMIT, "split grid too large");
    double by = 0.0;   // FP64 operand read twice (maxima, slices), NS FP16 slices written
    for (const auto &J : jobs) by += (double)J.rows * J.K * (16.0 + 2.0 * NS);
    KTime kt(KC_TC_SPLIT, s, 0.0, by);
    k_split_clear<<<(unsigned)tt, 64, 0, s>>>(dj, dpt, (int)jobs.size(), exps);
    CK_LAUNCH();
    k_split_max<<<(unsigned)tu, SPLIT_THREADS, 0, s>>>(src, dju, dpu, (int)jobs.size(), exps);
    CK_LAUNCH();
    k_split<<<(unsigned)tu, SPLIT_THREADS, 0, s>>>(src, dju, dpu, (int)jobs.size(), dst, exps);
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
    double by = 0.0;   // algorithmic bytes: the FP16 slices of A and B once, C read (beta != 0) and written
    const double cbytes = beta != 0.0 ? 16.0 : 8.0;
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
        by += 2.0 * NS * ((double)J.M + J.N) * J.K + (J.lower ? 0.5 : 1.0) * cbytes * J.M * (double)J.N;
    }
    if (js.empty()) return;
    DBuf<int64_t> buf;
    const GemmJob *dj = nullptr;
    const int64_t *dp = nullptr;
    const int64_t total = upload_jobs(js, cnt, buf, dj, dp, s);
    if (total == 0) return;
    if (total > 0x7fffffff) fail(LSAMG_LIMIT, "product grid too large");
    KTime kt(KC_TC_GEMM, s, fl, by);
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
    gemm_tc(slices, exps, C, jobs, alpha, beta, err, s, skip);
}

}  // namespace oz
}  // namespace lsamg
