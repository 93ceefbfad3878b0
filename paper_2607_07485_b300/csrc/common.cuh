// Shared device/host utilities of liblsamg: status handling, stream-ordered device
// buffers, prefix sums, in-CTA sorting networks and CSR transposition.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <utility>
#include <algorithm>

#include "../../include/lsamg.h"

namespace lsamg {

// ---------------------------------------------------------------------------------
// Errors: C++ exceptions stay inside the library; the C ABI converts them to codes.
// ---------------------------------------------------------------------------------
struct Failure {
    int code;
    std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string &msg) { throw Failure{code, msg}; }

inline void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    int code = (e == cudaErrorMemoryAllocation) ? LSAMG_OOM : LSAMG_CUDA;
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    fail(code, buf);
}
#define CK(x) ::lsamg::cuda_check((x), #x, __FILE__, __LINE__)
#define CK_LAUNCH() (::lsamg::count_launch(), ::lsamg::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))

// Number of kernel launches issued by the library (all streams, process-wide).
void count_launch();
int64_t launch_count();

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Stage trace on stderr when the environment variable LSAMG_TRACE is set.
void trace(const char *fmt, ...);

// Opt-in stage profiler (environment variable LSAMG_PROFILE): synchronises the stream around
// each named region and accumulates wall time; prof_report() prints and clears the totals.
bool prof_on();
void prof_mark(const char *name, cudaStream_t s, bool begin);
void prof_report(const char *title);
struct ProfScope {
    const char *n;
    cudaStream_t s;
    ProfScope(const char *name, cudaStream_t st) : n(name), s(st) { if (prof_on()) prof_mark(n, s, true); }
    ~ProfScope() { if (prof_on()) prof_mark(n, s, false); }
};
#define LSAMG_PROF(name, stream) ::lsamg::ProfScope _prof_scope_##__LINE__(name, stream)

// Per-kernel-class device timing with CUDA events on the launching stream (enabled by the
// `profile` option): algorithmic FLOPs / bytes per launch are supplied by the caller.
enum KClass {
    KC_ELEM_FACTOR = 0, KC_POTRF, KC_PSTRF, KC_TRSM, KC_SYRK, KC_SYTD2, KC_STEBZ, KC_STEIN,
    KC_ORMTR, KC_ASSEMBLE, KC_COARSE_GRAM, KC_SCHWARZ, KC_SPMV, KC_TRANSFER, KC_COARSE_SOLVE,
    KC_GRAPH, KC_TC_GEMM, KC_TC_SPLIT, KC_SYMV, KC_N
};
const char *kclass_name(int c);
void ktimer_enable(bool on);
bool ktimer_enabled();
struct KTime {
    int cls;
    cudaStream_t s;
    double flops, bytes;
    cudaEvent_t e0 = nullptr;
    KTime(int c, cudaStream_t st, double f = 0.0, double b = 0.0);
    ~KTime();
};
struct KStat {
    double ms = 0.0, flops = 0.0, bytes = 0.0;
    int64_t calls = 0;
};
void ktimer_collect(KStat out[KC_N]);  // synchronises, accumulates and clears pending events

// ---------------------------------------------------------------------------------
// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync), move-only.
// ---------------------------------------------------------------------------------
template <class T>
struct DBuf {
    T *p = nullptr;
    int64_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept { *this = std::move(o); }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(int64_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count > 0) {
            cudaError_t e = cudaMallocAsync((void **)&p, (size_t)count * sizeof(T), st);
            if (e == cudaErrorMemoryAllocation) {
                // memory freed earlier may still sit in the stream-ordered pool in blocks too small
                // for this request: return it to the device and try once more
                cudaGetLastError();
                int dev = 0;
                cudaMemPool_t pool;
                if (cudaStreamSynchronize(st) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess && cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
                    e = cudaMallocAsync((void **)&p, (size_t)count * sizeof(T), st);
            }
            if (e != cudaSuccess) {
                p = nullptr;
                n = 0;
                cudaGetLastError();
                char buf[160];
                snprintf(buf, sizeof buf, "device allocation of %.3f GB failed",
                         (double)count * sizeof(T) / 1e9);
                fail(e == cudaErrorMemoryAllocation ? LSAMG_OOM : LSAMG_CUDA, buf);
            }
        }
    }
    void zero(cudaStream_t st) {
        if (n) CK(cudaMemsetAsync(p, 0, (size_t)n * sizeof(T), st));
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    int64_t size() const { return n; }
    int64_t bytes() const { return n * (int64_t)sizeof(T); }
};

template <class T>
inline std::vector<T> to_host(const T *d, int64_t n, cudaStream_t s) {
    std::vector<T> h((size_t)std::max<int64_t>(n, 0));
    if (n > 0) {
        CK(cudaMemcpyAsync(h.data(), d, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return h;
}

template <class T>
inline T read1(const T *d, cudaStream_t s) {
    T v;
    CK(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return v;
}

template <class T>
inline void upload(DBuf<T> &b, const std::vector<T> &h, cudaStream_t s) {
    b.alloc((int64_t)h.size(), s);
    if (!h.empty())
        CK(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

// ---------------------------------------------------------------------------------
// Device error flag: kernels record the first failure (code, info) with atomicCAS.
// ---------------------------------------------------------------------------------
__device__ inline void flag_error(int *err, int code, int info) {
    if (err && atomicCAS(err, 0, code) == 0) err[1] = info;
}

// ---------------------------------------------------------------------------------
// Prefix sums (exclusive, int64 output with the total in out[n]).
// ---------------------------------------------------------------------------------
void exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------------
// Batcher odd-even merge sort network for arbitrary length n (comparators touching
// positions >= n are dropped, which is valid because the virtual tail is +infinity).
// Called by all threads of a CTA on shared or global memory.
// ---------------------------------------------------------------------------------
template <class K>
__device__ inline void cta_oem_sort(K *a, int n) {
    for (int p = 1; p < n; p <<= 1) {
        for (int k = p; k >= 1; k >>= 1) {
            const int r0 = k % p;
            for (int x = threadIdx.x; x + k < n; x += blockDim.x) {
                if (x < r0) continue;
                if (((x - r0) & (2 * k - 1)) >= k) continue;
                if ((x / (2 * p)) != ((x + k) / (2 * p))) continue;
                K u = a[x], v = a[x + k];
                if (v < u) { a[x] = v; a[x + k] = u; }
            }
            __syncthreads();
        }
    }
}

// Sort every CSR segment ascending in place and (optionally) count unique values.
// Segments longer than the shared-memory capacity raise LSAMG_LIMIT through err.
void seg_sort(int32_t *vals, const int64_t *ptr, int64_t nseg, int64_t *uniq_count, int *err,
              cudaStream_t s);
// Compact the sorted segments to their unique values: out[optr[i]..] = unique(vals[ptr[i]..]).
void seg_unique_compact(const int32_t *vals, const int64_t *ptr, int64_t nseg, const int64_t *optr,
                        int32_t *out, cudaStream_t s);

// Transpose a CSR map rows -> cols (ptr [nr+1], idx) into cols -> rows with each output
// list sorted ascending.  Allocates tptr [nc+1] and tidx.
void csr_transpose(const int64_t *ptr, const int32_t *idx, int64_t nr, int64_t nnz, int64_t nc,
                   DBuf<int64_t> &tptr, DBuf<int32_t> &tidx, int *err, cudaStream_t s);

// Device-wide sort of 64-bit keys (bitonic network, one launch per stage).
void sort_u64(uint64_t *keys, int64_t n, cudaStream_t s);

// Small reductions.
int32_t max_i32(const int32_t *d, int64_t n, cudaStream_t s);
int64_t sum_i64(const int64_t *d, int64_t n, cudaStream_t s);

constexpr int SEG_SMEM_MAX = 56 * 1024;  // max int32 entries of one segment sorted in smem

// size thresholds between one-CTA-per-matrix and multi-CTA kernels (set from the options)
extern int g_large_dense;
extern int g_split_sweep;
extern int g_sweep_block;

// ------------------------------------------------------------------ double-float arithmetic
// For FP64 multiply-add streams where this GPU's FP64 pipe (1/64 of the FP32 rate) is the limit:
// an FP64 value x is carried as an FP32 pair hi + lo holding its leading 48 bits (truncated;
// relative error below 2^-47 for |x| >= 2^-78), products keep their exact FP32 rounding error
// (fma) and the three leading cross terms, sums are error-free (two-sum).  For |x| < 2^-78 the
// low part underflows (absolute error below 2^-126) and below 2^-126 the value is flushed to
// zero: callers use it on quantities of norm of order one.
__device__ __forceinline__ float2 df_split(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff);                 // biased FP64 exponent
    const uint64_t m = b & 0xfffffffffffffull;              // 52 fraction bits
    const int fe = e - 896;                                  // FP32 biased exponent of hi
    if (fe <= 0) return make_float2(0.f, 0.f);
    if (fe >= 255) return make_float2(__uint_as_float(sgn | 0x7f800000u), 0.f);
    const uint32_t hib = sgn | ((uint32_t)fe << 23) | (uint32_t)(m >> 29);
    const uint32_t r = (uint32_t)(m & 0x1fffffffull);        // the 29 bits below hi: r 2^(e - 1075)
    const int lz = __clz((int)r) - 3;                        // r's top bit at 28 - lz
    const int le = 28 - lz + e - 1075 + 127;                 // FP32 biased exponent of lo
    const uint32_t lm = lz >= 5 ? (r << (lz - 5)) : (r >> (5 - lz));
    const uint32_t lob = (r == 0u || le <= 0) ? 0u : (sgn | ((uint32_t)le << 23) | (lm & 0x7fffffu));
    return make_float2(__uint_as_float(hib), __uint_as_float(lob));
}
// (sh, sl) += a v
__device__ __forceinline__ void df_mac(float &sh, float &sl, float2 a, float2 v) {
    const float p = __fmul_rn(a.x, v.x);
    float e = fmaf(a.x, v.x, -p);
    e = fmaf(a.x, v.y, e);
    e = fmaf(a.y, v.x, e);
    const float t = __fadd_rn(sh, p);
    const float bv = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    sl = __fadd_rn(sl, __fadd_rn(err, e));
    sh = t;
}
// (sh, sl) += (oh, ol)
__device__ __forceinline__ void df_add(float &sh, float &sl, float oh, float ol) {
    const float t = __fadd_rn(sh, oh);
    const float bv = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(oh, bv));
    sl = __fadd_rn(sl, __fadd_rn(err, ol));
    sh = t;
}


}  // namespace lsamg
