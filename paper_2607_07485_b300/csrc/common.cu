// Implementations of the shared utilities declared in common.cuh.
#include "common.cuh"

#include <cstdarg>
#include <deque>
#include <cstdlib>
#include <ctime>

namespace lsamg {

int g_large_dense = 2048;
int g_split_sweep = 128;
int g_sweep_block = 64;

static int64_t g_launches = 0;
void count_launch() { g_launches++; }
int64_t launch_count() { return g_launches; }

static const char *kKNames[KC_N] = {"elem_factor", "potrf", "pstrf", "trsm", "syrk", "sytd2",
                                    "stebz", "stein", "ormtr", "assemble", "coarse_gram",
                                    "schwarz_sweep", "gram_spmv", "transfer", "coarse_solve",
                                    "graph", "tc_dgemm", "tc_split", "sytd2_symv"};
const char *kclass_name(int c) { return (c >= 0 && c < KC_N) ? kKNames[c] : ""; }
static bool g_kt_on = false;
void ktimer_enable(bool on) { g_kt_on = on; }
bool ktimer_enabled() { return g_kt_on; }
struct KPending {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
};
static std::deque<KPending> g_kpend;
static KStat g_kacc[KC_N];

static std::vector<cudaEvent_t> g_evpool;
static cudaEvent_t ev_get() {
    if (!g_evpool.empty()) {
        cudaEvent_t e = g_evpool.back();
        g_evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

KTime::KTime(int c, cudaStream_t st, double f, double b) : cls(c), s(st), flops(f), bytes(b) {
    if (!g_kt_on) return;
    e0 = ev_get();
    cudaEventRecord(e0, s);
}
static void kt_account(const KPending &p) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    g_kacc[p.cls].ms += ms;
    g_kacc[p.cls].calls += 1;
    g_kacc[p.cls].flops += p.flops;
    g_kacc[p.cls].bytes += p.bytes;
    g_evpool.push_back(p.a);
    g_evpool.push_back(p.b);
}

KTime::~KTime() {
    if (!g_kt_on || !e0) return;
    cudaEvent_t e1 = ev_get();
    cudaEventRecord(e1, s);
    g_kpend.push_back({cls, e0, e1, flops, bytes});
    // fold the intervals the device has finished into the totals and recycle their events, so
    // that a long profiled run holds a bounded number of events (polling, never waiting)
    if (g_kpend.size() >= 4096 && cudaPeekAtLastError() == cudaSuccess) {
        while (!g_kpend.empty()) {
            const cudaError_t q = cudaEventQuery(g_kpend.front().b);
            if (q != cudaSuccess) {
                if (q == cudaErrorNotReady) (void)cudaGetLastError();   // not an error: still running
                break;
            }
            kt_account(g_kpend.front());
            g_kpend.pop_front();
        }
    }
}

void ktimer_collect(KStat out[KC_N]) {
    for (auto &p : g_kpend) {
        cudaEventSynchronize(p.b);
        kt_account(p);
    }
    g_kpend.clear();
    if (out)
        for (int c = 0; c < KC_N; c++) {
            out[c] = g_kacc[c];
            g_kacc[c] = KStat{};
        }
}

static std::vector<std::pair<std::string, double>> g_prof;
static std::vector<std::pair<std::string, double>> g_open;

bool prof_on() {
    static const bool on = std::getenv("LSAMG_PROFILE") != nullptr;
    return on;
}

static double wall() {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return t.tv_sec + 1e-9 * t.tv_nsec;
}

void prof_mark(const char *name, cudaStream_t s, bool begin) {
    cudaStreamSynchronize(s);
    double t = wall();
    if (begin) {
        g_open.push_back({name, t});
        return;
    }
    for (auto it = g_open.rbegin(); it != g_open.rend(); ++it)
        if (it->first == name) {
            double dt = t - it->second;
            g_open.erase(std::next(it).base());
            for (auto &q : g_prof)
                if (q.first == name) {
                    q.second += dt;
                    return;
                }
            g_prof.push_back({name, dt});
            return;
        }
}

void prof_report(const char *title) {
    if (!prof_on() || g_prof.empty()) return;
    fprintf(stderr, "[lsamg profile] %s\n", title);
    for (auto &q : g_prof) fprintf(stderr, "  %-28s %10.4f s\n", q.first.c_str(), q.second);
    fflush(stderr);
    g_prof.clear();
}

void trace(const char *fmt, ...) {
    static const bool on = std::getenv("LSAMG_TRACE") != nullptr;
    if (!on) return;
    va_list ap;
    va_start(ap, fmt);
    fprintf(stderr, "[lsamg] ");
    vfprintf(stderr, fmt, ap);
    fprintf(stderr, "\n");
    fflush(stderr);
    va_end(ap);
}

// ----------------------------------------------------------------------------- scans
namespace {
constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <class In>
__global__ void k_scan_tile(const In *in, int64_t *out, int64_t *bsum, int64_t n) {
    __shared__ int64_t warp_tot[SCAN_T / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t run = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t j = base + i;
        v[i] = (j < n) ? (int64_t)in[j] : 0;
        run += v[i];
    }
    // inclusive warp scan of per-thread totals
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < SCAN_T / 32) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < SCAN_T / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t excl = incl - run + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t j = base + i;
        if (j < n) out[j] = excl;
        excl += v[i];
    }
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = excl;
}

__global__ void k_scan_add(int64_t *out, const int64_t *boff, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    int64_t add = boff[blockIdx.x];
    for (int i = 0; i < SCAN_ITEMS; i++, j += SCAN_T)
        if (j < n) out[j] += add;
}

__global__ void k_set_total(int64_t *out, int64_t n, const int64_t *bsum_scan, int64_t nb) {
    out[n] = bsum_scan[nb];
}

template <class In>
void scan_impl(const In *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    int64_t nb = cdiv(n, SCAN_TILE);
    DBuf<int64_t> bsum, boff;
    bsum.alloc(nb, s);
    k_scan_tile<In><<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, bsum.p, n);
    CK_LAUNCH();
    if (nb == 1) {  // one tile: its sum is the total
        CK(cudaMemcpyAsync(out + n, bsum.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        return;
    }
    boff.alloc(nb + 1, s);
    scan_impl<int64_t>(bsum.p, boff.p, nb, s);
    k_scan_add<<<(unsigned)nb, SCAN_T, 0, s>>>(out, boff.p, n);
    CK_LAUNCH();
    k_set_total<<<1, 1, 0, s>>>(out, n, boff.p, nb);
    CK_LAUNCH();
}
}  // namespace

void exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    scan_impl<int32_t>(in, out, n, s);
}
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    scan_impl<int64_t>(in, out, n, s);
}

// ----------------------------------------------------------------------------- segmented sort
namespace {
__global__ void k_seg_sort(int32_t *vals, const int64_t *ptr, int64_t nseg, int64_t *ucount,
                           int *err) {
    extern __shared__ int32_t sm[];
    for (int64_t sgi = blockIdx.x; sgi < nseg; sgi += gridDim.x) {
        int64_t b = ptr[sgi], e = ptr[sgi + 1];
        int len = (int)(e - b);
        if (e - b > SEG_SMEM_MAX) {
            if (threadIdx.x == 0) flag_error(err, LSAMG_LIMIT, (int)sgi);
            continue;
        }
        for (int i = threadIdx.x; i < len; i += blockDim.x) sm[i] = vals[b + i];
        __syncthreads();
        cta_oem_sort<int32_t>(sm, len);
        for (int i = threadIdx.x; i < len; i += blockDim.x) vals[b + i] = sm[i];
        if (ucount) {
            __shared__ int cnt;
            if (threadIdx.x == 0) cnt = 0;
            __syncthreads();
            int local = 0;
            for (int i = threadIdx.x; i < len; i += blockDim.x)
                local += (i == 0 || sm[i] != sm[i - 1]);
            atomicAdd(&cnt, local);
            __syncthreads();
            if (threadIdx.x == 0) ucount[sgi] = cnt;
        }
        __syncthreads();
    }
}

__global__ void k_seg_unique(const int32_t *vals, const int64_t *ptr, int64_t nseg,
                             const int64_t *optr, int32_t *out) {
    // one warp per segment: stream-compact unique values with ballots
    int lane = threadIdx.x & 31;
    int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sgi = wid; sgi < nseg; sgi += nw) {
        int64_t b = ptr[sgi], e = ptr[sgi + 1];
        int64_t o = optr[sgi];
        for (int64_t base = b; base < e; base += 32) {
            int64_t i = base + lane;
            bool keep = false;
            int32_t v = 0;
            if (i < e) {
                v = vals[i];
                keep = (i == b) || (vals[i - 1] != v);
            }
            unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) out[o + __popc(m & ((1u << lane) - 1))] = v;
            o += __popc(m);
        }
    }
}
}  // namespace

void seg_sort(int32_t *vals, const int64_t *ptr, int64_t nseg, int64_t *uniq_count, int *err,
              cudaStream_t s) {
    if (nseg <= 0) return;
    static bool attr = false;
    if (!attr) {
        CK(cudaFuncSetAttribute(k_seg_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SEG_SMEM_MAX * (int)sizeof(int32_t)));
        attr = true;
    }
    int64_t grid = std::min<int64_t>(nseg, 148 * 8);
    // shared memory sized for the largest possible segment
    k_seg_sort<<<(unsigned)grid, 256, SEG_SMEM_MAX * sizeof(int32_t), s>>>(vals, ptr, nseg,
                                                                           uniq_count, err);
    CK_LAUNCH();
}

void seg_unique_compact(const int32_t *vals, const int64_t *ptr, int64_t nseg, const int64_t *optr,
                        int32_t *out, cudaStream_t s) {
    if (nseg <= 0) return;
    int64_t grid = std::min<int64_t>(cdiv(nseg * 32, 256), 148 * 32);
    k_seg_unique<<<(unsigned)grid, 256, 0, s>>>(vals, ptr, nseg, optr, out);
    CK_LAUNCH();
}

// ----------------------------------------------------------------------------- CSR transpose
namespace {
__global__ void k_count_cols(const int32_t *idx, int64_t nnz, int32_t *cnt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[idx[j]], 1);
}
__global__ void k_fill_transpose(const int64_t *ptr, const int32_t *idx, int64_t nr,
                                 const int64_t *tptr, int32_t *cursor, int32_t *tidx) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t j = ptr[r]; j < ptr[r + 1]; j++) {
            int32_t c = idx[j];
            int32_t pos = atomicAdd(&cursor[c], 1);
            tidx[tptr[c] + pos] = (int32_t)r;
        }
    }
}
}  // namespace

void csr_transpose(const int64_t *ptr, const int32_t *idx, int64_t nr, int64_t nnz, int64_t nc,
                   DBuf<int64_t> &tptr, DBuf<int32_t> &tidx, int *err, cudaStream_t s) {
    DBuf<int32_t> cnt;
    cnt.alloc(std::max<int64_t>(nc, 1), s);
    cnt.zero(s);
    if (nnz > 0) {
        k_count_cols<<<(unsigned)std::min<int64_t>(cdiv(nnz, 256), 148 * 16), 256, 0, s>>>(idx, nnz,
                                                                                          cnt.p);
        CK_LAUNCH();
    }
    tptr.alloc(nc + 1, s);
    exclusive_scan_i32(cnt.p, tptr.p, nc, s);
    tidx.alloc(std::max<int64_t>(nnz, 1), s);
    cnt.zero(s);
    if (nr > 0) {
        k_fill_transpose<<<(unsigned)std::min<int64_t>(cdiv(nr, 256), 148 * 16), 256, 0, s>>>(
            ptr, idx, nr, tptr.p, cnt.p, tidx.p);
        CK_LAUNCH();
    }
    seg_sort(tidx.p, tptr.p, nc, nullptr, err, s);
}

// ----------------------------------------------------------------------------- global sort
namespace {
__global__ void k_bitonic_step(uint64_t *a, int64_t npow, int64_t n, int64_t j, int64_t k) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npow;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = i ^ j;
        if (l > i) {
            uint64_t ai = (i < n) ? a[i] : ~0ull;
            uint64_t al = (l < n) ? a[l] : ~0ull;
            bool up = ((i & k) == 0);
            if ((up && ai > al) || (!up && ai < al)) {
                if (i < n) a[i] = al;
                if (l < n) a[l] = ai;
            }
        }
    }
}
}  // namespace

void sort_u64(uint64_t *keys, int64_t n, cudaStream_t s) {
    if (n <= 1) return;
    int64_t npow = 1;
    while (npow < n) npow <<= 1;
    // Padding positions (>= n) behave as +infinity and never swap into [0, n): in the
    // final ascending merges they stay at the tail; in intermediate descending runs the
    // network may move them, so they are materialised in a padded copy.
    DBuf<uint64_t> buf;
    buf.alloc(npow, s);
    CK(cudaMemsetAsync(buf.p, 0xff, npow * sizeof(uint64_t), s));
    CK(cudaMemcpyAsync(buf.p, keys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    unsigned grid = (unsigned)std::min<int64_t>(cdiv(npow, 256), 148 * 16);
    for (int64_t k = 2; k <= npow; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            k_bitonic_step<<<grid, 256, 0, s>>>(buf.p, npow, npow, j, k);
            CK_LAUNCH();
        }
    CK(cudaMemcpyAsync(keys, buf.p, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
}

// ----------------------------------------------------------------------------- reductions
namespace {
__global__ void k_max_i32(const int32_t *d, int64_t n, int32_t *out) {
    int32_t m = INT32_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, d[i]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
__global__ void k_sum_i64(const int64_t *d, int64_t n, unsigned long long *out) {
    long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m += d[i];
    for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)m);
}
}  // namespace

int32_t max_i32(const int32_t *d, int64_t n, cudaStream_t s) {
    DBuf<int32_t> o;
    o.alloc(1, s);
    int32_t init = INT32_MIN;
    CK(cudaMemcpyAsync(o.p, &init, 4, cudaMemcpyHostToDevice, s));
    if (n > 0) {
        k_max_i32<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 1184), 256, 0, s>>>(d, n, o.p);
        CK_LAUNCH();
    }
    return read1(o.p, s);
}

int64_t sum_i64(const int64_t *d, int64_t n, cudaStream_t s) {
    DBuf<unsigned long long> o;
    o.alloc(1, s);
    o.zero(s);
    if (n > 0) {
        k_sum_i64<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 1184), 256, 0, s>>>(d, n, o.p);
        CK_LAUNCH();
    }
    return (int64_t)read1(o.p, s);
}

}  // namespace lsamg
