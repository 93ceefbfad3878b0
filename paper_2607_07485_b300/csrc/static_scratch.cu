// Allocation-free element Gram SpMV, lsamg_gram_spmv_static (include/lsamg.h).  The paper has
// no counterpart: it is a library convenience that computes y = sum_T R_T^T G_T^T (G_T R_T x)
// for callers that cannot allocate device memory: applications whose GPU memory belongs to
// another allocator (a framework's caching pool), and latency-critical loops where
// cudaMalloc / cudaFree would synchronise the device.  It reads the element factors from caller
// buffers and keeps the intermediate t_T = G_T x_T in one file-scope device array instead of
// shared memory, so the call allocates nothing: no cudaMalloc, no cudaFree and no allocating
// library routine.
//
// The array's name is only a host-side stand-in in host code: the first call on each device
// looks up its device address with cudaGetSymbolAddress (that device current) and passes that
// address to the kernels.  Every call reads the error flag back and synchronises its stream, so
// it cannot be captured into a CUDA graph; a call on a capturing stream is rejected up front.
// The array keeps the previous call's contents; only the error flag must start at zero and is
// cleared.
//
// Scratch layout (per device): words [0, 32) a header whose first int is the error flag (set by
// the kernels for a DOF index outside [0, n_dofs); cleared at the start of every call), words
// [32, LSAMG_STATIC_SCRATCH_WORDS) the values t_T (n_elems * m of them).  Every call on a device
// shares the array, so calls that overlap on that device (other streams, other host threads)
// race; callers serialise them.
#include <mutex>
#include <string>

#include "impl.cuh"

namespace lsamg {
namespace {

constexpr int64_t kScratchWords = LSAMG_STATIC_SCRATCH_WORDS;
constexpr int64_t kHeaderWords = 32;   // 256 bytes: the error flag, then padding

static __device__ __align__(256) double g_static_scratch[kScratchWords];

// address of g_static_scratch on each device, looked up once per device with that device current
std::mutex g_scratch_mu;
double *g_scratch_ptr[64] = {};

double *scratch_for_current_device() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(LSAMG_LIMIT, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&p, g_static_scratch);
        if (rc != cudaSuccess || p == nullptr)
            fail(LSAMG_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                 cudaGetErrorString(rc));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    return g_scratch_ptr[dev];
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// t[e m + i] = sum_c G_e[i, c] x[dofs_e[c]]: a warp per (element, row), lanes over the columns
__global__ void k_static_rows(const int32_t *dofs, const double *G, const double *x, int64_t n, int64_t ne,
                              int nT, int m, double *t, int *flag) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < ne * m; q += nw) {
        const int64_t e = q / m;
        const double *g = G + q * nT;
        const int32_t *d = dofs + e * nT;
        double s = 0.0;
        for (int c = lane; c < nT; c += 32) {
            const int32_t j = d[c];
            if (j >= 0 && j < n) s += g[c] * x[j]; else atomicExch(flag, 1);
        }
        s = warp_sum_d(s);
        if (lane == 0) t[q] = s;
    }
}

// the same with a thread per (element, row), for small elements (n_T <= 16), where a warp over
// the columns would leave most lanes idle
__global__ void k_static_rows_thread(const int32_t *dofs, const double *G, const double *x, int64_t n,
                                     int64_t ne, int nT, int m, double *t, int *flag) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ne * m;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / m;
        const double *g = G + q * nT;
        const int32_t *d = dofs + e * nT;
        double s = 0.0;
        for (int c = 0; c < nT; c++) {
            const int32_t j = d[c];
            if (j >= 0 && j < n) s += g[c] * x[j]; else atomicExch(flag, 1);
        }
        t[q] = s;
    }
}

// y[dofs_e[c]] += sum_i G_e[i, c] t[e m + i]: a thread per (element, column)
__global__ void k_static_cols(const int32_t *dofs, const double *G, const double *t, int64_t n, int64_t ne,
                              int nT, int m, double *y, int *flag) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ne * nT;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / nT;
        const int c = (int)(q - e * nT);
        const double *g = G + e * m * nT + c;
        const double *te = t + e * m;
        double s = 0.0;
        for (int i = 0; i < m; i++) s += g[(int64_t)i * nT] * te[i];
        const int32_t j = dofs[q];
        if (j >= 0 && j < n) atomicAdd(&y[j], s); else atomicExch(flag, 1);
    }
}

unsigned grid_for(int64_t items, int per) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(items, per), 148 * 16));
}

}  // namespace
}  // namespace lsamg

extern "C" int lsamg_gram_spmv_static(int64_t n_dofs, int64_t n_elems, int32_t n_T, int32_t m,
                                      const int32_t *elem_dofs, const double *G, const double *x, double *y,
                                      void *stream) {
    using namespace lsamg;
    const int64_t cap = kScratchWords - kHeaderWords;
    if (n_dofs < 0 || n_elems < 0 || n_T < 1 || m < 0) {
        set_last_error("lsamg_gram_spmv_static: negative size or n_T < 1");
        return LSAMG_INVALID_ARG;
    }
    if (m > 0 && n_elems > cap / m) {
        set_last_error("lsamg_gram_spmv_static: n_elems * m = " + std::to_string(n_elems) + " * " +
                       std::to_string(m) + " exceeds the static scratch of " + std::to_string(cap) +
                       " doubles");
        return LSAMG_LIMIT;
    }
    if ((n_dofs > 0 && (!x || !y)) || (n_elems > 0 && (!elem_dofs || (m > 0 && !G)))) {
        set_last_error("lsamg_gram_spmv_static: null pointer");
        return LSAMG_INVALID_ARG;
    }
    try {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(s, &capst));
        if (capst != cudaStreamCaptureStatusNone) {
            set_last_error("lsamg_gram_spmv_static: the stream is capturing; this call synchronises and "
                           "cannot be captured");
            return LSAMG_INVALID_ARG;
        }
        double *base = scratch_for_current_device();
        int *flag = reinterpret_cast<int *>(base);
        double *t = base + kHeaderWords;
        CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
        if (n_dofs > 0) CK(cudaMemsetAsync(y, 0, (size_t)n_dofs * sizeof(double), s));
        if (n_elems > 0 && m > 0) {
            if (n_T <= 16)
                k_static_rows_thread<<<grid_for(n_elems * m, 256), 256, 0, s>>>(elem_dofs, G, x, n_dofs, n_elems,
                                                                              n_T, m, t, flag);
            else
                k_static_rows<<<grid_for(n_elems * m * 32, 256), 256, 0, s>>>(elem_dofs, G, x, n_dofs, n_elems, n_T,
                                                                              m, t, flag);
            CK_LAUNCH();
            k_static_cols<<<grid_for(n_elems * n_T, 256), 256, 0, s>>>(elem_dofs, G, t, n_dofs, n_elems, n_T, m,
                                                                      y, flag);
            CK_LAUNCH();
        }
        int h_flag = 0;
        CK(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h_flag) {
            set_last_error("lsamg_gram_spmv_static: a DOF index is outside [0, n_dofs)");
            return LSAMG_INVALID_ARG;
        }
    } catch (const Failure &e) {
        set_last_error(e.msg);
        return e.code;
    }
    set_last_error("");
    return LSAMG_OK;
}
