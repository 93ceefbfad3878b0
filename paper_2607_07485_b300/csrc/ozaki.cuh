// FP64 matrix products on the FP16 tensor cores by exact operand splitting (Ozaki's scheme).
//
// B300's FP64 pipes (DFMA and the FP64 MMA) deliver about 1 TFLOP/s, while its fifth-generation
// tensor cores run FP16 products with FP32 accumulation at over 2 PFLOP/s.  Every FP64 update of
// the set-up (Cholesky trailing updates, triangular-solve updates, Gram products, the
// tridiagonal reduction's rank-2k updates, back-transformations) is therefore computed as
// follows.
//
//   * Each row i of an operand is scaled by 2^-e_i (e_i: the exponent of the row's largest
//     entry, so |x| < 1) and cut into NS integer slices by round-to-nearest:
//         x = 2^-7 (a_1 + 2^-8 a_2 + ... + 2^-8(NS-1) a_NS) + r,   |a_p| <= 128,
//     each a_p exact in FP16.  NS = 7 slices hold 56 bits, more than the 53 of an FP64 entry.
//   * sum_k A_ik B_jk = 2^(e_i + f_j - 14) sum_d 2^-8(d-2) S_d,  S_d = sum_{p+q=d} sum_k a_p b_q.
//     Pairs with p + q <= ND = 8 are kept (28 products); the first dropped diagonal weighs
//     2^-56 relative to the leading one, below FP64 rounding of the result.
//   * S_d is accumulated by tcgen05.mma (FP16 x FP16 -> FP32, accumulator in tensor memory) over
//     K pieces of 128: every partial sum is an integer below 7 * 128 * 2^14 < 2^24, so the FP32
//     accumulation is exact.  After each piece the sums move into two 64-bit integers per
//     output, and the epilogue rounds the exact total to FP64 once.
//
// The error of an entry is at most a few units of 2^-53 times K max_k|A_ik| max_k|B_jk|, the
// same order as an FP64 dot product's normwise bound.
//
// Operands are staged per (slice, 64-row tile, 32-wide K chunk) as 4 KB blocks, pre-swizzled in
// global memory (the 64-byte-swizzle K-major layout of the tensor-core shared-memory
// descriptors), so that one 1-D bulk copy (cp.async.bulk, completion on an mbarrier) lands a
// block in shared memory ready for the tensor cores.
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace lsamg {
namespace oz {

constexpr int TM = 64;             // rows of a slice block and of a C tile
constexpr int TK = 32;             // K chunk
constexpr int BLK = TM * TK;       // halves per block (4 KB)
constexpr int NS = 7;              // slices per operand entry
constexpr int ND = 8;              // highest kept diagonal p + q

// One operand: `rows` rows of length K; element (i, k) at src[src_off + i * rs + k * ks].
struct SplitJob {
    int64_t src_off, rs, ks;
    int64_t dst_off;   // halves: NS * tiles * chunks blocks of BLK
    int64_t exp_off;   // ints: tiles * TM
    int32_t rows, K;
};

// C (M x N) = beta C + alpha A B^T with A, B split operands of the same K.  C element (i, j) at
// C[c_off + i * crs + j * ccs]; lower != 0: only i >= j is written (tiles above the diagonal
// are skipped).
struct GemmJob {
    int64_t a_off, b_off;        // slice storage (halves) of A and B
    int64_t a_exp, b_exp;        // exponent storage (ints)
    int64_t c_off, crs, ccs;
    int32_t M, N, K, lower;
    int32_t skip_idx, pad_;      // the job is skipped when skip != nullptr and skip[skip_idx] >= 0
    int32_t k0 = 0, ktot = 0;    // set by gemm(): first K index (0) and the operands' K
};

// 64-row blocks stored per slice and K chunk: rounded up to an even count, so that a 128-row
// operand tile of the tensor-core product always reads stored (zero-padded) rows.
__host__ __device__ inline int64_t stor_tiles(int64_t rows) {
    return 2 * (((rows > 1 ? rows : 1) + 2 * TM - 1) / (2 * TM));
}
// Slice storage needed for an operand of `rows` x K: (halves, exponent ints).
inline int64_t slice_halves(int64_t rows, int64_t K) {
    return (int64_t)NS * stor_tiles(rows) * cdiv(std::max<int64_t>(K, 1), TK) * BLK;
}
inline int64_t exp_ints(int64_t rows) { return stor_tiles(rows) * TM; }

// Split the operands of `jobs` (host vector) from `src` into `dst` / `exps`.
void split(const double *src, const std::vector<SplitJob> &jobs, __half *dst, int32_t *exps, cudaStream_t s);

// Run the products of `jobs`.  `err` receives LSAMG_DEVICE_TIMEOUT if a pipeline wait gives up.
void gemm(const __half *slices, const int32_t *exps, double *C, const std::vector<GemmJob> &jobs,
          double alpha, double beta, int *err, cudaStream_t s, const int32_t *skip = nullptr);

// A reusable device workspace for split operands (grown on demand, stream-ordered).
struct Workspace {
    DBuf<__half> sl;
    DBuf<int32_t> ex;
    void reserve(int64_t halves, int64_t ints, cudaStream_t s) {
        if (sl.size() < halves) sl.alloc(halves, s);
        if (ex.size() < ints) ex.alloc(ints, s);
    }
};

}  // namespace oz
}  // namespace lsamg
