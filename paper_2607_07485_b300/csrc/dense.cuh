// Batched variable-size FP64 dense linear algebra used by the local spectral problems
// (Section 2 eq. 2.9), the Schwarz factors and the coarsest factorisation.
// Matrices are column-major views (off, ld, n) into one device base array.
#pragma once
#include "common.cuh"

namespace lsamg {

struct MatBatch {
    DBuf<int64_t> off;  // element offset of each matrix view
    DBuf<int32_t> ld;   // leading dimension
    DBuf<int32_t> n;    // rows (= columns for square views)
    DBuf<int32_t> m;    // extra dimension (columns of a right-hand side, K of an update)
    int64_t count = 0;
    int32_t maxn = 0, maxm = 0;
    std::vector<int32_t> h_n, h_m;  // host copies of the sizes (FLOP accounting, product jobs)
    std::vector<int64_t> h_off;     // host copies of the offsets and leading dimensions
    std::vector<int32_t> h_ld;
    void set(const std::vector<int64_t> &o, const std::vector<int32_t> &l,
             const std::vector<int32_t> &nn, const std::vector<int32_t> &mm, cudaStream_t s) {
        count = (int64_t)o.size();
        upload(off, o, s);
        upload(ld, l, s);
        upload(n, nn, s);
        std::vector<int32_t> m2 = mm.empty() ? std::vector<int32_t>(o.size(), 0) : mm;
        upload(m, m2, s);
        h_n = nn;
        h_m = m2;
        h_off = o;
        h_ld = l;
        maxn = 0;
        maxm = 0;
        for (auto v : nn) maxn = std::max(maxn, v);
        for (auto v : m2) maxm = std::max(maxm, v);
    }
};

enum PotrfMode { POTRF_SPD = 0, POTRF_PSD = 1 };

// In-place lower Cholesky A = L L^T of each view (upper triangle left untouched).
// POTRF_SPD: a non-positive pivot flags LSAMG_SINGULAR.  POTRF_PSD: pivots below
// n*eps*max(diag) are treated as zero (column zeroed), giving a generalised inverse in the
// triangular solves below (used for the pseudo-inverse of the interface block).
void potrf_batched(double *base, const MatBatch &A, PotrfMode mode, int *err, cudaStream_t s);

// Pivoted (rank-revealing) Cholesky of a diagonal block of each view, LAPACK pstrf style:
// P A_bb P^T = L L^T with diagonal pivoting, stopping when the largest remaining diagonal is
// <= 10 * eps * max(diag); the trailing pivots are set to zero (generalised inverse in the
// triangular solves).  The block starts at row/column `b0[i]` of view i and has order bn[i];
// row and column swaps are applied to the whole view (order nfull[i]) so that the coupling
// blocks are permuted consistently.  perm receives the pivot order (block-local), rank the
// numerical rank.
void pstrf_batched(double *base, const MatBatch &A, const int32_t *b0, const int32_t *bn,
                   const std::vector<int32_t> &h_b0, const std::vector<int32_t> &h_bn,
                   int32_t max_bn, int32_t *perm, const int64_t *permoff, int32_t *rank,
                   int *err, cudaStream_t s);

// X = L^{-1} B (trans = false) or X = L^{-T} B (trans = true), in place on B.
// L views in Lb (n = order), B views in Bb (n = rows = order, m = columns).
// Zero diagonal entries of L (PSD mode) give zero solution rows.
void trsm_batched(const double *base_L, const MatBatch &Lb, double *base_B, const MatBatch &Bb,
                  bool trans, cudaStream_t s, int *err = nullptr);

// C += alpha W^T W over the full square C (n x n, column-major, ld); W views (n = K rows,
// m = columns = C order).  W(k, i) is base_W[off + k + i*ld] (column-major) or, with
// w_rowmajor, base_W[off + k*ld + i].
void syrk_tn_batched(double *base_C, const MatBatch &Cb, const double *base_W, const MatBatch &Wb,
                     double alpha, bool w_rowmajor, cudaStream_t s, int *err = nullptr);

// dst = src^T for square views (src n x n -> dst n x n).
void transpose_batched(const double *base_S, const MatBatch &Sb, double *base_D, const MatBatch &Db,
                       cudaStream_t s);

// Householder tridiagonalisation of the lower triangle (LAPACK sytd2 convention): d, e, tau at
// toff[i] (lengths n, n-1, n-1); reflector j stored below the subdiagonal of column j.
void sytd2_batched(double *base, const MatBatch &Ab, double *d, double *e, double *tau,
                   const int64_t *toff, cudaStream_t s);

// Eigenvalues below sigma of each tridiagonal (Sturm bisection, ascending): count k[i],
// values w[toff[i] ..], and gap[i] = min over all eigenvalues of |lambda / sigma - 1| using the
// two eigenvalues adjacent to sigma.
void stebz_batched(const double *d, const double *e, const int64_t *toff, const int32_t *n,
                   int64_t count, double sigma, int32_t *k, double *w, double *gap,
                   cudaStream_t s);

// Eigenvectors of the tridiagonals for w[toff[i]..+k[i]) by inverse iteration (one thread per
// eigenvalue over the batch), into V views (n rows, k columns); not orthogonalised.
void stein_batched(const double *d, const double *e, const int64_t *toff, const int32_t *n,
                   const double *w, const int32_t *k, double *base_V, const MatBatch &Vb, cudaStream_t s);

// Rectangular transpose: D (m x n, column-major, ld_d) = S^T with S n x m (column-major, ld_s);
// S views: n = rows, m = columns; D views: ld only.
void transpose_rect_batched(const double *base_S, const MatBatch &Sb, double *base_D, const MatBatch &Db,
                            cudaStream_t s);

// Orthonormalise the columns of each V (n x k, column-major) in place by CholeskyQR2 (two
// passes of G = V^T V = L L^T, V <- V L^{-T}; the first pass with a small diagonal shift).
void cholqr2_batched(double *base_V, const MatBatch &Vb, int *err, cudaStream_t s);

// V = Q V with Q the product of the sytd2 reflectors stored in A.
void ormtr_batched(const double *base_A, const MatBatch &Ab, const double *tau, const int64_t *toff,
                   double *base_V, const MatBatch &Vb, cudaStream_t s, int *err = nullptr);

}  // namespace lsamg
