"""The FP64 matrix product on the FP16 tensor cores (lsamg_dgemm_nt), which carries every dense
update of the set-up, against an extended-precision product on the host: exact on integer
operands, within the FP64 normwise dot-product bound on random and graded operands, for ragged
shapes (M, N not multiples of the 128 x 32 product tile, K not a multiple of 32) and for long K
(many 128-wide accumulation pieces carried in 64-bit integers)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_07485_b300 import dgemm_nt  # noqa: E402

DEV = "cuda:0"
U = 2.0 ** -53


def _ref(A, B):
    return (A.astype(np.longdouble) @ B.astype(np.longdouble).T)


def _bound(A, B):
    # a few units of 2^-53 K max_k|A_ik| max_k|B_jk|
    K = A.shape[1]
    return 8 * U * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]


def _run(A, B, C=None, alpha=1.0, beta=0.0):
    c = None if C is None else torch.from_numpy(C).to(DEV)
    out = dgemm_nt(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), c, alpha, beta)
    return out.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 32), (130, 70, 45), (200, 333, 257), (5, 700, 1000)])
def test_random_within_fp64_bound(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    got = _run(A, B)
    err = np.abs(got - _ref(A, B)).astype(np.float64)
    assert np.all(err <= _bound(A, B)), err.max()


def test_integer_operands_exact():
    rng = np.random.default_rng(3)
    # 21-bit integers: every slice product and sum is exact, so is the FP64 result (< 2^53)
    A = rng.integers(-2 ** 20, 2 ** 20, size=(150, 300)).astype(np.float64)
    B = rng.integers(-2 ** 20, 2 ** 20, size=(90, 300)).astype(np.float64)
    A[0, :] = 2 ** 20 - 1       # largest magnitudes: the FP32 sums reach their bound
    B[0, :] = 2 ** 20 - 1
    A[1, :] = -(2 ** 20)
    got = _run(A, B)
    np.testing.assert_array_equal(got, (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float64))


def test_graded_rows_and_alpha_beta():
    rng = np.random.default_rng(5)
    M, N, K = 96, 80, 200
    A = rng.standard_normal((M, K)) * np.logspace(-12, 0, K)[None, :]     # entries over 12 decades
    B = rng.standard_normal((N, K)) * np.logspace(0, -9, K)[None, :]
    A[3] *= 1e-200                                                      # tiny row: its own scale
    C0 = rng.standard_normal((M, N))
    got = _run(A, B, C0.copy(), alpha=-0.5, beta=2.0)
    ref = 2.0 * C0.astype(np.longdouble) - 0.5 * _ref(A, B)
    err = np.abs(got - ref).astype(np.float64)
    assert np.all(err <= 0.5 * _bound(A, B) + 4 * U * np.abs(ref).astype(np.float64)), err.max()
    assert np.abs(got[3] - 2.0 * C0[3]).max() <= 4 * U * np.abs(C0[3]).max() + 1e-200


def test_beta_zero_ignores_c_and_long_k_is_split():
    rng = np.random.default_rng(9)
    M, N, K = 70, 65, 20000          # 157 accumulation pieces of K = 128
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C0 = np.full((M, N), np.nan)
    got = _run(A, B, C0, beta=0.0)
    err = np.abs(got - _ref(A, B)).astype(np.float64)
    assert np.isfinite(got).all()
    assert np.all(err <= _bound(A, B)), err.max()


def test_accumulating_product_rounds_once():
    # C = C0 - A B^T with integer data: every exact sum is below 2^53, so the result must be exact
    # (the old C joins the integer sum before the single rounding)
    rng = np.random.default_rng(13)
    A = rng.integers(-2 ** 18, 2 ** 18, size=(200, 96)).astype(np.float64)
    B = rng.integers(-2 ** 18, 2 ** 18, size=(75, 96)).astype(np.float64)
    C0 = rng.integers(-2 ** 44, 2 ** 44, size=(200, 75)).astype(np.float64)
    got = _run(A, B, C0.copy(), alpha=-1.0, beta=1.0)
    ref = C0.astype(np.int64) - A.astype(np.int64) @ B.astype(np.int64).T
    np.testing.assert_array_equal(got, ref.astype(np.float64))
