"""The algebraic A-closure (Def. 5.2) against the G-row closure (Def. 5.3) on the GPU path:
overlaps, and the stationary V-cycle iteration counts of the Table 2 comparison (CG1 triangles,
kappa = 1 + x + y, Nitsche u = 0, tau_cut = max mult, random x0, b = 0, 1e-10 reduction), each
against the oracle on the same seeded input."""
import numpy as np
import pytest

import fegen
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_07485_b300 import Lsamg, LsamgError  # noqa: E402

DEV = "cuda:0"
OPTS = dict(tau_c=1.0)


def _problem(N):
    n, d, K = fegen.cg1_tri(N)
    return n, d, np.ascontiguousarray(K)


def _handle(n, d, K, closure, **extra):
    return Lsamg(n, torch.from_numpy(d).to(DEV), torch.from_numpy(K).to(DEV), closure=closure,
                 **dict(OPTS, **extra))


def _lists(ptr, idx):
    return [idx[ptr[i]:ptr[i + 1]] for i in range(len(ptr) - 1)]


def test_a_closure_is_inside_the_g_row_closure_and_cut_by_cancellation():
    n, d, K = _problem(32)
    hg, ha = _handle(n, d, K, "G"), _handle(n, d, K, "A")
    np.testing.assert_array_equal(hg.query(0, "AGG"), ha.query(0, "AGG"))
    OmG = _lists(hg.query(0, "OMEGA_PTR"), hg.query(0, "OMEGA_IDX"))
    OmA = _lists(ha.query(0, "OMEGA_PTR"), ha.query(0, "OMEGA_IDX"))
    assert all(set(a.tolist()) <= set(g.tolist()) for a, g in zip(OmA, OmG))
    assert sum(len(g) - len(a) for a, g in zip(OmA, OmG)) > 0
    # against the oracle's A-closure on the assembled matrix, every aggregate
    A = O.assemble(n, d, K)
    agg = hg.query(0, "AGG")
    *_, ref = O.closure(d, agg, int(agg.max()) + 1, A=A)
    for i, (a, r) in enumerate(zip(OmA, ref)):
        np.testing.assert_array_equal(a, r, err_msg=f"Omega^A_{i}")
    hg.close()
    ha.close()


@pytest.mark.parametrize("N", [32, 64])
@pytest.mark.parametrize("closure", ["G", "A"])
def test_stationary_iterations_match_oracle(N, closure):
    n, d, K = _problem(N)
    h = _handle(n, d, K, closure, rtol=1e-10, maxit=500)
    H = O.setup(n, d, K, opts=dict(OPTS, closure=closure))
    x0 = np.random.default_rng(N).uniform(-1, 1, n)
    b = np.zeros(n)
    x, its, rel, rc = h.solve(torch.from_numpy(b).to(DEV), x0=torch.from_numpy(x0).to(DEV), mode=2)
    assert rc == 0 and rel[0] <= 1e-10
    _, ito, _ = O.stationary(H, b, x0, rtol=1e-10)
    assert abs(int(its[0]) - ito) <= 1, (int(its[0]), ito)
    h.close()


def test_closure_option_is_checked():
    n, d, K = _problem(4)
    with pytest.raises(ValueError):
        _handle(n, d, K, "X")
    with pytest.raises(LsamgError):
        _handle(n, d, K, 2)
