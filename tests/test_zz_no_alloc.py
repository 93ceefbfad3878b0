"""The allocation-free Gram SpMV (lsamg_gram_spmv_static), for callers that must not allocate
device memory (GPU memory owned by another allocator, or latency-critical loops where
cudaMalloc would synchronise the device), against the handle's Gram SpMV (lsamg_gram_spmv) on
the same element factors.  It makes two calls in a row through the one static scratch array
(which keeps the previous call's contents), on two element families, and checks the size
limit.  Self-contained (it builds its own handles), so it passes alone in a fresh process and
after the other tests; the file sorts last so that a stop-at-first-failure run has already
run every other test."""
import numpy as np
import pytest

import fegen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_07485_b300 import Lsamg, LsamgError, gram_spmv_static  # noqa: E402

DEV = "cuda:0"
SCRATCH_WORDS = 1 << 20


def _padded_factors(amg):
    """Level-0 element maps and Gram factors read back from the handle, each G_T padded with
    zero rows to the largest row count m."""
    eptr, eidx = amg.query(0, "EPTR"), amg.query(0, "EIDX")
    goff, grows, G = amg.query(0, "GOFF"), amg.query(0, "GROWS"), amg.query(0, "G")
    ne = len(eptr) - 1
    nT = int(eptr[1] - eptr[0])
    m = int(grows.max())
    dofs = eidx.reshape(ne, nT).astype(np.int32)
    Gp = np.zeros((ne, m, nT))
    for e in range(ne):
        Gp[e, :grows[e]] = G[goff[e]:goff[e] + grows[e] * nT].reshape(grows[e], nT)
    return dofs, Gp


@pytest.mark.parametrize("cfg", [1, 3])
def test_static_scratch_matches_gram_spmv(cfg):
    c = fegen.config(cfg, N=16)
    mats = c["elem_mats"] if c["coef"] is None else c["elem_mats"] * c["coef"][:, None, None]
    amg = Lsamg(c["n"], torch.from_numpy(c["elem_dofs"]).to(DEV),
                torch.from_numpy(np.ascontiguousarray(mats)).to(DEV), tau_c=c["c_tau"])
    dofs, Gp = _padded_factors(amg)
    assert dofs.shape[0] * Gp.shape[1] <= SCRATCH_WORDS - 32
    d_dofs = torch.from_numpy(dofs).to(DEV)
    d_G = torch.from_numpy(Gp).to(DEV)
    rng = np.random.default_rng(77 + cfg)
    y = torch.empty(c["n"], dtype=torch.float64, device=DEV)
    for call in range(2):   # two calls in a row share the scratch
        x = torch.from_numpy(rng.standard_normal(c["n"])).to(DEV)
        ref = amg.gram_spmv(x, level=0).cpu().numpy()
        y.fill_(np.nan)
        got = gram_spmv_static(d_dofs, d_G, x, y).cpu().numpy()
        scale = np.abs(ref).max()
        # FP64, same products, atomics in a different order: agreement to a few ulps of the scale
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * scale,
                                   err_msg=f"cfg {cfg} call {call}")
    amg.close()


def test_static_scratch_rejects_oversize():
    x = torch.zeros(8, dtype=torch.float64, device=DEV)
    y = torch.zeros(8, dtype=torch.float64, device=DEV)
    dofs = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
    G = torch.zeros((1, 2, 4), dtype=torch.float64, device=DEV)
    from paper_2607_07485_b300 import lsamg as LB
    # size check only (no launch): claim more element rows than the scratch holds
    rc = LB._lib.lsamg_gram_spmv_static(8, SCRATCH_WORDS, 4, 2, LB._ptr(dofs), LB._ptr(G), LB._ptr(x),
                                        LB._ptr(y), LB._stream(None))
    assert rc == 9   # LSAMG_LIMIT
    assert b"exceeds the static scratch" in LB._lib.lsamg_last_error()
    with pytest.raises(LsamgError):
        gram_spmv_static(torch.full((1, 4), 99, dtype=torch.int32, device=DEV), G, x, y)
