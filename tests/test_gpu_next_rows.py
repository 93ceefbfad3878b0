"""GPU parity for the additive Schwarz smoother (option smoother=1, the parallel block smoother
Section 2 allows) and the stationary V-cycle solve mode (mode 2, the standalone iteration of
the Section 6 tests), against the oracle's ``vcycle(smoother="additive")`` and ``stationary``;
CUDA-graph replay of the V-cycle against eager launches; the tile-shape autotuner on the GPU."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import CASES, DEV, case  # noqa: E402


def _handle(name, **extra):
    from paper_2607_07485_b300 import Lsamg
    p, H, _, ptol, vtol, band = case(name)
    o = dict(CASES[name][1])
    if "tau_c" not in o and "c_tau" in p:
        o["tau_c"] = p["c_tau"]
    o.update(extra)
    amg = Lsamg(p["n"], torch.from_numpy(p["elem_dofs"]).to(DEV), torch.from_numpy(p["mats"]).to(DEV), **o)
    return p, H, amg, vtol


@pytest.mark.parametrize("name", ["rt1_beta1", "cfg1", "cfg3_16"])
def test_additive_vcycle_matches_oracle(name):
    p, H, amg, vtol = _handle(name, smoother=1)
    r = np.random.default_rng(21).standard_normal(p["n"])
    z = amg.apply(torch.from_numpy(r).to(DEV), fp32=0).cpu().numpy()
    zo = O.vcycle(H, r, smoother="additive")
    assert np.linalg.norm(z - zo) <= vtol * np.linalg.norm(zo)
    amg.close()


# Residual-reduction target per case, above the FP64 evaluation floor 64 eps || |A| |x| || / ||r_0||
# of its data (rt1_beta1: ~1e-13; cfg1, beta = 1e-4: 5.5e-8, where the oracle's iteration
# stagnates near 2e-10 and never reaches 1e-10).
STATIONARY_RTOL = {"rt1_beta1": 1e-10, "cfg1": 1e-8}


@pytest.mark.parametrize("name", ["rt1_beta1", "cfg1"])
@pytest.mark.parametrize("smoother", [0, 1])
def test_stationary_mode_matches_oracle(name, smoother):
    import scipy.sparse.linalg as spla
    rtol = STATIONARY_RTOL[name]
    p, H, amg, vtol = _handle(name, smoother=smoother, rtol=rtol, maxit=300)
    n = p["n"]
    b = p["b"][0]
    x0 = np.random.default_rng(22).standard_normal(n)
    x, its, rel, rc = amg.solve(torch.from_numpy(b).to(DEV), x0=torch.from_numpy(x0).to(DEV), mode=2)
    assert rc == 0 and rel[0] <= rtol
    A = H.levels[0].A
    xs = spla.spsolve(A.tocsc(), b)
    xg = x.cpu().numpy()
    # the residual reduction bounds the error by kappa(A) times it; compare residuals
    assert np.linalg.norm(b - A @ xg) <= rtol * np.linalg.norm(b - A @ x0) * 1.01 + 64 * np.finfo(float).eps * \
        np.linalg.norm(abs(A) @ abs(xs))
    xo, ito, _ = O.stationary(H, b, x0, rtol=rtol, smoother="additive" if smoother else "multiplicative")
    assert ito < 500 and abs(int(its[0]) - ito) <= 1
    amg.close()


def test_autotune_on_gpu_returns_options_with_the_same_cycle(tmp_path):
    # tile shapes change rounding only: the tuned handle's V-cycle matches the default's
    from paper_2607_07485_b300 import Lsamg
    from paper_2607_07485_b300.autotune import autotune
    p, H, amg, ptol, vtol, band = case("cfg3_16")
    o = dict(CASES["cfg3_16"][1])
    dofs = torch.from_numpy(p["elem_dofs"]).to(DEV)
    mats = torch.from_numpy(p["mats"]).to(DEV)
    cache = str(tmp_path / "tune.json")
    best = autotune(p["n"], dofs, mats, cache_file=cache, cycles=5, base_opts=o,
                    space={"split_sweep": (16, 128), "sweep_block": (32, 64)})
    assert set(best) == {"large_dense", "split_sweep", "sweep_block"}
    assert autotune(p["n"], dofs, mats, cache_file=cache, base_opts=o) == best
    tuned = Lsamg(p["n"], dofs, mats, **dict(o, **best))
    r = torch.from_numpy(np.random.default_rng(23).standard_normal(p["n"])).to(DEV)
    z1 = tuned.apply(r, fp32=0).cpu().numpy()
    z0 = amg.apply(r, fp32=0).cpu().numpy()
    assert np.linalg.norm(z1 - z0) <= vtol * np.linalg.norm(z0)
    tuned.close()


@pytest.mark.parametrize("name", ["cfg1", "cfg3_16"])
def test_graph_vcycle_matches_eager(name):
    # use_graph=1: first apply captures, later ones replay; a new right-hand-side count re-captures
    p, H, amg, vtol = _handle(name, use_graph=1)
    eager = case(name)[2]
    rng = np.random.default_rng(24)
    r = torch.from_numpy(rng.standard_normal(p["n"])).to(DEV)
    z0 = eager.apply(r, fp32=0).cpu().numpy()
    for _ in range(2):
        z = amg.apply(r, fp32=0).cpu().numpy()
        assert np.linalg.norm(z - z0) <= vtol * np.linalg.norm(z0)
    R = torch.stack([r, 2 * r])
    Z = amg.apply(R, fp32=0).cpu().numpy()
    assert np.linalg.norm(Z[1] - 2 * z0) <= vtol * np.linalg.norm(2 * z0)
    b = torch.from_numpy(p["b"][0]).to(DEV)
    _, its_e, _, rc_e = eager.solve(b, mode=0)
    _, its_g, _, rc_g = amg.solve(b, mode=0)
    assert rc_e == rc_g == 0 and abs(int(its_e[0]) - int(its_g[0])) <= 1
    amg.close()
