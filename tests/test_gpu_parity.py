"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.  Integer results (aggregates, overlaps, multiplicities, mode counts,
colours, coarse element maps) must match bit for bit; floating-point results within the
tolerances stated at each check.

Tolerances (per case in CASES).  Projectors onto span Z_i are held to 1e-8 where two
independent FP64 evaluations of eq. 2.9 from the same element data agree to better than
that; the beta = 1e-6 grad-div data (kappa(A_T) ~ 1e13-1e14) fix the projectors only to ~1e-4,
so there the bar is 1e-3.  Coarse-level quantities are compared in fine-level coordinates
(span of P_0 ... R^T Z_i), which is independent of the rotation freedom of degenerate local
eigenspaces.  Solutions are checked through their residual against the FP64 evaluation floor
eps * || |A| |x| ||.
"""
import numpy as np
import pytest

import fegen
import oracle as O
import oracle.lsamg_oracle as OL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_07485_b300 import Lsamg, LsamgError  # noqa: E402

DEV = "cuda:0"

# name -> (generator, options, projector tolerance, V-cycle tolerance, rank-flip band)
# Projector tolerances: 1e-8 where the data resolve the local spectra (beta = 1, cfg1, cfg3,
# cfg4: two independent FP64 evaluations of eq. 2.9 agree to ~2e-9); 1e-3 for the beta = 1e-6
# grad-div data, whose element blocks have kappa(A_T) ~ 1e13-1e14 so that the beta part of A_T
# carries only ~3 significant digits (independent FP64 evaluations agree to ~1e-4).
# The projector tolerance applies to the difference times delta_i tau (capped at 1), the
# separation of the retained from the discarded eigenvalues (Davis-Kahan).
# Rank-flip band: a mode count may differ only by eigenvalues with |mu tau - 1| < 1e-9, where the
# rank decision is flagged as unstable rather than a parity failure.  The smallest |mu tau - 1|
# of these cases is 0.013 (cfg2_16, cfg5_16), far outside the band: their counts must agree.
BAND = 1e-9
CASES = {
    "rt1_beta1": (lambda: _rt(8, 1, 1.0), dict(agg_passes=1, agg_passes_coarse=1, max_density=1.0), 1e-8, 1e-7, BAND),
    "cfg1": (lambda: _cfg(1, 16), dict(), 1e-8, 1e-6, BAND),
    "cfg2_16": (lambda: _cfg(2, 16), dict(), 1e-3, 1e-2, BAND),
    "cfg3_16": (lambda: _cfg(3, 16), dict(tau_c=1.0), 1e-6, 1e-4, BAND),
    "cfg5_16": (lambda: _cfg(5, 16), dict(), 1e-3, 1e-2, BAND),
    "cfg4_6": (lambda: _cfg(4, 6), dict(agg_passes=1, agg_passes_coarse=1), 1e-8, 1e-6, BAND),
    # CG1 triangles, kappa = 1 + x + y, 1,089 DOFs, tau_cut = max mult (the Table 2 set-up) with
    # the G-row closure and with the algebraic A-closure (Def. 5.2)
    "cg1_G": (lambda: _cg1(32), dict(tau_c=1.0), 1e-8, 1e-6, BAND),
    "cg1_A": (lambda: _cg1(32), dict(tau_c=1.0, closure="A"), 1e-8, 1e-6, BAND),
}


def _cg1(N):
    n, d, K = fegen.cg1_tri(N)
    rng = np.random.default_rng(7)
    return dict(n=n, elem_dofs=d, mats=np.ascontiguousarray(K), b=rng.uniform(-1, 1, (1, n)))


def _rt(N, k, beta):
    n, d, K = fegen.rt_quad(N, k, beta)
    mats = np.ascontiguousarray(np.broadcast_to(K, (d.shape[0],) + K.shape))
    rng = np.random.default_rng(5)
    return dict(n=n, elem_dofs=d, mats=mats, b=rng.uniform(-1, 1, (1, n)))


def _cfg(cfg, N):
    c = fegen.config(cfg, N=N)
    mats = c["elem_mats"] if c["coef"] is None else c["elem_mats"] * c["coef"][:, None, None]
    return dict(n=c["n"], elem_dofs=c["elem_dofs"], mats=np.ascontiguousarray(mats), b=c["b"][:1],
                c_tau=c["c_tau"])


_cache = {}


def case(name):
    if name not in _cache:
        gen, opts, ptol, vtol, band = CASES[name]
        p = gen()
        o = dict(opts)
        if "tau_c" not in o and "c_tau" in p:
            o["tau_c"] = p["c_tau"]
        H = O.setup(p["n"], p["elem_dofs"], p["mats"], opts=o)
        amg = Lsamg(p["n"], torch.from_numpy(p["elem_dofs"]).to(DEV), torch.from_numpy(p["mats"]).to(DEV), **o)
        _cache[name] = (p, H, amg, ptol, vtol, band)
    return _cache[name]


def _csr_lists(ptr, idx):
    return [idx[ptr[i]:ptr[i + 1]] for i in range(len(ptr) - 1)]


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_structure_bit_exact(name):
    p, H, amg, _, _, _ = case(name)
    st = amg.stats()
    assert st["n_levels"] == len(H.levels), (st["n"], [L.n for L in H.levels])
    assert st["n"] == [L.n for L in H.levels]
    for l, L in enumerate(H.levels):
        assert st["nnz"][l] == L.nnz, f"level {l} structural nnz"
        if L.coarsest:
            continue
        np.testing.assert_array_equal(amg.query(l, "AGG"), L.agg, err_msg=f"aggregates level {l}")
        np.testing.assert_array_equal(amg.query(l, "MULT"), L.mult, err_msg=f"mult level {l}")
        assert st["tau"][l] == pytest.approx(L.tau)
        optr, oidx = amg.query(l, "OMEGA_PTR"), amg.query(l, "OMEGA_IDX")
        for i, Om in enumerate(_csr_lists(optr, oidx)):
            np.testing.assert_array_equal(Om, L.Omega[i], err_msg=f"Omega_{i} level {l}")
        # colours depend on the overlaps only (not on the mode counts): always compared
        np.testing.assert_array_equal(amg.query(l, "COLOUR"), L.colour, err_msg=f"colours level {l}")
        kg = amg.query(l, "K")
        band = CASES[name][4]
        flagged = []
        for i in np.flatnonzero(kg != L.k):
            near = int((np.abs(L.mu[i] * L.tau - 1.0) < band).sum())
            assert abs(int(kg[i]) - int(L.k[i])) <= near, \
                f"level {l} aggregate {i}: k {kg[i]} vs {L.k[i]} with {near} eigenvalues in the band"
            flagged.append(int(i))
        if flagged:
            # a flagged (unstable) rank decision renumbers the coarse DOFs after it: the coarse
            # maps of this level and the coarser levels are not comparable
            pytest.skip(f"level {l}: rank decision unstable (|mu tau - 1| < {band}) at aggregates {flagged}")
        # next level's element maps (merged coarse elements) and the element -> group map
        cptr, cidx = amg.query(l, "CELEM_PTR"), amg.query(l, "CELEM_IDX")
        C = H.levels[l + 1]
        assert len(cptr) - 1 == len(C.elems)
        for g, cm in enumerate(_csr_lists(cptr, cidx)):
            np.testing.assert_array_equal(cm, C.elems[g])
        cg = amg.query(l, "CGROUP")
        ref = np.full(len(L.elems), -1)
        for g, members in enumerate(L.cgroups):
            ref[members] = g
        np.testing.assert_array_equal(cg, ref)


@pytest.mark.parametrize("name", list(CASES))
def test_two_handles_bit_identical(name):
    """The set-up is deterministic: a second handle on the same input reproduces every integer
    structure and every interpolation value bit for bit (no atomics in any summation that feeds
    the local eigenproblems)."""
    p, H, amg, _, _, _ = case(name)
    o = dict(CASES[name][1])
    if "tau_c" not in o and "c_tau" in p:
        o["tau_c"] = p["c_tau"]
    other = Lsamg(p["n"], torch.from_numpy(p["elem_dofs"]).to(DEV), torch.from_numpy(p["mats"]).to(DEV), **o)
    st = amg.stats()
    assert other.stats()["n"] == st["n"]
    for l in range(st["n_levels"]):
        for what in ("EPTR", "EIDX", "GROWS", "G"):
            np.testing.assert_array_equal(other.query(l, what), amg.query(l, what), err_msg=f"{what} level {l}")
        if l == st["n_levels"] - 1:
            continue
        for what in ("AGG", "K", "COLOUR", "CELEM_PTR", "CELEM_IDX", "Z"):
            np.testing.assert_array_equal(other.query(l, what), amg.query(l, what), err_msg=f"{what} level {l}")
    other.close()


@pytest.mark.parametrize("name", list(CASES))
def test_element_gram_factors(name):
    p, H, amg, _, _, _ = case(name)
    for l, L in enumerate(H.levels):
        goff, grows, G = amg.query(l, "GOFF"), amg.query(l, "GROWS"), amg.query(l, "G")
        eptr = amg.query(l, "EPTR")
        for e in range(len(L.elems)):
            nT = eptr[e + 1] - eptr[e]
            Ge = G[goff[e]:goff[e] + grows[e] * nT].reshape(grows[e], nT)
            Ae = L.mats[e]
            scale = np.abs(Ae).max() if l == 0 else np.linalg.norm(Ae, 2)
            if l == 0:
                np.testing.assert_allclose(Ge.T @ Ge, Ae, rtol=0, atol=1e-12 * scale,
                                           err_msg=f"G_T^T G_T != A_T, element {e}")


def _projector(Z):
    if Z.shape[1] == 0:
        return np.zeros((Z.shape[0], Z.shape[0]))
    Q, _ = np.linalg.qr(Z)
    return Q @ Q.T


def _oracle_prolong(H, l):
    """Product P_0 P_1 ... P_{l-1} of the oracle hierarchy (identity for l = 0)."""
    import scipy.sparse as sp
    M = sp.identity(H.levels[0].n, format="csr")
    for j in range(l):
        M = M @ H.levels[j].P
    return M


def _separation(L, i):
    """delta_i tau capped at 1: distance between the largest retained and the smallest discarded
    eigenvalue of eq. 2.9 for aggregate i, in units of the cutoff 1/tau.  By the Davis-Kahan
    sin-Theta bound a perturbation E of the local problem moves the projector onto the retained
    eigenspace by at most ||E|| / delta, so the projector tolerance is divided by it."""
    return _sep(L.mu[i], int(L.k[i]), L.tau)


def _sep(mu, k, tau):
    mu = np.sort(np.asarray(mu, float))
    if k == 0 or k >= len(mu):
        return 1.0
    return float(min(1.0, (mu[k] - mu[k - 1]) * tau))


@pytest.mark.parametrize("name", list(CASES))
def test_interpolation_projectors(name):
    p, H, amg, ptol, _, band = case(name)
    Pg = None   # library's prolongation P_0 ... P_{l-1}
    for l, L in enumerate(H.levels):
        if L.coarsest:
            continue
        zoff, Z, kg = amg.query(l, "ZOFF"), amg.query(l, "Z"), amg.query(l, "K")
        Po = _oracle_prolong(H, l)
        worst = 0.0
        for i in range(L.nagg):
            nw, k = len(L.omega[i]), int(kg[i])
            Zg = Z[zoff[i]:zoff[i + 1]].reshape(nw, k)
            if k != L.k[i]:
                continue  # rank flip inside the band (checked in the structure test)
            w = L.omega[i]
            if l == 0:
                A, B = Zg, L.Z[i]
            else:   # compare the fine-level images, invariant to coarse-basis rotations
                A = Pg[:, w] @ Zg
                B = Po[:, w] @ L.Z[i]
            d = np.linalg.norm(_projector(A) - _projector(B), 2) * _separation(L, i)
            worst = max(worst, d)
        assert worst <= ptol, f"level {l}: gap-scaled projector difference {worst:.3e} > {ptol:.1e}"
        if (kg != L.k).any():
            break
        Pl = gpu_P(amg, l, L.n)
        Pg = Pl if Pg is None else (Pg @ Pl)
        Pg = Pg.toarray() if hasattr(Pg, "toarray") else Pg


def gpu_level_matrix(amg, l, n):
    """Assembled operator of level l from the library's own element maps and Gram blocks."""
    import scipy.sparse as sp
    eptr, eidx = amg.query(l, "EPTR"), amg.query(l, "EIDX")
    goff, grows, G = amg.query(l, "GOFF"), amg.query(l, "GROWS"), amg.query(l, "G")
    rows, cols, vals = [], [], []
    for e in range(len(eptr) - 1):
        d = eidx[eptr[e]:eptr[e + 1]]
        nT = len(d)
        Ge = G[goff[e]:goff[e] + grows[e] * nT].reshape(grows[e], nT)
        Ae = Ge.T @ Ge
        rows.append(np.repeat(d, nT)); cols.append(np.tile(d, nT)); vals.append(Ae.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def gpu_P(amg, l, n):
    """Interpolation P of level l from the library's aggregates and Z blocks."""
    import scipy.sparse as sp
    agg, k, zoff, Z = amg.query(l, "AGG"), amg.query(l, "K"), amg.query(l, "ZOFF"), amg.query(l, "Z")
    off = np.concatenate([[0], np.cumsum(k)])
    rows, cols, vals = [], [], []
    for i in range(len(k)):
        w = np.flatnonzero(agg == i)
        Zi = Z[zoff[i]:zoff[i + 1]].reshape(len(w), k[i])
        rows.append(np.repeat(w, k[i])); cols.append(np.tile(np.arange(off[i], off[i + 1]), len(w)))
        vals.append(Zi.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, off[-1]))


@pytest.mark.parametrize("name", list(CASES))
def test_gram_spmv_and_galerkin(name):
    # level 0: G^T G x against the oracle's assembled A; coarser levels: the library's coarse
    # Gram must satisfy A_c = P^T A P = (G P)^T (G P) (Section 2) for its own P, and its SpMV
    # must apply that operator (the coarse basis itself is fixed only up to rotations)
    p, H, amg, _, _, _ = case(name)
    st = amg.stats()
    rng = np.random.default_rng(3)
    A_prev = None
    for l in range(st["n_levels"]):
        n = st["n"][l]
        A_l = gpu_level_matrix(amg, l, n)
        if l == 0:
            ref_op = H.levels[0].A
        else:
            P = gpu_P(amg, l - 1, st["n"][l - 1])
            ref_op = (P.T @ A_prev @ P).tocsr()
            # rounding bound of the product: eps-multiples of |P|^T |A| |P| (Z entries of the
            # near-kernel modes are large when beta is small)
            bound = (abs(P).T @ abs(A_prev) @ abs(P)).max()
            assert abs(A_l - ref_op).max() <= 1e-12 * bound, f"Galerkin identity level {l}"
        x = rng.standard_normal(n)
        ref = A_l @ x       # the library's own element blocks, assembled in FP64
        if l == 0:
            np.testing.assert_allclose(A_l.toarray(), ref_op.toarray(), rtol=0, atol=1e-12 * abs(ref_op).max())
        xs = torch.from_numpy(x).to(DEV)
        y = amg.gram_spmv(xs, level=l).cpu().numpy()
        scale = (abs(A_l) @ np.abs(x)).max()
        assert np.abs(y - ref).max() <= 1e-10 * scale, f"level {l} FP64 SpMV"
        y32 = amg.gram_spmv(xs.float(), level=l, fp32=True).double().cpu().numpy()
        assert np.abs(y32 - ref).max() <= 1e-4 * scale, f"level {l} FP32 SpMV"
        A_prev = A_l


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_fp64_matches_oracle(name):
    p, H, amg, _, vtol, _ = case(name)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(p["n"])
    ref = O.vcycle(H, r)
    z = amg.apply(torch.from_numpy(r).to(DEV), fp32=0).cpu().numpy()
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= vtol, f"V-cycle relative difference {err:.3e} > {vtol:.1e}"


@pytest.mark.parametrize("name", list(CASES))
def test_pcg_fp64_solution_and_iterations(name):
    p, H, amg, _, _, _ = case(name)
    A = H.levels[0].A
    b = p["b"][0]
    xo, ito, _ = O.pcg(lambda v: A @ v, b, lambda r: O.vcycle(H, r))
    x, its, rel, rc = amg.solve(torch.from_numpy(b).to(DEV), mode=0)
    x = x.cpu().numpy()
    assert rc == 0
    assert abs(int(its[0]) - ito) <= 1, f"iterations {its[0]} vs oracle {ito}"
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    floor = 64 * np.finfo(float).eps * np.linalg.norm(abs(A) @ np.abs(x)) / np.linalg.norm(b)
    assert res <= 1.5e-8 + floor, f"true relative residual {res:.2e} (FP64 evaluation floor {floor:.1e})"
    if name == "rt1_beta1":
        assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["rt1_beta1", "cfg3_16", "cfg4_6"])
def test_fcg_fp32_vcycle_converges(name):
    p, H, amg, _, _, _ = case(name)
    A = H.levels[0].A
    b = p["b"][0]
    x, its, rel, rc = amg.solve(torch.from_numpy(b).to(DEV), mode=1)
    x = x.cpu().numpy()
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert rc == 0 and res <= 1.5e-8, f"FP32-cycle FCG: rc {rc}, residual {res:.2e}, its {its}"
    xo, ito, _ = O.fcg(lambda v: A @ v, b, lambda r: O.vcycle(H, r, np.float32).astype(np.float64))
    assert abs(int(its[0]) - ito) <= max(2, ito // 5), f"iterations {its[0]} vs oracle FP32 emulation {ito}"


def test_multi_rhs_matches_single_and_host_path():
    p, H, amg, _, _, _ = case("cfg4_6")
    rng = np.random.default_rng(9)
    B = rng.uniform(-1, 1, (4, p["n"]))
    X, its, rel, rc = amg.solve(torch.from_numpy(B).to(DEV), mode=0)
    assert rc == 0
    for j in range(4):
        x1, it1, _, _ = amg.solve(torch.from_numpy(B[j]).to(DEV), mode=0)
        assert int(it1[0]) == int(its[j])
        np.testing.assert_allclose(X[j].cpu().numpy(), x1.cpu().numpy(), rtol=1e-10, atol=1e-12)
    Xh, itsh, relh, rch = amg.solve_host(B, mode=0)
    np.testing.assert_allclose(Xh, X.cpu().numpy(), rtol=1e-10, atol=1e-12)


def _adjoint_case(beta):
    c = fegen.config(5, N=8)
    n, d, K0 = fegen.rt_quad(8, 1, beta, 3)
    K = np.ascontiguousarray(np.broadcast_to(K0, (d.shape[0],) + K0.shape))
    return n, d, K, c["coef"], c["b"][0], c["x_star"]


def _gpu_grad(n, d, K, theta, b, xs, rtol):
    from paper_2607_07485_b300 import solve_with_grad
    th = torch.from_numpy(theta).to(DEV).requires_grad_(True)
    x = solve_with_grad(th, torch.from_numpy(b).to(DEV), n, torch.from_numpy(d).to(DEV),
                        torch.from_numpy(K).to(DEV), mode=0, rtol=rtol)
    loss = 0.5 * ((x - torch.from_numpy(xs).to(DEV)) ** 2).sum()
    loss.backward()
    return th.grad.cpu().numpy(), float(loss)


def test_adjoint_gradient_matches_oracle():
    # the adjoint workload's mesh and coefficients with beta = 1 (kappa(A) ~ 1e3): FP64 fixes the
    # gradient far below 1e-8, the bar of the adjoint row
    n, d, K, theta, b, xs = _adjoint_case(1.0)
    A = O.assemble(n, d, K * theta[:, None, None])
    Ho = O.setup(n, d, K * theta[:, None, None])

    def solve(rhs):
        return O.pcg(lambda v: A @ v, rhs, lambda r: O.vcycle(Ho, r), rtol=1e-13)[0]

    _, _, g_ref = O.adjoint_grad(n, d, K, theta, b, xs, solve)
    g, _ = _gpu_grad(n, d, K, theta, b, xs, 1e-13)
    np.testing.assert_allclose(g, g_ref, rtol=1e-8, atol=1e-8 * np.abs(g_ref).max())


def test_adjoint_gradient_on_the_adjoint_workload_form():
    # the adjoint workload itself (RT_[1], beta = 1e-6, theta_e = exp(N(0,1))) at 8 x 8:
    # kappa(A) ~ 9e11, so FP64 fixes x, lambda and g only to ~kappa eps ~ 2e-4 in the worst case;
    # the oracle's own PCG and a sparse direct solve agree on g to 2.6e-7 (max-normalised).
    # Reference: the direct solve; bar: 1e-6, about 4x that observed FP64 spread.
    import scipy.sparse.linalg as spla
    n, d, K, theta, b, xs = _adjoint_case(1e-6)
    A = O.assemble(n, d, K * theta[:, None, None])
    lu = spla.splu(A.tocsc())
    _, _, g_ref = O.adjoint_grad(n, d, K, theta, b, xs, lu.solve)
    g, _ = _gpu_grad(n, d, K, theta, b, xs, 1e-13)
    assert np.abs(g - g_ref).max() <= 1e-6 * np.abs(g_ref).max()


def test_adjoint_gradient_central_differences_on_gpu():
    # central differences of the GPU loss itself (h = 1e-6 relative) on 32 seeded elements of
    # the beta = 1 adjoint case: truncation ~h^2, solve error / h ~1e-13 / 1e-6
    n, d, K, theta, b, xs = _adjoint_case(1.0)
    g, _ = _gpu_grad(n, d, K, theta, b, xs, 1e-14)
    from paper_2607_07485_b300 import Lsamg as _L
    dd, KK, bb = torch.from_numpy(d).to(DEV), torch.from_numpy(K).to(DEV), torch.from_numpy(b).to(DEV)

    def loss(th):
        amg = _L(n, dd, KK, coef=torch.from_numpy(th).to(DEV), rtol=1e-14, maxit=500)
        x, its, rel, rc = amg.solve(bb, mode=0)
        amg.close()
        r = x.cpu().numpy() - xs
        return 0.5 * float(r @ r)

    rng = np.random.default_rng(32)
    for e in rng.choice(len(theta), size=32, replace=False):
        h = 1e-6 * theta[e]
        tp, tm = theta.copy(), theta.copy()
        tp[e] += h
        tm[e] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * np.abs(g).max(), f"element {e}: FD {fd:.6e} vs adjoint {g[e]:.6e}"


def test_beta_small_solution_against_direct_solve():
    # cfg2's form (RT_[3], beta = 1e-6, lognormal theta) at 4 x 4: the GPU solution (FP64 PCG
    # to 1e-12) against a sparse direct solve, element-wise, within kappa(A) eps ||x||
    import scipy.sparse.linalg as spla
    c = fegen.config(2, N=4)
    mats = np.ascontiguousarray(c["elem_mats"] * c["coef"][:, None, None])
    A = O.assemble(c["n"], c["elem_dofs"], mats)
    ev = np.linalg.eigvalsh(A.toarray())
    kappa = ev[-1] / ev[0]
    b = c["b"][0]
    xs = spla.spsolve(A.tocsc(), b)
    amg = Lsamg(c["n"], torch.from_numpy(c["elem_dofs"]).to(DEV), torch.from_numpy(mats).to(DEV),
                tau_c=c["c_tau"], rtol=1e-12, maxit=500)
    x, its, rel, rc = amg.solve(torch.from_numpy(b).to(DEV), mode=0)
    assert rc == 0
    x = x.cpu().numpy()
    bound = kappa * np.finfo(float).eps * np.linalg.norm(xs)
    assert np.abs(x - xs).max() <= bound, (np.abs(x - xs).max(), bound, kappa)
    amg.close()


# ------------------------------------------------------------------------------- failures
def test_error_codes_on_bad_input():
    n, d, K = fegen.rt_quad(4, 0, 1.0)
    mats = np.ascontiguousarray(np.broadcast_to(K, (d.shape[0],) + K.shape)).copy()
    dd = torch.from_numpy(d).to(DEV)
    bad = mats.copy()
    bad[3] = -bad[3]                                    # negative definite element
    with pytest.raises(LsamgError) as e:
        Lsamg(n, dd, torch.from_numpy(bad).to(DEV))
    assert e.value.code == 2
    d2 = d.copy()
    d2[0, 0] = n + 5                                    # DOF out of range
    with pytest.raises(LsamgError) as e:
        Lsamg(n, torch.from_numpy(d2).to(DEV), torch.from_numpy(mats).to(DEV))
    assert e.value.code == 1
    d3 = d.copy()
    d3[0, 1] = d3[0, 0]                                 # duplicate DOF in one element
    with pytest.raises(LsamgError) as e:
        Lsamg(n, torch.from_numpy(d3).to(DEV), torch.from_numpy(mats).to(DEV))
    assert e.value.code == 1
    c = fegen.config(1)
    amg = Lsamg(c["n"], torch.from_numpy(c["elem_dofs"]).to(DEV),
                torch.from_numpy(np.ascontiguousarray(c["elem_mats"])).to(DEV), maxit=1)
    b = torch.from_numpy(c["b"][0].copy()).to(DEV)
    x, its, rel, rc = amg.solve(b, mode=0)
    assert rc == 4                                      # maxit reached
    b[5] = float("nan")
    with pytest.raises(LsamgError) as e:
        amg.solve(b, mode=0)
    assert e.value.code == 8


@pytest.mark.parametrize("name", ["rt1_beta1", "cfg1", "cfg3_16", "cfg4_6"])
def test_local_eigenpairs_self_consistent(name):
    """Each level's local problems rebuilt in NumPy from the library's own data (element maps,
    element Gram blocks, aggregates, overlaps, multiplicities) and solved by the oracle's
    least-squares route: the library's Z must span the same subspaces (same coordinates, so
    no basis freedom beyond degenerate eigenspaces)."""
    p, H, amg, ptol, _, band = case(name)
    st = amg.stats()
    for l in range(st["n_levels"] - 1):
        eptr, eidx = amg.query(l, "EPTR"), amg.query(l, "EIDX")
        goff, grows, G = amg.query(l, "GOFF"), amg.query(l, "GROWS"), amg.query(l, "G")
        agg, mult = amg.query(l, "AGG"), amg.query(l, "MULT")
        optr, oidx = amg.query(l, "OMEGA_PTR"), amg.query(l, "OMEGA_IDX")
        kg, zoff, Z = amg.query(l, "K"), amg.query(l, "ZOFF"), amg.query(l, "Z")
        tau = st["tau"][l]
        elems = [eidx[eptr[e]:eptr[e + 1]] for e in range(len(eptr) - 1)]
        nagg = len(kg)
        ael = [[] for _ in range(nagg)]
        for t, d in enumerate(elems):
            for a in np.unique(agg[d]):
                ael[a].append(t)
        omega = [np.flatnonzero(agg == a) for a in range(nagg)]
        Omega = [oidx[optr[a]:optr[a + 1]] for a in range(nagg)]
        Gs = []
        for e, d in enumerate(elems):
            Gs.append(G[goff[e]:goff[e] + grows[e] * len(d)].reshape(grows[e], len(d)))
        worst = 0.0
        for a in range(nagg):
            Hm, F, _ = OL.local_gram_rows(a, elems, Gs, mult, ael, omega, Omega)
            nw = len(omega[a])
            Zr, mu, _ = OL.local_problem(Hm, F, nw, tau)
            if Zr.shape[1] != kg[a]:   # a flip is legitimate only by eigenvalues inside the band
                near = int((np.abs(np.asarray(mu) * tau - 1.0) < band).sum())
                assert abs(int(kg[a]) - Zr.shape[1]) <= near, \
                    f"level {l} aggregate {a}: k {kg[a]} vs {Zr.shape[1]} with {near} in the band"
                continue
            Zg = Z[zoff[a]:zoff[a + 1]].reshape(nw, kg[a])
            Aww = F.T @ F
            np.testing.assert_allclose(Zg.T @ Aww @ Zg, np.eye(kg[a]), atol=1e-6,
                                       err_msg=f"level {l} aggregate {a}: Z not A_ww-orthonormal")
            d = np.linalg.norm(_projector(Zg) - _projector(Zr), 2) * _sep(mu, int(kg[a]), tau)
            worst = max(worst, d)
        assert worst <= ptol, f"level {l}: self-consistency projector difference {worst:.3e}"


@pytest.mark.parametrize("name", ["cfg1", "cfg3_16"])
def test_multi_cta_paths_match_single_cta(name):
    """The multi-CTA tridiagonalisation and the split Schwarz sweep (used for large local
    problems) forced on a small case: same coarse space and the same V-cycle as the
    one-CTA-per-matrix kernels (and so as the oracle)."""
    p, H, amg, ptol, vtol, band = case(name)
    gen, opts, *_ = CASES[name]
    o = dict(opts)
    if "tau_c" not in o and "c_tau" in p:
        o["tau_c"] = p["c_tau"]
    big = Lsamg(p["n"], torch.from_numpy(p["elem_dofs"]).to(DEV), torch.from_numpy(p["mats"]).to(DEV),
                large_dense=16, split_sweep=16, sweep_block=32, **o)
    L0 = H.levels[0]
    kb, ka = big.query(0, "K"), amg.query(0, "K")
    zoff, Z = big.query(0, "ZOFF"), big.query(0, "Z")
    for i in range(L0.nagg):
        # mode counts agree except where the oracle has eigenvalues inside the rank-flip band
        if kb[i] != ka[i] or kb[i] != L0.k[i]:
            near = int((np.abs(L0.mu[i] * L0.tau - 1.0) < band).sum())
            assert max(abs(int(kb[i]) - int(L0.k[i])), abs(int(ka[i]) - int(L0.k[i]))) <= near, \
                f"aggregate {i}: k {kb[i]} (forced) vs {ka[i]} vs oracle {L0.k[i]}, {near} in the band"
            continue
        nw, k = len(L0.omega[i]), int(kb[i])
        Zg = Z[zoff[i]:zoff[i + 1]].reshape(nw, k)
        assert np.linalg.norm(_projector(Zg) - _projector(L0.Z[i]), 2) * _separation(L0, i) <= ptol
    r = np.random.default_rng(6).standard_normal(p["n"])
    rt = torch.from_numpy(r).to(DEV)
    z1 = big.apply(rt, fp32=0).cpu().numpy()
    z0 = amg.apply(rt, fp32=0).cpu().numpy()
    assert np.linalg.norm(z1 - z0) <= vtol * np.linalg.norm(z0)
    zo = O.vcycle(H, r)
    assert np.linalg.norm(z1 - zo) <= vtol * np.linalg.norm(zo)
    big.close()
