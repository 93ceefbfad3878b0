"""Plain FP64 oracle of LS-AMG-DD for conforming finite elements.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; never by the library.

Every function follows one passage of the paper (Krzysik, Southworth, Wimmer,
"A black-box, multilevel algebraic preconditioning framework for conforming
finite elements"), cited by section / equation:

* Section 2, eq. (2.1)          Gram row convention A = G^T G
* Section 5.1, Prop. 5.1        elementwise Gram stacking G = [G_T R_T]
* Section 5.2                   local factors (eigen range factor used here)
* Section 2, eq. (2.2)          disjoint aggregates (MIS(2) aggregation, two passes,
                                the Section 6 tests use two aggregation passes)
* Section 2, eqs. (2.3)-(2.4)   row-touching set and G-row closure Omega_i
* Section 5.4, Def. 5.4/Thm 5.6 element closure (= G-row closure structurally)
* Section 5.3, Def. 5.2         algebraic A-closure (the Table 2 comparison), option A=
* Section 2, eqs. (2.5)-(2.7)   multiplicity, weights, exact SPSD splitting
* Section 2, eqs. (2.8)-(2.9)   local GEP and its Schur-complement reduction
* Section 2, eq. (2.10)         tau_cut = c * max_j mult(j)
* Section 2 (end)               P = [R_w^T Z_i], G_c = G P, recursion, direct coarsest solve
* Section 6 preamble            multiplicative Schwarz pre/post smoothing, level limits,
                                the standalone V-cycle iteration (random x0, 1e-10 reduction)
* Section 2 (smoother choice)   additive (fully parallel) block Schwarz variant, damped
* (outer solver, adjoint)       FP64 PCG / flexible CG(1) and the adjoint gradient
                                g_e = -lambda_e^T K_e x_e  (not in the paper)

Readings where the paper is silent (aggregation algorithm, hash, colouring order,
pseudo-inverse tolerance, eigenvector normalisation) are stated at each function.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` against a property the paper or the mathematics
fixes (identities, brute force, textbook routines, bounds, and the Table 2 counts the
paper prints for the two smallest CG(1) meshes, stored under tests/golden/).  Parity
unpinned: absolute iteration counts and operator complexity relative to the paper's
own larger (triangle/Firedrake) runs, and the sign/rotation of individual Z_i columns
(only the spanned projectors are pinned).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps

__all__ = [
    "hash32", "assemble", "element_gram", "structural_graph", "mis2", "aggregate_mis2", "aggregate_greedy",
    "aggregate_two_pass", "closure", "local_problem", "local_problem_pinv", "local_gram_rows", "Level", "Hierarchy", "setup",
    "vcycle", "stationary", "pcg", "fcg", "elem_grad", "adjoint_grad", "gram_spmv", "greedy_colouring",
    "options_default",
]


# -----------------------------------------------------------------------------
# Options (Section 6 preamble values)
# -----------------------------------------------------------------------------
def options_default():
    """Paper defaults: c = 0.75 (Section 6.1/6.3), 2 aggregation passes, at most 3 levels,
    stop below 10 DOFs or above 25 % density (Section 6 preamble); the G-row closure
    (closure="A" selects the algebraic A-closure of the Section 5 comparison).  Two
    comparison options: aggregation="greedy" (the sequential greedy pass instead of MIS(2))
    and sweep_order="natural" (the multiplicative sweep in aggregate index order instead of
    colour-major order)."""
    return dict(tau_c=0.75, agg_passes=2, agg_passes_coarse=2, max_levels=3, min_coarse=10,
                max_density=0.25, rtol=1e-8, maxit=1000, closure="G", aggregation="mis2",
                sweep_order="colour")


# -----------------------------------------------------------------------------
# Hash priority (reading: the paper names no aggregation algorithm; priorities
# for the MIS(2) rounds use the "lowbias32" integer mix of C. Wellons'
# hash-prospector, a published 32-bit bijection)
# -----------------------------------------------------------------------------
def hash32(x):
    """lowbias32: x ^= x>>16; x *= 0x7feb352d; x ^= x>>15; x *= 0x846ca68b; x ^= x>>16 (mod 2^32)."""
    x = np.asarray(x, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    m = np.uint64(0xFFFFFFFF)
    x = x ^ (x >> np.uint64(16))
    x = (x * np.uint64(0x7FEB352D)) & m
    x = x ^ (x >> np.uint64(15))
    x = (x * np.uint64(0x846CA68B)) & m
    x = x ^ (x >> np.uint64(16))
    return x.astype(np.uint64)


# -----------------------------------------------------------------------------
# Assembly and element Gram factors (Section 4 eq. 4.1; Section 5.1 Prop. 5.1;
# Section 5.2)
# -----------------------------------------------------------------------------
def assemble(n, elems, mats):
    """A = sum_T R_T^T A_T R_T as scipy CSR (Section 4, eq. 4.1)."""
    rows, cols, vals = [], [], []
    for dofs, AT in zip(elems, mats):
        dofs = np.asarray(dofs, np.int64)
        if len(dofs) == 0:
            continue
        rows.append(np.repeat(dofs, len(dofs)))
        cols.append(np.tile(dofs, len(dofs)))
        vals.append(np.asarray(AT, float).ravel())
    if not rows:
        return sp.csr_matrix((n, n))
    if n <= 6000:
        D = np.zeros((n, n))
        for dofs, AT in zip(elems, mats):
            dofs = np.asarray(dofs, np.int64)
            if len(dofs):
                D[np.ix_(dofs, dofs)] += AT
        return sp.csr_matrix(D)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A.tocsr()


class NotSPSD(ValueError):
    pass


def element_gram(AT, check=True):
    """Range factor G_T = Lambda_+^{1/2} Q_+^T of an SPSD block (Section 5.2; the paper's
    runs use the eigendecomposition).  Keeps eigenvalues > n_T * eps * lambda_max and,
    with ``check`` (user input), raises NotSPSD if an eigenvalue is below
    -1e-12 * lambda_max.  Computed coarse blocks skip the check: their negative
    eigenvalues are rounding of an exactly SPSD product."""
    AT = np.asarray(AT, float)
    nT = AT.shape[0]
    if nT == 0:
        return np.zeros((0, 0))
    w, Q = np.linalg.eigh(AT)
    lmax = max(w[-1], 0.0)
    if check and lmax > 0 and w[0] < -1e-12 * lmax:
        raise NotSPSD(f"element eigenvalue {w[0]:.3e} < -1e-12*{lmax:.3e}")
    keep = w > nT * EPS * lmax
    return np.sqrt(w[keep])[:, None] * Q[:, keep].T


def gram_spmv(elems, G, x):
    """y = G^T (G x) = sum_T R_T^T G_T^T (G_T x_T) (Section 2 eq. 2.1; Prop. 5.1)."""
    y = np.zeros_like(x, dtype=float)
    for dofs, GT in zip(elems, G):
        if GT.size:
            y[dofs] += GT.T @ (GT @ x[dofs])
    return y


# -----------------------------------------------------------------------------
# Aggregation (Section 2 eq. 2.2; the Section 6 tests aggregate in two passes and name
# no algorithm).  Reading: each pass is the distance-2 maximal-independent-set
# aggregation of Bell, Dalton & Olson (SISC 2012) on the structural graph
# (p ~ q iff they share an element, i.e. strength threshold 0), with priorities
# (state, hash32(index), index); pass 2 runs on the aggregate graph.
# -----------------------------------------------------------------------------
def structural_graph(n, elems):
    """Boolean CSR S with S[p,q] = 1 iff p and q share an element (diagonal included)."""
    rows, cols = [], []
    for t, dofs in enumerate(elems):
        dofs = np.asarray(dofs, np.int64)
        if len(dofs):
            rows.append(dofs)
            cols.append(np.full(len(dofs), t, np.int64))
    ne = len(elems)
    if rows:
        E = sp.csr_matrix((np.ones(sum(len(r) for r in rows)), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, ne))
    else:
        E = sp.csr_matrix((n, ne))
    S = (E @ E.T).tocsr()
    S = S + sp.identity(n, format="csr")
    S.data[:] = 1.0
    S.sort_indices()
    return S


def _rowmax(S, v):
    return np.maximum.reduceat(v[S.indices], S.indptr[:-1])


def _rowmin(S, v):
    return np.minimum.reduceat(v[S.indices], S.indptr[:-1])


def mis2(S, prio):
    """Distance-2 maximal independent set by synchronous Luby rounds (Bell-Dalton-Olson):
    key(p) = (state+1, prio(p), p) packed in 64 bits; an undecided node whose 2-hop
    maximum is itself joins the set, one whose 2-hop maximum is a set member leaves.
    Returns state (+1 in the set, -1 out)."""
    n = S.shape[0]
    assert n < (1 << 30)
    idx = np.arange(n, dtype=np.uint64)
    prio = np.asarray(prio, np.uint64)
    state = np.zeros(n, np.int64)
    mask30 = np.uint64((1 << 30) - 1)
    while True:
        und = state == 0
        if not und.any():
            return state
        key = ((state + 1).astype(np.uint64) << np.uint64(62)) | (prio << np.uint64(30)) | idx
        m2 = _rowmax(S, _rowmax(S, key))
        win = und & ((m2 & mask30) == idx)
        lose = und & ~win & ((m2 >> np.uint64(62)) == np.uint64(2))
        state[win] = 1
        state[lose] = -1


def aggregate_mis2(S, prio):
    """One aggregation pass: MIS(2) roots take their distance-1 neighbourhoods (ids in
    ascending root order); every remaining node joins the aggregate of its aggregated
    distance-1 neighbour with the smallest (prio, index), in synchronous rounds."""
    n = S.shape[0]
    state = mis2(S, prio)
    roots = np.flatnonzero(state == 1)
    rootval = np.zeros(n, np.int64)
    rootval[roots] = np.arange(1, len(roots) + 1)
    m = _rowmax(S, rootval)
    agg = m - 1
    big = np.uint64(0xFFFFFFFFFFFFFFFF)
    prio = np.asarray(prio, np.uint64)
    while (agg < 0).any():
        key = np.where(agg >= 0, (prio << np.uint64(32)) | np.arange(n, dtype=np.uint64), big)
        mn = _rowmin(S, key)
        upd = (agg < 0) & (mn != big)
        if not upd.any():
            raise RuntimeError("aggregation stalled")
        q = (mn[upd] & np.uint64(0xFFFFFFFF)).astype(np.int64)
        agg = agg.copy()
        agg[upd] = agg[q]
    return agg, len(roots)


def aggregate_greedy(S):
    """One pass of the sequential greedy ("standard", Vanek-Mandel-Brezina) aggregation, the
    kind of routine the paper's serial implementation used; kept as a second option to show
    that iteration counts and operator complexity do not hinge on the MIS(2) reading.
    Step 1: visiting nodes in index order, a node whose whole distance-1 neighbourhood is
    still free becomes a root and its neighbourhood an aggregate (ids in root order).
    Step 2: every node left free joins the aggregate of its first (lowest-index) neighbour
    that step 1 aggregated.  Step 3: nodes still free (none on a structural graph, where each
    of them has an aggregated neighbour) form aggregates with their free neighbours, in
    index order.  Returns (labels, number of aggregates)."""
    n = S.shape[0]
    ptr, idx = S.indptr, S.indices
    agg = np.full(n, -1, np.int64)
    nagg = 0
    for i in range(n):
        nb = idx[ptr[i]:ptr[i + 1]]
        if agg[i] < 0 and (agg[nb] < 0).all():
            agg[nb] = nagg
            agg[i] = nagg
            nagg += 1
    step1 = agg.copy()
    for i in range(n):
        if agg[i] < 0:
            nb = idx[ptr[i]:ptr[i + 1]]
            joined = nb[step1[nb] >= 0]
            if len(joined):
                agg[i] = step1[joined.min()]
    for i in range(n):
        if agg[i] < 0:
            nb = idx[ptr[i]:ptr[i + 1]]
            free = nb[agg[nb] < 0]
            agg[free] = nagg
            agg[i] = nagg
            nagg += 1
    return agg, nagg


def aggregate_two_pass(S, passes=2, method="mis2"):
    """Compose ``passes`` aggregation passes (MIS(2), or the greedy pass with
    method="greedy"): pass 1 on the node graph S, pass k+1 on the graph of pass-k aggregates
    (adjacent iff any members are adjacent)."""
    if method not in ("mis2", "greedy"):
        raise ValueError(f"unknown aggregation {method!r}")
    n = S.shape[0]
    agg = np.arange(n)
    Sk = S
    nagg = n
    for _ in range(passes):
        if method == "greedy":
            a, nagg = aggregate_greedy(Sk)
        else:
            a, nagg = aggregate_mis2(Sk, hash32(np.arange(Sk.shape[0])))
        agg = a[agg]
        C = sp.csr_matrix((np.ones(len(a)), (np.arange(len(a)), a)), shape=(len(a), nagg))
        Sk = (C.T @ Sk @ C).tocsr()
        Sk.data[:] = 1.0
        Sk.sort_indices()
    return agg, nagg


# -----------------------------------------------------------------------------
# Closure, multiplicity, splitting (Section 2 eqs. 2.3-2.7; Section 5.4 Thm 5.6)
# -----------------------------------------------------------------------------
def closure(elems, agg, nagg, A=None):
    """Element-form closure.  With structural row supports, the rows touching omega_i are
    the rows of the elements T with N(T) & omega_i != {} (eq. 2.3), the G-row closure is
    Omega_i = U N(T) over those elements (eq. 2.4 = element closure, Thm 5.6), and
    mult(j) = mult(T) = #aggregates meeting N(T) (eq. 2.5).

    With the assembled matrix A given, Omega_i is instead the algebraic A-closure of
    Section 5 (Def. of Omega^A): omega_i together with every p such that A(q, p) is nonzero
    for some q in omega_i.  Reading of "nonzero" (the paper removes cancelled entries and
    notes that zero or near-zero entries are commonly dropped from the graph of A): an
    entry counts when |A(q, p)| > ACUT sqrt(|A(q, q)| |A(p, p)|).  Entries that cancel in
    exact arithmetic are exact zeros on the finest level (orthogonal gradients) but carry
    rounding after the Galerkin products of coarser levels; the relative cut treats both as
    zero.  Only the closure changes; rows touching omega_i and multiplicities stay those of
    eqs. 2.3-2.5.

    Returns (eagg, mult, ael, omega, Omega)."""
    eagg = [np.unique(agg[np.asarray(d, np.int64)]) for d in elems]
    mult = np.array([len(a) for a in eagg], np.int64)
    ael = [[] for _ in range(nagg)]
    for t, a in enumerate(eagg):
        for i in a:
            ael[i].append(t)
    ael = [np.array(x, np.int64) for x in ael]
    order = np.argsort(agg, kind="stable")
    counts = np.bincount(agg, minlength=nagg)
    starts = np.concatenate([[0], np.cumsum(counts)])
    omega = [order[starts[i]:starts[i + 1]] for i in range(nagg)]
    Omega = []
    if A is not None:
        Ac = sp.coo_matrix(A)
        dg = np.abs(sp.csr_matrix(A).diagonal())
        keep = np.abs(Ac.data) > ACUT * np.sqrt(dg[Ac.row] * dg[Ac.col])
        Ak = sp.csr_matrix((np.ones(int(keep.sum())), (Ac.row[keep], Ac.col[keep])), shape=A.shape)
        for i in range(nagg):
            nb = Ak[omega[i]].indices
            Omega.append(np.union1d(np.asarray(omega[i], np.int64), nb.astype(np.int64)))
        return eagg, mult, ael, omega, Omega
    for i in range(nagg):
        if len(ael[i]):
            Omega.append(np.unique(np.concatenate([np.asarray(elems[t], np.int64) for t in ael[i]])))
        else:
            Omega.append(np.array(omega[i], np.int64))
    return eagg, mult, ael, omega, Omega


def local_blocks(i, elems, mats, mult, ael, omega, Omega):
    """Local matrices of aggregate i in the order [omega_i; Gamma_i] (Section 2):
    At  = sum_{T in ael(i)} mult(T)^{-1} R_Omega R_T^T A_T R_T R_Omega^T   (eq. 2.6-2.7),
    Aww = R_omega A R_omega^T (principal submatrix of A on omega_i, eq. 2.8-2.9).
    Returns (At, Aww, loc) with loc = global DOFs in local order."""
    w = np.asarray(omega[i], np.int64)
    gam = np.setdiff1d(Omega[i], w)
    loc = np.concatenate([w, gam])
    pos = {int(g): j for j, g in enumerate(loc)}
    nO = len(loc)
    nw = len(w)
    At = np.zeros((nO, nO))
    Aww = np.zeros((nw, nw))
    for t in ael[i]:
        d = np.asarray(elems[t], np.int64)
        p = np.array([pos[int(g)] for g in d])
        AT = np.asarray(mats[t], float)
        At[np.ix_(p, p)] += AT / mult[t]
        inw = p < nw
        Aww[np.ix_(p[inw], p[inw])] += AT[np.ix_(inw, inw)]
    return At, Aww, loc


def pinv_sym(M):
    """Moore-Penrose pseudo-inverse of a symmetric PSD matrix by eigh, dropping
    eigenvalues <= size * eps * lambda_max (NumPy's matrix_rank convention)."""
    if M.shape[0] == 0:
        return np.zeros_like(M)
    w, V = np.linalg.eigh(M)
    tol = M.shape[0] * EPS * max(abs(w[-1]), abs(w[0]))
    keep = w > tol
    return (V[:, keep] / w[keep]) @ V[:, keep].T


ACUT = 1e-12  # reading: relative size below which an assembled entry counts as zero (A-closure)
TIE = 1e-9  # reading: keep mu*tau < 1 - TIE, so exact ties mu = 1/tau (from mesh symmetry) are
            # discarded deterministically; tau_max <= tau_cut is unaffected


def local_problem_pinv(At, Aww, tau):
    """Reduced local GEP (Section 2 eq. 2.9) in the assembled form S y = mu A_ww y with
    mu = 1/lambda: S = At_ww - At_wG pinv(At_GG) At_Gw.  Used by the pins on well-conditioned
    inputs only: the eigh pseudo-inverse loses ~eps*kappa(At_GG)^2, so ill-conditioned blocks
    go through the least-squares form ``local_problem``.  Returns (Z, mu, gap)."""
    nw = Aww.shape[0]
    Sw = At[:nw, :nw] - At[:nw, nw:] @ pinv_sym(At[nw:, nw:]) @ At[nw:, :nw]
    Sw = 0.5 * (Sw + Sw.T)
    mu, Y = sla.eigh(Sw, Aww)
    return _select(Y, mu, tau)


def _select(Y, mu, tau):
    keep = mu * tau < 1.0 - TIE
    Z = Y[:, keep].copy()
    for j in range(Z.shape[1]):
        k = int(np.argmax(np.abs(Z[:, j])))
        if Z[k, j] < 0:
            Z[:, j] = -Z[:, j]
    gap = float(np.min(np.abs(mu * tau - 1.0))) if len(mu) else np.inf
    return Z, mu, gap


def local_gram_rows(i, elems, G, mult, ael, omega, Omega):
    """Least-squares data of aggregate i (Section 2 eqs. 2.3-2.7), DOFs ordered [omega_i; Gamma_i]:
    H = W^{1/2} G(R_omega_i, Omega_i) (rows of the elements touching omega_i, each scaled by
    mult(T)^{-1/2}, eq. 2.6) so that At = H^T H (eq. 2.7), and F = G(R_omega_i, omega_i) so that
    A_ww = R_w A R_w^T = F^T F (rows not touching omega_i vanish on omega_i)."""
    w = np.asarray(omega[i], np.int64)
    loc = np.concatenate([w, np.setdiff1d(Omega[i], w)])
    pos = {int(g): j for j, g in enumerate(loc)}
    nw = len(w)
    blocks = []
    for t in ael[i]:
        GT = np.asarray(G[t], float)
        if GT.size == 0:
            continue
        B = np.zeros((GT.shape[0], len(loc)))
        cols = np.array([pos.get(int(g), -1) for g in elems[t]])
        inside = cols >= 0          # always all of N(T) for the G-row closure; the A-closure
        B[:, cols[inside]] = GT[:, inside]   # may cut element DOFs (their columns are lost)
        blocks.append((B, float(mult[t])))
    Hm = np.vstack([B / np.sqrt(m) for B, m in blocks]) if blocks else np.zeros((0, len(loc)))
    F = np.vstack([B[:, :nw] for B, _ in blocks]) if blocks else np.zeros((0, nw))
    return Hm, F, loc


def local_problem(Hm, F, nw, tau):
    """Reduced local GEP (Section 2 eq. 2.9) A_ww u = lambda S u, solved as S y = mu A_ww y
    with mu = 1/lambda, in least-squares form.  With At = H^T H the Schur complement with the
    Moore-Penrose pseudo-inverse is S = Y^T Y, Y = (I - Q Q^T) H_omega, Q an orthonormal basis of
    range(H_Gamma) (numerical rank at max(m, n) * eps * sigma_max, NumPy's matrix_rank rule);
    A_ww = F^T F = R^T R (QR of F).  Then mu are the squared singular values of Y R^{-1} (zeros
    for ker S, the +infinity modes) and y = R^{-1} v is A_ww-orthonormal.  Keep mu*tau < 1 - TIE,
    ascending mu, largest-magnitude entry of each column positive.  Returns (Z, mu, gap)."""
    HG = Hm[:, nw:]
    Hw = Hm[:, :nw]
    if HG.shape[1] > 0 and HG.shape[0] > 0:
        U, sg, _ = np.linalg.svd(HG, full_matrices=False)
        r = int((sg > max(HG.shape) * EPS * sg[0]).sum()) if sg[0] > 0 else 0
        Q = U[:, :r]
        Y = Hw - Q @ (Q.T @ Hw)
    else:
        Y = Hw
    R = np.linalg.qr(F, mode="r")
    M = sla.solve_triangular(R, Y.T, trans="T", lower=False).T      # Y R^{-1}
    _, s, Vt = np.linalg.svd(M, full_matrices=True)
    mu = np.zeros(nw)
    mu[:len(s)] = s * s
    order = np.argsort(mu, kind="stable")
    mu = mu[order]
    V = Vt.T[:, order]
    Yv = sla.solve_triangular(R, V, lower=False)
    return _select(Yv, mu, tau)


# -----------------------------------------------------------------------------
# Smoother colouring (reading: subdomains conflict iff some element meets both
# overlaps; greedy colouring in aggregate index order; sweep colours ascending)
# -----------------------------------------------------------------------------
def greedy_colouring(conflict):
    """Sequential greedy colouring of a symmetric boolean CSR conflict graph in index order:
    colour(i) = smallest colour unused by conflicting k < i."""
    n = conflict.shape[0]
    col = np.full(n, -1, np.int64)
    for i in range(n):
        nb = conflict.indices[conflict.indptr[i]:conflict.indptr[i + 1]]
        used = set(int(col[k]) for k in nb if k < i)
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


# -----------------------------------------------------------------------------
# Hierarchy
# -----------------------------------------------------------------------------
@dataclass
class Level:
    n: int
    elems: list
    mats: list            # A_T (FP64 dense) of this level
    G: list               # G_T with G_T^T G_T = A_T
    A: sp.csr_matrix = None
    S: sp.csr_matrix = None
    nnz: int = 0
    coarsest: bool = False
    # set-up products (non-coarsest levels)
    agg: np.ndarray = None
    nagg: int = 0
    eagg: list = None
    mult: np.ndarray = None
    tau: float = 0.0
    ael: list = None
    omega: list = None
    Omega: list = None
    Z: list = None
    k: np.ndarray = None
    off: np.ndarray = None
    gaps: np.ndarray = None
    mu: list = None               # local eigenvalues mu (ascending) of every aggregate
    P: sp.csr_matrix = None
    colour: np.ndarray = None
    sweep: list = None            # aggregate order of the forward sweep
    chol: list = None             # Cholesky factors (lower) of A_Omega
    cgroups: list = None          # level-l elements merged into each coarse element
    # coarsest
    Ldense: np.ndarray = None


@dataclass
class Hierarchy:
    levels: list = field(default_factory=list)
    opts: dict = None

    def stats(self):
        nnz0 = self.levels[0].nnz
        return dict(n=[L.n for L in self.levels], nnz=[L.nnz for L in self.levels],
                    OC=sum(L.nnz for L in self.levels) / nnz0,
                    GC=sum(L.n for L in self.levels) / self.levels[0].n,
                    tau=[L.tau for L in self.levels], nagg=[L.nagg for L in self.levels])


def setup(n, elems, mats, opts=None, c_tau=None):
    """LS-AMG-DD setup (Section 2; Section 6 preamble), level by level:
    factor A_T -> G_T (level 0, Section 5.2); aggregate (two passes); closure and
    mult; tau_cut = c max mult (eq. 2.10); local GEPs -> Z_i, P; coarse element maps
    and A_c,T = (R_T P)^T A_T (R_T P), G_c,T = G_T (R_T P); Schwarz factors and colours.
    Stops at max_levels, n < min_coarse or structural density > max_density; the last
    level is factored densely."""
    o = options_default()
    if opts:
        o.update(opts)
    if c_tau is not None:
        o["tau_c"] = c_tau
    elems = [np.asarray(d, np.int64) for d in elems]
    mats = [np.asarray(m, float) for m in mats]
    G = [element_gram(m) for m in mats]
    H = Hierarchy(opts=o)
    lev = Level(n=n, elems=elems, mats=mats, G=G)
    while True:
        lev.A = assemble(lev.n, lev.elems, lev.mats)
        lev.S = structural_graph(lev.n, lev.elems)
        lev.nnz = int(lev.S.nnz)
        H.levels.append(lev)
        li = len(H.levels) - 1
        last = (li == o["max_levels"] - 1 or lev.n < o["min_coarse"]
                or lev.nnz / float(lev.n) ** 2 > o["max_density"])
        if not last:
            nxt = _coarsen(lev, o, o["agg_passes"] if li == 0 else o["agg_passes_coarse"])
            if nxt is None:
                last = True
        if last:
            lev.coarsest = True
            Ad = lev.A.toarray()
            lev.Ldense = np.linalg.cholesky(0.5 * (Ad + Ad.T))
            return H
        _smoother_setup(lev, o.get("sweep_order", "colour"))
        lev = nxt


def _coarsen(lev, o, passes):
    agg, nagg = aggregate_two_pass(lev.S, passes, o.get("aggregation", "mis2"))
    if o.get("closure", "G") not in ("G", "A"):
        raise ValueError(f"unknown closure {o['closure']!r}")
    eagg, mult, ael, omega, Omega = closure(lev.elems, agg, nagg, A=lev.A if o.get("closure") == "A" else None)
    tau = o["tau_c"] * float(mult.max())
    Z, gaps, mus = [], [], []
    for i in range(nagg):
        Hm, F, _ = local_gram_rows(i, lev.elems, lev.G, mult, ael, omega, Omega)
        Zi, mui, gap = local_problem(Hm, F, len(omega[i]), tau)
        Z.append(Zi)
        gaps.append(gap)
        mus.append(mui)
    k = np.array([z.shape[1] for z in Z], np.int64)
    nc = int(k.sum())
    if nc == 0 or nc >= lev.n:
        # reading: a level whose coarse space is empty or does not shrink is the coarsest
        return None
    off = np.concatenate([[0], np.cumsum(k)])
    rows, cols, vals = [], [], []
    for i in range(nagg):
        if k[i]:
            rows.append(np.repeat(omega[i], k[i]))
            cols.append(np.tile(np.arange(off[i], off[i + 1]), len(omega[i])))
            vals.append(Z[i].ravel())
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(lev.n, nc))
    lev.agg, lev.nagg, lev.eagg, lev.mult, lev.tau = agg, nagg, eagg, mult, tau
    lev.ael, lev.omega, lev.Omega, lev.Z, lev.k, lev.off, lev.P = ael, omega, Omega, Z, k, off, P
    lev.gaps = np.array(gaps)
    lev.mu = mus
    # Coarse cover (Section 2 end: A_c = P^T A P = (GP)^T (GP); Remark 5.2: a cover by
    # collections of elements induces a coarser Gram).  Elements whose coarse DOF maps
    # coincide (same set of touching aggregates) are merged into one coarse element with
    # A_g = sum_T (R_T P)^T A_T (R_T P) and a range factor G_g of A_g.  Merged members share
    # eagg, hence mult, closure and splitting weights, so every next-level quantity
    # (graph, Omega, At, A_ww) is unchanged by the merge.  Groups are ordered by their
    # smallest member element.  The coarse element's Gram rows are the members' rows of
    # G_c = G P stacked (no truncation), so G_g^T G_g = A_g.
    groups = {}
    order = []
    for t in range(len(lev.elems)):
        key = tuple(int(a) for a in eagg[t])
        if len(key) == 0 or int(k[list(key)].sum()) == 0:
            continue
        if key not in groups:
            groups[key] = []
            order.append(key)
        groups[key].append(t)
    celems, cmats, cG, members = [], [], [], []
    for key in order:
        cm = np.concatenate([np.arange(off[a], off[a + 1]) for a in key]).astype(np.int64)
        Ag = np.zeros((len(cm), len(cm)))
        Gg = []
        for t in groups[key]:
            d = lev.elems[t]
            RTP = P[d][:, cm].toarray()
            Ag += RTP.T @ lev.mats[t] @ RTP
            Gg.append(lev.G[t] @ RTP)            # G_c = G P, rows of the member element
        Ag = 0.5 * (Ag + Ag.T)
        celems.append(cm)
        cmats.append(Ag)
        cG.append(np.vstack(Gg) if Gg else np.zeros((0, len(cm))))
        members.append(np.array(groups[key], np.int64))
    lev.cgroups = members
    return Level(n=nc, elems=celems, mats=cmats, G=cG)


def _smoother_setup(lev, order="colour"):
    """Multiplicative Schwarz on the overlaps Omega_i with exact local solves
    A_Omega = R_Omega A R_Omega^T (Section 2; Section 6 preamble); the forward sweep visits
    the subdomains colour by colour (order="colour") or in index order (order="natural")."""
    if order not in ("colour", "natural"):
        raise ValueError(f"unknown sweep order {order!r}")
    nagg = lev.nagg
    ne = len(lev.elems)
    # B[i, T] = 1 iff element T meets Omega_i
    lens = [len(o) for o in lev.Omega]
    M = sp.csr_matrix((np.ones(sum(lens)), (np.concatenate(lev.Omega), np.repeat(np.arange(nagg), lens))),
                      shape=(lev.n, nagg))
    el = [np.asarray(d, np.int64) for d in lev.elems]
    elens = [len(d) for d in el]
    E = sp.csr_matrix((np.ones(sum(elens)), (np.concatenate(el), np.repeat(np.arange(ne), elens))),
                      shape=(lev.n, ne))
    B = (M.T @ E).tocsr()
    B.data[:] = 1.0
    C = (B @ B.T).tocsr()
    C.data[:] = 1.0
    C.setdiag(0)
    C.eliminate_zeros()
    C.sort_indices()
    lev.colour = greedy_colouring(C)
    lev.sweep = (sorted(range(nagg), key=lambda i: (lev.colour[i], i)) if order == "colour"
                 else list(range(nagg)))
    lev.chol = []
    for i in range(nagg):
        Om = lev.Omega[i]
        AO = lev.A[Om][:, Om].toarray()
        lev.chol.append(np.linalg.cholesky(0.5 * (AO + AO.T)))


# -----------------------------------------------------------------------------
# V-cycle and Krylov drivers
# -----------------------------------------------------------------------------
def _cast(H, dtype):
    """Per-level operators cast to ``dtype`` (FP32 emulation of the mixed-precision cycle)."""
    key = np.dtype(dtype).name
    cache = getattr(H, "_cast_cache", {})
    if key in cache:
        return cache[key]
    out = []
    for L in H.levels:
        d = dict(A=L.A.astype(dtype))
        if L.coarsest:
            d["L"] = L.Ldense.astype(dtype)
        else:
            d["P"] = L.P.astype(dtype)
            d["chol"] = [c.astype(dtype) for c in L.chol]
        out.append(d)
    cache[key] = out
    H._cast_cache = cache
    return out


def vcycle(H, b, dtype=np.float64, level=0, smoother="multiplicative"):
    """One LS-AMG-DD V-cycle B^{-1} b (Section 2 error propagator E_TG, Section 6
    preamble): Schwarz pre-smoothing on the overlaps, coarse-grid correction, the adjoint
    post-smoothing; exact dense solve on the coarsest level.

    smoother="multiplicative": forward multiplicative Schwarz over colours ascending, the
    exact reverse order after the correction (the paper's numerical tests).
    smoother="additive": the fully parallel block Schwarz variant that Section 2 also allows,
    x += theta sum_i R_Omega_i^T A_Omega_i^{-1} R_Omega_i r before and after the correction.
    Reading (the paper gives no damping): theta = 1 / (number of colours).  Subdomains of one
    colour do not conflict, so the A-projections of a colour sum to an A-orthogonal
    projection and lambda_max(theta sum_i P_i) <= 1: the smoother is A-non-expansive."""
    if smoother not in ("multiplicative", "additive"):
        raise ValueError(f"unknown smoother {smoother!r}")
    ops = _cast(H, dtype)
    return _vc(H, ops, np.asarray(b, dtype), level, dtype, smoother)


def _vc(H, ops, b, l, dtype, smoother="multiplicative"):
    L = H.levels[l]
    op = ops[l]
    if L.coarsest:
        y = sla.solve_triangular(op["L"], b, lower=True)
        return sla.solve_triangular(op["L"].T, y, lower=False).astype(dtype)
    A = op["A"]
    x = np.zeros(L.n, dtype)
    res = b.copy()

    def solve_local(i, r):
        Lc = op["chol"][i]
        y = sla.solve_triangular(Lc, r[L.Omega[i]], lower=True)
        return sla.solve_triangular(Lc.T, y, lower=False).astype(dtype)

    def local(i):
        Om = L.Omega[i]
        d = solve_local(i, res)
        x[Om] += d
        res[:] = res - (A[:, Om] @ d).astype(dtype)

    def additive():
        theta = dtype(1.0 / (int(np.max(L.colour)) + 1))
        dx = np.zeros(L.n, dtype)
        for i in range(L.nagg):
            dx[L.Omega[i]] += solve_local(i, res)
        x[:] = x + theta * dx
        res[:] = b - (A @ x).astype(dtype)

    if smoother == "additive":
        additive()
    else:
        for i in L.sweep:
            local(i)
    rc = (op["P"].T @ res).astype(dtype)
    ec = _vc(H, ops, rc, l + 1, dtype, smoother)
    x += (op["P"] @ ec).astype(dtype)
    res[:] = b - (A @ x).astype(dtype)
    if smoother == "additive":
        additive()
    else:
        for i in reversed(L.sweep):
            local(i)
    return x


def stationary(H, b, x0, rtol=1e-10, maxit=500, smoother="multiplicative"):
    """The standalone V-cycle iteration of the paper's tests (Section 6 preamble):
    x <- x + B^{-1}(b - A x) from the given (random) initial iterate, stopped when the l2 norm
    of the residual has fallen by rtol relative to the initial residual.
    Returns (x, iterations, residual history ||r_k|| / ||r_0||)."""
    A = H.levels[0].A
    x = np.array(x0, float)
    r = b - A @ x
    r0 = np.linalg.norm(r)
    hist = [1.0]
    for it in range(1, maxit + 1):
        x += vcycle(H, r, smoother=smoother)
        r = b - A @ x
        hist.append(np.linalg.norm(r) / r0)
        if hist[-1] <= rtol:
            return x, it, hist
    return x, maxit, hist


def pcg(A, b, prec, rtol=1e-8, maxit=1000, x0=None):
    """Preconditioned CG in FP64 (x0 = 0 by default), stop at ||r|| <= rtol ||b||.
    Returns (x, iters, relres_history)."""
    b = np.asarray(b, float)
    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    r = b - A(x)
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= rtol:
            return x, it, hist
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist


def fcg(A, b, prec, rtol=1e-8, maxit=1000, x0=None):
    """Flexible CG(1) with the Polak-Ribiere coefficient
    beta_k = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k) (Notay 2000), FP64 vectors."""
    b = np.asarray(b, float)
    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    r = b - A(x)
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r_old = r.copy()
        r -= alpha * q
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= rtol:
            return x, it, hist
        z = prec(r)
        rz_new = r @ z
        beta = (z @ (r - r_old)) / rz
        p = z + beta * p
        rz = rz_new
    return x, maxit, hist


# -----------------------------------------------------------------------------
# Adjoint gradient (outer-solver layer; not in the paper)
# -----------------------------------------------------------------------------
def elem_grad(elems, K, lam, x):
    """g_e = -lambda_e^T K_e x_e for A(theta) = sum_e theta_e R_e^T K_e R_e, because
    dx/dtheta_e = -A^{-1} R_e^T K_e R_e x and A is symmetric."""
    return np.array([-(lam[d] @ (Ke @ x[d])) for d, Ke in zip(elems, K)])


def adjoint_grad(n, elems, K, theta, b, x_star, solve):
    """Loss L = 1/2 ||x - x*||^2 with x = A(theta)^{-1} b; returns (L, x, g)."""
    x = solve(b)
    gx = x - x_star
    lam = solve(gx)
    return 0.5 * float(gx @ gx), x, elem_grad(elems, K, lam, x)
