"""Seeded synthetic finite-element inputs for the LS-AMG-DD workloads.

This module only *generates inputs*: element DOF maps, element matrices A_T,
per-element coefficients and right-hand sides.  It holds none of the LS-AMG-DD
arithmetic (no factorization, aggregation, splitting, eigenproblem or cycle),
so both the FP64 oracle and the CUDA path can consume it without sharing any
of the method's code.

The discretisations are quad/hex analogues of the paper's Section 6 problems
(conforming assembly A = sum_T R_T^T A_T R_T with A_T >= 0, Section 4 eq. 4.1):

* ``rt_quad``      -- classical Raviart-Thomas RT_[k] = Q_{k+1,k} x Q_{k,k+1} on a
                      uniform N x N quad mesh of the unit square, form
                      (div u, div v) + beta (u, v)   (cf. Section 6.1);
* ``bfs_quad``     -- bicubic Bogner-Fox-Schmit (Hermite) on N x N squares,
                      anisotropic hyperdiffusion in H^2 (cf. Section 6.2);
* ``q2_elasticity``-- vector Q2 hexahedra on N^3 cubes, small-strain elasticity,
                      clamp on x = 0 imposed by symmetric Nitsche (cf. Section 6.3);
* ``cg1_tri``      -- P1 (CG1) on N x N squares split into right triangles, scalar
                      diffusion with kappa = 1 + x + y and u = 0 by symmetric Nitsche
                      (the closure comparison of Section 5, Table 2).

Workload configurations (``config``) use ``seed = 20260700 + cfg``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rt_quad", "bfs_quad", "q2_elasticity", "cg1_tri", "config", "CONFIGS", "gauss01", "gll01",
]


# ----------------------------------------------------------------------------
# 1-D helpers on [0, 1]
# ----------------------------------------------------------------------------
def gauss01(q: int):
    """Gauss-Legendre points/weights mapped to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def gll01(p: int):
    """p Gauss-Lobatto-Legendre points on [0, 1] (p >= 2)."""
    if p == 2:
        return np.array([0.0, 1.0])
    # interior points: roots of P'_{p-1}
    c = np.zeros(p)
    c[-1] = 1.0
    dc = np.polynomial.legendre.legder(c)
    r = np.sort(np.real(np.polynomial.legendre.legroots(dc)))
    x = np.concatenate([[-1.0], r, [1.0]])
    return 0.5 * (x + 1.0)


def lagrange_1d(nodes, x):
    """Values and first derivatives of the Lagrange basis on ``nodes`` at ``x``.

    Returns (V, D) with shape [len(nodes), len(x)]."""
    nodes = np.asarray(nodes, float)
    x = np.asarray(x, float)
    p = len(nodes)
    V = np.ones((p, len(x)))
    D = np.zeros((p, len(x)))
    for a in range(p):
        others = [b for b in range(p) if b != a]
        denom = np.prod([nodes[a] - nodes[b] for b in others]) if others else 1.0
        for b in others:
            V[a] *= (x - nodes[b])
        V[a] /= denom
        # derivative by the product rule
        for c in others:
            term = np.ones(len(x))
            for b in others:
                if b != c:
                    term = term * (x - nodes[b])
            D[a] += term
        D[a] /= denom
    return V, D


# ----------------------------------------------------------------------------
# Raviart-Thomas RT_[k] on quads
# ----------------------------------------------------------------------------
def _rt_ref(k: int, beta_h2: float, q: int):
    """Reference RT_[k] element matrix of (div u, div v) + beta*h^2 (u, v) on [0,1]^2.

    For an axis-aligned square of side h with nodal normal-component DOFs,
    (div u, div v)_T equals the reference div-div integral and (u, v)_T equals h^2
    times the reference mass, so the physical matrix is D_ref + beta h^2 M_ref.
    Local DOF order: x-component nodes (a in GLL_{k+2}, b in GL_{k+1}) with b fastest,
    then y-component nodes (a in GL_{k+1}, b in GLL_{k+2}) with b fastest."""
    xg = gll01(k + 2)
    xl, _ = gauss01(k + 1)
    qp, qw = gauss01(q)
    Vg, Dg = lagrange_1d(xg, qp)  # [k+2, q]
    Vl, _ = lagrange_1d(xl, qp)   # [k+1, q]
    nx = (k + 2) * (k + 1)
    nT = 2 * nx
    # values and divergence at quad points (ix over xi, iy over eta)
    val = np.zeros((nT, 2, q, q))
    div = np.zeros((nT, q, q))
    for a in range(k + 2):
        for b in range(k + 1):
            i = a * (k + 1) + b
            val[i, 0] = np.outer(Vg[a], Vl[b])
            div[i] = np.outer(Dg[a], Vl[b])
    for a in range(k + 1):
        for b in range(k + 2):
            i = nx + a * (k + 2) + b
            val[i, 1] = np.outer(Vl[a], Vg[b])
            div[i] = np.outer(Vl[a], Dg[b])
    W = np.outer(qw, qw)
    Dm = np.einsum("ixy,jxy,xy->ij", div, div, W)
    Mm = np.einsum("icxy,jcxy,xy->ij", val, val, W)
    K = Dm + beta_h2 * Mm
    return 0.5 * (K + K.T)


def rt_quad(N: int, k: int, beta: float, q: int | None = None):
    """RT_[k] on a uniform N x N quad mesh of the unit square.

    Returns (n, elem_dofs[int32, ne x nT], K_ref[nT x nT]) where every element's
    unit-coefficient matrix equals K_ref (uniform mesh, no boundary terms)."""
    if q is None:
        q = k + 2
    h = 1.0 / N
    K = _rt_ref(k, beta * h * h, q)
    kp = k + 1
    nV = (N + 1) * N * kp          # vertical edges: (i in 0..N, j in 0..N-1)
    nH = N * (N + 1) * kp          # horizontal edges: (i in 0..N-1, j in 0..N)
    nI = 2 * k * (k + 1)           # interior DOFs per element
    n = nV + nH + N * N * nI
    nx = (k + 2) * (k + 1)
    nT = 2 * nx
    ne = N * N
    dofs = np.empty((ne, nT), dtype=np.int64)
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    e = (jj * N + ii).ravel()
    ii = ii.ravel()
    jj = jj.ravel()
    for a in range(k + 2):
        for b in range(k + 1):
            loc = a * (k + 1) + b
            if a == 0:
                g = (ii * N + jj) * kp + b
            elif a == k + 1:
                g = ((ii + 1) * N + jj) * kp + b
            else:
                g = nV + nH + e * nI + (a - 1) * (k + 1) + b
            dofs[e, loc] = g
    for a in range(k + 1):
        for b in range(k + 2):
            loc = nx + a * (k + 2) + b
            if b == 0:
                g = nV + (jj * N + ii) * kp + a
            elif b == k + 1:
                g = nV + ((jj + 1) * N + ii) * kp + a
            else:
                g = nV + nH + e * nI + k * (k + 1) + a * k + (b - 1)
            dofs[e, loc] = g
    return n, dofs.astype(np.int32), K


# ----------------------------------------------------------------------------
# Bogner-Fox-Schmit bicubic on squares
# ----------------------------------------------------------------------------
def _hermite(t):
    """Cubic Hermite basis on [0,1]: (value0, slope0, value1, slope1), with 1st/2nd derivs."""
    H = np.stack([1 - 3 * t**2 + 2 * t**3, t - 2 * t**2 + t**3, 3 * t**2 - 2 * t**3, -t**2 + t**3])
    H1 = np.stack([-6 * t + 6 * t**2, 1 - 4 * t + 3 * t**2, 6 * t - 6 * t**2, -2 * t + 3 * t**2])
    H2 = np.stack([-6 + 12 * t, -4 + 6 * t, 6 - 12 * t, -2 + 6 * t])
    return H, H1, H2


def bfs_quad(N: int, eps: float = 1e-6, q: int = 4):
    """BFS bicubic elements on an N x N mesh of the unit square for
    a(u,v) = int (b^T Hu b)(b^T Hv b) + eps int Hu:Hv + int u v,
    b = (-(y-1/2), x-1/2)/r (unit circular field about the centre).

    Vertex DOFs (u, u_x, u_y, u_xy) in physical units.  Returns (n, elem_dofs, elem_mats)."""
    h = 1.0 / N
    qp, qw = gauss01(q)
    H, H1, H2 = _hermite(qp)          # [4, q]
    # 1-D basis in physical units: (node, kind) with kind 0 = value, 1 = slope (scaled by h)
    scale = np.array([1.0, h, 1.0, h])
    V = H * scale[:, None]
    Dx = H1 * scale[:, None] / h
    DDx = H2 * scale[:, None] / (h * h)
    # local DOF order: vertex v in (0,0),(1,0),(0,1),(1,1) -> (a,b); DOF d in (u, ux, uy, uxy)
    verts = [(0, 0), (1, 0), (0, 1), (1, 1)]
    comps = [(0, 0), (1, 0), (0, 1), (1, 1)]   # (slope in x?, slope in y?)
    nT = 16
    fx = np.zeros((nT, 3, q))   # x-factor value, d/dx, d2/dx2
    fy = np.zeros((nT, 3, q))
    for vi, (a, b) in enumerate(verts):
        for di, (sx, sy) in enumerate(comps):
            loc = 4 * vi + di
            ix = 2 * a + sx
            iy = 2 * b + sy
            fx[loc] = [V[ix], Dx[ix], DDx[ix]]
            fy[loc] = [V[iy], Dx[iy], DDx[iy]]
    u = np.einsum("ix,iy->ixy", fx[:, 0], fy[:, 0])
    uxx = np.einsum("ix,iy->ixy", fx[:, 2], fy[:, 0])
    uyy = np.einsum("ix,iy->ixy", fx[:, 0], fy[:, 2])
    uxy = np.einsum("ix,iy->ixy", fx[:, 1], fy[:, 1])
    Wq = np.outer(qw, qw) * h * h
    Mloc = np.einsum("ixy,jxy,xy->ij", u, u, Wq)
    Hloc = np.einsum("ixy,jxy,xy->ij", uxx, uxx, Wq) + np.einsum("ixy,jxy,xy->ij", uyy, uyy, Wq) \
        + 2 * np.einsum("ixy,jxy,xy->ij", uxy, uxy, Wq)
    ne = N * N
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    X = (ii[:, None, None] + qp[None, :, None]) * h   # [ne, qx, qy]
    Y = (jj[:, None, None] + qp[None, None, :]) * h
    dx = X - 0.5
    dy = Y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    bx = -dy / r
    by = dx / r
    # b^T H b for each basis function at each quad point: [ne, nT, q, q]
    bHb = (bx * bx)[:, None] * uxx[None] + (by * by)[:, None] * uyy[None] + 2 * (bx * by)[:, None] * uxy[None]
    A = np.einsum("eixy,ejxy,xy->eij", bHb, bHb, Wq)
    A += eps * Hloc[None] + Mloc[None]
    A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    dofs = np.empty((ne, nT), dtype=np.int64)
    for vi, (a, b) in enumerate(verts):
        node = (jj + b) * (N + 1) + (ii + a)
        for di in range(4):
            dofs[:, 4 * vi + di] = 4 * node + di
    n = 4 * (N + 1) ** 2
    return n, dofs.astype(np.int32), A


# ----------------------------------------------------------------------------
# Q2 hexahedral vector elasticity
# ----------------------------------------------------------------------------
def _q2_ref(nu: float, h: float, q: int = 3, nitsche_face: bool = False):
    """Unit-E Q2 elasticity matrix on a cube of side h (plus the symmetric Nitsche
    clamp terms on its x = 0 face if ``nitsche_face``).  Local DOF = 3*node + comp,
    node = (c*3 + b)*3 + a with a the x-index (fastest)."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    nodes = np.array([0.0, 0.5, 1.0])
    qp, qw = gauss01(q)
    V, D = lagrange_1d(nodes, qp)   # [3, q]
    D = D / h
    nn = 27
    # gradients of scalar shape functions at quad points: [nn, 3, q, q, q]
    phi = np.zeros((nn, q, q, q))
    grad = np.zeros((nn, 3, q, q, q))
    for c in range(3):
        for b in range(3):
            for a in range(3):
                i = (c * 3 + b) * 3 + a
                phi[i] = np.einsum("x,y,z->xyz", V[a], V[b], V[c])
                grad[i, 0] = np.einsum("x,y,z->xyz", D[a], V[b], V[c])
                grad[i, 1] = np.einsum("x,y,z->xyz", V[a], D[b], V[c])
                grad[i, 2] = np.einsum("x,y,z->xyz", V[a], V[b], D[c])
    W = np.einsum("x,y,z->xyz", qw, qw, qw) * h**3
    nT = 3 * nn
    # grad of vector basis (node i, comp c): G[dof, comp_row, deriv, ...]
    Gv = np.zeros((nT, 3, 3, q, q, q))
    for i in range(nn):
        for c in range(3):
            Gv[3 * i + c, c] = grad[i]
    eps = 0.5 * (Gv + np.swapaxes(Gv, 1, 2))
    divv = np.einsum("iccxyz->ixyz", Gv)
    K = 2 * mu * np.einsum("iabxyz,jabxyz,xyz->ij", eps, eps, W) + lam * np.einsum("ixyz,jxyz,xyz->ij", divv, divv, W)
    if nitsche_face:
        # face x = 0 (xi = 0): outward normal n = (-1, 0, 0); facet size h
        Vf0, Df0 = lagrange_1d(nodes, np.array([0.0]))
        Df0 = Df0 / h
        Wf = np.outer(qw, qw) * h * h
        gamma = 24.0 * 2**2 * (lam + 2 * mu) / h
        phif = np.zeros((nn, q, q))
        gradf = np.zeros((nn, 3, q, q))
        for c in range(3):
            for b in range(3):
                for a in range(3):
                    i = (c * 3 + b) * 3 + a
                    phif[i] = Vf0[a, 0] * np.outer(V[b], V[c])
                    gradf[i, 0] = Df0[a, 0] * np.outer(V[b], V[c])
                    gradf[i, 1] = Vf0[a, 0] * np.outer(D[b], V[c])
                    gradf[i, 2] = Vf0[a, 0] * np.outer(V[b], D[c])
        Gf = np.zeros((nT, 3, 3, q, q))
        Uf = np.zeros((nT, 3, q, q))
        for i in range(nn):
            for c in range(3):
                Gf[3 * i + c, c] = gradf[i]
                Uf[3 * i + c, c] = phif[i]
        epsf = 0.5 * (Gf + np.swapaxes(Gf, 1, 2))
        divf = np.einsum("iccyz->iyz", Gf)
        nvec = np.array([-1.0, 0.0, 0.0])
        sig = 2 * mu * epsf + lam * divf[:, None, None] * np.eye(3)[None, :, :, None, None]
        sn = np.einsum("iabyz,b->iayz", sig, nvec)          # sigma(u) n
        C = np.einsum("iayz,jayz,yz->ij", sn, Uf, Wf)        # <sigma(phi_i) n, phi_j>
        Mf = np.einsum("iayz,jayz,yz->ij", Uf, Uf, Wf)
        K = K - C - C.T + gamma * Mf
    return 0.5 * (K + K.T)


def q2_elasticity(N: int, nu: float = 0.45, E_elem=None, nitsche: bool = True):
    """Q2 vector elasticity on N^3 cubes of the unit cube, clamp x = 0 by symmetric Nitsche.

    ``E_elem`` (length N^3, default ones) scales each element's form.
    Returns (n, elem_dofs, elem_mats)."""
    h = 1.0 / N
    K0 = _q2_ref(nu, h)
    K1 = _q2_ref(nu, h, nitsche_face=True) if nitsche else K0
    M = 2 * N + 1
    ne = N**3
    kk, jj, ii = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    kk = kk.ravel()
    dofs = np.empty((ne, 81), dtype=np.int64)
    for c in range(3):
        for b in range(3):
            for a in range(3):
                loc = (c * 3 + b) * 3 + a
                node = ((2 * kk + c) * M + (2 * jj + b)) * M + (2 * ii + a)
                for comp in range(3):
                    dofs[:, 3 * loc + comp] = 3 * node + comp
    if E_elem is None:
        E_elem = np.ones(ne)
    A = np.where((ii == 0)[:, None, None], K1[None], K0[None]) * np.asarray(E_elem, float)[:, None, None]
    n = 3 * M**3
    return n, dofs.astype(np.int32), A


# ----------------------------------------------------------------------------
# Workload configurations
# ----------------------------------------------------------------------------
CONFIGS = {
    1: dict(kind="rt", N=16, k=0, beta=1e-4, q=2, c_tau=0.75, coef=None),
    2: dict(kind="rt", N=256, k=3, beta=1e-6, q=5, c_tau=0.75, coef="lognormal"),
    3: dict(kind="bfs", N=512, eps=1e-6, c_tau=1.0),
    4: dict(kind="q2", N=48, nu=0.45, E=(1.0, 1e4), block=6, nrhs=16, c_tau=0.75),
    5: dict(kind="rt", N=128, k=1, beta=1e-6, q=3, c_tau=0.75, coef="lognormal", adjoint=True),
}


def cg1_tri(N: int, gamma: float = 10.0):
    """P1 elements on a uniform N x N grid of the unit square, every square split along its
    (i, j)-(i+1, j+1) diagonal into two right triangles; -div(kappa grad u) = f with
    kappa(x, y) = 1 + x + y and u = 0 on the boundary imposed weakly by symmetric Nitsche.

    Element matrices (exact: grad phi is constant and kappa linear, so the volume term is
    (grad phi_p . grad phi_q) |T| kappa(centroid); edge terms use 2-point Gauss, exact for the
    cubic integrands):  K_T + sum over the element's boundary edges e of
        -<kappa d_n phi_q, phi_p>_e - <kappa d_n phi_p, phi_q>_e + (gamma / h) <kappa phi_p, phi_q>_e.
    gamma = 10 keeps every boundary element block positive semidefinite for this mesh.

    Returns (n, elem_dofs [2N^2, 3] int32, elem_mats [2N^2, 3, 3]) with DOF = j (N + 1) + i
    for the vertex (i h, j h).  The gradients of the two vertices on a hypotenuse are
    orthogonal, so their assembled entry of A cancels exactly (it is 0 in both triangles)."""
    h = 1.0 / N
    n = (N + 1) ** 2

    def vid(i, j):
        return j * (N + 1) + i

    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    dofs, mats = [], []
    for j in range(N):
        for i in range(N):
            for tri in (((i, j), (i + 1, j), (i + 1, j + 1)), ((i, j), (i + 1, j + 1), (i, j + 1))):
                X = np.array([[a * h, b * h] for a, b in tri])
                M = np.array([[1.0, X[0, 0], X[0, 1]], [1.0, X[1, 0], X[1, 1]], [1.0, X[2, 0], X[2, 1]]])
                C = np.linalg.inv(M)                 # phi_k(x, y) = C[0, k] + C[1, k] x + C[2, k] y
                grad = C[1:, :].T                    # [3, 2]
                area = 0.5 * abs(np.linalg.det(M))
                cen = X.mean(axis=0)
                K = (grad @ grad.T) * area * (1.0 + cen[0] + cen[1])
                for a, b in ((0, 1), (1, 2), (2, 0)):
                    P, Q = tri[a], tri[b]
                    on = ((P[0] == Q[0] and P[0] in (0, N)) or (P[1] == Q[1] and P[1] in (0, N)))
                    if not on:
                        continue
                    t = np.array([Q[0] - P[0], Q[1] - P[1]], float)
                    nvec = np.array([t[1], -t[0]])
                    if nvec @ (np.array([P[0] * h, P[1] * h]) - cen) < 0:
                        nvec = -nvec                 # outward
                    for qp in gp:
                        xy = (1 - qp) * X[a] + qp * X[b]
                        w = 0.5 * h                      # 2-point Gauss on an edge of length h
                        kap = 1.0 + xy[0] + xy[1]
                        phi = C[0, :] + C[1, :] * xy[0] + C[2, :] * xy[1]
                        dn = grad @ nvec
                        K += w * kap * (-np.outer(phi, dn) - np.outer(dn, phi) + (gamma / h) * np.outer(phi, phi))
                dofs.append([vid(*v) for v in tri])
                mats.append(0.5 * (K + K.T))
    return n, np.array(dofs, np.int32), np.array(mats)


def config(cfg: int, N: int | None = None, expand: bool = True):
    """Seeded inputs for workload ``cfg`` (1..5), optionally on a smaller mesh ``N``.

    Returns a dict with n, elem_dofs [ne, nT] int32, elem_mats [ne, nT, nT] f64
    (unit-coefficient matrices K_e), coef [ne] f64 or None (A_T = coef_e K_e),
    b [nrhs, n] f64, c_tau, and for the adjoint workload x_star [n]."""
    spec = dict(CONFIGS[cfg])
    if N is not None:
        spec["N"] = N
    rng = np.random.default_rng(20260700 + cfg)
    out = dict(cfg=cfg, c_tau=spec["c_tau"], N=spec["N"], kind=spec["kind"])
    if spec["kind"] == "rt":
        n, dofs, K = rt_quad(spec["N"], spec["k"], spec["beta"], spec["q"])
        ne = dofs.shape[0]
        mats = np.broadcast_to(K, (ne,) + K.shape)
        if expand:
            mats = np.ascontiguousarray(mats)
        coef = rng.lognormal(0.0, 1.0, size=ne) if spec["coef"] == "lognormal" else None
        out.update(k=spec["k"], beta=spec["beta"])
    elif spec["kind"] == "bfs":
        n, dofs, mats = bfs_quad(spec["N"], spec["eps"])
        coef = None
    else:
        Nm = spec["N"]
        nb = max(1, Nm // spec["block"])
        Eblk = np.where(rng.random(nb**3) < 0.5, spec["E"][0], spec["E"][1])
        kk, jj, ii = np.meshgrid(np.arange(Nm), np.arange(Nm), np.arange(Nm), indexing="ij")
        bsz = max(1, Nm // nb)
        bid = ((np.minimum(kk.ravel() // bsz, nb - 1) * nb + np.minimum(jj.ravel() // bsz, nb - 1)) * nb
               + np.minimum(ii.ravel() // bsz, nb - 1))
        n, dofs, mats = q2_elasticity(Nm, spec["nu"], Eblk[bid])
        coef = None
    nrhs = spec.get("nrhs", 1)
    b = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    out.update(n=n, elem_dofs=dofs, elem_mats=mats, coef=coef, b=b)
    if spec.get("adjoint"):
        out["x_star"] = np.random.default_rng(20260700 + cfg + 1).uniform(-1.0, 1.0, size=n)
    return out
