"""Finite-element part of the oracle (test infrastructure only).

Sec. 1.1 (Eqs. 6-9): linear elasticity -div sigma = f, sigma = E(x) C0 : eps,
discretised with bilinear (2D Q4) / trilinear (3D Hex8) Lagrange vector basis
functions on a uniform mesh of unit square/cube elements.  2D is plane stress
(Sec. 1.4).  Element moduli follow the SIMP law of Eq. 4:
    E_e = Emin + rho_e^p (Emax - Emin).
The element stiffness of element e is E_e * KE(nu), KE integrated with 2-point
Gauss rules per axis (exact for these polynomial integrands).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

GAUSS2 = (-1.0 / np.sqrt(3.0), 1.0 / np.sqrt(3.0))

# reference-element node signs, counter-clockwise (2D) / bottom then top face (3D)
Q4_NODES = ((-1, -1), (1, -1), (1, 1), (-1, 1))
HEX8_NODES = ((-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1),
              (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1))


def simp(rho, E0, Emin, p):
    """Eq. 4: E_e = Emin + rho_e^p (E0 - Emin)."""
    rho = np.asarray(rho, dtype=np.float64)
    return Emin + rho ** p * (E0 - Emin)


def d_plane_stress(nu):
    """Plane-stress constitutive matrix for E = 1 (C0 of Eq. 8 in 2D, Voigt
    order xx, yy, xy with engineering shear)."""
    return (1.0 / (1.0 - nu * nu)) * np.array(
        [[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]])


def d_iso3(nu):
    """Isotropic 3D constitutive matrix for E = 1 (Voigt xx, yy, zz, yz, xz, xy)."""
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] += 2.0 * mu
        D[3 + i, 3 + i] = mu
    return D


def _grad_shape(nodes, xi):
    """Gradients d N_a / d x of the (bi/tri)linear shape functions on a unit
    element (h = 1, so d xi / d x = 2) at reference point xi."""
    dim = len(xi)
    G = np.zeros((len(nodes), dim))
    for a, s in enumerate(nodes):
        for d in range(dim):
            g = 0.5 * s[d]
            for e in range(dim):
                if e != d:
                    g *= 0.5 * (1.0 + s[e] * xi[e])
            G[a, d] = g * 2.0
    return G


def _shape(nodes, xi):
    N = np.ones(len(nodes))
    for a, s in enumerate(nodes):
        for d in range(len(xi)):
            N[a] *= 0.5 * (1.0 + s[d] * xi[d])
    return N


def ke_q4(nu):
    """8x8 plane-stress Q4 stiffness, E = 1, unit square; DOF order
    [u0x, u0y, u1x, u1y, u2x, u2y, u3x, u3y]."""
    D = d_plane_stress(nu)
    KE = np.zeros((8, 8))
    detJ = 0.25  # (h/2)^2
    for xi in itertools.product(GAUSS2, GAUSS2):
        G = _grad_shape(Q4_NODES, xi)
        B = np.zeros((3, 8))
        for a in range(4):
            B[0, 2 * a] = G[a, 0]
            B[1, 2 * a + 1] = G[a, 1]
            B[2, 2 * a] = G[a, 1]
            B[2, 2 * a + 1] = G[a, 0]
        KE += B.T @ D @ B * detJ
    return KE


def ke_hex8(nu):
    """24x24 isotropic Hex8 stiffness, E = 1, unit cube; DOF = 3*a + c."""
    D = d_iso3(nu)
    KE = np.zeros((24, 24))
    detJ = 0.125
    for xi in itertools.product(GAUSS2, GAUSS2, GAUSS2):
        G = _grad_shape(HEX8_NODES, xi)
        B = np.zeros((6, 24))
        for a in range(8):
            B[0, 3 * a] = G[a, 0]
            B[1, 3 * a + 1] = G[a, 1]
            B[2, 3 * a + 2] = G[a, 2]
            B[3, 3 * a + 1] = G[a, 2]
            B[3, 3 * a + 2] = G[a, 1]
            B[4, 3 * a] = G[a, 2]
            B[4, 3 * a + 2] = G[a, 0]
            B[5, 3 * a] = G[a, 1]
            B[5, 3 * a + 1] = G[a, 0]
        KE += B.T @ D @ B * detJ
    return KE


def heat_element(dim):
    """Scalar Q1 element matrices for kappa = 1 on a unit element: stiffness
    int grad N_a . grad N_b and consistent mass int N_a N_b (used by the heat
    eigenproblem of Sec. 4.1)."""
    nodes = Q4_NODES if dim == 2 else HEX8_NODES
    n = len(nodes)
    Kh = np.zeros((n, n))
    Mh = np.zeros((n, n))
    detJ = 0.5 ** dim
    for xi in itertools.product(*([GAUSS2] * dim)):
        G = _grad_shape(nodes, xi)
        N = _shape(nodes, xi)
        Kh += G @ G.T * detJ
        Mh += np.outer(N, N) * detJ
    return Kh, Mh


# ----------------------------------------------------------------------------
# mesh numbering (same contract as the input generators)
# ----------------------------------------------------------------------------

def element_nodes(prob):
    """[n_el, 4] (2D) or [n_el, 8] (3D) global node ids in local node order."""
    nx, ny = prob.nx, prob.ny
    if prob.dim == 2:
        ey, ex = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ex, ey = ex.ravel(), ey.ravel()
        out = np.empty((ex.size, 4), dtype=np.int64)
        for a, (sx, sy) in enumerate(Q4_NODES):
            out[:, a] = (ey + (sy > 0)) * (nx + 1) + ex + (sx > 0)
        return out
    nz = prob.nz
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    out = np.empty((ex.size, 8), dtype=np.int64)
    for a, (sx, sy, sz) in enumerate(HEX8_NODES):
        out[:, a] = ((ez + (sz > 0)) * (ny + 1) + ey + (sy > 0)) * (nx + 1) + ex + (sx > 0)
    return out


def element_dofs(prob):
    en = element_nodes(prob)
    d = prob.dim
    return (d * en[:, :, None] + np.arange(d)[None, None, :]).reshape(en.shape[0], -1)


def node_coords(prob):
    """[n_nodes, dim] integer coordinates (unit spacing)."""
    nx, ny = prob.nx, prob.ny
    if prob.dim == 2:
        j, i = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel()], axis=1).astype(np.float64)
    k, j, i = np.meshgrid(np.arange(prob.nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)


def element_stiffness(prob):
    return ke_q4(prob.nu) if prob.dim == 2 else ke_hex8(prob.nu)


def assemble_K(prob, E=None):
    """Global stiffness (all DOFs, Dirichlet not yet removed) as CSR:
    K = sum_e E_e P_e^T KE P_e (standard FE assembly, Eq. 2)."""
    if E is None:
        E = simp(prob.rho, prob.E0, prob.Emin, prob.p)
    KE = element_stiffness(prob)
    edofs = element_dofs(prob)
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).ravel()
    cols = np.tile(edofs, (1, nd)).ravel()
    vals = (E[:, None] * KE.ravel()[None, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(prob.ndof, prob.ndof)).tocsr()
    K.sum_duplicates()
    return K


def apply_K_free(prob, x, E=None):
    """K x with Dirichlet rows and columns replaced by the identity (the
    operator of constrained_K), element by element without assembling K:
    y = sum_e E_e P_e^T KE P_e x (Eq. 2), x read as zero at Dirichlet DOFs
    and y[D] = x[D].  For residual checks at sizes where forming the CSR
    matrix costs more than the product."""
    if E is None:
        E = simp(prob.rho, prob.E0, prob.Emin, prob.p)
    free = free_mask(prob)
    xf = np.where(free, x, 0.0)
    KE = element_stiffness(prob)
    edofs = element_dofs(prob)
    ye = (xf[edofs] @ KE.T) * E[:, None]
    y = np.bincount(edofs.ravel(), weights=ye.ravel(), minlength=prob.ndof)
    return np.where(free, y, x)


def free_mask(prob):
    m = np.ones(prob.ndof, dtype=bool)
    m[prob.dirichlet] = False
    return m


def constrained_K(prob, K=None):
    """K with Dirichlet rows/columns replaced by the identity; for u with zeros
    at Dirichlet DOFs this applies the eliminated operator of Eq. 7/9 (V_0)."""
    if K is None:
        K = assemble_K(prob)
    m = free_mask(prob).astype(np.float64)
    Dm = sp.diags(m)
    return (Dm @ K @ Dm + sp.diags(1.0 - m)).tocsr()


def _residual_ext(A, x, b):
    """b - A x with every product and sum in extended precision (long double),
    so that the residual of an FP64 iterate is seen below FP64's own floor."""
    prod = A.data.astype(np.longdouble) * x.astype(np.longdouble)[A.indices]
    s = np.add.reduceat(prod, A.indptr[:-1]) if A.nnz else np.zeros(A.shape[0], np.longdouble)
    s[np.diff(A.indptr) == 0] = 0
    return b.astype(np.longdouble) - s


def true_residual(prob, u, f, K=None):
    """(relative residual ||f - K u|| / ||f|| with every product and sum in
    extended precision, the FP64 rounding floor eps ||(|K| |u|)|| / ||f|| of
    the same residual evaluated in FP64) on the free DOFs.  A solution
    rounded to FP64 cannot have a residual much below that floor, and an FP64
    evaluation of the residual cannot see below it."""
    if K is None:
        K = assemble_K(prob)
    free = np.flatnonzero(free_mask(prob))
    Kff = K[free][:, free].tocsr()
    r = _residual_ext(Kff, np.asarray(u, dtype=np.float64)[free], np.asarray(f, dtype=np.float64)[free])
    nf = float(np.linalg.norm(f[free]))
    rel = float(np.sqrt(np.sum(r * r))) / nf
    floor = np.finfo(np.float64).eps * float(np.linalg.norm(abs(Kff) @ np.abs(u[free]))) / nf
    return rel, floor


def direct_solve(prob, K=None, f=None, refine=8):
    """Sparse direct solve of K u = f on the free DOFs (Dirichlet DOFs = 0).

    The factorisation is SuperLU with symmetric (diagonal) pivoting, a library
    primitive.  Iterative refinement follows with the residual and the iterate
    kept in extended precision: with contrast 1e6-1e8 and a point load on soft
    material the displacements reach 1e6-1e7, and a plain FP64 solve (or FP64
    refinement) stalls at a K-norm error near 1e-8, the size of the parity
    tolerance itself.  Returns u rounded to FP64 with zeros at Dirichlet DOFs,
    one row per right-hand side."""
    if K is None:
        K = assemble_K(prob)
    if f is None:
        f = prob.f
    f = np.atleast_2d(f)
    free = np.flatnonzero(free_mask(prob))
    Kff = K[free][:, free].tocsr()
    lu = spla.splu(Kff.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    u = np.zeros_like(f)
    for k in range(f.shape[0]):
        b = f[k, free]
        x = lu.solve(b).astype(np.longdouble)
        for _ in range(refine):
            r = _residual_ext(Kff, x, b)
            d = lu.solve(np.asarray(r, dtype=np.float64))
            x = x + d.astype(np.longdouble)
        u[k, free] = np.asarray(x, dtype=np.float64)
    return u


def compliance(f, u):
    """g_0 = f^T u (Eq. 1)."""
    return float(np.dot(f, u))


def sensitivity(prob, u):
    """Eq. 1003 for the compliance objective: dg_0/drho_e = -u^T (dK/drho_e) u.
    With K = sum_e E_e P_e^T KE P_e and E_e of Eq. 4,
        dg_0/drho_e = -p rho_e^(p-1) (Emax - Emin) u_e^T KE u_e.
    Returns (dc [n_el], g_0 = sum_e E_e u_e^T KE u_e), the latter equal to
    f^T u (Eq. 1) when u solves K u = f."""
    KE = element_stiffness(prob)
    ue = np.asarray(u, dtype=np.float64)[element_dofs(prob)]
    q = np.einsum("ei,ij,ej->e", ue, KE, ue)
    rho = np.asarray(prob.rho, dtype=np.float64)
    dc = -prob.p * rho ** (prob.p - 1.0) * (prob.E0 - prob.Emin) * q
    E = simp(rho, prob.E0, prob.Emin, prob.p)
    return dc, float(np.sum(E * q))


def oc_update(rho, dc, volfrac, move=0.2, steps=80, lam_lo=1e-40, lam_hi=1e40):
    """Optimality-criteria density update of the topology-optimisation loop
    the state solve serves (Sec. 1: 'the densities are usually updated using
    ... the optimality criteria method'): with B_e = max(-dc_e, 0),
        rho_e(lam) = clamp(rho_e sqrt(B_e / lam), max(0, rho_e - move), min(1, rho_e + move)),
    and the multiplier lam chosen by bisection of log(lam) (steps halvings of
    [lam_lo, lam_hi]) so that the mean density equals volfrac (elements of
    equal volume): the mean is non-increasing in lam."""
    rho = np.asarray(rho, dtype=np.float64)
    B = np.maximum(-np.asarray(dc, dtype=np.float64), 0.0)
    lo_b = np.maximum(0.0, rho - move)
    hi_b = np.minimum(1.0, rho + move)

    def update(lam):
        return np.clip(rho * np.sqrt(B / lam), lo_b, hi_b)

    lo, hi = lam_lo, lam_hi
    target = volfrac * rho.size
    for _ in range(steps):
        mid = np.sqrt(lo * hi)
        if np.sum(update(mid)) > target:
            lo = mid
        else:
            hi = mid
    return update(np.sqrt(lo * hi))
