"""Two-level overlapping additive Schwarz preconditioner M_EH(+Rot) (oracle;
test infrastructure only).

Sec. 2 and Sec. 4.3 (Eqs. juan001/juan002):
    M^{-1} r = sum_i R_i^T K_i^{-1} R_i r  +  R_0^T K_0^{-1} R_0 r,
    K_i = R_i K R_i^T (Eq. localproblemsE),   K_0 = R_0 K R_0^T (Sec. 2.1),
with the columns of R_0^T the coarse basis of V_{0,H} (Sec. 4.1): chi_l [psi, 0]
and chi_l [0, psi] for the heat-operator eigenfunctions psi of each coarse-node
neighbourhood omega_l (Eq. juaneheateigenproblem), plus the rotation
enrichment chi_l r of Sec. 4.2 (Eq. juan002c).

Readings of what the paper leaves open (each restated where used):
  * overlap: D'_i is the coarse block D_i grown by `overlap` element layers in
    every axis direction (box distance), clipped to the domain; overlap = -1
    takes the paper's Sec. 5 geometry D'_i = omega_i.
  * local DOFs of D'_i: the free DOFs at nodes strictly inside D'_i plus nodes
    of D'_i on the domain boundary (so K_i is a principal submatrix of K).
  * chi_l: the bilinear/trilinear hat of coarse node y_l on the coarse grid.
  * heat eigenproblem: kappa = E_e per element; Q1 stiffness and kappa-weighted
    consistent mass on omega_l; natural (Neumann) on the part of the boundary
    of omega_l that is not Dirichlet for component c; Dirichlet at the nodes of
    omega_l where component c is Dirichlet globally.
  * threshold: keep every eigenpair with lambda < tau = tau_scale / H^2
    (H the coarse block width in elements, tau_scale = 2), at least one and at
    most max_modes (16) per (omega_l, component): the threshold decides, the
    cap only bounds storage (the 400x400 example of Sec. 1.4 caps at 6).
  * a coarse node lying on Gamma_D,c gets no component-c heat basis; its
    rotation is dropped when it is Dirichlet in every component.
  * rotation about y_l: (-(y - Y_l), x - X_l) in 2D; the three axis rotations
    in 3D.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem


def _axis_sizes(prob):
    return (prob.nx, prob.ny) if prob.dim == 2 else (prob.nx, prob.ny, prob.nz)


def subdomain_boxes(prob):
    """Element boxes [(lo, hi) per axis] of the overlapping subdomains D'_i
    (Eq. def:overlapping-subdomains)."""
    n = _axis_sizes(prob)
    H = prob.blk
    for a in range(prob.dim):
        if n[a] % H[a] != 0:
            raise ValueError("block size must divide the mesh")
    nb = [n[a] // H[a] for a in range(prob.dim)]
    boxes = []
    if prob.overlap >= 0:
        d = prob.overlap
        # row-major over blocks, x fastest
        for idx in itertools.product(*[range(nb[a]) for a in reversed(range(prob.dim))]):
            idx = idx[::-1]
            boxes.append(tuple((max(0, idx[a] * H[a] - d), min(n[a], (idx[a] + 1) * H[a] + d))
                               for a in range(prob.dim)))
    else:
        # D'_i = omega_i: one subdomain per coarse node
        for idx in itertools.product(*[range(nb[a] + 1) for a in reversed(range(prob.dim))]):
            idx = idx[::-1]
            boxes.append(tuple((max(0, (idx[a] - 1) * H[a]), min(n[a], (idx[a] + 1) * H[a]))
                               for a in range(prob.dim)))
    return boxes


def box_nodes(prob, box, strict=True):
    """Global node ids of the nodes of an element box, row-major (x fastest).
    strict: drop box-boundary nodes that are not on the domain boundary."""
    n = _axis_sizes(prob)
    rng = []
    for a, (lo, hi) in enumerate(box):
        if strict:
            rng.append(np.arange(lo + (lo > 0), hi - (hi < n[a]) + 1))
        else:
            rng.append(np.arange(lo, hi + 1))
    if prob.dim == 2:
        j, i = np.meshgrid(rng[1], rng[0], indexing="ij")
        return (j * (n[0] + 1) + i).ravel()
    k, j, i = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    return ((k * (n[1] + 1) + j) * (n[0] + 1) + i).ravel()


def box_elements(prob, box):
    n = _axis_sizes(prob)
    rng = [np.arange(lo, hi) for lo, hi in box]
    if prob.dim == 2:
        j, i = np.meshgrid(rng[1], rng[0], indexing="ij")
        return (j * n[0] + i).ravel()
    k, j, i = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    return ((k * n[1] + j) * n[0] + i).ravel()


def local_dofs(prob, box, free):
    nodes = box_nodes(prob, box, strict=True)
    d = prob.dim
    dofs = (d * nodes[:, None] + np.arange(d)[None, :]).ravel()
    return dofs[free[dofs]]


def coarse_nodes(prob):
    """Coarse vertex grid of T^H: list of (index tuple, fine-node coordinates)."""
    n = _axis_sizes(prob)
    H = prob.blk
    nb = [n[a] // H[a] for a in range(prob.dim)]
    out = []
    for idx in itertools.product(*[range(nb[a] + 1) for a in reversed(range(prob.dim))]):
        idx = idx[::-1]
        out.append((idx, tuple(idx[a] * H[a] for a in range(prob.dim))))
    return out


def neighbourhood_box(prob, idx):
    """omega_l: union of the coarse elements that touch coarse node idx."""
    n = _axis_sizes(prob)
    H = prob.blk
    return tuple((max(0, (idx[a] - 1) * H[a]), min(n[a], (idx[a] + 1) * H[a])) for a in range(prob.dim))


def chi(prob, y, coords):
    """Coarse hat of the node at fine coordinates y (multilinear on T^H)."""
    v = np.ones(coords.shape[0])
    for a in range(prob.dim):
        v *= np.maximum(0.0, 1.0 - np.abs(coords[:, a] - y[a]) / prob.blk[a])
    return v


def heat_matrices(prob, box, E):
    """Q1 heat stiffness and kappa-weighted consistent mass on an element box,
    kappa = E_e (Eq. juaneheateigenproblem); returns dense (K^l, M^l) over the
    closed box's nodes (row-major, x fastest) and those global node ids."""
    Kh, Mh = fem.heat_element(prob.dim)
    nodes = box_nodes(prob, box, strict=False)
    loc = {int(g): a for a, g in enumerate(nodes)}
    els = box_elements(prob, box)
    en = fem.element_nodes(prob)[els]
    nn = nodes.size
    Kl = np.zeros((nn, nn))
    Ml = np.zeros((nn, nn))
    for e, enodes in zip(els, en):
        li = np.array([loc[int(g)] for g in enodes])
        Kl[np.ix_(li, li)] += E[e] * Kh
        Ml[np.ix_(li, li)] += E[e] * Mh
    return Kl, Ml, nodes


def heat_eigenpairs(Kl, Ml, tau, max_modes):
    """Smallest eigenpairs of K^l psi = lambda M^l psi (dense LAPACK eigh as a
    library step).  Returns (eigenvalues checked: the first max_modes+1,
    the number below tau, the selected eigenvectors)."""
    n = Kl.shape[0]
    k = min(max_modes + 1, n)
    lam, vec = sla.eigh(Kl, Ml, subset_by_index=[0, k - 1])
    # the count below tau over the whole spectrum (it may exceed max_modes + 1)
    below = int(sla.eigh(Kl, Ml, eigvals_only=True, subset_by_value=(-np.inf, tau)).size)
    m = min(max(below, 1), max_modes, n)
    return lam, below, vec[:, :m]


_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 output function (Steele, Lea & Flood, 2014) of the 64-bit
    counters x (numpy uint64 array): the published counter-based generator
    both sides use for the random loads of the randomized coarse space."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
    return z ^ (z >> np.uint64(31))


def random_loads(node, n, snapshots):
    """Uniform values in [-1/2, 1/2) for snapshot s at box node i of coarse
    node `node`: counter (node << 40) | (s << 32) | i, top 53 bits (distinct
    counters for s < 256 and i < 2^32)."""
    i = np.arange(n, dtype=np.uint64)
    F = np.empty((n, snapshots))
    for s in range(snapshots):
        ctr = (np.uint64(node) << np.uint64(40)) | (np.uint64(s) << np.uint64(32)) | i
        F[:, s] = (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 - 0.5
    return F


def heat_eigenpairs_rand(Kl, Ml, tau, max_modes, F, sigma):
    """Randomized coarse basis of the heat problem, following the randomized
    algorithm of the paper's Sec. 'A randomized algorithm for eigenvalues
    computation': random loads of zero total (columns of F, free nodes),
    local solves (K + sigma M) u_l = f_l (sigma: the small shift that makes
    the Neumann problem solvable, as in the deterministic eigensolve), the
    span of the snapshots and the constant (the heat operator's rigid mode)
    by SVD, and the reduced generalized eigenproblem in that span.  Returns
    (reduced eigenvalues, count below tau, selected vectors)."""
    F = F - F.mean(axis=0, keepdims=True)
    U = np.linalg.solve(Kl + sigma * Ml, F)
    Wsnap = np.column_stack([U, np.ones(Kl.shape[0])])
    Q, sv, _ = np.linalg.svd(Wsnap, full_matrices=False)
    Q = Q[:, sv > 1e-12 * sv[0]]
    lam, phi = sla.eigh(Q.T @ Kl @ Q, Q.T @ Ml @ Q)
    below = int(np.sum(lam < tau))
    m = min(max(below, 1), max_modes, lam.size)
    return lam, below, Q @ phi[:, :m]


class CoarseSpace:
    """V_{0,H} (+ rotations): the rows of R_0 and per-neighbourhood records."""

    def __init__(self, prob, E, rotations=True, tau_scale=2.0, max_modes=16, method="eig", snapshots=15):
        self.prob = prob
        self.tau = tau_scale / float(max(prob.blk)) ** 2
        # shift of the local solves of the randomized basis (the GPU's heat shift)
        sigma = self.tau * max(prob.Emin / prob.E0, 1e-10)
        free = fem.free_mask(prob)
        coords = fem.node_coords(prob)
        d = prob.dim
        rows, cols, vals = [], [], []
        self.records = []  # (coarse idx, component or 'rot', eigenvalues, n_below, m)
        self.cap_hits = 0
        nb = 0
        cache = {}
        for idx, y in coarse_nodes(prob):
            box = neighbourhood_box(prob, idx)
            ynode = fem_node_id(prob, y)
            Kl = Ml = None
            nodes = box_nodes(prob, box, strict=False)
            ch = chi(prob, y, coords[nodes])
            for c in range(d):
                if not free[d * ynode + c]:
                    continue
                keep = free[d * nodes + c]
                key = (box, keep.tobytes())
                if key not in cache:
                    if Kl is None:
                        Kl, Ml, _ = heat_matrices(prob, box, E)
                    ki = np.flatnonzero(keep)
                    Kf, Mf = Kl[np.ix_(ki, ki)], Ml[np.ix_(ki, ki)]
                    if method == "eig":
                        cache[key] = heat_eigenpairs(Kf, Mf, self.tau, max_modes)
                    else:
                        # snapshots: at least `snapshots`, and the wanted modes + 5
                        exact = int(sla.eigh(Kf, Mf, eigvals_only=True, subset_by_value=(-np.inf, self.tau)).size)
                        M = max(snapshots, min(max(exact, 1), max_modes) + 5)
                        # no more loads than the free nodes can span beside the constant
                        M = max(0, min(M, Kf.shape[0] - 1))
                        lin = idx[0] + (prob.nx // prob.blk[0] + 1) * (
                            idx[1] + ((prob.ny // prob.blk[1] + 1) * idx[2] if prob.dim == 3 else 0))
                        F = random_loads(lin, nodes.size, M)[ki]
                        cache[key] = heat_eigenpairs_rand(Kf, Mf, self.tau, max_modes, F, sigma)
                lam, below, vec = cache[key]
                if below > max_modes:
                    self.cap_hits += 1
                ki = np.flatnonzero(keep)
                for j in range(vec.shape[1]):
                    v = np.zeros(nodes.size)
                    v[ki] = vec[:, j]
                    w = ch * v
                    nz = np.flatnonzero(w)
                    rows += [nb] * nz.size
                    cols += list(d * nodes[nz] + c)
                    vals += list(w[nz])
                    nb += 1
                self.records.append((idx, c, lam, below, vec.shape[1]))
            if rotations and any(free[d * ynode + c] for c in range(d)):
                rel = coords[nodes] - np.array(y, dtype=np.float64)[None, :]
                if d == 2:
                    rots = [np.stack([-rel[:, 1], rel[:, 0]], axis=1)]
                else:
                    rots = [np.stack([np.zeros(nodes.size), -rel[:, 2], rel[:, 1]], axis=1),
                            np.stack([rel[:, 2], np.zeros(nodes.size), -rel[:, 0]], axis=1),
                            np.stack([-rel[:, 1], rel[:, 0], np.zeros(nodes.size)], axis=1)]
                for rv in rots:
                    w = (ch[:, None] * rv)
                    gd = d * nodes[:, None] + np.arange(d)[None, :]
                    w = w.ravel()
                    gd = gd.ravel()
                    msk = (w != 0.0) & free[gd]
                    rows += [nb] * int(msk.sum())
                    cols += list(gd[msk])
                    vals += list(w[msk])
                    nb += 1
                self.records.append((idx, "rot", None, None, len(rots)))
        self.dim = nb
        self.R0 = sp.csr_matrix((np.array(vals), (np.array(rows), np.array(cols))), shape=(nb, prob.ndof))


def fem_node_id(prob, y):
    if prob.dim == 2:
        return int(y[1] * (prob.nx + 1) + y[0])
    return int((y[2] * (prob.ny + 1) + y[1]) * (prob.nx + 1) + y[0])


class Schwarz:
    """M_EH+Rot (rotations=True) or M_EH (rotations=False); with
    method="elastic" M_EE, the coarse space of oracle/elastic.py (Eq. 2lEp;
    modes_scale 2 takes twice as many eigenvectors), and with
    method="elastic_rand" its randomized variant M_EE;Rand."""

    def __init__(self, prob, rotations=True, tau_scale=2.0, max_modes=16, K=None, coarse=True, method="eig",
                 snapshots=15, modes_scale=1):
        self.prob = prob
        self.E = fem.simp(prob.rho, prob.E0, prob.Emin, prob.p)
        self.K = fem.assemble_K(prob, self.E) if K is None else K
        self.free = fem.free_mask(prob)
        self.boxes = subdomain_boxes(prob)
        self.dofs = []
        self.factors = []
        for box in self.boxes:
            dofs = local_dofs(prob, box, self.free)
            self.dofs.append(dofs)
            if dofs.size:
                Ki = self.K[dofs][:, dofs].toarray()
                self.factors.append(sla.cho_factor(Ki, lower=True))
            else:
                self.factors.append(None)
        self.coarse = None
        if coarse:
            if method == "elastic":
                from .elastic import ElasticCoarseSpace
                self.coarse = ElasticCoarseSpace(prob, self.E, modes_scale)
            elif method == "elastic_rand":
                from .elastic import ElasticCoarseSpace
                self.coarse = ElasticCoarseSpace(prob, self.E, modes_scale, "rand", snapshots)
            else:
                self.coarse = CoarseSpace(prob, self.E, rotations, tau_scale, max_modes, method, snapshots)
            R0 = self.coarse.R0
            self.K0 = (R0 @ self.K @ R0.T).toarray()
            # K_0^+ on span(R_0^T): the rotation vectors chi_l r_l are linearly
            # dependent whenever every coarse node keeps its rotation
            # (sum_l chi_l r_l = 0, the hats reproducing linear functions), so
            # the Galerkin correction is taken as the pseudo-inverse of the
            # diagonally scaled K_0 with numerically null directions dropped.
            d = 1.0 / np.sqrt(np.diag(self.K0))
            lam, V = np.linalg.eigh(self.K0 * d[:, None] * d[None, :])
            keep = lam > 1e-12 * lam.max()
            self.K0_scale = d
            self.K0_eig = (lam[keep], V[:, keep])
            self.coarse_dropped = int((~keep).sum())

    def local_part(self, r):
        """sum_i R_i^T K_i^{-1} R_i r (Eq. localproblemsE)."""
        z = np.zeros_like(r)
        for dofs, F in zip(self.dofs, self.factors):
            if F is not None:
                z[dofs] += sla.cho_solve(F, r[dofs])
        return z

    def coarse_part(self, r):
        """R_0^T K_0^{-1} R_0 r."""
        if self.coarse is None:
            return np.zeros_like(r)
        R0 = self.coarse.R0
        d = self.K0_scale
        lam, V = self.K0_eig
        c = d * (V @ ((V.T @ (d * (R0 @ r))) / lam))
        return R0.T @ c

    def apply(self, r):
        return self.local_part(r) + self.coarse_part(r)
