"""Elasticity-eigenproblem coarse space of M_EE (oracle; test infrastructure
only).

Sec. "Generalized multiscale coarse finite element spaces for the elasticity
equation" (Eq. juanelasticityeigenproblem, Eq. 3001): on each coarse-node
neighbourhood omega_l,
    -div sigma(psi) = lambda E(x) psi   in omega_l,
Neumann on the boundary of omega_l, Dirichlet where that boundary meets the
Dirichlet part of the domain boundary; in matrix form K_E^l phi = lambda M^l phi.
The coarse space V_{0,E} (Eq. juaneq:VOE) is spanned by chi_l psi_{i,l}; the
two-level preconditioner M_EE (Eq. 2lEp) pairs it with the same elasticity
local solves as M_EH.

Readings of what the paper leaves open (each restated where used):
  * M^l is the E-weighted consistent vector mass: sum_e E_e (M_Q1 x I_d), the
    matrix of the right-hand side lambda E psi.
  * Dirichlet: the DOFs of the closed box that are Dirichlet globally are
    removed (Dirichlet on the boundary of omega_l meeting Gamma_D, per
    component); the remaining boundary is natural (Neumann).
  * number of modes: the paper finds no automatic threshold and takes, per
    neighbourhood, the rigid-body count (3 in 2D, 6 in 3D) for every
    disconnected high-stiffness region (the remark after Eq. 3001 and its
    figure: two regions, six contrast-dependent modes, the seventh contrast
    independent).  Here a region is a set of stiff elements connected through
    element faces (edges in 2D), stiff meaning E_e >= sqrt(E0 Emin) (every
    element at contrast 1); a neighbourhood with no stiff element counts as
    one region.  `modes_scale` = 2 gives the "twice as many eigenvectors"
    rows of the tables.
  * a coarse node that is Dirichlet in every component gets no basis (the
    coarse dimension 243 = 81 x 3 of the contrast-1 table).
  * randomized variant (M_EE;Rand, Sec. "A randomized algorithm for
    eigenvalues computation"): the loads are uniform in [-1/2, 1/2) per free
    DOF from the SplitMix64 counters of the heat variant (coarse node << 40 |
    load << 32 | box DOF), made zero-total per component on the free DOFs
    (the integral of f vanishes); the local solves use K + sigma M with the
    heat eigensolve's shift sigma = tau max(Emin/E0, 1e-10), tau = 2/H^2,
    which keeps the Neumann problem solvable; the snapshot span (SVD) is
    enriched with the rigid-body modes; M = max(snapshots, wanted + 5).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.ndimage as ndi
import scipy.sparse as sp

from . import fem
from .schwarz import box_elements, box_nodes, chi, coarse_nodes, fem_node_id, neighbourhood_box, random_loads


def elastic_matrices(prob, box, E):
    """K_E^l and M^l of Eq. 3001 on an element box: sum_e E_e KE and
    sum_e E_e (M_Q1 x I_d) over the box's elements (natural boundary on the
    box), dense over the closed box's DOFs (node-major, component fastest);
    returns (K, M, global node ids of the box)."""
    d = prob.dim
    KE = fem.element_stiffness(prob)
    _, Mh = fem.heat_element(d)
    ME = np.kron(Mh, np.eye(d))  # same DOF order as KE: d * local node + component
    nodes = box_nodes(prob, box, strict=False)
    loc = {int(g): a for a, g in enumerate(nodes)}
    els = box_elements(prob, box)
    en = fem.element_nodes(prob)[els]
    nd = d * nodes.size
    Kl = np.zeros((nd, nd))
    Ml = np.zeros((nd, nd))
    for e, enodes in zip(els, en):
        ln = np.array([loc[int(g)] for g in enodes])
        li = (d * ln[:, None] + np.arange(d)[None, :]).ravel()
        Kl[np.ix_(li, li)] += E[e] * KE
        Ml[np.ix_(li, li)] += E[e] * ME
    return Kl, Ml, nodes


def stiff_regions(prob, box, E):
    """Number of disconnected high-stiffness regions in an element box:
    connected components (through element faces) of the elements with
    E_e >= sqrt(E0 Emin)."""
    thr = np.sqrt(prob.E0 * prob.Emin)
    els = box_elements(prob, box)
    shape = tuple(hi - lo for lo, hi in reversed(box))  # (ny, nx) or (nz, ny, nx)
    mask = (E[els] >= thr).reshape(shape)
    _, count = ndi.label(mask)  # default structure: face neighbours only
    return int(count)


def elastic_eigenpairs(Kl, Ml, m):
    """The m smallest eigenpairs of K_E^l phi = lambda M^l phi (dense LAPACK
    eigh as a library step)."""
    m = min(m, Kl.shape[0])
    lam, vec = sla.eigh(Kl, Ml, subset_by_index=[0, m - 1])
    return lam, vec


def rigid_modes(coords, d):
    """Rigid-body modes of the nodes at coords (DOFs node-major): the d
    translations and the rotations (-y, x) in 2D; the three axis rotations in
    3D."""
    n = coords.shape[0]
    R = []
    for c in range(d):
        t = np.zeros((n, d))
        t[:, c] = 1.0
        R.append(t.ravel())
    x = coords - coords.mean(axis=0, keepdims=True)
    if d == 2:
        R.append(np.stack([-x[:, 1], x[:, 0]], axis=1).ravel())
    else:
        z0 = np.zeros(n)
        R.append(np.stack([z0, -x[:, 2], x[:, 1]], axis=1).ravel())
        R.append(np.stack([x[:, 2], z0, -x[:, 0]], axis=1).ravel())
        R.append(np.stack([-x[:, 1], x[:, 0], z0], axis=1).ravel())
    return np.column_stack(R)


def elastic_eigenpairs_rand(Kl, Ml, m, F, sigma, Rb):
    """Randomized M_EE basis, the paper's steps in order: zero-total random
    loads (columns of F, free DOFs), local solves (K + sigma M) u_l = f_l, the span of the snapshots (SVD)
    and the rigid-body modes Rb, the reduced generalized eigenproblem in it.
    Returns (reduced eigenvalues, the m selected vectors)."""
    U = np.linalg.solve(Kl + sigma * Ml, F)
    Q, sv, _ = np.linalg.svd(U, full_matrices=False)
    Q = Q[:, sv > 1e-12 * sv[0]]
    Q, sv, _ = np.linalg.svd(np.column_stack([Q, Rb]), full_matrices=False)
    Q = Q[:, sv > 1e-12 * sv[0]]
    lam, phi = sla.eigh(Q.T @ Kl @ Q, Q.T @ Ml @ Q)
    m = min(m, lam.size)
    return lam, Q @ phi[:, :m]


class ElasticCoarseSpace:
    """V_{0,E} (Eq. juaneq:VOE): the rows of R_0 and per-neighbourhood records
    (coarse idx, eigenvalues, stiff regions, modes taken)."""

    def __init__(self, prob, E, modes_scale=1, method="eig", snapshots=15):
        d = prob.dim
        n_rbm = 3 if d == 2 else 6
        tau = 2.0 / float(max(prob.blk)) ** 2
        sigma = tau * max(prob.Emin / prob.E0, 1e-10)
        free = fem.free_mask(prob)
        coords = fem.node_coords(prob)
        rows, cols, vals = [], [], []
        self.records = []
        nb = 0
        for idx, y in coarse_nodes(prob):
            ynode = fem_node_id(prob, y)
            if not any(free[d * ynode + c] for c in range(d)):
                continue  # y_l Dirichlet in every component: no basis
            box = neighbourhood_box(prob, idx)
            Kl, Ml, nodes = elastic_matrices(prob, box, E)
            gd = (d * nodes[:, None] + np.arange(d)[None, :]).ravel()
            ki = np.flatnonzero(free[gd])
            regions = stiff_regions(prob, box, E)
            m = modes_scale * n_rbm * max(regions, 1)
            Kf, Mf = Kl[np.ix_(ki, ki)], Ml[np.ix_(ki, ki)]
            if method == "eig":
                lam, vec = elastic_eigenpairs(Kf, Mf, m)
            else:
                M = max(0, min(max(snapshots, m + 5), ki.size - 1))
                lin = idx[0] + (prob.nx // prob.blk[0] + 1) * (
                    idx[1] + ((prob.ny // prob.blk[1] + 1) * idx[2] if d == 3 else 0))
                F = random_loads(lin, gd.size, M)[ki]
                comp = (ki % d)
                for c in range(d):  # zero total force per component
                    rc = comp == c
                    F[rc] -= F[rc].mean(axis=0, keepdims=True)
                Rb = rigid_modes(coords[nodes], d)[ki]
                lam, vec = elastic_eigenpairs_rand(Kf, Mf, m, F, sigma, Rb)
            ch = np.repeat(chi(prob, y, coords[nodes]), d)  # chi_l per DOF
            for j in range(vec.shape[1]):
                v = np.zeros(gd.size)
                v[ki] = vec[:, j]
                w = ch * v
                nz = np.flatnonzero(w)
                rows += [nb] * nz.size
                cols += list(gd[nz])
                vals += list(w[nz])
                nb += 1
            self.records.append((idx, lam, regions, vec.shape[1]))
        self.dim = nb
        self.R0 = sp.csr_matrix((np.array(vals), (np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64))),
                                shape=(nb, prob.ndof))
