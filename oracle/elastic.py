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
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.ndimage as ndi
import scipy.sparse as sp

from . import fem
from .schwarz import box_elements, box_nodes, chi, coarse_nodes, fem_node_id, neighbourhood_box


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


class ElasticCoarseSpace:
    """V_{0,E} (Eq. juaneq:VOE): the rows of R_0 and per-neighbourhood records
    (coarse idx, eigenvalues, stiff regions, modes taken)."""

    def __init__(self, prob, E, modes_scale=1):
        d = prob.dim
        n_rbm = 3 if d == 2 else 6
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
            lam, vec = elastic_eigenpairs(Kl[np.ix_(ki, ki)], Ml[np.ix_(ki, ki)], m)
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
