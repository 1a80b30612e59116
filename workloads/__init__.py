"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only: mesh sizes, density fields shaped like
topology-optimisation designs, load vectors and Dirichlet DOF lists. It contains
none of the solver's arithmetic (no stiffness, no preconditioner, no PCG), so
the oracle and the CUDA path can both consume it without sharing method code.

Numbering conventions (the contract both sides follow):
  2D: node (i, j), 0<=i<=nx, 0<=j<=ny, id = j*(nx+1) + i; DOF = 2*node + c.
  3D: node (i, j, k), id = (k*(ny+1) + j)*(nx+1) + i; DOF = 3*node + c.
  Elements are row-major: 2D e = ey*nx + ex; 3D e = (ez*ny + ey)*nx + ex.
  Unit element size h = 1.

The paper's own workloads (the TO design of its first figure and the inclusion
material of Sec. 5) exist only as missing figures, so every generator below is a
seeded stand-in with the shapes, sizes and value structure those workloads have
(near-0/1 multiscale channels at a set volume fraction).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One state-solve instance K(rho) u = f (Eq. 2 with the SIMP law Eq. 4)."""

    dim: int
    nx: int
    ny: int
    nz: int
    blk: tuple            # coarse block size in elements (per axis)
    overlap: int          # delta in element layers; -1 means D'_i = omega_i (paper Sec. 5)
    rho: np.ndarray       # element densities in [0, 1], float64, row-major elements
    E0: float
    Emin: float
    p: float
    nu: float
    dirichlet: np.ndarray  # sorted unique int64 DOF ids with u = 0
    f: np.ndarray          # float64 [nrhs, ndof]; zero at Dirichlet DOFs
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        if self.dim == 2:
            return (self.nx + 1) * (self.ny + 1)
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def ndof(self) -> int:
        return self.dim * self.n_nodes

    @property
    def n_el(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def nrhs(self) -> int:
        return self.f.shape[0]


# ----------------------------------------------------------------------------
# node ids for boundary conditions
# ----------------------------------------------------------------------------

def node2(nx, i, j):
    return j * (nx + 1) + i


def node3(nx, ny, i, j, k):
    return (k * (ny + 1) + j) * (nx + 1) + i


def bc_cantilever_2d(nx, ny):
    """Left edge clamped; unit downward load at the bottom-right node."""
    nodes = np.array([node2(nx, 0, j) for j in range(ny + 1)], dtype=np.int64)
    dir_ = np.sort(np.concatenate([2 * nodes, 2 * nodes + 1]))
    f = np.zeros(2 * (nx + 1) * (ny + 1))
    f[2 * node2(nx, nx, 0) + 1] = -1.0
    return dir_, f


def bc_mbb_2d(nx, ny):
    """MBB half-beam: u_x = 0 on the left edge (symmetry roller), u_y = 0 at the
    bottom-right node (support), unit downward load at the top-left node."""
    left = np.array([node2(nx, 0, j) for j in range(ny + 1)], dtype=np.int64)
    dir_ = np.sort(np.concatenate([2 * left, [2 * node2(nx, nx, 0) + 1]])).astype(np.int64)
    f = np.zeros(2 * (nx + 1) * (ny + 1))
    f[2 * node2(nx, 0, ny) + 1] = -1.0
    return dir_, f


def bc_clamped_box_2d(nx, ny):
    """Zero Dirichlet on all four sides, two opposing unit x-loads at
    (0.2, 0.2) and (0.8, 0.8) of the unit square (Sec. 5 forcing figure)."""
    nodes = []
    for i in range(nx + 1):
        nodes += [node2(nx, i, 0), node2(nx, i, ny)]
    for j in range(ny + 1):
        nodes += [node2(nx, 0, j), node2(nx, nx, j)]
    nodes = np.unique(np.array(nodes, dtype=np.int64))
    dir_ = np.sort(np.concatenate([2 * nodes, 2 * nodes + 1]))
    f = np.zeros(2 * (nx + 1) * (ny + 1))
    a = node2(nx, round(0.2 * nx), round(0.2 * ny))
    b = node2(nx, round(0.8 * nx), round(0.8 * ny))
    f[2 * a] = 1.0
    f[2 * b] = -1.0
    return dir_, f


def bc_cantilever_3d(nx, ny, nz):
    """x = 0 face clamped; unit load -z at the mid node of the far bottom edge."""
    nodes = np.array([node3(nx, ny, 0, j, k) for k in range(nz + 1) for j in range(ny + 1)], dtype=np.int64)
    dir_ = np.sort(np.concatenate([3 * nodes, 3 * nodes + 1, 3 * nodes + 2]))
    f = np.zeros(3 * (nx + 1) * (ny + 1) * (nz + 1))
    f[3 * node3(nx, ny, nx, ny // 2, 0) + 2] = -1.0
    return dir_, f


def extra_top_loads_2d(nx, ny, count, rng):
    """Seeded unit point loads (0, -1) at random top-edge nodes, one per column."""
    out = []
    for _ in range(count):
        i = int(rng.integers(0, nx + 1))
        f = np.zeros(2 * (nx + 1) * (ny + 1))
        f[2 * node2(nx, i, ny) + 1] = -1.0
        out.append(f)
    return out


# ----------------------------------------------------------------------------
# density fields
# ----------------------------------------------------------------------------

def binary_channels(nx, ny, seed, vol=0.5):
    """Binary 0/1 field of random straight channels (width 1-4, length 8-64,
    horizontal/vertical/diagonal) and small rectangular inclusions, stopped at
    exactly round(vol * n_el) solid elements.  Returns rho[ny, nx] flattened."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = np.zeros((ny, nx), dtype=np.float64)
    target = int(round(vol * nx * ny))
    last = None
    while g.sum() < target:
        cells = []
        if rng.random() < 0.7:
            w = int(rng.integers(1, 5))
            L = int(rng.integers(8, 65))
            x0 = int(rng.integers(0, nx))
            y0 = int(rng.integers(0, ny))
            d = int(rng.integers(0, 4))
            dx, dy = [(1, 0), (0, 1), (1, 1), (1, -1)][d]
            for t in range(L):
                cx, cy = x0 + dx * t, y0 + dy * t
                for s in range(w):
                    # widen perpendicular to the direction
                    px, py = (cx, cy + s) if dx != 0 and dy == 0 else (cx + s, cy)
                    if 0 <= px < nx and 0 <= py < ny:
                        cells.append((py, px))
        else:
            a = int(rng.integers(1, 5))
            b = int(rng.integers(1, 5))
            x0 = int(rng.integers(0, nx))
            y0 = int(rng.integers(0, ny))
            for yy in range(y0, min(ny, y0 + b)):
                for xx in range(x0, min(nx, x0 + a)):
                    cells.append((yy, xx))
        new = [c for c in dict.fromkeys(cells) if g[c] == 0.0]
        for c in new:
            g[c] = 1.0
        last = new
    excess = int(g.sum()) - target
    if excess > 0:
        idx = rng.permutation(len(last))[:excess]
        for k in idx:
            g[last[k]] = 0.0
    return g.reshape(-1)


def _cone_filter(g, R):
    """Cone-weighted average with weights max(0, R - dist), normalised by the
    weights that fall inside the domain (works for 2D and 3D arrays)."""
    r = int(math.ceil(R))
    out = np.zeros_like(g)
    wsum = np.zeros_like(g)
    nd = g.ndim
    rngs = [range(-r, r + 1)] * nd
    import itertools
    for off in itertools.product(*rngs):
        w = R - math.sqrt(sum(o * o for o in off))
        if w <= 0:
            continue
        src = [slice(max(0, -o), g.shape[a] - max(0, o)) for a, o in enumerate(off)]
        dst = [slice(max(0, o), g.shape[a] - max(0, -o)) for a, o in enumerate(off)]
        out[tuple(dst)] += w * g[tuple(src)]
        wsum[tuple(dst)] += w
    return out / wsum


def _projection(t, beta, theta):
    return (np.tanh(beta * theta) + np.tanh(beta * (t - theta))) / (
        np.tanh(beta * theta) + np.tanh(beta * (1.0 - theta)))


def filtered_projected(shape, seed, vol, R=3.0, beta=8.0):
    """Gaussian white noise -> cone filter (radius R elements) -> standardise ->
    normal CDF -> tanh Heaviside projection (beta) with the threshold found by
    bisection so that mean(rho) = vol.  `shape` is (ny, nx) or (nz, ny, nx);
    returns the row-major flattened field."""
    from scipy.special import ndtr
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(shape)
    gf = _cone_filter(g, R)
    gf = (gf - gf.mean()) / gf.std()
    t = ndtr(gf)
    lo, hi = 0.0, 1.0
    for _ in range(80):
        th = 0.5 * (lo + hi)
        m = _projection(t, beta, th).mean()
        if m > vol:
            lo = th
        else:
            hi = th
    rho = _projection(t, beta, 0.5 * (lo + hi))
    return np.clip(rho, 0.0, 1.0).reshape(-1)


def smooth_drift(shape, seed, R=8.0):
    """Seeded smooth perturbation: filtered Gaussian field scaled to max|s| = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = _cone_filter(rng.standard_normal(shape), R)
    return (s / np.abs(s).max()).reshape(-1)


# ----------------------------------------------------------------------------
# the workloads used by tests and the bench
# ----------------------------------------------------------------------------

def _finish(dim, nx, ny, nz, blk, overlap, rho, E0, Emin, nu, dir_, fs, name, p=3.0, meta=None):
    f = np.atleast_2d(np.asarray(fs, dtype=np.float64)).copy()
    f[:, dir_] = 0.0
    return Problem(dim=dim, nx=nx, ny=ny, nz=nz, blk=tuple(blk), overlap=overlap,
                   rho=np.ascontiguousarray(rho, dtype=np.float64), E0=E0, Emin=Emin, p=p, nu=nu,
                   dirichlet=np.ascontiguousarray(dir_, dtype=np.int64), f=f, name=name,
                   meta=dict(meta or {}))


def cantilever_channels(nx=64, ny=32, seed=0, blk=8, overlap=1, contrast=1e6, vol=0.5):
    """64x32 binary channels at 50 % volume, E in {Emin, 1}, cantilever BCs,
    8x8-element blocks with one element layer of overlap (small case)."""
    rho = binary_channels(nx, ny, seed, vol)
    d, f = bc_cantilever_2d(nx, ny)
    return _finish(2, nx, ny, 0, (blk, blk), overlap, rho, 1.0, 1.0 / contrast, 0.3, d, f,
                   f"cantilever_channels_{nx}x{ny}_s{seed}", meta=dict(seed=seed, contrast=contrast))


def cantilever_field(nx=512, ny=256, seed=0, blk=16, overlap=2, contrast=1e6, vol=0.4):
    """Filtered/projected random field (R = 3, beta = 8) at 40 % volume,
    cantilever BCs, 16x16-element blocks with two layers of overlap."""
    rho = filtered_projected((ny, nx), seed, vol)
    d, f = bc_cantilever_2d(nx, ny)
    return _finish(2, nx, ny, 0, (blk, blk), overlap, rho, 1.0, 1.0 / contrast, 0.3, d, f,
                   f"cantilever_field_{nx}x{ny}_s{seed}_c{contrast:g}", meta=dict(seed=seed, contrast=contrast))


def mbb_field(nx=2048, ny=1024, seed=0, blk=16, overlap=2, contrast=1e6, vol=0.3, nrhs=8):
    """MBB boundary conditions, nrhs load cases: column 0 the MBB load,
    the rest seeded unit point loads on the top edge."""
    rho = filtered_projected((ny, nx), seed, vol)
    d, f = bc_mbb_2d(nx, ny)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    fs = [f] + extra_top_loads_2d(nx, ny, nrhs - 1, rng)
    return _finish(2, nx, ny, 0, (blk, blk), overlap, rho, 1.0, 1.0 / contrast, 0.3, d, fs,
                   f"mbb_field_{nx}x{ny}_s{seed}", meta=dict(seed=seed, contrast=contrast))


def paper_box(n=100, H=10, contrast=1.0, rho=None):
    """Sec. 5 geometry: n x n elements, H x H coarse blocks, D'_i = omega_i,
    Dirichlet on all sides, two opposing point loads.  With contrast 1 the
    material is uniform (the only case whose material the paper fixes)."""
    if rho is None:
        rho = np.ones(n * n)
    d, f = bc_clamped_box_2d(n, n)
    return _finish(2, n, n, 0, (H, H), -1, rho, 1.0, 1.0 / contrast, 0.3, d, f,
                   f"paper_box_{n}_H{H}", meta=dict(contrast=contrast))


def cantilever_3d(a=4, seed=0, blk=4, overlap=1, contrast=1e6, vol=0.4):
    """3D Hex8: (nx, ny, nz) = 4*(2a, a, a) elements, filtered/projected field,
    4x4x4-element blocks with one layer of overlap."""
    nx, ny, nz = 8 * a, 4 * a, 4 * a
    rho = filtered_projected((nz, ny, nx), seed, vol)
    d, f = bc_cantilever_3d(nx, ny, nz)
    return _finish(3, nx, ny, nz, (blk, blk, blk), overlap, rho, 1.0, 1.0 / contrast, 0.3, d, f,
                   f"cantilever3d_{nx}x{ny}x{nz}_s{seed}", meta=dict(seed=seed, contrast=contrast))


def custom_2d(nx, ny, rho, blk, overlap, contrast=1e6, bc="cantilever", nu=0.3, name="custom"):
    bcs = {"cantilever": bc_cantilever_2d, "mbb": bc_mbb_2d, "box": bc_clamped_box_2d}
    d, f = bcs[bc](nx, ny)
    return _finish(2, nx, ny, 0, (blk, blk) if np.isscalar(blk) else blk, overlap, rho, 1.0,
                   1.0 / contrast, nu, d, f, name)


def custom_3d(nx, ny, nz, rho, blk, overlap, contrast=1e6, nu=0.3, name="custom3d"):
    """3D Hex8 with the cantilever conditions of cantilever_3d and given densities."""
    d, f = bc_cantilever_3d(nx, ny, nz)
    return _finish(3, nx, ny, nz, (blk, blk, blk) if np.isscalar(blk) else blk, overlap, rho, 1.0,
                   1.0 / contrast, nu, d, f, name)
