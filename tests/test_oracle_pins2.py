"""Further pins of the oracle against facts fixed outside it: hand-counted
overlapping-subdomain sizes (Sec. 2, D'_i grown by delta element layers), the
Strakos-Tichy identity behind the delayed energy estimate (Sec. 5 stopping
rule), and the flexible CG variant reducing to PCG for a fixed SPD
preconditioner (Notay's FCG(1))."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, pcg, schwarz


def _box_dofs(prob, box, free=None):
    if free is None:
        free = np.ones(prob.ndof, bool)
    return schwarz.local_dofs(prob, box, free).size


@pytest.mark.parametrize("delta", [1, 2])
def test_overlapping_subdomain_counts_by_hand(delta):
    """64 x 64 elements, H = 16.  D'_i is the block grown by delta element
    layers and clipped; its unknowns are the nodes strictly inside D'_i plus
    the nodes of D'_i on the domain boundary.
      interior:  H + 2 delta elements per axis -> H + 2 delta - 1 nodes
      corner:    H + delta elements, the domain-boundary side kept -> H + delta nodes
      edge:      one axis like the corner, the other like the interior
    H = 16, delta = 2: interior 2 * 19^2 = 722, corner 2 * 18^2 = 648,
    edge 2 * 18 * 19 = 684; delta = 1: 2 * 17^2 = 578 for all three."""
    n, H = 64, 16
    prob = W.custom_2d(n, n, np.ones(n * n), H, delta, contrast=1.0)
    boxes = schwarz.subdomain_boxes(prob)
    assert len(boxes) == (n // H) ** 2
    ni = H + 2 * delta - 1   # interior nodes per axis
    nc = H + delta           # nodes per axis at a domain side
    # block (1, 1) interior, (0, 0) corner, (1, 0) edge (x interior, y at the bottom side)
    interior, corner, edge = boxes[1 * 4 + 1], boxes[0], boxes[1]
    assert interior == ((H - delta, 2 * H + delta),) * 2
    assert corner == ((0, H + delta),) * 2
    assert edge == ((H - delta, 2 * H + delta), (0, H + delta))
    assert _box_dofs(prob, interior) == 2 * ni * ni
    assert _box_dofs(prob, corner) == 2 * nc * nc
    assert _box_dofs(prob, edge) == 2 * ni * nc
    if delta == 2:
        assert _box_dofs(prob, interior) == 722
        assert _box_dofs(prob, corner) == 648
        assert _box_dofs(prob, edge) == 684
    # far corner (3, 3): clipped at the top and right sides
    assert boxes[-1] == ((3 * H - delta, n),) * 2
    assert _box_dofs(prob, boxes[-1]) == 2 * nc * nc
    # cantilever: the clamped left edge (x = 0) removes both DOFs of its nodes
    pc = W.custom_2d(n, n, np.ones(n * n), H, delta, contrast=1.0, bc="cantilever")
    free = fem.free_mask(pc)
    assert _box_dofs(pc, corner, free) == 2 * (nc - 1) * nc
    assert _box_dofs(pc, interior, free) == 2 * ni * ni
    # every node of the mesh lies in at least one D'_i, at most two per axis
    cover = np.zeros(prob.n_nodes if hasattr(prob, "n_nodes") else (n + 1) ** 2, int)
    for b in boxes:
        cover[schwarz.box_nodes(prob, b)] += 1
    assert cover.min() >= 1 and cover.max() <= 4


def _system(contrast=1e3, seed=4):
    prob = W.cantilever_channels(32, 16, seed=seed, blk=8, overlap=1, contrast=contrast)
    M = schwarz.Schwarz(prob)
    # Dirichlet rows and columns replaced by the identity (the eliminated operator)
    K = fem.constrained_K(prob, fem.assemble_K(prob, M.E))
    u = fem.direct_solve(prob, K)[0]
    f = prob.f[0].copy()
    Kop = lambda x: K @ x
    return prob, M, K, f, u


def _iterate(Kop, f, Minv, k, flexible=False):
    """x_k of PCG after exactly k iterations (no stopping test)."""
    x, info = pcg.pcg(Kop, f, Minv, rtol=0.0, etol=1e-300, maxit=k, flexible=flexible)
    assert info["iters"] == k
    return x, info


def test_strakos_tichy_identity():
    """For CG, alpha_j r_j^T z_j = ||e_j||_K^2 - ||e_{j+1}||_K^2 exactly (the
    iterates are K-orthogonal corrections), so the delayed estimate over
    d = 4 steps equals ||e_{k-4}||_K^2 - ||e_k||_K^2 (Sec. 5 stopping rule)."""
    prob, M, K, f, u = _system()
    Kop = lambda x: K @ x
    norm2 = lambda e: float(e @ (K @ e))
    e0 = norm2(u)
    for k in (6, 12, 20):
        xk, info = _iterate(Kop, f, M.apply, k)
        xd, _ = _iterate(Kop, f, M.apply, k - 4)
        drop = norm2(u - xd) - norm2(u - xk)
        est = info["energy_est"]
        assert est > 0.0
        assert abs(est - drop) <= 1e-8 * e0 + 1e-6 * drop, (k, est, drop)
        # each single term too: alpha_j r_j^T z_j = ||e_j||^2 - ||e_{j+1}||^2
        x1, _ = _iterate(Kop, f, M.apply, k - 1)
        a_last = info["alphas"][-1]
        # r_{k-1}^T z_{k-1} from the (k-1)-iterate
        r = f - K @ x1
        rz = float(r @ M.apply(r))
        term = a_last * rz
        assert abs(term - (norm2(u - x1) - norm2(u - xk))) <= 1e-8 * e0 + 1e-6 * term


def test_flexible_cg_equals_pcg_for_fixed_preconditioner():
    """Notay's FCG(1) beta = r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k equals the
    PCG beta when M is fixed and SPD, since then r_{k+1}^T z_k = 0: the two
    produce the same iterates up to rounding and stop at the same step."""
    prob, M, K, f, u = _system(contrast=1e4, seed=2)
    Kop = lambda x: K @ x
    x_p, i_p = pcg.pcg(Kop, f, M.apply, rtol=1e-10)
    x_f, i_f = pcg.pcg(Kop, f, M.apply, rtol=1e-10, flexible=True)
    assert i_p["converged"] and i_f["converged"]
    assert abs(i_p["iters"] - i_f["iters"]) <= 1
    # before rounding builds up (PCG loses orthogonality over many steps)
    for k in (5, 20):
        xa, ia = _iterate(Kop, f, M.apply, k)
        xb, ib = _iterate(Kop, f, M.apply, k, flexible=True)
        assert np.allclose(ia["betas_used"], ib["betas_used"], rtol=1e-9, atol=0.0), k
        assert np.linalg.norm(xa - xb) <= 1e-10 * np.linalg.norm(xa), k
    # a sign slip in the flexible beta would not match: r_{k+1}^T z_k is tiny
    # next to r_{k+1}^T z_{k+1}, so the two betas agree term by term
    assert pcg.energy_error(K, x_f, u) <= 1e-8


@pytest.mark.parametrize("dim", [2, 3])
def test_matrix_free_product_equals_assembled(dim):
    """The element-by-element product equals the assembled constrained K
    (Eq. 2) on a small mesh, Dirichlet rows as the identity."""
    prob = (W.cantilever_channels(16, 8, seed=3, blk=8, overlap=1, contrast=1e3) if dim == 2
            else W.cantilever_3d(a=1, seed=2, blk=4, overlap=1, contrast=1e3))
    rng = np.random.default_rng(9)
    x = rng.standard_normal(prob.ndof)
    y = fem.apply_K_free(prob, x)
    yref = fem.constrained_K(prob) @ x
    assert np.allclose(y, yref, rtol=0.0, atol=1e-13 * np.abs(yref).max())


def test_true_residual_sees_below_the_fp64_floor():
    """The extended-precision residual of the refined direct solution lies
    below the FP64 rounding floor eps ||(|K||u|)|| (rounding u itself to FP64
    leaves a residual of that order, here about a tenth of it), while the
    residual of a perturbed solution u + d is K d (to that precision)."""
    prob = W.mbb_field(64, 32, seed=1, contrast=1e6, vol=0.3, nrhs=1)
    K = fem.assemble_K(prob)
    u = fem.direct_solve(prob, K)[0]
    rel, floor = fem.true_residual(prob, u, prob.f[0], K)
    assert floor > 0 and rel < 0.5 * floor, (rel, floor)
    free = fem.free_mask(prob)
    rng = np.random.default_rng(3)
    d = np.where(free, rng.standard_normal(prob.ndof), 0.0) * 1e-6
    rel2, _ = fem.true_residual(prob, u + d, prob.f[0], K)
    Kd = fem.constrained_K(prob, K) @ d
    expect = np.linalg.norm(Kd[free]) / np.linalg.norm(prob.f[0][free])
    assert abs(rel2 - expect) <= 1e-6 * expect + 10 * floor, (rel2, expect)
