"""3D (Hex8) path of the CUDA library against the CPU oracle, on the same
seeded inputs: 16 x 8 x 8 elements, 4 x 4 x 4-element subdomains with one
layer of overlap (the 3D geometry of the serving workload), filtered and
projected densities, cantilever conditions (x = 0 face clamped).

Tolerances as in the 2D parity tests: K x to 1e-13 of (|K| |x|)_i; level-1
part to 1e-9 in the K-norm (twisted block LU against the oracle's dense
Cholesky, both backward stable; here the FP64 line blocks are too large for
the shared-memory rings and are read in place); coarse part to the
forward-error bound max(1e-8, 10 cond(K_0) eps); exact counts of heat
eigenvalues below tau with the selected eigenvalues to 1e-9 tau; solution
within the instance's FP64 sensitivity (parity_tol.py) and plain-FP64
iteration counts within +-1 of the oracle's PCG.
"""
import numpy as np
import pytest

import parity_tol as PT
import workloads as W
from oracle import fem, pcg, schwarz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13387_gb300 import Context
    c = Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def prob():
    return W.cantilever_3d(a=2, seed=0, blk=4, overlap=1, contrast=1e4)


@pytest.fixture(scope="module")
def oracle(prob):
    K = fem.assemble_K(prob)
    S = schwarz.Schwarz(prob)
    uref = fem.direct_solve(prob, K)[0]
    return K, S, uref


def _design(ctx, prob, **kw):
    from paper_2006_13387_gb300 import design_from_problem
    return design_from_problem(ctx, prob, **kw)


def _knorm(K, v):
    return float(np.sqrt(max(v @ (K @ v), 0.0)))


def test_hex8_spmv_parity(ctx, prob, oracle):
    K = oracle[0]
    d = _design(ctx, prob, coarse=False)
    Kc = fem.constrained_K(prob, K)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(prob.ndof)
    x[prob.dirichlet] = 0.0
    y = d.apply_K(torch.as_tensor(x, device="cuda")).cpu().numpy()
    yref = Kc @ x
    yref[prob.dirichlet] = 0.0
    scale = abs(K) @ np.abs(x) + 1e-300
    assert np.all(np.abs(y - yref) <= 1e-13 * scale)
    d.close()


@pytest.mark.parametrize("layout", ["dense", "blockline", "nd"])
def test_hex8_preconditioner_parity(ctx, prob, oracle, layout):
    K, S, _ = oracle
    d = _design(ctx, prob, coarse_layout=layout)
    assert d.coarse_dim == S.coarse.dim
    rng = np.random.default_rng(1)
    r = rng.standard_normal(prob.ndof)
    r[prob.dirichlet] = 0.0
    zl, zc = d.apply_M_parts(torch.as_tensor(r, device="cuda"))
    zl = zl.cpu().numpy()
    zc = zc.cpu().numpy()
    zl_ref = S.local_part(r)
    zc_ref = S.coarse_part(r)
    assert _knorm(K, zl - zl_ref) <= 1e-9 * _knorm(K, zl_ref)
    lam = S.K0_eig[0]
    ctol = max(1e-8, 10.0 * (lam.max() / lam.min()) * np.finfo(float).eps)
    assert _knorm(K, zc - zc_ref) <= ctol * _knorm(K, zc_ref)
    d.close()


def test_hex8_coarse_space_counts(ctx, prob, oracle):
    S = oracle[1]
    d = _design(ctx, prob)
    info = d.coarse_info()
    tau = S.coarse.tau
    ora = {(idx, c): (lam, below, m) for idx, c, lam, below, m in S.coarse.records if c != "rot"}
    ncx = prob.nx // prob.blk[0] + 1
    ncy = prob.ny // prob.blk[1] + 1
    assert len(info["node"]) == len(ora)
    for i in range(len(info["node"])):
        l = int(info["node"][i])
        idx = (l % ncx, (l // ncx) % ncy, l // (ncx * ncy))
        lam, below, m = ora[(idx, int(info["comp"][i]))]
        assert info["below"][i] == below
        assert info["selected"][i] == m
        got = info["eig"][i, :m]
        assert np.all(np.abs(got - lam[:m]) <= 1e-9 * tau), (got, lam[:m])
    d.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hex8_solve_parity(ctx, prob, oracle, precision):
    K, S, uref = oracle
    d = _design(ctx, prob, precision=precision)
    u, st = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-8)
    u = u[0].cpu().numpy()
    assert st[0]["converged"]
    err = pcg.energy_error(K, u, uref)
    tol, ctol = PT.tolerances(prob, K, uref)
    assert err <= tol, (err, tol)
    c, cref = prob.f[0] @ u, prob.f[0] @ uref
    assert abs(c - cref) <= ctol * abs(cref), (c, cref, ctol)
    if precision == "fp64":
        Kc = fem.constrained_K(prob, K)
        _, info = pcg.pcg(lambda v: Kc @ v, prob.f[0], S.apply, rtol=1e-8)
        assert abs(st[0]["first_iters"] - info["iters"]) <= 1, (st[0], info["iters"])
    d.close()


def test_hex8_bcr_with_dependent_coarse_vectors(ctx):
    """32 x 16 x 16 elements: 2367 coarse DOFs on 9 coarse lines (block
    cyclic reduction), eight of them exactly dependent (one per free coarse
    plane).  The dependent vectors are dropped at every reduction level, and
    the coarse correction equals the dense factor's and the oracle's
    pseudo-inverse correction."""
    prob = W.cantilever_3d(a=4, seed=103, blk=4, overlap=1, contrast=1e4)
    S = schwarz.Schwarz(prob)
    db = _design(ctx, prob, coarse_layout="blockline")
    dd = _design(ctx, prob, coarse_layout="dense")
    dn = _design(ctx, prob, coarse_layout="nd")  # nested dissection of the 9 x 5 x 5 coarse grid
    assert db.coarse_dim == dd.coarse_dim == dn.coarse_dim == S.coarse.dim
    rng = np.random.default_rng(4)
    r = rng.standard_normal(prob.ndof)
    r[prob.dirichlet] = 0.0
    rt = torch.as_tensor(r, device="cuda")
    zb = db.apply_M_parts(rt)[1].cpu().numpy()
    zd = dd.apply_M_parts(rt)[1].cpu().numpy()
    zn = dn.apply_M_parts(rt)[1].cpu().numpy()
    zref = S.coarse_part(r)
    K = S.K
    lam = S.K0_eig[0]
    ctol = max(1e-8, 10.0 * (lam.max() / lam.min()) * np.finfo(float).eps)
    assert _knorm(K, zb - zref) <= ctol * _knorm(K, zref)
    assert _knorm(K, zd - zref) <= ctol * _knorm(K, zref)
    assert _knorm(K, zn - zref) <= ctol * _knorm(K, zref)
    db.close()
    dd.close()
    dn.close()
