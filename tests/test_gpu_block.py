"""The block path: 8 load cases of one design solved together, every kernel
launch shared by the columns (Sec. 2 PCG per column; level 1 of Eq.
localproblemsE on the tensor cores; coarse correction of Sec. 2.1).

Parity, against the CPU oracle on the same seeded inputs:
  * preconditioner: each column of the block application equals the oracle's
    level-1 part, coarse part and their sum within the rounding bound of the
    arithmetic used: 4x the error of the one-column FP32 sweeps for 3xTF32
    and FP32, that error times 2^13 (the ratio of the unit roundoffs) for TF32;
  * solution: every column's relative K-norm error against the oracle's
    refined direct solve within max(1e-8, 3x that column's FP64 sensitivity),
    compliance within the larger of max(1e-10, 3x its sensitivity) and the
    energy bound (first order for flexible CG, see below);
  * a column's result does not depend on the other columns of its group
    (bit for bit), a zero load gives u = 0 at once, and more than 8 columns
    run as several groups.
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


def _design(ctx, prob, **kw):
    from paper_2006_13387_gb300 import design_from_problem
    return design_from_problem(ctx, prob, **kw)


def _knorm(K, v):
    return float(np.sqrt(max(v @ (K @ v), 0.0)))


CASES = {
    # MBB, 8 load cases, 6 x 4 subdomains of 16 x 16 with overlap 2 (ragged:
    # 96 is not a multiple of the 32-node SpMV tile), one coarse line
    "mbb_96x64_c1e4": lambda: W.mbb_field(96, 64, seed=3, contrast=1e4, vol=0.3, nrhs=8),
    # channels, cantilever, 8 random loads on the free DOFs
    "channels_64x32_c1e6": lambda: _random_loads(W.cantilever_channels(64, 32, seed=0, blk=8, overlap=1,
                                                                       contrast=1e6), 8, 11),
}


def _random_loads(prob, n, seed):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n, prob.ndof))
    f[:, prob.dirichlet] = 0.0
    prob.f = f
    return prob


@pytest.mark.parametrize("precision,layout", [("3xtf32", "auto"), ("tf32", "auto"), ("fp32", "blockline"),
                                              ("3xtf32", "nd")])
@pytest.mark.parametrize("name", list(CASES))
def test_block_preconditioner_parity(ctx, name, precision, layout):
    prob = CASES[name]()
    S = schwarz.Schwarz(prob)
    K = S.K
    d = _design(ctx, prob, precision=precision, coarse_layout=layout)
    assert d.coarse_dim == S.coarse.dim
    rng = np.random.default_rng(5)
    r = rng.standard_normal((6, prob.ndof))
    r[:, prob.dirichlet] = 0.0
    rt = torch.as_tensor(r, device="cuda")
    zl = d.apply_M_block(rt, which=1).cpu().numpy()
    zc = d.apply_M_block(rt, which=2).cpu().numpy()
    z = d.apply_M_block(rt, which=3).cpu().numpy()
    # the one-column FP32 path on the same stored factors, for the bound
    lam = S.K0_eig[0]
    # the rounding error of the level-1 products scales with the unit
    # roundoff of the arithmetic: 2^-24 (FP32, and 3xTF32 which carries
    # FP32's accuracy), 2^-11 (TF32, 10 explicit mantissa bits)
    ratio = 2.0 ** 13 if precision == "tf32" else 1.0
    ctol = max(1e-5, 10.0 * (lam.max() / lam.min()) * 2.0 ** -24)
    for j in range(r.shape[0]):
        zl_ref = S.local_part(r[j])
        zc_ref = S.coarse_part(r[j])
        zl1, zc1 = d.apply_M_parts(rt[j])
        e1 = _knorm(K, zl1.cpu().numpy() - zl_ref) / _knorm(K, zl_ref)  # FP32 sweeps
        eb = _knorm(K, zl[j] - zl_ref) / _knorm(K, zl_ref)
        # the block level 1 is as accurate as the FP32 sweeps (3xTF32), or
        # that error scaled by the ratio of unit roundoffs (TF32)
        bound = 4.0 * e1 * ratio + 64.0 * 2.0 ** -24
        assert eb <= bound, (j, eb, e1)
        # coarse part: FP32 stage matrices in both paths, the sums in another
        # order; within 4x the one-column path's own error (and the
        # conditioning bound, which is the looser one at high contrast)
        ec1 = _knorm(K, zc1.cpu().numpy() - zc_ref) / _knorm(K, zc_ref)
        ecb = _knorm(K, zc[j] - zc_ref) / _knorm(K, zc_ref)
        assert ecb <= min(ctol, 4.0 * ec1 + 1e-6), (j, ecb, ec1, ctol)
        zr = zl_ref + zc_ref
        assert _knorm(K, z[j] - zr) <= (bound + ctol) * _knorm(K, zr), j


@pytest.mark.parametrize("precision", ["3xtf32", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_block_solve_parity(ctx, name, precision):
    prob = CASES[name]()
    K = fem.assemble_K(prob)
    uref = fem.direct_solve(prob, K)
    d = _design(ctx, prob, precision=precision)
    f = torch.as_tensor(prob.f, device="cuda")
    u, st = d.solve(f, rtol=1e-8)
    u = u.cpu().numpy()
    one = []
    for c in range(prob.f.shape[0]):
        assert st[c]["converged"], (c, st[c])
        tol, ctol = PT.tolerances(prob, K, uref[c], rhs=c)
        err = pcg.energy_error(K, u[c], uref[c])
        assert err <= tol, (c, err, tol)
        cc, cref = prob.f[c] @ u[c], prob.f[c] @ uref[c]
        # f^T (u* - u) = u*^T K e is first order in the energy error once the
        # varying FP32 / TF32 preconditioner has cost FCG its Galerkin
        # orthogonality (with it, the compliance error is the square, P5)
        ctol = max(ctol, tol)
        assert abs(cc - cref) <= ctol * abs(cref), (c, cc, cref, ctol)
        one.append(st[c]["iters"])
    # FCG iterations of the block columns against one-column FP32 solves of
    # the same loads: the 3xTF32 products keep FP32 accuracy.  (At contrast
    # 1e6 the FP32 coarse stages leave the count sensitive to the order of
    # the sums, +-25 %, so the comparison runs on the contrast-1e4 case.)
    if precision == "3xtf32" and prob.Emin >= 1e-4:
        d1 = _design(ctx, prob, precision="fp32")
        for c in range(2):
            _, s1 = d1.solve(f[c:c + 1], rtol=1e-8)
            assert abs(one[c] - s1[0]["iters"]) <= max(2, 0.03 * s1[0]["iters"]), (c, one[c], s1[0]["iters"])


def test_block_columns_independent_and_groups(ctx):
    prob = CASES["mbb_96x64_c1e4"]()
    d = _design(ctx, prob, precision="3xtf32")
    f = torch.as_tensor(prob.f, device="cuda")
    u8, s8 = d.solve(f, rtol=1e-8)
    # the same columns in another group composition: a zero load and a
    # different neighbour set
    f3 = torch.stack([f[2], torch.zeros_like(f[0]), f[5]])
    u3, s3 = d.solve(f3, rtol=1e-8)
    assert torch.equal(u3[0], u8[2]) and torch.equal(u3[2], u8[5])
    assert s3[0]["iters"] == s8[2]["iters"] and s3[2]["iters"] == s8[5]["iters"]
    assert float(u3[1].abs().max()) == 0.0 and s3[1]["iters"] == 0 and s3[1]["converged"]
    # 10 columns: two groups (8 + 2)
    f10 = torch.cat([f, f[:2]])
    u10, s10 = d.solve(f10, rtol=1e-8)
    assert torch.equal(u10[:8], u8) and torch.equal(u10[8:], u8[:2])
    assert [s["iters"] for s in s10] == [s["iters"] for s in s8] + [s8[0]["iters"], s8[1]["iters"]]


def test_block_warm_start(ctx):
    prob = CASES["mbb_96x64_c1e4"]()
    d = _design(ctx, prob, precision="3xtf32", warm_start=True)
    f = torch.as_tensor(prob.f, device="cuda")
    u0 = torch.zeros_like(f)
    u, st = d.solve(f, u0.clone(), rtol=1e-8)
    cold = [s["iters"] for s in st]
    u2, st2 = d.solve(f, u.clone(), rtol=1e-8)
    for c in range(f.shape[0]):
        assert st2[c]["converged"] and st2[c]["iters"] <= max(4, cold[c] // 4), (c, st2[c]["iters"], cold[c])


@pytest.mark.slow
def test_block_parity_bench_recipe_512x256(ctx):
    """The benchmark's recipe (MBB, 30 % volume, contrast 1e6, 16 x 16 blocks,
    overlap 2, 8 load cases, 3xTF32 level 1) at the largest size the
    oracle's direct solve handles in a test: every column within the energy
    and compliance bounds against the refined direct solve."""
    prob = W.mbb_field(512, 256, seed=0, contrast=1e6, vol=0.3, nrhs=8)
    K = fem.assemble_K(prob)
    uref = fem.direct_solve(prob, K)
    tols = PT.tolerances_all(prob, K, uref)
    d = _design(ctx, prob, precision="3xtf32")
    u, st = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-8)
    u = u.cpu().numpy()
    for c in range(8):
        assert st[c]["converged"], (c, st[c])
        tol, ctol = tols[c]
        err = pcg.energy_error(K, u[c], uref[c])
        assert err <= tol, (c, err, tol)
        cc, cref = prob.f[c] @ u[c], prob.f[c] @ uref[c]
        assert abs(cc - cref) <= ctol * abs(cref), (c, cc, cref, ctol)
