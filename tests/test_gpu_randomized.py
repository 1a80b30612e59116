"""Randomized heat coarse basis (coarse_method = rand, the paper's M_EH+Rot;Rand)
on the GPU against the oracle's restatement: the same SplitMix64 random loads
on both sides, so the snapshot spans agree up to the local solves' rounding
and so do the reduced (Ritz) eigenvalues, their counts below tau, the
preconditioner and the solution."""
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


CASES = {
    "channels_1e4": lambda: W.cantilever_channels(32, 16, seed=2, blk=8, overlap=1, contrast=1e4),
    "field_mbb_1e6": lambda: W.custom_2d(48, 32, W.filtered_projected((32, 48), 3, 0.4), 16, 2, contrast=1e6,
                                         bc="mbb", name="mbb48"),
}


def _design(ctx, prob, **kw):
    from paper_2006_13387_gb300 import design_from_problem
    return design_from_problem(ctx, prob, coarse_method="rand", snapshots=10, **kw)


@pytest.mark.parametrize("name", list(CASES))
def test_randomized_counts_and_ritz_values(ctx, name):
    prob = CASES[name]()
    S = schwarz.Schwarz(prob, method="rand", snapshots=10)
    d = _design(ctx, prob, precision="fp64")
    info = d.coarse_info()
    tau = S.coarse.tau
    ora = {(idx, c): (lam, below, m) for idx, c, lam, below, m in S.coarse.records if c != "rot"}
    ncx = prob.nx // prob.blk[0] + 1
    assert len(info["node"]) == len(ora)
    for i in range(len(info["node"])):
        l = int(info["node"][i])
        lam, below, m = ora[((l % ncx, l // ncx), int(info["comp"][i]))]
        assert info["below"][i] == below
        assert info["selected"][i] == m
        assert np.all(np.abs(info["eig"][i, :m] - lam[:m]) <= 1e-9 * tau), (info["eig"][i, :m], lam[:m])
    assert d.coarse_dim == S.coarse.dim
    d.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_randomized_solve_parity(ctx, name, precision):
    prob = CASES[name]()
    K = fem.assemble_K(prob)
    uref = fem.direct_solve(prob, K)[0]
    d = _design(ctx, prob, precision=precision)
    u, st = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-10)
    un = u[0].cpu().numpy()
    tol_e, _ = PT.tolerances(prob, K, uref)
    assert st[0]["converged"]
    assert pcg.energy_error(K, un, uref) <= max(1e-8, tol_e)
    if precision == "fp64":
        # iteration counts at the bench's 1e-8 (deeper, rounding differences
        # of the two implementations steer the Krylov sequences apart).  The
        # reduced eigenvectors inside a cluster of near-equal Ritz values are
        # fixed only up to a rotation, so the coarse space itself depends on
        # the rounding order of the Jacobi sweeps and the snapshot
        # orthogonalisation: counts agree within 3 %.
        _, st8 = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-8)
        S = schwarz.Schwarz(prob, method="rand", snapshots=10, K=K)
        Kc = fem.constrained_K(prob, K)
        _, info = pcg.pcg(lambda v: Kc @ v, prob.f[0], S.apply, rtol=1e-8)
        assert abs(st8[0]["iters"] - info["iters"]) <= max(1, int(0.03 * info["iters"])), (st8[0]["iters"], info["iters"])
    d.close()


def test_randomized_paper_box(ctx):
    """Sec. 5 geometry, contrast 1, 10 snapshots on the GPU: coarse dimension
    243 (the printed value) and the oracle's iteration count within one."""
    prob = W.paper_box(100, 10)
    d = _design(ctx, prob, precision="fp64", energy_tol=0.0)
    assert d.coarse_dim == 243
    _, st = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-6)
    S = schwarz.Schwarz(prob, method="rand", snapshots=10)
    Kc = fem.constrained_K(prob, S.K)
    _, info = pcg.pcg(lambda v: Kc @ v, prob.f[0], S.apply, rtol=1e-6, etol=0)
    assert abs(st[0]["iters"] - info["iters"]) <= 1
    d.close()
