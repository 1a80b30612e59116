"""Request loop (ts_submit / ts_poll) and density updates on the GPU.

* A request computes exactly what ts_solve computes: every solve of the path
  uses fixed-order reductions, so the results of the designs solved one at a
  time and the same solves queued together (running concurrently on the
  loop's workers, kernels of different designs overlapping on the device)
  must agree bit for bit, and with the oracle's direct solve to the parity
  tolerance.
* ts_update_density / ts_submit_update with rebuild_policy 0 give the same
  preconditioner and solution as a design set up from scratch for the new
  densities (bit for bit), and a warm start from the previous step's
  solution saves iterations.
* rebuild_policy 1 keeps the preconditioner while the threshold counts of
  the heat eigenproblems keep their total (a stale-preconditioner solve still meets the
  parity tolerance against the oracle's direct solve for the new densities),
  rebuilds when they change (then bit for bit a fresh setup), and rebuilds
  after a solve that exceeded rebuild_factor x the first solve's iterations.
* Misuse is reported: a handle with queued requests is busy for ts_solve,
  an unknown ticket is invalid.
"""
import dataclasses

import numpy as np
import pytest

import parity_tol as PT
import workloads as W
from oracle import fem, pcg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13387_gb300 import Context
    c = Context()
    c.set_slots(3)
    yield c
    c.close()


def _design(ctx, prob, **kw):
    from paper_2006_13387_gb300 import design_from_problem
    return design_from_problem(ctx, prob, **kw)


def _mix():
    return [
        (W.cantilever_channels(32, 16, seed=1, blk=8, overlap=1, contrast=1e4), "fp64"),
        (W.custom_2d(48, 32, W.filtered_projected((32, 48), 3, 0.4), 16, 2, contrast=1e6, bc="mbb",
                     name="mbb48"), "mixed"),
        (W.custom_2d(40, 24, W.filtered_projected((24, 40), 5, 0.4), 8, 2, contrast=1e3), "fp64"),
        (W.cantilever_3d(a=2, seed=0, blk=4, overlap=1, contrast=1e4), "mixed"),
    ]


def test_request_loop_matches_alone(ctx):
    mix = _mix()
    designs = [_design(ctx, p, precision=prec) for p, prec in mix]
    fs = [torch.as_tensor(p.f, device="cuda") for p, _ in mix]
    alone = []
    for d, f in zip(designs, fs):
        u, st = d.solve(f, rtol=1e-8)
        torch.cuda.synchronize()
        alone.append((u.clone(), st[0]["iters"]))
    # two requests per design, interleaved: requests of one design run in
    # order, those of different designs concurrently
    tickets = []
    for rep in range(2):
        for i, (d, f) in enumerate(zip(designs, fs)):
            tickets.append((i, ctx.submit(d, f, rtol=1e-8)))
    for i, t in tickets:
        u, st = ctx.wait(t)
        assert st[0]["converged"]
        assert st[0]["iters"] == alone[i][1]
        assert torch.equal(u, alone[i][0]), i
    for (p, _), (u, _) in zip(mix, alone):
        K = fem.assemble_K(p)
        uref = fem.direct_solve(p, K)[0]
        tol, _ = PT.tolerances(p, K, uref)
        assert pcg.energy_error(K, u[0].cpu().numpy(), uref) <= tol
    for d in designs:
        d.close()


def test_update_density_equals_fresh_setup(ctx):
    p0 = W.cantilever_field(64, 32, seed=3, blk=16, overlap=2, contrast=1e4)
    drift = W.smooth_drift((32, 64), seed=9)
    rho1 = np.clip(p0.rho + 0.02 * drift, 0.0, 1.0)
    p1 = dataclasses.replace(p0, rho=rho1)
    f = torch.as_tensor(p0.f, device="cuda")
    fresh = _design(ctx, p1, precision="mixed")
    u_fresh, st_fresh = fresh.solve(f, rtol=1e-8)
    # synchronous update
    d = _design(ctx, p0, precision="mixed", rebuild="always")
    d.update_density(rho1)
    assert d.coarse_dim == fresh.coarse_dim
    u_upd, st_upd = d.solve(f, rtol=1e-8)
    assert st_upd[0]["iters"] == st_fresh[0]["iters"]
    assert torch.equal(u_upd, u_fresh)
    # the same through the request loop
    d2 = _design(ctx, p0, precision="mixed", rebuild="always")
    u_req, st_req = ctx.wait(ctx.submit(d2, f, rtol=1e-8, rho=rho1))
    assert d2.coarse_dim == fresh.coarse_dim
    assert torch.equal(u_req, u_fresh)
    for x in (fresh, d, d2):
        x.close()


def test_warm_start_after_drift(ctx):
    p0 = W.cantilever_field(64, 32, seed=4, blk=16, overlap=2, contrast=1e4)
    f = torch.as_tensor(p0.f, device="cuda")
    d = _design(ctx, p0, precision="fp64", warm_start=True, rebuild="always")
    u, st0 = d.solve(f, rtol=1e-8)  # u = 0 on entry: a cold start
    drift = W.smooth_drift((32, 64), seed=5)
    rho1 = np.clip(p0.rho + 0.02 * drift, 0.0, 1.0)
    u1, st1 = ctx.wait(ctx.submit(d, f, u=u.clone(), rtol=1e-8, rho=rho1))
    cold = _design(ctx, p0, precision="fp64", rebuild="always")
    cold.update_density(rho1)
    uc, stc = cold.solve(f, rtol=1e-8)
    assert st1[0]["converged"]
    assert st1[0]["iters"] < stc[0]["iters"], (st1[0]["iters"], stc[0]["iters"])
    K = fem.assemble_K(dataclasses.replace(p0, rho=rho1))
    e = u1[0].cpu().numpy() - uc[0].cpu().numpy()
    assert np.sqrt(max(e @ (K @ e), 0.0)) <= 1e-7 * np.sqrt(uc[0].cpu().numpy() @ (K @ uc[0].cpu().numpy()))
    d.close()
    cold.close()


def _wanted(d):
    """Heat modes the threshold asks for in a design's last build, summed
    over its eigenproblems: the count below tau, at least one, at most
    max_modes each (the heat part of the coarse dimension)."""
    info = d.coarse_info()
    return int(np.clip(info["below"], 1, d.max_modes).sum())


def test_rebuild_policy(ctx):
    p0 = W.cantilever_field(64, 32, seed=6, blk=16, overlap=2, contrast=1e4)
    f = torch.as_tensor(p0.f, device="cuda")
    d = _design(ctx, p0, precision="mixed", warm_start=True)  # policy 1 (default)
    u, st = d.solve(f, rtol=1e-8)
    assert st[0]["precond_age"] == 0
    want0 = _wanted(d)
    # a small drift: the operator moves, the preconditioner stays unless a
    # threshold count changes (decided by a fresh design for the same rho)
    rho1 = np.clip(p0.rho + 1e-3 * W.smooth_drift((32, 64), seed=7), 0.0, 1.0)
    p1 = dataclasses.replace(p0, rho=rho1)
    fresh1 = _design(ctx, p1, precision="mixed")
    same = _wanted(fresh1) == want0
    u1, st1 = ctx.wait(ctx.submit(d, f, u=u.clone(), rtol=1e-8, rho=rho1))
    assert st1[0]["converged"]
    assert st1[0]["precond_age"] == (1 if same else 0)
    # the stale-preconditioner solve meets the parity tolerance for rho1
    K1 = fem.assemble_K(p1)
    uref1 = fem.direct_solve(p1, K1)[0]
    tol, _ = PT.tolerances(p1, K1, uref1)
    assert pcg.energy_error(K1, u1[0].cpu().numpy(), uref1) <= tol
    # the operator did move: K u matches the new design's K
    x = torch.as_tensor(np.random.default_rng(0).standard_normal(p0.ndof), device="cuda") * torch.as_tensor(
        fem.free_mask(p0).astype(np.float64), device="cuda")
    assert torch.allclose(d.apply_K(x), fresh1.apply_K(x), rtol=0, atol=1e-12 * float(x.abs().max()))
    # a different design field: the threshold counts change, so the update
    # rebuilds, bit for bit as a fresh setup
    p2 = W.cantilever_field(64, 32, seed=11, blk=16, overlap=2, contrast=1e4)
    fresh2 = _design(ctx, p2, precision="mixed")
    assert _wanted(fresh2) != _wanted(d)
    u_f2, st_f2 = fresh2.solve(f, rtol=1e-8)
    d.update_density(p2.rho)
    assert d.coarse_dim == fresh2.coarse_dim
    u2, st2 = d.solve(f, u=torch.zeros_like(f), rtol=1e-8)  # a cold start
    assert st2[0]["precond_age"] == 0
    assert st2[0]["iters"] == st_f2[0]["iters"]
    assert torch.allclose(u2, u_f2, rtol=0, atol=1e-10 * float(u_f2.abs().max()))
    d.close()
    for x_ in (fresh1, fresh2):
        x_.close()


def test_rebuild_policy_iteration_trigger(ctx):
    """rebuild_factor 1: a stale solve that takes more iterations than the
    first solve after the build marks the preconditioner for a rebuild at the
    next update."""
    p0 = W.cantilever_field(64, 32, seed=8, blk=16, overlap=2, contrast=1e4)
    f = torch.as_tensor(p0.f, device="cuda")
    d = _design(ctx, p0, precision="fp64", rebuild_factor=1.0)
    _, st = d.solve(f, rtol=1e-8)
    ref = st[0]["iters"]
    ages = []
    rho = p0.rho
    grew = False
    for k in range(4):
        rho = np.clip(rho + 0.01 * W.smooth_drift((32, 64), seed=20 + k), 0.0, 1.0)
        fresh = _design(ctx, dataclasses.replace(p0, rho=rho), precision="fp64")
        same = _wanted(fresh) == _wanted(d)
        fresh.close()
        d.update_density(rho)
        _, st = d.solve(f, rtol=1e-8)
        age = st[0]["precond_age"]
        if grew or not same:
            assert age == 0, (k, grew, same)  # rebuilt
            ref = st[0]["iters"]
            grew = False
        else:
            assert age == (ages[-1] if ages else 0) + 1
            grew = st[0]["iters"] > ref
        ages.append(age)
    d.close()


def test_request_loop_errors(ctx):
    from paper_2006_13387_gb300 import TopSolveError
    from paper_2006_13387_gb300 import _native as N
    p = W.cantilever_channels(32, 16, seed=2, blk=8, overlap=1, contrast=1e2)
    d = _design(ctx, p)
    f = torch.as_tensor(p.f, device="cuda")
    tickets = [ctx.submit(d, f) for _ in range(3)]
    u_direct = torch.zeros_like(f)
    busy = N.lib().ts_solve(d._h, f.data_ptr(), u_direct.data_ptr(), 1, 1e-8, None)
    # the loop may already have finished all three; then the solve ran
    assert busy in (N.TS_ERR_BUSY, N.TS_OK)
    for t in tickets:
        ctx.wait(t)
    assert N.lib().ts_poll(ctx._p, 10 ** 9, None) == N.TS_ERR_INVALID
    with pytest.raises(TopSolveError):
        ctx.set_slots(2)  # the loop is running already
    d.close()
