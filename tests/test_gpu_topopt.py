"""Compliance sensitivities (Eq. 1003) and the optimality-criteria update on
the GPU, against the oracle, and a short topology-optimisation loop driven
through the request loop (density update, warm-started solve, sensitivity,
OC step), the outer iteration this state solve serves (Sec. 1)."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13387_gb300 import Context
    c = Context()
    c.set_slots(2)
    yield c
    c.close()


def _design(ctx, prob, **kw):
    from paper_2006_13387_gb300 import design_from_problem
    return design_from_problem(ctx, prob, **kw)


CASES = {
    "q4_cantilever_1e4": lambda: W.cantilever_field(64, 32, seed=3, blk=16, overlap=2, contrast=1e4, vol=0.4),
    "q4_mbb_1e6": lambda: W.custom_2d(48, 32, W.filtered_projected((32, 48), 3, 0.4), 16, 2, contrast=1e6,
                                      bc="mbb", name="mbb48"),
    "hex8_1e3": lambda: W.cantilever_3d(a=2, seed=1, blk=4, overlap=1, contrast=1e3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sensitivity_parity(ctx, name):
    """dc and the compliance from the GPU's own solution against the oracle's
    Eq. 1003 on the same displacements (every element compared)."""
    prob = CASES[name]()
    d = _design(ctx, prob, precision="mixed")
    u, st = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-10)
    dc, c = d.sensitivity(u[0])
    un = u[0].cpu().numpy()
    dc_ref, c_ref = fem.sensitivity(prob, un)
    dcn = dc.cpu().numpy()
    # a quadratic form u_e^T KE u_e evaluated in FP64 in any order carries an
    # error of at most a few eps |u_e|^T |KE| |u_e| (KE annihilates rigid
    # motions, so nearly rigid elements cancel): the per-element bound of the
    # difference between two such evaluations, scaled like dc
    KE = fem.element_stiffness(prob)
    ue = np.abs(un[fem.element_dofs(prob)])
    qa = np.einsum("ei,ij,ej->e", ue, np.abs(KE), ue)
    eps = np.finfo(float).eps
    scale = prob.p * prob.rho ** (prob.p - 1.0) * (prob.E0 - prob.Emin)
    bound = 64 * eps * scale * qa + 1e-14 * np.abs(dc_ref)
    assert np.all(np.abs(dcn - dc_ref) <= bound), np.max(np.abs(dcn - dc_ref) / bound)
    E = fem.simp(prob.rho, prob.E0, prob.Emin, prob.p)
    assert abs(c - c_ref) <= 64 * eps * np.sum(E * qa) + 1e-14 * abs(c_ref)
    # at the solution the element sum is the compliance f^T u (Eq. 1)
    assert abs(c - fem.compliance(prob.f[0], un)) <= 1e-8 * abs(c)
    assert np.all(dcn <= 0.0)
    d.close()


def test_oc_update_parity(ctx):
    """OC densities against the oracle's update on the same inputs; volume kept."""
    prob = CASES["q4_cantilever_1e4"]()
    d = _design(ctx, prob, precision="mixed")
    u, _ = d.solve(torch.as_tensor(prob.f, device="cuda"), rtol=1e-10)
    dc, _ = d.sensitivity(u[0])
    for vf, mv in ((0.4, 0.2), (0.37, 0.05)):  # targets the move limit can reach
        new = d.oc_update(dc, vf, mv).cpu().numpy()
        ref = fem.oc_update(prob.rho, dc.cpu().numpy(), vf, mv)
        assert np.max(np.abs(new - ref)) <= 1e-9
        assert abs(new.mean() - vf) <= 1e-9
        assert np.all(np.abs(new - prob.rho) <= mv + 1e-15)
    with pytest.raises(Exception):
        d.oc_update(dc, 1.5, 0.2)
    d.close()


def test_topopt_loop_through_request_loop(ctx):
    """Four optimisation steps of a 64x32 cantilever from a uniform design:
    each step rebuilds the preconditioner for the new densities and solves
    warm-started through ts_submit_update / ts_poll, then updates the
    densities by OC.  The compliance decreases at every step and the volume
    fraction is kept; the last step's compliance equals the oracle's direct
    solve for the same densities."""
    vf = 0.5
    prob = W.custom_2d(64, 32, np.full(64 * 32, vf), 16, 2, contrast=1e6)
    d = _design(ctx, prob, precision="mixed", warm_start=True)
    f = torch.as_tensor(prob.f, device="cuda")
    u = torch.zeros_like(f)
    rho = torch.as_tensor(prob.rho, device="cuda")
    comps = []
    for step in range(4):
        t = ctx.submit(d, f, u=u, rtol=1e-10, rho=rho if step > 0 else None)
        res = None
        t0 = time.time()
        while res is None:
            res = ctx.poll(t)
            assert time.time() - t0 < 120
        u = res[0]
        dc, c = d.sensitivity(u[0])
        comps.append(c)
        rho = d.oc_update(dc, vf, 0.2)
        assert abs(float(rho.mean()) - vf) <= 1e-9
    assert all(b < a for a, b in zip(comps, comps[1:])), comps
    # the last solve against the oracle for the densities it used
    last_rho = d._keep.cpu().numpy() if hasattr(d._keep, "cpu") else np.asarray(d._keep)
    pl = W.custom_2d(64, 32, last_rho, 16, 2, contrast=1e6)
    uref = fem.direct_solve(pl)[0]
    cref = fem.compliance(pl.f[0], uref)
    assert abs(comps[-1] - cref) <= 1e-8 * abs(cref)
    d.close()
