"""ts_apply_K_dot_static: the entry point that allocates nothing at call time
(for callers that cannot allocate device memory when they call, such as code
recorded into a CUDA graph or a serving loop under a fixed memory budget).

It must give the same y = K x as ts_apply_K and the energy x^T K x, on two
calls in a row (the shared fixed scratch keeps the previous call's contents,
which must not leak into the next result), for the Q4 stencil product and
the Hex8 element product.  A mesh whose product needs more blocks than the
fixed scratch holds is rejected with TS_ERR_INVALID and leaves y untouched.
This file is collected last so that a failure here does not hide the other
tests' results.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call(L, d, xt, y, out):
    return L.ts_apply_K_dot_static(d._h, C.c_void_p(xt.data_ptr()), C.c_void_p(y.data_ptr()),
                                   C.c_void_p(out.data_ptr()))


def test_static_scratch_matches_regular_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13387_gb300 import Context, _native as N, design_from_problem
    ctx = Context()
    try:
        L = N.lib()
        for prob in (W.cantilever_channels(64, 32, seed=0, blk=8, overlap=1, contrast=1e6),
                     W.custom_2d(48, 32, W.filtered_projected((32, 48), 3, 0.4), 16, 2, contrast=1e4, bc="mbb"),
                     W.cantilever_3d(a=2, seed=5, blk=4, overlap=1, contrast=1e4)):
            d = design_from_problem(ctx, prob, coarse=False)
            rng = np.random.default_rng(7)
            for call in range(2):
                x = rng.standard_normal(prob.ndof)
                x[prob.dirichlet] = 0.0
                xt = torch.as_tensor(x, device="cuda")
                y_ref = d.apply_K(xt)
                y = torch.full_like(xt, float("nan"))
                out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
                st = _call(L, d, xt, y, out)
                assert st == N.TS_OK, L.ts_last_error(ctx._p)
                torch.cuda.synchronize()
                # same kernel as ts_apply_K: identical products, identical sums
                assert torch.equal(y, y_ref), (prob.name, call)
                # energy: a different summation order than the reference dot
                e_ref = float(torch.dot(xt, y_ref))
                scale = float(torch.dot(xt.abs(), y_ref.abs()))
                assert abs(float(out[0]) - e_ref) <= 1e-13 * scale, (prob.name, call, float(out[0]), e_ref)
            d.close()
    finally:
        ctx.close()


def test_static_scratch_rejects_meshes_beyond_its_limit():
    """4096 x 4096 Q4 elements: 4097 x 4097 nodes need ceil(4097/32) *
    ceil(4097/8) = 66,177 product blocks, more than the 65,536 slots of the
    fixed scratch.  Level 1 only and FP32 local factors keep the setup small."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13387_gb300 import Context, _native as N
    from paper_2006_13387_gb300.api import Design
    n = 4096
    blocks = -(-(n + 1) // 32) * -(-(n + 1) // 8)
    assert blocks > 65536
    d_, _ = W.bc_cantilever_2d(n, n)
    ctx = Context()
    try:
        L = N.lib()
        d = Design(ctx, dim=2, nx=n, ny=n, blk=32, overlap=1, rho=np.ones(n * n), E0=1.0, Emin=1e-4, p=3.0,
                   nu=0.3, dirichlet=d_, precision="mixed", coarse=False)
        xt = torch.zeros(d.ndof, dtype=torch.float64, device="cuda")
        y = torch.full_like(xt, 7.0)
        out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
        st = _call(L, d, xt, y, out)
        assert st == N.TS_ERR_INVALID
        assert b"fixed scratch" in L.ts_last_error(ctx._p)
        torch.cuda.synchronize()
        assert bool((y == 7.0).all()) and float(out[0]) == 7.0
        d.close()
    finally:
        ctx.close()
