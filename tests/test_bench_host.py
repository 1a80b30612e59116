"""Host logic of bench.py that needs no GPU: the requests of the serving leg
(sizes that the blocks divide, both dimensions, the contrast range), the
instances of the batch leg
(configuration 4's size, volume and contrast ranges, blocks dividing the
mesh, reproducible) and the oracle baseline's linear extrapolation model."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_batch_instances_ranges_and_blocks():
    sizes = set()
    for i in range(24):
        p = bench._batch_instance(i)
        assert p.dim == 2 and 128 <= p.nx <= 384 and p.ny == p.nx // 2
        assert p.nx % 16 == 0 and p.ny % 16 == 0 and tuple(p.blk[:2]) == (16, 16) and p.overlap == 2
        assert 1e4 * (1 - 1e-12) <= p.E0 / p.Emin <= 1e8 * (1 + 1e-12)
        assert 0.30 - 1e-3 <= float(np.mean(p.rho)) <= 0.50 + 1e-3
        assert p.f.shape == (1, p.ndof)
        sizes.add(p.nx)
    assert len(sizes) >= 4  # uneven sizes
    a, b = bench._batch_instance(5), bench._batch_instance(5)
    assert a.nx == b.nx and np.array_equal(a.rho, b.rho) and a.Emin == b.Emin


def test_extrapolation_model():
    # setup scales with the subdomain count, an iteration with the DOF count,
    # 8 load cases at the given iteration count
    nd3 = 2 * (bench.C3["nx"] + 1) * (bench.C3["ny"] + 1)
    nsub3 = (bench.C3["nx"] // 16) * (bench.C3["ny"] // 16)
    t = bench._extrapolate(2.0, 0.01, nd3 / 4, nsub3 / 8, 100.0)
    assert np.isclose(t, 2.0 * 8 + bench.C3["nrhs"] * 100.0 * 0.01 * 4)


def test_serving_requests_fit_their_blocks():
    # half 2D (nx = 32 U{8..32}, ny = nx / 2, 16 x 16 blocks), half 3D
    # (4 (2a, a, a), a in U{4..8}, 4 x 4 x 4 blocks); contrast in [1e4, 1e6]
    class _Pool:  # small stand-in fields: windows are cut at seeded offsets
        rho = {2: np.random.default_rng(0).random((1024, 2048)), 3: np.random.default_rng(1).random((48, 48, 96))}
        window = staticmethod(bench._ServePool.window)
    seen = set()
    for i in range(16):
        prob, shape = bench._serve_request(i, _Pool())
        assert prob.dim == (2 if i % 2 == 0 else 3)
        if prob.dim == 2:
            assert 256 <= prob.nx <= 1024 and prob.nx % 32 == 0 and prob.ny == prob.nx // 2
            assert prob.ny % prob.blk[1] == 0 and prob.nx % prob.blk[0] == 0 and prob.blk[0] == 16
        else:
            a = prob.ny // 4
            assert 4 <= a <= 8 and (prob.nx, prob.ny, prob.nz) == (8 * a, 4 * a, 4 * a) and prob.blk[0] == 4
        assert 1e4 * (1 - 1e-12) <= prob.E0 / prob.Emin <= 1e6 * (1 + 1e-12)
        assert prob.rho.size == int(np.prod(shape))
        seen.add(prob.dim)
    assert seen == {2, 3}
