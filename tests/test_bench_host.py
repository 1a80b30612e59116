"""Host logic of bench.py that needs no GPU: the instances of the batch leg
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
