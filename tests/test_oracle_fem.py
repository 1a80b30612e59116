"""Pins of the oracle's finite-element layer (Sec. 1.1, Eqs. 4-9) against
facts that do not come from the oracle itself."""
import numpy as np
import pytest

import workloads as W
from oracle import fem


def _rbm_2d(prob):
    X = fem.node_coords(prob)
    n = X.shape[0]
    t1 = np.zeros(2 * n); t1[0::2] = 1
    t2 = np.zeros(2 * n); t2[1::2] = 1
    rot = np.zeros(2 * n); rot[0::2] = -X[:, 1]; rot[1::2] = X[:, 0]
    return [t1, t2, rot]


def _rbm_3d(prob):
    X = fem.node_coords(prob)
    n = X.shape[0]
    out = []
    for c in range(3):
        t = np.zeros(3 * n); t[c::3] = 1; out.append(t)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    for a, b in [((1, -z), (2, y)), ((0, z), (2, -x)), ((0, -y), (1, x))]:
        v = np.zeros(3 * n); v[a[0]::3] = a[1]; v[b[0]::3] = b[1]; out.append(v)
    return out


def test_ke_q4_symbolic():
    """P1: KE equals the exact symbolic integral of B^T D B over the unit square."""
    sympy = pytest.importorskip("sympy")
    x, y, nu = sympy.symbols("x y nu")
    N = [(1 - x) * (1 - y), x * (1 - y), x * y, (1 - x) * y]
    B = sympy.zeros(3, 8)
    for a in range(4):
        B[0, 2 * a] = sympy.diff(N[a], x)
        B[1, 2 * a + 1] = sympy.diff(N[a], y)
        B[2, 2 * a] = sympy.diff(N[a], y)
        B[2, 2 * a + 1] = sympy.diff(N[a], x)
    D = sympy.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
    KEs = (B.T * D * B).applyfunc(lambda t: sympy.integrate(sympy.integrate(t, (x, 0, 1)), (y, 0, 1)))
    for v in (0.0, 0.3, 0.45):
        ref = np.array(KEs.subs(nu, v).evalf(), dtype=np.float64)
        assert np.allclose(fem.ke_q4(v), ref, rtol=1e-14, atol=1e-15)


def test_ke_hex8_symbolic_diagonal_and_kernel():
    """P1 (3D): KE symmetric, exactly 6 zero eigenvalues (rigid modes), and the
    first row equals the exact symbolic integral."""
    sympy = pytest.importorskip("sympy")
    KE = fem.ke_hex8(0.3)
    assert np.allclose(KE, KE.T, atol=1e-15)
    ev = np.linalg.eigvalsh(KE)
    assert np.sum(np.abs(ev) < 1e-12) == 6 and ev[6] > 1e-3
    x, y, z = sympy.symbols("x y z")
    nodes = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    N = [((x if a else 1 - x) * (y if b else 1 - y) * (z if c else 1 - z)) for a, b, c in nodes]
    nu = sympy.Rational(3, 10)
    lam = nu / ((1 + nu) * (1 - 2 * nu)); mu = 1 / (2 * (1 + nu))
    D = sympy.zeros(6, 6)
    for i in range(3):
        for j in range(3):
            D[i, j] = lam
        D[i, i] += 2 * mu
        D[3 + i, 3 + i] = mu
    B = sympy.zeros(6, 24)
    for a in range(8):
        gx, gy, gz = [sympy.diff(N[a], s) for s in (x, y, z)]
        B[0, 3 * a] = gx; B[1, 3 * a + 1] = gy; B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1] = gz; B[3, 3 * a + 2] = gy
        B[4, 3 * a] = gz; B[4, 3 * a + 2] = gx
        B[5, 3 * a] = gy; B[5, 3 * a + 1] = gx
    row = (B[:, 0].T * D * B)
    ref = [float(sympy.integrate(row[0, j], (x, 0, 1), (y, 0, 1), (z, 0, 1))) for j in range(24)]
    assert np.allclose(KE[0], ref, rtol=1e-13, atol=1e-15)


def test_heat_element_textbook():
    """Q1 heat element matrices: the textbook unit-square values."""
    Kh, Mh = fem.heat_element(2)
    Kref = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    Mref = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0
    assert np.allclose(Kh, Kref, atol=1e-15) and np.allclose(Mh, Mref, atol=1e-15)
    Kh3, Mh3 = fem.heat_element(3)
    assert abs(Mh3.sum() - 1.0) < 1e-14 and np.allclose(Kh3.sum(axis=1), 0, atol=1e-15)
    assert abs(Kh3[0, 0] - 1.0 / 3.0) < 1e-15 and abs(Mh3[0, 0] - 1.0 / 27.0) < 1e-15


def test_simp():
    """Eq. 4 at its end points and p = 3."""
    E = fem.simp(np.array([0.0, 1.0, 0.5]), 1.0, 1e-6, 3.0)
    assert E[0] == 1e-6 and E[1] == 1.0 and abs(E[2] - (1e-6 + 0.125 * (1 - 1e-6))) < 1e-16


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_body_modes_in_kernel(dim):
    """P2: K (unconstrained) annihilates the rigid body modes (Sec. 2.1, RBM
    space), K symmetric, and the Dirichlet-constrained K is SPD."""
    rng = np.random.default_rng(1)
    if dim == 2:
        prob = W.custom_2d(6, 4, rng.random(24), 2, 1)
        modes = _rbm_2d(prob)
    else:
        prob = W.cantilever_3d(a=1)
        prob.rho[:] = rng.random(prob.rho.size)
        modes = _rbm_3d(prob)
    K = fem.assemble_K(prob)
    assert abs(K - K.T).max() < 1e-15
    scale = abs(K).max()
    for m in modes:
        assert np.abs(K @ m).max() <= 1e-13 * scale * np.abs(m).max()
    Kc = fem.constrained_K(prob, K).toarray()
    assert np.linalg.eigvalsh(Kc).min() > 0


def test_patch_test():
    """P3: homogeneous material, a linear displacement field prescribed on the
    whole boundary gives the same linear field inside (to 1e-12)."""
    nx, ny = 7, 5
    prob = W.custom_2d(nx, ny, np.ones(nx * ny), 1, 0)
    K = fem.assemble_K(prob).toarray()
    X = fem.node_coords(prob)
    ulin = np.zeros(prob.ndof)
    ulin[0::2] = 0.3 + 0.01 * X[:, 0] - 0.02 * X[:, 1]
    ulin[1::2] = -0.1 + 0.03 * X[:, 0] + 0.015 * X[:, 1]
    bnd = (X[:, 0] == 0) | (X[:, 0] == nx) | (X[:, 1] == 0) | (X[:, 1] == ny)
    bd = np.flatnonzero(np.repeat(bnd, 2))
    fr = np.flatnonzero(~np.repeat(bnd, 2))
    uf = np.linalg.solve(K[np.ix_(fr, fr)], -K[np.ix_(fr, bd)] @ ulin[bd])
    assert np.abs(uf - ulin[fr]).max() < 1e-12


@pytest.mark.parametrize("nx,ny,bc", [(4, 2, "cantilever"), (8, 4, "mbb"), (16, 8, "cantilever"), (6, 6, "box")])
def test_direct_solve_brute_force(nx, ny, bc):
    """P4: the sparse direct solve agrees with a dense LAPACK solve of the
    eliminated system within the dense solve's cond*eps error bound, and
    f^T u = u^T K u."""
    rng = np.random.default_rng(nx * 100 + ny)
    rho = (rng.random(nx * ny) > 0.5).astype(float)
    prob = W.custom_2d(nx, ny, rho, 2, 1, contrast=1e4, bc=bc)
    K = fem.assemble_K(prob)
    u = fem.direct_solve(prob, K)[0]
    free = np.flatnonzero(fem.free_mask(prob))
    Kd = K.toarray()[np.ix_(free, free)]
    ud = np.linalg.solve(Kd, prob.f[0, free])
    # dense LU's forward error bound: cond(K) * eps (times a small constant)
    bound = 10.0 * np.linalg.cond(Kd) * np.finfo(float).eps
    assert np.abs(u[free] - ud).max() <= bound * np.abs(ud).max()
    assert abs(prob.f[0] @ u - u @ (K @ u)) <= 1e-10 * abs(prob.f[0] @ u)
    assert np.all(u[prob.dirichlet] == 0.0)


def test_sensitivity_finite_differences():
    """Eq. 1003 against central differences of the compliance g_0 = f^T u(rho)
    computed by the direct solve (the adjoint of the compliance is u itself)."""
    rng = np.random.default_rng(7)
    prob = W.custom_2d(8, 4, rng.uniform(0.2, 1.0, 32), blk=4, overlap=1, contrast=1e3)
    u = fem.direct_solve(prob)[0]
    dc, c = fem.sensitivity(prob, u)
    assert abs(c - fem.compliance(prob.f[0], u)) <= 1e-12 * abs(c)
    h = 1e-5
    for e in (0, 5, 17, 31):
        cs = []
        for sgn in (1.0, -1.0):
            rho = prob.rho.copy()
            rho[e] += sgn * h
            pe = W.custom_2d(8, 4, rho, blk=4, overlap=1, contrast=1e3)
            cs.append(fem.compliance(pe.f[0], fem.direct_solve(pe)[0]))
        fd = (cs[0] - cs[1]) / (2 * h)
        assert abs(fd - dc[e]) <= 1e-6 * abs(dc[e]), (e, fd, dc[e])


def test_oc_update_invariants():
    """The OC update keeps the volume fraction, the move limit and [0, 1], and
    moves densities up where the sensitivity is large and down where it is small."""
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.05, 0.95, 4000)
    dc = -np.exp(rng.normal(0.0, 3.0, 4000))
    new = fem.oc_update(rho, dc, volfrac=0.45, move=0.1)
    assert abs(new.mean() - 0.45) <= 1e-12
    assert np.all(new >= 0.0) and np.all(new <= 1.0)
    assert np.all(np.abs(new - rho) <= 0.1 + 1e-15)
    # the unclamped elements share one multiplier: new/rho = sqrt(-dc/lam)
    free = (new > np.maximum(0, rho - 0.1) + 1e-9) & (new < np.minimum(1, rho + 0.1) - 1e-9)
    lam = -dc[free] / (new[free] / rho[free]) ** 2
    assert np.ptp(lam) <= 1e-9 * lam.mean()
