"""Pins of the oracle's PBNG solver (Section "Position-Based Nonlinear
Gauss-Seidel": Eq. pbgn_update, Eq. pbgn_dx, Eq. mod_hess; Section
"Acceleration Techniques") and of its Newton and adjoint references."""

import numpy as np
import pytest

import workloads as W


def _rot(axis, ang):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _loaded_problem():
    """Small twisted block with gravity, springs and an active contact plane,
    so every term of the energy is exercised."""
    p = W.twist_block(2, 40.0, 0.1)
    p.body_accel = np.array([0.3, -0.2, -9.8])
    p.density = np.full(p.ne, 1000.0)
    p.spr_idx = np.array([4, 13], np.int32)
    p.spr_target = p.X[p.spr_idx] + np.array([[0.02, -0.01, -0.05], [0.0, 0.03, 0.01]])
    p.spr_k = np.array([1e4, 3e3])
    nrm = np.array([0.0, 0.1, 1.0]) / np.linalg.norm([0.0, 0.1, 1.0])
    p.plane = np.array([nrm[0], nrm[1], nrm[2], 0.6])  # cuts the free middle layer
    p.k_contact = 1e6
    return p


def test_residual_is_minus_energy_gradient(oracle_mod):
    p = _loaded_problem()
    m = oracle_mod.OracleMesh.from_problem(p)
    rng = np.random.default_rng(0)
    x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape) * (1 - p.dirichlet_mask()[:, None])
    _, r = m.residual(x, vector=True)
    free = np.flatnonzero(p.dirichlet_mask() == 0)
    h = 1e-7
    for i in free[:10]:
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h; xm[i, a] -= h
            g = (m.energy(xp) - m.energy(xm)) / (2 * h)
            assert -g == pytest.approx(r[i, a], rel=1e-6, abs=1e-6 * np.abs(r).max())


def test_local_system_at_rest(oracle_mod):
    p = W.twist_block(3)
    m = oracle_mod.OracleMesh.from_problem(p)
    B, V, mu, lam = m.tet_constants()
    for i in (21, 22, 37):
        r, A = m.local_system(p.X, i)
        assert np.abs(r).max() < 1e-9
        expect = np.zeros((3, 3))
        for e in np.flatnonzero((p.tets == i).any(1)):
            k = int(np.flatnonzero(p.tets[e] == i)[0])
            g = -B[e].sum(0) if k == 0 else B[e][k - 1]
            expect += V[e] * (2 * mu[e] * (g @ g) * np.eye(3) + lam[e] * np.outer(g, g))
        assert np.allclose(A, expect, rtol=1e-12)
        assert np.linalg.eigvalsh(A).min() > 0


def _affine_problem(n=3):
    p = W.twist_block(n)
    Q = _rot([0.3, -1.0, 0.5], 0.4)
    M = Q @ np.diag([1.1, 0.95, 1.0])
    b = np.array([0.1, -0.2, 0.05])
    xa = p.X @ M.T + b
    outer = np.flatnonzero((np.isclose(p.X, 0) | np.isclose(p.X, 1)).any(1)).astype(np.int32)
    p.dirichlet = outer
    p.x0 = xa.copy()
    return p, M, xa


def test_patch_test_affine_field(oracle_mod):
    p, M, xa = _affine_problem()
    m = oracle_mod.OracleMesh.from_problem(p)
    B, V, mu, lam = m.tet_constants()
    s = np.linalg.svd(M, compute_uv=False)
    psiM = mu[0] * np.sum((s - 1) ** 2) + 0.5 * lam[0] * (np.prod(s) - 1) ** 2
    assert m.energy(xa) == pytest.approx(psiM * 1.0 - 0.0, rel=1e-12)
    n, r = m.residual(xa, vector=True)
    scale = mu[0] * (1.0 / 3) ** 2  # stress times face area
    assert n <= 1e-12 * scale
    x1, st = m.sweeps(xa, 1)
    assert st == 0 and np.abs(x1 - xa).max() <= 1e-13
    rng = np.random.default_rng(1)
    xp = xa.copy()
    free = p.dirichlet_mask() == 0
    xp[free] += 1e-2 / 3 * rng.standard_normal((free.sum(), 3))
    x2, st = m.sweeps(xp, 200)
    assert np.abs(x2 - xa).max() <= 1e-9


def test_sweep_commutes_with_rigid_motion(oracle_mod):
    p = W.twist_block(3, 60.0, 0.2)
    m = oracle_mod.OracleMesh.from_problem(p)
    Q = _rot([1.0, 2.0, -0.5], 0.8)
    b = np.array([0.3, -1.0, 2.0])
    x1, _ = m.sweeps(p.x0, 3)
    x2, _ = m.sweeps(p.x0 @ Q.T + b, 3)
    assert np.abs(x2 - (x1 @ Q.T + b)).max() <= 1e-11


def test_single_free_vertex_is_modified_newton(oracle_mod):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tets = np.array([[0, 1, 2, 3]], np.int32)
    mask = np.array([1, 1, 1, 0], np.uint8)
    m = oracle_mod.OracleMesh(X, tets, 1e5, 0.3, mask, body_accel=[0, 0, -9.8],
                              density=[5e4])
    x0 = X.copy(); x0[3] = [0.3, -0.2, 1.4]
    xs, st, hist = m.sweeps(x0, 2000, history=True)
    xn, it, res = m.newton(x0, 1e-13, 100)
    assert it >= 0
    assert np.abs(xs - xn).max() <= 1e-10
    assert hist[-1] <= 1e-9 * hist[0]


@pytest.mark.parametrize("maker", [lambda: W.twist_block(2, 45.0, 0.2),
                                   lambda: W.twist_block(3, 90.0, 0.3),
                                   lambda: W.gravity_sag(3)])
@pytest.mark.parametrize("accel,order", [("none", "forward"), ("chebyshev", "forward"), ("sor", "forward"),
                                         ("none", "symmetric"), ("chebyshev", "symmetric")])
def test_pbng_reaches_newton_equilibrium(oracle_mod, maker, accel, order):
    p = maker()
    m = oracle_mod.OracleMesh.from_problem(p)
    xn, it, res = m.newton(p.x0, 1e-13, 60)
    assert it >= 0
    omega = 1.5 if accel == "sor" else 1.7
    gamma = 1.0 if (accel == "chebyshev" and p.body_accel is None and p.nv > 30) else 1.7
    xs, st, hist = m.sweeps(p.x0, 3000, accel=accel, omega=omega, gamma=gamma, history=True, order=order)
    assert st == 0
    assert hist[-1] <= 1e-9 * hist[0]
    assert np.abs(xs - xn).max() <= 1e-9 * max(1.0, np.abs(xn - p.X).max())


def test_acceleration_reduces_to_plain(oracle_mod):
    p = W.twist_block(3)
    m = oracle_mod.OracleMesh.from_problem(p)
    xp, _ = m.sweeps(p.x0, 20)
    xc, _ = m.sweeps(p.x0, 20, accel="chebyshev", rho=0.0, gamma=1.0)
    xs, _ = m.sweeps(p.x0, 20, accel="sor", omega=1.0)
    assert np.abs(xc - xp).max() <= 1e-12 and np.abs(xs - xp).max() <= 1e-12


def test_symmetric_order_chebyshev_beats_forward_on_a_sag_cube(oracle_mod):
    # The symmetric colour order's real spectrum is what the Chebyshev weights
    # assume: on a bending-dominated, nearly incompressible cube it reaches a
    # residual that the ascending order does not, for the same number of
    # colour passes, with rho near the measured plain rate.
    p = W.gravity_sag(6)
    m = oracle_mod.OracleMesh.from_problem(p)
    C = m.ncolours
    nf = 300
    ns = nf * C // (2 * C - 1)
    _, _, hf = m.sweeps(p.x0, nf, accel="chebyshev", rho=0.98, history=True, threads=4)
    _, _, hs = m.sweeps(p.x0, ns, accel="chebyshev", rho=0.995, history=True, threads=4, order="symmetric")
    assert hs[-1] < 1e-6 * hs[0]
    assert hs[-1] < 1e-2 * hf[-1]


def test_chebyshev_beats_plain_at_equal_sweeps(oracle_mod):
    # Section "Acceleration Comparison": acceleration boosts the residual
    # reduction at a fixed number of iterations.
    p = W.twist_block(6, 90.0, 0.3)
    m = oracle_mod.OracleMesh.from_problem(p)
    _, _, hp = m.sweeps(p.x0, 60, history=True)
    _, _, hc = m.sweeps(p.x0, 60, accel="chebyshev", history=True)
    assert hc[-1] < hp[-1]


def test_skip_tol_freezes_converged_nodes(oracle_mod):
    p = W.twist_block(2)
    m = oracle_mod.OracleMesh.from_problem(p)
    x1, _ = m.sweeps(p.x0, 1, skip_tol=1e30)
    assert np.array_equal(x1, p.x0)


def test_dense_hessian_is_residual_derivative(oracle_mod):
    p = _loaded_problem()
    m = oracle_mod.OracleMesh.from_problem(p)
    rng = np.random.default_rng(2)
    x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape)
    H = m.hessian(x)
    assert np.allclose(H, H.T, rtol=1e-8, atol=1e-6 * np.abs(H).max())
    h = 1e-7
    for k in rng.choice(3 * p.nv, 8, replace=False):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[k] += h; xm[k] -= h
        # -d(f + f^ext)/dx via the residual, which zeroes clamped rows
        _, rp = m.residual(xp.reshape(-1, 3), vector=True)
        _, rm = m.residual(xm.reshape(-1, 3), vector=True)
        col = -(rp - rm).ravel() / (2 * h)
        free = np.repeat(p.dirichlet_mask() == 0, 3)
        assert np.allclose(col[free], H[free, k], rtol=1e-5, atol=1e-5 * np.abs(H).max())


def test_adjoint_matches_finite_differences(oracle_mod):
    p = W.twist_block(2, 30.0, 0.1)
    p.body_accel = np.array([0.0, 0.0, -9.8])
    p.density = np.full(p.ne, 3000.0)
    m = oracle_mod.OracleMesh.from_problem(p)
    xeq, it, _ = m.newton(p.x0, 1e-13, 60)
    assert it >= 0
    top = np.flatnonzero(np.isclose(p.X[:, 2], 0.5))
    target = xeq[top] + 0.01
    w = np.zeros(p.nv); w[top] = 1.0

    tgt_full = np.zeros((p.nv, 3)); tgt_full[top] = target

    def L(x):
        return float(np.sum(w[:, None] * (x - tgt_full) ** 2))

    dLdx = 2 * w[:, None] * (xeq - tgt_full)
    dE, dD = m.adjoint(xeq, dLdx)

    def solve(young, xd_shift):
        q = W.twist_block(2, 30.0, 0.1)
        q.body_accel, q.density = p.body_accel, p.density
        q.young = young
        x0 = p.x0.copy()
        x0[q.dirichlet] += xd_shift
        mq = oracle_mod.OracleMesh.from_problem(q)
        x, it, _ = mq.newton(x0, 1e-13, 60)
        assert it >= 0
        return x

    eps = 1e-4
    for e in (0, 5, 17):
        yp, ym = p.young.copy(), p.young.copy()
        yp[e] *= np.exp(eps); ym[e] *= np.exp(-eps)
        z = np.zeros((len(p.dirichlet), 3))
        fd = (L(solve(yp, z)) - L(solve(ym, z))) / (2 * eps)
        assert dE[e] == pytest.approx(fd, rel=1e-5, abs=1e-10)
    rng = np.random.default_rng(3)
    d = rng.standard_normal((len(p.dirichlet), 3))
    h = 1e-6
    fd = (L(solve(p.young, h * d)) - L(solve(p.young, -h * d))) / (2 * h)
    assert np.sum(dD * d) == pytest.approx(fd, rel=1e-5)


def test_local_hessian_is_contracted_density_hessian(oracle_mod):
    # Eq. mod_hess: A_ab = sum_e V_e sum_{g,d} C~_{a g b d} dN_i/dX_g dN_i/dX_d.
    p = W.twist_block(3, 70.0, 0.25)
    m = oracle_mod.OracleMesh.from_problem(p)
    B, V, mu, lam = m.tet_constants()
    rng = np.random.default_rng(4)
    x = p.x0 + 0.02 * rng.standard_normal(p.x0.shape)
    for i in (21, 26, 38):
        _, A = m.local_system(x, i)
        expect = np.zeros((3, 3))
        for e in np.flatnonzero((p.tets == i).any(1)):
            G = np.vstack([-B[e].sum(0), B[e]])          # rows g_0..g_3
            F = x[p.tets[e]].T @ G                        # sum_j x_j g_j^T
            k = int(np.flatnonzero(p.tets[e] == i)[0])
            C = oracle_mod.modified_density_hessian(F, mu[e], lam[e]).reshape(3, 3, 3, 3)
            expect += V[e] * np.einsum("agbd,g,d->ab", C, G[k], G[k])
        assert np.allclose(A, expect, rtol=1e-12)
