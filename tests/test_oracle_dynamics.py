"""Pins of the oracle's backward-Euler step (Eq. fem_be, lumped mass
m_ii = sum_e rho_e V_e / 4) as the incremental potential PBNG minimises:

* free fall: a rigid translation has no internal force, so every solved step
  follows the closed-form recurrence x^{n+1} = 2 x^n - x^{n-1} + dt^2 g;
* residual = -gradient of the incremental potential (FD);
* dt -> infinity recovers the quasistatic equilibrium;
* dt -> 0: (x^{n+1} - xhat) / dt^2 -> M^{-1} (f(xhat) + f^ext), which pins
  the m_ii / dt^2 scaling;
* PBNG with inertia reaches the Newton solution of the step."""

import numpy as np
import pytest

import workloads as W


def _free_block(n=2):
    p = W.twist_block(n, 0.0, 0.0)
    p.dirichlet = np.zeros(0, np.int32)
    p.body_accel = np.array([0.5, -1.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    p.x0 = p.X.copy()
    return p


def test_free_fall_follows_the_backward_euler_recurrence(oracle_mod):
    p = _free_block(2)
    m = oracle_mod.OracleMesh.from_problem(p)
    dt, g = 1e-2, p.body_accel
    v0 = np.array([0.3, 0.1, -0.2])
    x_prev, x = p.X - dt * v0, p.X.copy()
    for n in range(1, 6):
        m.set_inertia(dt, p.density, 2 * x - x_prev)
        x_new, st, hist = m.sweeps(x, 60, history=True)
        assert st == 0 and hist[-1] <= 1e-10 * max(hist[0], 1e-30) + 1e-12
        expect = p.X + n * dt * v0 + dt * dt * g * n * (n + 1) / 2
        assert np.abs(x_new - expect).max() <= 1e-10
        x_prev, x = x, x_new


def test_lumped_mass_is_total_mass(oracle_mod):
    p = _free_block(3)
    m = oracle_mod.OracleMesh.from_problem(p)
    m.set_inertia(1e-2, p.density, p.X)
    B, V, mu, lam = m.tet_constants()
    assert m.lumped_mass().sum() == pytest.approx((p.density * V).sum(), rel=1e-13)
    assert m.lumped_mass().sum() == pytest.approx(1000.0 * 1.0, rel=1e-12)   # unit cube


def test_residual_is_minus_gradient_of_the_incremental_potential(oracle_mod):
    p = W.twist_block(2, 40.0, 0.1)
    p.body_accel = np.array([0.3, -0.2, -9.8])
    p.density = np.full(p.ne, 1000.0)
    m = oracle_mod.OracleMesh.from_problem(p)
    rng = np.random.default_rng(1)
    free = p.dirichlet_mask() == 0
    m.set_inertia(3e-3, p.density, p.x0 + 0.02 * rng.standard_normal(p.x0.shape) * free[:, None])
    x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape) * free[:, None]
    _, r = m.residual(x, vector=True)
    h = 1e-7
    for i in np.flatnonzero(free)[:9]:
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (m.energy(xp) - m.energy(xm)) / (2 * h)
            assert -g == pytest.approx(r[i, a], rel=1e-6, abs=1e-6 * np.abs(r).max())


def test_large_dt_recovers_quasistatics(oracle_mod):
    p = W.gravity_sag(3)
    m = oracle_mod.OracleMesh.from_problem(p)
    xq, it, _ = m.newton(p.x0, 1e-13, 60)
    assert it >= 0
    m.set_inertia(1e5, p.density, p.X + 0.1)
    xd, it, _ = m.newton(p.x0, 1e-13, 60)
    assert it >= 0
    assert np.abs(xd - xq).max() <= 1e-6 * np.abs(xq - p.X).max()


def test_small_dt_limit_is_explicit_acceleration(oracle_mod):
    p = W.twist_block(2, 60.0, 0.2)
    p.body_accel = np.array([0.0, 0.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    m = oracle_mod.OracleMesh.from_problem(p)
    xhat = p.x0.copy()
    _, f = m.residual(xhat, vector=True)          # f(xhat) + f^ext on free vertices
    m.set_inertia(1.0, p.density, xhat)
    mass = m.lumped_mass()
    free = p.dirichlet_mask() == 0
    acc = f[free] / mass[free][:, None]
    errs = []
    for dt in (1e-3, 1e-4):
        m.set_inertia(dt, p.density, xhat)
        x, it, _ = m.newton(xhat, 1e-9, 30)   # k = m / dt^2 puts the rounding floor near 1e-10
        assert it >= 0
        errs.append(np.abs((x[free] - xhat[free]) / dt ** 2 - acc).max() / np.abs(acc).max())
    assert errs[0] < 1e-2 and errs[1] < 0.2 * errs[0]


def test_pbng_with_inertia_reaches_the_newton_step(oracle_mod):
    p = W.twist_block(3, 90.0, 0.3)
    p.body_accel = np.array([0.0, 0.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    m = oracle_mod.OracleMesh.from_problem(p)
    m.set_inertia(1e-2, p.density, p.x0)
    xn, it, _ = m.newton(p.x0, 1e-13, 60)
    assert it >= 0
    xs, st, hist = m.sweeps(p.X.copy() * 0 + p.x0, 400, accel="chebyshev", history=True)
    assert st == 0 and hist[-1] <= 1e-10 * hist[0]
    assert np.abs(xs - xn).max() <= 1e-9 * max(1.0, np.abs(xn - p.X).max())
