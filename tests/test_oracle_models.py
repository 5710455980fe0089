"""Pins of the oracle's Neo-Hookean (Eq. nh) and stable Neo-Hookean (Eq. snh)
models, Section "Constitutive Models", against what the paper and the
mathematics fix rather than against a retyped formula:

* every model is free of stress at rest and under any rotation;
* Section "Lame Coefficients": a model set from Lame coefficients must have
  the linear-elasticity Hessian at F = I, mu (dF + dF^T) + lambda tr(dF) I.
  That pins lambda_hat = mu + lambda of Eq. nh and the reading of Eq. snh
  (its missing lambda and the Lame reparametrisation);
* isotropy and frame invariance of Psi;
* P = dPsi/dF and the density Hessian = dP/dF by central differences, also
  for inverted F;
* at mesh level: residual = -grad(energy) and PBNG reaches the Newton
  equilibrium of the same model; the modified Hessian of Eq. mod_hess_dens
  is the same for every model."""

import numpy as np
import pytest

import workloads as W

MU, LAM = 38461.538461538461, 57692.307692307692
MODELS = [0, 1, 2]


def _rot(axis, ang):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _random_F(rng, n, inverted=False, scale=0.35):
    out = []
    while len(out) < n:
        F = np.eye(3) + scale * rng.standard_normal((3, 3))
        d = np.linalg.det(F)
        if abs(d) < 0.05:
            continue
        if (d < 0) != inverted:
            F[:, 2] *= -1
        out.append(F)
    return out


@pytest.mark.parametrize("model", MODELS)
def test_stress_free_at_rest_and_under_rotation(oracle_mod, model):
    assert np.abs(oracle_mod.pk1(np.eye(3), MU, LAM, model)).max() < 1e-9 * MU
    for ax, ang in (([1, 0, 0], 0.3), ([1, 2, 3], 2.5), ([0, -1, 1], 3.0)):
        Q = _rot(ax, ang)
        assert np.abs(oracle_mod.pk1(Q, MU, LAM, model)).max() < 1e-8 * MU
        assert oracle_mod.psi(Q, MU, LAM, model) == pytest.approx(oracle_mod.psi(np.eye(3), MU, LAM, model),
                                                                  rel=1e-12, abs=1e-9 * MU)


@pytest.mark.parametrize("model", MODELS)
def test_hessian_at_rest_is_linear_elasticity(oracle_mod, model):
    # Section "Lame Coefficients": d2Psi/dF2 at F = I must be that of Eq. le.
    rng = np.random.default_rng(11 + model)
    for _ in range(10):
        dF = rng.standard_normal((3, 3))
        expect = MU * (dF + dF.T) + LAM * np.trace(dF) * np.eye(3)
        got = oracle_mod.dpk1(np.eye(3), dF, MU, LAM, model)
        assert np.allclose(got, expect, rtol=1e-10, atol=1e-9 * MU * np.abs(dF).max())


@pytest.mark.parametrize("model", [1, 2])
def test_energy_is_isotropic_and_frame_invariant(oracle_mod, model):
    rng = np.random.default_rng(3)
    for F in _random_F(rng, 8) + _random_F(rng, 4, inverted=True):
        Q1, Q2 = _rot(rng.standard_normal(3), 1.1), _rot(rng.standard_normal(3), -2.2)
        v = oracle_mod.psi(F, MU, LAM, model)
        assert oracle_mod.psi(Q1 @ F, MU, LAM, model) == pytest.approx(v, rel=1e-11)
        assert oracle_mod.psi(F @ Q2, MU, LAM, model) == pytest.approx(v, rel=1e-11)


@pytest.mark.parametrize("model", [1, 2])
def test_pk1_is_gradient_of_psi(oracle_mod, model):
    rng = np.random.default_rng(5)
    h = 1e-6
    for F in _random_F(rng, 6) + _random_F(rng, 4, inverted=True):
        P = oracle_mod.pk1(F, MU, LAM, model)
        G = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += h
                Fm[i, j] -= h
                G[i, j] = (oracle_mod.psi(Fp, MU, LAM, model) - oracle_mod.psi(Fm, MU, LAM, model)) / (2 * h)
        assert np.allclose(P, G, rtol=1e-6, atol=1e-6 * np.abs(P).max())


@pytest.mark.parametrize("model", [1, 2])
def test_density_hessian_is_derivative_of_pk1(oracle_mod, model):
    rng = np.random.default_rng(7)
    h = 1e-6
    for F in _random_F(rng, 5) + _random_F(rng, 3, inverted=True):
        dF = rng.standard_normal((3, 3))
        fd = (oracle_mod.pk1(F + h * dF, MU, LAM, model) - oracle_mod.pk1(F - h * dF, MU, LAM, model)) / (2 * h)
        got = oracle_mod.dpk1(F, dF, MU, LAM, model)
        assert np.allclose(got, fd, rtol=1e-6, atol=1e-6 * np.abs(got).max())


def test_models_differ_away_from_rest(oracle_mod):
    # The three models agree to first order at rest but not at finite strain.
    F = np.diag([1.3, 0.9, 1.1]) @ _rot([1, 1, 0], 0.4)
    P = [oracle_mod.pk1(F, MU, LAM, m) for m in MODELS]
    for a in range(3):
        for b in range(a + 1, 3):
            assert np.abs(P[a] - P[b]).max() > 1e-3 * np.abs(P[a]).max()


def _loaded_problem():
    p = W.twist_block(2, 40.0, 0.1)
    p.body_accel = np.array([0.3, -0.2, -9.8])
    p.density = np.full(p.ne, 1000.0)
    p.spr_idx = np.array([4, 13], np.int32)
    p.spr_target = p.X[p.spr_idx] + np.array([[0.02, -0.01, -0.05], [0.0, 0.03, 0.01]])
    p.spr_k = np.array([1e4, 3e3])
    return p


@pytest.mark.parametrize("model", [1, 2])
def test_mesh_residual_is_minus_energy_gradient(oracle_mod, model):
    p = _loaded_problem()
    m = oracle_mod.OracleMesh.from_problem(p, model=model)
    rng = np.random.default_rng(0)
    x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape) * (1 - p.dirichlet_mask()[:, None])
    _, r = m.residual(x, vector=True)
    free = np.flatnonzero(p.dirichlet_mask() == 0)
    h = 1e-7
    for i in free[:9]:
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (m.energy(xp) - m.energy(xm)) / (2 * h)
            assert -g == pytest.approx(r[i, a], rel=1e-6, abs=1e-6 * np.abs(r).max())


@pytest.mark.parametrize("model", [1, 2])
def test_modified_hessian_is_model_independent(oracle_mod, model):
    # Eq. mod_hess_dens: the same SPD approximation for every model.
    p = W.twist_block(3, 60.0, 0.2)
    m0 = oracle_mod.OracleMesh.from_problem(p)
    m1 = oracle_mod.OracleMesh.from_problem(p, model=model)
    for i in (21, 22, 37):
        r0, A0 = m0.local_system(p.x0, i)
        r1, A1 = m1.local_system(p.x0, i)
        assert np.array_equal(A0, A1)
        assert np.abs(r0 - r1).max() > 1e-6 * np.abs(r0).max()


@pytest.mark.parametrize("model", [1, 2])
@pytest.mark.parametrize("accel", ["none", "chebyshev"])
def test_pbng_reaches_newton_equilibrium_of_the_model(oracle_mod, model, accel):
    p = W.twist_block(3, 90.0, 0.3)
    m = oracle_mod.OracleMesh.from_problem(p, model=model)
    xn, it, res = m.newton(p.x0, 1e-13, 60)
    assert it >= 0
    xs, st, hist = m.sweeps(p.x0, 3000, accel=accel, history=True)
    assert st == 0 and hist[-1] <= 1e-9 * hist[0]
    assert np.abs(xs - xn).max() <= 1e-9 * max(1.0, np.abs(xn - p.X).max())
    m0 = oracle_mod.OracleMesh.from_problem(p)
    x0n, _, _ = m0.newton(p.x0, 1e-13, 60)
    assert np.abs(x0n - xn).max() > 1e-4 * np.abs(xn - p.X).max()   # a different equilibrium


def test_small_strain_models_agree(oracle_mod):
    # Linear-elasticity consistency at mesh level: for a displacement of size
    # eps the three residuals agree up to O(eps^2).
    p = W.twist_block(3, 0.0, 0.0)
    rng = np.random.default_rng(4)
    d = rng.standard_normal(p.X.shape) * (1 - p.dirichlet_mask()[:, None])
    out = []
    for eps in (1e-4, 1e-5):
        x = p.X + eps * d
        rs = [oracle_mod.OracleMesh.from_problem(p, model=k).residual(x, vector=True)[1] for k in MODELS]
        out.append(max(np.abs(rs[k] - rs[0]).max() for k in (1, 2)) / np.abs(rs[0]).max())
    assert out[0] < 1e-3 and out[1] < 0.2 * out[0]
