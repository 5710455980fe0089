"""Pins of the oracle's constitutive layer (Section "Constitutive Models",
Eq. cor / Eq. lame / Eq. mod_hess_dens) against closed forms, library
routines and finite differences."""

import numpy as np
import pytest
import scipy.linalg as sla


def _rot(axis, ang):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _random_F(rng, n, inverted=False):
    out = []
    for _ in range(n):
        F = np.eye(3) + 0.4 * rng.standard_normal((3, 3))
        if inverted and np.linalg.det(F) > 0:
            F[:, 2] *= -1
        if not inverted and np.linalg.det(F) < 0:
            F[:, 2] *= -1
        out.append(F)
    return out


MU, LAM = 38461.538461538461, 57692.307692307692


def test_lame_inverse_relations(oracle_mod):
    # The inverse textbook relations E = mu(3 lam + 2 mu)/(lam + mu) and
    # nu = lam / (2 (lam + mu)) recover the inputs.
    for E, nu in [(1e5, 0.3), (1e3, 0.45), (3e3, 0.0), (2.5e4, 0.25)]:
        mu, lam = oracle_mod.lame(E, nu)
        assert mu * (3 * lam + 2 * mu) / (lam + mu) == pytest.approx(E, rel=1e-14)
        assert lam / (2 * (lam + mu)) == pytest.approx(nu, rel=1e-14, abs=1e-15)
    mu, lam = oracle_mod.lame(2.5e4, 0.25)
    assert lam == pytest.approx(mu, rel=1e-14)  # nu = 1/4 gives lam = mu


def test_svd_matches_numpy(oracle_mod):
    rng = np.random.default_rng(1)
    Fs = _random_F(rng, 30) + _random_F(rng, 30, inverted=True)
    Fs += [np.diag([1.0, 1.0, 1e-9]), np.diag([2.0, 2.0, 2.0]), np.zeros((3, 3)),
           np.outer([1, 2, 3], [0.5, -1, 2.0])]
    for F in Fs:
        U, s, V = oracle_mod.svd3(F)
        assert np.allclose(s, np.linalg.svd(F, compute_uv=False), rtol=1e-13, atol=1e-13)
        assert np.allclose(U @ U.T, np.eye(3), atol=1e-12)
        assert np.allclose(V @ V.T, np.eye(3), atol=1e-12)
        assert np.allclose(U @ np.diag(s) @ V.T, F, atol=1e-12 * max(1, s[0]))


def test_polar_is_closest_rotation(oracle_mod):
    rng = np.random.default_rng(2)
    for F in _random_F(rng, 25) + _random_F(rng, 25, inverted=True):
        R, sh = oracle_mod.polar(F)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        # Kabsch/Umeyama through numpy's SVD: U diag(1, 1, det(U V^T)) V^T.
        U, s, Vt = np.linalg.svd(F)
        D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
        assert np.allclose(R, U @ D @ Vt, atol=1e-10)
        if np.linalg.det(F) > 0:
            assert np.allclose(R, sla.polar(F)[0], atol=1e-10)
        # R maximises tr(Q^T F) over sampled rotations.
        best = np.trace(R.T @ F)
        for _ in range(50):
            Q = _rot(rng.standard_normal(3), rng.uniform(0, np.pi))
            assert np.trace((Q @ R).T @ F) <= best + 1e-12
        assert np.prod(sh) == pytest.approx(np.linalg.det(F), rel=1e-10)


def test_psi_diagonal_closed_form(oracle_mod):
    for sig in ([1.2, 0.9, 1.05], [2.0, 0.5, 0.5], [1.3, 1.1, -0.4], [0.9, 0.7, -0.2]):
        F = np.diag(sig)
        expect = MU * sum((s - 1) ** 2 for s in sig) + 0.5 * LAM * (np.prod(sig) - 1) ** 2
        assert oracle_mod.psi(F, MU, LAM) == pytest.approx(expect, rel=1e-13)


def test_rest_and_rigid_states(oracle_mod):
    assert oracle_mod.psi(np.eye(3), MU, LAM) == 0.0
    assert np.abs(oracle_mod.pk1(np.eye(3), MU, LAM)).max() == 0.0
    Q = _rot([1, 2, 3], 1.1)
    assert oracle_mod.psi(Q, MU, LAM) == pytest.approx(0.0, abs=1e-9)
    assert np.abs(oracle_mod.pk1(Q, MU, LAM)).max() < 1e-9


def test_frame_invariance(oracle_mod):
    rng = np.random.default_rng(3)
    for F in _random_F(rng, 10) + _random_F(rng, 10, inverted=True):
        Q = _rot(rng.standard_normal(3), rng.uniform(0, np.pi))
        p = oracle_mod.psi(F, MU, LAM)
        assert oracle_mod.psi(Q @ F, MU, LAM) == pytest.approx(p, rel=1e-10)
        assert oracle_mod.psi(F @ Q, MU, LAM) == pytest.approx(p, rel=1e-10)
        assert np.allclose(oracle_mod.pk1(Q @ F, MU, LAM), Q @ oracle_mod.pk1(F, MU, LAM),
                           rtol=1e-9, atol=1e-6)


def test_pk1_is_gradient_of_psi(oracle_mod):
    rng = np.random.default_rng(4)
    for F in _random_F(rng, 10) + _random_F(rng, 10, inverted=True):
        P = oracle_mod.pk1(F, MU, LAM)
        h = 1e-6
        G = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                E = np.zeros((3, 3)); E[a, b] = h
                G[a, b] = (oracle_mod.psi(F + E, MU, LAM) - oracle_mod.psi(F - E, MU, LAM)) / (2 * h)
        assert np.abs(G - P).max() <= 1e-7 * np.abs(P).max() + 1e-6


def test_dpk1_is_derivative_of_pk1(oracle_mod):
    rng = np.random.default_rng(5)
    Fs = _random_F(rng, 8) + _random_F(rng, 8, inverted=True) + [_rot([0, 0, 1], 0.7) @ np.diag([1.1, 0.9, 1.0])]
    for F in Fs:
        dF = rng.standard_normal((3, 3))
        h = 1e-6
        fd = (oracle_mod.pk1(F + h * dF, MU, LAM) - oracle_mod.pk1(F - h * dF, MU, LAM)) / (2 * h)
        an = oracle_mod.dpk1(F, dF, MU, LAM)
        assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max() + 1e-4


def test_cofactor(oracle_mod):
    rng = np.random.default_rng(6)
    for F in _random_F(rng, 5) + _random_F(rng, 5, inverted=True):
        assert np.allclose(oracle_mod.cofactor(F), np.linalg.det(F) * np.linalg.inv(F).T, atol=1e-12)
    S = np.array([[1.0, 2.0, 3.0], [0.5, -1.0, 2.0], [1.5, 1.0, 5.0]])  # rank 2
    C = oracle_mod.cofactor(S)
    assert np.abs(C).max() > 0.1
    assert np.allclose(C @ S.T, 0.0, atol=1e-12)  # cof(F) F^T = det(F) I = 0


def test_modified_hessian_is_spd(oracle_mod):
    rng = np.random.default_rng(7)
    for F in _random_F(rng, 5) + _random_F(rng, 5, inverted=True) + [np.diag([1.0, 1.0, 0.0])]:
        C = oracle_mod.modified_density_hessian(F, MU, LAM)
        assert np.allclose(C, C.T)
        w = np.linalg.eigvalsh(C)
        assert w.min() == pytest.approx(2 * MU, rel=1e-10)  # 2 mu I plus a PSD rank-one term
        c = oracle_mod.cofactor(F).ravel()
        assert w.max() == pytest.approx(2 * MU + LAM * c @ c, rel=1e-10)


def test_small_strain_matches_linear_elasticity(oracle_mod):
    # Section "Lame Coefficients" (Eq. le): near F = I the corotated energy
    # agrees with mu tr(eps^2) + lam/2 tr(eps)^2 to second order.
    rng = np.random.default_rng(8)
    G = rng.standard_normal((3, 3))
    for t in (1e-3, 1e-4):
        F = np.eye(3) + t * G
        eps = 0.5 * (F + F.T) - np.eye(3)
        le = MU * np.trace(eps @ eps) + 0.5 * LAM * np.trace(eps) ** 2
        assert oracle_mod.psi(F, MU, LAM) == pytest.approx(le, rel=20 * t)


def test_modified_hessian_index_order(oracle_mod):
    # Eq. mod_hess_dens with the cofactor det(F) F^{-T} = dJ/dF from numpy.
    rng = np.random.default_rng(9)
    F = _random_F(rng, 1)[0]
    cof = np.linalg.det(F) * np.linalg.inv(F).T
    C = oracle_mod.modified_density_hessian(F, MU, LAM).reshape(3, 3, 3, 3)
    expect = 2 * MU * np.einsum("ab,gd->agbd", np.eye(3), np.eye(3)) + LAM * np.einsum("ag,bd->agbd", cof, cof)
    assert np.allclose(C, expect, rtol=1e-13)
