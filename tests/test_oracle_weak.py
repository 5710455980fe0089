"""Pins of the oracle's general weak constraints (Section "Weak Constraints":
C_c(y) = sum_j w0_cj y_j - sum_j w1_cj y_j, energy (1/2) C^T K_c C) and of the
incremental recolouring of Section "Collision Coloring":

* residual = -gradient of the energy with the constraints, dense Hessian =
  derivative of the residual;
* the colouring is valid with constraints treated like elements and equals a
  brute-force greedy colouring; incremental recolouring is valid, leaves
  every node off the constraints untouched and keeps any colour still valid;
* physics: at equilibrium the constraints carry exactly the weight of the
  hanging block (global force balance), and PBNG reaches the Newton
  equilibrium."""

import numpy as np
import pytest

import workloads as W


def _two_blocks(k=1e5, n_top=3, n_bottom=2):
    p = W.two_blocks_hanging(n_top, n_bottom, k=k)
    return p, p.meta["weak"]


def _mesh(oracle_mod, p, weak, recolour=False):
    m = oracle_mod.OracleMesh.from_problem(p)
    m.set_weak_constraints(*weak, recolour=recolour)
    return m


def _neighbours(p, weak):
    nb = [set() for _ in range(p.nv)]
    for t in p.tets:
        for a in t:
            nb[a].update(int(b) for b in t if b != a)
    idx = weak[0]
    for row in idx:
        vs = [int(v) for v in row if v >= 0]
        for a in vs:
            nb[a].update(b for b in vs if b != a)
    return nb


def test_residual_is_minus_energy_gradient_with_constraints(oracle_mod):
    p, weak = _two_blocks()
    m = _mesh(oracle_mod, p, weak)
    rng = np.random.default_rng(2)
    free = p.dirichlet_mask() == 0
    x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape) * free[:, None]
    _, r = m.residual(x, vector=True)
    bound = sorted({int(v) for v in weak[0].reshape(-1) if v >= 0 and free[v]})
    h = 1e-7
    for i in bound[:6]:
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (m.energy(xp) - m.energy(xm)) / (2 * h)
            assert -g == pytest.approx(r[i, a], rel=1e-6, abs=1e-6 * np.abs(r).max())


def test_dense_hessian_is_residual_derivative_with_constraints(oracle_mod):
    p, weak = _two_blocks(n_top=2, n_bottom=1)
    m = _mesh(oracle_mod, p, weak)
    rng = np.random.default_rng(5)
    x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape) * (p.dirichlet_mask() == 0)[:, None]
    H = m.hessian(x)
    d = rng.standard_normal(p.x0.shape) * (p.dirichlet_mask() == 0)[:, None]
    h = 1e-6
    _, rp = m.residual(x + h * d, vector=True)
    _, rm = m.residual(x - h * d, vector=True)
    fd = -(rp - rm) / (2 * h)
    free = np.repeat(p.dirichlet_mask() == 0, 3)
    got = (H @ d.reshape(-1))[free]
    assert np.allclose(got, fd.reshape(-1)[free], rtol=1e-6, atol=1e-6 * np.abs(got).max())


def test_colouring_with_constraints_is_valid_and_greedy(oracle_mod):
    p, weak = _two_blocks()
    m = _mesh(oracle_mod, p, weak)
    col = m.colours()
    nb = _neighbours(p, weak)
    free = p.dirichlet_mask() == 0
    for i in np.flatnonzero(free):
        assert all(col[j] != col[i] for j in nb[i] if free[j])
    # brute-force greedy: ascending ids, least colour unused by coloured neighbours
    ref = np.full(p.nv, -1)
    for i in np.flatnonzero(free):
        used = {ref[j] for j in nb[i] if ref[j] >= 0}
        c = 0
        while c in used:
            c += 1
        ref[i] = c
    assert np.array_equal(col, ref)
    assert m.ncolours > oracle_mod.OracleMesh.from_problem(p).ncolours   # the bindings couple the blocks


def test_incremental_recolouring(oracle_mod):
    p, weak = _two_blocks()
    m = oracle_mod.OracleMesh.from_problem(p)
    before = m.colours()
    m.set_weak_constraints(*weak, recolour=True)
    after = m.colours()
    nb = _neighbours(p, weak)
    free = p.dirichlet_mask() == 0
    on = np.zeros(p.nv, bool)
    on[[v for v in weak[0].reshape(-1) if v >= 0]] = True
    for i in np.flatnonzero(free):
        assert all(after[j] != after[i] for j in nb[i] if free[j])
        if not on[i]:
            assert after[i] == before[i]
    # adding constraints again that are already satisfied by the colouring changes nothing
    m.set_weak_constraints(*weak, recolour=True)
    assert np.array_equal(m.colours(), after)
    # a node whose old colour stays valid keeps it
    for i in np.flatnonzero(free & on):
        if all(before[i] != after[j] for j in nb[i] if free[j] and j != i):
            assert after[i] == before[i]


def test_constraints_carry_the_weight_of_the_hanging_block(oracle_mod):
    p, weak = _two_blocks()
    m = _mesh(oracle_mod, p, weak)
    xn, it, _ = m.newton(p.x0, 1e-11, 80)
    assert it >= 0
    idx, w, kn, kt, nrm = weak
    side0 = (w[:, :4, None] * xn[np.where(idx[:, :4] < 0, 0, idx[:, :4])]).sum(1)
    side1 = (w[:, 4:, None] * xn[np.where(idx[:, 4:] < 0, 0, idx[:, 4:])]).sum(1)
    force_on_bottom = -(kn[:, None] * (side0 - side1)).sum(0)   # isotropic K = k I
    na = W.box_grid(3, 3, 3, 1.0)[0].shape[0]
    B, V, mu, lam = m.tet_constants()
    weight = (p.density * V)[np.any(p.tets >= na, axis=1)].sum() * 9.8
    assert np.allclose(force_on_bottom, [0.0, 0.0, weight], rtol=1e-8, atol=1e-8 * weight)
    assert np.abs(side0 - side1).max() < 1e-2          # the binding holds


@pytest.mark.parametrize("accel", ["none", "chebyshev"])
def test_pbng_reaches_the_newton_equilibrium_with_constraints(oracle_mod, accel):
    p, weak = _two_blocks(n_top=2, n_bottom=2, k=3e4)
    m = _mesh(oracle_mod, p, weak)
    xn, it, _ = m.newton(p.x0, 1e-11, 80)
    assert it >= 0
    xs, st, hist = m.sweeps(p.x0, 20000 if accel == "none" else 4000, accel=accel, history=True)
    assert st == 0 and hist[-1] <= 1e-8 * hist[0]
    assert np.abs(xs - xn).max() <= 1e-7 * np.abs(xn - p.X).max()
