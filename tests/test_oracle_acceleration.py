"""Pins of the oracle's acceleration steps (Section "Acceleration
Techniques") against linear-iteration theory, independent of the update
formulas they implement.

Near the equilibrium x* one plain PBNG sweep is the linear map
x -> x* + B (x - x*) up to second order, with B its Jacobian (taken here by
central differences of the oracle's plain sweep).  An acceleration applied
after every sweep then moves the error e = x - x* by a linear recurrence
whose solution is known in closed form:

* Chebyshev, x^{l+1} = w_{l+1} (g (x_P - x^l) + x^l - x^{l-1}) + x^{l-1},
  with two plain sweeps first and then the weights 2/(2 - rho^2),
  4/(4 - rho^2 w): the Chebyshev semi-iterative method (Golub & Varga 1961)
  started after the first sweep.  With B' = g B + (1 - g) I its error is
  e_l = P_{l-1}(B') B' e_0, where P_k(t) = T_k(t / rho) / T_k(1 / rho) and
  T_k are the Chebyshev polynomials of the first kind (T_0 = 1, T_1 = t,
  T_{k+1} = 2 t T_k - T_{k-1}).
* SOR as printed, x^{l+1} = w (x_P - x^{l-1}) + x^{l-1} with x^{-1} = x^0:
  e_{l+1} = w B e_l + (1 - w) e_{l-1}.  Along an eigenvector of B with
  eigenvalue b this is s_{l+1} = w b s_l + (1 - w) s_{l-1}, solved by the
  roots of z^2 - w b z - (1 - w) = 0.

A wrong weight index, a misplaced g or a swapped iterate changes e_l at
first order and fails these checks."""

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def linearised(oracle_mod):
    p = W.gravity_sag(3, young=1e4)
    om = oracle_mod.OracleMesh.from_problem(p)
    xs, it, _ = om.newton(p.x0, 1e-14, 60)
    assert it >= 0
    free = np.flatnonzero(p.dirichlet_mask() == 0)
    dofs = [(i, a) for i in free for a in range(3)]
    n = len(dofs)
    B = np.zeros((n, n))
    h = 1e-6
    for c, (i, a) in enumerate(dofs):
        xp, xm = xs.copy(), xs.copy()
        xp[i, a] += h
        xm[i, a] -= h
        yp, _ = om.sweeps(xp, 1)
        ym, _ = om.sweeps(xm, 1)
        B[:, c] = np.array([(yp[j, b] - ym[j, b]) / (2 * h) for (j, b) in dofs])
    return p, om, xs, dofs, B


def _err(x, xs, dofs):
    return np.array([x[i, a] - xs[i, a] for (i, a) in dofs])


def _start(xs, dofs, seed, scale=1e-7):
    rng = np.random.default_rng(seed)
    e0 = scale * rng.standard_normal(len(dofs))
    x0 = xs.copy()
    for c, (i, a) in enumerate(dofs):
        x0[i, a] += e0[c]
    return x0, e0


def test_plain_sweep_is_a_contraction_with_gauss_seidel_structure(linearised):
    p, om, xs, dofs, B = linearised
    rho_b = np.max(np.abs(np.linalg.eigvals(B)))
    assert 0.05 < rho_b < 1.0                      # converging, and not trivially exact
    assert np.abs(B - B.T).max() > 1e-3 * np.abs(B).max()   # Gauss-Seidel, not Jacobi


@pytest.mark.parametrize("rho,gamma", [(0.9, 1.0), (0.95, 1.7), (0.8, 1.3)])
def test_chebyshev_error_is_the_scaled_chebyshev_polynomial(linearised, rho, gamma):
    p, om, xs, dofs, B = linearised
    x0, e0 = _start(xs, dofs, 11)
    n = len(dofs)
    Bp = gamma * B + (1.0 - gamma) * np.eye(n)
    y0 = Bp @ e0
    # T_k(Bp / rho) y0 and T_k(1 / rho) by their own recurrence
    Tm, T = y0, (Bp / rho) @ y0
    tm, t = 1.0, 1.0 / rho
    expected = {1: y0, 2: T / t}
    for k in range(2, 9):
        Tm, T = T, 2.0 * (Bp / rho) @ T - Tm
        tm, t = t, 2.0 * t / rho - tm
        expected[k + 1] = T / t
    for l in range(1, 10):
        x, st = om.sweeps(x0, l, accel="chebyshev", rho=rho, gamma=gamma)
        assert st == 0
        e = _err(x, xs, dofs)
        assert np.abs(e - expected[l]).max() <= 1e-5 * np.abs(expected[l]).max() + 1e-13, l


@pytest.mark.parametrize("omega", [0.7, 1.3, 1.6])
def test_sor_error_follows_the_two_step_recurrence_closed_form(linearised, omega):
    p, om, xs, dofs, B = linearised
    x0, e0 = _start(xs, dofs, 12)
    lam, V = np.linalg.eig(B)
    c0 = np.linalg.solve(V, e0.astype(complex))
    for l in range(1, 9):
        # s_{-1} = s_0 = c0, s_{l+1} = w b s_l + (1 - w) s_{l-1}: roots z1, z2
        disc = np.sqrt((omega * lam) ** 2 + 4.0 * (1.0 - omega) + 0j)
        z1, z2 = (omega * lam + disc) / 2.0, (omega * lam - disc) / 2.0
        # s_m = A z1^m + C z2^m fitted to s_{-1} = s_0 = c0
        A = c0 * (1.0 - 1.0 / z2) / (1.0 / z1 - 1.0 / z2)
        C = c0 - A
        s = A * z1 ** l + C * z2 ** l
        expected = np.real(V @ s)
        x, st = om.sweeps(x0, l, accel="sor", omega=omega)
        assert st == 0
        e = _err(x, xs, dofs)
        assert np.abs(e - expected).max() <= 1e-5 * np.abs(expected).max() + 1e-13, l
