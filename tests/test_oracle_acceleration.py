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


def _sweep_jacobian(om, xs, dofs, order):
    n = len(dofs)
    B = np.zeros((n, n))
    h = 1e-6
    for c, (i, a) in enumerate(dofs):
        xp, xm = xs.copy(), xs.copy()
        xp[i, a] += h
        xm[i, a] -= h
        yp, _ = om.sweeps(xp, 1, order=order)
        ym, _ = om.sweeps(xm, 1, order=order)
        B[:, c] = np.array([(yp[j, b] - ym[j, b]) / (2 * h) for (j, b) in dofs])
    return B


@pytest.fixture(scope="module")
def equilibrium(oracle_mod):
    p = W.gravity_sag(3, young=1e4)
    om = oracle_mod.OracleMesh.from_problem(p)
    xs, it, _ = om.newton(p.x0, 1e-14, 60)
    assert it >= 0
    free = np.flatnonzero(p.dirichlet_mask() == 0)
    dofs = [(i, a) for i in free for a in range(3)]
    return p, om, xs, dofs


@pytest.fixture(scope="module")
def linearised(equilibrium):
    p, om, xs, dofs = equilibrium
    return p, om, xs, dofs, _sweep_jacobian(om, xs, dofs, "forward")


@pytest.fixture(scope="module")
def linearised_symmetric(equilibrium):
    p, om, xs, dofs = equilibrium
    return p, om, xs, dofs, _sweep_jacobian(om, xs, dofs, "symmetric")


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


def _free_hessian(om, xs, dofs):
    H = om.hessian(xs)
    idx = [3 * i + a for (i, a) in dofs]
    return H[np.ix_(idx, idx)]


def test_symmetric_sweep_is_self_adjoint_with_spectrum_in_unit_interval(linearised, linearised_symmetric):
    """Linearised at the equilibrium, the update of colour c is
    T_c = I - E_c A_c^{-1} E_c^T H (A_c the SPD nodal Hessians of Eq. mod_hess,
    H the true Hessian): each T_c is self-adjoint in the H inner product, so
    the palindromic product T_0 ... T_{C-1} ... T_0 of the symmetric order is
    too, i.e. H B is a symmetric matrix and B has a real spectrum; the
    ascending order's product is not.  At this near-rest equilibrium the
    modified Hessian dominates the true diagonal blocks, which puts the
    spectrum in [0, 1)."""
    p, om, xs, dofs, Bs = linearised_symmetric
    Bf = linearised[4]
    H = _free_hessian(om, xs, dofs)
    HB = H @ Bs
    assert np.abs(HB - HB.T).max() <= 1e-6 * np.abs(HB).max()
    HBf = H @ Bf
    assert np.abs(HBf - HBf.T).max() > 1e-2 * np.abs(HBf).max()
    ev = np.linalg.eigvals(Bs)
    assert np.abs(ev.imag).max() <= 1e-6
    assert ev.real.min() >= -1e-6
    assert 0.05 < ev.real.max() < 1.0
    # the forward order's spectrum has complex pairs
    assert np.abs(np.linalg.eigvals(Bf).imag).max() > 1e-3


def test_symmetric_sweep_is_the_forward_sweep_then_the_reverse_pass(linearised_symmetric, oracle_mod):
    """One symmetric sweep from x equals, to first order around the
    equilibrium, the ascending pass followed by the descending colours
    C-2..0: checked through the linear maps, B_s = R B_f with R the Jacobian
    of the descending passes, which is itself the product of the single-colour
    maps T_c = I - E_c A_c^{-1} E_c^T H built from the oracle's own local
    systems (Eq. pbgn_dx)."""
    p, om, xs, dofs, Bs = linearised_symmetric
    H = _free_hessian(om, xs, dofs)
    pos = {d: k for k, d in enumerate(dofs)}
    colours = om.colours()
    n = len(dofs)
    T = []
    for c in range(om.ncolours):
        M = np.zeros((n, n))
        for i in np.flatnonzero(colours == c):
            _, A = om.local_system(xs, i)
            k = [pos[(i, a)] for a in range(3)]
            M[np.ix_(k, k)] = np.linalg.inv(A)
        T.append(np.eye(n) - M @ H)
    C = len(T)
    seq = list(range(C)) + list(range(C - 2, -1, -1))
    B = np.eye(n)
    for c in seq:
        B = T[c] @ B
    assert np.abs(B - Bs).max() <= 1e-5 * np.abs(Bs).max()


def _chebyshev_expected(B, e0, rho, gamma):
    n = len(e0)
    Bp = gamma * B + (1.0 - gamma) * np.eye(n)
    y0 = Bp @ e0
    Tm, T = y0, (Bp / rho) @ y0
    tm, t = 1.0, 1.0 / rho
    expected = {1: y0, 2: T / t}
    for k in range(2, 9):
        Tm, T = T, 2.0 * (Bp / rho) @ T - Tm
        tm, t = t, 2.0 * t / rho - tm
        expected[k + 1] = T / t
    return expected


@pytest.mark.parametrize("rho,gamma", [(0.9, 1.7), (0.97, 1.7)])
def test_symmetric_order_chebyshev_error_is_the_scaled_chebyshev_polynomial(linearised_symmetric, rho, gamma):
    p, om, xs, dofs, B = linearised_symmetric
    x0, e0 = _start(xs, dofs, 13)
    expected = _chebyshev_expected(B, e0, rho, gamma)
    for l in range(1, 10):
        x, st = om.sweeps(x0, l, accel="chebyshev", rho=rho, gamma=gamma, order="symmetric")
        assert st == 0
        e = _err(x, xs, dofs)
        assert np.abs(e - expected[l]).max() <= 1e-5 * np.abs(expected[l]).max() + 1e-13, l


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
