"""EquilibriumModel (torch.autograd.Function over pbng_solve / pbng_adjoint):
gradients of L = |x_top - target|^2 with respect to per-tet log E and the
clamped positions, against the oracle's dense adjoint and against central
finite differences of GPU solves along random directions."""

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# The model's adjoint is refined with the float-float force (past the float32
# sweeps' floor near 1e-5 on these blocks).
ADJ_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _setup(n=4, seed=21):
    p = W.adjoint_block(n)
    xd, acc = W.adjoint_load_cases(p, count=1, seed=seed)
    p.x0 = p.X.copy()
    p.x0[p.dirichlet] = xd[0]
    p.body_accel = acc[0]
    rng = np.random.default_rng(seed)
    log_e = np.log(1e5) + 0.2 * rng.standard_normal(p.ne)
    top = np.flatnonzero(np.isclose(p.X[:, 2], 1.0))
    target = p.X[top] + np.array([0.0, 0.0, -0.01]) + 0.005 * rng.standard_normal((len(top), 3))
    return p, log_e, xd[0], top, target


def _loss(model, p, log_e, xd, top, target):
    le = torch.tensor(log_e, dtype=torch.float64, device="cuda", requires_grad=True)
    xdt = torch.tensor(xd, dtype=torch.float64, device="cuda", requires_grad=True)
    u = model(le, xdt)
    x_top = u[top].double() + torch.tensor(p.X[top], device="cuda")
    L = ((x_top - torch.tensor(target, device="cuda")) ** 2).sum()
    return L, le, xdt


@pytest.mark.parametrize("energy", ["corotated", "neohookean", "stable_neohookean"])
def test_autograd_matches_dense_oracle_adjoint(oracle_mod, energy):
    from paper_2306_09021_gb300 import EquilibriumModel
    p, log_e, xd, top, target = _setup()
    model = EquilibriumModel(p, rel_tol=1e-6, model=energy, adjoint_tol=ADJ_TOL)
    L, le, xdt = _loss(model, p, log_e, xd, top, target)
    L.backward()
    # oracle: same log E and boundary, Newton equilibrium, dense adjoint
    q = W.adjoint_block(4)
    q.young = np.exp(log_e)
    q.body_accel = p.body_accel
    q.x0 = p.x0
    om = oracle_mod.OracleMesh.from_problem(q, model=energy)
    xeq, it, _ = om.newton(q.x0, 1e-12, 60)
    assert it >= 0
    dLdx = np.zeros_like(xeq)
    dLdx[top] = 2.0 * (xeq[top] - target)
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)
    gE = le.grad.cpu().numpy()
    gD = xdt.grad.cpu().numpy()
    assert np.abs(gE - dE_ref).max() <= 2e-3 * np.abs(dE_ref).max()
    assert np.abs(gD - dD_ref).max() <= 2e-3 * np.abs(dD_ref).max()


def test_autograd_matches_finite_differences():
    from paper_2306_09021_gb300 import EquilibriumModel
    p, log_e, xd, top, target = _setup(n=4, seed=5)
    model = EquilibriumModel(p, rel_tol=1e-6, max_sweeps=30000, adjoint_tol=ADJ_TOL)
    L, le, xdt = _loss(model, p, log_e, xd, top, target)
    L.backward()
    gE, gD = le.grad.cpu().numpy(), xdt.grad.cpu().numpy()
    rng = np.random.default_rng(1)
    h = 1.0 / 4
    for k in range(16):   # 16 random directions in (log E, x_D)
        dE = rng.standard_normal(p.ne)
        dD = rng.standard_normal(xd.shape)
        epsE, epsD = 1e-3, 1e-4 * h
        vals = []
        for sgn in (1.0, -1.0):
            Ls, _, _ = _loss(model, p, log_e + sgn * epsE * dE, xd + sgn * epsD * dD, top, target)
            vals.append(Ls.item())
        # directional derivative along (epsE dE, epsD dD) with step 1
        fd = (vals[0] - vals[1]) / 2.0
        an = epsE * (gE @ dE) + epsD * np.sum(gD * dD)
        assert fd == pytest.approx(an, rel=2e-2, abs=1e-3 * abs(an) + 1e-12)


def test_unconverged_solves_raise_unless_allowed():
    """A forward or adjoint solve that stops at its sweep limit gives no
    equilibrium gradient: the autograd function raises, or warns with the
    residual reached when the model allows it."""
    from paper_2306_09021_gb300 import EquilibriumModel
    from paper_2306_09021_gb300.autograd import NotConvergedError
    p, log_e, xd, top, target = _setup(n=4, seed=7)
    model = EquilibriumModel(p, rel_tol=1e-9, max_sweeps=20)
    with pytest.raises(NotConvergedError, match="relative residual"):
        _loss(model, p, log_e, xd, top, target)
    model = EquilibriumModel(p, rel_tol=1e-6, max_sweeps=30000, adjoint_tol=1e-9, adjoint_max_sweeps=5)
    L, le, xdt = _loss(model, p, log_e, xd, top, target)
    assert model.last_solve[0] == 0
    with pytest.raises(NotConvergedError, match="adjoint"):
        L.backward()
    model = EquilibriumModel(p, rel_tol=1e-9, max_sweeps=20, allow_unconverged=True)
    with pytest.warns(RuntimeWarning, match="relative residual"):
        L, le, xdt = _loss(model, p, log_e, xd, top, target)
    assert model.last_solve[0] == 7


def _smooth(points, rng, k=2.0 * np.pi):
    """A smooth random field on points: a sum of two random plane waves."""
    out = np.zeros(len(points))
    for _ in range(2):
        kv = rng.standard_normal(3)
        kv *= k / np.linalg.norm(kv)
        out += np.sin(points @ kv + rng.uniform(0.0, 2.0 * np.pi))
    return out


def test_full_size_gradients_match_finite_differences():
    """One load case of the adjoint workload at full size (48^3 cells,
    552,960 tets): autograd's dL/d(log E) and dL/dx_D at the equilibrium,
    from the refined coloured Gauss-Seidel adjoint, against central
    differences of extended-precision forward solves along 4 smooth random
    directions in (log E, x_D)."""
    from paper_2306_09021_gb300 import EquilibriumModel
    p, log_e, xd, top, target = _setup(n=48, seed=5)
    model = EquilibriumModel(p, rel_tol=1e-9, max_sweeps=40000, adjoint_tol=1e-6, adjoint_max_sweeps=40000)
    L, le, xdt = _loss(model, p, log_e, xd, top, target)
    assert model.last_solve[0] == 0
    L.backward()
    assert model.last_adjoint[0] == 0
    gE, gD = le.grad.cpu().numpy(), xdt.grad.cpu().numpy()
    rng = np.random.default_rng(3)
    cent = p.X[p.tets].mean(axis=1)
    Xd = p.X[p.dirichlet]
    h = 1.0 / 48
    for k in range(4):
        dE = _smooth(cent, rng)
        dD = np.stack([_smooth(Xd, rng) for _ in range(3)], axis=1)
        epsE, epsD = 3e-3, 3e-2 * h
        vals = []
        for sgn in (1.0, -1.0):
            Ls, _, _ = _loss(model, p, log_e + sgn * epsE * dE, xd + sgn * epsD * dD, top, target)
            assert model.last_solve[0] == 0
            vals.append(Ls.item())
        fd = (vals[0] - vals[1]) / 2.0
        an = epsE * (gE @ dE) + epsD * np.sum(gD * dD)
        print(f"48^3 direction {k}: finite difference {fd:.6e}, adjoint {an:.6e}")
        assert fd == pytest.approx(an, rel=1e-2)
