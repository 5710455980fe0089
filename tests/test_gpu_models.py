"""GPU parity of the Neo-Hookean (Eq. nh) and stable Neo-Hookean (Eq. snh)
sweeps against the FP64 oracle of the same model, through the C ABI."""

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODELS = ["neohookean", "stable_neohookean"]
RES_FLOOR = 1e-5  # relative-residual target of the float32 path


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _u0(p):
    return torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("accel", ["none", "chebyshev", "sor"])
def test_twist_block_200_sweeps(model, accel):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(10, 90.0, 0.3)
    kw = dict(accel=accel, omega=1.5) if accel == "sor" else dict(accel=accel)
    m = Mesh.from_problem(p)
    u = _u0(p)
    rel = m.sweep(u, 200, default_params(model=model, **kw), want_residual=True)
    om = oracle.OracleMesh.from_problem(p, model=model)
    x_ora, st = om.sweeps(p.x0, 200, **kw)
    assert st == 0
    x_gpu = u.cpu().double().numpy() + p.X
    err = np.abs(x_gpu - x_ora).max() / np.abs(x_ora - p.X).max()
    assert err <= 1e-5, err
    rr = om.residual(x_ora) / om.residual(p.x0)
    assert abs(rel[0] - rr) <= 1e-3 * rr + RES_FLOOR


@pytest.mark.parametrize("model", MODELS)
def test_residual_uses_the_model_of_the_last_sweep(model):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(6, 90.0, 0.3)    # large strain: the models' stresses differ
    m = Mesh.from_problem(p)
    u = _u0(p)
    m.sweep(u, 15, default_params(model=model))
    x = u.cpu().double().numpy() + p.X
    r_gpu = m.residual(u)[0]
    r_ora = oracle.OracleMesh.from_problem(p, model=model).residual(x)
    r_cor = oracle.OracleMesh.from_problem(p).residual(x)
    assert abs(r_gpu - r_ora) <= 1e-4 * r_ora + 1e-6 * oracle.OracleMesh.from_problem(p).residual(p.x0)
    assert abs(r_cor - r_ora) > 1e-2 * r_ora   # the models really differ here


@pytest.mark.parametrize("model", MODELS)
def test_solve_reaches_newton_equilibrium_of_the_model(model):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(3, 90.0, 0.3)
    om = oracle.OracleMesh.from_problem(p, model=model)
    xn, it, _ = om.newton(p.x0, 1e-13, 60)
    assert it >= 0
    m = Mesh.from_problem(p)
    u = _u0(p)
    st, sweeps, rel = m.solve(u, RES_FLOOR, 20000, default_params(model=model, accel="chebyshev"))
    assert st == 0 and rel[0] <= RES_FLOOR
    x_gpu = u.cpu().double().numpy() + p.X
    assert np.abs(x_gpu - xn).max() <= 1e-4 * np.abs(xn - p.X).max()


@pytest.mark.parametrize("model", MODELS)
def test_ragged_bar_with_weak_constraints(model):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.contact_bar(3, 4, 7, h=0.1, k_contact=1e6)
    p.body_accel = np.array([0.0, 0.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    m = Mesh.from_problem(p)
    u = _u0(p)
    m.sweep(u, 60, default_params(model=model))
    x_ora, st = oracle.OracleMesh.from_problem(p, model=model).sweeps(p.x0, 60)
    assert st == 0
    x_gpu = u.cpu().double().numpy() + p.X
    assert np.abs(x_gpu - x_ora).max() / np.abs(x_ora - p.X).max() <= 1e-5


def test_direct_and_ring_paths_agree_for_each_model():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(6, 60.0, 0.2)
    for model in MODELS:
        out = []
        for path in (0, 1):
            m = Mesh.from_problem(p)
            u = _u0(p)
            m.sweep(u, 30, default_params(model=model, accel="chebyshev", kernel_path=path))
            out.append(u.cpu().double().numpy())
        assert np.abs(out[0] - out[1]).max() <= 1e-6 * np.abs(out[0]).max()


@pytest.mark.parametrize("model", MODELS)
def test_hessian_apply_and_newton_cg_for_the_model(model):
    """pbng_hessian_apply against the oracle's dense true Hessian of the model,
    and Newton-CG to the oracle's Newton equilibrium of the model."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(3, 60.0, 0.2)
    om = oracle.OracleMesh.from_problem(p, model=model)
    x, st = om.sweeps(p.x0, 4)
    x = x.astype(np.float32).astype(np.float64)
    free = p.dirichlet_mask() == 0
    idx = np.flatnonzero(np.repeat(free, 3))
    H = om.hessian(x)
    d = np.random.default_rng(5).standard_normal(p.X.shape)
    m = Mesh.from_problem(p)
    prm = default_params(model=model)
    hp = m.hessian_apply(_u0_of(x - p.X), _u0_of(d), params=prm).cpu().double().numpy()
    expect = (H[np.ix_(idx, idx)] @ (d * free[:, None]).reshape(-1)[idx]).reshape(-1, 3)
    assert np.abs(hp[free] - expect).max() <= 1e-3 * np.abs(expect).max()
    f = m.force(_u0_of(x - p.X), params=prm).cpu().double().numpy()
    _, r = om.residual(x, vector=True)
    assert np.abs(f[free] - r[free]).max() <= 2e-4 * np.abs(r[free]).max()
    xn, it, _ = om.newton(p.x0, 1e-12, 60)
    assert it >= 0
    u = _u0(p)
    st, info = m.newton_cg(u, 1e-5, max_newton=60, max_cg=2000, cg_tol=1e-2, params=prm)
    assert st == 0
    assert np.abs(u.cpu().double().numpy() + p.X - xn).max() <= 1e-4 * np.abs(xn - p.X).max()


def _u0_of(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()
