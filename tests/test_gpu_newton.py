"""The GPU Newton-CG reference solver and its building blocks (pbng_force,
pbng_hessian_apply) against the FP64 oracle: its residual vector, its dense
true Hessian (Eq. hess) and its dense Newton solve."""

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def _state(p, sweeps=4):
    om = oracle.OracleMesh.from_problem(p)
    x, st = om.sweeps(p.x0, sweeps)
    assert st == 0
    return om, x.astype(np.float32).astype(np.float64)   # representable in float32


def _loaded():
    p = W.twist_block(4, 90.0, 0.3)
    p.body_accel = np.array([0.2, 0.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    return p


def test_force_matches_the_oracle_residual_vector():
    from paper_2306_09021_gb300 import Mesh
    p = _loaded()
    om, x = _state(p)
    m = Mesh.from_problem(p)
    f = m.force(_t(x - p.X)).cpu().double().numpy()
    _, r = om.residual(x, vector=True)
    free = p.dirichlet_mask() == 0
    assert np.abs(f[~free]).max() == 0.0
    assert np.abs(f[free] - r[free]).max() <= 2e-4 * np.abs(r[free]).max()


def test_hessian_apply_matches_the_dense_oracle_hessian():
    from paper_2306_09021_gb300 import Mesh
    p = W.twist_block(3, 60.0, 0.2)
    om, x = _state(p)
    m = Mesh.from_problem(p)
    free = p.dirichlet_mask() == 0
    H = om.hessian(x)
    idx = np.flatnonzero(np.repeat(free, 3))
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal(p.X.shape)
        hp = m.hessian_apply(_t(x - p.X), _t(d)).cpu().double().numpy()
        dfree = (d * free[:, None]).reshape(-1)
        expect = (H[np.ix_(idx, idx)] @ dfree[idx]).reshape(-1, 3)
        assert np.abs(hp[~free]).max() == 0.0
        assert np.abs(hp[free] - expect).max() <= 1e-3 * np.abs(expect).max()


# The relative-residual floor of the float32 force evaluation is about 7e-6
# on the 6^3 sag cube, so that case stops at 3e-5.
@pytest.mark.parametrize("maker,tol", [(lambda: W.twist_block(4, 90.0, 0.3), 1e-5), (lambda: W.gravity_sag(6), 3e-5)])
def test_newton_cg_reaches_the_oracle_newton_equilibrium(maker, tol):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = maker()
    om = oracle.OracleMesh.from_problem(p)
    xn, it, _ = om.newton(p.x0, 1e-12, 60)   # the sag cube's FP64 floor is near 1.5e-13
    assert it >= 0
    m = Mesh.from_problem(p)
    u = _t(p.x0 - p.X)
    st, info = m.newton_cg(u, tol, max_newton=60, max_cg=2000, cg_tol=1e-2, params=default_params())
    assert st == 0 and info["rel_residual"] <= tol
    assert 1 <= info["newton_iterations"] <= 60 and info["cg_iterations"] >= info["newton_iterations"]
    x_gpu = u.cpu().double().numpy() + p.X
    assert np.abs(x_gpu - xn).max() <= 1e-4 * np.abs(xn - p.X).max()
    # the residual of the result, measured by the sweep library, agrees
    r = m.residual(u)[0] / oracle.OracleMesh.from_problem(p).residual(p.x0)
    assert r <= 2 * tol


def test_newton_cg_argument_errors():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.twist_block(3, 30.0, 0.1)
    m = Mesh.from_problem(p)
    u = _t(p.x0 - p.X)
    with pytest.raises(PbngError):
        m.newton_cg(u, 1e-5, params=default_params(kernel_path=1))
    with pytest.raises(PbngError):
        m.newton_cg(u, 1e-5, cg_tol=0.0)
