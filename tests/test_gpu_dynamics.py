"""Backward-Euler time steps (Eq. fem_be) on the GPU: pbng_set_inertia,
pbng_step and pbng_set_dirichlet_targets, against the closed-form free fall
and the FP64 oracle's step loop."""

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


def test_free_fall_matches_the_backward_euler_recurrence():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(4, 0.0, 0.0)
    p.dirichlet = np.zeros(0, np.int32)
    p.body_accel = np.array([0.5, -1.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    m = Mesh.from_problem(p)
    dt = 1e-2
    m.set_inertia(dt, p.density)
    v0 = np.array([0.3, 0.1, -0.2])
    u = _t(np.zeros_like(p.X))
    u_prev = _t(np.tile(-dt * v0, (p.nv, 1)))
    for n in range(1, 11):
        m.step(u, u_prev, 20, default_params())
        expect = n * dt * v0 + dt * dt * p.body_accel * n * (n + 1) / 2
        got = u.cpu().double().numpy()
        assert np.abs(got - expect).max() <= 1e-5 * np.abs(expect).max(), n
        prev = (n - 1) * dt * v0 + dt * dt * p.body_accel * (n - 1) * n / 2
        assert np.abs(u_prev.cpu().double().numpy() - prev).max() <= 1e-5 * np.abs(expect).max()


def _released_twist():
    p = W.twist_block(5, 60.0, 0.2)
    bottom = np.flatnonzero(np.isclose(p.X[:, 2], 0.0)).astype(np.int32)
    p.dirichlet = bottom                      # the top face is let go
    p.body_accel = np.array([0.0, 0.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    return p


@pytest.mark.parametrize("accel", ["none", "chebyshev"])
def test_released_twist_matches_the_oracle_step_loop(accel):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _released_twist()
    dt, steps, sweeps = 1e-2, 5, 40
    m = Mesh.from_problem(p)
    m.set_inertia(dt, p.density)
    u = _t(p.x0 - p.X)
    u_prev = u.clone()                        # released at rest
    for _ in range(steps):
        m.step(u, u_prev, sweeps, default_params(accel=accel))
    om = oracle.OracleMesh.from_problem(p)
    free = p.dirichlet_mask() == 0
    x_prev, x = p.x0.copy(), p.x0.copy()
    for _ in range(steps):
        xhat = 2 * x - x_prev
        om.set_inertia(dt, p.density, xhat)
        guess = x.copy()
        guess[free] = xhat[free] + dt * dt * p.body_accel   # f_ext / m_ii = body acceleration
        x_new, st = om.sweeps(guess, sweeps, accel=accel)
        assert st == 0
        x_prev, x = x, x_new
    x_gpu = u.cpu().double().numpy() + p.X
    err = np.abs(x_gpu - x).max() / np.abs(x - p.x0).max()
    assert err <= 1e-4, err
    assert np.abs(x - p.x0).max() > 1e-3          # the block really moved


def test_step_to_a_tolerance():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _released_twist()
    m = Mesh.from_problem(p)
    m.set_inertia(5e-3, p.density)
    u = _t(p.x0 - p.X)
    u_prev = u.clone()
    for _ in range(3):
        st, sweeps, rel = m.step(u, u_prev, 5000, default_params(accel="chebyshev"), rel_tol=1e-5)
        assert st == 0 and rel[0] <= 1e-5 and 0 < sweeps < 5000


def test_dirichlet_targets_update_without_relayout():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(5, 30.0, 0.1)
    q = W.twist_block(5, 75.0, 0.25)
    m = Mesh.from_problem(p)
    u = _t(p.x0 - p.X)
    m.sweep(u, 5, default_params())
    m.set_dirichlet_targets(q.x0[q.dirichlet])
    u1 = _t(q.x0 - q.X)
    m.sweep(u1, 25, default_params(accel="chebyshev"))
    ref = Mesh.from_problem(q)
    u2 = _t(q.x0 - q.X)
    ref.sweep(u2, 25, default_params(accel="chebyshev"))
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)


def test_step_argument_errors():
    from paper_2306_09021_gb300 import Mesh, PbngError
    p = W.twist_block(3, 30.0, 0.1)
    m = Mesh.from_problem(p)
    u = _t(p.x0 - p.X)
    with pytest.raises(PbngError):
        m.step(u, u.clone(), 5)                   # no pbng_set_inertia yet
    with pytest.raises(PbngError):
        m.set_inertia(1e-2, None)                 # densities required
    with pytest.raises(PbngError):
        m.set_inertia(1e-2, np.zeros(p.ne))
    m.set_inertia(1e-2, np.full(p.ne, 1000.0))
    m.step(u, u.clone(), 5)
    m.set_inertia(0.0)                            # back to quasistatics
    with pytest.raises(PbngError):
        m.step(u, u.clone(), 5)
