"""The symmetric colour order (pbng_params.colour_order) on the GPU against
the oracle's symmetric sweep, and its automatic-rho schedule.

One symmetric sweep runs the colour passes 0..C-1 and then C-2..0 (Section
"Coloring and Parallelism" leaves the order of the colour loop open).  The
oracle pins that this sweep, linearised at an equilibrium, is self-adjoint
in the Hessian's inner product with a real spectrum in [0, 1), which is what
the Chebyshev weights of Section "Acceleration Techniques" assume."""

import numpy as np
import pytest

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


def _u0(p):
    return torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("accel,kw", [("none", {}), ("chebyshev", dict(rho=0.95, gamma=1.7)),
                                      ("sor", dict(omega=1.5))])
def test_symmetric_twist_200_sweeps_match_the_oracle(oracle_mod, accel, kw):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(10, 90.0, 0.3)
    om = oracle_mod.OracleMesh.from_problem(p)
    m = Mesh.from_problem(p)
    u = _u0(p)
    rel = m.sweep(u, 200, default_params(accel=accel, colour_order="symmetric", **kw), want_residual=True)[0]
    xo, st = om.sweeps(p.x0, 200, accel=accel, order="symmetric", threads=4, **kw)
    assert st == 0
    x = u.cpu().double().numpy() + p.X
    err = np.abs(x - xo).max() / np.abs(xo - p.X).max()
    assert err <= 1e-5, err
    r_ora = om.residual(xo) / om.residual(p.x0)
    assert abs(rel - r_ora) <= 1e-3 * r_ora + 2e-6, (rel, r_ora)


def test_symmetric_auto_rho_schedule_replays_on_the_oracle(oracle_mod):
    """The solve's recorded schedule (plain sweeps, then Chebyshev restarts
    with the rho of each) run on the oracle gives the same iterate."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(10)
    om = oracle_mod.OracleMesh.from_problem(p)
    m = Mesh.from_problem(p)
    u = _u0(p)
    total = 700
    st, sweeps, rel = m.solve(u, 0.0, total, default_params(accel="chebyshev", rho=-1.0,
                                                            colour_order="symmetric"), raise_on_status=False)
    assert sweeps == total
    info = m.solve_info()
    ev_s, ev_r = info["event_sweep"], info["event_rho"]
    assert info["nevents"] >= 1 and ev_s[0] == info["estimate_sweeps"] == 30
    assert ev_r[0] == pytest.approx(min(1 - 1e-6, max(0.5, 1 - 1.7 * (1 - info["plain_rate"]))), abs=1e-15)
    assert all(b > a for a, b in zip(ev_s, ev_s[1:]))
    x = p.x0.copy()
    x, s0 = om.sweeps(x, ev_s[0], order="symmetric", threads=4)
    bounds = ev_s + [total]
    for k, rho in enumerate(ev_r):
        n = bounds[k + 1] - bounds[k]
        if n > 0:
            acc = "chebyshev" if rho > 0 else "none"
            x, s1 = om.sweeps(x, n, accel=acc, rho=rho, gamma=1.7, order="symmetric", threads=4)
            assert s1 == 0
    xg = u.cpu().double().numpy() + p.X
    err = np.abs(xg - x).max() / np.abs(x - p.X).max()
    assert err <= 1e-5, err


def test_symmetric_order_converges_where_the_forward_order_crawls():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(16)
    m = Mesh.from_problem(p)
    res = {}
    for order in ("forward", "symmetric"):
        u = _u0(p)
        st, sweeps, rel = m.solve(u, 1e-4, 6000, default_params(accel="chebyshev", rho=-1.0, colour_order=order),
                                  raise_on_status=False)
        res[order] = (st, sweeps)
    assert res["symmetric"][0] == 0
    # a symmetric sweep is 2C - 1 = 9 passes against 5
    assert res["symmetric"][1] * 9 < 0.5 * res["forward"][1] * 5 or res["forward"][0] != 0, res
