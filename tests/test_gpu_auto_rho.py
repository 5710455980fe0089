"""Chebyshev acceleration with rho estimated from the FP64 residual checks
(pbng_solve with rho <= 0).

Section "Acceleration Techniques" takes rho as a spectral-radius estimate of
the plain iteration.  The library measures the plain per-sweep contraction
q, runs Chebyshev with rho = clamp(1 - 2 (1 - q), 0.5, 0.98) restarted at
the current iterate, and backs rho off when a residual check grows.  These
tests pin the schedule against the oracle (plain sweeps, then the printed
Chebyshev update from a fresh history with that rho) and check that the
estimate pays off."""

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


def _u0(p):
    return torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")


def test_auto_rho_follows_plain_then_chebyshev_of_the_oracle():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(8)
    m = Mesh.from_problem(p)
    u = _u0(p)
    extra = 60
    st, sweeps, rel = m.solve(u, 0.0, 30 + extra, default_params(accel="chebyshev", rho=-1.0, residual_every=10),
                              raise_on_status=False)
    info = m.solve_info()
    assert sweeps == 30 + extra
    assert info["estimate_sweeps"] == 30 and info["restarts"] == 0
    assert 0.9 < info["plain_rate"] < 1.0
    expect = min(0.98, max(0.5, 1.0 - 2.0 * (1.0 - info["plain_rate"])))
    assert info["rho"] == pytest.approx(expect, rel=0, abs=1e-15)
    om = oracle.OracleMesh.from_problem(p)
    xa, s1 = om.sweeps(p.x0, 30)
    xb, s2 = om.sweeps(xa, extra, accel="chebyshev", rho=info["rho"], gamma=1.7)
    assert s1 == 0 and s2 == 0
    x_gpu = u.cpu().double().numpy() + p.X
    err = np.abs(x_gpu - xb).max() / np.abs(xb - p.X).max()
    assert err <= 1e-5, err
    r_ora = om.residual(xb) / om.residual(p.x0)
    assert abs(rel[0] - r_ora) <= 1e-3 * r_ora + 1e-5


def test_auto_rho_beats_the_fixed_default_on_a_slow_problem():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(12)
    m = Mesh.from_problem(p)
    out = {}
    for name, rho in (("auto", -1.0), ("fixed", 0.95)):
        u = _u0(p)
        st, sweeps, rel = m.solve(u, 0.0, 600, default_params(accel="chebyshev", rho=rho), raise_on_status=False)
        out[name] = rel[0]
    assert m.solve_info()["rho"] == 0.95
    assert out["auto"] < 0.7 * out["fixed"], out


def test_auto_rho_on_a_batch_converges_every_mesh():
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=5, side_lo=3, side_hi=7, seed=23)
    batch, mid, _ = W.concat_problems(probs)
    m = Mesh.from_problem(batch, mesh_id=mid)
    u = _u0(batch)
    st, sweeps, rel = m.solve(u, 1e-5, 20000, default_params(accel="chebyshev", rho=-1.0))
    assert st == 0 and np.all(rel <= 1e-5)
    info = m.solve_info()
    assert 0.5 <= info["rho"] <= 0.98 or info["restarts"] > 4


def test_pbng_sweep_rejects_automatic_rho():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.twist_block(3, 30.0, 0.1)
    m = Mesh.from_problem(p)
    with pytest.raises(PbngError):
        m.sweep(_u0(p), 5, default_params(accel="chebyshev", rho=0.0))
