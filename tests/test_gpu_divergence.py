"""Divergence reporting of pbng_solve and the state a failed solve leaves.

An iterate that grows is made on purpose with the Newton step scale of
Eq. pbgn_dx set well above 2 (the modified nodal Hessian exceeds the true
diagonal block, so the local step over-relaxes only beyond about 2.7 here):
each node update then overshoots its local minimum by more than it
corrects, and the residual grows while every value stays finite.  pbng_solve must call that PBNG_EDIVERGED, both when the residual
passes 1e3 r_0 and when it grows steadily (above r_0 and 100 times its
smallest value), never PBNG_ENOTCONVERGED.  A batched handle whose solve
ends in an error must leave every component active for later calls."""

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PBNG_EDIVERGED = 5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _u0(p):
    return torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")


def test_fast_divergence_is_reported():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(3, 45.0, 0.2)
    m = Mesh.from_problem(p)
    u = _u0(p)
    st, sweeps, rel = m.solve(u, 1e-6, 2000, default_params(step=5.0, residual_every=2), raise_on_status=False)
    assert st == PBNG_EDIVERGED
    assert sweeps < 2000
    assert torch.isfinite(u).all()


def test_sustained_growth_is_reported_below_the_hard_limit():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(4, 45.0, 0.2)
    m = Mesh.from_problem(p)
    u = _u0(p)
    st, sweeps, rel = m.solve(u, 1e-6, 5000, default_params(step=3.0, residual_every=1), raise_on_status=False)
    assert st == PBNG_EDIVERGED
    assert 1.0 < rel[0] <= 1e3      # the growth rule, not the 1e3 r_0 limit, stopped it
    assert torch.isfinite(u).all()


def test_batched_handle_is_whole_again_after_a_failed_solve():
    """Component 0 starts at its equilibrium (it is frozen at once),
    component 1 diverges.  After the failed solve a sweep on the same handle
    must update both, bit for bit like a fresh handle."""
    from paper_2306_09021_gb300 import Mesh, default_params
    rest = W.twist_block(3, 0.0, 0.0)
    twisted = W.twist_block(3, 45.0, 0.2)
    batch, mid, offs = W.concat_problems([rest, twisted], spacing=2.0)
    m = Mesh.from_problem(batch, mesh_id=mid)
    u = _u0(batch)
    st, _, rel = m.solve(u, 1e-6, 2000, default_params(step=5.0, residual_every=2), raise_on_status=False)
    assert st == PBNG_EDIVERGED
    assert rel[0] == 0.0
    # a displaced start for both components (clamped entries are reset by the library)
    both, _, _ = W.concat_problems([W.twist_block(3, 30.0, 0.1), twisted], spacing=2.0)
    params = default_params(accel="chebyshev")
    u1 = torch.tensor(both.x0 - batch.X, dtype=torch.float32, device="cuda")
    m.sweep(u1, 20, params)
    ref = Mesh.from_problem(batch, mesh_id=mid)
    u2 = torch.tensor(both.x0 - batch.X, dtype=torch.float32, device="cuda")
    ref.sweep(u2, 20, params)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)
    moved = (u1 - torch.tensor(both.x0 - batch.X, dtype=torch.float32, device="cuda")).abs()
    assert moved[offs[0]:offs[1]].max() > 0.0      # component 0 was updated
