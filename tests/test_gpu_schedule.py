"""Launch schedules of the colour passes and the autotuner that picks them.

The vertex updates of one colour are independent (Section "Coloring and
Parallelism": same-colour vertices share no element), so the grid size and
the order in which warps take work items cannot change the iterate: every
schedule must give bit-identical displacements.  The autotuner times the
schedules on a scratch copy and must leave the caller's iterate and the
handle's iteration history untouched."""

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


_SCHED_PROBLEMS = {
    "twist": lambda: W.twist_block(10, 90.0, 0.3),           # 90 degree twist: large rotations
    "sag": lambda: W.gravity_sag(12),                        # lane widths 8 and 32
    "bar": lambda: W.contact_bar(4, 4, 20, h=0.05, seed=3),  # springs, contact, lognormal E
}


@pytest.mark.parametrize("model", ["corotated", "neohookean", "stable_neohookean"])
@pytest.mark.parametrize("prob", list(_SCHED_PROBLEMS))
@pytest.mark.parametrize("precision", ["compensated", "fp32"])
def test_every_schedule_gives_the_same_iterate(prob, model, precision):
    from paper_2306_09021_gb300 import Mesh, default_params
    from paper_2306_09021_gb300._lib import MAX_CTAS_PER_SM
    p = _SCHED_PROBLEMS[prob]()
    params = default_params(accel="chebyshev", model=model, precision=precision)
    ref = Mesh.from_problem(p)
    u_ref = _u0(p)
    ref.sweep(u_ref, 25, params)
    ncol = ref.colouring()[1]
    m = Mesh.from_problem(p)
    for cps in range(1, MAX_CTAS_PER_SM + 1):
        for blocked in (0, 1):
            for balanced in (0, 1):
                m.set_schedule([cps] * ncol, [blocked] * ncol, balanced=[balanced] * ncol, params=params)
                s = m.schedule()
                assert s["ctas_per_sm"] == [cps] * ncol and s["blocked"] == [blocked] * ncol
                assert s["balanced"] == [balanced] * ncol
                u = _u0(p)
                m.sweep(u, 25, params)
                torch.cuda.synchronize()
                assert torch.equal(u, u_ref), (cps, blocked, balanced)


def test_mixed_schedules_on_a_batch_give_the_same_iterate():
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=6, side_lo=3, side_hi=9, seed=5)
    batch, mid, _ = W.concat_problems(probs)
    params = default_params(accel="chebyshev")
    ref = Mesh.from_problem(batch, mesh_id=mid)
    u_ref = _u0(batch)
    ref.sweep(u_ref, 30, params)
    m = Mesh.from_problem(batch, mesh_id=mid)
    ncol = m.colouring()[1]
    m.set_schedule([1 + c % 3 for c in range(ncol)], [c % 2 for c in range(ncol)],
                   balanced=[(c // 2) % 2 for c in range(ncol)])
    u = _u0(batch)
    m.sweep(u, 30, params)
    torch.cuda.synchronize()
    assert torch.equal(u, u_ref)


def test_autotune_leaves_iterate_and_history_untouched():
    from paper_2306_09021_gb300 import Mesh, default_params
    from paper_2306_09021_gb300._lib import MAX_CTAS_PER_SM
    p = W.gravity_sag(12)
    first = default_params(accel="chebyshev")
    cont = default_params(accel="chebyshev", resume=1)
    a, b = Mesh.from_problem(p), Mesh.from_problem(p)
    ua, ub = _u0(p), _u0(p)
    a.sweep(ua, 7, first)
    b.sweep(ub, 7, first)
    probe = ua.clone() + 1e-3
    probe_before = probe.clone()
    sched = a.autotune(probe, reps=3, params=first)
    torch.cuda.synchronize()
    assert torch.equal(probe, probe_before)
    ncol = sched["ncolours"]
    assert ncol == 5 and sched["candidates"] == 4 * MAX_CTAS_PER_SM
    assert all(1 <= c <= MAX_CTAS_PER_SM for c in sched["ctas_per_sm"])
    assert all(x in (0, 1) for x in sched["blocked"]) and all(x in (0, 1) for x in sched["balanced"])
    assert 0.0 < sched["tuned_ms_per_sweep"] <= sched["default_ms_per_sweep"]
    assert a.schedule()["ctas_per_sm"] == sched["ctas_per_sm"]
    ra = a.sweep(ua, 9, cont, want_residual=True)
    rb = b.sweep(ub, 9, cont, want_residual=True)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    assert np.array_equal(ra, rb)


def test_schedule_survives_constraint_changes_and_rejects_bad_arguments():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    from paper_2306_09021_gb300._lib import MAX_CTAS_PER_SM
    p = W.twist_block(6, 45.0, 0.2)
    m = Mesh.from_problem(p)
    ncol = m.colouring()[1]
    m.set_schedule([2] * ncol, [1] * ncol)
    m.set_constraints(p.dirichlet, p.x0[p.dirichlet])
    assert m.colouring()[1] == ncol
    assert m.schedule()["ctas_per_sm"] == [2] * ncol
    m.set_schedule([99] * ncol, [1] * ncol)          # clamped
    assert m.schedule()["ctas_per_sm"] == [MAX_CTAS_PER_SM] * ncol
    with pytest.raises(PbngError):
        m.autotune(_u0(p), reps=0)
    # direct-load layout: no ring colours, nothing to schedule
    m.set_schedule([1] * ncol, [0] * ncol, params=default_params(kernel_path=1))
    assert m.schedule()["ctas_per_sm"] == [0] * ncol
