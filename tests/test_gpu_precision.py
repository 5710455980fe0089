"""The residual and the sweep in extended precision (PBNG_PREC_EXTENDED).

Near an equilibrium the nodal force is a small sum of per-element terms
V P(F) g_i that are much larger than it (Section "Discretization",
Eq. fem_qs; the residual is the 2-norm of the Newton residual of Section
"PBNG vs. PBD and Limited Newton").  These tests take the oracle's Newton
equilibrium of a gravity-sag cube, round it to float32 (which leaves a
relative residual near 1e-5) and require the library's residual of that
state to match the oracle's FP64 residual of the same state to 1e-3
relative; they also check that extended-precision sweeps follow the oracle's
trajectory and converge to the Newton equilibrium far below the float32
passes' floor."""

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


def _equilibrium(oracle_mod, n, model="corotated"):
    p = W.gravity_sag(n)
    om = oracle_mod.OracleMesh.from_problem(p, model=model)
    xs, it, _ = om.newton(p.x0, 1e-11, 40)
    assert it >= 0
    assert om.residual(xs) <= 1e-12 * om.residual(p.x0)
    return p, om, xs


@pytest.mark.parametrize("n,model", [(6, "corotated"), (8, "corotated"), (6, "neohookean"),
                                     (6, "stable_neohookean")])
def test_residual_near_equilibrium_matches_the_oracle(oracle_mod, n, model):
    from paper_2306_09021_gb300 import Mesh, default_params
    p, om, xs = _equilibrium(oracle_mod, n, model)
    u32 = (xs - p.X).astype(np.float32)
    x32 = p.X + u32.astype(np.float64)
    r0 = om.residual(p.x0)
    r_ora = om.residual(x32)
    assert 1e-7 < r_ora / r0 < 1e-4            # near the equilibrium
    m = Mesh.from_problem(p)
    u = torch.tensor(u32, device="cuda")
    m.sweep(u, 0, default_params(model=model))   # the handle's model
    r_ext = m.residual(u)[0]
    assert abs(r_ext - r_ora) <= 1e-3 * r_ora, (r_ext, r_ora)
    # the same through a sweep call's relative residual (no sweep, r_0 at x^0)
    u0 = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    prm = default_params(model=model, precision="extended")
    rel0 = m.sweep(u0, 0, prm, want_residual=True)[0]
    assert rel0 == pytest.approx(1.0)
    r0_gpu = m.residual(u0)[0]
    assert r0_gpu == pytest.approx(r0, rel=1e-6)


def test_float32_element_residual_is_far_less_accurate_near_equilibrium(oracle_mod):
    """The float32-element residual (FP64 vertex sums) at the same state: its
    error is reported, and it must be larger than the extended one's."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p, om, xs = _equilibrium(oracle_mod, 8)
    u32 = (xs - p.X).astype(np.float32)
    r_ora = om.residual(p.X + u32.astype(np.float64))
    r0 = om.residual(p.x0)
    m = Mesh.from_problem(p)
    errs = {}
    for prec in ("compensated", "extended"):
        # pbng_sweep_host with no sweep: the absolute residual of the loaded
        # state, in the residual precision of `prec`
        r = m.sweep_host(u32.copy(), 0, default_params(precision=prec), want_residual=True)[0]
        errs[prec] = abs(r - r_ora) / r_ora
    print("relative error of the residual at r/r0 = %.1e: float32 elements %.2e, extended %.2e"
          % (r_ora / r0, errs["compensated"], errs["extended"]))
    assert errs["extended"] <= 1e-3
    assert errs["extended"] < errs["compensated"]


def test_extended_sweeps_follow_the_oracle_trajectory(oracle_mod):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(8)
    om = oracle_mod.OracleMesh.from_problem(p)
    m = Mesh.from_problem(p)
    for order in ("forward", "symmetric"):
        u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
        rel = m.sweep(u, 120, default_params(accel="chebyshev", rho=0.99, precision="extended",
                                             colour_order=order), want_residual=True)[0]
        xo, st = om.sweeps(p.x0, 120, accel="chebyshev", rho=0.99, gamma=1.7, order=order)
        assert st == 0
        x = u.cpu().double().numpy() + p.X
        err = np.abs(x - xo).max() / np.abs(xo - p.X).max()
        assert err <= 1e-5, (order, err)
        r_ora = om.residual(xo) / om.residual(p.x0)
        assert abs(rel - r_ora) <= 1e-3 * r_ora, (order, rel, r_ora)


@pytest.mark.parametrize("prec", ["extended", "auto"])
def test_extended_solve_reaches_the_newton_equilibrium(oracle_mod, prec):
    """Symmetric order, automatic rho: the extended-precision passes take the
    iterate to the oracle's Newton equilibrium within float32 rounding of
    the output, and the library's own (extended) residual agrees with the
    oracle's along the way; AUTO first stalls at the float32 passes' floor."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p, om, xs = _equilibrium(oracle_mod, 8)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    st, sweeps, rel = m.solve(u, 1e-9, 20000, default_params(accel="chebyshev", rho=-1.0, precision=prec,
                                                             colour_order="symmetric"))
    assert st == 0 and rel[0] <= 1e-9
    info = m.solve_info()
    if prec == "auto":
        assert info["extended_from"] > 0
    else:
        assert info["extended_from"] == 0
    x = u.cpu().double().numpy() + p.X
    err = np.abs(x - xs).max() / np.abs(xs - p.X).max()
    assert err <= 1e-6, err


def test_extended_precision_needs_the_ring_layout():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.twist_block(3, 30.0, 0.1)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    with pytest.raises(PbngError):
        m.sweep(u, 2, default_params(precision="extended", kernel_path=1))


@pytest.mark.parametrize("prec,floor", [("compensated", 1e-4), ("extended", 1e-10)])
def test_residual_history_matches_the_oracle_down_to_the_floor(oracle_mod, prec, floor):
    """A 10^3 gravity-sag cube, symmetric colour order, Chebyshev rho 0.998:
    the GPU's relative residual every 10 sweeps against the oracle's history
    of the same run agrees to 1e-3 relative plus the GPU path's floor (1e-4
    for the float32 passes, 1e-10 extended), at every check where the
    oracle's residual is above ten times that floor."""
    import os
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(10)
    om = oracle_mod.OracleMesh.from_problem(p)
    total, every = 700, 10
    _, st, hist = om.sweeps(p.x0, total, accel="chebyshev", rho=0.998, gamma=1.7, order="symmetric",
                            threads=oracle_mod.threads_available(os.cpu_count() or 1), history=True)
    assert st == 0
    hist = hist / hist[0]
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    prm = default_params(accel="chebyshev", rho=0.998, colour_order="symmetric", precision=prec)
    compared = 0
    for k in range(total // every):
        rel = m.sweep(u, every, prm, want_residual=True)[0]
        prm.resume = 1
        r_ora = hist[(k + 1) * every]
        if r_ora > 10.0 * floor:
            assert abs(rel - r_ora) <= 1e-3 * r_ora + floor, (prec, (k + 1) * every, rel, r_ora)
            compared += 1
    assert compared >= 10
    if prec == "extended":
        assert hist[-1] < 1e-8 and rel < 1e-8


def test_forward_order_history_matches_the_oracle_on_a_16_cube(oracle_mod):
    """The paper's setting (ascending colours, Chebyshev rho 0.95, gamma 1.7)
    on a 16^3 gravity-sag cube over 2,000 sweeps: the GPU's relative residual
    every 100 sweeps follows the oracle's FP64 history to 1e-3 relative (plus
    the float32 passes' floor, 1e-4), so the slow decay of the ascending order
    (§ "Acceleration Techniques" with a complex-spectrum iteration) is the
    method's, not the GPU's."""
    import os
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(16)
    om = oracle_mod.OracleMesh.from_problem(p)
    total, every, floor = 2000, 100, 1e-4
    _, st, hist = om.sweeps(p.x0, total, accel="chebyshev", rho=0.95, gamma=1.7,
                            threads=oracle_mod.threads_available(os.cpu_count() or 1), history=True)
    assert st == 0
    hist = hist / hist[0]
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    prm = default_params(accel="chebyshev", rho=0.95)
    for k in range(total // every):
        rel = m.sweep(u, every, prm, want_residual=True)[0]
        prm.resume = 1
        r_ora = hist[(k + 1) * every]
        assert abs(rel - r_ora) <= 1e-3 * r_ora + floor, ((k + 1) * every, rel, r_ora)
    assert hist[-1] > 1e-4          # still far from 1e-5 after 2,000 ascending sweeps
