"""General two-sided weak constraints (Section "Weak Constraints") and the
incremental recolouring of Section "Collision Coloring" on the GPU, against
the FP64 oracle, on the two-blocks-hanging example."""

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


def _pair(p, recolour=False):
    from paper_2306_09021_gb300 import Mesh
    m = Mesh.from_problem(p)
    om = oracle.OracleMesh.from_problem(p)
    if recolour:          # colour the plain mesh first, then add the bindings
        m.colouring()
    m.set_weak_constraints(*p.meta["weak"], recolour=recolour)
    om.set_weak_constraints(*p.meta["weak"], recolour=recolour)
    return m, om


@pytest.mark.parametrize("recolour", [False, True])
def test_colouring_matches_the_oracle(recolour):
    p = W.two_blocks_hanging(4, 3, k=1e5)
    m, om = _pair(p, recolour)
    col, ncol = m.colouring()
    assert np.array_equal(col, om.colours()) and ncol == om.ncolours
    prof = m.profile()
    assert prof["colour_ms"] >= 0.0 and prof["layout_ms"] >= prof["colour_ms"]


@pytest.mark.parametrize("accel", ["none", "chebyshev"])
def test_sweeps_match_the_oracle(accel):
    from paper_2306_09021_gb300 import default_params
    p = W.two_blocks_hanging(3, 2, k=1e5)
    m, om = _pair(p)
    u = _u0(p)
    rel = m.sweep(u, 300, default_params(accel=accel), want_residual=True)
    x_ora, st = om.sweeps(p.x0, 300, accel=accel)
    assert st == 0
    x_gpu = u.cpu().double().numpy() + p.X
    err = np.abs(x_gpu - x_ora).max() / np.abs(x_ora - p.X).max()
    assert err <= 1e-5, err
    rr = om.residual(x_ora) / om.residual(p.x0)
    assert abs(rel[0] - rr) <= 1e-3 * rr + 1e-5


def test_solved_bindings_carry_the_weight():
    from paper_2306_09021_gb300 import default_params
    p = W.two_blocks_hanging(3, 2, k=1e5)
    m, om = _pair(p)
    u = _u0(p)
    st, sweeps, rel = m.solve(u, 1e-5, 40000, default_params(accel="chebyshev"))
    assert st == 0 and rel[0] <= 1e-5
    x = u.cpu().double().numpy() + p.X
    idx, w, kn, kt, nrm = p.meta["weak"]
    side0 = (w[:, :4, None] * x[np.where(idx[:, :4] < 0, 0, idx[:, :4])]).sum(1)
    side1 = (w[:, 4:, None] * x[np.where(idx[:, 4:] < 0, 0, idx[:, 4:])]).sum(1)
    force = -(kn[:, None] * (side0 - side1)).sum(0)
    na = W.box_grid(3, 3, 3, 1.0)[0].shape[0]
    _, V, _, _ = om.tet_constants()
    weight = (p.density * V)[np.any(p.tets >= na, axis=1)].sum() * 9.8
    assert abs(force[2] - weight) <= 1e-3 * weight and np.abs(force[:2]).max() <= 1e-3 * weight


def test_removing_constraints_restores_the_plain_mesh():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.two_blocks_hanging(3, 2, k=1e5)
    m, _ = _pair(p)
    m.set_weak_constraints(np.zeros((0, 8), np.int32), np.zeros((0, 8)), [], [], np.zeros((0, 3)))
    ref = Mesh.from_problem(p)
    assert np.array_equal(m.colouring()[0], ref.colouring()[0])
    u1, u2 = _u0(p), _u0(p)
    m.sweep(u1, 20, default_params())
    ref.sweep(u2, 20, default_params())
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)


def test_weak_constraint_errors():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.two_blocks_hanging(2, 1, k=1e5)
    idx, w, kn, kt, nrm = p.meta["weak"]
    m = Mesh.from_problem(p)
    bad = w.copy()
    bad[0, 4:] *= 0.5                              # side 1 no longer sums to one
    with pytest.raises(PbngError):
        m.set_weak_constraints(idx, bad, kn, kt, nrm)
    m.set_weak_constraints(idx, w, kn, kt, nrm)
    # a constraint across two batch components is rejected
    mid = np.zeros(p.nv, np.int32)
    mid[W.box_grid(2, 2, 2, 1.0)[0].shape[0]:] = 1
    mb = Mesh.from_problem(p, mesh_id=mid)
    with pytest.raises(PbngError):
        mb.set_weak_constraints(idx, w, kn, kt, nrm)


def _blocks_equilibrium(k=1e4, young=1e4):
    p = W.two_blocks_hanging(3, 2, young=young, k=k)
    m, om = _pair(p)
    xeq, it, _ = om.newton(p.x0, 1e-11, 60)
    assert it >= 0
    return p, m, om, xeq


def test_adjoint_with_two_sided_constraints_matches_the_dense_oracle():
    """The coloured block Gauss-Seidel adjoint on the two-blocks scene: the
    constraints' true Hessian blocks beta_i beta_j K (Section "Weak
    Constraints") in the diagonal blocks, in the off-diagonal products and in
    dL/dx_D, against the oracle's dense adjoint."""
    from paper_2306_09021_gb300 import default_params
    p, m, om, xeq = _blocks_equilibrium()
    rng = np.random.default_rng(4)
    low = np.isclose(p.X[:, 2], 0.0)          # the hanging block's bottom face
    dLdx = np.where(low[:, None], 2.0 * 0.01 * rng.standard_normal(xeq.shape), 0.0)
    dLdx[p.dirichlet] = 0.05 * rng.standard_normal((len(p.dirichlet), 3))
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)
    u = torch.tensor(xeq - p.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dLdx, dtype=torch.float32, device="cuda")
    st, dE, dD, sweeps, rel = m.adjoint(u, g, rel_tol=1e-5, max_sweeps=200000,
                                        params=default_params(accel="chebyshev", rho=-1.0,
                                                              colour_order="symmetric"))
    assert st == 0
    dE, dD = dE.cpu().double().numpy(), dD.cpu().double().numpy()
    assert np.abs(dE - dE_ref).max() <= 1e-3 * np.abs(dE_ref).max()
    assert np.abs(dD - dD_ref).max() <= 1e-3 * np.abs(dD_ref).max()


def test_newton_cg_with_two_sided_constraints_reaches_the_oracle_equilibrium():
    """Newton-CG with the constraints in the force, the preconditioner blocks
    and the Hessian apply reaches the oracle's Newton equilibrium."""
    from paper_2306_09021_gb300 import default_params
    p, m, om, xeq = _blocks_equilibrium()
    u = _u0(p)
    st, info = m.newton_cg(u, 1e-6, max_newton=60, max_cg=2000, cg_tol=0.05, params=default_params())
    assert st == 0, info
    x = u.cpu().double().numpy() + p.X
    assert np.abs(x - xeq).max() <= 1e-4 * np.abs(xeq - p.X).max()
