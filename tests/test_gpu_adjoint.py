"""The coloured Gauss-Seidel adjoint (pbng_adjoint) against the oracle's
dense adjoint (itself pinned by finite differences of the loss)."""

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-3  # relative, float32 adjoint vs FP64 dense adjoint


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _loaded(n=4):
    p = W.adjoint_block(n)
    xd, acc = W.adjoint_load_cases(p, count=1, seed=9)
    p.x0 = p.X.copy()
    p.x0[p.dirichlet] = xd[0]
    p.body_accel = acc[0]
    return p


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n,accel", [(3, "none"), (4, "chebyshev"), (5, "sor")])
def test_adjoint_matches_dense_oracle(oracle_mod, n, accel):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _loaded(n)
    om = oracle_mod.OracleMesh.from_problem(p)
    xeq, it, _ = om.newton(p.x0, 1e-12, 60)
    assert it >= 0
    top = np.isclose(p.X[:, 2], 1.0)
    rng = np.random.default_rng(n)
    target = xeq + 0.01 * rng.standard_normal(xeq.shape)
    dLdx = np.where(top[:, None], 2.0 * (xeq - target), 0.0)
    dLdx[p.dirichlet] = 0.05 * rng.standard_normal((len(p.dirichlet), 3))  # direct boundary term
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)

    m = Mesh.from_problem(p)
    u = torch.tensor(xeq - p.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dLdx, dtype=torch.float32, device="cuda")
    kw = dict(accel=accel)
    if accel == "sor":
        kw["omega"] = 1.5
    st, dE, dD, sweeps, rel = m.adjoint(u, g, rel_tol=1e-6, max_sweeps=20000, params=default_params(**kw),
                                        raise_on_status=False)
    print(f"adjoint {n}^3 {accel}: status {st}, {sweeps} sweeps, rel residual {rel:.2e}")
    assert st == 0 or (st == 7 and rel <= 1e-5), (st, sweeps, rel)
    dE = dE.cpu().double().numpy()
    dD = dD.cpu().double().numpy()
    assert _rel(dE, dE_ref) <= ADJ_TOL
    # dir_idx order of pbng_set_constraints is the ascending clamped ids, as in the oracle
    assert _rel(dD, dD_ref) <= ADJ_TOL


@pytest.mark.parametrize("model", ["neohookean", "stable_neohookean"])
def test_adjoint_of_the_neohookean_models_matches_dense_oracle(oracle_mod, model):
    """The adjoint with the true Hessian of Eq. nh / Eq. snh (no polar
    factor) against the oracle's dense adjoint of the same model."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _loaded(4)
    om = oracle_mod.OracleMesh.from_problem(p, model=model)
    xeq, it, _ = om.newton(p.x0, 1e-12, 60)
    assert it >= 0
    top = np.isclose(p.X[:, 2], 1.0)
    rng = np.random.default_rng(17)
    dLdx = np.where(top[:, None], 2.0 * (xeq - (xeq + 0.01 * rng.standard_normal(xeq.shape))), 0.0)
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)
    m = Mesh.from_problem(p)
    u = torch.tensor(xeq - p.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dLdx, dtype=torch.float32, device="cuda")
    st, dE, dD, sweeps, rel = m.adjoint(u, g, rel_tol=1e-6, max_sweeps=20000,
                                        params=default_params(model=model, accel="chebyshev"), raise_on_status=False)
    assert st == 0 or (st == 7 and rel <= 1e-5), (st, sweeps, rel)
    assert _rel(dE.cpu().double().numpy(), dE_ref) <= ADJ_TOL
    assert _rel(dD.cpu().double().numpy(), dD_ref) <= ADJ_TOL


def test_adjoint_zero_rhs_gives_zero():
    from paper_2306_09021_gb300 import Mesh
    p = _loaded(3)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    st, dE, dD, sweeps, rel = m.adjoint(u, torch.zeros_like(u))
    assert st == 0 and sweeps == 0
    assert torch.count_nonzero(dE) == 0 and torch.count_nonzero(dD) == 0


@pytest.mark.parametrize("n", [4, 6])
def test_refined_adjoint_matches_dense_oracle_tightly(oracle_mod, n):
    """Extended precision: iterative refinement with the float-float force's
    central differences takes the adjoint residual far below the float32
    sweeps' floor, and the sensitivities to the dense oracle adjoint's within
    float32 rounding of the gradients themselves."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _loaded(n)
    om = oracle_mod.OracleMesh.from_problem(p)
    xeq, it, _ = om.newton(p.x0, 1e-11, 60)
    assert it >= 0
    top = np.isclose(p.X[:, 2], 1.0)
    rng = np.random.default_rng(n + 1)
    dLdx = np.where(top[:, None], 2.0 * 0.01 * rng.standard_normal(xeq.shape), 0.0)
    dLdx[p.dirichlet] = 0.05 * rng.standard_normal((len(p.dirichlet), 3))
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)
    m = Mesh.from_problem(p)
    # the equilibrium as the float pair nearest the oracle's (float32 input)
    u = torch.tensor(xeq - p.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dLdx, dtype=torch.float32, device="cuda")
    st, dE, dD, sweeps, rel = m.adjoint(u, g, rel_tol=1e-8, max_sweeps=200000,
                                        params=default_params(accel="chebyshev", rho=-1.0, colour_order="symmetric",
                                                              precision="extended"))
    print(f"refined adjoint {n}^3: {sweeps} sweeps, rel residual {rel:.2e}")
    assert st == 0 and rel <= 1e-8
    # the float32 rounding of u_eq moves the gradients by about its own size
    assert _rel(dE.cpu().double().numpy(), dE_ref) <= 2e-5
    assert _rel(dD.cpu().double().numpy(), dD_ref) <= 2e-5


@pytest.mark.parametrize("model", ["corotated", "neohookean"])
def test_cg_adjoint_matches_dense_oracle(oracle_mod, model):
    """PBNG_ACCEL_CG: conjugate gradients preconditioned by the symmetric
    block Gauss-Seidel sweep, in float32, against the oracle's dense adjoint;
    the reported residual is the true one of the returned multipliers."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _loaded(5)
    om = oracle_mod.OracleMesh.from_problem(p, model=model)
    xeq, it, _ = om.newton(p.x0, 1e-12, 60)
    assert it >= 0
    top = np.isclose(p.X[:, 2], 1.0)
    rng = np.random.default_rng(23)
    dLdx = np.where(top[:, None], 2.0 * 0.01 * rng.standard_normal(xeq.shape), 0.0)
    dLdx[p.dirichlet] = 0.05 * rng.standard_normal((len(p.dirichlet), 3))
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)
    m = Mesh.from_problem(p)
    u = torch.tensor(xeq - p.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dLdx, dtype=torch.float32, device="cuda")
    prm = default_params(model=model, accel="cg", colour_order="symmetric")
    st, dE, dD, its, rel = m.adjoint(u, g, rel_tol=1e-5, max_sweeps=5000, params=prm, raise_on_status=False)
    print(f"cg adjoint 5^3 {model}: status {st}, {its} iterations, rel residual {rel:.2e}")
    assert st == 0 and rel <= 1e-5, (st, its, rel)
    assert _rel(dE.cpu().double().numpy(), dE_ref) <= ADJ_TOL
    assert _rel(dD.cpu().double().numpy(), dD_ref) <= ADJ_TOL


def test_refined_cg_adjoint_matches_dense_oracle_tightly(oracle_mod):
    """Conjugate-gradient corrections inside the refinement reach the same
    1e-8 residual and oracle agreement as the refined sweeps."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _loaded(6)
    om = oracle_mod.OracleMesh.from_problem(p)
    xeq, it, _ = om.newton(p.x0, 1e-11, 60)
    assert it >= 0
    top = np.isclose(p.X[:, 2], 1.0)
    rng = np.random.default_rng(7)
    dLdx = np.where(top[:, None], 2.0 * 0.01 * rng.standard_normal(xeq.shape), 0.0)
    dLdx[p.dirichlet] = 0.05 * rng.standard_normal((len(p.dirichlet), 3))
    dE_ref, dD_ref = om.adjoint(xeq, dLdx)
    m = Mesh.from_problem(p)
    u = torch.tensor(xeq - p.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dLdx, dtype=torch.float32, device="cuda")
    st, dE, dD, its, rel = m.adjoint(u, g, rel_tol=1e-8, max_sweeps=20000,
                                     params=default_params(accel="cg", colour_order="symmetric", precision="extended"))
    print(f"refined cg adjoint 6^3: {its} iterations, rel residual {rel:.2e}")
    assert st == 0 and rel <= 1e-8
    assert _rel(dE.cpu().double().numpy(), dE_ref) <= 2e-5
    assert _rel(dD.cpu().double().numpy(), dD_ref) <= 2e-5


def test_cg_adjoint_needs_the_symmetric_order_and_is_rejected_elsewhere():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = _loaded(3)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    g = torch.ones_like(u)
    with pytest.raises(PbngError):
        m.adjoint(u, g, 1e-5, 100, default_params(accel="cg", colour_order="forward"))
    with pytest.raises(PbngError):
        m.sweep(u, 1, default_params(accel="cg", colour_order="symmetric"))


def test_cg_and_sweeps_agree_on_a_larger_block():
    """On a 16^3 block the refined conjugate-gradient and refined sweep
    adjoints give the same sensitivities, the former in far fewer
    iterations than the latter has sweeps."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _loaded(16)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    st, _, _ = m.solve(u, 1e-7, 40000, default_params(accel="chebyshev", rho=-1.0, colour_order="symmetric",
                                                       precision="auto"))
    assert st == 0
    top = torch.tensor(np.isclose(p.X[:, 2], 1.0), device="cuda")
    g = torch.where(top[:, None], 0.02 * torch.ones_like(u), torch.zeros_like(u))
    out = {}
    for name, prm in (("cg", default_params(accel="cg", colour_order="symmetric", precision="extended")),
                      ("sweeps", default_params(accel="chebyshev", rho=-1.0, colour_order="symmetric",
                                                precision="extended"))):
        st, dE, dD, n, rel = m.adjoint(u, g, 1e-7, 100000, prm)
        assert st == 0 and rel <= 1e-7
        out[name] = (dE.cpu().double().numpy(), dD.cpu().double().numpy(), n)
    print(f"16^3 refined adjoint: cg {out['cg'][2]} iterations, sweeps {out['sweeps'][2]}")
    assert _rel(out["cg"][0], out["sweeps"][0]) <= 1e-5
    assert _rel(out["cg"][1], out["sweeps"][1]) <= 1e-5
    assert out["cg"][2] < out["sweeps"][2]
