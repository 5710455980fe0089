"""Batched solves: many independent meshes of uneven size in one handle
(one launch per colour across all of them), each stopping at its own
tolerance.  Each mesh's result must equal solving it on its own."""

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


def test_batched_solve_equals_separate_solves():
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=5, side_lo=3, side_hi=7, seed=11)
    batch, mid, offs = W.concat_problems(probs)
    params = default_params(accel="chebyshev", residual_every=10)
    m = Mesh.from_problem(batch, mesh_id=mid)
    assert m.ncomp == len(probs)
    u = torch.tensor(batch.x0 - batch.X, dtype=torch.float32, device="cuda")
    st, sweeps, rel = m.solve(u, 1e-5, 20000, params)
    assert st == 0 and np.all(rel <= 1e-5)
    ub = u.cpu().double().numpy()
    for k, p in enumerate(probs):
        ms = Mesh.from_problem(p)
        us = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
        st1, sw1, rel1 = ms.solve(us, 1e-5, 20000, params)
        assert st1 == 0
        part = ub[offs[k]:offs[k + 1]]
        ref = us.cpu().double().numpy()
        scale = np.abs(ref).max()
        assert np.abs(part - ref).max() <= 1e-6 * scale, k
        assert rel[k] == pytest.approx(rel1[0], rel=1e-6)


def test_batched_colouring_is_per_mesh():
    from paper_2306_09021_gb300 import Mesh
    probs = W.batched_blocks(count=4, side_lo=3, side_hi=6, seed=3)
    batch, mid, offs = W.concat_problems(probs)
    col, n = Mesh.from_problem(batch, mesh_id=mid).colouring()
    for k, p in enumerate(probs):
        ck, _ = Mesh.from_problem(p).colouring()
        assert np.array_equal(col[offs[k]:offs[k + 1]], ck)


def test_batched_sweep_residuals_per_mesh(oracle_mod):
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=3, side_lo=3, side_hi=5, seed=5)
    batch, mid, offs = W.concat_problems(probs)
    m = Mesh.from_problem(batch, mesh_id=mid)
    u = torch.tensor(batch.x0 - batch.X, dtype=torch.float32, device="cuda")
    m.sweep(u, 15, default_params(accel="sor", omega=1.5))
    r = m.residual(u)
    x = u.cpu().double().numpy() + batch.X
    for k, p in enumerate(probs):
        om = oracle_mod.OracleMesh.from_problem(p)
        assert r[k] == pytest.approx(om.residual(x[offs[k]:offs[k + 1]]), rel=1e-5)


def test_auto_precision_batch_meets_the_tolerance_in_extended_residuals():
    """A batch in PBNG_PREC_AUTO (symmetric order, automatic rho): every mesh
    stops at the tolerance of its extended-precision residual, which
    pbng_residual (extended) confirms after the solve."""
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=6, side_lo=4, side_hi=9, seed=31)
    batch, mid, offs = W.concat_problems(probs)
    m = Mesh.from_problem(batch, mesh_id=mid)
    u0 = torch.tensor(batch.x0 - batch.X, dtype=torch.float32, device="cuda")
    r0 = m.residual(u0)
    u = u0.clone()
    tol = 1e-7
    st, sweeps, rel = m.solve(u, tol, 40000, default_params(accel="chebyshev", rho=-1.0, colour_order="symmetric",
                                                            precision="auto"))
    assert st == 0 and np.all(rel <= tol)
    # the output is float32: its own residual is that of the rounded iterate,
    # so check the solve's report against a fresh extended evaluation of the
    # iterate it stopped at (resume keeps the float pairs)
    rel_again = m.sweep(u, 0, default_params(precision="extended", resume=1), want_residual=True)
    assert np.all(rel_again <= tol * (1 + 1e-6))


def test_batched_cg_adjoint_matches_each_meshs_dense_adjoint(oracle_mod):
    """One conjugate-gradient adjoint (refined) over a batch of three meshes
    of uneven size: H is block diagonal over the meshes, so each mesh's
    sensitivities must match the oracle's dense adjoint of that mesh alone."""
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=3, side_lo=3, side_hi=5, seed=21)
    batch, mid, offs = W.concat_problems(probs)
    rng = np.random.default_rng(4)
    xeq, dldx, refs = [], [], []
    for p in probs:
        om = oracle_mod.OracleMesh.from_problem(p)
        x, it, _ = om.newton(p.x0, 1e-11, 60)
        assert it >= 0
        g = 0.01 * rng.standard_normal(x.shape)
        xeq.append(x)
        dldx.append(g)
        refs.append(om.adjoint(x, g))
    xeq, dldx = np.vstack(xeq), np.vstack(dldx)
    m = Mesh.from_problem(batch, mesh_id=mid)
    u = torch.tensor(xeq - batch.X, dtype=torch.float32, device="cuda")
    g = torch.tensor(dldx, dtype=torch.float32, device="cuda")
    st, dE, dD, its, rel = m.adjoint(u, g, 1e-8, 20000,
                                     default_params(accel="cg", colour_order="symmetric", precision="extended"))
    assert st == 0 and rel <= 1e-8
    dE, dD = dE.cpu().double().numpy(), dD.cpu().double().numpy()
    te = np.cumsum([0] + [p.ne for p in probs])
    td = np.cumsum([0] + [len(p.dirichlet) for p in probs])
    for k, (dE_ref, dD_ref) in enumerate(refs):
        e, d = dE[te[k]:te[k + 1]], dD[td[k]:td[k + 1]]
        assert np.abs(e - dE_ref).max() <= 2e-5 * np.abs(dE_ref).max(), k
        assert np.abs(d - dD_ref).max() <= 2e-5 * np.abs(dD_ref).max(), k
