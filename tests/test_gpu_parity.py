"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: positions after a fixed number of sweeps agree to
max_i |x_gpu - x_oracle| / max_i |x_oracle - X| <= 1e-5 in compensated
precision (float32 element arithmetic, float32-pair iterate); colourings agree
bit for bit.
"""

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
RES_FLOOR = 1e-5  # relative-residual target of the float32 path


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _gpu_run(p, sweeps, **kw):
    from paper_2306_09021_gb300 import Mesh, default_params
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    rel = m.sweep(u, sweeps, default_params(**kw), want_residual=True)
    return m, u.cpu().double().numpy() + p.X, rel


def _oracle(oracle_mod, p):
    return oracle_mod.OracleMesh.from_problem(p)


def _pos_err(x, xr, X):
    return np.abs(x - xr).max() / max(np.abs(xr - X).max(), 1e-300)


ACCELS = [dict(accel="none"), dict(accel="chebyshev"), dict(accel="sor", omega=1.5)]


@pytest.mark.parametrize("kw", ACCELS, ids=lambda k: k["accel"])
def test_twist_block_200_sweeps(oracle_mod, kw):
    """Unit cube 10^3 cells (1331 vertices, 5000 tets), E = 1e5, nu = 0.3,
    bottom clamped, top lifted 30% and twisted 90 degrees; 200 sweeps."""
    p = W.twist_block(10, 90.0, 0.3)
    _, x, rel = _gpu_run(p, 200, **kw)
    om = _oracle(oracle_mod, p)
    xr, st = om.sweeps(p.x0, 200, accel=kw["accel"], omega=kw.get("omega", 1.7))
    assert st == 0
    err = _pos_err(x, xr, p.X)
    rr = om.residual(xr) / om.residual(p.x0)
    print(f"twist 10^3 {kw['accel']}: pos err {err:.2e}, rel residual gpu {rel[0]:.3e} oracle {rr:.3e}")
    assert err <= POS_TOL
    # float32 element arithmetic floors the relative residual near 1e-6 here;
    # above that floor the two residuals agree.
    assert abs(rel[0] - rr) <= 1e-3 * rr + RES_FLOOR


def test_fp32_mode_is_close(oracle_mod):
    p = W.twist_block(6, 90.0, 0.3)
    _, x, _ = _gpu_run(p, 60, precision="fp32")
    xr, _ = _oracle(oracle_mod, p).sweeps(p.x0, 60)
    assert _pos_err(x, xr, p.X) <= 1e-4


def _ragged_problem():
    """Bar of 3 x 2 x 5 cells with lognormal stiffness, gravity, springs on 10%
    of the vertices and an active contact plane; boundary vertices give every
    lane-group width and ragged colour tails."""
    p = W.contact_bar(3, 2, 5, 0.1, seed=7, spring_frac=0.1)
    p.body_accel = np.array([0.0, 0.0, -9.8])
    p.density = np.full(p.ne, 1000.0)
    p.dirichlet = np.array([0, 1], np.int32)
    p.plane = np.array([0.0, 0.0, 1.0, 0.01])  # n.x < 0.01 is in contact
    return p


@pytest.mark.parametrize("kw", ACCELS, ids=lambda k: k["accel"])
def test_ragged_bar_with_weak_constraints(oracle_mod, kw):
    p = _ragged_problem()
    if kw["accel"] == "chebyshev":
        # With the 1e8 contact penalty, gamma = 1.7 Chebyshev does not converge
        # (the FP64 residual oscillates near 3e6 and 1e-9 input noise moves the
        # iterate by 1e-5): no reference trajectory exists.  Check the springs
        # and gravity part of the path under Chebyshev with the plane removed.
        p.plane = None
    _, x, _ = _gpu_run(p, 80, **kw)
    xr, st = _oracle(oracle_mod, p).sweeps(p.x0, 80, accel=kw["accel"], omega=kw.get("omega", 1.7))
    assert st == 0
    assert _pos_err(x, xr, p.X) <= POS_TOL


@pytest.mark.parametrize("maker", [lambda: W.twist_block(5), lambda: W.gravity_sag(7),
                                   lambda: W.contact_bar(4, 3, 9, 0.05, spring_frac=0.05),
                                   _ragged_problem])
def test_colouring_matches_oracle(oracle_mod, maker):
    from paper_2306_09021_gb300 import Mesh
    p = maker()
    col, n = Mesh.from_problem(p).colouring()
    om = _oracle(oracle_mod, p)
    assert n == om.ncolours
    assert np.array_equal(col, om.colours())


def test_table1_colour_counts():
    """Table 1: 5 particle colours for the Res 16 / 32 / 64 / 128 boxes."""
    from paper_2306_09021_gb300 import Mesh
    from tests.golden.values import paper_values
    pv = paper_values()
    for res in (16, 32, 64, 128):
        X, tets = W.box_grid(res, res, res, 1.0 / res)
        m = Mesh(X, tets, 1e5, 0.3)
        m.set_constraints()
        _, n = m.colouring()
        assert n == int(pv[f"box_res{res}_particle_colours"])


def test_residual_matches_oracle(oracle_mod):
    from paper_2306_09021_gb300 import Mesh
    p = _ragged_problem()
    m = Mesh.from_problem(p)
    om = _oracle(oracle_mod, p)
    rng = np.random.default_rng(3)
    for k in range(3):
        x = p.x0 + 0.01 * rng.standard_normal(p.x0.shape)
        x[p.dirichlet] = p.x0[p.dirichlet]
        u = torch.tensor(x - p.X, dtype=torch.float32, device="cuda")
        xs = u.cpu().double().numpy() + p.X  # the float32-rounded state both sides see
        r_gpu = m.residual(u)[0]
        r_ora = om.residual(xs)
        assert r_gpu == pytest.approx(r_ora, rel=1e-5)


def test_sweep_commutes_with_rigid_motion():
    p = W.twist_block(5, 60.0, 0.2)
    _, x1, _ = _gpu_run(p, 20)
    a = 0.7
    Q = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    Q = Q @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    b = np.array([0.2, -0.1, 0.3])
    q = W.twist_block(5, 60.0, 0.2)
    q.X = p.X @ Q.T + b
    q.x0 = p.x0 @ Q.T + b
    _, x2, _ = _gpu_run(q, 20)
    assert np.abs(x2 - (x1 @ Q.T + b)).max() / np.abs(x1 - p.X).max() <= POS_TOL


def test_solve_reaches_newton_equilibrium(oracle_mod):
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(6)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    st, sweeps, rel = m.solve(u, RES_FLOOR, 20000, default_params(accel="chebyshev", residual_every=20),
                              raise_on_status=False)
    print(f"sag 6^3 chebyshev: status {st}, {sweeps} sweeps, rel residual {rel[0]:.3e}")
    assert st == 0 and rel[0] <= RES_FLOOR
    xn, it, _ = _oracle(oracle_mod, p).newton(p.x0, 1e-12, 60)
    assert it >= 0
    x = u.cpu().double().numpy() + p.X
    assert _pos_err(x, xn, p.X) <= 1e-4


def test_resume_is_bit_exact():
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(6, 90.0, 0.3)
    m = Mesh.from_problem(p)
    u1 = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    m.sweep(u1, 50, default_params(accel="chebyshev"))
    m.sweep(u1, 50, default_params(accel="chebyshev", resume=1))
    m2 = Mesh.from_problem(p)
    u2 = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    m2.sweep(u2, 100, default_params(accel="chebyshev"))
    assert torch.equal(u1, u2)


def test_full_size_gravity_sag_sampled(oracle_mod):
    """64^3 cells (274,625 vertices, 1,310,720 tets), the benchmark's mesh and
    launch configuration: the update of sampled vertices of every colour in one
    GPU sweep equals the oracle's node update from the same state."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.gravity_sag(64)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    m.sweep(u, 5, default_params())
    s0 = u.cpu().double().numpy() + p.X
    m.sweep(u, 1, default_params())
    s1 = u.cpu().double().numpy() + p.X
    col, ncol = m.colouring()
    om = _oracle(oracle_mod, p)
    rng = np.random.default_rng(11)
    for c in range(ncol):
        ids = rng.choice(np.flatnonzero(col == c), 12, replace=False)
        mixed = np.where((col < c)[:, None] & (col >= 0)[:, None], s1, s0)
        for i in ids:
            r, A = om.local_system(mixed, i)
            d_ora = np.linalg.solve(A, r)
            d_gpu = s1[i] - s0[i]
            assert np.abs(d_gpu - d_ora).max() <= 2e-4 * np.abs(d_ora).max() + 1e-9


def test_edge_cases():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    # every vertex clamped: a sweep leaves the targets in place
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tets = np.array([[0, 1, 2, 3]], np.int32)
    m = Mesh(X, tets, 1e5, 0.3)
    m.set_constraints(np.arange(4), X + 0.1)
    u = torch.zeros(4, 3, device="cuda")
    m.sweep(u, 3, default_params())
    assert torch.allclose(u, torch.full_like(u, 0.1))
    # one free vertex, pulled by gravity: converges
    m.set_constraints(np.arange(3), X[:3], body_accel=[0, 0, -9.8], density=[1e3])
    st, n, rel = m.solve(u, 1e-7, 5000, default_params())
    assert st == 0
    # bad inputs fail with a status, never a crash
    with pytest.raises(PbngError):
        Mesh(X, np.array([[0, 1, 2, 7]], np.int32), 1e5, 0.3)
    with pytest.raises(PbngError):
        Mesh(np.zeros((4, 3)), tets, 1e5, 0.3)  # zero-volume tet
    with pytest.raises(PbngError):
        m.set_constraints(np.array([9], np.int32), np.zeros((1, 3)))
    with pytest.raises(ValueError):
        m.sweep(torch.zeros(5, 3, device="cuda"), 1)


@pytest.mark.parametrize("maker", [lambda: W.twist_block(10, 90.0, 0.3), lambda: W.gravity_sag(12),
                                   _ragged_problem])
def test_pipelined_equals_direct(maker):
    """The ring-layout kernels (TMA-staged records, 1-ring gathers) and the
    direct-load kernels run the same per-vertex arithmetic in the same lane
    order; they differ only where the compiler fuses multiply-adds
    differently, i.e. at float32 rounding level."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = maker()
    out = []
    for path in (0, 1):
        m = Mesh.from_problem(p)
        u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
        rel = m.sweep(u, 30, default_params(accel="sor", omega=1.5, kernel_path=path), want_residual=True)
        out.append((u, rel, m.residual(u)))
    scale = (out[1][0]).abs().max().item()
    assert (out[0][0] - out[1][0]).abs().max().item() <= 1e-6 * scale
    assert out[0][1][0] == pytest.approx(out[1][1][0], rel=1e-3, abs=1e-7)
    assert out[0][2][0] == pytest.approx(out[1][2][0], rel=1e-3, abs=1e-7 * out[1][2][0] + 1e-12)


def test_checkpoint_across_handles_is_bit_exact():
    """100 sweeps == 50 sweeps, checkpoint, restore in a new handle, 50 more."""
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.twist_block(6, 90.0, 0.3)
    params = default_params(accel="chebyshev")
    m1 = Mesh.from_problem(p)
    u1 = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    m1.sweep(u1, 100, params)
    m2 = Mesh.from_problem(p)
    u2 = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    m2.sweep(u2, 50, params)
    blob = m2.get_state()
    del m2
    m3 = Mesh.from_problem(p)
    m3.set_state(blob)
    u3 = torch.zeros_like(u2)
    m3.sweep(u3, 50, default_params(accel="chebyshev", resume=1))
    assert torch.equal(u1, u3)
    other = Mesh.from_problem(W.twist_block(5))
    with pytest.raises(PbngError):
        other.set_state(blob)


def _fan_problem():
    """A centre vertex joined to the 80 faces of a once-subdivided icosahedron:
    the centre has 80 incident tets (more than one warp's lanes), the surface
    vertices 5 or 6.  Five surface vertices are clamped; gravity loads it."""
    t = (1 + 5 ** 0.5) / 2
    V = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    F = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
         [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5], [2, 4, 11],
         [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    V = [list(np.asarray(v, float) / np.linalg.norm(v)) for v in V]
    mid = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            m = (np.asarray(V[a]) + np.asarray(V[b])) / 2
            V.append(list(m / np.linalg.norm(m)))
            mid[key] = len(V) - 1
        return mid[key]

    F2 = []
    for a, b, c in F:
        ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        F2 += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
    X = np.vstack([np.zeros((1, 3)), np.asarray(V)])
    tets = np.array([[0, a + 1, b + 1, c + 1] for a, b, c in F2], np.int32)
    ne = len(tets)
    dirichlet = np.array([1, 2, 3, 4, 5], np.int32)
    rng = np.random.default_rng(8)
    x0 = X + 0.05 * rng.standard_normal(X.shape)
    x0[dirichlet] = X[dirichlet]
    return W.Problem(name="fan", X=X, tets=tets, young=np.full(ne, 1e5), poisson=np.full(ne, 0.3),
                     dirichlet=dirichlet, x0=x0, body_accel=np.array([0.0, 0.0, -9.8]),
                     density=np.full(ne, 1000.0))


def test_high_degree_vertex_uses_direct_loads_and_matches_the_oracle(oracle_mod):
    """A colour whose vertex has more incident tets than a warp has lanes is
    laid out for direct loads while the other colours keep the ring layout;
    the mixed sweep and residual match the oracle."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _fan_problem()
    assert np.bincount(p.tets.reshape(-1))[0] == 80
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    rel = m.sweep(u, 60, default_params(accel="chebyshev"), want_residual=True)
    sched = m.schedule()
    assert 0 in sched["ctas_per_sm"] and any(c > 0 for c in sched["ctas_per_sm"])  # mixed layout
    om = _oracle(oracle_mod, p)
    x_ora, st = om.sweeps(p.x0, 60, accel="chebyshev")
    assert st == 0
    x_gpu = u.cpu().double().numpy() + p.X
    assert np.abs(x_gpu - x_ora).max() <= 1e-5 * np.abs(x_ora - p.X).max()
    rr = om.residual(x_ora) / om.residual(p.x0)
    assert abs(rel[0] - rr) <= 1e-3 * rr + RES_FLOOR


def test_isolated_vertex(oracle_mod):
    """A free vertex in no tetrahedron: with a spring its nodal system is the
    spring alone (A = k I) and it lands on the target in one update, as in the
    oracle; without one its nodal Hessian is zero and the sweep reports
    PBNG_EDEGENERATE instead of writing a non-finite value."""
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.twist_block(3, 30.0, 0.1)
    X = np.vstack([p.X, [[2.0, 2.0, 2.0]]])
    iso = X.shape[0] - 1
    x0 = np.vstack([p.x0, [[2.0, 2.0, 2.0]]])
    target = np.array([[2.1, 1.9, 2.05]])
    m = Mesh(X, p.tets, p.young, p.poisson)
    m.set_constraints(p.dirichlet, p.x0[p.dirichlet], np.array([iso], np.int32), target, np.array([1e3]))
    u = torch.tensor(x0 - X, dtype=torch.float32, device="cuda")
    m.sweep(u, 20, default_params())
    om = oracle_mod.OracleMesh(X, p.tets, p.young, p.poisson,
                               np.isin(np.arange(len(X)), p.dirichlet).astype(np.uint8),
                               spr_idx=np.array([iso]), spr_target=target, spr_k=np.array([1e3]))
    x_ora, st = om.sweeps(x0, 20)
    assert st == 0
    x_gpu = u.cpu().double().numpy() + X
    assert np.abs(x_gpu[iso] - target[0]).max() <= 1e-6
    assert np.abs(x_gpu - x_ora).max() <= 1e-5 * np.abs(x_ora - X).max()
    m.set_constraints(p.dirichlet, p.x0[p.dirichlet])      # spring removed
    u = torch.tensor(x0 - X, dtype=torch.float32, device="cuda")
    with pytest.raises(PbngError) as e:
        m.sweep(u, 2, default_params())
    assert "DEGENERATE" in str(e.value)


@pytest.mark.parametrize("angle", [150.0, 179.0])
def test_large_rotation_matches_oracle(oracle_mod, angle):
    """The deformed state and the clamp targets of a twisted block turned
    rigidly by more than 120 degrees about an oblique axis: every element's
    polar factor takes the adjugate column with the largest diagonal instead
    of column 0 (Horn's eigenvector for rotations near 180 degrees), and the
    iterate still follows the FP64 oracle."""
    p = W.twist_block(4, 45.0, 0.1)
    axis = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    t = np.radians(angle)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Q = np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K
    c = p.X.mean(axis=0)
    p.x0 = (p.x0 - c) @ Q.T + c
    _, x_gpu, _ = _gpu_run(p, 30)
    x_ora, st = _oracle(oracle_mod, p).sweeps(p.x0, 30)
    assert st == 0
    assert np.abs(x_gpu - x_ora).max() <= POS_TOL * np.abs(x_ora - p.X).max()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_sweep_equals_device_sweep(pinned):
    """pbng_sweep_host (host iterate in and out, one synchronisation) gives the
    bits of pbng_sweep with resume = 0 on a device copy, and the absolute
    residual that pbng_residual reports for the result."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = W.twist_block(8, 60.0, 0.2)
    # pbng_residual evaluates the element forces in extended precision, so
    # the sweeps' residuals are taken in that precision too
    params = default_params(accel="chebyshev", precision="extended")
    m = Mesh.from_problem(p)
    u_dev = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    r_start = m.residual(u_dev)[0]
    rel = m.sweep(u_dev, 23, params, want_residual=True)
    h = torch.tensor(p.x0 - p.X, dtype=torch.float32)
    if pinned:
        h = h.pin_memory()
    r_host = m.sweep_host(h, 23, params, want_residual=True)
    torch.cuda.synchronize()
    assert torch.equal(h, u_dev.cpu())
    # the same FP64 residual of the same (compensated) state
    assert r_host[0] == pytest.approx(rel[0] * r_start, rel=1e-12)
    # twice in a row from the returned host iterate: a fresh history each call
    m.sweep_host(h, 5, params)
    u2 = u_dev.clone()
    m.sweep(u2, 5, params)
    assert torch.equal(h, u2.cpu())
    # no sweep: the residual of the loaded iterate
    r0 = m.sweep_host(h.clone(), 0, params, want_residual=True)
    assert r0[0] == pytest.approx(m.residual(u2)[0], rel=1e-12)


def _full_size_case(name):
    if name == "bar":
        return W.contact_bar(), None, {}
    if name == "blocks":
        return W.two_blocks_hanging(64, 48, k=1e5), None, {}
    if name == "batched":
        p, mid, _ = W.concat_problems(W.batched_blocks())
        return p, mid, {}
    if name == "adjoint_case":
        # one load case of the adjoint workload's 48^3 block: the clamp's
        # rigid motion extended to the block, its own gravity direction
        p = W.adjoint_block(48)
        xall, accs = W.adjoint_load_cases(p, count=32, full_body=True)
        p.x0 = xall[5]
        p.body_accel = np.asarray(accs[5], dtype=np.float64)
        return p, None, {}
    model = {"sag64_nh": "neohookean", "sag64_snh": "stable_neohookean"}[name]
    return W.gravity_sag(64), None, {"model": model}


@pytest.mark.parametrize("name,kw", [
    ("sag64", dict(accel="chebyshev")),
    ("sag64_symmetric", dict(accel="chebyshev", rho=0.999, colour_order="symmetric")),
    ("bar", dict(accel="none", precision="extended")),
], ids=["sag64_chebyshev", "sag64_symmetric_chebyshev", "bar_plain_without_plane_extended"])
def test_full_size_trajectory_matches_the_oracle(oracle_mod, name, kw):
    """Every position after 30 sweeps from x^0 at full size, in the benchmark's
    launch configuration (Eq. pbgn_update colour by colour, Section "Coloring
    and Parallelism"; acceleration after each sweep, Section "Acceleration
    Techniques"): the 64^3 gravity-sag cube (274,625 vertices, 1,310,720
    tets) with Chebyshev rho = 0.95 in ascending and rho = 0.999 in symmetric
    colour order, and the 40x40x200 bar (1.6 M tets, lognormal E, 2 % of the
    vertices on springs) with plain sweeps.  The bar runs without its contact
    plane here: with k_n = 1e8 a vertex in contact settles within about 1e-11
    of the plane, below float32 resolution of its position, so whether the
    penalty is active (n.x < d) is decided differently in float32 and FP64
    and the two trajectories part (1.5e-2 after 30 sweeps); the plane is
    covered by the ragged-bar trajectory and the sampled full-size step.  Its
    springs pull single vertices 5 cm on 5 mm elements, which inverts and
    flattens elements around them, where the polar factor is ill-conditioned
    (two singular values summing to nearly zero): the float32 rotation
    estimate and the oracle's FP64 SVD then part by more than rounding, and
    the trajectory ends 2.3e-4 (float32 passes) or 4.6e-5 (extended
    precision) from the oracle's after 30 sweeps.  The bar runs in extended
    precision and is held to 1e-4.  The oracle runs on every host core (its
    colour loop parallelises without changing a bit)."""
    import os
    if name == "bar":
        p = W.contact_bar()
        p.plane, p.k_contact = None, 0.0
    else:
        p = W.gravity_sag(64)
    sweeps = 30
    _, x, rel = _gpu_run(p, sweeps, **kw)
    om = _oracle(oracle_mod, p)
    threads = oracle_mod.threads_available(os.cpu_count() or 1)
    okw = {k: v for k, v in kw.items() if k not in ("colour_order", "precision")}
    xr, st = om.sweeps(p.x0, sweeps, threads=threads, order=kw.get("colour_order", "forward"), **okw)
    assert st == 0
    err = _pos_err(x, xr, p.X)
    rr = om.residual(xr) / om.residual(p.x0)
    print(f"{name} {sweeps} sweeps: pos err {err:.2e}, rel residual gpu {rel[0]:.4e} oracle {rr:.4e}")
    assert err <= (1e-4 if name == "bar" else POS_TOL)
    assert abs(rel[0] - rr) <= 1e-3 * rr


@pytest.mark.parametrize("name", ["bar", "blocks", "batched", "adjoint_case", "sag64_nh", "sag64_snh"])
def test_full_size_workloads_sampled(oracle_mod, name):
    """The other benchmark workloads at full size, in the benchmark's launch
    configuration: the contact bar (1.6 M tets, springs, plane, lognormal E),
    the weak-constraint blocks (1.86 M tets, 2,401 bindings), the 256-mesh
    batch (14.2 M tets), one load case of the adjoint workload's 48^3 block
    and the Neo-Hookean models on the 64^3 cube.  After
    three sweeps, one more GPU sweep moves sampled vertices of every colour
    (constraint vertices among them) by the oracle's Newton step on its local
    system, taken from the state that vertex's update saw."""
    from paper_2306_09021_gb300 import Mesh, default_params
    from paper_2306_09021_gb300._lib import MODEL
    p, mid, kw = _full_size_case(name)
    m = Mesh.from_problem(p, mesh_id=mid)
    om = oracle_mod.OracleMesh.from_problem(p, model=MODEL[kw.get("model", "corotated")])
    bound = np.zeros(p.nv, bool)
    if "weak" in p.meta:
        m.set_weak_constraints(*p.meta["weak"])
        om.set_weak_constraints(*p.meta["weak"])
        idx = p.meta["weak"][0]
        bound[idx[idx >= 0]] = True
    params = default_params(**kw)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    m.sweep(u, 3, params)
    s0 = u.cpu().double().numpy() + p.X
    m.sweep(u, 1, params)
    s1 = u.cpu().double().numpy() + p.X
    col, ncol = m.colouring()
    rng = np.random.default_rng(17)
    for c in range(ncol):
        members = np.flatnonzero(col == c)
        ids = list(rng.choice(members, min(8, len(members)), replace=False))
        on = np.flatnonzero(bound[members])
        ids += list(members[rng.choice(on, min(4, len(on)), replace=False)]) if len(on) else []
        mixed = np.ascontiguousarray(np.where((col < c)[:, None] & (col >= 0)[:, None], s1, s0))
        for i in ids:
            r, A = om.local_system(mixed, i)
            d_ora = np.linalg.solve(A, r)
            d_gpu = s1[i] - s0[i]
            # the states are read back as float32 displacements: a few ulps of
            # u on top of the relative tolerance
            ulps = 4.0 * 2.0 ** -23 * np.abs(s0[i] - p.X[i]).max()
            assert np.abs(d_gpu - d_ora).max() <= 2e-4 * np.abs(d_ora).max() + ulps + 1e-12, (name, c, i)


def test_host_buffer_sweep_on_a_batch_reports_every_component():
    """Three meshes in one handle: pbng_sweep_host gives the device sweep's
    iterate and, per component, its residual (relative residual times the
    starting residual)."""
    from paper_2306_09021_gb300 import Mesh, default_params
    probs = W.batched_blocks(count=3, side_lo=3, side_hi=6, seed=9)
    p, mid, _ = W.concat_problems(probs)
    params = default_params(accel="chebyshev", precision="extended")  # as pbng_residual
    m = Mesh.from_problem(p, mesh_id=mid)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    r_start = m.residual(u)
    rel = m.sweep(u, 17, params, want_residual=True)
    h = torch.tensor(p.x0 - p.X, dtype=torch.float32).pin_memory()
    r_host = m.sweep_host(h, 17, params, want_residual=True)
    torch.cuda.synchronize()
    assert len(r_host) == 3
    assert torch.equal(h, u.cpu())
    assert np.allclose(r_host, rel * r_start, rtol=1e-12, atol=0.0)


def _full_pair_problem():
    """A centre vertex with exactly 32 incident tets and 32 1-ring vertices:
    two rings of 16 vertices (z = +-0.5, the lower one turned by half a step)
    joined to the centre by the tets (c, a_i, a_i+1, b_i) and
    (c, b_i, b_i+1, a_i+1).  Its pair item uses every lane of a 16-lane group
    with both tets and both 1-ring slots filled, and its ring item all 32
    lanes; the ring vertices have 3 tets and 5 neighbours.  Four ring
    vertices are clamped; gravity loads it."""
    n = 16
    ang = 2 * np.pi * np.arange(n) / n
    a = np.stack([np.cos(ang), np.sin(ang), np.full(n, 0.5)], 1)
    b = np.stack([np.cos(ang + np.pi / n), np.sin(ang + np.pi / n), np.full(n, -0.5)], 1)
    X = np.vstack([np.zeros((1, 3)), a, b])
    A = lambda i: 1 + i % n
    B = lambda i: 1 + n + i % n
    tets = []
    for i in range(n):
        for t in ([0, A(i), A(i + 1), B(i)], [0, B(i), B(i + 1), A(i + 1)]):
            P = X[t]
            if np.linalg.det(P[1:] - P[0]) < 0:
                t = [t[0], t[2], t[1], t[3]]
            tets.append(t)
    tets = np.array(tets, np.int32)
    ne = len(tets)
    dirichlet = np.array([A(0), A(8), B(4), B(12)], np.int32)
    rng = np.random.default_rng(12)
    x0 = X + 0.03 * rng.standard_normal(X.shape)
    x0[dirichlet] = X[dirichlet]
    return W.Problem(name="full_pair", X=X, tets=tets, young=np.full(ne, 1e5), poisson=np.full(ne, 0.3),
                     dirichlet=dirichlet, x0=x0, body_accel=np.array([0.0, 0.0, -9.8]),
                     density=np.full(ne, 1000.0))


@pytest.mark.parametrize("precision", ["compensated", "extended"])
def test_full_32_tet_32_ring_vertex_matches_the_oracle(oracle_mod, precision):
    """The widest vertex the ring layout holds (32 tets, 32 1-ring vertices):
    the float32 passes' pair item fills both tets and both 1-ring slots of all
    16 lanes of its group, the extended passes' ring item all 32 lanes; 30
    Chebyshev sweeps (to about 3e-4 of the initial residual) match the
    oracle's positions and residual."""
    from paper_2306_09021_gb300 import Mesh, default_params
    p = _full_pair_problem()
    assert np.bincount(p.tets.reshape(-1))[0] == 32
    assert len(np.setdiff1d(np.unique(p.tets[np.any(p.tets == 0, axis=1)]), [0])) == 32
    m = Mesh.from_problem(p)
    sched = m.schedule()
    assert all(c > 0 for c in sched["ctas_per_sm"])  # every colour in the ring layout
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    rel = m.sweep(u, 30, default_params(accel="chebyshev", precision=precision), want_residual=True)
    om = _oracle(oracle_mod, p)
    x_ora, st = om.sweeps(p.x0, 30, accel="chebyshev")
    assert st == 0
    x_gpu = u.cpu().double().numpy() + p.X
    assert np.abs(x_gpu - x_ora).max() <= 1e-5 * np.abs(x_ora - p.X).max()
    rr = om.residual(x_ora) / om.residual(p.x0)
    assert abs(rel[0] - rr) <= 1e-3 * rr + RES_FLOOR
