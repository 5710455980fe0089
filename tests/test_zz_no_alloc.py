"""pbng_residual_noalloc: the allocation-free residual entry point.

Some callers cannot allocate GPU memory while their solve loop runs (their
device memory is owned by their own pool allocator, or a cudaMalloc/cudaFree
would stall a real-time loop).  For them the library offers a residual that
keeps its FP64 partial sums in one fixed array reserved when the library is
loaded.  This checks, through the C ABI, that two calls in a row give the
same norms as pbng_residual, for one mesh and for a batch of two meshes
(whose per-mesh sums must be cleared between calls).  The file is named to be
collected last.
"""

import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES_REL_TOL = 1e-5  # residual tolerance used by the parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    from paper_2306_09021_gb300 import _lib
    return _lib.load()


def _noalloc(lib, mesh, u):
    out = np.zeros(mesh.ncomp)
    st = lib.pbng_residual_noalloc(mesh.h, ctypes.c_void_p(u.data_ptr()),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == 0, lib.pbng_last_error(mesh.h)
    return out


def _states(p, mesh, n):
    from paper_2306_09021_gb300 import default_params
    u1 = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    u2 = u1.clone()
    mesh.sweep(u2, n, default_params(accel="chebyshev"))
    return u1, u2


def test_noalloc_residual_single_mesh(lib):
    from paper_2306_09021_gb300 import Mesh
    p = W.gravity_sag(12)
    m = Mesh.from_problem(p)
    u1, u2 = _states(p, m, 30)
    ref1, ref2 = m.residual(u1), m.residual(u2)
    got1 = _noalloc(lib, m, u1)
    got2 = _noalloc(lib, m, u2)
    assert ref1[0] != pytest.approx(ref2[0], rel=1e-3)  # the two states differ
    np.testing.assert_allclose(got1, ref1, rtol=RES_REL_TOL)
    np.testing.assert_allclose(got2, ref2, rtol=RES_REL_TOL)


def test_noalloc_residual_batch_of_two(lib):
    from paper_2306_09021_gb300 import Mesh
    a = W.twist_block(4, 60.0, 0.2)
    b = W.gravity_sag(5)
    X = np.vstack([a.X, b.X + np.array([3.0, 0.0, 0.0])])
    tets = np.vstack([a.tets, b.tets + a.nv]).astype(np.int32)
    mid = np.concatenate([np.zeros(a.nv), np.ones(b.nv)]).astype(np.int32)
    m = Mesh(X, tets, 1e5, np.concatenate([a.poisson, b.poisson]), mesh_id=mid)
    dirs = np.concatenate([a.dirichlet, b.dirichlet + a.nv]).astype(np.int32)
    x0 = np.vstack([a.x0, b.x0 + np.array([3.0, 0.0, 0.0])])
    m.set_constraints(dirs, x0[dirs], body_accel=[0.0, 0.0, -9.8],
                      density=np.full(len(tets), 1000.0))
    u1 = torch.tensor(x0 - X, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(5)
    u2 = (u1 + 1e-3 * torch.randn(u1.shape, generator=g, device="cuda")).contiguous()
    ref1, ref2 = m.residual(u1), m.residual(u2)
    assert ref1.shape == (2,)
    got1 = _noalloc(lib, m, u1)
    got2 = _noalloc(lib, m, u2)
    np.testing.assert_allclose(got1, ref1, rtol=RES_REL_TOL)
    np.testing.assert_allclose(got2, ref2, rtol=RES_REL_TOL)


def test_noalloc_residual_rejects_an_unbuilt_layout_and_allocates_nothing(lib):
    """Before the layout exists the call must fail with PBNG_EINVAL (building
    the layout allocates); once it exists, repeated calls leave the device's
    free memory and torch's allocator untouched."""
    from paper_2306_09021_gb300 import Mesh
    p = W.gravity_sag(6)
    m = Mesh.from_problem(p)
    u = torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")
    out = np.zeros(1)
    st = lib.pbng_residual_noalloc(m.h, ctypes.c_void_p(u.data_ptr()),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == 1  # PBNG_EINVAL
    assert b"layout" in lib.pbng_last_error(m.h)
    ref = m.residual(u)           # builds the layout
    _noalloc(lib, m, u)           # first call: looks the scratch address up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    got = _noalloc(lib, m, u)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    np.testing.assert_allclose(got, ref, rtol=RES_REL_TOL)
