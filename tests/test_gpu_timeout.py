"""Device-side timeouts of the ring passes, exercised without a GPU fault:
the test hook makes each warp's first record-copy wait expect 16 bytes more
than its copy carries.  The wait gives up after its bounded time, the kernel
records the timeout, lets its other copies land and returns, and the sweep
fails with PBNG_ETIMEOUT.  The handle stays usable: with the hook off, a
fresh run gives the same bits as a fresh handle."""

import time

import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PBNG_ETIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09021_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _u0(p):
    return torch.tensor(p.x0 - p.X, dtype=torch.float32, device="cuda")


def test_copy_wait_timeout_is_reported_and_the_handle_recovers():
    from paper_2306_09021_gb300 import Mesh, PbngError, default_params
    p = W.twist_block(6, 45.0, 0.2)
    params = default_params(accel="chebyshev")
    m = Mesh.from_problem(p)
    u = _u0(p)
    m.sweep(u, 2, params)
    with pytest.raises(PbngError):
        m.test_set_copy_shortfall(8)                 # not a multiple of 16
    m.test_set_copy_shortfall(16)
    t0 = time.perf_counter()
    with pytest.raises(PbngError) as e:
        m.sweep(u, 1, params)
    assert e.value.status == PBNG_ETIMEOUT
    assert time.perf_counter() - t0 < 60.0
    with pytest.raises(PbngError) as e:
        m.residual(u)
    assert e.value.status == PBNG_ETIMEOUT
    m.test_set_copy_shortfall(0)
    u1 = _u0(p)
    m.sweep(u1, 20, params)
    ref = Mesh.from_problem(p)
    u2 = _u0(p)
    ref.sweep(u2, 20, params)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)
