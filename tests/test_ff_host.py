"""The extended-precision element force (csrc/pbng_ff.cuh, the float-float
V P(F) s of Section "Constitutive Models" with the corotated rotation refined
from a float32 quaternion) against the FP64 oracle's first Piola-Kirchhoff
stress, on the CPU: the header's host path is compiled with g++.

The inputs are the float pairs the extended passes store (each FP64 value
split into hi + lo) and the reference is formed in FP64 from exactly those
pairs, so the float-float path must agree to far below float32 rounding: a
dropped low word, a sign or index slip, or a float32 step anywhere fails the
1e-12 bound (measured: about 3e-15), which float32 inputs break by four orders of
magnitude (2e-8)."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2306_09021_gb300", "csrc")
TOL = 1e-12


@pytest.fixture(scope="module")
def ff(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("ffhost") / "libffhost.so")
    # no contraction of a * b + c into FMAs: the error-free transformations
    # depend on separate roundings (the device path uses explicit intrinsics)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "ff_host.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_double)
    lib.ff_element_force.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_float), P]
    lib.ff_element_force.restype = ctypes.c_int

    def call(model, g, d, a, b, q):
        g = np.ascontiguousarray(g, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        q = np.ascontiguousarray(q, np.float32)
        out = np.zeros(3)
        assert lib.ff_element_force(model, g.ctypes.data_as(P), d.ctypes.data_as(P), a, b,
                                    q.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    out.ctypes.data_as(P)) == 0
        return out
    return call


def _pair(x):
    """The FP64 value of the float pair (hi, lo) a double is stored as."""
    x = np.asarray(x, np.float64)
    h = x.astype(np.float32)
    return h.astype(np.float64) + (x - h.astype(np.float64)).astype(np.float32).astype(np.float64)


def _rotation(axis, theta):
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(theta) * K + (1 - np.cos(theta)) * K @ K


def _quaternion(R):
    """Unit quaternion (w, x, y, z) of a rotation matrix (largest-component branch)."""
    tr = np.trace(R)
    if tr > 0:
        w = 0.5 * np.sqrt(1 + tr)
        return np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)])
    i = int(np.argmax(np.diag(R)))
    j, k = (i + 1) % 3, (i + 2) % 3
    t = 0.5 * np.sqrt(1 + 2 * R[i, i] - tr)
    q = np.zeros(4)
    q[1 + i] = t
    q[0] = (R[k, j] - R[j, k]) / (4 * t)
    q[1 + j] = (R[j, i] + R[i, j]) / (4 * t)
    q[1 + k] = (R[k, i] + R[i, k]) / (4 * t)
    return q


def _cases(seed, n):
    """Random tets under F = Rot(theta) (I + eps S): strains 1e-3 .. 0.2,
    rotations 0 .. 2.8 rad; the rest shape gradients and the displacement
    differences as their stored float pairs."""
    rng = np.random.default_rng(seed)
    for t in range(n):
        X = np.vstack([np.zeros(3), np.eye(3) + 0.3 * rng.uniform(-1, 1, (3, 3))])
        Dm = (X[1:] - X[0]).T
        g = np.linalg.inv(Dm)                                  # row k = dN_k / dX
        theta = [0.0, 0.05, 1.0, 2.8][t % 4]
        eps = [1e-3, 1e-2, 0.2][(t // 4) % 3]
        S = rng.uniform(-1, 1, (3, 3))
        Ft = _rotation(rng.uniform(-1, 1, 3) + [0, 0, 1e-3], theta) @ (np.eye(3) + eps * 0.5 * (S + S.T))
        d = (X[1:] - X[0]) @ (Ft - np.eye(3)).T                # row k = (Ft - I)(X_k - X_0)
        mu, lam = rng.uniform(0.5, 1.5), rng.uniform(2.0, 4.0)
        yield _pair(g), _pair(d), _pair(2.0 * mu), _pair(lam)


def _reference(model, g, d, a, b):
    """FP64: F = I + sum_k d_k g_k^T, V P(F) s with V = 1, mu = a / 2,
    lambda = b, s = g_1 + g_2 + g_3; and the scale of its largest parts."""
    F = np.eye(3) + d.T @ g
    s = g.sum(axis=0)
    P = oracle.pk1(F, a / 2.0, b, model)
    C = oracle.cofactor(F)
    J = np.linalg.det(F)
    ns, nF, nC = np.linalg.norm(s), np.linalg.norm(F), np.linalg.norm(C)
    scale = ns * (a * (nF + 3.0) + b * nC * (abs(J - 1.0) + nF ** 3))
    return P @ s, F, scale


@pytest.mark.parametrize("model", [0, 1, 2])
def test_float_float_element_force_matches_the_fp64_oracle(ff, model):
    worst, float32_worst = 0.0, 0.0
    for g, d, a, b in _cases(11 + model, 240):
        ref, F, scale = _reference(model, g, d, a, b)
        R, _ = oracle.polar(F)
        q = _quaternion(R).astype(np.float32)            # the float32 estimate of the passes
        f = ff(model, g, d, a, b, q)
        worst = max(worst, np.abs(f - ref).max() / scale)
        # the same with float32 inputs (low words zero): the bound must see it
        g32 = g.astype(np.float32).astype(np.float64)
        d32 = d.astype(np.float32).astype(np.float64)
        f32 = ff(model, g32, d32, float(np.float32(a)), float(np.float32(b)), q)
        float32_worst = max(float32_worst, np.abs(f32 - ref).max() / scale)
    print(f"model {model}: float-float {worst:.2e}, float32 inputs {float32_worst:.2e} of the term scale")
    assert worst <= TOL
    assert float32_worst > 1000 * TOL


def test_a_perturbed_quaternion_is_refined_away(ff):
    """The rotation is refined from the estimate: a quaternion a few float32
    ulps off (the device's estimate is accurate to a few ulps) gives the same
    force to the float-float bound."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for g, d, a, b in _cases(3, 120):
        ref, F, scale = _reference(0, g, d, a, b)
        R, _ = oracle.polar(F)
        q = (_quaternion(R) * (1.0 + 4e-7 * rng.uniform(-1, 1, 4))).astype(np.float32)
        worst = max(worst, np.abs(ff(0, g, d, a, b, q) - ref).max() / scale)
    assert worst <= TOL
