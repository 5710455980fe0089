"""FP64 PBNG oracle — TEST INFRASTRUCTURE ONLY.

A ctypes wrapper over ``pbng_oracle.cpp``, a plain serial double-precision
restatement of Position-Based Nonlinear Gauss-Seidel (arXiv 2306.09021).
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It imports nothing from the CUDA library and the
CUDA library imports nothing from it.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  lame, svd3, polar, psi, pk1, dpk1, cofactor  pinned (closed forms, numpy/scipy
                                               special cases, finite differences)
  colouring                                    pinned (validity, brute-force greedy,
                                               Table 1's 5 colours on box grids)
  local_system, residual, energy               pinned (FD gradient of the energy,
                                               patch test, rest closed form)
  sweeps (plain)                               pinned (fixed point = Newton
                                               equilibrium, patch test, rotation
                                               invariance, single-vertex Newton)
  sweeps (Chebyshev / SOR)                     pinned (linear-iteration theory on
                                               the linearised sweep: the scaled
                                               Chebyshev polynomial, the closed
                                               form of the two-step recurrence)
  sweeps (symmetric colour order)              pinned (the linearised sweep is
                                               self-adjoint in the Hessian's inner
                                               product with spectrum in [0, 1);
                                               Chebyshev polynomial error)
  newton, hessian_dense                        pinned (FD of the residual)
  adjoint_dense                                pinned (FD of the loss)
"""

import ctypes
import os

import numpy as np

from .build import build as _build

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        sig = {
            "ora_lame": (None, [ctypes.c_double, ctypes.c_double, _D, _D]),
            "ora_svd3": (ctypes.c_int, [_D, _D, _D, _D]),
            "ora_polar": (None, [_D, _D, _D]),
            "ora_psi": (ctypes.c_double, [_D, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
            "ora_pk1": (None, [_D, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]),
            "ora_dpk1": (None, [_D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]),
            "ora_set_model": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
            "ora_set_colour_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
            "ora_set_inertia": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, _D, _D]),
            "ora_lumped_mass": (None, [ctypes.c_void_p, _D]),
            "ora_set_weak_constraints": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _I, _D, _D, _D, _D,
                                                        ctypes.c_int]),
            "ora_cofactor": (None, [_D, _D]),
            "ora_modified_density_hessian": (None, [_D, ctypes.c_double, ctypes.c_double, _D]),
            "ora_create": (ctypes.c_void_p, [ctypes.c_int, _D, ctypes.c_int, _I, _D, _D, _U8,
                                             _D, _D, ctypes.c_int, _I, _D, _D, _D,
                                             ctypes.c_double, _I]),
            "ora_destroy": (None, [ctypes.c_void_p]),
            "ora_num_colours": (ctypes.c_int, [ctypes.c_void_p]),
            "ora_get_colours": (None, [ctypes.c_void_p, _I]),
            "ora_get_tet_constants": (None, [ctypes.c_void_p, _D, _D, _D, _D]),
            "ora_get_fext": (None, [ctypes.c_void_p, _D]),
            "ora_local_system": (None, [ctypes.c_void_p, _D, ctypes.c_int, _D, _D]),
            "ora_residual": (ctypes.c_double, [ctypes.c_void_p, _D, _D]),
            "ora_energy": (ctypes.c_double, [ctypes.c_void_p, _D]),
            "ora_sweeps": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, _D]),
            "ora_newton": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_int, _D]),
            "ora_hessian_dense": (None, [ctypes.c_void_p, _D, _D]),
            "ora_adjoint_dense": (ctypes.c_int, [ctypes.c_void_p, _D, _D, _D, _D]),
            "ora_threads_available": (ctypes.c_int, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------- density level
def lame(E, nu):
    mu, lam = ctypes.c_double(), ctypes.c_double()
    lib().ora_lame(E, nu, ctypes.byref(mu), ctypes.byref(lam))
    return mu.value, lam.value


def svd3(F):
    F = _f64(F, (3, 3))
    U, s, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    lib().ora_svd3(_d(F), _d(U), _d(s), _d(V))
    return U, s, V


def polar(F):
    F = _f64(F, (3, 3))
    R, sh = np.zeros((3, 3)), np.zeros(3)
    lib().ora_polar(_d(F), _d(R), _d(sh))
    return R, sh


MODELS = {"corotated": 0, "neohookean": 1, "stable_neohookean": 2}
COLOUR_ORDERS = {"forward": 0, "symmetric": 1}


def _model(model):
    return MODELS[model] if isinstance(model, str) else int(model)


def psi(F, mu, lam, model=0):
    F = _f64(F, (3, 3))
    return lib().ora_psi(_d(F), mu, lam, _model(model))


def pk1(F, mu, lam, model=0):
    F = _f64(F, (3, 3))
    P = np.zeros((3, 3))
    lib().ora_pk1(_d(F), mu, lam, _model(model), _d(P))
    return P


def dpk1(F, dF, mu, lam, model=0):
    F, dF = _f64(F, (3, 3)), _f64(dF, (3, 3))
    dP = np.zeros((3, 3))
    lib().ora_dpk1(_d(F), _d(dF), mu, lam, _model(model), _d(dP))
    return dP


def cofactor(F):
    F = _f64(F, (3, 3))
    C = np.zeros((3, 3))
    lib().ora_cofactor(_d(F), _d(C))
    return C


def modified_density_hessian(F, mu, lam):
    F = _f64(F, (3, 3))
    C = np.zeros((9, 9))
    lib().ora_modified_density_hessian(_d(F), mu, lam, _d(C))
    return C


# ------------------------------------------------------------------ mesh
class OracleMesh:
    """FP64 PBNG on one mesh.  Positions are absolute (x = X + u)."""

    def __init__(self, X, tets, young, poisson, dirichlet_mask=None, body_accel=None,
                 density=None, spr_idx=None, spr_target=None, spr_k=None, plane=None,
                 k_contact=0.0):
        self.X = _f64(X, (-1, 3))
        self.nv = self.X.shape[0]
        self.tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        self.ne = self.tets.shape[0]
        young = _f64(np.broadcast_to(young, (self.ne,)))
        poisson = _f64(np.broadcast_to(poisson, (self.ne,)))
        mask = (np.zeros(self.nv, np.uint8) if dirichlet_mask is None
                else np.ascontiguousarray(dirichlet_mask, dtype=np.uint8))
        self.dir_mask = mask
        ba = None if body_accel is None else _f64(body_accel, (3,))
        dens = None if density is None else _f64(np.broadcast_to(density, (self.ne,)))
        ns = 0 if spr_idx is None else int(len(spr_idx))
        si = np.ascontiguousarray(spr_idx if ns else np.zeros(1), dtype=np.int32)
        st = _f64(spr_target if ns else np.zeros((1, 3)), (-1, 3))
        sk = _f64(spr_k if ns else np.zeros(1))
        pl = None if plane is None else _f64(plane, (4,))
        st_code = ctypes.c_int(0)
        self._keep = (young, poisson, mask, ba, dens, si, st, sk, pl)
        self.h = lib().ora_create(
            self.nv, _d(self.X), self.ne, self.tets.ctypes.data_as(_I), _d(young), _d(poisson),
            mask.ctypes.data_as(_U8), None if ba is None else _d(ba),
            None if dens is None else _d(dens), ns, si.ctypes.data_as(_I), _d(st), _d(sk),
            None if pl is None else _d(pl), float(k_contact), ctypes.byref(st_code))
        if not self.h:
            raise ValueError(f"oracle mesh rejected (status {st_code.value})")

    @classmethod
    def from_problem(cls, p, model=0):
        m = cls(p.X, p.tets, p.young, p.poisson, p.dirichlet_mask(), p.body_accel,
                p.density, p.spr_idx, p.spr_target, p.spr_k, p.plane, p.k_contact)
        m.set_model(model)
        return m

    def set_inertia(self, dt, density, xhat):
        """Backward Euler (Eq. fem_be) with inertial target xhat = 2 x^n - x^{n-1};
        dt <= 0 returns to quasistatics."""
        dens = _f64(np.broadcast_to(density, (self.ne,)))
        xh = _f64(xhat, (-1, 3))
        self._inertia_keep = (dens, xh)
        if lib().ora_set_inertia(self.h, float(dt), _d(dens), _d(xh)) != 0:
            raise ValueError("bad inertia arguments")

    def set_weak_constraints(self, idx, w, kn, kt, normal, recolour=False):
        """General weak constraints: idx, w [nc, 8] (side 0 = columns 0..3,
        side 1 = 4..7, idx -1 unused), kn, kt [nc], normal [nc, 3]."""
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 8)
        nc = idx.shape[0]
        w = _f64(w, (nc, 8)) if nc else np.zeros((0, 8))
        kn = _f64(np.broadcast_to(kn, (nc,))) if nc else np.zeros(0)
        kt = _f64(np.broadcast_to(kt, (nc,))) if nc else np.zeros(0)
        nrm = _f64(np.broadcast_to(normal, (nc, 3))) if nc else np.zeros((0, 3))
        self._wc_keep = (idx, w, kn, kt, nrm)
        if lib().ora_set_weak_constraints(self.h, nc, idx.ctypes.data_as(_I), _d(w), _d(kn), _d(kt), _d(nrm),
                                          1 if recolour else 0) != 0:
            raise ValueError("bad weak constraints")

    def lumped_mass(self):
        out = np.zeros(self.nv)
        lib().ora_lumped_mass(self.h, _d(out))
        return out

    def set_model(self, model):
        """Constitutive model: 0 / 'corotated', 1 / 'neohookean', 2 / 'stable_neohookean'."""
        if lib().ora_set_model(self.h, _model(model)) != 0:
            raise ValueError(f"unknown model {model!r}")

    def __del__(self):
        if getattr(self, "h", None):
            lib().ora_destroy(self.h)
            self.h = None

    @property
    def ncolours(self):
        return lib().ora_num_colours(self.h)

    def colours(self):
        out = np.zeros(self.nv, np.int32)
        lib().ora_get_colours(self.h, out.ctypes.data_as(_I))
        return out

    def tet_constants(self):
        B = np.zeros((self.ne, 3, 3)); V = np.zeros(self.ne)
        mu = np.zeros(self.ne); lam = np.zeros(self.ne)
        lib().ora_get_tet_constants(self.h, _d(B), _d(V), _d(mu), _d(lam))
        return B, V, mu, lam

    def fext(self):
        f = np.zeros((self.nv, 3))
        lib().ora_get_fext(self.h, _d(f))
        return f

    def local_system(self, x, i):
        x = _f64(x, (-1, 3))
        r, A = np.zeros(3), np.zeros((3, 3))
        lib().ora_local_system(self.h, _d(x), int(i), _d(r), _d(A))
        return r, A

    def residual(self, x, vector=False):
        x = _f64(x, (-1, 3))
        r = np.zeros((self.nv, 3))
        n = lib().ora_residual(self.h, _d(x), _d(r))
        return (n, r) if vector else n

    def energy(self, x):
        x = _f64(x, (-1, 3))
        return lib().ora_energy(self.h, _d(x))

    def sweeps(self, x, n, accel="none", omega=1.7, rho=0.95, gamma=1.7, skip_tol=0.0,
               threads=1, history=False, order="forward"):
        """Returns (x_new, status[, residual history]).  order: "forward"
        (colours 0..C-1 per sweep) or "symmetric" (0..C-1, then C-2..0)."""
        if lib().ora_set_colour_order(self.h, COLOUR_ORDERS[order]) != 0:
            raise ValueError(f"unknown colour order {order!r}")
        xx = _f64(x, (-1, 3)).copy()
        code = {"none": 0, "chebyshev": 1, "sor": 2}[accel]
        hist = np.zeros(n + 1) if history else None
        st = lib().ora_sweeps(self.h, _d(xx), int(n), code, omega, rho, gamma, skip_tol,
                              int(threads), None if hist is None else _d(hist))
        return (xx, st, hist) if history else (xx, st)

    def newton(self, x, rel_tol=1e-12, maxit=50):
        xx = _f64(x, (-1, 3)).copy()
        res = ctypes.c_double()
        it = lib().ora_newton(self.h, _d(xx), rel_tol, maxit, ctypes.byref(res))
        return xx, it, res.value

    def hessian(self, x):
        x = _f64(x, (-1, 3))
        H = np.zeros((3 * self.nv, 3 * self.nv))
        lib().ora_hessian_dense(self.h, _d(x), _d(H))
        return H

    def adjoint(self, x, dLdx):
        x = _f64(x, (-1, 3))
        g = _f64(dLdx, (-1, 3))
        nd = int(self.dir_mask.sum())
        dE = np.zeros(self.ne)
        dD = np.zeros((nd, 3))
        st = lib().ora_adjoint_dense(self.h, _d(x), _d(g), _d(dE), _d(dD))
        if st != 0:
            raise RuntimeError("singular Hessian in the dense adjoint")
        return dE, dD


def threads_available(n):
    """Threads the oracle's sweep would use when asked for n."""
    return lib().ora_threads_available(int(n))


def build():
    """Compile the oracle library (used by __graft_entry__.build)."""
    return _build(force=False)
