"""Python face of the PBNG C ABI: one ``Mesh`` per pbng_mesh handle.

Host arrays go in as numpy arrays; the iterate u = x - X is a float32 CUDA
tensor [nv, 3] owned by the caller (PyTorch provides the memory and the
stream).  Methods map one-to-one onto pbng_* entry points.
"""

import ctypes

import numpy as np

from ._lib import (ACCEL, MODEL, ORDER, PRECISION, PbngNewtonInfo, PbngParams, PbngProfile, PbngSchedule, PbngSolveInfo,
                   check, load)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def default_params(**kw):
    """pbng_default_params, then overrides: model ('corotated'|'neohookean'|
    'stable_neohookean'), accel ('none'|'chebyshev'|'sor'), precision
    ('fp32'|'compensated'|'extended'|'auto'), omega, rho, gamma, step, skip_tol, residual_every,
    resume, kernel_path, colour_order ('forward'|'symmetric')."""
    p = PbngParams()
    load().pbng_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "accel":
            v = ACCEL[v] if isinstance(v, str) else int(v)
        elif k == "precision":
            v = PRECISION[v] if isinstance(v, str) else int(v)
        elif k == "model":
            v = MODEL[v] if isinstance(v, str) else int(v)
        elif k == "colour_order":
            v = ORDER[v] if isinstance(v, str) else int(v)
        setattr(p, k, v)
    return p


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_u(u, nv):
    import torch
    if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float32
            and u.is_contiguous() and tuple(u.shape) == (nv, 3)):
        raise ValueError(f"u must be a contiguous float32 CUDA tensor of shape ({nv}, 3)")


def measure_fp32_peak(stream=None):
    """pbng_measure_fp32_peak: FP32 FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double()
    check(load().pbng_measure_fp32_peak(_stream_ptr(stream), ctypes.byref(out)), "pbng_measure_fp32_peak")
    return out.value


class Mesh:
    """A pbng_mesh handle (pbng_create_mesh / pbng_destroy)."""

    def __init__(self, X, tets, young, poisson, mesh_id=None, stream=None):
        L = load()
        self.X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        self.nv, self.ne = self.X.shape[0], self.tets.shape[0]
        young = np.ascontiguousarray(np.broadcast_to(young, (self.ne,)), dtype=np.float64)
        poisson = np.ascontiguousarray(np.broadcast_to(poisson, (self.ne,)), dtype=np.float64)
        mid = None if mesh_id is None else np.ascontiguousarray(mesh_id, dtype=np.int32)
        self._stream = _stream_ptr(stream)
        h = ctypes.c_void_p()
        st = L.pbng_create_mesh(_dptr(self.X), self.nv, _iptr(self.tets), self.ne, _dptr(young),
                                _dptr(poisson), None if mid is None else _iptr(mid), self._stream,
                                ctypes.byref(h))
        check(st, "pbng_create_mesh")
        self.h = h
        self.ncomp = L.pbng_num_components(self.h)
        self.dirichlet = np.zeros(0, np.int32)

    @classmethod
    def from_problem(cls, p, stream=None, mesh_id=None):
        m = cls(p.X, p.tets, p.young, p.poisson, mesh_id=mesh_id, stream=stream)
        m.set_constraints(p.dirichlet, p.x0[p.dirichlet], p.spr_idx, p.spr_target, p.spr_k,
                          p.plane, p.k_contact, p.body_accel, p.density)
        return m

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            load().pbng_destroy(h)
            self.h = None

    def set_constraints(self, dir_idx=None, dir_xyz=None, spr_idx=None, spr_target=None,
                        spr_k=None, plane=None, k_contact=0.0, body_accel=None, density=None):
        di = np.ascontiguousarray(np.zeros(0) if dir_idx is None else dir_idx, dtype=np.int32)
        dx = np.ascontiguousarray(np.zeros((0, 3)) if dir_xyz is None else dir_xyz, dtype=np.float64)
        si = np.ascontiguousarray(np.zeros(0) if spr_idx is None else spr_idx, dtype=np.int32)
        stg = np.ascontiguousarray(np.zeros((0, 3)) if spr_target is None else spr_target, dtype=np.float64)
        sk = np.ascontiguousarray(np.zeros(0) if spr_k is None else spr_k, dtype=np.float64)
        pl = None if plane is None else np.ascontiguousarray(plane, dtype=np.float64)
        ba = None if body_accel is None else np.ascontiguousarray(body_accel, dtype=np.float64)
        de = None if density is None else np.ascontiguousarray(np.broadcast_to(density, (self.ne,)), dtype=np.float64)
        st = load().pbng_set_constraints(
            self.h, _iptr(di), _dptr(dx), len(di), _iptr(si), _dptr(stg), _dptr(sk), len(si),
            None if pl is None else _dptr(pl), float(k_contact),
            None if ba is None else _dptr(ba), None if de is None else _dptr(de))
        check(st, "pbng_set_constraints", self.h)
        self.dirichlet = di.copy()

    def set_body_accel(self, accel, density=None):
        """pbng_set_body_accel: accel [ncomp, 3] (host), density [ne] or None."""
        acc = np.ascontiguousarray(accel, dtype=np.float64).reshape(-1, 3)
        if acc.shape[0] != self.ncomp:
            raise ValueError("one acceleration per component")
        de = None if density is None else np.ascontiguousarray(np.broadcast_to(density, (self.ne,)), dtype=np.float64)
        check(load().pbng_set_body_accel(self.h, _dptr(acc), None if de is None else _dptr(de)),
              "pbng_set_body_accel", self.h)

    def set_material(self, young, poisson):
        """pbng_set_material (per-tet E and nu, host arrays)."""
        young = np.ascontiguousarray(np.broadcast_to(young, (self.ne,)), dtype=np.float64)
        poisson = np.ascontiguousarray(np.broadcast_to(poisson, (self.ne,)), dtype=np.float64)
        check(load().pbng_set_material(self.h, _dptr(young), _dptr(poisson)), "pbng_set_material", self.h)

    def adjoint(self, u_eq, dLdu, rel_tol=1e-6, max_sweeps=100000, params=None, raise_on_status=True):
        """pbng_adjoint: returns (status, dL/dlogE [ne], dL/dx_D [nd, 3], sweeps, rel residual)."""
        import torch
        _check_u(u_eq, self.nv)
        _check_u(dLdu, self.nv)
        p = params if params is not None else default_params()
        dE = torch.empty(self.ne, dtype=torch.float32, device=u_eq.device)
        dD = torch.empty((max(1, len(self.dirichlet)), 3), dtype=torch.float32, device=u_eq.device)
        sweeps = ctypes.c_int32()
        rel = ctypes.c_double()
        st = load().pbng_adjoint(self.h, ctypes.c_void_p(u_eq.data_ptr()), ctypes.c_void_p(dLdu.data_ptr()),
                                 ctypes.c_void_p(dE.data_ptr()),
                                 ctypes.c_void_p(dD.data_ptr()) if len(self.dirichlet) else None,
                                 float(rel_tol), int(max_sweeps), ctypes.byref(p), ctypes.byref(sweeps),
                                 ctypes.byref(rel))
        if raise_on_status:
            check(st, "pbng_adjoint", self.h)
        return st, dE, dD[:len(self.dirichlet)], sweeps.value, rel.value

    def colouring(self):
        col = np.zeros(self.nv, np.int32)
        n = ctypes.c_int32()
        check(load().pbng_get_colouring(self.h, _iptr(col), ctypes.byref(n)), "pbng_get_colouring", self.h)
        return col, n.value

    def sweep(self, u, nsweeps, params=None, want_residual=False):
        """pbng_sweep in place on u; returns the relative residuals (or None)."""
        _check_u(u, self.nv)
        p = params if params is not None else default_params()
        out = np.zeros(self.ncomp) if want_residual else None
        st = load().pbng_sweep(self.h, ctypes.c_void_p(u.data_ptr()), int(nsweeps), ctypes.byref(p),
                               None if out is None else _dptr(out))
        check(st, "pbng_sweep", self.h)
        return out

    def sweep_host(self, u_host, nsweeps, params=None, want_residual=False):
        """pbng_sweep_host in place on a host float32 [nv, 3] array or CPU
        tensor (pinned memory for asynchronous copies); returns the absolute
        residual norms per component (or None)."""
        import torch
        if isinstance(u_host, torch.Tensor):
            if u_host.is_cuda or u_host.dtype != torch.float32 or not u_host.is_contiguous() \
                    or tuple(u_host.shape) != (self.nv, 3):
                raise ValueError(f"u_host must be a contiguous float32 host tensor of shape ({self.nv}, 3)")
            ptr = u_host.data_ptr()
        else:
            if not (isinstance(u_host, np.ndarray) and u_host.dtype == np.float32 and u_host.flags["C_CONTIGUOUS"]
                    and u_host.shape == (self.nv, 3)):
                raise ValueError(f"u_host must be a C-contiguous float32 array of shape ({self.nv}, 3)")
            ptr = u_host.ctypes.data
        p = params if params is not None else default_params()
        out = np.zeros(self.ncomp) if want_residual else None
        st = load().pbng_sweep_host(self.h, ctypes.c_void_p(ptr), int(nsweeps), ctypes.byref(p),
                                    None if out is None else _dptr(out))
        check(st, "pbng_sweep_host", self.h)
        return out

    def solve(self, u, rel_tol, max_sweeps, params=None, raise_on_status=True):
        """pbng_solve in place on u; returns (status, sweeps, rel_residuals)."""
        _check_u(u, self.nv)
        p = params if params is not None else default_params()
        sweeps = ctypes.c_int32()
        out = np.zeros(self.ncomp)
        st = load().pbng_solve(self.h, ctypes.c_void_p(u.data_ptr()), float(rel_tol), int(max_sweeps),
                               ctypes.byref(p), ctypes.byref(sweeps), _dptr(out))
        if raise_on_status:
            check(st, "pbng_solve", self.h)
        return st, sweeps.value, out

    def set_weak_constraints(self, idx, w, kn, kt, normal, recolour=False):
        """pbng_set_weak_constraints: idx, w [nc, 8] (side 0 = columns 0..3,
        side 1 = 4..7, idx -1 unused), kn, kt [nc], normal [nc, 3]."""
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 8)
        nc = idx.shape[0]
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(nc, 8)
        kn = np.ascontiguousarray(np.broadcast_to(kn, (nc,)), dtype=np.float64)
        kt = np.ascontiguousarray(np.broadcast_to(kt, (nc,)), dtype=np.float64)
        nrm = np.ascontiguousarray(np.broadcast_to(normal, (nc, 3)), dtype=np.float64)
        check(load().pbng_set_weak_constraints(self.h, nc, _iptr(idx), _dptr(w), _dptr(kn), _dptr(kt), _dptr(nrm),
                                               1 if recolour else 0), "pbng_set_weak_constraints", self.h)

    def set_inertia(self, dt, density=None):
        """pbng_set_inertia: backward Euler with lumped masses (dt <= 0: quasistatic)."""
        de = None if density is None else np.ascontiguousarray(np.broadcast_to(density, (self.ne,)), dtype=np.float64)
        check(load().pbng_set_inertia(self.h, float(dt), None if de is None else _dptr(de)), "pbng_set_inertia",
              self.h)

    def step(self, u, u_prev, nsweeps, params=None, rel_tol=0.0, raise_on_status=True):
        """pbng_step: one backward-Euler step in place (u: u^n -> u^{n+1},
        u_prev: u^{n-1} -> u^n).  Returns (status, sweeps, rel_residuals)."""
        _check_u(u, self.nv)
        _check_u(u_prev, self.nv)
        p = params if params is not None else default_params()
        sweeps = ctypes.c_int32()
        out = np.zeros(self.ncomp)
        st = load().pbng_step(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u_prev.data_ptr()),
                              int(nsweeps), float(rel_tol), ctypes.byref(p), ctypes.byref(sweeps), _dptr(out))
        if raise_on_status:
            check(st, "pbng_step", self.h)
        return st, sweeps.value, out

    def set_dirichlet_targets(self, dir_xyz):
        """pbng_set_dirichlet_targets (positions in the order of set_constraints' dir_idx)."""
        dx = np.ascontiguousarray(dir_xyz, dtype=np.float64).reshape(-1, 3)
        if dx.shape[0] != len(self.dirichlet):
            raise ValueError("one target per clamped vertex")
        check(load().pbng_set_dirichlet_targets(self.h, _dptr(dx)), "pbng_set_dirichlet_targets", self.h)

    def force(self, u, params=None):
        """pbng_force: f(u) + f^ext as a float32 CUDA tensor [nv, 3] (zero at clamped rows)."""
        import torch
        _check_u(u, self.nv)
        out = torch.empty_like(u)
        p = params if params is not None else default_params()
        check(load().pbng_force(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.byref(p),
                                ctypes.c_void_p(out.data_ptr())), "pbng_force", self.h)
        return out

    def hessian_apply(self, u, direction, params=None):
        """pbng_hessian_apply: H(u) direction on free rows (zero at clamped rows)."""
        import torch
        _check_u(u, self.nv)
        _check_u(direction, self.nv)
        out = torch.empty_like(u)
        p = params if params is not None else default_params()
        check(load().pbng_hessian_apply(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(direction.data_ptr()),
                                        ctypes.byref(p), ctypes.c_void_p(out.data_ptr())),
              "pbng_hessian_apply", self.h)
        return out

    def newton_cg(self, u, rel_tol, max_newton=50, max_cg=1000, cg_tol=0.1, params=None, raise_on_status=True):
        """pbng_newton_cg in place on u; returns (status, info dict)."""
        _check_u(u, self.nv)
        p = params if params is not None else default_params()
        info = PbngNewtonInfo()
        st = load().pbng_newton_cg(self.h, ctypes.c_void_p(u.data_ptr()), float(rel_tol), int(max_newton),
                                   int(max_cg), float(cg_tol), ctypes.byref(p), ctypes.byref(info))
        if raise_on_status:
            check(st, "pbng_newton_cg", self.h)
        return st, {k: getattr(info, k) for k, _ in PbngNewtonInfo._fields_}

    def solve_info(self):
        """pbng_get_solve_info of the last solve as a dict."""
        i = PbngSolveInfo()
        check(load().pbng_get_solve_info(self.h, ctypes.byref(i)), "pbng_get_solve_info", self.h)
        out = {k: getattr(i, k) for k, _ in PbngSolveInfo._fields_}
        n = i.nevents
        out["event_sweep"] = list(i.event_sweep)[:n]
        out["event_rho"] = list(i.event_rho)[:n]
        return out

    def residual(self, u):
        """pbng_residual: absolute FP64 residual norms per component."""
        _check_u(u, self.nv)
        out = np.zeros(self.ncomp)
        check(load().pbng_residual(self.h, ctypes.c_void_p(u.data_ptr()), _dptr(out)), "pbng_residual", self.h)
        return out

    def get_state(self):
        """pbng_get_state: the iteration checkpoint as bytes."""
        n = ctypes.c_size_t()
        check(load().pbng_get_state(self.h, None, ctypes.byref(n)), "pbng_get_state", self.h)
        buf = ctypes.create_string_buffer(n.value)
        check(load().pbng_get_state(self.h, buf, ctypes.byref(n)), "pbng_get_state", self.h)
        return buf.raw[:n.value]

    def set_state(self, blob):
        """pbng_set_state: restore a checkpoint taken on an identical mesh."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        check(load().pbng_set_state(self.h, buf, len(blob)), "pbng_set_state", self.h)

    @staticmethod
    def _schedule_dict(s):
        n = min(s.ncolours, len(s.ctas_per_sm))
        return {"ncolours": s.ncolours, "ctas_per_sm": list(s.ctas_per_sm[:n]), "blocked": list(s.blocked[:n]),
                "balanced": list(s.balanced[:n]),
                "default_ms_per_sweep": s.default_ms_per_sweep, "tuned_ms_per_sweep": s.tuned_ms_per_sweep,
                "candidates": s.candidates}

    def schedule(self):
        """pbng_get_schedule as a dict (per-colour ctas_per_sm and blocked)."""
        s = PbngSchedule()
        check(load().pbng_get_schedule(self.h, ctypes.byref(s)), "pbng_get_schedule", self.h)
        return self._schedule_dict(s)

    def set_schedule(self, ctas_per_sm, blocked, params=None, balanced=None):
        """pbng_set_schedule from per-colour lists."""
        s = PbngSchedule()
        s.ncolours = len(ctas_per_sm)
        bal = balanced if balanced is not None else [0] * len(ctas_per_sm)
        for c, (a, b, g) in enumerate(zip(ctas_per_sm, blocked, bal)):
            s.ctas_per_sm[c] = int(a)
            s.blocked[c] = int(b)
            s.balanced[c] = int(g)
        p = params if params is not None else default_params()
        check(load().pbng_set_schedule(self.h, ctypes.byref(p), ctypes.byref(s)), "pbng_set_schedule", self.h)

    def autotune(self, u, reps=10, params=None):
        """pbng_autotune on a scratch copy of u; returns the chosen schedule."""
        _check_u(u, self.nv)
        s = PbngSchedule()
        p = params if params is not None else default_params()
        check(load().pbng_autotune(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.byref(p), int(reps),
                                   ctypes.byref(s)), "pbng_autotune", self.h)
        return self._schedule_dict(s)

    def test_set_copy_shortfall(self, nbytes):
        """pbng_test_set_copy_shortfall: make each warp's first record-copy wait
        of the ring passes run out (test hook; 0 restores normal operation)."""
        check(load().pbng_test_set_copy_shortfall(self.h, int(nbytes)), "pbng_test_set_copy_shortfall", self.h)

    def set_profiling(self, enable=True):
        """pbng_set_profiling: per-launch event timing of the library's kernels."""
        check(load().pbng_set_profiling(self.h, 1 if enable else 0), "pbng_set_profiling", self.h)

    def profile(self):
        """pbng_get_profile as a dict."""
        pr = PbngProfile()
        check(load().pbng_get_profile(self.h, ctypes.byref(pr)), "pbng_get_profile", self.h)
        return {k: getattr(pr, k) for k, _ in PbngProfile._fields_ if k != "reserved"}
