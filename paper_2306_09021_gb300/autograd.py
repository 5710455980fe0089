"""Differentiable equilibrium: u = u*(log E, x_D) as a torch.autograd.Function.

Forward solves the quasistatic equilibrium with pbng_solve; backward calls
pbng_adjoint, which solves H lambda = dL/du by the same coloured
Gauss-Seidel and returns dL/dlog E (per tet) and dL/dx_D (clamped positions).

Gradients are those of the equilibrium only when both solves reach their
tolerances.  A solve that stops at its sweep limit (PBNG_ENOTCONVERGED)
raises ``NotConvergedError`` unless the model was built with
``allow_unconverged=True``, which turns it into a warning that carries the
relative residual reached.
"""

import warnings

import numpy as np
import torch

from .mesh import Mesh, default_params


PBNG_ENOTCONVERGED = 7


class NotConvergedError(RuntimeError):
    """A forward or adjoint solve ended at its sweep limit above its tolerance."""


def _unconverged(model, what, rel, tol, sweeps):
    msg = (f"{what} stopped after {sweeps} sweeps at relative residual {float(np.max(rel)):.3e} "
           f"(tolerance {tol:.1e}): the gradient is not that of the equilibrium")
    if not model.allow_unconverged:
        raise NotConvergedError(msg)
    warnings.warn(msg, RuntimeWarning, stacklevel=3)


class EquilibriumModel:
    """A mesh with fixed topology, Poisson ratios, springs, contact and body
    forces whose per-tet log Young's modulus and clamped positions are the
    differentiable inputs.  ``model(log_young, x_dirichlet)`` returns the
    equilibrium displacement u [nv, 3] (float32, CUDA).  ``model`` selects the
    energy density (Section "Constitutive Models"); the adjoint always uses the
    forward solve's model.  ``allow_unconverged`` turns a solve that ends at
    its sweep limit from an error into a warning."""

    def __init__(self, problem, mesh_id=None, body_accel=None, rel_tol=1e-6, max_sweeps=200000,
                 adjoint_tol=1e-6, adjoint_max_sweeps=200000, params=None, adjoint_params=None,
                 model="corotated", allow_unconverged=False):
        self.allow_unconverged = bool(allow_unconverged)
        self.p = problem
        self.mesh = Mesh.from_problem(problem, mesh_id=mesh_id)
        self.body_accel = None if body_accel is None else np.asarray(body_accel, dtype=np.float64)
        self.rel_tol, self.max_sweeps = rel_tol, max_sweeps
        self.adjoint_tol, self.adjoint_max_sweeps = adjoint_tol, adjoint_max_sweeps
        # forward: symmetric colour order with automatic Chebyshev rho, moving
        # to extended precision at the float32 floor; adjoint: conjugate
        # gradients preconditioned by the symmetric block Gauss-Seidel sweep,
        # refined with the float-float force (both past float32's floor)
        self.params = params if params is not None else default_params(
            model=model, accel="chebyshev", rho=-1.0, colour_order="symmetric", precision="auto")
        self.adjoint_params = (adjoint_params if adjoint_params is not None
                               else default_params(model=model, accel="cg", colour_order="symmetric",
                                                   precision="auto"))
        self.adjoint_params.model = self.params.model
        self.u_last = None
        self.last_solve = None
        self.last_adjoint = None

    def __call__(self, log_young, x_dirichlet):
        return _Equilibrium.apply(log_young, x_dirichlet, self)

    def _solve(self, log_young, x_dirichlet):
        p, m = self.p, self.mesh
        m.set_material(np.exp(log_young.detach().double().cpu().numpy()), p.poisson)
        xd = x_dirichlet.detach().double().cpu().numpy()
        m.set_constraints(p.dirichlet, xd, p.spr_idx, p.spr_target, p.spr_k, p.plane, p.k_contact,
                          p.body_accel, p.density)
        if self.body_accel is not None:
            m.set_body_accel(self.body_accel, p.density)
        u = self.u_last.clone() if self.u_last is not None else torch.tensor(
            p.x0 - p.X, dtype=torch.float32, device="cuda")
        st, sweeps, rel = m.solve(u, self.rel_tol, self.max_sweeps, self.params, raise_on_status=False)
        if st not in (0, PBNG_ENOTCONVERGED):
            raise RuntimeError(f"equilibrium solve failed with status {st}")
        self.last_solve = (st, sweeps, rel)
        if st == PBNG_ENOTCONVERGED:
            _unconverged(self, "the equilibrium solve", rel, self.rel_tol, sweeps)
        self.u_last = u.clone()
        return u


class _Equilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_young, x_dirichlet, model):
        u = model._solve(log_young, x_dirichlet)
        ctx.model = model
        ctx.save_for_backward(u)
        ctx.dtypes = (log_young.dtype, x_dirichlet.dtype, log_young.device, x_dirichlet.device)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        model = ctx.model
        g = grad_u.detach().to(torch.float32).contiguous()
        st, dE, dD, sweeps, rel = model.mesh.adjoint(u, g, model.adjoint_tol, model.adjoint_max_sweeps,
                                                     model.adjoint_params, raise_on_status=False)
        if st not in (0, PBNG_ENOTCONVERGED):
            raise RuntimeError(f"adjoint solve failed with status {st}")
        model.last_adjoint = (st, sweeps, rel)
        if st == PBNG_ENOTCONVERGED:
            _unconverged(model, "the adjoint solve", rel, model.adjoint_tol, sweeps)
        t_e, t_d, d_e, d_d = ctx.dtypes
        return dE.to(dtype=t_e, device=d_e), dD.to(dtype=t_d, device=d_d), None
