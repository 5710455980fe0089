"""Synthetic quasistatic problems on box grids.

The paper's scenes (muscle meshes, dropped shapes) are not available; these
seeded box problems stand in for its block examples (stretch/twist blocks,
the bar under gravity, weak-constraint springs and collision contact) with the
paper's material values (E = 1e5, nu = 0.3, density 1000).  Each builder
returns plain arrays; no PBNG arithmetic happens here.
"""

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .grids import box_grid
from .rng import standard_normal, uniform01


@dataclass
class Problem:
    name: str
    X: np.ndarray                      # [nv, 3] float64 rest positions
    tets: np.ndarray                   # [ne, 4] int32
    young: np.ndarray                  # [ne] float64
    poisson: np.ndarray                # [ne] float64
    dirichlet: np.ndarray              # [nd] int32 clamped vertex ids (sorted)
    x0: np.ndarray                     # [nv, 3] float64 initial positions (targets on clamped ids)
    body_accel: Optional[np.ndarray] = None   # [3] float64 body acceleration
    density: Optional[np.ndarray] = None      # [ne] float64 rest density
    spr_idx: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    spr_target: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    spr_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    plane: Optional[np.ndarray] = None        # [4] = (n, d): contact when n.x < d
    k_contact: float = 0.0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.X.shape[0])

    @property
    def ne(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_free(self) -> int:
        return self.nv - int(self.dirichlet.shape[0])

    def dirichlet_mask(self) -> np.ndarray:
        m = np.zeros(self.nv, dtype=np.uint8)
        m[self.dirichlet] = 1
        return m


def _twist_field(X, centre, angle, stretch, height):
    """Rotation about the z axis through ``centre`` by angle*z/height plus a
    z-translation stretch*z/height: the smooth extension of a twisted and
    stretched top face to the whole block."""
    t = (X[:, 2] - X[:, 2].min()) / height
    th = angle * t
    c, s = np.cos(th), np.sin(th)
    dx = X[:, 0] - centre[0]
    dy = X[:, 1] - centre[1]
    out = X.copy()
    out[:, 0] = centre[0] + c * dx - s * dy
    out[:, 1] = centre[1] + s * dx + c * dy
    out[:, 2] = X[:, 2] + stretch * t
    return out


def twist_block(n: int = 10, angle_deg: float = 90.0, stretch: float = 0.3,
                young: float = 1e5, poisson: float = 0.3) -> Problem:
    """Unit cube of n^3 cells; bottom face clamped at rest, top face rotated
    by ``angle_deg`` about the vertical centre line and lifted by ``stretch``.
    The initial guess applies the twist and stretch linearly in z."""
    h = 1.0 / n
    X, tets = box_grid(n, n, n, h)
    z = X[:, 2]
    bottom = np.flatnonzero(np.isclose(z, 0.0))
    top = np.flatnonzero(np.isclose(z, 1.0))
    dirichlet = np.union1d(bottom, top).astype(np.int32)
    x0 = _twist_field(X, (0.5, 0.5), np.deg2rad(angle_deg), stretch, 1.0)
    ne = tets.shape[0]
    return Problem(
        name=f"twist_{n}", X=X, tets=tets,
        young=np.full(ne, young), poisson=np.full(ne, poisson),
        dirichlet=dirichlet, x0=x0,
        meta=dict(angle_deg=angle_deg, stretch=stretch, cells=(n, n, n)),
    )


def gravity_sag(n: int = 64, young: float = 1e5, poisson: float = 0.45,
                density: float = 1000.0, g: float = 9.8) -> Problem:
    """Unit cube of n^3 cells clamped on the face x = 0, loaded by gravity
    (0, 0, -g) with the given density; starts from rest."""
    h = 1.0 / n
    X, tets = box_grid(n, n, n, h)
    dirichlet = np.flatnonzero(np.isclose(X[:, 0], 0.0)).astype(np.int32)
    ne = tets.shape[0]
    return Problem(
        name=f"sag_{n}", X=X, tets=tets,
        young=np.full(ne, young), poisson=np.full(ne, poisson),
        dirichlet=dirichlet, x0=X.copy(),
        body_accel=np.array([0.0, 0.0, -g]), density=np.full(ne, density),
        meta=dict(cells=(n, n, n)),
    )


def contact_bar(nx: int = 40, ny: int = 40, nz: int = 200, h: float = 0.005,
                seed: int = 20230615, log_sigma: float = 0.5, poisson: float = 0.4,
                spring_frac: float = 0.02, k_spring: float = 1e4,
                pull: float = 0.05, target_sigma: float = 0.02,
                k_contact: float = 1e8) -> Problem:
    """Bar of nx x ny x nz cells resting on the plane z = 0, no clamped
    vertices.  Per-tet Young's modulus is lognormal around 1e5; a random
    ``spring_frac`` of the vertices is tied by zero-rest-length springs to
    targets pulled ``pull`` below the rest position plus N(0, target_sigma^2)
    noise, which presses the bar into the contact plane."""
    X, tets = box_grid(nx, ny, nz, h)
    ne, nv = tets.shape[0], X.shape[0]
    young = np.exp(np.log(1e5) + log_sigma * standard_normal(seed, ne))
    ns = int(round(spring_frac * nv))
    order = np.argsort(uniform01(seed + 1, nv), kind="stable")
    spr_idx = np.sort(order[:ns]).astype(np.int32)
    noise = target_sigma * standard_normal(seed + 2, 3 * ns).reshape(ns, 3)
    spr_target = X[spr_idx] + np.array([0.0, 0.0, -pull]) + noise
    return Problem(
        name=f"bar_{nx}x{ny}x{nz}", X=X, tets=tets,
        young=young, poisson=np.full(ne, poisson),
        dirichlet=np.zeros(0, np.int32), x0=X.copy(),
        spr_idx=spr_idx, spr_target=spr_target, spr_k=np.full(ns, k_spring),
        plane=np.array([0.0, 0.0, 1.0, 0.0]), k_contact=k_contact,
        seed=seed, meta=dict(cells=(nx, ny, nz)),
    )


def batched_blocks(count: int = 256, side_lo: int = 8, side_hi: int = 32,
                   seed: int = 4242, max_stretch: float = 0.4,
                   max_twist_deg: float = 36.0) -> List[Problem]:
    """``count`` unit cubes with side s ~ U{side_lo..side_hi} cells, bottom
    clamped at rest, top clamped to a seeded stretch in [0, max_stretch] and
    twist in [-max_twist_deg, max_twist_deg]; initial guess = the boundary
    map extended linearly in z."""
    u = uniform01(seed, 3 * count).reshape(count, 3)
    sides = side_lo + np.minimum((u[:, 0] * (side_hi - side_lo + 1)).astype(int),
                                 side_hi - side_lo)
    out = []
    for m in range(count):
        s = int(sides[m])
        stretch = max_stretch * u[m, 1]
        twist = max_twist_deg * (2.0 * u[m, 2] - 1.0)
        p = twist_block(s, twist, stretch)
        p.name = f"batch{m}_{s}"
        p.seed = seed
        p.meta.update(index=m)
        out.append(p)
    return out


def adjoint_block(n: int = 48, young: float = 1e5, poisson: float = 0.3) -> Problem:
    """Unit cube of n^3 cells with its bottom face z = 0 clamped (at rest;
    load cases move it) and gravity of density 1000."""
    h = 1.0 / n
    X, tets = box_grid(n, n, n, h)
    dirichlet = np.flatnonzero(np.isclose(X[:, 2], 0.0)).astype(np.int32)
    ne = tets.shape[0]
    return Problem(
        name=f"adjoint_{n}", X=X, tets=tets,
        young=np.full(ne, young), poisson=np.full(ne, poisson),
        dirichlet=dirichlet, x0=X.copy(),
        body_accel=np.array([0.0, 0.0, -9.8]), density=np.full(ne, 1000.0),
        meta=dict(cells=(n, n, n)),
    )


def adjoint_load_cases(p: Problem, count: int = 32, seed: int = 777,
                       max_rot_deg: float = 5.0, max_trans: float = 0.02, g: float = 9.8,
                       full_body: bool = False):
    """Seeded load cases for ``adjoint_block``: per case a rigid motion of the
    clamped face (rotation angle <= max_rot_deg about a random axis through
    the face centre, translation <= max_trans) and a gravity direction in the
    lower hemisphere.  Returns (x [count, nd, 3], body_accel [count, 3]);
    with full_body the rigid motion is applied to every vertex (x [count,
    nv, 3]), the boundary map extended to the whole block as an initial
    guess."""
    u = uniform01(seed, 9 * count).reshape(count, 9)
    Xd = p.X if full_body else p.X[p.dirichlet]
    centre = np.array([0.5, 0.5, 0.0])
    xds, accs = [], []
    for c in range(count):
        ax = u[c, 0:3] * 2.0 - 1.0
        ax /= max(np.linalg.norm(ax), 1e-12)
        ang = np.deg2rad(max_rot_deg) * u[c, 3]
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        Q = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)
        tr = max_trans * (u[c, 4:7] * 2.0 - 1.0) / np.sqrt(3.0)
        xds.append((Xd - centre) @ Q.T + centre + tr)
        phi = 2 * np.pi * u[c, 7]
        cz = -u[c, 8]                       # lower hemisphere: z component <= 0
        sz = np.sqrt(max(0.0, 1.0 - cz * cz))
        accs.append(g * np.array([sz * np.cos(phi), sz * np.sin(phi), cz]))
    return np.stack(xds), np.stack(accs)


def concat_problems(problems: List[Problem], spacing: float = 0.0):
    """One batch of independent meshes: vertex, tet and constraint arrays
    concatenated with offsets, plus the component id of every vertex.
    Returns (Problem, mesh_id, vertex_offsets).  Body forces must agree."""
    offs = np.cumsum([0] + [p.nv for p in problems])
    shift = lambda k: np.array([spacing * k, 0.0, 0.0])
    X = np.vstack([p.X + shift(k) for k, p in enumerate(problems)])
    x0 = np.vstack([p.x0 + shift(k) for k, p in enumerate(problems)])
    tets = np.vstack([p.tets + offs[k] for k, p in enumerate(problems)]).astype(np.int32)
    dirichlet = np.concatenate([p.dirichlet + offs[k] for k, p in enumerate(problems)]).astype(np.int32)
    spr_idx = np.concatenate([p.spr_idx + offs[k] for k, p in enumerate(problems)]).astype(np.int32)
    spr_target = np.vstack([p.spr_target + shift(k) for k, p in enumerate(problems)])
    accels = {None if p.body_accel is None else tuple(p.body_accel) for p in problems}
    if len(accels) != 1:
        raise ValueError("problems of one batch must share the body acceleration")
    acc = problems[0].body_accel
    dens = None if acc is None else np.concatenate([p.density for p in problems])
    mesh_id = np.concatenate([np.full(p.nv, k, np.int32) for k, p in enumerate(problems)])
    batch = Problem(
        name=f"batch_of_{len(problems)}", X=X, tets=tets,
        young=np.concatenate([p.young for p in problems]),
        poisson=np.concatenate([p.poisson for p in problems]),
        dirichlet=dirichlet, x0=x0, body_accel=acc, density=dens,
        spr_idx=spr_idx, spr_target=spr_target,
        spr_k=np.concatenate([p.spr_k for p in problems]),
        meta=dict(count=len(problems), offsets=offs),
    )
    return batch, mesh_id, offs


def two_blocks_hanging(n_top: int = 4, n_bottom: int = 3, young: float = 1000.0, poisson: float = 0.3,
                       density: float = 10.0, k: float = 1e8, g: float = 9.8) -> Problem:
    """Two unit cubes stacked in z (the "Varying Stiffness" example): the top
    one (z in [1, 2], n_top cells, top face clamped) holds the bottom one
    (z in [0, 1], n_bottom cells, free) through zero-rest-length weak
    constraints, one per vertex of the bottom block's top face, to the point
    of the top block's bottom face at the same position.  That point is
    interpolated with the barycentric weights of a top-block tet with a face
    on z = 1 containing it.  Gravity -g in z, density and E as in the paper's
    example; k_n = k_tau = k.  The constraints are in meta["weak"] as
    (idx [nc, 8], w [nc, 8], kn [nc], kt [nc], normal [nc, 3])."""
    Xa, ta = box_grid(n_top, n_top, n_top, 1.0 / n_top)
    Xa = Xa + np.array([0.0, 0.0, 1.0])
    Xb, tb = box_grid(n_bottom, n_bottom, n_bottom, 1.0 / n_bottom)
    na = Xa.shape[0]
    X = np.vstack([Xa, Xb])
    tets = np.vstack([ta, tb + na]).astype(np.int32)
    dirichlet = np.flatnonzero(np.isclose(X[:, 2], 2.0)).astype(np.int32)
    bottom_faces = ta[np.isclose(Xa[ta][:, :, 2], 1.0).sum(axis=1) == 3]   # tets with a face on z = 1
    TF = Xa[bottom_faces]                                             # [nf, 4, 3]
    MF = np.stack([TF[:, 1] - TF[:, 0], TF[:, 2] - TF[:, 0], TF[:, 3] - TF[:, 0]], axis=2)
    MF_inv = np.linalg.inv(MF)
    idx, w = [], []
    verts = np.flatnonzero(np.isclose(Xb[:, 2], 1.0))
    # candidate tets by barycentric coordinates, vectorised over chunks of
    # binding points; the first containing one, in tet order, is then solved
    # exactly as one system
    cands = []
    for c0 in range(0, len(verts), 64):
        Pc = Xb[verts[c0:c0 + 64]]
        l_all = np.einsum("fij,vfj->vfi", MF_inv, Pc[:, None, :] - TF[None, :, 0])
        lmin = np.minimum(1.0 - l_all.sum(axis=2), l_all.min(axis=2))
        cands.extend(np.flatnonzero(row >= -1e-9) for row in lmin)
    for v, cand in zip(verts, cands):
        P = Xb[v]
        for f in cand:
            t = bottom_faces[f]
            T = Xa[t]
            M = np.column_stack([T[1] - T[0], T[2] - T[0], T[3] - T[0]])
            l123 = np.linalg.solve(M, P - T[0])
            lam = np.concatenate([[1.0 - l123.sum()], l123])
            if lam.min() >= -1e-12:
                lam = np.clip(lam, 0.0, None)
                lam /= lam.sum()
                idx.append([na + v, -1, -1, -1] + [int(i) for i in t])
                w.append([1.0, 0.0, 0.0, 0.0] + list(lam))
                break
        else:
            raise RuntimeError("no top-block tet contains a binding point")
    nc = len(idx)
    ne = tets.shape[0]
    p = Problem(
        name=f"two_blocks_{n_top}_{n_bottom}", X=X, tets=tets,
        young=np.full(ne, young), poisson=np.full(ne, poisson),
        dirichlet=dirichlet, x0=X.copy(),
        body_accel=np.array([0.0, 0.0, -g]), density=np.full(ne, density),
        meta=dict(cells=(n_top, n_bottom)),
    )
    p.meta["weak"] = (np.array(idx, np.int32), np.array(w), np.full(nc, k), np.full(nc, k),
                      np.tile([0.0, 0.0, 1.0], (nc, 1)))
    return p
