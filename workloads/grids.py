"""Five-tetrahedra-per-cell box grids.

The paper's box examples (Table 1: 32K/150K, 260K/1250K, 2097K/10242K vertices/
elements with K = 1024) match (n+1)^3 vertices and 5 n^3 tetrahedra, i.e. each
cube cell split into one central tetrahedron and four corner tetrahedra.  The
split alternates with the cell parity so that the face diagonals of
neighbouring cells agree and the mesh is conforming.
"""

import numpy as np

# Local cube corners (a, b, c) in {0,1}^3.  For an even cell the central
# tetrahedron uses the odd-parity corners and each even-parity corner is the
# apex of one corner tetrahedron together with its three axis neighbours.  An
# odd cell swaps the roles.  Central tetrahedron first, then the four corner
# tetrahedra.
_EVEN_CELL = (
    ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)),
    ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((1, 1, 0), (0, 1, 0), (1, 0, 0), (1, 1, 1)),
    ((1, 0, 1), (0, 0, 1), (1, 1, 1), (1, 0, 0)),
    ((0, 1, 1), (1, 1, 1), (0, 0, 1), (0, 1, 0)),
)
_ODD_CELL = (
    ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)),
    ((1, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1)),
    ((0, 1, 0), (1, 1, 0), (0, 0, 0), (0, 1, 1)),
    ((0, 0, 1), (1, 0, 1), (0, 1, 1), (0, 0, 0)),
    ((1, 1, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)),
)


def _orient(template):
    """Order each template's corners so the integer corner triple product is
    positive (swap the last two corners otherwise)."""
    out = []
    for tet in template:
        p = np.array(tet, dtype=np.int64)
        e = p[1:] - p[0]
        if int(np.linalg.det(e.astype(np.float64)).round()) < 0:
            tet = (tet[0], tet[1], tet[3], tet[2])
        out.append(tet)
    return tuple(out)


_TEMPLATES = (_orient(_EVEN_CELL), _orient(_ODD_CELL))


def grid_vertex_id(i, j, k, nx, ny):
    """Vertex id of lattice point (i, j, k): x fastest, then y, then z."""
    return (k * (ny + 1) + j) * (nx + 1) + i


def box_grid(nx: int, ny: int, nz: int, h: float, origin=(0.0, 0.0, 0.0)):
    """Rest positions X [(nx+1)(ny+1)(nz+1), 3] (float64) and tetrahedra
    [5 nx ny nz, 4] (int32) of a box of nx x ny x nz cubic cells of side h.

    Tetrahedra are listed cell by cell in lattice order (x fastest), five per
    cell, central one first.
    """
    ii, jj, kk = np.meshgrid(
        np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij"
    )
    order = np.lexsort((ii.ravel(), jj.ravel(), kk.ravel()))
    lat = np.stack([ii.ravel()[order], jj.ravel()[order], kk.ravel()[order]], 1)
    X = lat.astype(np.float64) * h + np.asarray(origin, dtype=np.float64)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    corder = np.lexsort((ci.ravel(), cj.ravel(), ck.ravel()))
    cells = np.stack([ci.ravel()[corder], cj.ravel()[corder], ck.ravel()[corder]], 1)
    parity = cells.sum(1) % 2
    ncell = cells.shape[0]
    tets = np.empty((ncell, 5, 4), dtype=np.int64)
    for p in (0, 1):
        sel = parity == p
        c = cells[sel]
        for t, tet in enumerate(_TEMPLATES[p]):
            for q, (a, b, cc) in enumerate(tet):
                tets[sel, t, q] = grid_vertex_id(c[:, 0] + a, c[:, 1] + b, c[:, 2] + cc, nx, ny)
    return X, tets.reshape(-1, 4).astype(np.int32)
