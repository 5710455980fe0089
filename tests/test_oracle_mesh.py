"""Pins of the oracle's discretisation (Section "Discretization", Eq.
disc_pe), its external forces and its greedy node colouring (Section
"Coloring and Parallelism", Table 1)."""

import numpy as np
import pytest

import workloads as W
from tests.golden.values import paper_values


def _mesh(oracle_mod, p):
    return oracle_mod.OracleMesh.from_problem(p)


def test_tet_constants(oracle_mod):
    n = 3
    p = W.twist_block(n)
    m = _mesh(oracle_mod, p)
    B, V, mu, lam = m.tet_constants()
    h = 1.0 / n
    assert V.sum() == pytest.approx(1.0, rel=1e-14)
    # Five-tet split: one central tet of volume h^3/3 and four corners of h^3/6.
    assert np.allclose(np.sort(V.reshape(-1, 5), axis=1),
                       np.array([1, 1, 1, 1, 2]) * h ** 3 / 6, rtol=1e-12)
    for e in (0, 7, len(V) - 1):
        Xe = p.X[p.tets[e]]
        Dm = (Xe[1:] - Xe[0]).T
        assert np.allclose(B[e] @ Dm, np.eye(3), atol=1e-12)
    assert np.allclose(mu, 1e5 / 2.6) and np.allclose(lam, 1e5 * 0.3 / (1.3 * 0.4))


def test_gravity_nodal_force(oracle_mod):
    p = W.gravity_sag(4)
    m = _mesh(oracle_mod, p)
    f = m.fext()
    # Total load is rho g times the volume; each vertex carries a quarter of
    # the volume of its incident tets (P1 shape functions integrate to V/4).
    assert f.sum(0) == pytest.approx(np.array([0, 0, -9.8 * 1000.0]), abs=1e-9)
    _, V, _, _ = m.tet_constants()
    share = np.zeros(p.nv)
    np.add.at(share, p.tets.ravel(), np.repeat(V / 4, 4))
    assert np.allclose(f[:, 2], -9800.0 * share, rtol=1e-13)


def _greedy_bruteforce(nv, tets, is_dir):
    """Plain restatement: for each free vertex in ascending id, the least
    colour not yet taken by any other vertex of any tet containing it."""
    col = -np.ones(nv, int)
    tets_of = [[] for _ in range(nv)]
    for e, t in enumerate(tets):
        for v in t:
            tets_of[v].append(e)
    for i in range(nv):
        if is_dir[i]:
            continue
        used = {col[v] for e in tets_of[i] for v in tets[e] if col[v] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


@pytest.mark.parametrize("maker", [lambda: W.twist_block(3), lambda: W.gravity_sag(4),
                                   lambda: W.contact_bar(3, 2, 5, 0.1, spring_frac=0.1)])
def test_colouring_is_greedy_and_valid(oracle_mod, maker):
    p = maker()
    m = _mesh(oracle_mod, p)
    col = m.colours()
    assert np.array_equal(col, _greedy_bruteforce(p.nv, p.tets, p.dirichlet_mask()))
    assert np.all(col[p.dirichlet] == -1)
    for t in p.tets:
        c = col[t][col[t] >= 0]
        assert len(set(c.tolist())) == len(c), "two nodes of one tet share a colour"


def test_table1_five_colours(oracle_mod):
    pv = paper_values()
    for res, key in ((16, "box_res16_particle_colours"), (32, "box_res32_particle_colours")):
        X, tets = W.box_grid(res, res, res, 1.0 / res)
        m = oracle_mod.OracleMesh(X, tets, 1e5, 0.3)
        assert m.ncolours == int(pv[key])
    for n in (3, 5, 8):  # also with clamped faces (two clamped faces leave too few layers below 3 cells)
        assert _mesh(oracle_mod, W.twist_block(n)).ncolours == 5
        assert _mesh(oracle_mod, W.gravity_sag(n)).ncolours == 5
