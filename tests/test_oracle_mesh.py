"""Pins of the oracle's levels, node classes, boundary sets and J2 numbering
(oracle/mesh.py), checked against brute-force geometric definitions and
closed-form DOF counts."""
import itertools

import numpy as np
import pytest

from oracle import mesh
from paper_1909_13201_gb300 import inputs as I


def _small(dim=2, n=8, levels=3, seed=3, **kw):
    if dim == 2:
        return I.make_channel_2d(n, levels, 1, seed, **kw)
    return I.make_valve_3d(n, levels, 1, seed)


def test_dof_count_closed_form_config0():
    p = I.make_config(0)
    fine = mesh.build_levels(p)[-1]
    # 2 fields x 2 comps on 33^2 Q2 nodes + 17^2 Q1 nodes + 17 duplicated
    # interface pressures (the band's top edge y = 0.25 is a row of 17 vertices)
    assert fine.n_dofs == 4 * 33 ** 2 + 17 ** 2 + 17 == 4662


@pytest.mark.parametrize("dim", [2, 3])
def test_dof_count_general(dim):
    p = _small(dim, n=8 if dim == 2 else 4, levels=2, bulge=True) if dim == 2 else _small(3, n=4, levels=2)
    for lev in mesh.build_levels(p):
        both = int((lev.q1_has_s & lev.q1_has_f).sum())
        assert lev.n_dofs == 2 * dim * lev.nq2 + lev.nq1 + both


def test_any_descendant_coarsening_bruteforce():
    p = _small(n=16, levels=3, bulge=True, seed=11)
    levs = mesh.build_levels(p)
    for c, f in zip(levs[:-1], levs[1:]):
        for I_ in range(c.n):
            for J in range(c.n):
                kids = [f.material[(2 * I_ + a) + f.n * (2 * J + b)] for a in (0, 1) for b in (0, 1)]
                assert c.material[I_ + c.n * J] == int(any(kids))


def test_node_classes_bruteforce_geometry():
    p = _small(n=8, levels=1, bulge=True, seed=5)
    lev = mesh.build_levels(p)[0]
    h = lev.h
    xs = np.arange(2 * lev.n + 1) * h / 2
    for q, y in enumerate(xs):
        for pidx, x in enumerate(xs):
            node = pidx + (2 * lev.n + 1) * q
            solid = False
            for e in np.flatnonzero(lev.material == 1):
                i, j = e % lev.n, e // lev.n
                if i * h - 1e-12 <= x <= (i + 1) * h + 1e-12 and j * h - 1e-12 <= y <= (j + 1) * h + 1e-12:
                    solid = True
            assert lev.q2_solid[node] == solid


def test_j2_group_order_and_map():
    p = _small(n=8, levels=1, seed=2)
    lev = mesh.build_levels(p)[0]
    off = lev.group_offsets
    # groups: d^s, d^f, p^s, u^s, u^f, p^f (Eq. matrix_J2)
    fld = lev.dof_field
    assert np.all(fld[off[0]:off[2]] == 0) and np.all(fld[off[3]:off[5]] == 1)
    assert np.all(fld[off[2]:off[3]] == 2) and np.all(fld[off[5]:off[6]] == 2)
    assert np.all(lev.dof_comp[off[2]:off[3]] == 0) and np.all(lev.dof_comp[off[5]:off[6]] == 1)
    sol = lev.q2_solid[lev.dof_node]
    assert np.all(sol[off[0]:off[1]]) and not np.any(sol[off[1]:off[2]])
    assert np.all(sol[off[3]:off[4]]) and not np.any(sol[off[4]:off[5]])
    # nodes increase within a group, components consecutive
    for g in (0, 1, 3, 4):
        nodes = lev.dof_node[off[g]:off[g + 1]]
        assert np.all(np.diff(nodes) >= 0)
        comps = lev.dof_comp[off[g]:off[g + 1]]
        assert np.all(comps == np.tile(np.arange(2), comps.size // 2))
    # bijection onto (field, comp, node) keys
    keys = set(zip(fld.tolist(), lev.dof_comp.tolist(), lev.dof_node.tolist()))
    assert len(keys) == lev.n_dofs


def test_boundary_sets_channel():
    p = _small(n=8, levels=1, seed=2)
    lev = mesh.build_levels(p)[0]
    m2 = 2 * lev.n + 1
    for node in range(lev.nq2):
        x, y = node % m2, node // m2
        x0, x1, y0, y1 = x == 0, x == m2 - 1, y == 0, y == m2 - 1
        if lev.q2_solid[node]:
            assert lev.d_fixed[node] == (x0 or x1 or y0) == lev.v_fixed[node]
        else:
            assert lev.d_fixed[node] == (x0 or x1 or y0 or y1)
            assert lev.v_fixed[node] == (x0 or y0 or y1)
    # fixed dofs and only those
    expect = np.zeros(lev.n_dofs, bool)
    expect[lev.d_dof[lev.d_fixed].ravel()] = True
    expect[lev.v_dof[lev.v_fixed].ravel()] = True
    assert np.array_equal(expect, lev.fixed)
    assert not lev.fixed[lev.dof_field == 2].any()


def test_boundary_sets_box3d():
    p = _small(3, n=4, levels=1)
    lev = mesh.build_levels(p)[0]
    c = mesh.lex(3, 2 * lev.n + 1)
    top = 2 * lev.n
    face = (c[:, 0] == 0) | (c[:, 1] == 0) | (c[:, 1] == top) | (c[:, 2] == 0) | (c[:, 2] == top)
    assert np.array_equal(lev.d_fixed, face) and np.array_equal(lev.v_fixed, face)


def test_level_advection_sampling():
    p = _small(n=8, levels=3, seed=4)
    levs = mesh.build_levels(p)
    w = mesh.level_advection(p, levs[0])
    m_c, m_f = 2 * levs[0].n + 1, 2 * p.n_fine + 1
    for node in range(levs[0].nq2):
        x, y = node % m_c, node // m_c
        fine_node = 4 * x + m_f * 4 * y
        expect = 0.0 if levs[0].q2_solid[node] else p.advection[:, fine_node]
        np.testing.assert_array_equal(w[:, node], expect)
