"""Level hierarchy, materials, node classes, boundary conditions and the J2
dof numbering.

Paper passages followed:
  * Sec. 3.3: levels by midpoint refinement of a conforming coarse mesh; the
    same fluid/solid decomposition is kept on every level.  Reading: a coarse
    element is solid when any of its descendants is solid, so thin solids stay
    visible on coarse grids and coarse solid nodes never interpolate from
    fluid ones.
  * Sec. 3.1 (notation) and the remarks after Eq. jac_orig: kinematic and
    momentum test functions on the interface belong to the solid rows, so a
    node is solid-class when it touches a solid element.
  * Eq. matrix_J2: unknowns ordered d^s, d^f, p^s, u^s, u^f, p^f.  Numbering
    convention inside each group (shared format with the CUDA library):
    nodes in lexicographic order (x fastest), components of a node
    consecutive; pressure copies exist on Q1 vertices touching an element of
    that material (interface vertices carry both p^s and p^f).
  * Boundary conditions (the paper's are geometry specific, Sec. 4): preset 0
    (2D channel): solid-class nodes fixed (d = u = 0) on x=0, x=1, y=0;
    fluid-class nodes: d fixed on every outer side, u fixed on x=0, y=0, y=1,
    do-nothing outflow at x=1.  Preset 1 (3D box): d = u = 0 on every face
    but x=1.  A fixed dof keeps an identity row and a zero column.
"""
from __future__ import annotations

import itertools

import numpy as np

FIELD_D, FIELD_V, FIELD_P = 0, 1, 2


def lex(dim: int, m: int) -> np.ndarray:
    """(m^dim, dim) integer coordinates in flat lexicographic order, x fastest."""
    idx = np.arange(m ** dim)
    return np.stack([(idx // m ** a) % m for a in range(dim)], 1)


def flat(coords: np.ndarray, m: int) -> np.ndarray:
    dim = coords.shape[-1]
    return sum(coords[..., a] * m ** a for a in range(dim))


def coarsen_material(material: np.ndarray, dim: int, n: int) -> np.ndarray:
    """Material of the n/2 grid: solid when any of the 2^dim children is solid."""
    nc = n // 2
    ce = lex(dim, nc)
    out = np.zeros(nc ** dim, np.uint8)
    for off in itertools.product(range(2), repeat=dim):
        child = flat(2 * ce + np.array(off[::-1]), n)
        out |= material[child]
    return out


class Level:
    """One grid level: n^dim elements of side h = 1/n on [0,1]^dim."""

    def __init__(self, dim: int, n: int, material: np.ndarray, bc_preset: int):
        self.dim, self.n, self.h = dim, n, 1.0 / n
        self.material = material.astype(np.uint8)
        m2, m1 = 2 * n + 1, n + 1
        self.nq2, self.nq1 = m2 ** dim, m1 ** dim
        ec = lex(dim, n)                                   # element coords
        loc2 = lex(dim, 3)                                 # local Q2 offsets
        loc1 = lex(dim, 2)
        # element -> global Q2 nodes (n_el, 3^dim) and Q1 vertices (n_el, 2^dim)
        self.elem_q2 = flat(2 * ec[:, None, :] + loc2[None], m2)
        self.elem_q1 = flat(ec[:, None, :] + loc1[None], m1)

        solid_el = self.material == 1
        self.q2_solid = np.zeros(self.nq2, bool)
        self.q2_solid[self.elem_q2[solid_el].ravel()] = True
        self.q1_has_s = np.zeros(self.nq1, bool)
        self.q1_has_s[self.elem_q1[solid_el].ravel()] = True
        self.q1_has_f = np.zeros(self.nq1, bool)
        self.q1_has_f[self.elem_q1[~solid_el].ravel()] = True

        # boundary flags of Q2 nodes
        c2 = lex(dim, m2)
        lo = c2 == 0
        hi = c2 == 2 * n
        if bc_preset == 0:
            assert dim == 2
            x0, x1, y0, y1 = lo[:, 0], hi[:, 0], lo[:, 1], hi[:, 1]
            s = self.q2_solid
            self.d_fixed = np.where(s, x0 | x1 | y0, x0 | x1 | y0 | y1)
            self.v_fixed = np.where(s, x0 | x1 | y0, x0 | y0 | y1)
        elif bc_preset == 1:
            assert dim == 3
            fixed = lo[:, 0] | lo[:, 1] | hi[:, 1] | lo[:, 2] | hi[:, 2]
            self.d_fixed = fixed.copy()
            self.v_fixed = fixed.copy()
        else:
            raise ValueError(bc_preset)
        self._number()

    def _number(self):
        """J2 numbering: d^s, d^f, p^s, u^s, u^f, p^f (Eq. matrix_J2)."""
        dim = self.dim
        s_nodes = np.flatnonzero(self.q2_solid)
        f_nodes = np.flatnonzero(~self.q2_solid)
        ps_nodes = np.flatnonzero(self.q1_has_s)
        pf_nodes = np.flatnonzero(self.q1_has_f)
        ns, nf = s_nodes.size, f_nodes.size
        sizes = [ns * dim, nf * dim, ps_nodes.size, ns * dim, nf * dim, pf_nodes.size]
        off = np.concatenate([[0], np.cumsum(sizes)])
        self.group_offsets = off                     # 7 entries
        self.n_dofs = int(off[-1])
        comps = np.arange(dim)
        self.d_dof = np.full((self.nq2, dim), -1, np.int64)
        self.v_dof = np.full((self.nq2, dim), -1, np.int64)
        self.d_dof[s_nodes] = off[0] + np.arange(ns)[:, None] * dim + comps
        self.d_dof[f_nodes] = off[1] + np.arange(nf)[:, None] * dim + comps
        self.v_dof[s_nodes] = off[3] + np.arange(ns)[:, None] * dim + comps
        self.v_dof[f_nodes] = off[4] + np.arange(nf)[:, None] * dim + comps
        self.ps_dof = np.full(self.nq1, -1, np.int64)
        self.pf_dof = np.full(self.nq1, -1, np.int64)
        self.ps_dof[ps_nodes] = off[2] + np.arange(ps_nodes.size)
        self.pf_dof[pf_nodes] = off[5] + np.arange(pf_nodes.size)

        # dof map: field, comp (pressure copy for p), node
        n = self.n_dofs
        self.dof_field = np.empty(n, np.int64)
        self.dof_comp = np.empty(n, np.int64)
        self.dof_node = np.empty(n, np.int64)
        allq2 = np.arange(self.nq2)
        for fld, table in ((0, self.d_dof), (1, self.v_dof)):
            idx = table.ravel()
            self.dof_field[idx] = fld
            self.dof_comp[idx] = np.tile(comps, self.nq2)
            self.dof_node[idx] = np.repeat(allq2, dim)
        for copy, table, nodes in ((0, self.ps_dof, ps_nodes), (1, self.pf_dof, pf_nodes)):
            self.dof_field[table[nodes]] = 2
            self.dof_comp[table[nodes]] = copy
            self.dof_node[table[nodes]] = nodes

        fixed = np.zeros(n, bool)
        fixed[self.d_dof[self.d_fixed].ravel()] = True
        fixed[self.v_dof[self.v_fixed].ravel()] = True
        self.fixed = fixed
        self.group = np.searchsorted(off, np.arange(n), side="right") - 1


def build_levels(prob) -> list[Level]:
    """Levels 0 (coarse) .. L-1 (fine)."""
    mats = [prob.material.astype(np.uint8)]
    n = prob.n_fine
    for _ in range(prob.n_levels - 1):
        assert n % 2 == 0, "fine size must be divisible by 2^(levels-1)"
        mats.append(coarsen_material(mats[-1], prob.dim, n))
        n //= 2
    mats = mats[::-1]
    return [Level(prob.dim, prob.n_fine >> (prob.n_levels - 1 - l), mats[l], prob.bc_preset)
            for l in range(prob.n_levels)]


def level_advection(prob, lev: Level) -> np.ndarray:
    """Frozen advection w at the level's Q2 nodes: the fine nodal values
    sampled at the coinciding nodes (nested grids), zero at solid-class
    nodes (the solid does not advect)."""
    stride = prob.n_fine // lev.n
    c = lex(lev.dim, 2 * lev.n + 1) * stride
    fine_idx = flat(c, 2 * prob.n_fine + 1)
    w = prob.advection[:, fine_idx].copy()
    w[:, lev.q2_solid] = 0.0
    return w
