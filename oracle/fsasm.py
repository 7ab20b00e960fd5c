"""Field-split additive Schwarz smoother (the FS preconditioner P2 of Sec. 3.2).

P2 = blockdiag( [S_d^s S_d^f S_p^s; A_d^s A_d^f 0; V_d^s 0 V_p^s],
                [K_u^s 0 0; F_u^s F_u^f F_p^f; W_u^s W_u^f 0] )
and each diagonal block is itself replaced by an additive Schwarz method:
  AS1: solid blocks [S_d^s S_p^s; V_d^s V_p^s]_j and fluid blocks [A_d^f]_j,
  AS2: the lumped mass K_u^s inverted exactly by one Jacobi step, and fluid
       blocks [F_u^f F_p^f; W_u^f 0]_j,
each block solved by LU (Sec. 3.2, "solved using LU decomposition").

Blocks follow the paper's Vanka selection rule (Sec. 3.2): a block takes a
set of pressure dofs and then every displacement/velocity dof whose support
meets the support of those pressures.  For the continuous Q1 pressure used
here the pressure sets are non-overlapping groups of b^dim pressure vertices
(tiles of the Q1 vertex lattice, truncated at the domain edge; b = ``patch``).
Per group:
  solid block   [d^s, p^s]: the group's p^s vertices, plus the d^s dofs on the
                closure of the solid elements touching them;
  fluid-d block [d^f]     : the d^f dofs on the closure of the fluid elements
                touching the group's p^f vertices (overlapping blocks, AS1);
  fluid-u block [u^f, p^f]: the group's p^f vertices plus the u^f dofs on the
                same closure (AS2);
fixed dofs are excluded.  With b = 1 in 2D a fluid-u block spans 2x2 elements
(50 + 1 dofs), with b = 3 it spans 4x4 elements (162 + 9 dofs), with b = 1 in
3D 2x2x2 elements (375 + 1 dofs).  Because every pressure row of a block sees
its complete support, the block saddle problems are the true local Vanka
problems.  The additive combination (Sec. 3.2, additive update formula) uses
partition-of-unity weights W_j = diag(1/multiplicity):

    P2^{-1} r = sum_j R_j^T W_j A_jj^{-1} R_j r  +  D^{-1} r |_{u^s and fixed dofs},
    x <- x + omega P2^{-1} (b - A x)        (damped Richardson, Sec. 3.2).

With multiplicative=True the blocks are combined instead by the paper's
locally multiplicative update (Sec. 3.2, multiplicative update formula), per
field system of P2: FSASM.sweep corrects one block after another from the
residual of the field operator at the latest iterate (see _setup_sweep).

The oracle factors each block with partial-pivoting LU (scipy/LAPACK getrf).
Storage emulations of the mixed modes: ``dtype=float32`` factors and solves
in float32; ``half=True`` forms the float64 inverse from the LU factors,
normalises each row by its max-abs entry, rounds it to float16 and applies it
in float32 times the float32 row scale.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp

from .mesh import Level, flat, lex
from .transfer import G_DF, G_DS, G_PS, G_US


def vertex_groups(lev: Level, b: int) -> list[np.ndarray]:
    """Q1 vertices of the b^dim tiles of the vertex lattice, tiles in lex order."""
    m1 = lev.n + 1
    npd = -(-m1 // b)
    tile = flat(lex(lev.dim, m1) // b, npd)           # tile of every vertex
    order = np.argsort(tile, kind="stable")            # vertices in lex order inside a tile
    bounds = np.searchsorted(tile[order], np.arange(npd ** lev.dim + 1))
    return [order[bounds[t]:bounds[t + 1]] for t in range(npd ** lev.dim)]


def vertex_elements(lev: Level) -> np.ndarray:
    """(nq1, 2^dim) elements touching each Q1 vertex, -1 where absent."""
    nv = 2 ** lev.dim
    out = np.full((lev.nq1, nv), -1, np.int64)
    fill = np.zeros(lev.nq1, np.int64)
    for al in range(nv):                      # each element touches its 2^dim vertices once
        z = lev.elem_q1[:, al]
        out[z, fill[z]] = np.arange(lev.material.size)
        fill[z] += 1
    return out


def blocks_tagged(lev: Level, b: int) -> list[tuple[int, int, np.ndarray]]:
    """(vertex group, kind, sorted dof indices) of every non-empty block, per
    group in the order solid (kind 0, [d^s, p^s]), fluid-d (kind 1, [d^f]),
    fluid-u (kind 2, [u^f, p^f])."""
    touch = vertex_elements(lev)
    blocks = []
    for g, grp in enumerate(vertex_groups(lev, b)):
        cand = []
        zs = grp[lev.ps_dof[grp] >= 0]
        els = touch[zs].ravel()
        els = np.unique(els[(els >= 0)])
        els = els[lev.material[els] == 1]
        if els.size:
            q2 = np.unique(lev.elem_q2[els])
            cand.append((0, np.concatenate([lev.d_dof[q2].ravel(), lev.ps_dof[zs]])))
        zf = grp[lev.pf_dof[grp] >= 0]
        els = touch[zf].ravel()
        els = np.unique(els[(els >= 0)])
        els = els[lev.material[els] == 0]
        if els.size:
            q2 = np.unique(lev.elem_q2[els])
            q2 = q2[~lev.q2_solid[q2]]
            cand.append((1, lev.d_dof[q2].ravel()))
            cand.append((2, np.concatenate([lev.v_dof[q2].ravel(), lev.pf_dof[zf]])))
        for kind, idx in cand:
            idx = np.unique(idx)
            idx = idx[~lev.fixed[idx]]
            if idx.size:
                blocks.append((g, kind, idx))
    return blocks


def block_index_sets(lev: Level, b: int) -> list[np.ndarray]:
    """Sorted dof index sets of all blocks: per vertex group solid, fluid-d, fluid-u."""
    return [idx for _, _, idx in blocks_tagged(lev, b)]


def colour_period(b: int) -> int:
    """Colours per direction k of the vertex groups in a multiplicative sweep.
    Group t spans the element closure [t b - 1, (t + 1) b] (in vertex units);
    groups t and t + k leave a gap of (k - 1) b - 1 vertex spacings, and two
    dofs are coupled only when they share an element (gap <= 1).  The
    smallest k with (k - 1) b - 1 >= 2: 4 for b = 1, 3 for b = 2, else 2."""
    return 4 if b == 1 else (3 if b == 2 else 2)


def group_colours(lev: Level, b: int) -> np.ndarray:
    """Colour of every vertex group: sum_a ((t_a mod k) k^a) over the group's
    tile coordinates t_a (groups in the lex order of vertex_groups)."""
    npd = -(-(lev.n + 1) // b)
    k = colour_period(b)
    t = lex(lev.dim, npd)
    return sum((t[:, a] % k) * k ** a for a in range(lev.dim))


def block_index_sets_monolithic(lev: Level, b: int) -> list[np.ndarray]:
    """Blocks of the monolithic additive Schwarz preconditioner AS (Sec. 3.2):
    the same pressure groups, but one block per group holding every variable
    whose support meets the support of the group's pressures: the group's p^s
    and p^f vertices and all displacement and velocity dofs, of both classes,
    on the closure of all elements touching them (fixed dofs excluded)."""
    touch = vertex_elements(lev)
    blocks = []
    for grp in vertex_groups(lev, b):
        els = touch[grp].ravel()
        els = np.unique(els[els >= 0])
        q2 = np.unique(lev.elem_q2[els])
        p = np.concatenate([lev.ps_dof[grp], lev.pf_dof[grp]])
        idx = np.concatenate([lev.d_dof[q2].ravel(), lev.v_dof[q2].ravel(), p[p >= 0]])
        idx = np.unique(idx)
        idx = idx[~lev.fixed[idx]]
        if idx.size:
            blocks.append(idx)
    return blocks


class FSASM:
    """The smoother's preconditioner on one level: the field-split P2^{-1}
    (default) or, with monolithic=True, the additive Schwarz method AS whose
    blocks hold all fields (Sec. 3.2); fixed dofs take a Jacobi step in both,
    the lumped K_u^s rows only in the field split."""

    def __init__(self, A: sp.csr_matrix, lev: Level, b: int, *, dtype=np.float64,
                 weighted: bool = True, half: bool = False, monolithic: bool = False,
                 multiplicative: bool = False):
        self.n = A.shape[0]
        self.dtype = np.float32 if half else dtype
        self.half = half
        self.multiplicative = multiplicative and not monolithic
        if monolithic:
            self.blocks = block_index_sets_monolithic(lev, b)
        else:
            tagged = blocks_tagged(lev, b)
            self.blocks = [idx for _, _, idx in tagged]
        mult = np.zeros(self.n)
        for idx in self.blocks:
            mult[idx] += 1.0
        self.multiplicity = mult
        self.weight = np.where(mult > 0, 1.0 / np.maximum(mult, 1.0), 0.0) if weighted \
            else (mult > 0).astype(np.float64)
        Ad = A.tocsr()
        self.lu = []
        local = np.full(self.n, -1, np.int64)         # global dof -> position in the block
        for idx in self.blocks:
            # A_jj = A[I_j, I_j]: the block's rows, columns mapped into the block
            sub = Ad[idx]
            local[idx] = np.arange(idx.size)
            cols = local[sub.indices]
            keep = cols >= 0
            rows = np.repeat(np.arange(idx.size), np.diff(sub.indptr))
            blk = np.zeros((idx.size, idx.size))
            blk[rows[keep], cols[keep]] = sub.data[keep]
            local[idx] = -1
            if half:
                inv = la.lu_solve(la.lu_factor(blk), np.eye(idx.size))
                scale = np.abs(inv).max(1)
                scale[scale == 0] = 1.0
                m16 = (inv / scale[:, None]).astype(np.float16)
                self.lu.append((m16, scale.astype(np.float32)))
            else:
                self.lu.append(la.lu_factor(blk.astype(dtype), check_finite=True))
        self.jacobi = np.flatnonzero(lev.fixed if monolithic else (lev.group == G_US) | lev.fixed)
        self.inv_diag = 1.0 / Ad.diagonal()[self.jacobi]
        if self.multiplicative:
            self._setup_sweep(Ad, lev, b, tagged)

    # ---------------------------------------------- locally multiplicative
    # Sec. 3.2: the two field systems of P2 (block diagonal: displacement /
    # solid pressure, velocity / fluid pressure) are solved separately, each
    # by a locally multiplicative Schwarz sweep: block j is updated from the
    # field residual of the most recent iterate, y <- y + R_j^T A_jj^{-1}
    # R_j (r_F - A_FF y), blocks one after another (the paper's multiplicative
    # update formula), starting from y = 0.  A_FF is A restricted to the
    # field's rows and columns (P2 drops the couplings between the fields).
    # In the velocity field the lumped K_u^s rows come first (one exact Jacobi
    # step, Sec. 3.2), then the fluid blocks.  Fixed dofs take a Jacobi step.
    # Block order: by pass (kind, colour) with kind 0 solid, 1 fluid-d, 2
    # fluid-u and the colour of the block's vertex group, then by group.
    def _setup_sweep(self, Ad, lev, b, tagged):
        dt = self.dtype
        col = group_colours(lev, b)
        nc = colour_period(b) ** lev.dim
        self.block_pass = np.array([kind * nc + col[g] for g, kind, _ in tagged], np.int64)
        self.block_field = np.array([int(kind == 2) for _, kind, _ in tagged], np.int64)
        self.order = np.argsort(self.block_pass, kind="stable")
        dfield = np.isin(lev.group, (G_DS, G_DF, G_PS)) & ~lev.fixed
        ufield = ~np.isin(lev.group, (G_DS, G_DF, G_PS)) & ~lev.fixed
        C = Ad.tocoo()
        self.AFF = []
        for m in (dfield, ufield):
            keep = m[C.row] & m[C.col]
            self.AFF.append(sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=Ad.shape).astype(dt))
        AFT = [M.T.tocsr() for M in self.AFF]
        self.rows_f = [self.AFF[f][idx] for f, idx in zip(self.block_field, self.blocks)]
        self.rows_t = [AFT[f][idx] for f, idx in zip(self.block_field, self.blocks)]
        jac = np.zeros(self.n, bool)
        jac[self.jacobi] = True
        self.kdofs = np.flatnonzero((lev.group == G_US) & ~lev.fixed)
        self.fdofs = np.flatnonzero(lev.fixed)
        diag = Ad.diagonal()
        self.k_inv = (1.0 / diag[self.kdofs]).astype(dt)
        self.f_inv = (1.0 / diag[self.fdofs]).astype(dt)
        self.k_rows = self.AFF[1][self.kdofs]
        self.k_rows_t = AFT[1][self.kdofs]

    def _solve(self, j, v, transpose=False):
        lu = self.lu[j]
        if self.half:
            m16, scale = lu
            if transpose:
                return m16.astype(np.float32).T @ (scale * v)
            return scale * (m16.astype(np.float32) @ v)
        return la.lu_solve(lu, v, trans=1 if transpose else 0)

    def sweep(self, r: np.ndarray, transpose: bool = False) -> np.ndarray:
        """y = M r: one multiplicative sweep per field from y = 0; with
        transpose, M^T r (the blocks in reverse order with A_jj^{-T} and the
        residual of A_FF^T: the velocity field's K_u^s step comes last)."""
        dt = self.dtype
        r = r.astype(dt)
        y = np.zeros(self.n, dt)
        rows = self.rows_t if transpose else self.rows_f
        order = self.order[::-1] if transpose else self.order
        d_blocks = [j for j in order if self.block_field[j] == 0]
        u_blocks = [j for j in order if self.block_field[j] == 1]
        for j in d_blocks:
            idx = self.blocks[j]
            y[idx] += self._solve(j, r[idx] - rows[j] @ y, transpose).astype(dt)
        if not transpose:
            k = self.kdofs
            y[k] += ((r[k] - self.k_rows @ y) * self.k_inv).astype(dt)
        for j in u_blocks:
            idx = self.blocks[j]
            y[idx] += self._solve(j, r[idx] - rows[j] @ y, transpose).astype(dt)
        if transpose:
            k = self.kdofs
            y[k] += ((r[k] - self.k_rows_t @ y) * self.k_inv).astype(dt)
        y[self.fdofs] += (r[self.fdofs] * self.f_inv).astype(dt)
        return y

    def apply(self, r: np.ndarray) -> np.ndarray:
        """P2^{-1} r (additive), or the multiplicative sweep M r."""
        if self.multiplicative:
            return self.sweep(r)
        dt = self.dtype
        r = r.astype(dt)
        y = np.zeros(self.n, dt)
        w = self.weight.astype(dt)
        for idx, lu in zip(self.blocks, self.lu):
            if self.half:
                m16, scale = lu
                y[idx] += w[idx] * (scale * (m16.astype(np.float32) @ r[idx]))
            else:
                y[idx] += w[idx] * la.lu_solve(lu, r[idx])
        y[self.jacobi] += (r[self.jacobi] * self.inv_diag.astype(dt)).astype(dt)
        return y

    def apply_transpose(self, r: np.ndarray) -> np.ndarray:
        """P2^{-T} r = sum_j R_j^T A_jj^{-T} W_j R_j r + D^{-1} r (adjoint smoother),
        or M^T r for the multiplicative sweep."""
        if self.multiplicative:
            return self.sweep(r, transpose=True)
        dt = self.dtype
        r = r.astype(dt)
        y = np.zeros(self.n, dt)
        w = self.weight.astype(dt)
        for idx, lu in zip(self.blocks, self.lu):
            if self.half:
                m16, scale = lu
                y[idx] += m16.astype(np.float32).T @ (scale * w[idx] * r[idx])
            else:
                y[idx] += la.lu_solve(lu, w[idx] * r[idx], trans=1)
        y[self.jacobi] += (r[self.jacobi] * self.inv_diag.astype(dt)).astype(dt)
        return y
