"""Prolongation P2 and equation-aware restriction R2 (Sec. 3.3).

P_{l,l-1} is the natural injection of the coarse FE space into the fine one,
written as nodal interpolation: a fine Q2 node takes the coarse Q2
interpolant of a coarse element containing it; a fine p^s (p^f) vertex takes
the coarse Q1 interpolant of a containing coarse solid (fluid) element, or a
zero row for p^f when no coarse fluid element contains it.  Fixed fine rows
and fixed coarse columns are zero (homogeneous corrections).

R_{l-1,l} is not P^T (Sec. 3.3, block structure of R2): each coarse equation
gathers fine residuals of the same equation with the transpose of the
interpolation of its test functions,
  S <- S (P_{d^s,d^s}^T) and F (P_{u^f,u^s}^T);  A <- A (P_{d^f,d^f}^T);
  V <- V (P_{p^s,p^s}^T);  K <- K (P_{u^s,u^s}^T);  F <- F (P_{u^f,u^f}^T);
  W <- W (P_{p^f,p^f}^T);
and the fluid residual never reaches the coarse K rows (the transpose of
P_{u^f,u^s} is dropped there).  Reading: the paper writes R_{S,F} =
P_{d^f,d^s}^T; the momentum residual is restricted with the momentum (velocity)
test space, which coincides with P_{d^f,d^s} wherever d and u share their
fixed set and differs only at outflow nodes (u free, d fixed).
``classical=True`` returns R = P^T instead.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .fem import q1_1d, q2_1d
from .mesh import Level, flat, lex


def prolongation(fine: Level, coarse: Level) -> sp.csr_matrix:
    """Nodal interpolation, vectorised over the fine nodes."""
    dim = fine.dim
    nc = coarse.n
    rows, cols, vals = [], [], []
    # --- Q2 fields (d and u) ---
    pos = lex(dim, 2 * fine.n + 1)                     # fine Q2 lattice indices
    el = np.minimum(pos // 4, nc - 1)                  # coarse element spans 4 fine Q2 steps
    frac = (pos - 4 * el) / 4.0
    w1 = [q2_1d(frac[:, k])[0] for k in range(dim)]    # (3, nq2) per direction
    for a in itertools.product(range(3), repeat=dim):
        a = np.array(a[::-1])                          # local coarse node, x fastest
        wt = np.ones(fine.nq2)
        for k in range(dim):
            wt = wt * w1[k][a[k]]
        Y = flat(2 * el + a, 2 * nc + 1)
        for comp in range(dim):
            for tab_f, tab_c in ((fine.d_dof, coarse.d_dof), (fine.v_dof, coarse.v_dof)):
                r, c = tab_f[:, comp], tab_c[Y, comp]
                keep = (wt != 0.0) & ~fine.fixed[r] & ~coarse.fixed[c]
                rows.append(r[keep]); cols.append(c[keep]); vals.append(wt[keep])
    # --- Q1 pressure copies ---
    pos = lex(dim, fine.n + 1)                         # fine Q1 lattice; coarse element spans 2 steps
    lo = np.maximum((pos - 1) // 2, 0)
    hi = np.minimum(pos // 2, nc - 1)
    # candidate containing coarse elements, x fastest; both choices contain the vertex
    cand = []
    for t in range(2 ** dim):
        e = np.where(np.array([(t >> k) & 1 for k in range(dim)])[None, :] == 1, hi, lo)
        cand.append(e)
    cand = np.stack(cand, 1)                           # (nq1, 2^dim, dim)
    cmat = coarse.material[flat(cand, nc)]             # (nq1, 2^dim)
    for has_f, dof_f, dof_c, mat in ((fine.q1_has_s, fine.ps_dof, coarse.ps_dof, 1),
                                     (fine.q1_has_f, fine.pf_dof, coarse.pf_dof, 0)):
        match = cmat == mat
        ok = has_f & match.any(1)                      # p^f with no coarse fluid parent: zero row
        first = np.argmax(match, 1)
        E = cand[np.arange(pos.shape[0]), first]       # chosen coarse element
        fr = (pos - 2 * E) / 2.0
        for a in itertools.product(range(2), repeat=dim):
            a = np.array(a[::-1])
            wt = np.ones(pos.shape[0])
            for k in range(dim):
                wt = wt * (fr[:, k] if a[k] else 1.0 - fr[:, k])
            keep = ok & (wt != 0.0)
            Z = flat(E + a, nc + 1)
            rows.append(dof_f[keep]); cols.append(dof_c[Z[keep]]); vals.append(wt[keep])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.n_dofs, coarse.n_dofs)).tocsr()
    P.sum_duplicates()
    P.sort_indices()
    return P


# J2 group ids: 0 d^s (S rows), 1 d^f (A rows), 2 p^s (V), 3 u^s (K), 4 u^f (F), 5 p^f (W)
G_DS, G_DF, G_PS, G_US, G_UF, G_PF = range(6)


def restriction(P: sp.csr_matrix, fine: Level, coarse: Level, classical: bool = False) -> sp.csr_matrix:
    if classical:
        return P.T.tocsr()
    Pc = P.tocoo()
    gf = fine.group[Pc.row]           # fine dof group
    gc = coarse.group[Pc.col]         # coarse dof group
    rr, cc, vv = [], [], []
    # same-group blocks: S<-S, A<-A, V<-V, K<-K, F<-F, W<-W
    same = gf == gc
    rr.append(Pc.col[same]); cc.append(Pc.row[same]); vv.append(Pc.data[same])
    # S <- F through the momentum interpolation P_{u^f,u^s}: fine F residual
    # (u^f rows) to coarse S (d^s rows) of the same node and component.
    m = (gf == G_UF) & (gc == G_US)
    fine_uf = Pc.row[m]
    coarse_us = Pc.col[m]
    node_c, comp_c = coarse.dof_node[coarse_us], coarse.dof_comp[coarse_us]
    coarse_ds = coarse.d_dof[node_c, comp_c]
    ok = ~coarse.fixed[coarse_ds]
    rr.append(coarse_ds[ok]); cc.append(fine_uf[ok]); vv.append(Pc.data[m][ok])
    R = sp.coo_matrix((np.concatenate(vv), (np.concatenate(rr), np.concatenate(cc))),
                      shape=(coarse.n_dofs, fine.n_dofs)).tocsr()
    R.sum_duplicates()
    R.sort_indices()
    return R
