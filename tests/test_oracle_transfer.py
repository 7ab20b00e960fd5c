"""Pins of the oracle's prolongation and restriction (oracle/transfer.py):
exact reproduction of Q2/Q1 fields (natural injection, Sec. 3.3), the block
zero pattern of P2, and the blockwise R2 relations of Sec. 3.3."""
import numpy as np
import pytest

from oracle import mesh, transfer
from oracle.transfer import G_DF, G_DS, G_PF, G_PS, G_UF, G_US
from paper_1909_13201_gb300 import inputs as I


def _interp(lev, f2, f1):
    """Nodal values of Q2 field f2 (both comps, both d and u) and Q1 field f1."""
    dim = lev.dim
    c = mesh.lex(dim, 2 * lev.n + 1) / (2 * lev.n)
    x = np.zeros(lev.n_dofs)
    for tab in (lev.d_dof, lev.v_dof):
        for k in range(dim):
            x[tab[:, k]] = f2(c) * (k + 1)
    c1 = mesh.lex(dim, lev.n + 1) / lev.n
    for tab in (lev.ps_dof, lev.pf_dof):
        m = tab >= 0
        x[tab[m]] = f1(c1[m])
    x[lev.fixed] = 0.0
    return x


CASES = [
    (2, lambda: I.make_channel_2d(16, 3, 1, 5, bulge=True),
     lambda c: c[:, 0] * (1 - c[:, 0]) * c[:, 1] * (1 - c[:, 1]), lambda c: (1 + c[:, 0]) * (2 - c[:, 1])),
    (3, lambda: I.make_valve_3d(8, 2, 1, 5),
     lambda c: c[:, 0] * (1 - c[:, 0]) * c[:, 1] * (1 - c[:, 1]) * c[:, 2] * (1 - c[:, 2]),
     lambda c: (1 + c[:, 0]) * (2 - c[:, 1]) * (1 + 0.5 * c[:, 2])),
]


@pytest.mark.parametrize("dim,mk,f2,f1", CASES)
def test_prolongation_reproduces_fields(dim, mk, f2, f1):
    p = mk()
    levs = mesh.build_levels(p)
    fine, coarse = levs[-1], levs[-2]
    P = transfer.prolongation(fine, coarse)
    y = P @ _interp(coarse, f2, f1)
    xf = _interp(fine, f2, f1)
    nz = np.diff(P.indptr) > 0
    # every non-empty row reproduces the fine interpolant exactly
    assert np.abs(y - xf)[nz].max() < 1e-13
    # empty rows are exactly: fixed dofs and p^f vertices without a coarse fluid parent
    empty = ~nz
    pf_orphan = empty & (fine.group == G_PF)
    assert np.all(empty == (fine.fixed | pf_orphan | (np.abs(xf) == 0) & empty))
    assert not np.any(empty & ~fine.fixed & (fine.group != G_PF) & (xf != 0))


def test_prolongation_block_pattern_and_weights():
    p = I.make_channel_2d(16, 2, 1, 8, bulge=True)
    fine, coarse = mesh.build_levels(p)[1], mesh.build_levels(p)[0]
    P = transfer.prolongation(fine, coarse).tocoo()
    gf, gc = fine.group[P.row], coarse.group[P.col]
    pairs = set(zip(gf.tolist(), gc.tolist()))
    allowed = {(G_DS, G_DS), (G_DF, G_DS), (G_DF, G_DF), (G_PS, G_PS),
               (G_US, G_US), (G_UF, G_US), (G_UF, G_UF), (G_PF, G_PF)}
    assert pairs <= allowed
    assert (G_DF, G_DS) in pairs and (G_UF, G_US) in pairs
    # same component, and Q2 weights from {1, 3/4, 3/8, 1/2, -1/8, ...} products
    assert np.all(fine.dof_comp[P.row] == coarse.dof_comp[P.col])
    w1 = {1.0, 0.75, 0.375, -0.125, 0.5}
    prods = {a * b for a in w1 | {1.0} for b in w1 | {1.0}}
    assert all(any(abs(v - q) < 1e-15 for q in prods) for v in P.data)


def _block(M, rows_lev, rg, cols_lev, cg):
    r = np.flatnonzero(rows_lev.group == rg)
    c = np.flatnonzero(cols_lev.group == cg)
    return M.tocsr()[r][:, c].toarray()


def test_restriction_blockwise_relations():
    p = I.make_channel_2d(16, 2, 1, 8, bulge=True)
    levs = mesh.build_levels(p)
    fine, coarse = levs[1], levs[0]
    P = transfer.prolongation(fine, coarse)
    R = transfer.restriction(P, fine, coarse)
    # R_SS = P_{ds,ds}^T, R_AA = P_{df,df}^T, R_VV = P_{ps,ps}^T, R_KK = P_{us,us}^T,
    # R_FF = P_{uf,uf}^T, R_WW = P_{pf,pf}^T   (Sec. 3.3)
    for g in (G_DS, G_DF, G_PS, G_US, G_UF, G_PF):
        np.testing.assert_array_equal(_block(R, coarse, g, fine, g), _block(P, fine, g, coarse, g).T)
    # R_SF: coarse S rows (d^s dofs) gather fine F residuals (u^f dofs) with the
    # transpose of P_{uf,us}; the d^s/u^s dofs of a node are in the same order
    np.testing.assert_array_equal(_block(R, coarse, G_DS, fine, G_UF),
                                  _block(P, fine, G_UF, coarse, G_US).T)
    # fluid residuals never reach the coarse K rows; A never reaches S
    assert not _block(R, coarse, G_US, fine, G_UF).any()
    assert not _block(R, coarse, G_DS, fine, G_DF).any()
    # no other cross blocks
    Rc = R.tocoo()
    pairs = set(zip(coarse.group[Rc.row].tolist(), fine.group[Rc.col].tolist()))
    assert pairs <= {(g, g) for g in range(6)} | {(G_DS, G_UF)}
    # R_SF really is present on this geometry
    assert (G_DS, G_UF) in pairs


def test_classical_restriction_is_transpose():
    p = I.make_channel_2d(8, 2, 1, 8)
    levs = mesh.build_levels(p)
    P = transfer.prolongation(levs[1], levs[0])
    R = transfer.restriction(P, levs[1], levs[0], classical=True)
    assert abs(R - P.T).max() == 0
