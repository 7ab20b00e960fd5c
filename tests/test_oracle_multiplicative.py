"""Pins of the oracle's locally multiplicative Schwarz sweep (Sec. 3.2: the
field systems of P2 solved by multiplicative AS, the multiplicative update
formula).  Checked against things other than the sweep's own loop: the
coupling structure of the passes, the textbook closed form of a sequential
subspace-correction sweep (a product of dense projections), the adjoint
identity between the forward and transposed sweeps, and the direct solution
of the whole system."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import fgmres, fsasm, gmg, mesh
from oracle.assemble import assemble
from oracle.transfer import G_DF, G_DS, G_PS, G_US
from paper_1909_13201_gb300 import inputs as I


def _field_masks(lev):
    d = np.isin(lev.group, (G_DS, G_DF, G_PS)) & ~lev.fixed
    u = ~np.isin(lev.group, (G_DS, G_DF, G_PS)) & ~lev.fixed
    return d, u


@pytest.mark.parametrize("mk,b", [
    (lambda: I.make_channel_2d(16, 3, 1, 3), 1),
    (lambda: I.make_channel_2d(16, 3, 2, 3, bulge=True), 2),
    (lambda: I.make_channel_2d(24, 3, 3, 5), 3),
    (lambda: I.make_channel_2d(32, 3, 4, 7, bulge=True), 4),
    (lambda: I.make_valve_3d(4, 2, 1, 9), 1),
    (lambda: I.make_valve_3d(4, 2, 2, 9), 2),
])
def test_blocks_of_a_pass_are_uncoupled(mk, b):
    """Blocks that share a pass (kind, colour) are disjoint and no entry of the
    field operator A_FF couples two of them: updating them one after another
    or all at once gives the same result, so a pass may run in parallel."""
    p = mk()
    lev = mesh.build_levels(p)[-1]
    A = assemble(p, lev).tocoo()
    d, u = _field_masks(lev)
    tagged = fsasm.blocks_tagged(lev, b)
    col = fsasm.group_colours(lev, b)
    nc = fsasm.colour_period(b) ** lev.dim
    passes = {}
    for j, (g, kind, idx) in enumerate(tagged):
        passes.setdefault(kind * nc + col[g], []).append(j)
    assert len(passes) > 1
    for f, m in ((0, d), (1, u)):
        keep = m[A.row] & m[A.col] & (A.data != 0)
        rows, cols = A.row[keep], A.col[keep]
        for key, js in passes.items():
            owner = np.full(lev.n_dofs, -1)
            for j in js:
                idx = tagged[j][2]
                assert (owner[idx] < 0).all()
                owner[idx] = j
            cross = (owner[rows] >= 0) & (owner[cols] >= 0) & (owner[rows] != owner[cols])
            assert not cross.any(), (key, int(cross.sum()))


def _closed_form(S, A, lev, transpose=False, block_inverse=None):
    """Dense M (or M^T) of the sweep from its textbook form: for a field F with
    corrections B_1..B_m (in sweep order, B_j = R_j^T A_jj^{-1} R_j),
    M_F = (I - (I - B_m A_FF) ... (I - B_1 A_FF)) A_FF^{-1}.  block_inverse(j,
    A_jj) replaces the exact inverse of block j (default numpy inv)."""
    n = lev.n_dofs
    Ad = A.toarray()
    d, u = _field_masks(lev)
    M = np.zeros((n, n))
    for f, m in ((0, d), (1, u)):
        F = np.flatnonzero(m)
        AFF = Ad[np.ix_(F, F)]
        pos = np.full(n, -1)
        pos[F] = np.arange(F.size)
        corr = []
        if f == 1:
            k = np.flatnonzero((lev.group == G_US) & ~lev.fixed)
            Bk = np.zeros((F.size, F.size))
            Bk[pos[k], pos[k]] = 1.0 / np.diag(Ad)[k]
            corr.append(Bk)
        for j in S.order:
            if S.block_field[j] != f:
                continue
            idx = pos[S.blocks[j]]
            Bj = np.zeros((F.size, F.size))
            Ajj = AFF[np.ix_(idx, idx)]
            Bj[np.ix_(idx, idx)] = np.linalg.inv(Ajj) if block_inverse is None else block_inverse(j, Ajj)
            corr.append(Bj)
        E = np.eye(F.size)
        for Bj in corr:
            E = (np.eye(F.size) - Bj @ AFF) @ E
        MF = (np.eye(F.size) - E) @ np.linalg.inv(AFF)
        M[np.ix_(F, F)] = MF
    fx = np.flatnonzero(lev.fixed)
    M[fx, fx] = 1.0 / np.diag(Ad)[fx]
    return M.T if transpose else M


@pytest.mark.parametrize("mk,b", [
    (lambda: I.make_channel_2d(8, 2, 2, 11, bulge=True), 2),
    (lambda: I.make_channel_2d(8, 2, 1, 12), 1),
])
def test_sweep_equals_closed_form(mk, b):
    p = mk()
    lev = mesh.build_levels(p)[-1]
    A = assemble(p, lev)
    S = fsasm.FSASM(A, lev, b, multiplicative=True)
    M = _closed_form(S, A, lev)
    rng = np.random.default_rng(0)
    for _ in range(2):
        r = rng.standard_normal(lev.n_dofs)
        y = S.apply(r)
        ref = M @ r
        assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
        yt = S.apply_transpose(r)
        reft = M.T @ r
        assert np.linalg.norm(yt - reft) <= 1e-10 * np.linalg.norm(reft)
    # the sweep is not the additive P2^{-1}: the order of the blocks matters
    Sa = fsasm.FSASM(A, lev, b)
    assert np.linalg.norm(Sa.apply(r) - S.apply(r)) > 1e-3 * np.linalg.norm(S.apply(r))


def test_sweep_adjoint_identity_mixed_half():
    """<M r1, r2> = <r1, M^T r2> for the float16-inverse emulation too (the
    transposed sweep is an independent loop, not a transposed matrix)."""
    p = I.make_channel_2d(16, 3, 2, 21, bulge=True)
    lev = mesh.build_levels(p)[-1]
    A = assemble(p, lev)
    rng = np.random.default_rng(1)
    r1, r2 = rng.standard_normal((2, lev.n_dofs))
    for kw in ({}, {"half": True}):
        S = fsasm.FSASM(A, lev, 2, multiplicative=True, **kw)
        lhs = float(np.dot(S.apply(r1).astype(np.float64), r2))
        rhs = float(np.dot(r1, S.apply_transpose(r2).astype(np.float64)))
        tol = 1e-12 if not kw else 1e-5
        assert abs(lhs - rhs) <= tol * (abs(lhs) + abs(rhs)), (kw, lhs, rhs)


class _HalfScaleDropped(fsasm.FSASM):
    """Planted mistake: the float16 rows applied without their row scale."""

    def _solve(self, j, v, transpose=False):
        m16, scale = self.lu[j]
        m = m16.astype(np.float32)
        return m.T @ v if transpose else m @ v


@pytest.mark.parametrize("mk,b", [
    (lambda: I.make_channel_2d(8, 2, 2, 11, bulge=True), 2),
    (lambda: I.make_channel_2d(8, 2, 1, 12), 1),
])
def test_half_sweep_equals_closed_form_of_its_stored_inverses(mk, b):
    """The float16-storage sweep (the emulation behind the headline's stored
    iteration count) equals the closed form built from its own stored
    inverses diag(s) m16 (dequantized in float64) up to its float32
    arithmetic, and differs from the exact-inverse closed form at float16
    level: the tolerance separates the two, and a sweep that drops the row
    scale fails it."""
    p = mk()
    lev = mesh.build_levels(p)[-1]
    A = assemble(p, lev)
    S = fsasm.FSASM(A, lev, b, multiplicative=True, half=True)

    def stored(j, Ajj):
        m16, scale = S.lu[j]
        return scale.astype(np.float64)[:, None] * m16.astype(np.float64)

    Mh = _closed_form(S, A, lev, block_inverse=stored)
    M = _closed_form(S, A, lev)
    bad = _HalfScaleDropped(A, lev, b, multiplicative=True, half=True)
    rng = np.random.default_rng(3)
    for _ in range(2):
        r = rng.standard_normal(lev.n_dofs).astype(np.float32).astype(np.float64)
        for tr in (False, True):
            y = (S.apply_transpose(r) if tr else S.apply(r)).astype(np.float64)
            ref = (Mh.T if tr else Mh) @ r
            exact = (M.T if tr else M) @ r
            nr = np.linalg.norm(ref)
            # float32 arithmetic of the sweep: a few u = 2^-24 (measured
            # 4e-8 to 9e-8), allowed 1e-6
            assert np.linalg.norm(y - ref) <= 1e-6 * nr, (tr, np.linalg.norm(y - ref) / nr)
            # the stored inverses are visibly not the exact ones: float16
            # rounding (2^-11 per stored entry, averaging in the products;
            # measured 1.6e-5 to 1.1e-4) stays above 4x that tolerance
            assert np.linalg.norm(exact - ref) > 4e-6 * nr
        yb = bad.apply(r).astype(np.float64)
        assert np.linalg.norm(yb - Mh @ r) > 1e-2 * np.linalg.norm(Mh @ r)


@pytest.mark.parametrize("mult_levels", [1, 99])
def test_multiplicative_gmg_fgmres_reaches_direct_solution(mult_levels):
    p = I.make_config(0)
    H = gmg.Hierarchy(p, mult_levels=mult_levels)
    lev = H.levels[-1]
    b = I.gather_natural(I.natural_vector(p, 1), lev.dof_field, lev.dof_comp, lev.dof_node)
    x_ref = spl.spsolve(H.fine.tocsc(), b)
    x, st = fgmres.solve(H, b, rtol=1e-12)
    assert st["converged"]
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # and the multiplicative smoother needs fewer iterations than the additive one
    Ha = gmg.Hierarchy(p)
    _, sa = fgmres.solve(Ha, b, rtol=1e-8)
    _, sm = fgmres.solve(H, b, rtol=1e-8)
    assert sm["iterations"] < sa["iterations"]
    # transposed cycle (reverse sweeps with A_jj^{-T}): the adjoint system
    xt, stt = fgmres.fgmres(H.fine.T.tocsr(), b, H.vcycle_transpose, rtol=1e-12)
    xt_ref = spl.spsolve(H.fine.T.tocsc(), b)
    assert stt["converged"]
    assert np.linalg.norm(xt - xt_ref) <= 1e-9 * np.linalg.norm(xt_ref)
