"""Pins of the oracle's smoother, V-cycle, FGMRES and adjoint.

* FS-ASM (Sec. 3.2): block index sets against a brute-force geometric
  statement of the Vanka rule; partition of unity; with one vertex group
  covering the whole level the smoother equals the exact solve with the
  field-split block-diagonal matrix (AS1 solid/fluid, AS2 Jacobi + fluid);
  the Jacobi step on K_u^s is exact; the transposed apply is the adjoint.
* AS (the paper's monolithic comparison method, Sec. 3.2): block sets against
  a brute-force statement of the Vanka rule over all fields; partition of
  unity; one group covering the level gives the exact solve; GMG-FGMRES with
  AS smoothing matches a sparse direct solve.
* GMG: a 1-level hierarchy is the direct solve; the transposed V-cycle is the
  adjoint of the V-cycle; a two-grid spectral radius below 1 on this
  workload; mixed mode stays within float32 rounding of the float64 cycle.
* FGMRES: the residual estimates equal the true minimal residuals over the
  Krylov spaces (dense least squares), an exact preconditioner converges in
  one step, and the solve matches a sparse direct solve.
* Adjoint: lambda matches a sparse direct transposed solve, lambda^T b =
  w^T x, and gradients agree with central differences.
"""
import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import adjoint, fgmres, fsasm, gmg, mesh
from oracle.assemble import assemble
from paper_1909_13201_gb300 import inputs as I


@pytest.fixture(scope="module")
def c0():
    p = I.make_config(0)
    return p, gmg.Hierarchy(p)


def test_block_sets_bruteforce_geometry():
    p = I.make_channel_2d(8, 1, 2, 5, bulge=True, band_width=0.3)
    lev = mesh.build_levels(p)[0]
    h = lev.h
    got = fsasm.block_index_sets(lev, 2)
    q2xy = mesh.lex(2, 2 * lev.n + 1) * (h / 2)
    q1xy = mesh.lex(2, lev.n + 1) * h
    expect = []
    for gy in range(0, lev.n + 1, 2):
        for gx in range(0, lev.n + 1, 2):
            verts = [z for z in range(lev.nq1) if gx <= q1xy[z, 0] / h < gx + 2 - 1e-9
                     and gy <= q1xy[z, 1] / h < gy + 2 - 1e-9]
            for mat in (1, 0):
                # elements of this material whose closed box contains a selected vertex
                # that carries this material's pressure
                pv = [z for z in verts if any(
                    lev.material[e] == mat and
                    (e % lev.n) * h - 1e-12 <= q1xy[z, 0] <= (e % lev.n + 1) * h + 1e-12 and
                    (e // lev.n) * h - 1e-12 <= q1xy[z, 1] <= (e // lev.n + 1) * h + 1e-12
                    for e in range(lev.material.size))]
                els = [e for e in range(lev.material.size) if lev.material[e] == mat and any(
                    (e % lev.n) * h - 1e-12 <= q1xy[z, 0] <= (e % lev.n + 1) * h + 1e-12 and
                    (e // lev.n) * h - 1e-12 <= q1xy[z, 1] <= (e // lev.n + 1) * h + 1e-12 for z in pv)]
                nodes = [y for y in range(lev.nq2) if any(
                    (e % lev.n) * h - 1e-12 <= q2xy[y, 0] <= (e % lev.n + 1) * h + 1e-12 and
                    (e // lev.n) * h - 1e-12 <= q2xy[y, 1] <= (e // lev.n + 1) * h + 1e-12 for e in els)]
                if mat == 1:
                    sets = [[lev.d_dof[y, c] for y in nodes for c in (0, 1)] + [lev.ps_dof[z] for z in pv]]
                else:
                    fn = [y for y in nodes if not lev.q2_solid[y]]
                    sets = [[lev.d_dof[y, c] for y in fn for c in (0, 1)],
                            [lev.v_dof[y, c] for y in fn for c in (0, 1)] + [lev.pf_dof[z] for z in pv]]
                for s in sets:
                    s = np.array(sorted(d for d in set(s) if not lev.fixed[d]), np.int64)
                    if s.size:
                        expect.append(s)
    assert len(got) == len(expect)
    for a, b in zip(got, expect):
        np.testing.assert_array_equal(a, b)


def test_partition_of_unity_and_coverage(c0):
    p, H = c0
    for l in range(1, len(H.levels)):
        S, lev = H.smoothers[l], H.levels[l]
        tot = np.zeros(S.n)
        for idx in S.blocks:
            tot[idx] += S.weight[idx]
        jac = np.zeros(S.n, bool)
        jac[S.jacobi] = True
        np.testing.assert_allclose(tot[~jac], 1.0, rtol=1e-15)
        assert np.all(tot[jac] == 0)           # u^s and fixed dofs are Jacobi-only


def test_whole_level_group_is_exact_field_split_solve():
    p = I.make_channel_2d(6, 1, 1, 3, bulge=True, band_width=0.4)
    lev = mesh.build_levels(p)[0]
    A = assemble(p, lev)
    S = fsasm.FSASM(A, lev, lev.n + 1)     # one vertex group = the whole level
    assert len(S.blocks) == 3
    Ad = A.toarray()
    g = lev.group
    free = ~lev.fixed
    M = np.zeros_like(Ad)
    # AS1 solid [d^s, p^s], AS1 fluid [d^f], AS2 fluid [u^f, p^f]: S_d^f and
    # A_d^s couplings drop out because the solid and fluid sets are separate
    for grp in ((0, 2), (1,), (4, 5)):
        idx = np.flatnonzero(np.isin(g, grp) & free)
        M[np.ix_(idx, idx)] = Ad[np.ix_(idx, idx)]
    jac = (g == 3) | lev.fixed
    M[jac, jac] = np.diag(Ad)[jac]
    r = np.random.default_rng(0).standard_normal(lev.n_dofs)
    np.testing.assert_allclose(S.apply(r), np.linalg.solve(M, r), rtol=1e-9, atol=1e-12)


def test_jacobi_rows_exact_and_transpose_adjoint(c0):
    p, H = c0
    S, lev, A = H.smoothers[-1], H.levels[-1], H.A[-1]
    rng = np.random.default_rng(2)
    r = rng.standard_normal(S.n)
    y = S.apply(r)
    us = lev.group == 3
    np.testing.assert_allclose(y[us], r[us] / A.diagonal()[us], rtol=1e-14)
    r2 = rng.standard_normal(S.n)
    assert S.apply(r) @ r2 == pytest.approx(r @ S.apply_transpose(r2), rel=1e-11)


def test_one_level_is_direct_solve():
    p = I.make_channel_2d(8, 1, 1, 4, band_width=0.25, mu_s=1e2, mu_f=1e-2)
    H = gmg.Hierarchy(p)
    b = np.random.default_rng(1).standard_normal(H.fine.shape[0])
    x, st = fgmres.solve(H, b, rtol=1e-12)
    assert st["iterations"] == 1
    np.testing.assert_allclose(x, spl.spsolve(H.fine.tocsc(), b), rtol=1e-9, atol=1e-12)


def test_vcycle_transpose_is_adjoint(c0):
    p, H = c0
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((2, H.fine.shape[0]))
    assert H.vcycle(a) @ b == pytest.approx(a @ H.vcycle_transpose(b), rel=1e-10)


def test_two_grid_contraction():
    p = I.make_channel_2d(16, 2, 1, 13201, band_width=0.25, mu_s=1e2, mu_f=1e-2)
    H = gmg.Hierarchy(p)
    A = H.fine
    rng = np.random.default_rng(4)
    e = rng.standard_normal(A.shape[0])
    for _ in range(40):                    # power iteration on I - M^{-1} A
        e = e - H.vcycle(A @ e)
        nrm = np.linalg.norm(e)
        e /= nrm
    assert nrm < 1.0


def test_mixed_vcycle_close_to_fp64(c0):
    p, H = c0
    Hm = gmg.Hierarchy(p, mixed=True)
    b = np.random.default_rng(5).standard_normal(H.fine.shape[0])
    z64, z32 = H.vcycle(b), Hm.vcycle(b)
    assert np.linalg.norm(z64 - z32) / np.linalg.norm(z64) < 1e-3
    assert z32.dtype == np.float64 and np.all(z32 == z32.astype(np.float32))


def test_fgmres_estimates_are_minimal_residuals():
    rng = np.random.default_rng(6)
    n = 40
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.5
    b = rng.standard_normal(n)
    x, st = fgmres.fgmres(sp.csr_matrix(A), b, lambda v: v, rtol=1e-13, restart=n, maxit=12)
    K = np.zeros((n, 12))
    v = b.copy()
    for k in range(12):
        K[:, k] = v
        v = A @ v
    for k in range(1, 13):
        Q, _ = np.linalg.qr(K[:, :k])
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        true_min = np.linalg.norm(b - A @ Q @ y) / np.linalg.norm(b)
        assert st["estimates"][k - 1] == pytest.approx(true_min, rel=1e-8)
    assert st["rel_residual"] == pytest.approx(st["estimates"][-1], rel=1e-8)


def test_fgmres_exact_preconditioner_one_step(c0):
    p, H = c0
    lu = spl.splu(H.fine.tocsc())
    b = np.random.default_rng(7).standard_normal(H.fine.shape[0])
    x, st = fgmres.fgmres(H.fine, b, lu.solve, rtol=1e-9)
    assert st["iterations"] == 1 and st["converged"]


def test_fgmres_gmg_matches_direct_solve(c0):
    p, H = c0
    b = np.random.default_rng(8).standard_normal(H.fine.shape[0])
    x, st = fgmres.solve(H, b, rtol=1e-12)
    xd = spl.spsolve(H.fine.tocsc(), b)
    assert st["converged"]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
    assert 5 <= st["iterations"] <= 60
    assert st["rho"] == pytest.approx((st["rN"] / st["r0"]) ** (1 / st["iterations"]))


def test_adjoint_solution_and_identity(c0):
    p, H = c0
    rng = np.random.default_rng(9)
    b, w = rng.standard_normal((2, H.fine.shape[0]))
    x, _ = fgmres.solve(H, b, rtol=1e-12)
    lam, st = adjoint.adjoint_solve(H, w, rtol=1e-12)
    assert st["converged"]
    lam_d = spl.spsolve(H.fine.T.tocsc(), w)
    assert np.linalg.norm(lam - lam_d) / np.linalg.norm(lam_d) < 1e-9
    assert lam @ b == pytest.approx(w @ x, rel=1e-9)


def test_adjoint_gradients_central_differences():
    p = I.make_channel_2d(8, 2, 1, 21, band_width=0.3, mu_s=50.0, mu_f=0.05)
    H = gmg.Hierarchy(p)
    A = H.fine
    rng = np.random.default_rng(10)
    b, w = rng.standard_normal((2, A.shape[0]))
    solve = lambda M, rhs: spl.spsolve(M.tocsc(), rhs)
    x = solve(A, b)
    lam = solve(A.T, w)
    J = lambda M, rhs: w @ solve(M, rhs)
    h = 1e-6
    # dJ/db along a random direction
    d = rng.standard_normal(b.size)
    fd = (J(A, b + h * d) - J(A, b - h * d)) / (2 * h)
    assert lam @ d == pytest.approx(fd, rel=1e-5)
    # dJ/dA on the pattern, along a random direction scaled entry-wise by |A_ij|
    # (entries span 1e-5..1e3; a single tiny entry gives an FD signal below the
    # solve's rounding noise)
    g = adjoint.pattern_gradient(A, lam, x)
    D = A.copy()
    D.data = rng.standard_normal(A.nnz) * np.abs(A.data)
    fd = (J(A + h * D, b) - J(A - h * D, b)) / (2 * h)
    assert g @ D.data == pytest.approx(fd, rel=1e-5)
    # and one large entry on its own
    k = int(np.argmax(np.abs(A.data)))
    E = A.copy()
    E.data[:] = 0
    E.data[k] = h * abs(A.data[k])
    fd = (J(A + E, b) - J(A - E, b)) / (2 * E.data[k])
    assert g[k] == pytest.approx(fd, rel=1e-3)     # single entry: FD near the noise floor
    # dJ/dmu_s through the assembly (lambda_s held fixed)
    lev = H.levels[-1]
    gmu = adjoint.mu_s_gradient(p, lev, lam, x)
    Js = []
    for sgn in (1, -1):
        q = I.make_channel_2d(8, 2, 1, 21, band_width=0.3, mu_s=50.0, mu_f=0.05)
        q.mu_s += sgn * h * 50.0
        q.lambda_s = p.lambda_s
        Js.append(J(assemble(q, lev), b))
    assert gmu == pytest.approx((Js[0] - Js[1]) / (2 * h * 50.0), rel=1e-5)


# ---- monolithic additive Schwarz AS (the paper's comparison preconditioner, Sec. 3.2)

def test_monolithic_block_sets_bruteforce_geometry():
    """AS block of a pressure group = its p^s and p^f dofs plus every d and u
    dof (both classes) on the closure of the elements touching its vertices
    (the union of the supports of its pressures), fixed dofs removed."""
    p = I.make_channel_2d(8, 1, 2, 5, bulge=True, band_width=0.3)
    lev = mesh.build_levels(p)[0]
    h = lev.h
    got = fsasm.block_index_sets_monolithic(lev, 2)
    q2xy = mesh.lex(2, 2 * lev.n + 1) * (h / 2)
    q1xy = mesh.lex(2, lev.n + 1) * h

    def inside(e, xy):
        return ((e % lev.n) * h - 1e-12 <= xy[0] <= (e % lev.n + 1) * h + 1e-12 and
                (e // lev.n) * h - 1e-12 <= xy[1] <= (e // lev.n + 1) * h + 1e-12)

    expect = []
    for gy in range(0, lev.n + 1, 2):
        for gx in range(0, lev.n + 1, 2):
            verts = [z for z in range(lev.nq1) if gx <= q1xy[z, 0] / h < gx + 2 - 1e-9
                     and gy <= q1xy[z, 1] / h < gy + 2 - 1e-9]
            els = [e for e in range(lev.material.size) if any(inside(e, q1xy[z]) for z in verts)]
            nodes = [y for y in range(lev.nq2) if any(inside(e, q2xy[y]) for e in els)]
            s = [lev.d_dof[y, c] for y in nodes for c in (0, 1)] + [lev.v_dof[y, c] for y in nodes for c in (0, 1)]
            s += [lev.ps_dof[z] for z in verts if lev.ps_dof[z] >= 0] + [lev.pf_dof[z] for z in verts if lev.pf_dof[z] >= 0]
            s = np.array(sorted(d for d in set(s) if not lev.fixed[d]), np.int64)
            if s.size:
                expect.append(s)
    assert len(got) == len(expect)
    for a, b in zip(got, expect):
        np.testing.assert_array_equal(a, b)


def test_monolithic_partition_of_unity_and_whole_level_exact_solve():
    """AS weights sum to one on every free dof (fixed dofs: Jacobi only), and
    with one pressure group covering the level AS is the exact solve."""
    p = I.make_channel_2d(6, 1, 1, 3, bulge=True, band_width=0.4)
    lev = mesh.build_levels(p)[0]
    A = assemble(p, lev)
    S = fsasm.FSASM(A, lev, 2, monolithic=True)
    tot = np.zeros(S.n)
    for idx in S.blocks:
        tot[idx] += S.weight[idx]
    np.testing.assert_allclose(tot[~lev.fixed], 1.0, rtol=1e-15)
    assert np.all(tot[lev.fixed] == 0) and np.array_equal(np.sort(S.jacobi), np.flatnonzero(lev.fixed))
    S1 = fsasm.FSASM(A, lev, lev.n + 1, monolithic=True)
    assert len(S1.blocks) == 1
    r = np.random.default_rng(0).standard_normal(lev.n_dofs)
    np.testing.assert_allclose(S1.apply(r), spl.spsolve(A.tocsc(), r), rtol=1e-9, atol=1e-12)
    r2 = np.random.default_rng(1).standard_normal(lev.n_dofs)
    assert S.apply(r) @ r2 == pytest.approx(r @ S.apply_transpose(r2), rel=1e-11)


def test_monolithic_gmg_fgmres_matches_direct_solve(c0):
    p, _ = c0
    H = gmg.Hierarchy(p, monolithic=True)
    lev = H.levels[-1]
    b = I.gather_natural(I.natural_vector(p, 4), lev.dof_field, lev.dof_comp, lev.dof_node)
    x, st = fgmres.solve(H, b, rtol=1e-10)
    xd = spl.spsolve(H.fine.tocsc(), b)
    assert st["converged"]
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
