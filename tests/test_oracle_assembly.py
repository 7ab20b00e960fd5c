"""Pins of the oracle's operator assembly (oracle/assemble.py).

* method of manufactured solutions (sympy-derived forcing, load vectors by a
  6-point Gauss rule and an independent polynomial basis) for the ALE block
  (Eq. kinfld), mixed elasticity (S/V rows) and the Oseen block (F/W rows),
  with the expected Q2 convergence rates;
* closed forms of the lumped K rows, the momentum rows applied to constant
  fields (interface rows summed over both materials), the continuity rows;
* rigid motions in the kernel of the ALE rows; symmetry of the elastic and
  ALE blocks; the zero-block pattern of Eq. matrix_J2.
"""
import numpy as np
import numpy.polynomial.legendre as leg
import pytest
import scipy.sparse.linalg as spl
import sympy as sy

from oracle import assemble as asm
from oracle import mesh
from paper_1909_13201_gb300 import inputs as I

X, Y = sy.symbols("x y")


def _basis_q2(t):
    return np.array([(2 * t - 1) * (t - 1), 4 * t * (1 - t), t * (2 * t - 1)])


def _basis_q1(t):
    return np.array([1 - t, t])


def _load(lev, f_funcs, rows_fn, kind):
    """Load vector int f phi over all elements with a 6-point Gauss rule.
    kind 'q2': f_funcs[i] is component i, rows_fn(node, i) the row;
    kind 'q1': f_funcs[0] scalar, rows_fn(vertex) the row."""
    g, wg = leg.leggauss(6)
    g = 0.5 * (g + 1)
    wg = 0.5 * wg
    F = np.zeros(lev.n_dofs)
    h = lev.h
    for e in range(lev.material.size):
        i, j = e % lev.n, e // lev.n
        for qa, wa in zip(g, wg):
            for qb, wb in zip(g, wg):
                x, y = (i + qa) * h, (j + qb) * h
                w = wa * wb * h * h
                if kind == "q2":
                    phi = np.outer(_basis_q2(qb), _basis_q2(qa)).ravel()   # local a0 + 3 a1
                    for comp, f in enumerate(f_funcs):
                        val = f(x, y)
                        for a, node in enumerate(lev.elem_q2[e]):
                            r = rows_fn(node, comp)
                            if r >= 0:
                                F[r] += w * val * phi[a]
                else:
                    psi = np.outer(_basis_q1(qb), _basis_q1(qa)).ravel()
                    val = f_funcs[0](x, y)
                    for al, z in enumerate(lev.elem_q1[e]):
                        r = rows_fn(z)
                        if r >= 0:
                            F[r] += w * val * psi[al]
    return F


def _nodes_xy(lev):
    c = mesh.lex(2, 2 * lev.n + 1) / (2 * lev.n)
    return c[:, 0], c[:, 1]


def _verts_xy(lev):
    c = mesh.lex(2, lev.n + 1) / lev.n
    return c[:, 0], c[:, 1]


def _interior_nodes(lev):
    m2 = 2 * lev.n + 1
    c = mesh.lex(2, m2)
    return np.all((c > 0) & (c < m2 - 1), 1)


def _deep_nodes(lev):
    """Q2 nodes whose touching elements have no node on the outer boundary."""
    onb = ~_interior_nodes(lev)
    bad_el = onb[lev.elem_q2].any(1)
    deep = np.ones(lev.nq2, bool)
    deep[lev.elem_q2[bad_el].ravel()] = False
    return deep


def _lam(expr):
    return sy.lambdify((X, Y), expr, "numpy")


def _ale_error(n):
    p = I.make_channel_2d(n, 1, 1, 1, band_width=0.0, mu_s=1.0, mu_f=1.0)
    lev = mesh.build_levels(p)[0]
    A = asm.assemble(p, lev)
    k = float(n) ** 2
    d = [sy.sin(sy.pi * X) * sy.sin(sy.pi * Y), sy.sin(2 * sy.pi * X) * sy.sin(sy.pi * Y)]
    grad = [[sy.diff(d[i], v) for v in (X, Y)] for i in range(2)]
    f = [-k * sum(sy.diff(grad[i][j] + grad[j][i], (X, Y)[j]) for j in range(2)) for i in range(2)]
    interior = _interior_nodes(lev)
    rows = np.concatenate([lev.d_dof[interior].ravel()])
    F = _load(lev, [_lam(fi) for fi in f], lambda node, c: lev.d_dof[node, c], "q2")
    sol = spl.spsolve(A[rows][:, rows].tocsc(), F[rows])
    x, y = _nodes_xy(lev)
    exact = np.stack([_lam(d[0])(x, y), _lam(d[1])(x, y)], 1)[interior].ravel()
    return np.abs(sol - exact).max()


def test_mms_ale_block_rate():
    e1, e2 = _ale_error(4), _ale_error(8)
    assert e2 < 2e-3
    assert np.log2(e1 / e2) > 2.8


def _elasticity_error(n, mu=3.0, lam=7.0):
    p = I.make_channel_2d(n, 1, 1, 1, band_width=2.0, mu_s=mu, mu_f=1.0)
    p.lambda_s = lam
    lev = mesh.build_levels(p)[0]
    A = asm.assemble(p, lev)
    d = [sy.sin(sy.pi * X) * sy.sin(sy.pi * Y) ** 2, X * (1 - X) * sy.sin(sy.pi * Y)]
    pr = sy.cos(sy.pi * X) * sy.cos(2 * sy.pi * Y) + X
    eps = [[(sy.diff(d[i], (X, Y)[j]) + sy.diff(d[j], (X, Y)[i])) / 2 for j in range(2)] for i in range(2)]
    f = [-sum(sy.diff(2 * mu * eps[i][j], (X, Y)[j]) for j in range(2)) + sy.diff(pr, (X, Y)[i])
         for i in range(2)]
    div = sy.diff(d[0], X) + sy.diff(d[1], Y)
    g = -div - pr / lam
    interior = _interior_nodes(lev)
    drows = lev.d_dof[interior].ravel()
    prows = lev.ps_dof[lev.ps_dof >= 0]
    rows = np.concatenate([drows, prows])
    F = _load(lev, [_lam(fi) for fi in f], lambda node, c: lev.d_dof[node, c], "q2")
    F += _load(lev, [_lam(g)], lambda z: lev.ps_dof[z], "q1")
    sol = spl.spsolve(A[rows][:, rows].tocsc(), F[rows])
    x, y = _nodes_xy(lev)
    ex_d = np.stack([_lam(d[0])(x, y), _lam(d[1])(x, y)], 1)[interior].ravel()
    vx, vy = _verts_xy(lev)
    ex_p = _lam(pr)(vx, vy)[lev.ps_dof >= 0]
    return np.abs(sol[:drows.size] - ex_d).max(), np.abs(sol[drows.size:] - ex_p).max()


def test_mms_mixed_elasticity_rates():
    (d1, p1), (d2, p2) = _elasticity_error(4), _elasticity_error(8)
    assert np.log2(d1 / d2) > 2.8
    assert np.log2(p1 / p2) > 1.8


def _oseen_error(n, mu=0.7, rho=1.3, dt=0.5):
    wexpr = [Y * (1 - Y) + 0.5 * X, -0.5 * Y + X * X]          # quadratic: Q2-exact
    p = I.make_channel_2d(n, 1, 1, 1, band_width=0.0, mu_s=1.0, mu_f=mu, dt=dt)
    p.rho_f = rho
    fine = mesh.build_levels(p)[0]
    xs, ys = _nodes_xy(fine)
    p.advection = np.stack([_lam(wexpr[0])(xs, ys) * np.ones_like(xs), _lam(wexpr[1])(xs, ys)])
    lev = fine
    A = asm.assemble(p, lev)
    psi = sy.sin(sy.pi * X) ** 2 * sy.sin(sy.pi * Y) ** 2
    u = [sy.diff(psi, Y), -sy.diff(psi, X)]                     # divergence free, zero on the boundary
    pr = sy.cos(sy.pi * X) * sy.sin(sy.pi * Y) + Y
    f = []
    for i in range(2):
        visc = sum(sy.diff(mu * (sy.diff(u[i], (X, Y)[j]) + sy.diff(u[j], (X, Y)[i])), (X, Y)[j])
                   for j in range(2))
        conv = sum(wexpr[j] * sy.diff(u[i], (X, Y)[j]) for j in range(2))
        f.append(rho / dt * u[i] + rho * conv - visc + sy.diff(pr, (X, Y)[i]))
    interior = _interior_nodes(lev)
    urows = lev.v_dof[interior].ravel()
    pf = lev.pf_dof[lev.pf_dof >= 0]
    pin, prows = pf[0], pf[1:]
    rows = np.concatenate([urows, prows])
    F = _load(lev, [_lam(fi) for fi in f], lambda node, c: lev.v_dof[node, c], "q2")
    vx, vy = _verts_xy(lev)
    ex_p_all = _lam(pr)(vx, vy)
    ex_p = ex_p_all[lev.pf_dof >= 0]
    rhs = F[rows] - A[rows][:, [pin]].toarray().ravel() * ex_p[0]
    sol = spl.spsolve(A[rows][:, rows].tocsc(), rhs)
    ex_u = np.stack([_lam(u[0])(xs, ys), _lam(u[1])(xs, ys)], 1)[interior].ravel()
    return np.abs(sol[:urows.size] - ex_u).max(), np.abs(sol[urows.size:] - ex_p[1:]).max()


def test_mms_oseen_rates():
    (u1, p1), (u2, p2) = _oseen_error(4), _oseen_error(8)
    assert np.log2(u1 / u2) > 2.8
    assert np.log2(p1 / p2) > 1.8


def _band_problem(n=8, seed=7, bulge=False):
    p = I.make_channel_2d(n, 1, 1, seed, band_width=0.3, bulge=bulge, mu_s=5.0, mu_f=0.3)
    return p, mesh.build_levels(p)[0]


def test_lumped_kinematic_rows_closed_form():
    p, lev = _band_problem()
    A = asm.assemble(p, lev).tocsr()
    h = lev.h
    m2 = 2 * lev.n + 1
    for node in np.flatnonzero(lev.q2_solid & ~lev.v_fixed):
        px, py = node % m2, node // m2
        lump = 0.0
        for e in np.flatnonzero(lev.material == 1):
            if node in lev.elem_q2[e]:
                kind = (px % 2) + (py % 2)              # 0 vertex, 1 edge, 2 centre
                lump += h * h * (1.0, 4.0, 16.0)[kind] / 36.0
        for c in range(2):
            r = lev.v_dof[node, c]
            row = A.getrow(r)
            assert row.nnz == (2 if not lev.d_fixed[node] else 1)
            assert A[r, r] == pytest.approx(lump, rel=1e-13)
            if not lev.d_fixed[node]:
                assert A[r, lev.d_dof[node, c]] == pytest.approx(-lump / p.dt, rel=1e-13)


def test_momentum_rows_on_constant_velocity_and_pressure():
    p, lev = _band_problem(bulge=False)
    p.rho_s = p.rho_f = 1.0
    A = asm.assemble(p, lev).tocsr()
    n = lev.n_dofs
    interior = _deep_nodes(lev)
    h = lev.h
    m2 = 2 * lev.n + 1
    for comp in range(2):
        u = np.zeros(n)
        u[lev.v_dof[:, comp]] = 1.0
        u[lev.fixed] = 0.0
        res = A @ u
        for node in np.flatnonzero(interior):
            # all neighbours of an interior node are free for v (fixed only on the boundary)
            px, py = node % m2, node // m2
            kind = (px % 2) + (py % 2)
            touching = 1 if kind == 2 else (2 if kind == 1 else 4)
            lump = touching * h * h * (1.0, 4.0, 16.0)[kind] / 36.0
            row = lev.d_dof[node, comp] if lev.q2_solid[node] else lev.v_dof[node, comp]
            # mass (rho/dt) over BOTH materials at interface nodes; advection of a
            # constant vanishes; no stress from a constant field
            assert res[row] == pytest.approx(lump / p.dt, rel=1e-12, abs=1e-12)
    # pressure 1 in both copies: -(1, div phi) vanishes for interior momentum rows
    q = np.zeros(n)
    q[lev.ps_dof[lev.ps_dof >= 0]] = 1.0
    q[lev.pf_dof[lev.pf_dof >= 0]] = 1.0
    res = A @ q
    for node in np.flatnonzero(interior):
        for comp in range(2):
            row = lev.d_dof[node, comp] if lev.q2_solid[node] else lev.v_dof[node, comp]
            assert abs(res[row]) < 1e-13


def test_continuity_rows_closed_form():
    p, lev = _band_problem(bulge=True, seed=3)
    A = asm.assemble(p, lev).tocsr()
    x, _ = _nodes_xy(lev)
    n = lev.n_dofs
    d = np.zeros(n)
    d[lev.d_dof[:, 0]] = x                 # d = (x, 0): div d = 1
    d[lev.fixed] = 0.0
    u = np.zeros(n)
    u[lev.v_dof[:, 0]] = x
    u[lev.fixed] = 0.0
    rd, ru = A @ d, A @ u
    onb = ~_interior_nodes(lev)
    checked = 0
    for z in range(lev.nq1):
        els = [e for e in range(lev.material.size) if z in lev.elem_q1[e]]
        if onb[lev.elem_q2[els]].any():
            continue                        # the stencil sees fixed dofs
        checked += 1
        ns = sum(lev.material[e] == 1 for e in els)
        nf = len(els) - ns
        if lev.ps_dof[z] >= 0:
            assert rd[lev.ps_dof[z]] == pytest.approx(-ns * lev.h ** 2 / 4, rel=1e-12)
        if lev.pf_dof[z] >= 0:
            assert ru[lev.pf_dof[z]] == pytest.approx(-nf * lev.h ** 2 / 4, rel=1e-12)
    assert checked > 10


def test_ale_rows_rigid_kernel_and_symmetry():
    p, lev = _band_problem(bulge=True, seed=9)
    raw = asm.assemble(p, lev, apply_bc=False).tocsr()      # before fixed rows/columns
    x, y = _nodes_xy(lev)
    arow = np.flatnonzero(lev.group == 1)
    for field in ([np.ones_like(x), 0 * x], [0 * x, np.ones_like(x)], [-y, x]):
        d = np.zeros(lev.n_dofs)
        d[lev.d_dof[:, 0]] = field[0]
        d[lev.d_dof[:, 1]] = field[1]
        # rigid motions have zero symmetric gradient: every A row vanishes
        assert np.abs((raw @ d)[arow]).max() < 1e-9
    # a non-rigid field does not vanish (guards against an all-zero block)
    d = np.zeros(lev.n_dofs)
    d[lev.d_dof[:, 0]] = x * x
    assert np.abs((raw @ d)[arow]).max() > 1.0
    A = asm.assemble(p, lev).tocsr()
    df = np.flatnonzero(lev.group == 1)
    Add = A[df][:, df]
    assert abs(Add - Add.T).max() < 1e-9 * abs(Add).max()


def test_elastic_block_symmetric_without_fluid():
    p = I.make_channel_2d(6, 1, 1, 1, band_width=2.0, mu_s=4.0)
    lev = mesh.build_levels(p)[0]
    A = asm.assemble(p, lev).tocsr()
    g = np.flatnonzero(np.isin(lev.group, (0, 2)))   # [d^s, p^s]
    B = A[g][:, g]
    assert abs(B - B.T).max() < 1e-12 * abs(B).max()


def test_mesh_velocity_coupling_closed_form():
    # all fluid, w = (y, 0): (d.grad) w = (d_y, 0), so the F row (a, x) times
    # d = e_y is -(rho/dt) int phi_a, and d = e_x gives nothing
    p = I.make_channel_2d(6, 1, 1, 1, band_width=0.0, mu_f=0.2)
    lev = mesh.build_levels(p)[0]
    x, y = _nodes_xy(lev)
    p.advection = np.stack([y, 0 * y])
    A = asm.assemble(p, lev).tocsr()
    interior = _deep_nodes(lev)
    h = lev.h
    m2 = 2 * lev.n + 1
    for comp, expect_scale in ((1, -p.rho_f / p.dt), (0, 0.0)):
        d = np.zeros(lev.n_dofs)
        d[lev.d_dof[:, comp]] = 1.0
        d[lev.fixed] = 0.0
        res = A @ d
        for node in np.flatnonzero(interior):
            px, py = node % m2, node // m2
            kind = (px % 2) + (py % 2)
            touching = 1 if kind == 2 else (2 if kind == 1 else 4)
            lump = touching * h * h * (1.0, 4.0, 16.0)[kind] / 36.0
            assert res[lev.v_dof[node, 0]] == pytest.approx(expect_scale * lump, abs=1e-12)
            assert abs(res[lev.v_dof[node, 1]]) < 1e-12


def test_j2_zero_block_pattern():
    p, lev = _band_problem(bulge=True, seed=5)
    A = asm.assemble(p, lev).tocoo()
    off = A.row != A.col
    gr, gc = lev.group[A.row[off]], lev.group[A.col[off]]
    nz = A.data[off] != 0
    present = set(zip(gr[nz].tolist(), gc[nz].tolist()))
    # groups 0 d^s/S, 1 d^f/A, 2 p^s/V, 3 u^s/K, 4 u^f/F, 5 p^f/W
    allowed = {
        0: {0, 1, 2, 3, 4, 5},
        1: {0, 1},              # A_d^s, A_d^f
        2: {0, 2},              # V_d^s (and the penalty V_p^s of the linear solid)
        3: {0, 3},              # K_d^s, K_u^s
        4: {0, 1, 3, 4, 5},     # F_d^s F_d^f F_u^s F_u^f F_p^f (no p^s)
        5: {3, 4},              # W_u^s W_u^f (W_d vanishes in the linearisation at d = 0)
    }
    for g_r, g_c in present:
        assert g_c in allowed[g_r], (g_r, g_c)
    # K rows are diagonal in each field: K_d^s and K_u^s couple node to itself
    K = A.row[(lev.group[A.row] == 3) & (A.data != 0)]
    Kc = A.col[(lev.group[A.row] == 3) & (A.data != 0)]
    assert np.all(lev.dof_node[K] == lev.dof_node[Kc])


def test_mu_s_derivative_matches_difference():
    p, lev = _band_problem(bulge=True, seed=5)
    dA = asm.assemble(p, lev, only_mu_s_derivative=True)
    h = 1e-3
    p.mu_s += h
    Ap = asm.assemble(p, lev)
    p.mu_s -= 2 * h
    Am = asm.assemble(p, lev)
    fd = (Ap - Am) / (2 * h)
    assert abs(fd - dA).max() < 1e-9 * abs(dA).max()
