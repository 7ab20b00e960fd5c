"""Pins of the oracle's nonlinear FSI residual and Newton loop (Sec. 2.2).

* the complex-step Jacobian equals central finite differences of the
  residual along random directions;
* at the rest state with no body force the residual vanishes, and the
  Jacobian there equals the linear operator assembled independently by
  oracle/assemble.py with the matching coefficients (Crank-Nicolson halves
  the solid and fluid stiffness, mu_lin = mu / 2; incompressible solid: no
  pressure mass; no frozen advection) -- the 3-point rule is exact for these
  polynomial integrands, so the two agree to rounding;
* Mooney-Rivlin objectivity: a rigid rotation of a solid element (B = I,
  stress free with p = 0 in the rest-state pressure convention) leaves zero
  momentum residual, and J = 1 gives zero continuity residual; simple shear
  (J = 1) also gives zero continuity residual;
* lambda_k of an undeformed square element equals the closed form of the
  bubble eigenproblem (sympy integration);
* Newton converges quadratically on a seeded time step.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as oasm
from oracle import mesh
from oracle import nonlinear as NL
from paper_1909_13201_gb300 import inputs as I


@pytest.fixture(scope="module")
def c0():
    p = I.make_config(0)
    return p, NL.Problem(p)


def _rand_state(pr, rng, scale):
    lev = pr.levels[-1]
    U = scale * rng.standard_normal(lev.n_dofs)
    U[lev.fixed] = 0.0
    return U


def test_complex_step_jacobian_matches_central_differences(c0):
    p, pr = c0
    fine = pr.nl[-1]
    rng = np.random.default_rng(1)
    U = _rand_state(pr, rng, 1e-3)
    Un = _rand_state(pr, rng, 1e-3)
    t = 3 * p.dt
    tau = NL.tau_lambda(fine.lev, fine.P, U, fine.maps)[0]
    J = fine.jacobian(U, Un, t, tau=tau)
    for seed in range(3):
        v = _rand_state(pr, np.random.default_rng(10 + seed), 1.0)
        eps = 1e-6
        fd = (fine.residual(U + eps * v, Un, t, tau=tau) - fine.residual(U - eps * v, Un, t, tau=tau)) / (2 * eps)
        assert np.linalg.norm(J @ v - fd) <= 1e-6 * np.linalg.norm(fd)


def test_rest_state_and_linearisation(c0):
    p, pr = c0
    P0 = NL.Params(p, force=0.0)
    lev = pr.levels[-1]
    fine = NL.LevelNL(p, lev, P0)
    Z = np.zeros(lev.n_dofs)
    t = p.dt
    assert np.abs(fine.residual(Z, Z, t)).max() == 0.0
    Jn = fine.jacobian(Z, Z, t)
    q = I.make_config(0)
    q.mu_s = p.mu_s / 2.0
    q.mu_f = p.mu_f / 2.0
    q.lambda_s = math.inf
    q.advection = np.zeros_like(p.advection)
    Al = oasm.assemble(q, lev)
    D = (Jn - Al).tocsr()
    scale = abs(Al).max(axis=1).toarray().ravel()
    rows = np.repeat(np.arange(D.shape[0]), np.diff(D.indptr))
    assert D.nnz == 0 or (np.abs(D.data) / np.maximum(scale[rows], 1e-300)).max() < 1e-12


def _solid_element(lev):
    ids = np.flatnonzero(lev.material == 1)
    return int(ids[len(ids) // 2])


def test_mooney_rivlin_objectivity_and_incompressibility(c0):
    p, pr = c0
    lev = pr.levels[-1]
    P = NL.Params(p, force=0.0)
    fine = NL.LevelNL(p, lev, P)
    e = _solid_element(lev)
    m = fine.maps
    n2 = 2 * lev.n + 1
    xy = np.stack([np.arange(n2 ** 2) % n2, np.arange(n2 ** 2) // n2], 1) / (2.0 * lev.n)   # Q2 node coordinates
    nodes = lev.elem_q2[e]
    X = xy[nodes]                                       # (9, 2)
    th = 0.3
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    for d, pressure, check_mom in (((Rm - np.eye(2)) @ X.T).T, 0.0, True), \
                                  (np.stack([0.2 * X[:, 1], np.zeros(9)], 1), 0.0, False):
        Ul = np.zeros((1, NL.NLOC))
        Ul[0, 0:18] = d.reshape(18)
        Ul[0, 36:40] = pressure
        one = NL.ElementMaps.__new__(NL.ElementMaps)
        one.solid, one.cols, one.rows = m.solid[[e]], m.cols[[e]], m.rows[[e]]
        tab = NL.shape_tables()
        fq = np.zeros((1, 9, 2))
        R = NL.element_residual(lev, P, Ul, Ul, np.zeros((1, 9)), fq, fq, one, tab)
        assert np.abs(R[0, 36:40]).max() < 1e-14                  # J = 1
        if check_mom:
            assert np.abs(R[0, 0:18]).max() < 1e-12 * max(P.C1, 1.0)   # B = I, p = 0: P = 0


def test_lambda_closed_form_on_square_element(c0):
    sympy = pytest.importorskip("sympy")
    p, pr = c0
    lev = pr.levels[-1]
    _, lam = NL.tau_lambda(lev, pr.P, np.zeros(lev.n_dofs), pr.nl[-1].maps)
    h = lev.h
    x, y = sympy.symbols("x y")
    b = 16 * x * (1 - x) * y * (1 - y) / 1                     # bubble on the unit square
    bx = lambda f, i: sympy.diff(f, [x, y][i]) / h
    H = [[bx(bx(b, i), j) for j in range(2)] for i in range(2)]
    lap = H[0][0] + H[1][1]
    K = [[sympy.integrate(sympy.integrate((lap ** 2 * (1 if i == j else 0) + 2 * lap * H[i][j]
                                            + H[i][0] * H[j][0] + H[i][1] * H[j][1]) * h * h, (x, 0, 1)), (y, 0, 1))
          for j in range(2)] for i in range(2)]
    M = sympy.integrate(sympy.integrate((bx(b, 0) ** 2 + bx(b, 1) ** 2) * h * h, (x, 0, 1)), (y, 0, 1))
    Kn = np.array([[float(K[i][j]) for j in range(2)] for i in range(2)])
    ref = np.linalg.eigvalsh(Kn).max() / float(M)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)


def test_newton_converges_quadratically():
    p = I.make_channel_2d(8, 2, 1, 5, band_width=0.3, mu_s=20.0, mu_f=0.02)
    pr = NL.Problem(p, NL.Params(p, force=400.0))
    U = np.zeros(pr.levels[-1].n_dofs)
    U, st = pr.step(U, 0.25, nl_rtol=1e-13, lin_rtol=1e-13)
    r = st["residuals"]
    assert r[-1] <= 1e-10 * r[0]
    # quadratic: r_{k+1} <= C r_k^2 with one constant once in the basin
    for k in range(1, len(r) - 1):
        if r[k] < 1e-3 * r[0] and r[k + 1] > 1e-12 * r[0]:
            assert r[k + 1] <= 100.0 * r[k] ** 2 / r[0], r


# ---------------------------------------------------------------------------
# single fluid elements with fields the Q2/Q1 spaces hold exactly, against
# integrals sympy evaluates in closed form (an evaluation independent of the
# oracle's tensor contractions and quadrature)

def _fluid_element(pr):
    lev = pr.levels[-1]
    m = pr.nl[-1].maps
    e = int(np.flatnonzero(lev.material == 0)[-1])            # top row: fluid
    one = NL.ElementMaps.__new__(NL.ElementMaps)
    one.solid, one.cols, one.rows = m.solid[[e]], m.cols[[e]], m.rows[[e]]
    return lev, one


def _sym_q2(h):
    """sympy Q2 basis on [0, h]^2 in the oracle's local order (x fastest) and
    Q1 basis; node coordinates."""
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    s, t = x / h, y / h
    L = [(2 * s - 1) * (s - 1), 4 * s * (1 - s), s * (2 * s - 1)]
    M = [(2 * t - 1) * (t - 1), 4 * t * (1 - t), t * (2 * t - 1)]
    phi = [L[a % 3] * M[a // 3] for a in range(9)]
    X = [(sympy.Rational(a % 3, 2) * h, sympy.Rational(a // 3, 2) * h) for a in range(9)]
    l1 = [1 - s, s]
    m1 = [1 - t, t]
    psi = [l1[b % 2] * m1[b // 2] for b in range(4)]
    return sympy, x, y, phi, X, psi


def _integrate(sympy, f, x, y, h):
    return float(sympy.integrate(sympy.integrate(sympy.expand(f), (x, 0, h)), (y, 0, h)))


def sympy_rational(h):
    sympy = pytest.importorskip("sympy")
    return sympy.nsimplify(h)


def test_fluid_convection_ale_and_viscous_terms_closed_form(c0):
    """Moving mesh with a uniform displacement increment (F = I, mesh velocity
    w0), a linear velocity field u with u_n = u, p = 0, f = 0, tau = 0:
    momentum row (a, i) = int rho ((u - w0).grad) u_i phi_a + mu (d_j u_i +
    d_i u_j) d_j phi_a, continuity row b = -int div u psi_b, A rows zero."""
    p, pr = c0
    lev, one = _fluid_element(pr)
    h = lev.h
    P = NL.Params(p, force=0.0)
    sympy_h = sympy_rational(h)
    sympy, x, y, phi, X, psi = _sym_q2(sympy_h)
    c = [0.3, -1.2, 0.7, 0.5, 0.9, -0.4]
    w0 = (0.8, -0.6)
    u = (c[0] + c[1] * x + c[2] * y, c[3] + c[4] * x + c[5] * y)
    Ul = np.zeros((1, NL.NLOC))
    Unl = np.zeros((1, NL.NLOC))
    for a in range(9):
        xa, ya = float(X[a][0]), float(X[a][1])
        for i in range(2):
            Ul[0, 2 * a + i] = P.dt * w0[i]                                   # d = d_n + dt w0
            val = float(u[i].subs({x: xa, y: ya}))
            Ul[0, 18 + 2 * a + i] = val
            Unl[0, 18 + 2 * a + i] = val
    fq = np.zeros((1, 9, 2))
    R = NL.element_residual(lev, P, Ul, Unl, np.zeros((1, 9)), fq, fq, one, NL.shape_tables())
    rho, mu = P.rho_f, P.mu_f
    grad = [[sympy.diff(u[i], v) for v in (x, y)] for i in range(2)]
    for a in range(9):
        for i in range(2):
            conv = sum((u[j] - w0[j]) * grad[i][j] for j in range(2))
            visc = sum(mu * (grad[i][j] + grad[j][i]) * sympy.diff(phi[a], (x, y)[j]) for j in range(2))
            ref = _integrate(sympy, rho * conv * phi[a] + visc, x, y, sympy_h)
            assert abs(R[0, 2 * a + i] - ref) <= 1e-12 * (1.0 + abs(ref)), (a, i, R[0, 2 * a + i], ref)
    assert np.abs(R[0, 18:36]).max() < 1e-12                                    # A rows: grad d = 0
    div = c[1] + c[5]
    for b in range(4):
        ref = -div * _integrate(sympy, psi[b], x, y, sympy_h)
        assert abs(R[0, 36 + b] - ref) <= 1e-13 * (1.0 + abs(ref))


@pytest.mark.parametrize("speed", [1e-4, 5.0])
def test_supg_term_closed_form(c0, speed):
    """Undeformed element, constant velocity U0 from rest (u_n = 0), p = 0,
    f = 0: the strong residual is rho U0 / dt, the SUPG test function
    rho U0.grad phi_a and tau = min(1/(4 lambda nu), 1/(sqrt(lambda) |U0|))
    with lambda of the square element in closed form; both branches of the
    minimum (slow and fast flow)."""
    p, pr = c0
    lev, one = _fluid_element(pr)
    h = lev.h
    P = NL.Params(p, force=0.0)
    sh = sympy_rational(h)
    sympy, x, y, phi, X, psi = _sym_q2(sh)
    # lambda_k of the square element (bubble eigenproblem, closed form)
    b = 16 * (x / sh) * (1 - x / sh) * (y / sh) * (1 - y / sh)
    H = [[sympy.diff(b, u_, v_) for v_ in (x, y)] for u_ in (x, y)]
    lap = H[0][0] + H[1][1]
    K = np.array([[_integrate(sympy, lap ** 2 * (1 if i == j else 0) + 2 * lap * H[i][j]
                              + H[i][0] * H[j][0] + H[i][1] * H[j][1], x, y, sh) for j in range(2)]
                  for i in range(2)])
    Mb = _integrate(sympy, sympy.diff(b, x) ** 2 + sympy.diff(b, y) ** 2, x, y, sh)
    lam = np.linalg.eigvalsh(K).max() / Mb
    nu = P.mu_f / P.rho_f
    U0 = speed * np.array([0.6, 0.8])
    tau = min(1.0 / (4.0 * lam * nu), 1.0 / (math.sqrt(lam) * np.linalg.norm(U0)))
    Ul = np.zeros((1, NL.NLOC))
    for a in range(9):
        Ul[0, 18 + 2 * a:18 + 2 * a + 2] = U0
    fq = np.zeros((1, 9, 2))
    R = NL.element_residual(lev, P, Ul, np.zeros((1, NL.NLOC)), None, fq, fq, one, NL.shape_tables())
    rho = P.rho_f
    for a in range(9):
        ip = _integrate(sympy, phi[a], x, y, sh)
        ig = _integrate(sympy, U0[0] * sympy.diff(phi[a], x) + U0[1] * sympy.diff(phi[a], y), x, y, sh)
        for i in range(2):
            ref = rho * U0[i] / P.dt * ip + tau * (rho * U0[i] / P.dt) * rho * ig
            assert abs(R[0, 2 * a + i] - ref) <= 1e-10 * (abs(ref) + rho * abs(U0[i]) / P.dt * abs(ip)), \
                (speed, a, i, R[0, 2 * a + i], ref)


def test_body_force_crank_nicolson_closed_form(c0):
    """At rest (u = u_n = 0, d = d_n = 0, p = 0) the fluid momentum rows hold
    only the body force, averaged over the two time levels: -rho/2 (f_new +
    f_old)_i int phi_a (the SUPG test function vanishes with u = w_m = 0)."""
    p, pr = c0
    lev, one = _fluid_element(pr)
    P = NL.Params(p, force=0.0)
    sh = sympy_rational(lev.h)
    sympy, x, y, phi, X, psi = _sym_q2(sh)
    fn, fo = np.array([1.5, -0.5]), np.array([-0.25, 2.0])
    fqn = np.broadcast_to(fn, (1, 9, 2)).copy()
    fqo = np.broadcast_to(fo, (1, 9, 2)).copy()
    Z = np.zeros((1, NL.NLOC))
    R = NL.element_residual(lev, P, Z, Z, None, fqn, fqo, one, NL.shape_tables())
    for a in range(9):
        ip = _integrate(sympy, phi[a], x, y, sh)
        for i in range(2):
            ref = -0.5 * P.rho_f * (fn[i] + fo[i]) * ip
            assert abs(R[0, 2 * a + i] - ref) <= 1e-13 * (1.0 + abs(ref))


def test_mooney_rivlin_homogeneous_deformation_closed_form(c0):
    """A solid element under the homogeneous deformation F = [[s1, g], [0, s2]]
    from rest (d_n = 0: P_el(F_n) = 0 in the rest-state convention), u = u_n =
    0, constant pressure p0: momentum row (a, i) = sum_J T_iJ int d_J phi_a with
    the constant stress T = 1/2 P_el(F) - p0 J F^{-T}, P_el = J sigma_el F^{-T}
    (the first Piola-Kirchhoff stress), sigma_el = 2 C1 (B - I) - 2 C2 (B^{-1} -
    I), B = F F^T -- the law's two invariant terms, which a rigid rotation
    cannot tell apart, and the transposes a shear exposes; V rows -(J - 1)
    int psi_b; K rows -M_L d / dt."""
    p, pr = c0
    lev = pr.levels[-1]
    m = pr.nl[-1].maps
    e = int(np.flatnonzero(lev.material == 1)[0])
    one = NL.ElementMaps.__new__(NL.ElementMaps)
    one.solid, one.cols, one.rows = m.solid[[e]], m.cols[[e]], m.rows[[e]]
    P = NL.Params(p, force=0.0)
    sh = sympy_rational(lev.h)
    sympy, x, y, phi, X, psi = _sym_q2(sh)
    s1, s2, g, p0 = 1.03, 0.98, 0.07, 0.37
    F = np.array([[s1, g], [0.0, s2]])
    Ul = np.zeros((1, NL.NLOC))
    for a in range(9):
        Xa = np.array([float(X[a][0]), float(X[a][1])])
        Ul[0, 2 * a:2 * a + 2] = (F - np.eye(2)) @ Xa
    Ul[0, 36:40] = p0
    fq = np.zeros((1, 9, 2))
    R = NL.element_residual(lev, P, Ul, np.zeros((1, NL.NLOC)), np.zeros((1, 9)), fq, fq, one, NL.shape_tables())
    J = np.linalg.det(F)
    FiT = np.linalg.inv(F).T
    B = F @ F.T
    sig = 2 * P.C1 * (B - np.eye(2)) - 2 * P.C2 * (np.linalg.inv(B) - np.eye(2))
    T = 0.5 * J * sig @ FiT - p0 * J * FiT
    for a in range(9):
        dphi = [_integrate(sympy, sympy.diff(phi[a], v), x, y, sh) for v in (x, y)]
        for i in range(2):
            ref = T[i, 0] * dphi[0] + T[i, 1] * dphi[1]
            assert abs(R[0, 2 * a + i] - ref) <= 1e-12 * (1.0 + np.abs(T).max() * lev.h), (a, i, R[0, 2 * a + i], ref)
        lump = _integrate(sympy, phi[a], x, y, sh)
        for i in range(2):
            assert abs(R[0, 18 + 2 * a + i] + lump * Ul[0, 2 * a + i] / P.dt) <= 1e-12 * (1 + abs(Ul[0, 2 * a + i]) / P.dt)
    for b in range(4):
        ref = -(J - 1.0) * _integrate(sympy, psi[b], x, y, sh)
        assert abs(R[0, 36 + b] - ref) <= 1e-13


def test_fluid_on_deformed_element_closed_form(c0):
    """Fluid element moved by the homogeneous deformation F = [[s1, g], [0,
    s2]] (d = d_n: no mesh velocity), a velocity u = G X linear in the
    reference coordinates with u_n = u, p = 0, f = 0, tau = 0: with the spatial
    gradient Gx = G F^{-1} (constant) and J = det F, momentum row (a, i) =
    int J [rho (u . Gx^T)_i phi_a + (mu (Gx + Gx^T) F^{-T})_iK d_K phi_a] dX
    and continuity row b = -J tr(Gx) int psi_b (the ALE map of gradients and
    volumes, Sec. 2.2)."""
    p, pr = c0
    lev, one = _fluid_element(pr)
    P = NL.Params(p, force=0.0)
    sh = sympy_rational(lev.h)
    sympy, x, y, phi, X, psi = _sym_q2(sh)
    F = np.array([[1.04, 0.06], [0.0, 0.97]])
    G = np.array([[0.4, -1.1], [0.8, 0.3]])
    Ul = np.zeros((1, NL.NLOC))
    for a in range(9):
        Xa = np.array([float(X[a][0]), float(X[a][1])])
        Ul[0, 2 * a:2 * a + 2] = (F - np.eye(2)) @ Xa
        Ul[0, 18 + 2 * a:18 + 2 * a + 2] = G @ Xa
    fq = np.zeros((1, 9, 2))
    R = NL.element_residual(lev, P, Ul, Ul.copy(), np.zeros((1, 9)), fq, fq, one, NL.shape_tables())
    J = np.linalg.det(F)
    Fi = np.linalg.inv(F)
    Gx = G @ Fi
    T = P.mu_f * (Gx + Gx.T) @ Fi.T
    uX = [G[i, 0] * x + G[i, 1] * y for i in range(2)]
    conv = [sum(uX[j] * Gx[i, j] for j in range(2)) for i in range(2)]
    for a in range(9):
        for i in range(2):
            ref = J * _integrate(sympy, P.rho_f * conv[i] * phi[a] + T[i, 0] * sympy.diff(phi[a], x)
                                 + T[i, 1] * sympy.diff(phi[a], y), x, y, sh)
            assert abs(R[0, 2 * a + i] - ref) <= 1e-12 * (1.0 + abs(ref)), (a, i, R[0, 2 * a + i], ref)
    for b in range(4):
        ref = -J * np.trace(Gx) * _integrate(sympy, psi[b], x, y, sh)
        assert abs(R[0, 36 + b] - ref) <= 1e-13 * (1.0 + abs(ref))


def test_supg_strong_residual_viscous_and_pressure_terms(c0):
    """Undeformed element, slow quadratic velocity u (tau in its 1/(4 lambda
    nu) branch: constant), u_n = 0, bilinear pressure p, f = 0: momentum row
    (a, i) = int [rho u_i / dt phi_a + 1/2 (rho (u.grad u)_i phi_a + mu (grad u +
    grad u^T) : grad (phi_a e_i)) - p d_i phi_a] + tau int r_i rho (u.grad phi_a)
    (Crank-Nicolson: the old state contributes nothing from rest; pressure
    and strong residual at the new level)
    with the strong residual r = rho u / dt + rho u.grad u + grad p - mu
    div(grad u + grad u^T) -- derivatives by sympy, integrals by the
    3-point Gauss rule of the method (the SUPG integrand's degree exceeds what
    the rule integrates exactly)."""
    p, pr = c0
    lev, one = _fluid_element(pr)
    P = NL.Params(p, force=0.0)
    sh = sympy_rational(lev.h)
    sympy, x, y, phi, X, psi = _sym_q2(sh)
    # |u| below 4 sqrt(lambda) nu (~4.7 here): tau takes its constant branch;
    # the viscous and pressure parts of r are a few per cent of it
    u = [0.3 + 2.0 * x - 1.5 * y + 40.0 * x * y - 30.0 * x ** 2,
         -0.2 + 1.0 * x + 0.5 * y + 25.0 * y ** 2 - 35.0 * x * y]
    pf = 0.01 * (0.6 - 2.0 * x / sh + 1.3 * y / sh + 0.9 * x * y / sh ** 2)
    Ul = np.zeros((1, NL.NLOC))
    for a in range(9):
        for i in range(2):
            Ul[0, 18 + 2 * a + i] = float(u[i].subs({x: X[a][0], y: X[a][1]}))
    for b in range(4):
        Ul[0, 36 + b] = float(pf.subs({x: sh * (b % 2), y: sh * (b // 2)}))
    fq = np.zeros((1, 9, 2))
    R = NL.element_residual(lev, P, Ul, np.zeros((1, NL.NLOC)), None, fq, fq, one, NL.shape_tables())
    tau, lam = NL.tau_local(float(sh), P, np.zeros((1, 9, 2)), Ul[:, 18:36].reshape(1, 9, 2), NL.shape_tables())
    assert np.allclose(tau, 1.0 / (4.0 * lam[0] * P.mu_f / P.rho_f), rtol=1e-14)     # the constant branch
    t = 1.0 / (4.0 * lam[0] * P.mu_f / P.rho_f)
    rho, mu, dt = P.rho_f, P.mu_f, P.dt
    gu = [[sympy.diff(u[i], v) for v in (x, y)] for i in range(2)]
    conv = [u[0] * gu[i][0] + u[1] * gu[i][1] for i in range(2)]
    gp = [sympy.diff(pf, x), sympy.diff(pf, y)]
    divs = [sum(sympy.diff(gu[i][j] + gu[j][i], (x, y)[j]) for j in range(2)) for i in range(2)]
    r = [rho * u[i] / dt + rho * conv[i] + gp[i] - mu * divs[i] for i in range(2)]
    gx = [0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)]
    gw = [5 / 18, 8 / 18, 5 / 18]
    hf = float(sh)
    for a in range(9):
        dphi = [sympy.diff(phi[a], v) for v in (x, y)]
        for i in range(2):
            integrand = (rho * u[i] / dt * phi[a]
                         + 0.5 * (rho * conv[i] * phi[a] + sum(mu * (gu[i][j] + gu[j][i]) * dphi[j] for j in range(2)))
                         - pf * dphi[i]
                         + t * r[i] * rho * (u[0] * dphi[0] + u[1] * dphi[1]))
            fn = sympy.lambdify((x, y), integrand, "math")
            ref = sum(gw[k] * gw[l] * hf * hf * fn(gx[k] * hf, gx[l] * hf) for k in range(3) for l in range(3))
            assert abs(R[0, 2 * a + i] - ref) <= 1e-11 * (1.0 + abs(ref)), (a, i, R[0, 2 * a + i], ref)


def test_injection_maps_coinciding_nodes(c0):
    """The coarse state takes each coarse dof's value from the fine dof of the
    same field and component at the same point (Q2 nodes and Q1 vertices of
    a coarse level are nodes of the finer one); fixed coarse dofs are zero."""
    p, pr = c0
    for l in range(1, len(pr.levels)):
        fine, coarse = pr.levels[l], pr.levels[l - 1]
        inj = pr.inj[l]
        def coords(lev, dof):
            q2 = lev.dof_field[dof] < 2                 # Q2 node (d, u) or Q1 vertex (p)
            node = lev.dof_node[dof]
            m = np.where(q2, 2 * lev.n + 1, lev.n + 1)
            step = np.where(q2, 0.5 * lev.h, lev.h)
            return np.stack([(node % m) * step, (node // m) * step], -1)
        has = inj >= 0
        cd = np.flatnonzero(has)
        fd = inj[has]
        assert np.array_equal(coarse.dof_field[cd], fine.dof_field[fd])
        assert np.array_equal(coarse.dof_comp[cd], fine.dof_comp[fd])
        np.testing.assert_allclose(coords(coarse, cd), coords(fine, fd), atol=1e-15)
        # every coarse d/u dof has a fine partner; pressure copies may not
        assert np.all(has[coarse.dof_field < 2])
        U = np.random.default_rng(l).standard_normal(fine.n_dofs)
        Uc = NL.inject(U, inj, coarse)
        assert np.all(Uc[coarse.fixed] == 0.0)
        free = has & ~coarse.fixed
        assert np.array_equal(Uc[free], U[inj[free]])
