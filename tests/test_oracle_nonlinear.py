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
