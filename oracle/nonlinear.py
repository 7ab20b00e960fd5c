"""Nonlinear monolithic FSI residual, its Newton Jacobian and the ALE Newton /
Crank-Nicolson time loop (Sec. 2.2), 2D -- test infrastructure (oracle).

Unknowns U = (d, u, p) in the J2 numbering of mesh.Level.  Per element of
the reference mesh (side h, 3-point Gauss rule per direction) the residual
has three groups of rows:

  momentum (Eq. momentum_supg; S rows at solid-class nodes, F rows at fluid
  nodes, test phi_a e_i), Crank-Nicolson for the spatial operator and a
  backward difference for the time derivatives (Sec. 2.2):
    solid elements (total Lagrangian on the reference solid, Mooney-Rivlin
    sigma = -p I + 2 C1 B - 2 C2 B^{-1}, B = F F^T, F = I + grad_X d,
    P = J sigma F^{-T}, C1 = mu_s / 3, C2 = C1 / 2; the pressure unknown is
    measured from the rest state's hydrostatic stress 2 (C1 - C2), i.e.
    sigma = -p I + 2 C1 (B - I) - 2 C2 (B^{-1} - I), so d = 0, p = 0 is
    stress free):
      int rho_s (u - u_n)/dt phi_a + [1/2 (P_el(U) + P_el(U_n)) - p J F^{-T}] : grad_X (phi_a e_i)
    (P_el the elastic part of P; the pressure, a Lagrange multiplier, acts at
    the new time level)
    fluid elements (ALE on the current element x = X + d: grad_x = F^{-T}
    grad_X, dx = J dX; sigma_f = -p I + mu (grad_x u + grad_x u^T); mesh
    velocity w_m = (d - d_n)/dt; body force rho_f f):
      int J rho_f (u - u_n)_i/dt phi_a + 1/2 (G(U) + G(U_n)),
        - int J p div_x (phi_a e_i)   (pressure at the new time level),
      G(U) = int J [rho_f ((u - w_m).grad_x) u_i phi_a + mu (grad_x u + grad_x u^T) : grad_x (phi_a e_i)
                    - rho_f f_i phi_a]
      + SUPG: int J tau r_i rho_f ((u - w_m).grad_x) phi_a with the strong
      residual r = rho_f (u - u_n)/dt + rho_f ((u - w_m).grad_x) u + grad_x p
      - mu div_x (grad_x u + grad_x u^T) - rho_f f (at the new state);
  kinematic rows: solid (K, Eq. kinsld): row-sum lumped mass, M_L (u - (d - d_n)/dt);
    fluid-class nodes (A, Eq. kinfld): int k (grad_X d + grad_X d^T) : grad_X phi_a, k = 1/V_el;
  continuity rows: solid (V, Eq. cntsld): -int (J - 1) psi_b; fluid (W, Eq. cntfld):
    -int J (div_x u) psi_b.
Fixed (Dirichlet) dofs: R_i = U_i.

tau (Eq. tausupg): xi(Re_k) / (sqrt(lambda_k) |u|), Re_k = |u| / (4 sqrt(lambda_k) nu),
nu = mu_f / rho_f, lambda_k the largest eigenvalue of the generalized
problem of Eq. lambda_k on the current element, V_0(T) = the element's bubble
(its centre node, both components), solved by the power method (50 steps
from (1, 1)); tau = min(1/(4 lambda nu), 1/(sqrt(lambda) |u|)).  tau is
a function of the state like the rest of the residual and is differentiated
with it (exact Newton).  Second derivatives on the moving element use the mapping at the quadrature
point (its curvature is not differentiated).

The exact Jacobian of the element residual is taken by complex-step
differentiation (Im R(U + i e h) / h, exact to rounding for this analytic
residual).  Coarse levels rediscretise the residual at the state injected
from the finer level (coinciding nodes).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .mesh import Level, level_advection

# 3-point Gauss-Legendre rule on [0, 1]
G3X = 0.5 + 0.5 * np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
G3W = 0.5 * np.array([5.0, 8.0, 5.0]) / 9.0
NLOC = 40            # 9 nodes x (2 d + 2 u) + 4 pressures


def _q2(x):
    v = np.array([(2 * x - 1) * (x - 1), 4 * x * (1 - x), x * (2 * x - 1)])
    d = np.array([4 * x - 3, 4 - 8 * x, 4 * x - 1])
    dd = np.array([4.0, -8.0, 4.0])
    return v, d, dd


def shape_tables():
    """At the 9 quadrature points (x fastest): Q2 values phi (9, 9),
    gradients dphi (9, 2, 9), second derivatives ddphi (9, 2, 2, 9), Q1
    values psi (9, 4), gradients dpsi (9, 2, 4), weights (9,)."""
    phi = np.zeros((9, 9)); dphi = np.zeros((9, 2, 9)); ddphi = np.zeros((9, 2, 2, 9))
    psi = np.zeros((9, 4)); dpsi = np.zeros((9, 2, 4)); wq = np.zeros(9)
    for q1i in range(3):
        for q0i in range(3):
            q = q0i + 3 * q1i
            x, y = G3X[q0i], G3X[q1i]
            wq[q] = G3W[q0i] * G3W[q1i]
            vx, dx, ddx = _q2(x)
            vy, dy, ddy = _q2(y)
            for a1 in range(3):
                for a0 in range(3):
                    a = a0 + 3 * a1
                    phi[q, a] = vx[a0] * vy[a1]
                    dphi[q, 0, a] = dx[a0] * vy[a1]
                    dphi[q, 1, a] = vx[a0] * dy[a1]
                    ddphi[q, 0, 0, a] = ddx[a0] * vy[a1]
                    ddphi[q, 1, 1, a] = vx[a0] * ddy[a1]
                    ddphi[q, 0, 1, a] = ddphi[q, 1, 0, a] = dx[a0] * dy[a1]
            lx, ly = np.array([1 - x, x]), np.array([1 - y, y])
            for b1 in range(2):
                for b0 in range(2):
                    b = b0 + 2 * b1
                    psi[q, b] = lx[b0] * ly[b1]
                    dpsi[q, 0, b] = (-1.0 if b0 == 0 else 1.0) * ly[b1]
                    dpsi[q, 1, b] = lx[b0] * (-1.0 if b1 == 0 else 1.0)
    return phi, dphi, ddphi, psi, dpsi, wq


class Params:
    """Physical and time-stepping data of the nonlinear problem."""

    def __init__(self, prob, force: float = 20.0, period: float = 1.0):
        self.rho_s, self.rho_f, self.mu_f, self.dt = prob.rho_s, prob.rho_f, prob.mu_f, prob.dt
        self.C1 = prob.mu_s / 3.0
        self.C2 = self.C1 / 2.0
        self.k_ale = float(prob.n_fine) ** 2
        self.force, self.period = force, period

    def force_factor(self, t: float) -> float:
        return self.force * math.sin(2.0 * math.pi * t / self.period)


class ElementMaps:
    """Per element: the local unknown -> global dof map (cols, -1 where the
    dof does not exist) and the local residual -> global row map (rows, -1
    where the equation is not assembled there)."""

    def __init__(self, lev: Level):
        assert lev.dim == 2, "the nonlinear residual is 2D"
        ne = lev.material.size
        q2, q1 = lev.elem_q2, lev.elem_q1
        self.solid = lev.material == 1
        cols = np.full((ne, NLOC), -1, np.int64)
        rows = np.full((ne, NLOC), -1, np.int64)
        d = lev.d_dof[q2]                       # (ne, 9, 2)
        v = lev.v_dof[q2]
        cols[:, 0:18] = d.reshape(ne, 18)
        cols[:, 18:36] = v.reshape(ne, 18)
        p = np.where(self.solid[:, None], lev.ps_dof[q1], lev.pf_dof[q1])
        cols[:, 36:40] = p
        sn = lev.q2_solid[q2]                   # (ne, 9) solid-class nodes
        mom = np.where(self.solid[:, None, None] | sn[..., None], d, v)
        rows[:, 0:18] = mom.reshape(ne, 18)
        kin = np.where(self.solid[:, None, None], v, np.where(sn[..., None], -1, d))
        rows[:, 18:36] = kin.reshape(ne, 18)
        rows[:, 36:40] = p
        self.cols, self.rows = cols, rows


def gather(U: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Local unknowns (ne, 40); 0 where a dof does not exist."""
    out = np.zeros(cols.shape, dtype=U.dtype)
    m = cols >= 0
    out[m] = U[cols[m]]
    return out


def _split(Ul):
    ne = Ul.shape[0]
    return Ul[:, 0:18].reshape(ne, 9, 2), Ul[:, 18:36].reshape(ne, 9, 2), Ul[:, 36:40]


def _kinematics(d, h, dphi):
    """F (ne, nq, 2, 2), J, F^{-1} from the nodal displacements d (ne, 9, 2)."""
    gd = np.einsum("eai,qJa->eqiJ", d, dphi) / h
    F = gd + np.eye(2)
    J = F[..., 0, 0] * F[..., 1, 1] - F[..., 0, 1] * F[..., 1, 0]
    Fi = np.empty_like(F)
    Fi[..., 0, 0] = F[..., 1, 1] / J
    Fi[..., 1, 1] = F[..., 0, 0] / J
    Fi[..., 0, 1] = -F[..., 0, 1] / J
    Fi[..., 1, 0] = -F[..., 1, 0] / J
    return gd, F, J, Fi


def tau_local(h: float, P: Params, d, u, tables):
    """SUPG parameter tau (ne, nq) and lambda_k (ne,) from local nodal d and u
    (Eqs. tausupg, lambda_k; power method on the bubble space).  Written
    without moduli or conjugates, so complex-step differentiation goes
    through it: tau is part of the exact Newton linearisation."""
    phi, dphi, ddphi, psi, dpsi, wq = tables
    _, F, J, Fi = _kinematics(d, h, dphi)
    b = 4                                                    # centre node: the bubble
    gb = np.einsum("qJ,eqJj->eqj", dphi[:, :, b] / h, Fi)   # grad_x b
    Hx = np.einsum("qJK,eqJj,eqKk->eqjk", ddphi[:, :, :, b] / h ** 2, Fi, Fi)
    lap = Hx[..., 0, 0] + Hx[..., 1, 1]
    dX = wq * h * h
    K = np.einsum("eq,eqij->eij", dX * J, lap[..., None, None] ** 2 * np.eye(2) + 2 * lap[..., None, None] * Hx
                  + np.einsum("eqik,eqjk->eqij", Hx, Hx))
    M = np.einsum("eq,eq->e", dX * J, np.sum(gb * gb, -1))
    a = np.ones((K.shape[0], 2), dtype=K.dtype)
    for _ in range(50):
        a = np.einsum("eij,ej->ei", K, a) / M[:, None]
        a = a / np.sqrt(np.sum(a * a, 1))[:, None]
    lam = np.einsum("ei,eij,ej->e", a, K, a) / (M * np.sum(a * a, 1))
    uq = np.einsum("eai,qa->eqi", u, phi)
    speed = np.sqrt(np.sum(uq * uq, -1))
    nu = P.mu_f / P.rho_f
    t1 = np.broadcast_to((1.0 / (4.0 * lam * nu))[:, None], speed.shape)
    moving = speed.real > 0
    t2 = 1.0 / (np.sqrt(lam)[:, None] * np.where(moving, speed, 1.0))
    tau = np.where(moving & (t2.real < t1.real), t2, t1)
    return tau, lam


def tau_lambda(lev: Level, P: Params, U: np.ndarray, maps: ElementMaps, tables=None):
    """tau and lambda_k at the global state U (real)."""
    d, u, _ = _split(gather(U, maps.cols))
    return tau_local(lev.h, P, d, u, tables or shape_tables())


def element_residual(lev: Level, P: Params, Ul, Unl, tau, fq_new, fq_old, maps: ElementMaps, tables=None):
    """Local residuals (ne, 40) in the row layout of ElementMaps; Ul may be
    complex (complex-step differentiation).  tau None: from Ul (differentiated
    with the rest); an array: held fixed."""
    tables = tables or shape_tables()
    phi, dphi, ddphi, psi, dpsi, wq = tables
    h = lev.h
    ne = Ul.shape[0]
    dX = wq * h * h                                            # (nq,)
    lump = np.einsum("q,qa->a", dX, phi)                       # int phi_a
    d, u, p = _split(Ul)
    dn, un, pn = _split(Unl)
    if tau is None:
        tau = tau_local(h, P, d, u, tables)[0]
    R = np.zeros((ne, NLOC), dtype=np.result_type(Ul, np.float64))
    sol = maps.solid
    dq, dnq = np.einsum("eai,qa->eqi", d, phi), np.einsum("eai,qa->eqi", dn, phi)
    uq, unq = np.einsum("eai,qa->eqi", u, phi), np.einsum("eai,qa->eqi", un, phi)
    wm = (dq - dnq) / P.dt
    gd, F, J, Fi = _kinematics(d, h, dphi)
    gdn, Fn, Jn, Fin = _kinematics(dn, h, dphi)
    pq, pnq = np.einsum("eb,qb->eq", p, psi), np.einsum("eb,qb->eq", pn, psi)
    # ---------------- solid elements
    if sol.any():
        s = sol

        def piola(F_, J_, Fi_):
            B = np.einsum("eqiK,eqjK->eqij", F_, F_)
            Bi = np.einsum("eqKi,eqKj->eqij", Fi_, Fi_)         # F^{-T} F^{-1}
            I2 = np.eye(2)
            sig = 2 * P.C1 * (B - I2) - 2 * P.C2 * (Bi - I2)
            return J_[..., None, None] * np.einsum("eqij,eqKj->eqiK", sig, Fi_)   # J sigma F^{-T}
        # elastic stress by Crank-Nicolson; the pressure (a multiplier) at the new state
        Pm = 0.5 * (piola(F[s], J[s], Fi[s]) + piola(Fn[s], Jn[s], Fin[s]))
        Pm = Pm - (pq[s] * J[s])[..., None, None] * np.swapaxes(Fi[s], -1, -2)
        mass = P.rho_s * np.einsum("q,eqi,qa->eai", dX, uq[s] - unq[s], phi) / P.dt
        stiff = np.einsum("q,eqiJ,qJa->eai", dX, Pm, dphi) / h
        R[s, 0:18] = (mass + stiff).reshape(-1, 18)
        kin = lump[None, :, None] * (u[s] - (d[s] - dn[s]) / P.dt)
        R[s, 18:36] = kin.reshape(-1, 18)
        R[s, 36:40] = -np.einsum("q,eq,qb->eb", dX, J[s] - 1.0, psi)
    # ---------------- fluid elements
    f = ~sol
    if f.any():
        Jf, Fif, Jnf, Finf = J[f], Fi[f], Jn[f], Fin[f]
        wmf = wm[f]

        def spatial(J_, Fi_, u_, uq_, fq_):
            gu = np.einsum("eai,qJa->eqiJ", u_, dphi) / h
            gxu = np.einsum("eqiJ,eqJj->eqij", gu, Fi_)
            gxphi = np.einsum("qJa,eqJj->eqaj", dphi / h, Fi_)
            conv = np.einsum("eqj,eqij->eqi", uq_ - wmf, gxu)
            sig = P.mu_f * (gxu + np.swapaxes(gxu, -1, -2))
            g = np.einsum("q,eq,eqi,qa->eai", dX, J_, P.rho_f * (conv - fq_), phi)
            g += np.einsum("q,eq,eqij,eqaj->eai", dX, J_, sig, gxphi)
            return g, gxu, gxphi, conv
        fqn, fqo = fq_new[f], fq_old[f]
        gN, gxu, gxphi, conv = spatial(Jf, Fif, u[f], uq[f], fqn)
        gO, _, _, _ = spatial(Jnf, Finf, un[f], unq[f], fqo)
        # pressure (a multiplier) at the new state: -int J p div_x phi
        pres = -np.einsum("q,eq,eq,eqaj->eaj", dX, Jf, pq[f], gxphi)
        mass = P.rho_f * np.einsum("q,eq,eqi,qa->eai", dX, Jf, uq[f] - unq[f], phi) / P.dt
        # SUPG at the new state (tau frozen)
        hu = np.einsum("eai,qJKa->eqiJK", u[f], ddphi) / h ** 2
        hxu = np.einsum("eqiJK,eqJj,eqKk->eqijk", hu, Fif, Fif)
        visc = np.einsum("eqijj->eqi", hxu) + np.einsum("eqjji->eqi", hxu)
        gp = np.einsum("eb,qJb,eqJj->eqj", p[f], dpsi / h, Fif)
        r = P.rho_f * (uq[f] - unq[f]) / P.dt + P.rho_f * conv + gp - P.mu_f * visc - P.rho_f * fqn
        sa = P.rho_f * np.einsum("eqj,eqaj->eqa", uq[f] - wmf, gxphi)
        supg = np.einsum("q,eq,eq,eqi,eqa->eai", dX, Jf, tau[f], r, sa)
        R[f, 0:18] = (mass + 0.5 * (gN + gO) + pres + supg).reshape(-1, 18)
        gdf = gd[f]
        ale = P.k_ale * np.einsum("q,eqiJ,qJa->eai", dX, gdf + np.swapaxes(gdf, -1, -2), dphi) / h
        R[f, 18:36] = ale.reshape(-1, 18)
        divu = np.einsum("eqii->eq", gxu)
        R[f, 36:40] = -np.einsum("q,eq,eq,qb->eb", dX, Jf, divu, psi)
    return R


def force_at_quadrature(prob, lev: Level, factor: float, tables=None) -> np.ndarray:
    """rho-free body force f (ne, nq, 2): the seeded divergence-free field of
    the workload (zero at solid-class nodes) times the time factor."""
    phi = (tables or shape_tables())[0]
    w = level_advection(prob, lev)                             # (2, nq2)
    wn = w[:, lev.elem_q2].transpose(1, 2, 0)                  # (ne, 9, 2)
    return factor * np.einsum("eai,qa->eqi", wn, phi)


class LevelNL:
    """One level of the nonlinear problem: maps, shape tables, fixed dofs."""

    def __init__(self, prob, lev: Level, P: Params):
        self.prob, self.lev, self.P = prob, lev, P
        self.maps = ElementMaps(lev)
        self.tables = shape_tables()
        self.n = lev.n_dofs

    def residual_local(self, U, Un, tau, t_new, Ul=None):
        m = self.maps
        Ul = gather(U, m.cols) if Ul is None else Ul
        fn = force_at_quadrature(self.prob, self.lev, self.P.force_factor(t_new), self.tables)
        fo = force_at_quadrature(self.prob, self.lev, self.P.force_factor(t_new - self.P.dt), self.tables)
        return element_residual(self.lev, self.P, Ul, gather(Un, m.cols), tau, fn, fo, m, self.tables)

    def residual(self, U, Un, t_new, tau=None):
        """Global residual R(U; U_n) (fixed rows: U); tau from U unless given."""
        Rl = self.residual_local(U, Un, tau, t_new)
        m = self.maps
        R = np.zeros(self.n)
        keep = m.rows >= 0
        np.add.at(R, m.rows[keep], Rl[keep].real)
        fx = self.lev.fixed
        R[fx] = U[fx]
        return R

    def jacobian(self, U, Un, t_new, tau=None, step=1e-30):
        """dR/dU at U (with tau differentiated, or held at a given array):
        element Jacobians by complex-step differentiation, assembled; fixed
        rows identity, fixed columns dropped."""
        m = self.maps
        Ul = gather(U, m.cols).astype(np.complex128)
        ne = Ul.shape[0]
        Jl = np.zeros((ne, NLOC, NLOC))
        for t in range(NLOC):
            Up = Ul.copy()
            Up[:, t] += 1j * step
            Jl[:, :, t] = self.residual_local(None, Un, tau, t_new, Ul=Up).imag / step
        r = np.broadcast_to(m.rows[:, :, None], Jl.shape)
        c = np.broadcast_to(m.cols[:, None, :], Jl.shape)
        fx = self.lev.fixed
        keep = (r >= 0) & (c >= 0)
        keep &= ~fx[np.where(r >= 0, r, 0)] & ~fx[np.where(c >= 0, c, 0)]
        A = sp.coo_matrix((Jl[keep], (r[keep], c[keep])), shape=(self.n, self.n)).tocsr()
        A = A + sp.diags(fx.astype(np.float64))
        A = A.tocsr()
        A.sum_duplicates()
        A.sort_indices()
        return A


def injection(fine: Level, coarse: Level) -> np.ndarray:
    """Coarse dof -> fine dof at the coinciding node (-1: no such fine dof),
    for states restricted by injection to the coarse level."""
    out = np.full(coarse.n_dofs, -1, np.int64)
    mc2, mf2 = 2 * coarse.n + 1, 2 * fine.n + 1
    cq = np.arange(mc2 ** 2)
    fq = (2 * (cq % mc2)) + mf2 * (2 * (cq // mc2))
    for i in range(2):
        out[coarse.d_dof[cq, i]] = fine.d_dof[fq, i]
        out[coarse.v_dof[cq, i]] = fine.v_dof[fq, i]
    mc1, mf1 = coarse.n + 1, fine.n + 1
    cv = np.arange(mc1 ** 2)
    fv = (2 * (cv % mc1)) + mf1 * (2 * (cv // mc1))
    for cmap, fmap in ((coarse.ps_dof, fine.ps_dof), (coarse.pf_dof, fine.pf_dof)):
        has = cmap[cv] >= 0
        out[cmap[cv[has]]] = fmap[fv[has]]
    return out


def inject(U_f: np.ndarray, inj: np.ndarray, coarse: Level) -> np.ndarray:
    U = np.zeros(coarse.n_dofs)
    has = inj >= 0
    U[has] = U_f[inj[has]]
    U[coarse.fixed] = 0.0
    return U


class Problem:
    """The nonlinear time loop on a hierarchy: state U (fine level), per time
    step Newton iterations J(U_k) dU = -R(U_k), each linear system solved by
    FGMRES with the GMG preconditioner whose level operators are the
    Jacobians rediscretised at the injected states (Sec. 2.2, Sec. 3.2)."""

    def __init__(self, prob, P: Params | None = None):
        from .mesh import build_levels
        self.prob = prob
        self.P = P or Params(prob)
        self.levels = build_levels(prob)
        self.nl = [LevelNL(prob, lev, self.P) for lev in self.levels]
        self.inj = [None] + [injection(self.levels[l], self.levels[l - 1]) for l in range(1, len(self.levels))]

    def level_states(self, U):
        out = [None] * len(self.levels)
        out[-1] = U
        for l in range(len(self.levels) - 1, 0, -1):
            out[l - 1] = inject(out[l], self.inj[l], self.levels[l - 1])
        return out

    def jacobians(self, U, Un, t_new):
        Us, Uns = self.level_states(U), self.level_states(Un)
        return [self.nl[l].jacobian(Us[l], Uns[l], t_new) for l in range(len(self.levels))]

    def step(self, U_n, t_new, nl_rtol=1e-8, lin_rtol=1e-8, max_newton=10, **hier_kw):
        """One time step from U_n: returns U, and per Newton step the linear
        iterations N and rates rho = (r_N / r_0)^(1/N), and the residual norms."""
        from . import fgmres, gmg
        fine = self.nl[-1]
        U = U_n.copy()
        R = fine.residual(U, U_n, t_new)
        r0 = np.linalg.norm(R)
        res, its, rates = [r0], [], []
        for _ in range(max_newton):
            if res[-1] <= nl_rtol * max(r0, 1e-300) or res[-1] == 0.0:
                break
            ops = self.jacobians(U, U_n, t_new)
            H = gmg.Hierarchy(self.prob, operators=ops, **hier_kw)
            dU, st = fgmres.solve(H, -R, rtol=lin_rtol)
            U = U + dU
            its.append(int(st["iterations"]))
            rates.append(float(st["rho"]))
            R = fine.residual(U, U_n, t_new)
            res.append(np.linalg.norm(R))
        return U, {"newton_steps": len(its), "iterations": its, "rho": rates, "residuals": res}
