"""Assembly of the linearised monolithic FSI operator in the J2 ordering.

Follows the weak form of Sec. 2.2 linearised about the reference
configuration (d = 0) with a frozen advection field w, backward Euler in
time, and the solid law read as mixed linear elasticity (the incompressible
Mooney-Rivlin law of Sec. 2.2 is replaced by sigma = 2 mu_s eps(d) - p I with
the penalty constraint -(q, div d) - (1/lambda_s)(q, p) = 0):

  S rows (momentum, solid-class nodes; d^s dofs)   and  F rows (momentum,
  fluid-class nodes; u^f dofs), test phi (Eq. momentum_supg without SUPG):
    solid elements:  rho_s/dt (u, phi) + (2 mu_s eps(d), eps(phi)) - (p^s, div phi)
    fluid elements:  rho_f/dt (u, phi) + rho_f ((w.grad) u, phi)
                     + (mu_f (grad u + grad u^T), grad phi) - (p^f, div phi)
                     - rho_f/dt ((d.grad) w, phi)         [mesh-velocity term]
  A rows (Eq. kinfld, fluid-class nodes; d^f dofs): (k (grad d + grad d^T), grad phi),
    k = 1 / V_el (Sec. 2.2).  k is a coefficient of the PDE, so V_el is the
    volume of the FINE element containing the point on every level (on the
    uniform grid k = n_fine^dim everywhere); taking the coarse element's
    volume would scale the coarse A rows by 2^-dim per level and break the
    coarse-grid correction.
  K rows (Eq. kinsld, solid-class nodes; u^s dofs): lumped solid mass
    M_L (u - d/dt), row-sum lumping (the diagonal K_u^s of Eq. matrix_J2)
  V rows (Eq. cntsld linearised; p^s dofs): -(q, div d) - (1/lambda_s)(q, p^s)
  W rows (Eq. cntfld; p^f dofs): -(q, div u)

Interface momentum test functions are summed over solid and fluid elements
into the S rows (remarks after Eq. jac_orig).  A fixed (Dirichlet) dof gets
an identity row and a zero column.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import Reference
from .mesh import Level, level_advection


def _sym_grad_block(ref: Reference, dim: int) -> np.ndarray:
    """E[(i, j), a, b] = int (grad phi_a e_i + ...) : 2 eps-form on the unit cell:
    delta_ij grad phi_a . grad phi_b + d_j phi_a d_i phi_b."""
    lap = sum(ref.G[k, k] for k in range(dim))
    E = np.zeros((dim, dim) + lap.shape)
    for i in range(dim):
        for j in range(dim):
            E[i, j] = ref.G[j, i] + (lap if i == j else 0.0)
    return E


class _COO:
    def __init__(self):
        self.r, self.c, self.v = [], [], []

    def add(self, rows, cols, vals):
        rows, cols, vals = np.broadcast_arrays(rows, cols, vals)
        keep = (rows >= 0) & (cols >= 0)
        self.r.append(rows[keep].astype(np.int64))
        self.c.append(cols[keep].astype(np.int64))
        self.v.append(vals[keep].astype(np.float64))

    def tocsr(self, n):
        r = np.concatenate(self.r)
        c = np.concatenate(self.c)
        v = np.concatenate(self.v)
        A = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
        A.sum_duplicates()
        A.sort_indices()
        return A


def _dirichlet(A: sp.csr_matrix, fixed: np.ndarray) -> sp.csr_matrix:
    keep = sp.diags((~fixed).astype(np.float64))
    A = (keep @ A @ keep).tocsr()
    A = A + sp.diags(fixed.astype(np.float64))
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble(prob, lev: Level, ref: Reference | None = None, *, only_mu_s_derivative=False,
             apply_bc=True) -> sp.csr_matrix:
    """Level operator A_l (rediscretisation on each level, Sec. 3.3).

    only_mu_s_derivative=True returns dA/dmu_s at fixed lambda_s (the solid
    elasticity term only), used by the adjoint gradient with respect to mu_s.
    """
    dim, h = lev.dim, lev.h
    ref = ref or Reference(dim)
    n2, n1 = ref.n2, ref.n1
    E = _sym_grad_block(ref, dim)                     # (dim, dim, n2, n2)
    eye = np.eye(dim)
    coo = _COO()
    s_el = np.flatnonzero(lev.material == 1)
    f_el = np.flatnonzero(lev.material == 0)
    hd, hd1, hd2 = h ** dim, h ** (dim - 1), h ** (dim - 2)

    # ---------------- solid elements ----------------
    if s_el.size:
        q2, q1 = lev.elem_q2[s_el], lev.elem_q1[s_el]
        d = lev.d_dof[q2]          # (ne, n2, dim)  S rows / d^s cols
        v = lev.v_dof[q2]          # (ne, n2, dim)  K rows / u^s cols
        ps = lev.ps_dof[q1]        # (ne, n1)
        # (2 mu eps, eps): rows (a,i) cols (b,j)
        mu = 1.0 if only_mu_s_derivative else prob.mu_s
        kel = mu * hd2 * E.transpose(2, 0, 3, 1)               # (a, i, b, j)
        rows = d[:, :, :, None, None]
        coo.add(rows, d[:, None, None, :, :], kel[None])
        if not only_mu_s_derivative:
            mel = (prob.rho_s / prob.dt) * hd * np.einsum("ab,ij->aibj", ref.M, eye)
            coo.add(rows, v[:, None, None, :, :], mel[None])
            # -(p, div phi_(a,i)) = -int psi_be d_i phi_a
            bel = -hd1 * ref.B.transpose(2, 0, 1)              # (a, i, be)
            coo.add(d[:, :, :, None], ps[:, None, None, :], bel[None])
            # V rows: -(q_al, div d) = -int psi_al d_j phi_b ; -(1/lambda) Mp
            vd = -hd1 * ref.B.transpose(1, 2, 0)               # (al, b, j)
            coo.add(ps[:, :, None, None], d[:, None, :, :], vd[None])
            coo.add(ps[:, :, None], ps[:, None, :], (-hd / prob.lambda_s) * ref.Mp[None])
            # K rows: lumped mass on the diagonal, M_L (u - d/dt)
            lump = hd * ref.lump[None, :, None] * np.ones((s_el.size, 1, dim))
            coo.add(v, v, lump)
            coo.add(v, d, -lump / prob.dt)

    # ---------------- fluid elements ----------------
    if f_el.size and not only_mu_s_derivative:
        q2, q1 = lev.elem_q2[f_el], lev.elem_q1[f_el]
        d = lev.d_dof[q2]
        v = lev.v_dof[q2]
        pf = lev.pf_dof[q1]
        solid_node = lev.q2_solid[q2]                           # (ne, n2)
        mom = np.where(solid_node[..., None], d, v)             # momentum rows
        w = level_advection(prob, lev)[:, q2].transpose(1, 0, 2)  # (ne, dim, n2) nodal w
        # velocity block: mass + advection + viscous
        adv = prob.rho_f * hd1 * np.einsum("ekc,kabc->eab", w, ref.T)      # (ne, a, b)
        scal = (prob.rho_f / prob.dt) * hd * ref.M[None] + adv
        vel = np.einsum("eab,ij->eaibj", scal, eye) + prob.mu_f * hd2 * E.transpose(2, 0, 3, 1)[None]
        coo.add(mom[:, :, :, None, None], v[:, None, None, :, :], vel)
        # pressure gradient
        bel = -hd1 * ref.B.transpose(2, 0, 1)
        coo.add(mom[:, :, :, None], pf[:, None, None, :], bel[None])
        # mesh-velocity coupling -(rho/dt)((d.grad) w, phi): rows (a,i) cols (b,j)
        # int phi_a phi_b d_j w_i = sum_c w_(i,c) int phi_a (d_j phi_c) phi_b = T[j, a, c, b]
        cpl = -(prob.rho_f / prob.dt) * hd1 * np.einsum("eic,jacb->eaibj", w, ref.T)
        coo.add(mom[:, :, :, None, None], d[:, None, None, :, :], cpl)
        # A rows at fluid-class nodes only: k (grad d + grad d^T, grad phi), k = 1/V_el
        a_rows = np.where(solid_node[..., None], -1, d)
        k_ale = float(prob.n_fine) ** dim          # 1 / V_el of the fine element
        kale = k_ale * hd2 * E.transpose(2, 0, 3, 1)
        coo.add(a_rows[:, :, :, None, None], d[:, None, None, :, :], kale[None])
        # W rows: -(q, div u)
        wd = -hd1 * ref.B.transpose(1, 2, 0)
        coo.add(pf[:, :, None, None], v[:, None, :, :], wd[None])

    A = coo.tocsr(lev.n_dofs)
    if apply_bc:
        if only_mu_s_derivative:
            keep = sp.diags((~lev.fixed).astype(np.float64))
            A = (keep @ A @ keep).tocsr()
            A.sort_indices()
        else:
            A = _dirichlet(A, lev.fixed)
    return A
