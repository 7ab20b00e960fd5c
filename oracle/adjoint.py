"""Adjoint solve and gradients (extension: the paper has no adjoint).

For J(x) = w^T x with A x = b:
    A^T lambda = w,   dJ/db = lambda,   dJ/dA_ij = -lambda_i x_j (on the
    sparsity pattern of A),   dJ/dmu_s = -lambda^T (dA/dmu_s) x.
The transposed system is solved by the same FGMRES with the transposed
V-cycle as right preconditioner (``Hierarchy.vcycle_transpose``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assemble import assemble
from .fem import Reference
from .fgmres import fgmres


def adjoint_solve(hier, w, rtol=1e-8, restart=30, maxit=1000):
    AT = hier.fine.T.tocsr()
    return fgmres(AT, w, hier.vcycle_transpose, rtol=rtol, restart=restart, maxit=maxit)


def pattern_gradient(A: sp.csr_matrix, lam: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dJ/dA on the CSR pattern of A (same order as A.data)."""
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    return -lam[rows] * x[A.indices]


def mu_s_gradient(prob, lev, lam: np.ndarray, x: np.ndarray) -> float:
    dA = assemble(prob, lev, Reference(prob.dim), only_mu_s_derivative=True)
    return float(-lam @ (dA @ x))
