"""Geometric multigrid V-cycle preconditioner (Sec. 3.2-3.3).

On every level l >= 1 the smoother is damped Richardson preconditioned by the
field-split additive Schwarz method (monolithic=True: the paper's AS
comparison method, blocks over all fields; on the mult_levels finest levels
the locally multiplicative sweep of fsasm.FSASM.sweep); level 0 is solved directly (Sec. 3.2,
"at the coarse level (l=0) a direct solver is employed").  Level operators
are rediscretised on each level; transfers are P2 and R2 of Sec. 3.3.

Mixed mode (extension, not in the paper): level operators, transfers,
Schwarz factors and V-cycle vectors are rounded to float32 and the cycle's
arithmetic runs in float32; the coarse direct solve stays float64.
mixed="half" additionally stores the Schwarz block inverses in float16 with
a float32 scale per row (see fsasm.FSASM).

The transposed cycle (adjoint extension) applies the transposed operators in
reverse order: transposed post-smoothing first, restriction by P^T,
transposed coarse solve, prolongation by R^T, transposed pre-smoothing.

cascade=True builds the swapped cascade of the paper's future work (Sec. 5,
the GMG and FS boxes of its solver diagram interchanged): the Krylov solver
is preconditioned by the field split FS, whose two diagonal blocks -- the
displacement system [d^s, d^f, p^s] (rows S, A, V) and the velocity system
[u^s, u^f, p^f] (rows K, F, W) of J2 -- are each preconditioned by a GMG
V-cycle with the same Schwarz (AS) smoothing.  Every operator the cycle
uses (level matrices, restrictions, prolongations, the coarse matrix) is
restricted to same-system entries, so one V-cycle over the whole vector is
exactly blockdiag(GMG_d, GMG_u); the outer Krylov operator stays the full
fine J2 (``fine``).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la

from .assemble import assemble
from .fem import Reference
from .fsasm import FSASM
from .mesh import build_levels
from .transfer import G_DF, G_DS, G_PS, prolongation, restriction


def system_of(lev) -> np.ndarray:
    """0 for the displacement system (d^s, d^f, p^s), 1 for the velocity
    system (u^s, u^f, p^f), per dof of the level (J2 groups, Sec. 3.2)."""
    return (~np.isin(lev.group, (G_DS, G_DF, G_PS))).astype(np.int64)


def split_systems(M, sys_rows: np.ndarray, sys_cols: np.ndarray):
    """M with the entries coupling the two systems removed."""
    C = M.tocoo()
    keep = sys_rows[C.row] == sys_cols[C.col]
    return type(M.tocsr())((C.data[keep], (C.row[keep], C.col[keep])), shape=M.shape).tocsr()


class Hierarchy:
    def __init__(self, prob, *, mixed: bool = False, omega: float | None = None, nu_pre: int = 1,
                 nu_post: int = 1, patch: int | None = None, classical_restriction: bool = False,
                 weighted: bool = True, monolithic: bool = False, mult_levels: int = 0,
                 cascade: bool = False, operators=None):
        self.prob = prob
        self.cascade = cascade
        self.mixed = bool(mixed)
        half = mixed == "half"
        omega = getattr(prob, "omega", 1.0) if omega is None else omega
        self.omega, self.nu_pre, self.nu_post = omega, nu_pre, nu_post
        self.wdtype = np.float32 if mixed else np.float64
        self.levels = build_levels(prob)
        ref = Reference(prob.dim)
        # level operators: rediscretised linear forms, or given matrices (the
        # Newton Jacobians of the nonlinear loop, oracle.nonlinear)
        self.A = list(operators) if operators is not None else [assemble(prob, lev, ref) for lev in self.levels]
        nl = len(self.levels)
        self.P = [None] + [prolongation(self.levels[l], self.levels[l - 1]) for l in range(1, nl)]
        self.R = [None] + [restriction(self.P[l], self.levels[l], self.levels[l - 1],
                                       classical=classical_restriction) for l in range(1, nl)]
        b = prob.patch if patch is None else patch
        self.smoothers = [None] + [FSASM(self.A[l], self.levels[l], b, dtype=self.wdtype,
                                         weighted=weighted, half=half, monolithic=monolithic,
                                         multiplicative=l >= nl - mult_levels)
                                   for l in range(1, nl)]
        # operators of the cycle: the full ones, or (cascade) their two
        # same-system diagonal blocks
        Ac, Pc, Rc = self.A, self.P, self.R
        if cascade:
            sy = [system_of(lev) for lev in self.levels]
            Ac = [split_systems(A, sy[l], sy[l]) for l, A in enumerate(self.A)]
            Pc = [None] + [split_systems(self.P[l], sy[l], sy[l - 1]) for l in range(1, nl)]
            Rc = [None] + [split_systems(self.R[l], sy[l - 1], sy[l]) for l in range(1, nl)]
        self.A_cycle = Ac
        self.coarse_lu = la.lu_factor(Ac[0].toarray())
        wd = self.wdtype
        self.Aw = [A.astype(wd) for A in Ac]
        self.Pw = [None] + [P.astype(wd) for P in Pc[1:]]
        self.Rw = [None] + [R.astype(wd) for R in Rc[1:]]
        self.AwT = [A.T.tocsr() for A in self.Aw]

    @property
    def fine(self):
        return self.A[-1]

    def _smooth(self, l, x, b, transpose=False):
        A = self.AwT[l] if transpose else self.Aw[l]
        S = self.smoothers[l]
        r = b - A @ x
        y = S.apply_transpose(r) if transpose else S.apply(r)
        return (x + self.wdtype(self.omega) * y).astype(self.wdtype)

    def vcycle_level(self, l: int, b: np.ndarray) -> np.ndarray:
        wd = self.wdtype
        b = b.astype(wd)
        if l == 0:
            return la.lu_solve(self.coarse_lu, b.astype(np.float64)).astype(wd)
        x = np.zeros_like(b)
        for _ in range(self.nu_pre):
            x = self._smooth(l, x, b)
        r = (b - self.Aw[l] @ x).astype(wd)
        xc = self.vcycle_level(l - 1, (self.Rw[l] @ r).astype(wd))
        x = (x + self.Pw[l] @ xc).astype(wd)
        for _ in range(self.nu_post):
            x = self._smooth(l, x, b)
        return x

    def vcycle_transpose_level(self, l: int, b: np.ndarray) -> np.ndarray:
        wd = self.wdtype
        b = b.astype(wd)
        if l == 0:
            return la.lu_solve(self.coarse_lu, b.astype(np.float64), trans=1).astype(wd)
        x = np.zeros_like(b)
        for _ in range(self.nu_post):
            x = self._smooth(l, x, b, transpose=True)
        r = (b - self.AwT[l] @ x).astype(wd)
        xc = self.vcycle_transpose_level(l - 1, (self.Pw[l].T @ r).astype(wd))
        x = (x + self.Rw[l].T @ xc).astype(wd)
        for _ in range(self.nu_pre):
            x = self._smooth(l, x, b, transpose=True)
        return x

    def vcycle(self, b: np.ndarray) -> np.ndarray:
        """One V-cycle from a zero guess on the fine level: M^{-1} b (float64 out)."""
        return self.vcycle_level(len(self.levels) - 1, b).astype(np.float64)

    def vcycle_transpose(self, b: np.ndarray) -> np.ndarray:
        return self.vcycle_transpose_level(len(self.levels) - 1, b).astype(np.float64)
