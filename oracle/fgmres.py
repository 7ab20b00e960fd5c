"""Restarted flexible GMRES with right preconditioning (outer Krylov solver).

The paper's outer solver is GMRES preconditioned by GMG (Sec. 3.2).  The
flexible variant is used so that the preconditioner may change between
iterations (mixed precision): the preconditioned vectors z_j are kept and the
update is x += Z y.  Arnoldi uses classical Gram-Schmidt applied twice
(CGS2); the least-squares problem is updated with Givens rotations.

Stopping rule: the Arnoldi estimate |g_{j+1}| <= rtol ||b|| ends a cycle, and
the solve is converged when the float64 TRUE residual ||b - A x|| <= rtol
||b||; otherwise the method restarts from the true residual.  A happy
breakdown (|h_{j+1,j}| <= 1e-14 ||A z_j||) also ends a cycle.

Statistics follow Sec. 4: N (iterations) and the average convergence rate
rho = (r_N / r_0)^(1/N).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as la


def fgmres(A, b, precond, x0=None, rtol=1e-8, restart=30, maxit=1000, breakdown=1e-14):
    n = b.size
    bnorm = float(np.linalg.norm(b))
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    stats = {"iterations": 0, "cycles": 0, "converged": False, "estimates": []}
    if bnorm == 0.0:
        x[:] = 0.0
        stats.update(converged=True, rel_residual=0.0, r0=0.0, rN=0.0, rho=0.0)
        return x, stats
    r = b - A @ x
    beta = float(np.linalg.norm(r))
    r0 = beta
    its = 0
    while beta > rtol * bnorm and its < maxit:
        m = restart
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            Z[:, j] = precond(V[:, j])
            w = A @ Z[:, j]
            wnorm0 = float(np.linalg.norm(w))
            Vj = V[:, : j + 1]
            h = Vj.T @ w
            w = w - Vj @ h
            h2 = Vj.T @ w
            w = w - Vj @ h2
            h = h + h2
            hn = float(np.linalg.norm(w))
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            est = abs(g[j + 1])
            stats["estimates"].append(est / bnorm)
            if est <= rtol * bnorm or hn <= breakdown * wnorm0 or its >= maxit:
                break
            V[:, j + 1] = w / hn
        y = la.solve_triangular(H[:k, :k], g[:k])
        x = x + Z[:, :k] @ y
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        stats["cycles"] += 1
    N = its
    stats.update(iterations=N, converged=beta <= rtol * bnorm, rel_residual=beta / bnorm,
                 r0=r0, rN=beta, rho=(beta / r0) ** (1.0 / N) if N and r0 > 0 else 0.0)
    return x, stats


def solve(hier, b, rtol=1e-8, restart=30, maxit=1000, x0=None):
    """FGMRES(restart) on the fine operator with one V-cycle per iteration."""
    return fgmres(hier.fine, b, hier.vcycle, x0=x0, rtol=rtol, restart=restart, maxit=maxit)
