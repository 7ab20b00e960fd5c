"""Reference-element integrals for the Q2 (d, u) / Q1 (p) discretisation.

The paper discretises displacement and velocity with biquadratic Lagrange
elements (Sec. 2.2, "finite element families chosen are biquadratic").  The
pressure space here is continuous Q1 per material, duplicated on the
interface (the reading that matches the workload DOF counts; the paper's P1
discontinuous space likewise leaves p^s and p^f unconstrained at the
interface, Sec. 3.3).

Everything is computed on the unit reference cell [0,1]^dim with the 4-point
Gauss rule per direction, exact to degree 7: the trilinear advection integrand
phi_a (d_k phi_b) phi_c has degree 6 per direction, so a 3-point rule would
not be exact.  Physical integrals on a cube of side h follow by
the scalings documented on each function.  Local numbering: Q2 node
(a0, a1[, a2]) in {0,1,2}^dim has local index a0 + 3 a1 (+ 9 a2); Q1 vertex
(b0, b1[, b2]) in {0,1}^dim has b0 + 2 b1 (+ 4 b2).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# 4-point Gauss-Legendre rule on [-1, 1] (nodes +-sqrt(3/7 -+ 2/7 sqrt(6/5))),
# mapped to [0, 1]
_a = math.sqrt(3.0 / 7.0 - 2.0 / 7.0 * math.sqrt(6.0 / 5.0))
_b = math.sqrt(3.0 / 7.0 + 2.0 / 7.0 * math.sqrt(6.0 / 5.0))
_wa = (18.0 + math.sqrt(30.0)) / 36.0
_wb = (18.0 - math.sqrt(30.0)) / 36.0
GAUSS_X = 0.5 + 0.5 * np.array([-_b, -_a, _a, _b])
GAUSS_W = 0.5 * np.array([_wb, _wa, _wa, _wb])


def q2_1d(x: float) -> tuple[np.ndarray, np.ndarray]:
    """Quadratic Lagrange basis on nodes 0, 1/2, 1 and its derivative."""
    v = np.array([(2 * x - 1) * (x - 1), 4 * x * (1 - x), x * (2 * x - 1)])
    d = np.array([4 * x - 3, 4 - 8 * x, 4 * x - 1])
    return v, d


def q1_1d(x: float) -> tuple[np.ndarray, np.ndarray]:
    return np.array([1 - x, x]), np.array([-1.0, 1.0])


def _tensor(dim: int, one_d, npd: int, pt) -> tuple[np.ndarray, np.ndarray]:
    """Values (nb,) and gradients (dim, nb) of a tensor-product basis at pt."""
    vals_1d = [one_d(pt[k]) for k in range(dim)]
    nb = npd ** dim
    val = np.ones(nb)
    grad = np.ones((dim, nb))
    for idx in itertools.product(range(npd), repeat=dim):
        # itertools.product varies the LAST index fastest; the local
        # numbering has x (index 0) fastest, so reverse.
        a = idx[::-1]
        lin = sum(a[k] * npd ** k for k in range(dim))
        v = 1.0
        for k in range(dim):
            v *= vals_1d[k][0][a[k]]
        val[lin] = v
        for g in range(dim):
            dv = 1.0
            for k in range(dim):
                dv *= vals_1d[k][1][a[k]] if k == g else vals_1d[k][0][a[k]]
            grad[g, lin] = dv
    return val, grad


def quadrature(dim: int):
    """Yield (point, weight) of the tensor Gauss rule on [0,1]^dim."""
    for idx in itertools.product(range(GAUSS_X.size), repeat=dim):
        pt = [GAUSS_X[i] for i in idx]
        w = 1.0
        for i in idx:
            w *= GAUSS_W[i]
        yield pt, w


class Reference:
    """Reference integrals on [0,1]^dim.

    M[a,b]      = int phi_a phi_b                 (scale h^dim)
    G[k,l,a,b]  = int d_k phi_a d_l phi_b         (scale h^(dim-2))
    B[k,al,b]   = int psi_al d_k phi_b            (scale h^(dim-1))
    Mp[al,be]   = int psi_al psi_be               (scale h^dim)
    T[k,a,b,c]  = int phi_a (d_k phi_b) phi_c     (scale h^(dim-1))
    lump[a]     = int phi_a                       (scale h^dim)
    """

    def __init__(self, dim: int):
        self.dim = dim
        n2, n1 = 3 ** dim, 2 ** dim
        self.n2, self.n1 = n2, n1
        M = np.zeros((n2, n2))
        G = np.zeros((dim, dim, n2, n2))
        B = np.zeros((dim, n1, n2))
        Mp = np.zeros((n1, n1))
        T = np.zeros((dim, n2, n2, n2))
        for pt, w in quadrature(dim):
            phi, dphi = _tensor(dim, q2_1d, 3, pt)
            psi, _ = _tensor(dim, q1_1d, 2, pt)
            M += w * np.outer(phi, phi)
            for k in range(dim):
                for l in range(dim):
                    G[k, l] += w * np.outer(dphi[k], dphi[l])
                B[k] += w * np.outer(psi, dphi[k])
                T[k] += w * np.einsum("a,b,c->abc", phi, dphi[k], phi)
            Mp += w * np.outer(psi, psi)
        self.M, self.G, self.B, self.Mp, self.T = M, G, B, Mp, T
        self.lump = M.sum(1)
