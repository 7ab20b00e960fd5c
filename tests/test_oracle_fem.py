"""Pins of the oracle's reference-element integrals (oracle/fem.py).

Independent checks: closed forms of the Q2 element (tests/golden), exact
polynomial integration with numpy.polynomial (a different method than the
oracle's Gauss rule), and invariants (partition of unity, zero derivative of
constants).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from oracle.fem import Reference

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "q2_reference_closed_forms.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if "=" not in line or "h" in line.split("=")[1]:
            continue
        k, v = (s.strip() for s in line.split("="))
        out[k] = float(Fraction(v))
    return out


# exact 1D polynomials (coefficients, increasing powers) of the Q2 / Q1 bases
L = [np.array([1.0, -3.0, 2.0]), np.array([0.0, 4.0, -4.0]), np.array([0.0, -1.0, 2.0])]
N = [np.array([1.0, -1.0]), np.array([0.0, 1.0])]


def _int01(c):
    ci = P.polyint(c)
    return P.polyval(1.0, ci) - P.polyval(0.0, ci)


def _q2_factors(dim, a, deriv=None):
    """1D polynomial factors of phi_a (local index a, x fastest), d/dx_deriv applied."""
    idx = [(a // 3 ** k) % 3 for k in range(dim)]
    return [P.polyder(L[idx[k]]) if k == deriv else L[idx[k]] for k in range(dim)]


def _q1_factors(dim, al):
    idx = [(al // 2 ** k) % 2 for k in range(dim)]
    return [N[idx[k]] for k in range(dim)]


def _int_prod(*factor_lists):
    dim = len(factor_lists[0])
    val = 1.0
    for k in range(dim):
        c = np.array([1.0])
        for fl in factor_lists:
            c = P.polymul(c, fl[k])
        val *= _int01(c)
    return val


def test_golden_1d_closed_forms_2d_tensor():
    g = _golden()
    ref = Reference(2)
    m1 = np.array([[g["M00"], g["M01"], g["M02"]],
                   [g["M01"], g["M11"], g["M01"]],
                   [g["M02"], g["M01"], g["M00"]]])
    k1 = np.array([[g["K00"], g["K01"], g["K02"]],
                   [g["K01"], g["K11"], g["K01"]],
                   [g["K02"], g["K01"], g["K00"]]])
    # local index a = a0 + 3 a1  ->  kron(y-factor, x-factor)
    np.testing.assert_allclose(ref.M, np.kron(m1, m1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(ref.G[0, 0], np.kron(m1, k1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(ref.G[1, 1], np.kron(k1, m1), rtol=0, atol=1e-14)
    w1 = np.array([g["int_L0"], g["int_L1"], g["int_L2"]])
    np.testing.assert_allclose(ref.lump, np.kron(w1, w1), rtol=0, atol=1e-15)
    # lumped weights (h^2/36){1, 4, 16}: vertex, edge, centre
    assert sorted(set(np.round(ref.lump * 36, 12))) == [1.0, 4.0, 16.0]


@pytest.mark.parametrize("dim", [2, 3])
def test_reference_tensors_exact_integration(dim):
    ref = Reference(dim)
    rng = np.random.default_rng(dim)
    n2, n1 = 3 ** dim, 2 ** dim
    for _ in range(30):
        a, b, c = rng.integers(0, n2, 3)
        k, l = rng.integers(0, dim, 2)
        al, be = rng.integers(0, n1, 2)
        assert ref.M[a, b] == pytest.approx(_int_prod(_q2_factors(dim, a), _q2_factors(dim, b)), abs=1e-14)
        assert ref.G[k, l, a, b] == pytest.approx(
            _int_prod(_q2_factors(dim, a, k), _q2_factors(dim, b, l)), abs=1e-13)
        assert ref.B[k, al, b] == pytest.approx(
            _int_prod(_q1_factors(dim, al), _q2_factors(dim, b, k)), abs=1e-14)
        assert ref.Mp[al, be] == pytest.approx(_int_prod(_q1_factors(dim, al), _q1_factors(dim, be)), abs=1e-15)
        assert ref.T[k, a, b, c] == pytest.approx(
            _int_prod(_q2_factors(dim, a), _q2_factors(dim, b, k), _q2_factors(dim, c)), abs=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_reference_invariants(dim):
    ref = Reference(dim)
    assert ref.M.sum() == pytest.approx(1.0, abs=1e-14)          # area of the unit cell
    assert ref.Mp.sum() == pytest.approx(1.0, abs=1e-14)
    for k in range(dim):
        for l in range(dim):
            # gradient of the constant (sum of all basis functions) vanishes
            np.testing.assert_allclose(ref.G[k, l].sum(1), 0.0, atol=1e-13)
        # sum over test functions of int phi_a d_k phi_b = int d_k phi_b
        np.testing.assert_allclose(ref.T[k].sum(axis=(0, 2)), ref.B[k].sum(0), atol=1e-14)
        # int d_k phi_b over the cell is (boundary flux): +-(1D Simpson weights)
        flux = ref.B[k].sum(0)
        for bidx in range(3 ** dim):
            digits = [(bidx // 3 ** m) % 3 for m in range(dim)]
            expect = {0: -1.0, 1: 0.0, 2: 1.0}[digits[k]]
            for m in range(dim):
                if m != k:
                    expect *= (1 / 6, 4 / 6, 1 / 6)[digits[m]]
            assert flux[bidx] == pytest.approx(expect, abs=1e-14)
