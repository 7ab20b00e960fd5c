"""Pins of the oracle's float16 row-scaled storage of the block inverses.

The mixed-half smoother stores every block inverse A_jj^{-1} (Sec. 3.2, the
blocks of AS1/AS2 solved by LU) as float16 rows m16 times a float32 row
scale s, with s the row's max-abs entry, and applies it in float32.  The
oracle's emulation of that storage (``FSASM(half=True)``) is the reference
the GPU's half smoother is compared against, so it is pinned here against
quantities computed without it:

* reconstruction: for every block, s * m16 equals the float64 inverse of the
  block (computed here by ``numpy.linalg.inv`` of the block sliced from the
  level matrix by scipy, not through the oracle's extraction or its LU) to the
  float16 rounding bound, entry by entry: relative 2^-11 for normal float16
  values, absolute 2^-25 s below the float16 normal range; every row of m16
  has max-abs exactly 1;
* apply and transposed apply: the float16 smoother stays, entry by entry,
  within a bound derived from those roundings and float32 accumulation
  (gamma_n = n u / (1 - n u), u = 2^-24) of the float64 additive smoother
  sum_j R_j^T W_j A_jj^{-1} R_j r + D^{-1} r (transposed: A_jj^{-T} W_j);
* the bound has teeth: the same check fails for an emulation with the row
  scale dropped, or applied to the columns instead of the rows, planted here
  in a subclass of the oracle.
"""
import numpy as np
import pytest

from oracle import fsasm, mesh
from oracle.assemble import assemble
from oracle.transfer import G_US
from paper_1909_13201_gb300 import inputs as I

U32 = 2.0 ** -24
H16 = 2.0 ** -11          # float16 unit roundoff (11 significant bits)
SUB16 = 2.0 ** -25        # half the spacing of float16 subnormals (2^-24)


def _gamma(n):
    return n * U32 / (1.0 - n * U32)


CASES = {
    "c0": lambda: I.make_config(0),
    "bulge48": lambda: I.make_channel_2d(48, 4, 3, 4242, bulge=True),
}


@pytest.fixture(scope="module", params=list(CASES))
def fine(request):
    p = CASES[request.param]()
    lev = mesh.build_levels(p)[-1]
    A = assemble(p, lev).tocsr()
    S = fsasm.FSASM(A, lev, p.patch, half=True)
    # float64 block inverses, independent of the oracle's extraction and LU
    invs = [np.linalg.inv(A[idx][:, idx].toarray()) for idx in S.blocks]
    jac = np.flatnonzero((lev.group == G_US) | lev.fixed)
    return request.param, A, lev, S, invs, jac


def test_blocks_are_the_vanka_sets(fine):
    """The emulation stores one inverse per block of the field split, in the
    order of the block index sets."""
    name, A, lev, S, invs, jac = fine
    ref = fsasm.block_index_sets(lev, CASES[name]().patch)
    assert len(S.blocks) == len(ref) == len(S.lu)
    for a, b in zip(S.blocks, ref):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(S.jacobi, jac)


def test_row_scaled_float16_reconstructs_inverse(fine):
    name, A, lev, S, invs, jac = fine
    for j, ((m16, scale), inv) in enumerate(zip(S.lu, invs)):
        assert m16.dtype == np.float16 and scale.dtype == np.float32
        s = np.abs(inv).max(1)
        # the row scale is the float32 rounding of the row's max-abs entry
        np.testing.assert_allclose(scale, s, rtol=U32 * (1 + 1e-6) + 1e-12, atol=0)
        m = m16.astype(np.float64)
        np.testing.assert_array_equal(np.abs(m).max(1), 1.0)
        err = np.abs(scale.astype(np.float64)[:, None] * m - inv)
        # float16 rounding of inv/s, the float32 scale, the float64 inverse's own error
        tol = (H16 + 2 * U32) * np.abs(inv) + SUB16 * (1 + U32) * s[:, None] \
            + 1e-11 * s[:, None]
        assert np.all(err <= tol), (name, j, float((err / tol).max()))


def _fp64_apply(invs, blocks, weight, jac, dinv, r, transpose):
    y = np.zeros_like(r)
    for idx, inv in zip(blocks, invs):
        y[idx] += inv.T @ (weight[idx] * r[idx]) if transpose else weight[idx] * (inv @ r[idx])
    y[jac] += r[jac] * dinv
    return y


def _bound(invs, blocks, weight, mult, jac, dinv, r, transpose):
    """Entrywise bound on |apply_half - apply_fp64| from the float16 rounding
    of every stored entry (relative H16, subnormal absolute SUB16 s) and
    float32 products and sums (gamma of the block size, of the overlap)."""
    n = r.size
    bnd = np.zeros(n)
    mag = np.zeros(n)
    ar = np.abs(r)
    for idx, inv in zip(blocks, invs):
        s = np.abs(inv).max(1)
        ai = np.abs(inv)
        w = weight[idx]
        g = H16 + _gamma(idx.size + 6)
        if transpose:
            v = w * ar[idx]
            bnd[idx] += g * (ai.T @ v) + SUB16 * np.dot(s, v)
            mag[idx] += ai.T @ v
        else:
            bnd[idx] += w * (g * (ai @ ar[idx]) + SUB16 * s * ar[idx].sum())
            mag[idx] += w * (ai @ ar[idx])
    bnd += _gamma(int(mult.max()) + 1) * mag
    bnd[jac] += 4 * U32 * np.abs(r[jac] * dinv)
    return 1.01 * bnd


def _check(S, invs, A, jac, r, transpose):
    dinv = 1.0 / A.diagonal()[jac]
    y64 = _fp64_apply(invs, S.blocks, S.weight, jac, dinv, r, transpose)
    yh = (S.apply_transpose(r) if transpose else S.apply(r)).astype(np.float64)
    bnd = _bound(invs, S.blocks, S.weight, S.multiplicity, jac, dinv, r, transpose)
    return np.abs(yh - y64), bnd


@pytest.mark.parametrize("transpose", [False, True])
def test_half_apply_within_rounding_bound_of_fp64(fine, transpose):
    name, A, lev, S, invs, jac = fine
    rng = np.random.default_rng(31)
    for _ in range(2):
        # float32-representable input: the emulation casts r to float32 first
        r = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
        err, bnd = _check(S, invs, A, jac, r, transpose)
        assert np.all(err <= bnd), (name, transpose, float((err / np.maximum(bnd, 1e-300)).max()))
        # the bound is not vacuous: it sits at float16 level of the result
        y = _fp64_apply(invs, S.blocks, S.weight, jac, 1.0 / A.diagonal()[jac], r, transpose)
        assert np.linalg.norm(bnd) < 5e-3 * np.linalg.norm(y)


class _DroppedScale(fsasm.FSASM):
    def apply(self, r):
        r = r.astype(np.float32)
        y = np.zeros(self.n, np.float32)
        w = self.weight.astype(np.float32)
        for idx, (m16, scale) in zip(self.blocks, self.lu):
            y[idx] += w[idx] * (m16.astype(np.float32) @ r[idx])
        y[self.jacobi] += r[self.jacobi] * self.inv_diag.astype(np.float32)
        return y

    def apply_transpose(self, r):
        r = r.astype(np.float32)
        y = np.zeros(self.n, np.float32)
        w = self.weight.astype(np.float32)
        for idx, (m16, scale) in zip(self.blocks, self.lu):
            y[idx] += m16.astype(np.float32).T @ (w[idx] * r[idx])
        y[self.jacobi] += r[self.jacobi] * self.inv_diag.astype(np.float32)
        return y


class _ColumnScale(fsasm.FSASM):
    def apply(self, r):
        r = r.astype(np.float32)
        y = np.zeros(self.n, np.float32)
        w = self.weight.astype(np.float32)
        for idx, (m16, scale) in zip(self.blocks, self.lu):
            y[idx] += w[idx] * (m16.astype(np.float32) @ (scale * r[idx]))
        y[self.jacobi] += r[self.jacobi] * self.inv_diag.astype(np.float32)
        return y

    def apply_transpose(self, r):
        r = r.astype(np.float32)
        y = np.zeros(self.n, np.float32)
        w = self.weight.astype(np.float32)
        for idx, (m16, scale) in zip(self.blocks, self.lu):
            y[idx] += scale * (m16.astype(np.float32).T @ (w[idx] * r[idx]))
        y[self.jacobi] += r[self.jacobi] * self.inv_diag.astype(np.float32)
        return y


@pytest.mark.parametrize("mutant", [_DroppedScale, _ColumnScale])
@pytest.mark.parametrize("transpose", [False, True])
def test_bound_rejects_planted_scale_mistakes(fine, mutant, transpose):
    name, A, lev, S, invs, jac = fine
    M = mutant.__new__(mutant)
    M.__dict__.update(S.__dict__)
    r = np.random.default_rng(32).standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    err, bnd = _check(M, invs, A, jac, r, transpose)
    assert np.any(err > bnd), (name, mutant.__name__, transpose)
