"""Parity of the nonlinear path (Sec. 2.2) at the benchmark's full size: the
256x256 channel (7 levels, 1.12 M unknowns) with the nonlinear patterns, as
bench.py's nonlinear leg runs it, on outputs the oracle computes element by
element: at a seeded deformed state,

- the residual R(U; U_n) of the fine level on sampled rows (every J2 field
  group), against the oracle's element residuals of the elements touching
  those rows, assembled in extended precision: within 1e-12 of the row's
  largest element contribution plus 10x the oracle's own float64 error;
- the exact Jacobian of the fine level on the same rows: every entry against
  the oracle's complex-step element Jacobians of those elements, 1e-10 of the
  row scale (the whole row, so a missing or extra entry fails too).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh
from oracle import nonlinear as NL
from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORCE = 20.0
T_NEW = 0.25
PER_GROUP = 64


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def full_nl():
    p = I.make_config(1)
    lev = mesh.build_levels(p)[-1]
    P = NL.Params(p, force=FORCE)
    nl = NL.LevelNL(p, lev, P)
    s = binding.FSISolver(p, nonlinear=True)
    s.nl_setup(force=FORCE)
    rng = np.random.default_rng(256)
    f = lev.dof_field

    def state():
        U = np.zeros(lev.n_dofs)
        U[f == 0] = 0.03 * lev.h * rng.standard_normal(int((f == 0).sum()))
        U[f == 1] = rng.standard_normal(int((f == 1).sum()))
        U[f == 2] = rng.standard_normal(int((f == 2).sum()))
        U[lev.fixed] = 0.0
        return U

    U, Un = state(), state()
    free = np.flatnonzero(~lev.fixed)
    rows = []
    for g in range(6):
        cand = free[lev.group[free] == g]
        rows.append(np.sort(rng.choice(cand, min(PER_GROUP, cand.size), replace=False)))
    rows = np.concatenate(rows)
    # the elements that assemble into the sampled rows, and the oracle's maps for them
    m = nl.maps
    els = np.unique(np.nonzero(np.isin(m.rows, rows))[0])
    sub = NL.ElementMaps.__new__(NL.ElementMaps)
    sub.solid, sub.cols, sub.rows = m.solid[els], m.cols[els], m.rows[els]
    tab = NL.shape_tables()
    fn = NL.force_at_quadrature(p, lev, P.force_factor(T_NEW), tab)[els]
    fo = NL.force_at_quadrature(p, lev, P.force_factor(T_NEW - p.dt), tab)[els]
    return p, lev, P, s, U, Un, rows, sub, tab, fn, fo


def _assemble_rows(sub, Rl, rows):
    """Row values of the sampled rows from element contributions Rl (ne, 40)."""
    out = {int(r): [] for r in rows}
    for e in range(sub.rows.shape[0]):
        for r in range(NL.NLOC):
            g = int(sub.rows[e, r])
            if g in out:
                out[g].append(Rl[e, r])
    return out


def test_full_size_residual_sampled_rows(full_nl):
    p, lev, P, s, U, Un, rows, sub, tab, fn, fo = full_nl
    got = s.nl_residual(_cuda(U), _cuda(Un), T_NEW).cpu().numpy()
    Ul, Unl = NL.gather(U, sub.cols), NL.gather(Un, sub.cols)
    R64 = NL.element_residual(lev, P, Ul, Unl, None, fn, fo, sub, tab)
    Rld = NL.element_residual(lev, P, Ul.astype(np.longdouble), Unl.astype(np.longdouble), None,
                              fn.astype(np.longdouble), fo.astype(np.longdouble), sub, tab)
    c64, cld = _assemble_rows(sub, R64, rows), _assemble_rows(sub, Rld, rows)
    for r in rows:
        r = int(r)
        ref = np.sum(np.array(cld[r], dtype=np.longdouble))
        own = abs(float(np.sum(np.array(c64[r])) - ref))
        scale = max(abs(float(v)) for v in c64[r])
        err = abs(float(got[r] - ref))
        assert err <= 1e-12 * scale + 10.0 * own, (r, lev.group[r], err, scale, own)


def test_full_size_jacobian_sampled_rows(full_nl):
    p, lev, P, s, U, Un, rows, sub, tab, fn, fo = full_nl
    s.nl_jacobian(_cuda(U), _cuda(Un), T_NEW)
    ptr, col, val = s.matrix(p.n_levels - 1)
    Ul, Unl = NL.gather(U, sub.cols).astype(np.complex128), NL.gather(Un, sub.cols)
    h = 1e-30
    ne = Ul.shape[0]
    Jl = np.zeros((ne, NL.NLOC, NL.NLOC))
    for t in range(NL.NLOC):
        Up = Ul.copy()
        Up[:, t] += 1j * h
        Jl[:, :, t] = NL.element_residual(lev, P, Up, Unl, None, fn, fo, sub, tab).imag / h
    want = {int(r): {} for r in rows}
    for e in range(ne):
        for r in range(NL.NLOC):
            g = int(sub.rows[e, r])
            if g not in want:
                continue
            for t in range(NL.NLOC):
                c = int(sub.cols[e, t])
                if c < 0 or lev.fixed[c]:
                    continue
                want[g][c] = want[g].get(c, 0.0) + Jl[e, r, t]
    for r in rows:
        r = int(r)
        ref = want[r]
        scale = max(abs(v) for v in ref.values())
        gpu = {int(c): v for c, v in zip(col[ptr[r]:ptr[r + 1]], val[ptr[r]:ptr[r + 1]])}
        for c in set(ref) | set(gpu):
            d = abs(gpu.get(c, 0.0) - ref.get(c, 0.0))
            assert d <= 1e-10 * scale, (r, c, lev.group[r], d, scale)
