"""Host checks of the nonlinear set-up (no GPU): the operator patterns built
with fsi_hier_opts.nonlinear = 1 hold every nonzero of the oracle's exact
Newton Jacobian of the nonlinear residual (Sec. 2.2) at a deformed state, on
every level, and differ from the linear patterns only by the d columns of
the W rows (the moving fluid element makes div_x u depend on d)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import nonlinear as NL
from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I


def _pattern(s, level):
    ptr, col = s.pattern(level)
    n = len(ptr) - 1
    return sp.csr_matrix((np.ones(len(col)), col, ptr), shape=(n, n))


@pytest.mark.parametrize("maker", [lambda: I.make_config(0), lambda: I.make_channel_2d(24, 3, 2, 77, bulge=True)])
def test_nonlinear_pattern_holds_the_jacobian(maker):
    p = maker()
    pr = NL.Problem(p)
    rng = np.random.default_rng(5)
    lev = pr.levels[-1]
    U = 1e-2 * rng.standard_normal(lev.n_dofs)
    Un = 1e-2 * rng.standard_normal(lev.n_dofs)
    U[lev.fixed] = 0.0
    Un[lev.fixed] = 0.0
    jac = pr.jacobians(U, Un, 0.3)
    snl = binding.FSISolver(p, host_only=True, nonlinear=True)
    slin = binding.FSISolver(p, host_only=True)
    for l, Jl in enumerate(jac):
        Pn = _pattern(snl, l)
        Pl = _pattern(slin, l)
        Jl = Jl.tocoo()
        nz = Jl.data != 0.0
        inside = np.asarray(Pn[Jl.row[nz], Jl.col[nz]]).ravel()
        assert np.all(inside == 1.0), (l, int((inside != 1.0).sum()))
        # the W rows' d columns are the only additions
        extra = (Pn - Pl).tocoo()
        assert extra.data.min() > 0 if extra.nnz else True
        levl = pr.levels[l]
        f, c = levl.dof_field, levl.dof_comp
        assert np.all((f[extra.row] == 2) & (c[extra.row] == 1)), l      # p^f rows (W)
        assert np.all(f[extra.col] == 0), l                             # d columns
        # and the Jacobian uses them: W rows couple to d somewhere
        if l == len(jac) - 1:
            w_rows = (f[Jl.row] == 2) & (c[Jl.row] == 1) & (f[Jl.col] == 0) & nz
            assert w_rows.any()
