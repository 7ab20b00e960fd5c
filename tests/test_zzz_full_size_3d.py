"""Iteration parity at the 3D benchmark size: the 32^3 valve box (4 levels,
1.69 M unknowns, field-split blocks of one pressure vertex, omega = 0.7) in
the configuration bench.py's valve3d leg times, against the oracle's FGMRES
iteration count on the same system.  The oracle needs hours for this solve,
so the count is stored in tests/golden/full_size_valve32.json, written by
tests/golden/make_full_size_reference_3d.py from oracle/ alone.

- float16 row-scaled inverses of float64 factors, float32 cycle, float64
  Krylov (the storage the oracle emulates), additive smoother: converged to
  the float64 true residual 1e-8, iterations within +-1 of the oracle's; a
  repeat solve gives the same iterate bit for bit;
- the bench's configuration (the same storage of tensor-core TF32 factors):
  converged, iterations within +-1 of the oracle's.

Collected after the other test files: it builds the largest 3D hierarchy of
the suite.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh
from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL = 1e-8


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "full_size_valve32.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def valve(golden):
    p = I.make_config(2)
    assert (golden["workload"], golden["patch"], golden["omega"]) == (p.name, p.patch, p.omega)
    lev = mesh.build_levels(p)[-1]
    s = binding.FSISolver(p)
    f, c, nd = s.dof_map(p.n_levels - 1)
    np.testing.assert_array_equal(f, lev.dof_field)
    np.testing.assert_array_equal(nd, lev.dof_node)
    b = I.gather_natural(I.natural_vector(p, 1), lev.dof_field, lev.dof_comp, lev.dof_node)
    assert b.size == golden["n"]
    return s, torch.from_numpy(b).cuda()


def _solve(s, b):
    x, st = s.solve(b, rtol=RTOL)
    assert st["converged"] and st["rel_residual"] <= RTOL, st
    return x, st


def test_valve32_iterations_float64_factors(valve, golden):
    s, b = valve
    s.setup_smoothers(precision=binding.FSI_MIXED_HALF, factor=binding.FSI_FACTOR_FP64)
    x, st = _solve(s, b)
    want = golden["iterations_half_additive"]
    assert abs(st["iterations"] - want) <= 1, (st["iterations"], want)
    x2, st2 = _solve(s, b)
    assert st2["iterations"] == st["iterations"]
    np.testing.assert_array_equal(x.cpu().numpy(), x2.cpu().numpy())


def test_valve32_iterations_bench_configuration(valve, golden):
    s, b = valve
    s.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    _, st = _solve(s, b)
    want = golden["iterations_half_additive"]
    assert abs(st["iterations"] - want) <= 1, (st["iterations"], want)
