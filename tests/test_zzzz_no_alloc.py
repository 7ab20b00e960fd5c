"""fsi_apply_smoother_noalloc: the smoother apply for callers that cannot
allocate GPU memory at call time (allocator-restricted or real-time code).

It must give the same y = P2^{-1} r as fsi_apply_smoother, which allocates its
working vectors per call, and keep doing so on consecutive calls that reuse
the library's static device array: on additive levels and on a level smoothed
by the multiplicative sweep, where a transposed call before the transposed
operators exist is refused (it would have to build them, which allocates).
A level above FSI_NOALLOC_MAX_DOFS is refused with FSI_ERR_ARG.  Collected
last (file name) so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# the tolerances of the smoother parity tests: float64 1e-9, float16 storage 2e-5
CASES = [(binding.FSI_FP64, 1e-9), (binding.FSI_MIXED, 1e-6), (binding.FSI_MIXED_HALF, 2e-5)]
NOALLOC_MAX_DOFS = 2097152          # FSI_NOALLOC_MAX_DOFS of include/fsi.h


def _compare(s, level, rng, tr, prec, tol, tag):
    n = s.sizes(level)["n"]
    r = torch.from_numpy(rng.standard_normal(n)).cuda()
    y_ref = s.apply_smoother(level, r, transpose=tr)
    y = torch.full_like(r, float("nan"))
    s.apply_smoother_noalloc(level, r, y, transpose=tr)
    a, b = y.cpu().numpy(), y_ref.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), (prec, level, tr, tag)


@pytest.mark.parametrize("mult_levels", [0, 1])
@pytest.mark.parametrize("prec,tol", CASES)
def test_noalloc_smoother_matches_allocating_entry_point(prec, tol, mult_levels):
    p = I.make_channel_2d(48, 4, 3, 4242, bulge=True)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=prec, mult_levels=mult_levels)
    rng = np.random.default_rng(31)
    fine = p.n_levels - 1
    if mult_levels:
        # the sweep's transposed operators do not exist yet: refused, not built
        n = s.sizes(fine)["n"]
        r = torch.from_numpy(rng.standard_normal(n)).cuda()
        y = torch.zeros_like(r)
        with pytest.raises(binding.FSIError) as e:
            s.apply_smoother_noalloc(fine, r, y, transpose=True)
        assert e.value.status == binding.FSI_ERR_STATE
    for level in range(1, p.n_levels):
        for call in range(2):                        # two calls in a row reuse the static array
            for tr in (False, True):
                # on the sweep level the allocating transposed call builds the
                # transposed operators before the no-alloc call runs
                _compare(s, level, rng, tr, prec, tol, call)


def test_noalloc_rejects_level_above_limit():
    # 2D 352^2 (6 levels from 11^2): 4 * 705^2 + 353^2 = 2 112 709 fine unknowns
    p = I.make_channel_2d(352, 6, 4, 77)
    s = binding.FSISolver(p)
    n = s.sizes(p.n_levels - 1)["n"]
    assert n > NOALLOC_MAX_DOFS
    s.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(r)
    with pytest.raises(binding.FSIError) as e:
        s.apply_smoother_noalloc(p.n_levels - 1, r, y)
    assert e.value.status == binding.FSI_ERR_ARG
    # a level within the limit still works on the same context
    _compare(s, p.n_levels - 2, np.random.default_rng(5), False, binding.FSI_MIXED_HALF, 2e-5, "coarser")
