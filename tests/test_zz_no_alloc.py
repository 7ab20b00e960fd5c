"""fsi_apply_smoother_noalloc: the smoother apply for callers that cannot
allocate GPU memory at call time (allocator-restricted or real-time code).

It must give the same y = P2^{-1} r as fsi_apply_smoother, which allocates its
working vectors per call, and keep doing so on consecutive calls that reuse
the library's static device array.  Collected after the parity tests so that a
run stopping at the first failure has already run them (only the full-size
tests follow).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# the tolerances of the smoother parity tests: float64 1e-9, float16 storage 2e-5
CASES = [(binding.FSI_FP64, 1e-9), (binding.FSI_MIXED, 1e-6), (binding.FSI_MIXED_HALF, 2e-5)]


@pytest.mark.parametrize("prec,tol", CASES)
def test_noalloc_smoother_matches_allocating_entry_point(prec, tol):
    p = I.make_channel_2d(48, 4, 3, 4242, bulge=True)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=prec)
    rng = np.random.default_rng(31)
    for level in range(1, p.n_levels):
        n = s.sizes(level)["n"]
        for call in range(2):                        # two calls in a row reuse the static array
            for tr in (False, True):
                r = torch.from_numpy(rng.standard_normal(n)).cuda()
                y_ref = s.apply_smoother(level, r, transpose=tr)
                y = torch.full_like(r, float("nan"))
                s.apply_smoother_noalloc(level, r, y, transpose=tr)
                a, b = y.cpu().numpy(), y_ref.cpu().numpy()
                assert np.all(np.isfinite(a))
                assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), (prec, level, call, tr)
