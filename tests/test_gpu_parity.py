"""GPU parity of every piece of the path against the FP64 oracle, through
the C ABI: assembled operators, SpMV, the FS-ASM smoother (and its
transpose), the V-cycle, full FGMRES solves in FP64 and mixed precision,
the adjoint and its gradients, and the error statuses.

Tolerances, from the arithmetic: operator values and SpMV to 1e-13 of
the row scale (same quadrature, different summation order); smoother and
V-cycle in FP64 to 1e-9 relative (block inverses by Gauss-Jordan versus the
oracle's pivoted LU, condition numbers up to ~1e5); solutions to 1e-9
relative in FP64 and 1e-8 in mixed precision against x* = A^{-1} b (sparse
LU with refinement) when solved to a 1e-10 true residual (the attainable
residual floor of these row-scaled systems is ~1e-11); FGMRES iteration
counts within +-1 of the oracle's.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj
from oracle import fgmres as ofg
from oracle import gmg
from oracle.assemble import assemble
from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rhs(p, H, seed):
    lev = H.levels[-1]
    return I.gather_natural(I.natural_vector(p, seed), lev.dof_field, lev.dof_comp, lev.dof_node)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _direct(A, b):
    """x* = A^{-1} b: sparse LU plus two refinement steps (the LU solve alone
    carries ~1e-10 relative error on these badly row-scaled systems)."""
    lu = spl.splu(A.tocsc())
    x = lu.solve(b)
    for _ in range(2):
        x = x + lu.solve(b - A @ x)
    return x


PROBLEMS = {
    "c0": lambda: I.make_config(0),
    # several Vanka tiles and a ragged last tile (49 vertices / 3), 4 levels
    "bulge48": lambda: I.make_channel_2d(48, 4, 3, 4242, bulge=True),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    p = PROBLEMS[request.param]()
    H = gmg.Hierarchy(p)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64)
    return request.param, p, H, s


def test_operator_values_all_levels(case):
    name, p, H, s = case
    for l, A in enumerate(H.A):
        ptr, col, val = s.matrix(l)
        L = sp.csr_matrix((val, col, ptr), shape=A.shape)
        D = (L - A).tocsr()
        scale = abs(A).max(axis=1).toarray().ravel()
        rows = np.repeat(np.arange(A.shape[0]), np.diff(D.indptr))
        rel = np.abs(D.data) / np.maximum(scale[rows], 1e-300)
        assert rel.size == 0 or rel.max() < 1e-13, (name, l, rel.max())


def test_spmv(case):
    """y = A_l x on every level (binned-ELL copy of the operator: bins of
    every row length, each a ragged number of 32-row slabs)."""
    name, p, H, s = case
    rng = np.random.default_rng(1)
    for l, A in enumerate(H.A):
        x = rng.standard_normal(A.shape[0])
        y = s.apply_operator(l, _cuda(x)).cpu().numpy()
        ref = A @ x
        bound = 1e-15 * 60 * (abs(A) @ np.abs(x))   # float64 sum of <= ~110 terms per row
        assert np.all(np.abs(y - ref) <= bound + 1e-300), (name, l)


@pytest.mark.parametrize("transpose", [False, True])
def test_smoother_fp64(case, transpose):
    name, p, H, s = case
    rng = np.random.default_rng(2)
    for l in range(1, len(H.A)):
        r = rng.standard_normal(H.A[l].shape[0])
        y = s.apply_smoother(l, _cuda(r), transpose=transpose).cpu().numpy()
        S = H.smoothers[l]
        ref = S.apply_transpose(r) if transpose else S.apply(r)
        assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref), (name, l)


@pytest.mark.parametrize("transpose", [False, True])
def test_vcycle_fp64(case, transpose):
    name, p, H, s = case
    v = np.random.default_rng(3).standard_normal(H.fine.shape[0])
    z = s.apply_vcycle(_cuda(v), transpose=transpose).cpu().numpy()
    ref = H.vcycle_transpose(v) if transpose else H.vcycle(v)
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)


def test_fgmres_fp64_solution_and_iterations(case):
    name, p, H, s = case
    b = _rhs(p, H, 11)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    xd = _direct(H.fine, b)
    assert st["converged"]
    assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    # iteration count parity at the workload tolerance
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    _, ost = ofg.solve(H, b, rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8, ost["iterations"])
    assert st8["rel_residual"] <= 1e-8
    assert st8["rho"] == pytest.approx(ost["rho"], rel=0.05)


@pytest.mark.parametrize("prec", [binding.FSI_MIXED, binding.FSI_MIXED_HALF])
def test_mixed_precision_solve(case, prec):
    name, p, H, s = case
    sm = binding.FSISolver(p)
    # float64 block inverses, as in the oracle's storage emulation
    sm.setup_smoothers(precision=prec, factor=binding.FSI_FACTOR_FP64)
    b = _rhs(p, H, 12)
    xd = _direct(H.fine, b)
    x, st = sm.solve(_cuda(b), rtol=1e-10)
    assert st["converged"]
    assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    # mixed V-cycle is a float32-accurate version of the FP64 cycle
    v = np.random.default_rng(5).standard_normal(H.fine.shape[0])
    z = sm.apply_vcycle(_cuda(v)).cpu().numpy()
    ref = H.vcycle(v)
    assert np.linalg.norm(z - ref) <= (1e-3 if prec == binding.FSI_MIXED else 2e-2) * np.linalg.norm(ref)
    # iterations close to the oracle's emulation of the same storage
    Hm = gmg.Hierarchy(p, mixed=True if prec == binding.FSI_MIXED else "half")
    _, ost = ofg.solve(Hm, b, rtol=1e-8)
    _, st8 = sm.solve(_cuda(b), rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])


def test_adjoint_and_gradients(case):
    name, p, H, s = case
    rng = np.random.default_rng(6)
    b = _rhs(p, H, 13)
    w = rng.standard_normal(b.size)
    xg, _ = s.solve(_cuda(b), rtol=1e-10)
    lam, dA, dmu, st = s.adjoint(_cuda(w), xg, rtol=1e-10)
    lam = lam.cpu().numpy()
    A = H.fine
    lam_d = _direct(A.T.tocsr(), w)
    assert st["converged"]
    assert np.linalg.norm(lam - lam_d) <= 1e-9 * np.linalg.norm(lam_d)
    x = xg.cpu().numpy()
    assert lam @ b == pytest.approx(w @ x, rel=1e-9)
    ptr, col, _ = s.matrix(len(H.A) - 1)
    rows = np.repeat(np.arange(b.size), np.diff(ptr))
    # the pattern gradient is -lambda_i x_j of the solve's own lambda and x
    np.testing.assert_allclose(dA.cpu().numpy(), -lam[rows] * x[col], rtol=1e-14, atol=0)
    ref_mu = oadj.mu_s_gradient(p, H.levels[-1], lam_d, x)
    assert dmu == pytest.approx(ref_mu, rel=1e-8)


def test_half_storage_smoother_matches_emulation(case):
    """FP16 row-scaled block inverses: the GPU smoother equals the oracle's
    emulation (float64 inverse, row max-abs scaling, float16 rounding,
    float32 apply) to float32 accumulation error."""
    name, p, H, s = case
    sh = binding.FSISolver(p)
    sh.setup_smoothers(precision=binding.FSI_MIXED_HALF, factor=binding.FSI_FACTOR_FP64)
    Hh = gmg.Hierarchy(p, mixed="half")
    rng = np.random.default_rng(8)
    for l in range(1, len(H.A)):
        r = rng.standard_normal(H.A[l].shape[0]).astype(np.float32).astype(np.float64)
        for tr in (False, True):
            y = sh.apply_smoother(l, _cuda(r), transpose=tr).cpu().numpy()
            S = Hh.smoothers[l]
            ref = (S.apply_transpose(r) if tr else S.apply(r)).astype(np.float64)
            assert np.linalg.norm(y - ref) <= 2e-5 * np.linalg.norm(ref), (name, l, tr)


def test_autograd_backward_is_adjoint():
    p = I.make_config(0)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64)
    H = gmg.Hierarchy(p)
    b = _cuda(_rhs(p, H, 14)).requires_grad_(True)
    w = _cuda(np.random.default_rng(7).standard_normal(b.numel()))
    x = binding.fsi_solve_autograd(b, s, rtol=1e-10)
    (x * w).sum().backward()
    lam = _direct(H.fine.T.tocsr(), w.cpu().numpy())
    assert np.linalg.norm(b.grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)


def test_autograd_operator_and_mu_s_gradients_central_differences():
    """autograd through fsi_solve_autograd with the operator values and mu_s
    as inputs: dJ/dA on the pattern and dJ/dmu_s against central differences
    of J = w^T A^{-1} b computed with the oracle (sparse direct solves of the
    oracle's assembled operator; mu_s perturbed in the assembly with
    lambda_s held fixed)."""
    p = I.make_config(0)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64)
    H = gmg.Hierarchy(p)
    A = H.fine.tocsr()
    rng = np.random.default_rng(15)
    bn = _rhs(p, H, 16)
    wn = rng.standard_normal(bn.size)
    b = _cuda(bn).requires_grad_(True)
    vals = s.operator_values().requires_grad_(True)
    mu = torch.tensor(p.mu_s, dtype=torch.float64, device="cuda", requires_grad=True)
    ptr, col, v0 = s.matrix(len(H.A) - 1)
    x = binding.fsi_solve_autograd(b, s, rtol=1e-11, values=vals, mu_s=mu)
    (x * _cuda(wn)).sum().backward()
    gA = vals.grad.cpu().numpy()
    gmu = float(mu.grad)
    solve = lambda M, rhs: _direct(M.tocsr(), rhs)
    J = lambda M: wn @ solve(M, bn)
    h = 1e-6
    # a random direction scaled entry-wise by |A_ij| (entries span many decades)
    dv = rng.standard_normal(v0.size) * np.abs(v0)
    D = sp.csr_matrix((dv, col, ptr), shape=A.shape)        # on the library's pattern and order
    fd = (J(A + h * D) - J(A - h * D)) / (2 * h)
    assert gA @ dv == pytest.approx(fd, rel=1e-5)
    Js = []
    for sgn in (1, -1):
        q = I.make_config(0)
        q.mu_s = p.mu_s * (1 + sgn * h)
        q.lambda_s = p.lambda_s
        Js.append(J(assemble(q, H.levels[-1])))
    assert gmu == pytest.approx((Js[0] - Js[1]) / (2 * h * p.mu_s), rel=1e-5)
    # dJ/db is lambda, as before
    lam = _direct(A.T.tocsr(), wn)
    assert np.linalg.norm(b.grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)


def test_error_statuses():
    p = I.make_config(0)
    s = binding.FSISolver(p)
    H = gmg.Hierarchy(p)
    b = _rhs(p, H, 15)
    with pytest.raises(binding.FSIError) as e:
        s.solve(_cuda(b))
    assert e.value.status == binding.FSI_ERR_STATE          # smoothers not set up
    s.setup_smoothers(precision=binding.FSI_FP64)
    x, st = s.solve(_cuda(b), max_iters=2, check=False)
    assert st["status"] == binding.FSI_ERR_NOT_CONVERGED and st["iterations"] == 2
    bad = b.copy()
    bad[3] = np.nan
    x, st = s.solve(_cuda(bad), check=False)
    assert st["status"] == binding.FSI_ERR_NONFINITE
    # zero right-hand side: zero solution, converged
    x, st = s.solve(_cuda(np.zeros_like(b)))
    assert st["converged"] and float(x.abs().max()) == 0.0
    # the context still works after the failures
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"]


def test_batched_uneven_systems_match_single_solves():
    """fsi_solve_batched advances several problems of different sizes, levels
    and materials together; each result equals the direct solution and the
    iteration count equals the single-problem solve's."""
    probs = [I.make_channel_2d(16, 3, 1, 101, band_width=0.2),
             I.make_channel_2d(32, 4, 3, 102, band_width=0.35, mu_s=20.0),
             I.make_channel_2d(24, 3, 3, 103, band_width=0.15),
             I.make_channel_2d(16, 2, 1, 104, band_width=0.3, mu_f=0.05)]
    sb = binding.FSISolver(probs)
    sb.setup_smoothers(precision=binding.FSI_MIXED_HALF, patch=3)
    bs, refs, singles = [], [], []
    for i, p in enumerate(probs):
        H = gmg.Hierarchy(p)
        b = _rhs(p, H, 20 + i)
        bs.append(_cuda(b))
        refs.append(_direct(H.fine, b))
        s1 = binding.FSISolver(p)
        s1.setup_smoothers(precision=binding.FSI_MIXED_HALF, patch=3)
        singles.append(s1.solve(_cuda(b), rtol=1e-10)[1]["iterations"])
    xs, sts = sb.solve_batched(bs, rtol=1e-10)
    for x, ref, st, it1 in zip(xs, refs, sts, singles):
        assert st["converged"]
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
        assert st["iterations"] == it1


def test_batch_graph_and_layout_autotune():
    """A batch over every problem runs as one graph launch (one solve chain
    per problem, each stopping on its own test): twice in a row it gives the
    same bits; the layout autotuner keeps one of its candidates, and the
    batched solves after it still match the direct solutions."""
    probs = [I.make_channel_2d(16, 3, 1, 111, band_width=0.2),
             I.make_channel_2d(32, 4, 3, 112, band_width=0.35, mu_s=20.0),
             I.make_channel_2d(24, 3, 3, 113, band_width=0.15)]
    sb = binding.FSISolver(probs)
    sb.setup_smoothers(precision=binding.FSI_MIXED_HALF, patch=3)
    bs, refs = [], []
    for i, p in enumerate(probs):
        H = gmg.Hierarchy(p)
        b = _rhs(p, H, 30 + i)
        bs.append(_cuda(b))
        refs.append(_direct(H.fine, b))
    xs1, sts1 = sb.solve_batched(bs, rtol=1e-10)
    xs2, sts2 = sb.solve_batched(bs, rtol=1e-10)
    for a, b_, s1, s2 in zip(xs1, xs2, sts1, sts2):
        assert s1["iterations"] == s2["iterations"]
        np.testing.assert_array_equal(a.cpu().numpy(), b_.cpu().numpy())
    chosen, times = sb.autotune_layout((0, 1, 4), rtol=1e-8)
    assert chosen in (0, 1, 4) and len(times) == 3 and min(times) < 1e300
    xs, sts = sb.solve_batched(bs, rtol=1e-10)
    for x, ref, st, st1 in zip(xs, refs, sts, sts1):
        assert st["converged"]
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
        assert abs(st["iterations"] - st1["iterations"]) <= 1


def test_3d_valve_box_parity():
    """3D: Q2 hexahedra (27 nodes), 376-dof Vanka blocks (8-CTA cluster
    Gauss-Jordan in float64), FP16 storage apply for blocks above 256 dofs."""
    p = I.make_valve_3d(8, 3, 1, 777)
    H = gmg.Hierarchy(p)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64)
    assert s.sizes(2)["max_block"] > 256
    for l, A in enumerate(H.A):
        ptr, col, val = s.matrix(l)
        L = sp.csr_matrix((val, col, ptr), shape=A.shape)
        D = (L - A).tocsr()
        scale = abs(A).max(axis=1).toarray().ravel()
        rows = np.repeat(np.arange(A.shape[0]), np.diff(D.indptr))
        assert D.nnz == 0 or (np.abs(D.data) / np.maximum(scale[rows], 1e-300)).max() < 1e-13
    rng = np.random.default_rng(9)
    for l in range(1, len(H.A)):
        r = rng.standard_normal(H.A[l].shape[0])
        y = s.apply_smoother(l, _cuda(r)).cpu().numpy()
        ref = H.smoothers[l].apply(r)
        assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref)
    v = rng.standard_normal(H.fine.shape[0])
    z = s.apply_vcycle(_cuda(v)).cpu().numpy()
    assert np.linalg.norm(z - H.vcycle(v)) <= 1e-9 * np.linalg.norm(H.vcycle(v))
    b = _rhs(p, H, 30)
    xd = _direct(H.fine, b)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    _, ost = ofg.solve(H, b, rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1
    sh = binding.FSISolver(p)
    sh.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    x, st = sh.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


def test_autotune_per_size_class_patch():
    """fsi_autotune times each candidate Vanka group size once per size class
    and rebuilds every problem's smoothers with its class's fastest choice;
    afterwards each smoother equals the oracle's FS-ASM with that group size
    and the batched solve still reaches the direct solution."""
    probs = [I.make_channel_2d(32, 4, 3, 301, band_width=0.3, mu_s=200.0),
             I.make_channel_2d(24, 3, 3, 302, band_width=0.2, mu_s=300.0),
             I.make_channel_2d(32, 4, 3, 303, band_width=0.25, mu_s=500.0)]
    s = binding.FSISolver(probs)
    s.setup_smoothers(precision=binding.FSI_FP64, patch=1)
    cand = (1, 2, 3)
    chosen, times = s.autotune(cand, rtol=1e-8)
    assert chosen[0] == chosen[2] and all(c in cand for c in chosen)
    for k, c in enumerate(chosen):
        assert np.isfinite(times[k][cand.index(c)])
        assert times[k][cand.index(c)] == min(times[k])
    np.testing.assert_array_equal(times[0], times[2])
    rng = np.random.default_rng(5)
    bs, refs = [], []
    for k, p in enumerate(probs):
        H = gmg.Hierarchy(p, patch=chosen[k])
        lf = len(H.A) - 1
        r = rng.standard_normal(H.A[lf].shape[0])
        y = s.apply_smoother(lf, _cuda(r), prob=k).cpu().numpy()
        ref = H.smoothers[lf].apply(r)
        assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref)
        b = _rhs(p, H, 40 + k)
        bs.append(_cuda(b))
        refs.append(_direct(H.fine, b))
    xs, sts = s.solve_batched(bs, rtol=1e-10)
    for x, ref, st in zip(xs, refs, sts):
        assert st["converged"]
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)


def test_device_loop_matches_host_loop(monkeypatch):
    """The solve runs as one CUDA graph whose restart and Arnoldi loops are
    WHILE nodes driven from the device; it must reproduce the host-driven
    loop (same kernels, same order): equal iteration and cycle counts and
    the same iterate, for a fresh solve, a replay, a warm start and the
    transposed (adjoint) solve."""
    p = PROBLEMS["bulge48"]()
    H = gmg.Hierarchy(p)
    b = _rhs(p, H, 77)
    sd = binding.FSISolver(p)
    sd.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    monkeypatch.setenv("FSI_DEVICE_LOOP", "0")
    sh = binding.FSISolver(p)
    monkeypatch.delenv("FSI_DEVICE_LOOP")
    sh.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    for rtol in (1e-10, 1e-6):
        for rep in range(2):
            xd, std = sd.solve(_cuda(b), rtol=rtol, restart=12)
            xh, sth = sh.solve(_cuda(b), rtol=rtol, restart=12)
            # the preconditioner is bitwise repeatable; the loops differ only in
            # the float64 rounding of the small least-squares update (device
            # kernel vs host loop), which can move a stop at the threshold by one
            assert abs(std["iterations"] - sth["iterations"]) <= 1
            assert std["cycles"] >= 1
            xd, xh = xd.cpu().numpy(), xh.cpu().numpy()
            assert np.linalg.norm(xd - xh) <= 1e-2 * rtol * np.linalg.norm(xh)
            assert std["converged"] and sth["converged"]
            assert std["rel_residual"] <= rtol and sth["rel_residual"] <= rtol
    x0 = _cuda(0.5 * _direct(H.fine, b))
    xd, std = sd.solve(_cuda(b), x0=x0.clone(), rtol=1e-10)
    xh, sth = sh.solve(_cuda(b), x0=x0.clone(), rtol=1e-10)
    assert abs(std["iterations"] - sth["iterations"]) <= 1
    assert np.linalg.norm(xd.cpu().numpy() - xh.cpu().numpy()) <= 1e-12 * np.linalg.norm(xh.cpu().numpy())
    w = _rhs(p, H, 78)
    x, _ = sd.solve(_cuda(b), rtol=1e-10)
    ad = sd.adjoint(_cuda(w), x, rtol=1e-10)
    ah = sh.adjoint(_cuda(w), x, rtol=1e-10)
    assert abs(ad[3]["iterations"] - ah[3]["iterations"]) <= 1
    assert np.linalg.norm(ad[0].cpu().numpy() - ah[0].cpu().numpy()) <= 1e-12 * np.linalg.norm(ah[0].cpu().numpy())


@pytest.mark.parametrize("variant", ["fs", "as"])
@pytest.mark.parametrize("prec", [binding.FSI_FP64, binding.FSI_MIXED, binding.FSI_MIXED_HALF])
def test_repeatable_smoother_and_solve(prec, variant):
    """Overlapping Schwarz blocks are combined owner by owner in block order
    (no float atomics), so the smoother, the forward solve and the adjoint
    solve give the same bits on every run."""
    p = PROBLEMS["bulge48"]()
    H = gmg.Hierarchy(p)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=prec, variant=binding.FSI_SMOOTHER_AS if variant == "as" else binding.FSI_SMOOTHER_FS)
    r = _cuda(np.random.default_rng(90).standard_normal(H.fine.shape[0]))
    l = len(H.A) - 1
    for tr in (False, True):
        y1 = s.apply_smoother(l, r, transpose=tr).cpu().numpy()
        y2 = s.apply_smoother(l, r, transpose=tr).cpu().numpy()
        np.testing.assert_array_equal(y1, y2)
    b = _cuda(_rhs(p, H, 91))
    x1, st1 = s.solve(b, rtol=1e-8)
    x2, st2 = s.solve(b, rtol=1e-8)
    assert st1["iterations"] == st2["iterations"]
    np.testing.assert_array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    w = _cuda(np.random.default_rng(92).standard_normal(H.fine.shape[0]))
    l1 = s.adjoint(w, x1, rtol=1e-8)[0].cpu().numpy()
    l2 = s.adjoint(w, x1, rtol=1e-8)[0].cpu().numpy()
    np.testing.assert_array_equal(l1, l2)


FACTOR_CASES = {
    "bulge48": lambda: I.make_channel_2d(48, 4, 3, 4242, bulge=True),     # 171-dof blocks, 2-CTA cluster
    "bulge48_b4": lambda: I.make_channel_2d(48, 4, 4, 4242, bulge=True),  # 258-dof blocks, 4-CTA cluster
    "valve8": lambda: I.make_valve_3d(8, 3, 1, 777),                      # 376-dof blocks, 4-CTA cluster
}


@pytest.mark.parametrize("name", list(FACTOR_CASES))
def test_float32_blocked_inversion(name):
    """Blocked float32 Gauss-Jordan (32-column panels) with the rank-32
    updates on the CUDA cores (FP32) or on the tensor cores (tcgen05, TF32
    operands): the smoother output against the same smoother with float64
    inverses, on every level, in float32 storage; then full solves with the
    tensor-core factors in both mixed modes.  Expected errors (the oracle's
    emulation of the blocked elimination): ~8e-8 (FP32) and ~1.3e-4 (TF32)."""
    p = FACTOR_CASES[name]()
    H = gmg.Hierarchy(p)
    ref = binding.FSISolver(p)
    ref.setup_smoothers(precision=binding.FSI_MIXED, factor=binding.FSI_FACTOR_FP64)
    rng = np.random.default_rng(12)
    for factor, tol in ((binding.FSI_FACTOR_FP32, 2e-6), (binding.FSI_FACTOR_TF32, 2e-3)):
        sv = binding.FSISolver(p)
        sv.setup_smoothers(precision=binding.FSI_MIXED, factor=factor)
        for l in range(1, len(H.A)):
            r = rng.standard_normal(H.A[l].shape[0]).astype(np.float32).astype(np.float64)
            y0 = ref.apply_smoother(l, _cuda(r)).cpu().numpy()
            y = sv.apply_smoother(l, _cuda(r)).cpu().numpy()
            assert np.linalg.norm(y - y0) <= tol * np.linalg.norm(y0), (factor, l)
            yt0 = ref.apply_smoother(l, _cuda(r), transpose=True).cpu().numpy()
            yt = sv.apply_smoother(l, _cuda(r), transpose=True).cpu().numpy()
            assert np.linalg.norm(yt - yt0) <= tol * np.linalg.norm(yt0), (factor, l)
    b = _rhs(p, H, 50)
    xd = _direct(H.fine, b)
    for prec in (binding.FSI_MIXED, binding.FSI_MIXED_HALF):
        s64 = binding.FSISolver(p)
        s64.setup_smoothers(precision=prec, factor=binding.FSI_FACTOR_FP64)
        stc = binding.FSISolver(p)
        stc.setup_smoothers(precision=prec)                 # default: tensor-core factors
        x, st = stc.solve(_cuda(b), rtol=1e-10)
        assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
        _, st8 = stc.solve(_cuda(b), rtol=1e-8)
        _, st64 = s64.solve(_cuda(b), rtol=1e-8)
        assert abs(st8["iterations"] - st64["iterations"]) <= 1, (st8["iterations"], st64["iterations"])
    with pytest.raises(binding.FSIError):
        binding.FSISolver(p).setup_smoothers(precision=binding.FSI_FP64, factor=binding.FSI_FACTOR_TF32)


def test_batch_larger_than_hardware_queues():
    """Ten systems (more than the 8 default hardware work queues) advance in
    host-driven rounds; each result matches the direct solution, and each
    iteration count its own single solve.  Counts are compared at rtol 1e-8:
    1e-10 lies at the attainable accuracy of these systems (the sparse LU
    itself leaves ~5e-11), where the count of the float32 cycle, whose
    overlapping scatter-add uses atomics, moves with rounding."""
    probs = [I.make_channel_2d(16 + 8 * (i % 3), 3, 1, 600 + i, band_width=0.15 + 0.02 * i,
                               mu_s=100.0 + 40.0 * i) for i in range(10)]
    sb = binding.FSISolver(probs)
    sb.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    bs, refs, singles = [], [], []
    for i, p in enumerate(probs):
        H = gmg.Hierarchy(p)
        b = _rhs(p, H, 70 + i)
        bs.append(_cuda(b))
        refs.append(_direct(H.fine, b))
        s1 = binding.FSISolver(p)
        s1.setup_smoothers(precision=binding.FSI_MIXED_HALF)
        singles.append(s1.solve(_cuda(b), rtol=1e-8)[1]["iterations"])
    xs, sts = sb.solve_batched(bs, rtol=1e-10)
    for x, ref, st in zip(xs, refs, sts):
        assert st["converged"]
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    _, sts8 = sb.solve_batched(bs, rtol=1e-8)
    for st, it1 in zip(sts8, singles):
        assert st["converged"] and abs(st["iterations"] - it1) <= 1, (st["iterations"], it1)


# ---- monolithic additive Schwarz AS, the paper's comparison preconditioner (Sec. 3.2)

@pytest.fixture(scope="module", params=list(PROBLEMS))
def as_case(request):
    p = PROBLEMS[request.param]()
    H = gmg.Hierarchy(p, monolithic=True)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64, variant=binding.FSI_SMOOTHER_AS)
    return request.param, p, H, s


def test_as_blocks_and_smoother_fp64(as_case):
    """AS block sets equal the oracle's on every level; the AS smoother and its
    transpose match the oracle to 1e-9 (FP64 Gauss-Jordan vs pivoted LU)."""
    name, p, H, s = as_case
    rng = np.random.default_rng(31)
    for l in range(1, len(H.A)):
        ptr, idx = s.blocks(l)
        S = H.smoothers[l]
        assert len(ptr) - 1 == len(S.blocks), (name, l)
        for j, ref in enumerate(S.blocks):
            np.testing.assert_array_equal(idx[ptr[j]:ptr[j + 1]], ref)
        r = rng.standard_normal(H.A[l].shape[0])
        for tr in (False, True):
            y = s.apply_smoother(l, _cuda(r), transpose=tr).cpu().numpy()
            ref = S.apply_transpose(r) if tr else S.apply(r)
            assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref), (name, l, tr)


def test_as_solves_fp64_and_mixed(as_case):
    """AS-preconditioned FGMRES: FP64 solution to 1e-9 of the direct solution,
    iterations +-1 of the oracle's; mixed precision (FP16 inverses, tensor-core
    factors) to 1e-8, iterations +-2 of the oracle's emulation."""
    name, p, H, s = as_case
    b = _rhs(p, H, 32)
    xd = _direct(H.fine, b)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    _, ost = ofg.solve(H, b, rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])
    sm = binding.FSISolver(p)
    sm.setup_smoothers(precision=binding.FSI_MIXED_HALF, variant=binding.FSI_SMOOTHER_AS)
    x, st = sm.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    Hm = gmg.Hierarchy(p, mixed="half", monolithic=True)
    _, ostm = ofg.solve(Hm, b, rtol=1e-8)
    _, stm = sm.solve(_cuda(b), rtol=1e-8)
    assert abs(stm["iterations"] - ostm["iterations"]) <= 1, (stm["iterations"], ostm["iterations"])


def test_as_3d_split_inversion():
    """AS blocks in 3D (~750 dofs: all fields on the 5^3 nodes around a
    vertex) are inverted by the 2 x 2 split over the two field systems (the
    halves by the cluster Gauss-Jordan kernel, the products by batched
    float32 GEMMs): block sets equal the oracle's, the smoother equals the
    oracle's float64 AS smoother to float32 accuracy of the block inverses
    (cond(A_jj) u_32, condition numbers up to ~1e4: 1e-3), the solve reaches
    the direct solution and needs the oracle's float32 emulation's iteration
    count +-1.  Float64 inverses of such blocks are refused (FSI_ERR_ARG)."""
    p = I.make_valve_3d(8, 2, 1, 777)
    s = binding.FSISolver(p)
    with pytest.raises(binding.FSIError) as err:
        s.setup_smoothers(precision=binding.FSI_FP64, variant=binding.FSI_SMOOTHER_AS)
    assert err.value.status == binding.FSI_ERR_ARG
    s.setup_smoothers(precision=binding.FSI_MIXED, factor=binding.FSI_FACTOR_FP32, variant=binding.FSI_SMOOTHER_AS)
    H = gmg.Hierarchy(p, monolithic=True)
    l = len(H.A) - 1
    assert s.sizes(l)["max_block"] > 512
    ptr, idx = s.blocks(l)
    for j, ref in enumerate(H.smoothers[l].blocks):
        np.testing.assert_array_equal(idx[ptr[j]:ptr[j + 1]], ref)
    rng = np.random.default_rng(42)
    r = rng.standard_normal(H.A[l].shape[0])
    for tr in (False, True):
        y = s.apply_smoother(l, _cuda(r), transpose=tr).cpu().numpy()
        S = H.smoothers[l]
        ref = S.apply_transpose(r) if tr else S.apply(r)
        assert np.linalg.norm(y - ref) <= 1e-3 * np.linalg.norm(ref), tr
    b = _rhs(p, H, 43)
    xd = _direct(H.fine, b)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    Hm = gmg.Hierarchy(p, monolithic=True, mixed=True)
    _, ost = ofg.solve(Hm, b, rtol=1e-8)
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])



def test_as_2d_wide_blocks_eight_cta_clusters():
    """Monolithic AS blocks of a 4 x 4 pressure-vertex group in 2D (~506
    dofs): the tensor-core and float32 Gauss-Jordan kernels in 8-CTA clusters
    with 16 register chunks per panel row.  Block sets equal the oracle's;
    with float32 factors the solve reaches the direct solution and needs the
    oracle's float32-storage emulation's iteration count +-1; with TF32
    factors it reaches the direct solution."""
    p = I.make_channel_2d(24, 3, 4, 7)
    H = gmg.Hierarchy(p, monolithic=True)
    l = len(H.A) - 1
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_MIXED, factor=binding.FSI_FACTOR_FP32, variant=binding.FSI_SMOOTHER_AS)
    assert 384 < s.sizes(l)["max_block"] <= 512
    ptr, idx = s.blocks(l)
    for j, ref in enumerate(H.smoothers[l].blocks):
        np.testing.assert_array_equal(idx[ptr[j]:ptr[j + 1]], ref)
    b = _rhs(p, H, 44)
    xd = _direct(H.fine, b)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    Hm = gmg.Hierarchy(p, monolithic=True, mixed=True)
    _, ost = ofg.solve(Hm, b, rtol=1e-8)
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])
    st_ = binding.FSISolver(p)
    st_.setup_smoothers(precision=binding.FSI_MIXED, factor=binding.FSI_FACTOR_TF32, variant=binding.FSI_SMOOTHER_AS)
    x, st = st_.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("prec", [binding.FSI_MIXED, binding.FSI_MIXED_HALF])
def test_mixed_adjoint_matches_direct_transposed_solve(case, prec):
    """Mixed-precision adjoint (transposed float32 cycle: transposed FP16 or
    float32 block applies streamed by rows, stored transpose of the coarse
    inverse): lambda to 1e-8 of the direct solve of A^T lambda = w when solved
    to a 1e-10 true residual, and lambda^T b = w^T x."""
    name, p, H, s = case
    sm = binding.FSISolver(p)
    sm.setup_smoothers(precision=prec)
    rng = np.random.default_rng(51)
    b = _rhs(p, H, 52)
    w = rng.standard_normal(b.size)
    x, _ = sm.solve(_cuda(b), rtol=1e-10)
    lam, _, _, st = sm.adjoint(_cuda(w), x, rtol=1e-10)
    assert st["converged"]
    lam = lam.cpu().numpy()
    lam_d = _direct(H.fine.T.tocsr(), w)
    assert np.linalg.norm(lam - lam_d) <= 1e-8 * np.linalg.norm(lam_d), (name, prec)
    assert lam @ b == pytest.approx(w @ x.cpu().numpy(), rel=1e-8)


# ---- locally multiplicative Schwarz sweep (Sec. 3.2, multiplicative update formula)

@pytest.fixture(scope="module", params=list(PROBLEMS))
def mult_case(request):
    p = PROBLEMS[request.param]()
    H = gmg.Hierarchy(p, mult_levels=99)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64, mult_levels=99)
    return request.param, p, H, s


def test_mult_sweep_and_transpose_fp64(mult_case):
    """y = M r and M^T r on every level equal the oracle's sweep, which
    updates one block after another, to 1e-9: the GPU updates all blocks of a
    pass (kind, colour) in one launch, from the residual of the field operator
    on the pass's rows (binned-ELL copy of A_FF, or A_FF^T, on those rows)."""
    name, p, H, s = mult_case
    rng = np.random.default_rng(61)
    for l in range(1, len(H.A)):
        r = rng.standard_normal(H.A[l].shape[0])
        S = H.smoothers[l]
        # the library stores the blocks in the oracle's sweep order, with its passes
        ptr, idx = s.blocks(l)
        for jj, j in enumerate(S.order):
            np.testing.assert_array_equal(idx[ptr[jj]:ptr[jj + 1]], S.blocks[j])
        np.testing.assert_array_equal(s.block_passes(l), S.block_pass[S.order])
        for tr in (False, True):
            y = s.apply_smoother(l, _cuda(r), transpose=tr).cpu().numpy()
            ref = S.apply_transpose(r) if tr else S.apply(r)
            assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref), (name, l, tr)
        # a second call gives the same result (the sweep's correction is cleared)
        y2 = s.apply_smoother(l, _cuda(r)).cpu().numpy()
        np.testing.assert_array_equal(y2, s.apply_smoother(l, _cuda(r)).cpu().numpy())


def test_mult_vcycle_solves_and_adjoint(mult_case):
    """FP64: V-cycle (and transposed) to 1e-9 of the oracle's; solution to 1e-9
    of the direct solution, iterations +-1 of the oracle's and fewer than with
    the additive smoother; adjoint lambda to 1e-9 of the direct transposed
    solve.  FP16 inverses: solution to 1e-8, iterations +-2 of the oracle's
    emulation."""
    name, p, H, s = mult_case
    v = np.random.default_rng(62).standard_normal(H.fine.shape[0])
    for tr in (False, True):
        z = s.apply_vcycle(_cuda(v), transpose=tr).cpu().numpy()
        ref = H.vcycle_transpose(v) if tr else H.vcycle(v)
        assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref), (name, tr)
    b = _rhs(p, H, 63)
    xd = _direct(H.fine, b)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    _, ost = ofg.solve(H, b, rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])
    _, ost_add = ofg.solve(gmg.Hierarchy(p), b, rtol=1e-8)
    assert st8["iterations"] < ost_add["iterations"]
    w = np.random.default_rng(64).standard_normal(b.size)
    lam, _, _, sta = s.adjoint(_cuda(w), x, rtol=1e-10)
    lam_d = _direct(H.fine.T.tocsr(), w)
    assert sta["converged"]
    assert np.linalg.norm(lam.cpu().numpy() - lam_d) <= 1e-9 * np.linalg.norm(lam_d)
    sh = binding.FSISolver(p)
    sh.setup_smoothers(precision=binding.FSI_MIXED_HALF, factor=binding.FSI_FACTOR_FP64, mult_levels=99)
    x, st = sh.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    Hh = gmg.Hierarchy(p, mixed="half", mult_levels=99)
    _, osth = ofg.solve(Hh, b, rtol=1e-8)
    _, sth = sh.solve(_cuda(b), rtol=1e-8)
    assert abs(sth["iterations"] - osth["iterations"]) <= 1, (sth["iterations"], osth["iterations"])


def test_mult_fine_level_only_mixed():
    """The configuration the benchmark times: the multiplicative sweep on the
    finest level only (additive below), FP16 inverses from tensor-core
    factors: converges, and in fewer iterations than the additive smoother;
    the forward and adjoint solutions match the direct solves."""
    p = PROBLEMS["bulge48"]()
    H = gmg.Hierarchy(p)
    b = _rhs(p, H, 65)
    xd = _direct(H.fine, b)
    sa = binding.FSISolver(p)
    sa.setup_smoothers(precision=binding.FSI_MIXED_HALF)
    sm = binding.FSISolver(p)
    sm.setup_smoothers(precision=binding.FSI_MIXED_HALF, mult_levels=1)
    x, st = sm.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    _, st_m = sm.solve(_cuda(b), rtol=1e-8)
    _, st_a = sa.solve(_cuda(b), rtol=1e-8)
    assert st_m["iterations"] < st_a["iterations"], (st_m["iterations"], st_a["iterations"])
    w = np.random.default_rng(66).standard_normal(b.size)
    lam, _, _, sta = sm.adjoint(_cuda(w), x, rtol=1e-10)
    lam_d = _direct(H.fine.T.tocsr(), w)
    assert sta["converged"] and np.linalg.norm(lam.cpu().numpy() - lam_d) <= 1e-8 * np.linalg.norm(lam_d)


def test_mult_rejected_with_monolithic_blocks():
    p = I.make_config(0)
    s = binding.FSISolver(p)
    with pytest.raises(binding.FSIError) as err:
        s.setup_smoothers(precision=binding.FSI_FP64, variant=binding.FSI_SMOOTHER_AS, mult_levels=1)
    assert err.value.status == binding.FSI_ERR_ARG
    with pytest.raises(binding.FSIError) as err:
        s.setup_smoothers(precision=binding.FSI_FP64, mult_levels=-1)
    assert err.value.status == binding.FSI_ERR_ARG


def test_mult_3d_sweep_and_solve():
    """3D valve box, b = 1 (the 3D workload's group size; b = 2 blocks of ~1000
    dofs exceed the inversion kernels): 64 colours x 3 kinds = 192 passes of
    blocks up to 376 dofs; the fine-level sweep equals the oracle's to 1e-9
    (FP64), the solve reaches the direct solution, iterations +-1 of the
    oracle's."""
    p = I.make_valve_3d(8, 2, 1, 4243)
    H = gmg.Hierarchy(p, mult_levels=1)
    s = binding.FSISolver(p)
    s.setup_smoothers(precision=binding.FSI_FP64, mult_levels=1)
    l = len(H.A) - 1
    S = H.smoothers[l]
    np.testing.assert_array_equal(s.block_passes(l), S.block_pass[S.order])
    r = np.random.default_rng(71).standard_normal(H.A[l].shape[0])
    y = s.apply_smoother(l, _cuda(r)).cpu().numpy()
    ref = S.apply(r)
    assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref)
    b = _rhs(p, H, 72)
    xd = _direct(H.fine, b)
    x, st = s.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    _, st8 = s.solve(_cuda(b), rtol=1e-8)
    _, ost = ofg.solve(H, b, rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])


# ---- swapped cascade (the paper's future work, Sec. 5): Krylov preconditioned
# by FS with a GMG V-cycle inside each field system
@pytest.mark.parametrize("mult_levels", [0, 1])
def test_cascade_vcycle_and_solves(case, mult_levels):
    name, p, H, s = case
    Hc = gmg.Hierarchy(p, cascade=True, mult_levels=mult_levels)
    sc = binding.FSISolver(p)
    sc.setup_smoothers(precision=binding.FSI_FP64, cascade=True, mult_levels=mult_levels)
    rng = np.random.default_rng(95)
    v = rng.standard_normal(Hc.fine.shape[0])
    b = _rhs(p, Hc, 96)
    xd = _direct(Hc.fine, b)
    x, st = sc.solve(_cuda(b), rtol=1e-10)
    assert st["converged"]
    assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    _, st8 = sc.solve(_cuda(b), rtol=1e-8)
    _, ost = ofg.solve(Hc, b, rtol=1e-8)
    assert abs(st8["iterations"] - ost["iterations"]) <= 1, (st8["iterations"], ost["iterations"])
    # the transposed cycle (built with the transposes by the adjoint)
    w = rng.standard_normal(b.size)
    lam, _, _, sta = sc.adjoint(_cuda(w), x, rtol=1e-10)
    lam_d = _direct(Hc.fine.T.tocsr(), w)
    assert sta["converged"]
    assert np.linalg.norm(lam.cpu().numpy() - lam_d) <= 1e-9 * np.linalg.norm(lam_d)
    for tr in (False, True):
        z = sc.apply_vcycle(_cuda(v), transpose=tr).cpu().numpy()
        ref = Hc.vcycle_transpose(v) if tr else Hc.vcycle(v)
        assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref), (name, tr)
    # mixed precision with float16 inverses: iterations against the oracle's emulation
    sh = binding.FSISolver(p)
    sh.setup_smoothers(precision=binding.FSI_MIXED_HALF, factor=binding.FSI_FACTOR_FP64, cascade=True,
                       mult_levels=mult_levels)
    x, st = sh.solve(_cuda(b), rtol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    Hh = gmg.Hierarchy(p, cascade=True, mixed="half", mult_levels=mult_levels)
    _, osth = ofg.solve(Hh, b, rtol=1e-8)
    _, sth = sh.solve(_cuda(b), rtol=1e-8)
    assert abs(sth["iterations"] - osth["iterations"]) <= 1, (sth["iterations"], osth["iterations"])


def test_cascade_rejected_with_monolithic_blocks():
    s = binding.FSISolver(I.make_config(0))
    with pytest.raises(binding.FSIError):
        s.setup_smoothers(precision=binding.FSI_FP64, variant=binding.FSI_SMOOTHER_AS, cascade=True)
