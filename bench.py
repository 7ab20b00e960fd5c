#!/usr/bin/env python
"""Benchmark of the FSI solve: fine DOF/s to reach a 1e-8 relative residual.

Workload: the 2D channel with an aneurysm-like wall pocket, 256 x 256 fine
elements, 7 GMG levels, 1.12 M unknowns (seeded synthetic stand-in for the
paper's 2D aneurysm meshes).  One step = one complete FGMRES(30) solve from
x0 = 0 to a float64 true relative residual <= 1e-8 (V-cycle with FS-ASM
smoothing, Arnoldi, refinement): every step of the solve path.  Set-up
(hierarchy, assembly, block factorisation) is timed separately.

  value      mixed precision (float32 cycle with float16 row-scaled block
             inverses, float64 Krylov) with the locally multiplicative Schwarz
             sweep per field system on the finest level (Sec. 3.2; additive
             on the coarser levels), device-resident right-hand side, CUDA
             events on the solver's stream;
  additive   the same with the additive field-split smoother everywhere;
  mixed_f32_inverses  the headline configuration with float32 inverses;
  fp64       the all-float64 path on the same system (mixed/fp64 speed-up);
  as_smoother  the paper's monolithic AS comparison smoother;
  cascade    the swapped cascade of the paper's future work (Sec. 5);
  e2e        the headline through the public call with host buffers
             (pinned H2D of b, solve, D2H of x inside the timed region);
  roofline   the fine-level sweep (its apply and pass-residual launches on
             two streams): algorithmic bytes / its mean time from CUDA
             events, against the measured HBM copy bandwidth;
  nonlinear  implicit time steps of the nonlinear problem (Sec. 2.2) on the
             same channel from rest: exact Newton, every Newton system solved
             by the headline configuration; the paper's s^max, N and rho;
  cpu_baseline  the FP64 oracle on this host, bounded sample (see "sample").

--impl reference runs the oracle itself as the reference arm.  With
torchrun, every rank solves its own replica of the workload (weak scaling).
"""
from __future__ import annotations

import os

# 32 hardware work queues instead of CUDA's default 8 (read when the CUDA
# context is created): the batched leg keeps 64 whole-solve graphs in flight
# on 64 streams, which otherwise share 8 queues and wait on one another
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fine DOF/s to 1e-8 rel residual (mixed vs FP64 GPU); smoother % HBM peak"
UNIT = "DOF/s"
RTOL = 1e-8
NL_FORCE = 20.0       # body-force amplitude of the nonlinear leg
NL_STEPS = 4          # implicit time steps of the nonlinear leg
NL_RTOL = 1e-8        # Newton tolerance on ||R|| relative to the step's initial residual
NL_JAC_INST_PER_ELEMENT = 142.1e3   # float64 thread-instructions per element of one Jacobian (ncu)
# the timed smoother: the locally multiplicative sweep on this many finest
# levels (additive below); 0 = additive everywhere
HEAD_MULT = 1
# FGMRES iterations the oracle's float64 algorithm with that smoother needs on
# each seeded workload to reach RTOL (oracle.fgmres.solve with
# gmg.Hierarchy(p, mult_levels=1) on the same right-hand side); used to
# project the oracle's per-iteration time to the metric.
ORACLE_ITERATIONS = {0: 12, 1: 24, 4: 18}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-iters", type=int, default=3, help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Replicas across ranks: every rank runs the whole workload on its own GPU;
# the only cross-rank traffic is the timing barrier and the max of the
# per-rank times (no collective on the data path).
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    """Slowest rank's value: the whole job takes as long as its slowest replica."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def its_summary(its):
    """min / median / max FGMRES iterations of the timed solves of one leg."""
    if not its:
        return None
    return {"min": min(its), "median": statistics.median(its), "max": max(its), "solves": len(its)}


def job_throughput(units_per_rank, ms, world):
    """Weak scaling: units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------- oracle leg
def oracle_rhs(p):
    from oracle import mesh
    from paper_1909_13201_gb300 import inputs as I
    lev = mesh.build_levels(p)[-1]
    return I.gather_natural(I.natural_vector(p, 1), lev.dof_field, lev.dof_comp, lev.dof_node)


def oracle_sample(cfg: int, iters: int, steps: int = 1, warmup: int = 0):
    """Time the FP64 oracle: set-up untimed, then `steps` samples of `iters`
    FGMRES iterations each.  Returns per-iteration seconds of every sample."""
    from oracle import fgmres, gmg
    from paper_1909_13201_gb300 import inputs as I
    p = I.make_config(cfg)
    t0 = time.time()
    H = gmg.Hierarchy(p, mult_levels=HEAD_MULT)
    setup_s = time.time() - t0
    b = oracle_rhs(p)
    per_it, cpu_it = [], []
    for k in range(warmup + steps):
        t, c = time.time(), time.process_time()
        _, st = fgmres.solve(H, b, rtol=RTOL, maxit=iters)
        its = max(st["iterations"], 1)
        dt, dc = (time.time() - t) / its, (time.process_time() - c) / its
        if k >= warmup:
            per_it.append(dt)
            cpu_it.append(dc)
    return {"n": int(H.fine.shape[0]), "setup_s": setup_s, "per_iteration_s": per_it,
            "cpu_per_iteration_s": cpu_it, "iterations_timed": iters * steps}


def _oracle_run(cfg: int, threads: int):
    """The oracle sample in a fresh process whose BLAS/OpenMP pools hold
    `threads` threads; None (and the error) if it failed."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", "--config", str(cfg)],
                         capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        return None, out.stderr.strip().splitlines()[-1][:200]
    return json.loads(out.stdout.strip().splitlines()[-1]), None


def cpu_baseline(cfg: int):
    """The FP64 oracle as it stands on this host's cores: a bounded sample
    (3 FGMRES iterations after an untimed set-up) with 1 thread and with
    nproc threads; cores = the threads the process kept busy (CPU time /
    wall time over the timed iterations).  The metric's value is projected
    to the iterations the oracle needs to reach RTOL."""
    n_it = ORACLE_ITERATIONS.get(cfg)
    nproc = os.cpu_count() or 1
    legs = {}
    for threads in (1, nproc):
        res, err = _oracle_run(cfg, threads)
        if res is None:
            legs[threads] = {"value": None, "error": err}
            continue
        t_it = statistics.median(res["per_iteration_s"])
        c_it = statistics.median(res["cpu_per_iteration_s"])
        legs[threads] = {"value": res["n"] / (t_it * n_it), "s_per_iteration": t_it,
                         "cores_busy": round(c_it / t_it, 2), "threads": threads, "setup_s": res["setup_s"],
                         "iterations_timed": res["iterations_timed"]}
    one = legs[1]
    out = {"value": one["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"FP64 oracle, {one.get('iterations_timed')} FGMRES its timed "
                      f"({one.get('s_per_iteration', 0):.2f} s each) after an untimed set-up; value projected "
                      f"to the {n_it} its it needs for {RTOL:g}"),
           "projected_iterations": n_it}
    many = legs[nproc]
    out["nproc"] = {"value": many["value"], "threads": nproc, "cores": many.get("cores_busy"),
                    "s_per_iteration": many.get("s_per_iteration")}
    return out


# ------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# GB300 float64 rate (nominal; the bench also measures it, fsi_profile mode
# 3): the outer product and the Gram-Schmidt passes are bound by it, not by HBM
FP64_NOMINAL_GFLOPS = 1250.0


def measured_tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst figure times the
    nominal TF32/bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16 = json.load(open(path)).get("bf16_tflops", 1900.0) if os.path.exists(path) else 1900.0
    return bf16 * 1.1 / 2.25


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def device_code_sha(path):
    """sha256[:16] of a CUDA source's device code: its text before the first
    host function definition (a line starting with "fsi_status ")."""
    text = []
    for line in open(path, encoding="utf-8"):
        if line.startswith("fsi_status "):
            break
        text.append(line)
    return hashlib.sha256("".join(text).encode()).hexdigest()[:16]


def ncu_traffic(summary="sweep_fine_c1_mult_half.md", key="dram bytes per sweep",
                sources=("kernels_block.cu", "kernels_sparse.cu")):
    """DRAM bytes per unit of the roofline's kernel(s) from a committed ncu
    summary, valid only while the device code of every source it covers is
    unchanged (the summary records each source's sha)."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            vals[k.strip()] = v.strip().split()[0]
    for src in sources:
        sha = device_code_sha(os.path.join(ROOT, "paper_1909_13201_gb300", "csrc", src))
        if vals.get(f"{src} device code sha256[:16]") != sha:
            return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------- our arm
def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1909_13201_gb300 import inputs as I
    from paper_1909_13201_gb300.binding import (FSI_FACTOR_FP32, FSI_FACTOR_FP64, FSI_FACTOR_TF32, FSI_FP64,
                                                FSI_MIXED, FSI_MIXED_HALF, FSI_SMOOTHER_AS, FSISolver)

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    p = I.make_config(args.config)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    s = FSISolver(p, stream=stream)
    torch.cuda.synchronize()
    setup_hier_s = time.time() - t0
    n = s.sizes(p.n_levels - 1)["n"]
    f, c, nd = s.dof_map(p.n_levels - 1)
    b_host = I.gather_natural(I.natural_vector(p, 1), f.astype(np.int64), c.astype(np.int64), nd.astype(np.int64))
    b = torch.from_numpy(b_host).to(dev)
    x = torch.empty_like(b)

    def timed(k, fn):
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1) / k, world, dev)

    stats = {}
    its_log = []          # iterations of every solve since the last reset

    def solve_dev():
        _, st = s.solve(b, rtol=RTOL, out=x)
        stats.update(st)
        its_log.append(int(st["iterations"]))

    def timed_its(k, fn):
        """timed() plus the iteration counts of the timed solves."""
        its_log.clear()
        t = timed(k, fn)
        return t, its_summary(its_log)

    # ---- headline: mixed precision, float16 block inverses, the locally
    # multiplicative sweep (Sec. 3.2) on the finest level, additive below
    t0 = time.time()
    s.setup_smoothers(precision=FSI_MIXED_HALF, mult_levels=HEAD_MULT)
    torch.cuda.synchronize()
    setup_mixed_s = time.time() - t0
    for _ in range(args.warmup):
        solve_dev()
    props = torch.cuda.get_device_properties(local)
    smi_id = str(local)
    if all(hasattr(props, a) for a in ("pci_domain_id", "pci_bus_id", "pci_device_id")):
        smi_id = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    clocks = Clocks(smi_id)
    clocks.start()
    ms, its_mixed = timed_its(args.steps, solve_dev)
    clk = clocks.stop()
    st_mixed = dict(stats)
    # whole solve against the HBM roofline: algorithmic bytes of every V-cycle,
    # outer product and Gram-Schmidt pass of the timed solve (fsi_get_cost)
    solve_bytes = s.solve_bytes(its_mixed["median"])
    # roofline of the fine-level sweep and launch count, from profiled solves
    s.profile(1)
    for _ in range(2):
        solve_dev()
    prof = s.profile(0)
    launches_per_step = prof["kernel_launches"] / 2.0
    sm_ms = prof["smoother_ms"] / max(prof["smoother_launches"], 1)
    achieved = prof["smoother_bytes"] / (sm_ms * 1e-3) / 1e9
    spmv_ms = prof["spmv_ms"] / max(prof["spmv_launches"], 1)
    spmv_gbs = prof["spmv_bytes"] / (spmv_ms * 1e-3) / 1e9
    rst_ms = prof["restrict_ms"] / max(prof["restrict_launches"], 1)
    rst_gbs = prof["restrict_bytes"] / (rst_ms * 1e-3) / 1e9
    pro_ms = prof["prolong_ms"] / max(prof["prolong_launches"], 1)
    pro_gbs = prof["prolong_bytes"] / (pro_ms * 1e-3) / 1e9
    outer_ms = prof["outer_ms"] / max(prof["outer_launches"], 1)
    outer_gbs = prof["outer_bytes"] / (outer_ms * 1e-3) / 1e9
    outer_gflops = 2.0 * prof["outer_fma"] / (outer_ms * 1e-3) / 1e9
    gs64_gflops = 2.0 * prof["gs64_fma"] / (prof["gs64_ms"] * 1e-3) / 1e9 if prof["gs64_ms"] > 0 else None
    gs64_gbs = prof["gs64_bytes"] / (prof["gs64_ms"] * 1e-3) / 1e9 if prof["gs64_ms"] > 0 else None
    gs1_gbs = prof["gs1_bytes"] / (prof["gs1_ms"] * 1e-3) / 1e9 if prof["gs1_ms"] > 0 else None
    fp64_peak = s.profile(3)["fp64_gflops"]          # measured float64 FMA rate of this GPU
    peak, peak_kind = measured_peaks()
    gs64_bound_frac = (max(2.0 * prof["gs64_fma"] / (fp64_peak * 1e9), prof["gs64_bytes"] / (peak * 1e9))
                       / (prof["gs64_ms"] * 1e-3) if prof["gs64_ms"] > 0 and fp64_peak else None)
    # ---- end to end through the public call with host buffers (mixed)
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()

    def solve_e2e():
        b.copy_(b_pin, non_blocking=True)
        _, st = s.solve(b, rtol=RTOL, out=x)
        its_log.append(int(st["iterations"]))
        x_pin.copy_(x, non_blocking=True)

    solve_e2e()
    ms_e2e, its_e2e = timed_its(max(2, args.steps // 2), solve_e2e)
    # ---- set-up: fine-level batched block inversion by each factorisation
    fact = {}
    for fname, fcode in (("tf32_tensor_cores", FSI_FACTOR_TF32), ("fp32_cuda_cores", FSI_FACTOR_FP32),
                         ("fp64_cuda_cores", FSI_FACTOR_FP64)):
        t0 = time.time()
        s.profile(1)
        s.setup_smoothers(precision=FSI_MIXED_HALF, factor=fcode)
        torch.cuda.synchronize()
        pf = s.profile(0)
        inv_ms = pf["invert_ms"] / max(pf["invert_launches"], 1)
        fact[fname] = {"fine_inversion_ms": inv_ms, "fine_blocks": pf["fine_blocks"],
                       "gflop": pf["invert_flops"] / 1e9,
                       "achieved_tflops": pf["invert_flops"] / (inv_ms * 1e-3) / 1e12,
                       "smoothers_setup_s": time.time() - t0}
    tf32_peak = measured_tf32_peak()
    fact["tf32_tensor_cores"]["frac_of_tf32_peak"] = fact["tf32_tensor_cores"]["achieved_tflops"] / tf32_peak
    fact["tf32_peak_tflops"] = tf32_peak
    # ---- mixed precision with float32 block inverses
    t0 = time.time()
    s.setup_smoothers(precision=FSI_MIXED, mult_levels=HEAD_MULT)
    torch.cuda.synchronize()
    setup_f32_s = time.time() - t0
    solve_dev()
    ms32, its32 = timed_its(max(2, args.steps // 2), solve_dev)
    st32 = dict(stats)
    # ---- all-float64 path on the same system
    t0 = time.time()
    s.setup_smoothers(precision=FSI_FP64, mult_levels=HEAD_MULT)
    torch.cuda.synchronize()
    setup_fp64_s = time.time() - t0
    solve_dev()
    ms64, its64 = timed_its(max(2, args.steps // 3), solve_dev)
    st64 = dict(stats)
    # ---- the paper's comparison: monolithic additive Schwarz (AS) level smoother, same cycle
    t0 = time.time()
    # float32 inverses: with FP16 storage the monolithic blocks make no progress on this system
    # (their inverses mix rows of every field, whose entries span beyond FP16's range)
    s.setup_smoothers(precision=FSI_MIXED, factor=FSI_FACTOR_FP32, variant=FSI_SMOOTHER_AS)
    torch.cuda.synchronize()
    setup_as_s = time.time() - t0
    def solve_as():
        _, st = s.solve(b, rtol=RTOL, out=x, check=False, max_iters=300)
        stats.update(st)
        its_log.append(int(st["iterations"]))

    solve_as()
    ms_as, its_as = timed_its(max(2, args.steps // 4), solve_as)
    st_as = dict(stats)

    # ---- the additive field-split smoother on every level (same storage)
    t0 = time.time()
    s.setup_smoothers(precision=FSI_MIXED_HALF, mult_levels=0)
    torch.cuda.synchronize()
    setup_add_s = time.time() - t0
    for _ in range(max(args.warmup, 1)):
        solve_dev()
    ms_add, its_add = timed_its(args.steps, solve_dev)
    st_add = dict(stats)
    s.profile(1)
    for _ in range(2):
        solve_dev()
    prof_add = s.profile(0)
    sm_add_ms = prof_add["smoother_ms"] / max(prof_add["smoother_launches"], 1)
    sm_add_gbs = prof_add["smoother_bytes"] / (sm_add_ms * 1e-3) / 1e9
    # ---- the swapped cascade (Sec. 5 future work): FGMRES preconditioned by
    # the field split, a GMG V-cycle inside each field system
    t0 = time.time()
    s.setup_smoothers(precision=FSI_MIXED_HALF, mult_levels=HEAD_MULT, cascade=True)
    torch.cuda.synchronize()
    setup_casc_s = time.time() - t0
    solve_dev()
    ms_casc, its_casc = timed_its(max(2, args.steps // 4), solve_dev)

    # ---- batched: 64 independent uneven 2D systems solved together
    batch = I.make_config(3)
    t0 = time.time()
    sb = FSISolver(batch, stream=stream)
    sb.setup_smoothers(precision=FSI_MIXED_HALF, patch=3)
    torch.cuda.synchronize()
    setup_batch_s = time.time() - t0
    bb = []
    for k, q in enumerate(batch):
        lv = q.n_levels - 1
        f_, c_, nd_ = sb.dof_map(lv, prob=k)
        bb.append(torch.from_numpy(I.gather_natural(I.natural_vector(q, 1), f_.astype(np.int64),
                                                    c_.astype(np.int64), nd_.astype(np.int64))).to(dev))
    xb = [torch.empty_like(v) for v in bb]
    bstats = []

    def solve_batch():
        _, sts = sb.solve_batched(bb, xs=xb, rtol=RTOL)
        bstats[:] = sts

    solve_batch()
    ms_batch_fixed = timed(max(2, args.steps // 4), solve_batch)
    # per size class, keep the fastest Vanka group size (native autotuner)
    t0 = time.time()
    tune_cand = (2, 3, 4)
    chosen, _ = sb.autotune(tune_cand, rtol=RTOL)
    torch.cuda.synchronize()
    tune_s = time.time() - t0
    # lanes per row of the sparse copies, timed on the whole batch (native autotuner)
    t0 = time.time()
    lanes_chosen, lanes_times = sb.autotune_layout((0, 1, 4), rtol=RTOL)
    tune_layout_s = time.time() - t0
    solve_batch()
    ms_batch = timed(max(2, args.steps // 4), solve_batch)
    batch_bytes = sum(sb.solve_bytes(t["iterations"], prob=k) for k, t in enumerate(bstats))
    chosen_by_size = {str(q.n_fine): c for q, c in zip(batch, chosen)}
    batch_dofs = sum(int(v.numel()) for v in bb)
    # ---- adjoint: forward solve plus the transposed solve with gradients (128^2)
    pa = I.make_config(4)
    sa = FSISolver(pa, stream=stream)
    sa.setup_smoothers(precision=FSI_MIXED_HALF)
    na = sa.sizes(pa.n_levels - 1)["n"]
    fa, ca, nda = sa.dof_map(pa.n_levels - 1)
    ba = torch.from_numpy(I.gather_natural(I.natural_vector(pa, 1), fa.astype(np.int64), ca.astype(np.int64),
                                           nda.astype(np.int64))).to(dev)
    wa = torch.from_numpy(I.gather_natural(I.natural_vector(pa, 2), fa.astype(np.int64), ca.astype(np.int64),
                                           nda.astype(np.int64))).to(dev)
    xa = torch.empty_like(ba)
    astats = {}

    def fwd_adj():
        _, st_f = sa.solve(ba, rtol=RTOL, out=xa)
        _, _, _, st_a = sa.adjoint(wa, xa, rtol=RTOL)
        astats.update(forward=st_f["iterations"], adjoint=st_a["iterations"])

    fwd_adj()
    ms_adj = timed(max(2, args.steps // 4), fwd_adj)

    # ---- 3D valve box, 32^3 hexahedra, 4 levels, mixed precision
    p3 = I.make_config(2)
    t0 = time.time()
    s3 = FSISolver(p3, stream=stream)
    torch.cuda.synchronize()
    setup_3d_hier_s = time.time() - t0
    t0 = time.time()
    s3.profile(1)
    s3.setup_smoothers(precision=FSI_MIXED_HALF)
    torch.cuda.synchronize()
    pf3 = s3.profile(0)
    setup_3d_smooth_s = time.time() - t0
    inv3_ms = pf3["invert_ms"] / max(pf3["invert_launches"], 1)
    n3 = s3.sizes(p3.n_levels - 1)["n"]
    f3, c3_, nd3 = s3.dof_map(p3.n_levels - 1)
    b3 = torch.from_numpy(I.gather_natural(I.natural_vector(p3, 1), f3.astype(np.int64), c3_.astype(np.int64),
                                           nd3.astype(np.int64))).to(dev)
    x3 = torch.empty_like(b3)
    st3 = {}

    def solve_3d():
        _, st = s3.solve(b3, rtol=RTOL, out=x3)
        st3.update(st)
        its_log.append(int(st["iterations"]))

    solve_3d()
    ms_3d, its_3d = timed_its(2, solve_3d)
    s3.profile(1)
    solve_3d()
    pr3 = s3.profile(0)
    sm3 = pr3["smoother_ms"] / max(pr3["smoother_launches"], 1)
    # ---- the paper's 3D comparison (Sec. 4.2): the monolithic AS smoother on the
    # same 3D system; its ~750-dof blocks are inverted by the split over the
    # two field systems, float32 inverses (FP16 storage does not converge for AS)
    t0 = time.time()
    s3.setup_smoothers(precision=FSI_MIXED, factor=FSI_FACTOR_FP32, variant=FSI_SMOOTHER_AS)
    torch.cuda.synchronize()
    setup_as3_s = time.time() - t0

    def solve_as3():
        _, st = s3.solve(b3, rtol=RTOL, out=x3, check=False, max_iters=300)
        st3.update(st)
        its_log.append(int(st["iterations"]))

    solve_as3()
    ms_as3, its_as3 = timed_its(2, solve_as3)
    conv_as3 = bool(st3.get("converged"))
    del s3, b3, x3
    torch.cuda.empty_cache()
    # ---- the nonlinear time loop (Sec. 2.2): implicit steps of the same 256^2
    # channel from rest under the pulsatile body force, exact Newton with the
    # headline solver on every Newton system (Jacobians on all levels, blocks
    # refactored per Newton step); the paper's s^max, N and rho (Sec. 4)
    t0 = time.time()
    snl = FSISolver(p, stream=stream, nonlinear=True)
    snl.nl_setup(force=NL_FORCE)
    snl.setup_smoothers(precision=FSI_MIXED_HALF, mult_levels=1)
    torch.cuda.synchronize()
    setup_nl_s = time.time() - t0
    Un_nl = torch.zeros(n, dtype=torch.float64, device=dev)
    U_nl = torch.empty_like(Un_nl)
    nl_steps = []
    for k in range(NL_STEPS):
        U_nl.copy_(Un_nl)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = snl.nl_step(Un_nl, U_nl, (k + 1) * p.dt, nl_rtol=NL_RTOL, lin_rtol=RTOL, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        g["ms"] = e0.elapsed_time(e1)
        nl_steps.append(g)
        Un_nl.copy_(U_nl)
    jac_ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        snl.nl_jacobian(U_nl, Un_nl, NL_STEPS * p.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        jac_ms.append(e0.elapsed_time(e1))
    del snl, Un_nl, U_nl
    torch.cuda.empty_cache()
    n_el_all = sum((p.n_fine >> l) ** 2 for l in range(p.n_levels))
    nl_newton = [st["newton_steps"] for st in nl_steps]
    nl_its = [i for st in nl_steps for i in st["iterations"]]
    nl_rho = [r for st in nl_steps for r in st["rho"]]
    nl_ms = [st["ms"] for st in nl_steps]
    nonlinear = {
        "what": "implicit time steps of the nonlinear FSI problem (Mooney-Rivlin solid, ALE Navier-Stokes with "
                "SUPG, Crank-Nicolson) from rest, exact Newton, each Newton system solved by the headline "
                "solver; Jacobians on every level by dual-number kernels",
        "workload": p.name + "-nonlinear", "force": NL_FORCE, "time_steps": NL_STEPS, "nl_rtol": NL_RTOL,
        "s_max": sum(nl_newton) / len(nl_newton), "N": sum(nl_its) / max(len(nl_its), 1),
        "rho": sum(nl_rho) / max(len(nl_rho), 1), "all_converged": all(st["converged"] for st in nl_steps),
        "ms_per_time_step": sum(nl_ms) / len(nl_ms),
        "ms_per_newton_step": {"jacobian": sum(st["jacobian_ms"] for st in nl_steps) / max(sum(nl_newton), 1),
                               "block_setup": sum(st["setup_ms"] for st in nl_steps) / max(sum(nl_newton), 1),
                               "solve": sum(st["solve_ms"] for st in nl_steps) / max(sum(nl_newton), 1)},
        "jacobian_all_levels_ms": min(jac_ms),
        # float64-pipe roofline of the assembly: float64 thread-instructions per
        # element counted by ncu on the 128^2 fine level (point + d/u/p seed
        # kernels, profiles/nl_jacobian_c4.md) x elements of all levels, over
        # the measured float64 FMA rate in instructions (half its flop rate)
        "jacobian_roofline": {
            "bound": "fp64", "inst_per_element": NL_JAC_INST_PER_ELEMENT,
            "achieved_ginst_s": NL_JAC_INST_PER_ELEMENT * n_el_all / (min(jac_ms) * 1e-3) / 1e9,
            "peak_ginst_s": fp64_peak / 2.0 if fp64_peak else None,
            "frac": (NL_JAC_INST_PER_ELEMENT * n_el_all / (min(jac_ms) * 1e-3) / 1e9 / (fp64_peak / 2.0)
                     if fp64_peak else None),
            "note": "includes the coarse-level inverse and the ELL refills of nl_jacobian"},
        "jacobian_elements_per_s": n_el_all / (min(jac_ms) * 1e-3),
        "newton_fine_dof_per_s": job_throughput(n * sum(nl_newton), sum(nl_ms), world),
        "setup_s": setup_nl_s,
        "steps": [{"newton": st["newton_steps"], "its": st["iterations"], "ms": round(st["ms"], 2)}
                  for st in nl_steps],
    }

    value = job_throughput(n, ms, world)
    if rank != 0:
        return
    cpu = cpu_baseline(args.config) if world == 1 else None
    traffic = ncu_traffic()
    # every leg in full, on a line of its own before the result line
    detail = {
        "detail": "legs of the bench run (the result line follows)",
        "mixed_half": {"ms_per_step": ms, "iterations": its_mixed, "rho": st_mixed.get("rho"),
                       "rel_residual": st_mixed.get("rel_residual"),
                       "solve_hbm": {"algorithmic_bytes": solve_bytes,
                                     "achieved_gbs": solve_bytes / (ms * 1e-3) / 1e9,
                                     "frac": solve_bytes / (ms * 1e-3) / 1e9 / peak}},
        "fp64": {"value": job_throughput(n, ms64, world), "ms_per_step": ms64, "iterations": its64,
                 "speedup_mixed_over_fp64": ms64 / ms},
        "mixed_f32_inverses": {"value": job_throughput(n, ms32, world), "ms_per_step": ms32, "iterations": its32},
        "as_smoother": {"what": "monolithic additive Schwarz (one block of all fields per pressure group), "
                                "the paper's comparison method; same cycle, mixed precision, float32 inverses "
                                "(FP16 storage does not converge for these blocks)",
                        "value": job_throughput(n, ms_as, world), "ms_per_step": ms_as,
                        "iterations": its_as, "converged": bool(st_as.get("converged")),
                        "rel_residual": st_as.get("rel_residual"), "setup_s": setup_as_s,
                        "fs_speedup_over_as": ms_as / ms},
        "additive": {"what": "the additive field-split smoother on every level (partition-of-unity weights, "
                             "owner-computes combination); mixed precision, FP16 inverses",
                     "value": job_throughput(n, ms_add, world), "ms_per_step": ms_add, "iterations": its_add,
                     "converged": bool(st_add.get("converged")), "setup_s": setup_add_s,
                     "mult_speedup_over_additive": ms_add / ms,
                     "smoother_fine": {"mean_launch_ms": sm_add_ms, "achieved_gbs": sm_add_gbs,
                                       "frac": sm_add_gbs / peak,
                                       "algorithmic_bytes_per_launch": prof_add["smoother_bytes"]}},
        "cascade": {"what": "swapped cascade (Sec. 5 future work): FGMRES preconditioned by the field split, "
                            "each field system by its own GMG V-cycle with the same smoothing",
                    "value": job_throughput(n, ms_casc, world), "ms_per_step": ms_casc, "iterations": its_casc,
                    "setup_s": setup_casc_s, "slowdown_vs_headline": ms_casc / ms},
        "batched": {"systems": len(batch), "unknowns_total": batch_dofs, "ms_per_batch": ms_batch,
                    "ms_per_batch_patch3": ms_batch_fixed,
                    "autotune": {"candidates": list(tune_cand), "chosen_by_n_fine": chosen_by_size,
                                 "tune_s": tune_s,
                                 "ell_lanes": {"candidates": [0, 1, 4], "chosen": lanes_chosen,
                                               "batch_ms": lanes_times, "tune_s": tune_layout_s,
                                               "note": "0 = size rule (1 lane per row inside a batch)"}},
                    "solves_per_s": job_throughput(len(batch), ms_batch, world),
                    "dof_per_s": job_throughput(batch_dofs, ms_batch, world),
                    "iterations_min_max": [min(t["iterations"] for t in bstats),
                                           max(t["iterations"] for t in bstats)],
                    "all_converged": all(t["converged"] for t in bstats), "setup_s": setup_batch_s,
                    "hbm": {"algorithmic_bytes": batch_bytes,
                            "achieved_gbs": batch_bytes / (ms_batch * 1e-3) / 1e9,
                            "frac": batch_bytes / (ms_batch * 1e-3) / 1e9 / peak,
                            "how": "sum over systems of its Arnoldi steps x (V-cycle + float64 outer product "
                                   "+ Gram-Schmidt bytes), fsi_get_cost; one graph launch for all systems"},
                    "workload": "64 seeded 2D channels, fine grids {32,48,64,96,128}^2, band width U[0.1,0.4]"},
        "valve3d": {"workload": p3.name, "unknowns": n3, "ms_per_solve": ms_3d,
                    "dof_per_s": job_throughput(n3, ms_3d, world), "iterations": its_3d,
                    "setup_s": {"hierarchy": setup_3d_hier_s, "smoothers": setup_3d_smooth_s,
                                "fine_inversion_ms": inv3_ms,
                                "fine_inversion_tflops": pf3["invert_flops"] / (inv3_ms * 1e-3) / 1e12,
                                "factor": "tf32_tensor_cores"},
                    "omega": p3.omega,
                    "smoother_fine": {"mean_launch_ms": sm3, "achieved_gbs": pr3["smoother_bytes"] / sm3 / 1e6,
                                      "frac": pr3["smoother_bytes"] / sm3 / 1e6 / peak}},
        "as_smoother_3d": {"what": "the paper's 3D FS-vs-AS comparison (Sec. 4.2) on the 32^3 valve box: monolithic "
                                   "AS blocks (~750 dofs) inverted by the split over the two field systems, "
                                   "float32 inverses; same cycle and Krylov solver",
                           "ms_per_solve": ms_as3, "iterations": its_as3, "converged": conv_as3,
                           "setup_s": setup_as3_s, "fs_ms_per_solve": ms_3d,
                           "fs_speedup_over_as": ms_as3 / ms_3d},
        "nonlinear": nonlinear,
        "adjoint": {"workload": pa.name, "unknowns": na, "ms_forward_plus_adjoint": ms_adj,
                    "iterations": astats, "dof_per_s": job_throughput(na, ms_adj, world)},
        "factorization": fact,
        "setup_s": {"hierarchy": setup_hier_s, "smoothers_mixed_half": setup_mixed_s,
                    "smoothers_mixed_f32": setup_f32_s, "smoothers_fp64": setup_fp64_s},
        "e2e_iterations": its_e2e,
        "kernels": {"sweep_fine": {"achieved_gbs": achieved, "frac": achieved / peak, "mean_sweep_ms": sm_ms,
                                   "algorithmic_bytes_per_sweep": prof["smoother_bytes"]},
                    "spmv_fine": {"achieved": spmv_gbs, "frac": spmv_gbs / peak, "mean_launch_ms": spmv_ms},
                    "restriction_fine": {"achieved": rst_gbs, "frac": rst_gbs / peak, "mean_launch_ms": rst_ms},
                    "prolongation_fine": {"achieved": pro_gbs, "frac": pro_gbs / peak, "mean_launch_ms": pro_ms},
                    "fp64_peak_gflops": {"measured": fp64_peak, "nominal": FP64_NOMINAL_GFLOPS,
                                         "how": "fsi_profile mode 3: 8 independent FMA chains per thread, "
                                                "8 CTAs x 256 threads per SM, best of 3 timed launches"},
                    "outer_spmv_f64": {"achieved_gbs": outer_gbs, "frac_hbm": outer_gbs / peak,
                                       "achieved_fp64_gflops": outer_gflops,
                                       "frac_fp64_measured": outer_gflops / fp64_peak if fp64_peak else None,
                                       "mean_launch_ms": outer_ms},
                    "gram_schmidt_f64": {"bound": "fp64 and hbm", "achieved_gflops": gs64_gflops,
                                         "frac_fp64_measured": (gs64_gflops / fp64_peak
                                                                if gs64_gflops and fp64_peak else None),
                                         "achieved_gbs": gs64_gbs,
                                         "frac_hbm": gs64_gbs / peak if gs64_gbs else None,
                                         # time the passes need at the slower of their two bounds
                                         # (float64 FMAs at the measured rate, bytes at the measured
                                         # copy bandwidth) over the time they take
                                         "frac_of_bound": gs64_bound_frac,
                                         "launches_timed": prof["gs64_launches"]},
                    "gram_schmidt_first_pass_f32": {"bound": "hbm", "achieved_gbs": gs1_gbs,
                                                    "frac": gs1_gbs / peak if gs1_gbs else None,
                                                    "launches_timed": prof["gs1_launches"]}},
        "cpu_baseline": cpu,
    }
    print(json.dumps(detail), flush=True)
    # the result line: short enough to survive a 1500-character log tail
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 cycle, f16 row-scaled inverses, f64 Krylov",
        "data": "synthetic (seeded)",
        "config": {"workload": p.name, "unknowns": n, "levels": p.n_levels, "vanka_group": p.patch,
                   "rtol": RTOL, "parallelism": f"replicas x{world}", "l2": "inputs > L2, no flush"},
        "iterations": its_mixed,
        "fp64": {"ms_per_step": round(ms64, 3), "its": its64["median"], "speedup_mixed": round(ms64 / ms, 3)},
        "additive": {"ms_per_step": round(ms_add, 3), "its": its_add["median"]},
        "cascade": {"ms_per_step": round(ms_casc, 3), "its": its_casc["median"]},
        "as": {"ms_per_step": round(ms_as, 3), "its": its_as["median"]},
        "fs_vs_as_3d": {"fs_ms": round(ms_3d, 2), "as_ms": round(ms_as3, 2), "as_its": its_as3["median"]},
        "nonlinear": {"ms_per_time_step": round(nonlinear["ms_per_time_step"], 1),
                      "s_max": nonlinear["s_max"], "N": round(nonlinear["N"], 2), "rho": round(nonlinear["rho"], 3),
                      "jacobian_ms": round(nonlinear["jacobian_all_levels_ms"], 2),
                      "jacobian_fp64_frac": (round(nonlinear["jacobian_roofline"]["frac"], 3)
                                             if nonlinear["jacobian_roofline"]["frac"] else None)},
        "e2e": {"value": job_throughput(n, ms_e2e, world), "unit": UNIT, "ms_per_step": round(ms_e2e, 3),
                "h2d_bytes_per_step": int(b_pin.numel() * 8), "d2h_bytes_per_step": int(x_pin.numel() * 8)},
        "roofline": {"bound": "hbm", "kernel": "fine-level sweep (12 apply + 11 residual passes, 2 streams)",
                     "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": traffic},
        "solve_hbm_frac": round(solve_bytes / (ms * 1e-3) / 1e9 / peak, 3),
        "batched": {"ms": round(ms_batch, 2), "hbm_frac": round(batch_bytes / (ms_batch * 1e-3) / 1e9 / peak, 3)},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
        "cpu_baseline": ({k: cpu[k] for k in ("value", "unit", "cores", "kind")} |
                         {"sample": "FP64 oracle, 3 its timed, projected; detail line has nproc"}
                         if cpu else None),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle as the reference arm: `steps` FGMRES iterations of the same
    workload, each a step (one V-cycle plus Arnoldi), timed after `warmup`
    untimed ones and an untimed set-up.  ms_per_step is the measured time of
    one iteration; the metric's value divides the unknowns by the projected
    time of the ORACLE_ITERATIONS[config] iterations a full solve needs."""
    if rank != 0:
        return
    from paper_1909_13201_gb300 import inputs as I
    p = I.make_config(args.config)
    res = oracle_sample(args.config, iters=1, steps=args.steps, warmup=args.warmup)
    n_it = ORACLE_ITERATIONS[args.config]
    t_it = statistics.mean(res["per_iteration_s"])
    c_it = statistics.mean(res["cpu_per_iteration_s"])
    value = res["n"] / (t_it * n_it)
    sample = (f"FP64 oracle (numpy/scipy); step = 1 FGMRES iteration, {args.steps} timed after an untimed "
              f"{res['setup_s']:.0f} s set-up; value projected to the {n_it} its a solve needs")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * 1e3,
        "step": "one FGMRES(30) iteration of the oracle",
        "projected": {"iterations_per_solve": n_it, "ms_per_solve": t_it * n_it * 1e3},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": p.name, "unknowns": res["n"], "levels": p.n_levels, "vanka_group": p.patch,
                   "rtol": RTOL, "parallelism": "cpu"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": round(c_it / t_it, 2), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(oracle_sample(args.config, args.sample_iters)), flush=True)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
