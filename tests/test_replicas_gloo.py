"""The multi-process path on CPU: two ranks over `gloo`, launched the way
bench.py is launched for N > 1 (torch.distributed.run, one process per rank,
rendezvous on 127.0.0.1).

The solve does not shard: with N ranks every rank solves its own replica of
the workload, the ranks exchange nothing but the timing barrier and the max
of their step times, and the job's throughput is N x the per-rank units over
the slowest rank's time (weak scaling).  These tests cover that host logic:
rank discovery from the launcher's environment, the barrier and max
reduction, the aggregation, identical replicas on every rank (the host-side
set-up of the C library is deterministic across processes), and that only
rank 0 prints a result line while the other ranks exit 0.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

from paper_1909_13201_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = textwrap.dedent("""
    import hashlib, json, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch.distributed as dist
    import bench
    from paper_1909_13201_gb300 import binding
    from paper_1909_13201_gb300 import inputs as I

    rank, world, local = bench.dist_env()
    assert (world, local) == (2, rank), (rank, world, local)
    dist.init_process_group("gloo")
    bench.barrier(world)
    # each rank reports a different step time; every rank must see the max
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    # each rank builds its own replica (host-side structure of the library)
    p = I.make_config(0)
    s = binding.FSISolver(p, host_only=True)
    h = hashlib.sha256()
    for l in range(p.n_levels):
        for a in s.dof_map(l) + s.pattern(l):
            h.update(np.ascontiguousarray(a).tobytes())
        if l >= 1:
            for a in s.blocks(l):
                h.update(np.ascontiguousarray(a).tobytes())
    n = s.sizes(p.n_levels - 1)["n"]
    digests = [None] * world
    dist.all_gather_object(digests, h.hexdigest())
    bench.barrier(world)
    if rank == 0:
        print(json.dumps({{"ms": ms, "n": n, "digests": digests,
                          "value": bench.job_throughput(n, ms, world)}}), flush=True)
    dist.destroy_process_group()
""")


def free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def torchrun(args, tmp_env=None, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    env.update(tmp_env or {})
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_job_throughput_is_weak_scaling():
    import bench
    assert bench.job_throughput(1000, 2.0, 1) == pytest.approx(5e5)
    assert bench.job_throughput(1000, 2.0, 4) == pytest.approx(2e6)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_two_gloo_ranks_barrier_max_and_identical_replicas(tmp_path):
    binding.load_library(build_if_missing=True)     # build once, before the ranks load it
    script = tmp_path / "replica_worker.py"
    script.write_text(WORKER.format(root=ROOT))
    out = torchrun([str(script)])
    assert out.returncode == 0, out.stderr[-3000:]
    lines = json_lines(out.stdout)
    assert len(lines) == 1, out.stdout
    r = lines[0]
    assert r["ms"] == 15.0                            # the slower rank's time, seen by rank 0
    assert len(r["digests"]) == 2 and r["digests"][0] == r["digests"][1]
    assert r["value"] == pytest.approx(2 * r["n"] / 15e-3)


def test_reference_arm_two_ranks_rank0_prints_once():
    out = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--config", "0",
                    "--steps", "2", "--warmup", "1"])
    assert out.returncode == 0, out.stderr[-3000:]
    lines = json_lines(out.stdout)
    assert len(lines) == 1, out.stdout
    r = lines[0]
    assert r["impl"] == "reference" and r["n_gpus"] == 2 and r["steps"] == 2 and r["warmup"] == 1
    assert r["value"] > 0 and r["higher_is_better"] is True
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["value"] == r["value"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
