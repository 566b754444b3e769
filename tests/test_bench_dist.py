"""The benchmark's multi-rank host logic on CPU: world size 2 over gloo.

Replicas only (a single factorization does not shard), so the ranks meet
only to take the max of the timed region; the aggregate counts every
replica's flops.  The reference arm prints from rank 0 alone.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group(backend="gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms = 100.0 + 50.0 * rank            # rank 1 is the slow replica
m = bench.max_over_ranks(ms, world, "cpu")
v = bench.aggregate_gflops(1e9, m, world)
with open(os.path.join({out!r}, "rank%d.json" % rank), "w") as f:   # one file per rank: no interleaving
    json.dump({{"rank": rank, "max": m, "value": v}}, f)
dist.destroy_process_group()
"""


def _torchrun(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update({"OMP_NUM_THREADS": "1"})
    if env_extra:
        env.update(env_extra)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(29500 + os.getpid() % 1000)] + args
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, env=env, cwd=ROOT)


def test_max_over_ranks_and_aggregate_gloo(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, out=str(tmp_path)))
    r = _torchrun([str(script)])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / ("rank%d.json" % k)).read_text()) for k in range(2)]
    assert [l["rank"] for l in lines] == [0, 1]
    for l in lines:
        assert l["max"] == 150.0
        assert l["value"] == pytest.approx(2 * 1e9 / 0.150 / 1e9)


def test_reference_arm_prints_once_under_two_ranks():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                   "--ref-n", "96"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
