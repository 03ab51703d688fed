"""Host-side multi-rank logic of bench.py on CPU with gloo (world size 2)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
rank, world = bench.dist_init("gloo")
assert world == 2
m = bench.max_over_ranks(1.5 + rank)
bench.barrier()
g = bench.whole_job_glups(1000, 10, world, m)
print(json.dumps({{"rank": rank, "max": m, "glups": g}}))
"""


def _launch(code, port, world=2):
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_weak_scaling_gloo():
    outs = _launch(WORKER.format(root=ROOT), _free_port())
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert all(r["max"] == 2.5 for r in res)
    # 2 replicas x 1000 nodes x 10 steps / 2.5 s
    assert all(abs(r["glups"] - 2 * 1000 * 10 / 2.5 / 1e9) < 1e-18 for r in res)


REF = r"""
import sys
sys.path.insert(0, {root!r})
import bench
sys.exit(bench.main(["--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3",
                     "--workload", "parity", "--ref-rows", "16"]))
"""


def test_reference_arm_prints_on_rank0_only():
    outs = _launch(REF.format(root=ROOT), _free_port())
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["unit"] == "GLUPS" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
