"""The multi-rank path of bench.py (independent replicas, one process per
GPU) with the gloo backend on CPU, world size 2: barrier, max-over-ranks
timing, weak-scaling aggregation, distinct member seeds, and the reference
arm's rank-0-only output."""
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
import json, os, sys
sys.path.insert(0, %(root)r)
from paper_2603_25282_gb300.replicas import Replicas
rep = Replicas("gloo")
rep.barrier()
local_time = 1.0 + rep.rank          # rank 1 is the slow one
t = rep.max_over_ranks(local_time)
v = rep.weak_throughput(100, t)
seeds = [rep.member_seed(m) for m in range(3)]
print(json.dumps({"rank": rep.rank, "world": rep.world, "t": t, "v": v, "seeds": seeds}))
rep.close()
"""


def _launch(nproc, code_or_args, script=True):
    port = _free_port()
    procs = []
    for r in range(nproc):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(nproc), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        cmd = [sys.executable, "-c", code_or_args] if script else [sys.executable] + code_or_args
        procs.append(subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        outs.append((p.returncode, o, e))
    return outs


def test_two_gloo_ranks_max_timing_and_weak_aggregate():
    outs = _launch(2, WORKER % {"root": ROOT})
    res = []
    for rc, o, e in outs:
        assert rc == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    for r in res:
        assert r["world"] == 2
        assert r["t"] == 2.0                 # max over ranks
        assert r["v"] == 2 * 100 / 2.0       # whole-job units per second
    assert set(res[0]["seeds"]).isdisjoint(res[1]["seeds"])


@pytest.mark.slow
def test_reference_arm_prints_on_rank_zero_only():
    args = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
            "--workload", "2d512_ts4_f32"]
    outs = _launch(2, args, script=False)
    lines = []
    for rc, o, e in outs:
        assert rc == 0, e
        lines.append([l for l in o.splitlines() if l.startswith("{")])
    assert len(lines[0]) == 1 and len(lines[1]) == 0
    d = json.loads(lines[0][0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints
    one JSON line with the keys the bench contract names."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["warmup"] >= 3 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
