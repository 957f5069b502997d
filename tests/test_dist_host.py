"""The multi-rank host logic of bench.py (replicas: one process per GPU, a
barrier and the max over ranks of the timings; no collective on the data
path), run as world_size-2 gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, %(root)r)
import bench
rank, world, local = bench.dist_init(2, backend="gloo")
assert (world, local) == (2, rank)
bench.barrier(world)
t = bench.max_over_ranks(1.5 * (rank + 1), world)           # per-rank times 1.5, 3.0
units = world * 100 / (t * 1e-3)                              # weak scaling: all ranks' units / max time
print(json.dumps({"rank": rank, "max": t, "value": units}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_barrier_and_max():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD % {"root": ROOT}], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(out.strip().splitlines()[-1])
    import json
    res = sorted((json.loads(o) for o in outs), key=lambda j: j["rank"])
    assert [r["max"] for r in res] == [3.0, 3.0]                 # every rank sees the slowest rank's time
    assert res[0]["value"] == res[1]["value"] == pytest.approx(2 * 100 / 3e-3)


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_init(1) == (0, 1, 0)
    assert bench.max_over_ranks(2.5, 1) == 2.5
    bench.barrier(1)


@pytest.mark.parametrize("workload", ["dense_4096x256_s1_m512", "csr_1000000x20000_s2_g2", "batched_256_ragged_g2"])
def test_reference_arm_runs_on_rank_zero_only(workload):
    # under torchrun the oracle arm is rank 0's alone: the other ranks exit 0
    # at once, without joining a process group or doing work
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--workload", workload], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_reference_arm_line_keeps_the_bench_contract():
    # the oracle arm on the small dense workload (CPU only): one JSON line with
    # every key of the benchmark line contract, its value equal to its own cpu_baseline and e2e
    import json
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "dense_4096x256_s1_m512", "--steps", "2", "--warmup", "1"], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in j, k
    assert j["impl"] == "reference" and j["steps"] == 2 and j["value"] > 0
    assert j["config"]["workload"] == "dense_4096x256_s1_m512"
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["value"] == j["value"]
    assert j["e2e"]["value"] == j["value"] and j["e2e"]["h2d_bytes_per_step"] == 0
