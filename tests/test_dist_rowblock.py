"""Row-block sharding, run as world_size-2 gloo ranks on the CPU.

The library's row-block solve (``ski_solve_rowblock``) sums, over the
processes, the m x (d + 1) partial sketches once, and A^T t with ||t||^2 in
every LSQR iteration; ``paper_2105_11815_gb300.sharded.TorchAllreduce`` is the
callback that does each sum through torch.distributed.  Here, on the host:
  - the callback sums host buffers in place over two gloo ranks;
  - the row split covers every row once;
  - partial sketches of the two ranks' row blocks, each drawn from the columns
    of S of the block's global rows (Def. 5), sum through the callback to the
    sketch of the whole A (the oracle's S A);
  - LSQR run with those sums -- each rank's W^T u formed from its own rows and
    summed -- follows the single-process LSQR iterate by iterate.
The library's own row-block kernels are checked on the GPU
(tests/test_gpu_rowblock.py).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, %(root)r)
import numpy as np
import torch.distributed as dist
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
from paper_2105_11815_gb300 import SKI_F32, SKI_F64, sharded, workloads
from oracle import hashing, lsqr as olsqr, sketch as osk
ar = sharded.TorchAllreduce(device="cpu")
out = {"rank": rank}
# (1) the callback on host buffers: FP64 and FP32, summed in place
for dt, npdt in ((SKI_F64, np.float64), (SKI_F32, np.float32)):
    buf = (np.arange(7, dtype=npdt) + 1) * (rank + 1)
    ar(buf.ctypes.data, buf.size, dt, None)
    out["sum_%%d" %% dt] = buf.tolist()
# (2) partial sketches of the row blocks sum to the sketch of A
n, d, m, s, seed = 3001, 40, 120, 2, 77
A, b, _ = workloads.gaussian_lls(n, d, seed=5)
start, cnt = sharded.row_blocks(n, world)[rank]
idx, sgn = hashing.hash_table(seed, s, m, n)          # column j of S: global row j
part = np.zeros((m, d + 1))
for k in range(s):
    coef = sgn[start:start + cnt, k] / np.sqrt(s)
    np.add.at(part[:, :d], idx[start:start + cnt, k], coef[:, None] * A[start:start + cnt])
    np.add.at(part[:, d], idx[start:start + cnt, k], coef * b[start:start + cnt])
ar(part.ctypes.data, part.size, SKI_F64, None)
full = osk.sketch_rows(seed, s, m, A, b)
out["sketch_err"] = float(np.linalg.norm(part - full) / np.linalg.norm(full))
out["sketch_sum"] = float(part.sum())
# (3) LSQR with the row-block sums: W = A R^-1, each rank applies W^T to its rows
R = np.linalg.qr(full[:, :d], mode="r")
Ab = A[start:start + cnt]
def Wmul_local(v):
    return Ab @ np.linalg.solve(R, v)
def WTmul_sum(u_local):
    g = np.linalg.solve(R.T, Ab.T @ u_local)
    ar(g.ctypes.data, g.size, SKI_F64, None)
    return g
def norm_sum(u_local):
    t = np.array([u_local @ u_local])
    ar(t.ctypes.data, 1, SKI_F64, None)
    return float(np.sqrt(t[0]))
# LSQR written over the local slices of the n-vectors: every length-n inner
# product is a sum over the ranks, every length-d one is local
u = b[start:start + cnt].copy()
beta = norm_sum(u); u /= beta
v = WTmul_sum(u); alpha = np.linalg.norm(v); v /= alpha
w = v.copy(); phibar, rhobar = beta, alpha; y = np.zeros(d)
ys = []
for it in range(12):
    u = Wmul_local(v) - alpha * u
    beta = norm_sum(u); u /= beta
    v = WTmul_sum(u) - beta * v
    alpha = np.linalg.norm(v); v /= alpha
    rho = np.hypot(rhobar, beta); c, sn = rhobar / rho, beta / rho
    theta = sn * alpha; rhobar = -c * alpha; phi = c * phibar; phibar = sn * phibar
    y = y + (phi / rho) * w; w = v - (theta / rho) * w
    ys.append(y.copy())
ref = []
olsqr.lsqr(lambda z: A @ np.linalg.solve(R, z), lambda t: np.linalg.solve(R.T, A.T @ t), b, d, 0.0, 12,
           history=lambda k, yk, *rest: ref.append(yk))
out["lsqr_err"] = max(float(np.linalg.norm(a - r) / np.linalg.norm(r)) for a, r in zip(ys, ref))
out["y_last"] = ys[-1][:3].tolist()
print(json.dumps(out))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_row_blocks_cover_every_row_once():
    from paper_2105_11815_gb300 import sharded
    for n, world in ((10, 3), (3001, 2), (5, 8), (0, 2), (7, 1)):
        blocks = sharded.row_blocks(n, world)
        assert len(blocks) == world
        assert sum(c for _, c in blocks) == n
        assert all(blocks[k][0] + blocks[k][1] == blocks[k + 1][0] for k in range(world - 1))
        assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1


def test_two_gloo_ranks_row_block_sums():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD % {"root": ROOT}], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    res = sorted(outs, key=lambda j: j["rank"])
    for j in res:
        assert j["sum_0"] == [3.0 * (i + 1) for i in range(7)]        # 1x + 2x summed
        assert j["sum_1"] == [3.0 * (i + 1) for i in range(7)]
        assert j["sketch_err"] <= 1e-13
        assert j["lsqr_err"] <= 1e-10
    # every rank holds the same sums
    assert res[0]["sketch_sum"] == res[1]["sketch_sum"]
    assert res[0]["y_last"] == res[1]["y_last"]
