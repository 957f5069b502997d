"""The autotuner on the GPU: it times candidate launch parameters on a small
ragged batch, returns valid options, caches them, and the batch solved with
the tuned options meets the tolerance."""
import numpy as np
import pytest

from paper_2105_11815_gb300 import autotune, workloads
from gpu_util import cuda

pytestmark = pytest.mark.gpu


def test_tune_batched_on_a_ragged_batch(tmp_path):
    torch, pkg = cuda()
    shapes, As, bs = workloads.ragged_batch_torch(6, 11, "cuda", n_hi=9000, d_hi=200)
    mats = [pkg.dense_matrix(a) for a in As]
    xs = [torch.empty(d, dtype=torch.float64, device="cuda") for _, d in shapes]
    o = pkg.ski_opts_default(m=-2000, s=1, seed=3, tol=1e-10, tau_r=1e-10)
    space = {"lsqr_pass": (1, 2, 3), "lsqr_ctas": (0, 304), "graphs": (0, 1), "streams": (8, 2)}
    path = str(tmp_path / "tune.json")
    ot, rec = autotune.tune_batched(mats, bs, xs, o, cache_path=path, sample=4, reps=1, rounds=1, space=space)
    assert not rec["cached"] and rec["trials"] >= 6 and np.isfinite(rec["seconds"])
    for f, v in rec["config"].items():
        assert v in space[f] and getattr(ot, f) == v
    infos = pkg.ski_solve_batched(mats, bs, ot, xs)
    assert all(i.status == 0 and i.metric <= 1e-10 for i in infos)
    ot2, rec2 = autotune.tune_batched(mats, bs, xs, o, cache_path=path, sample=4, reps=1, rounds=1, space=space)
    assert rec2["cached"] and rec2["config"] == rec["config"]
