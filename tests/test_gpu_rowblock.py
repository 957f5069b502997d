"""Row-block sharding on one GPU.

Partial sketches: the sketch of rows [r0, r0 + n) of A with
ski_opts.row_offset = r0 draws the columns of S of those global rows (Def. 5),
so the partial sketches of a row split sum to the sketch of the whole A.

Row-block solve: ``ski_solve_rowblock`` on k virtual processes, each a host
thread with its own stream and workspace on this one GPU.  Their sums go
through a host-side all-reduce (each thread synchronises its stream, copies
its buffer to the host, meets the others at a barrier, and writes back the sum
taken in rank order), so no kernel of one virtual process ever waits on
another's.  The row-block solve must agree with the one-process solve of the
whole A and meet the acceptance test, with every virtual process holding the
same x and report.
"""
import threading

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hashing, lsqr as olsqr, sketch as osk
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _partial_oracle(seed, s, m, A, b, start, cnt):
    """S[:, start:start+cnt] [A_blk | b_blk] from the oracle's draw of the whole S."""
    n, d = A.shape
    idx, sgn = hashing.hash_table(seed, s, m, n)
    out = np.zeros((m, d + 1))
    for k in range(s):
        coef = sgn[start:start + cnt, k] / np.sqrt(s)
        np.add.at(out[:, :d], idx[start:start + cnt, k], coef[:, None] * A[start:start + cnt])
        np.add.at(out[:, d], idx[start:start + cnt, k], coef * b[start:start + cnt])
    return out


@pytest.mark.parametrize("s", [1, 3])
def test_partial_sketches_of_row_blocks_sum_to_the_sketch(s):
    torch, pkg = cuda()
    from paper_2105_11815_gb300 import sharded
    n, d, m, seed = 5003, 60, 180, 31
    A, b, _ = workloads.gaussian_lls(n, d, seed=2)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    total = torch.zeros(m, d + 1, dtype=torch.float64, device="cuda")
    for start, cnt in sharded.row_blocks(n, 3):
        o = pkg.ski_opts_default(m=m, s=s, seed=seed, row_offset=start)
        SA = torch.empty(m, d + 1, dtype=torch.float64, device="cuda")
        pkg.ski_sketch_hash(pkg.dense_matrix(At[start:start + cnt]), bt[start:start + cnt], o, SA, d + 1)
        assert rel_fro(SA.cpu().numpy(), _partial_oracle(seed, s, m, A, b, start, cnt)) <= 1e-12
        total += SA
    full = osk.sketch_rows(seed, s, m, A, b)
    assert rel_fro(total.cpu().numpy(), full) <= 1e-12
    # a row offset with the premix (which mixes every row) is refused
    o = pkg.ski_opts_default(m=m, s=s, seed=seed, row_offset=7, premix=1)
    with pytest.raises(pkg.SkiError):
        pkg.ski_sketch_hash(pkg.dense_matrix(At), bt, o, total, d + 1)


class ThreadSum:
    """All-reduce among k host threads on one GPU (see the module docstring)."""

    def __init__(self, k):
        self.k = k
        self.bar = threading.Barrier(k, timeout=120)
        self.slots = [None] * k

    def callback(self, rank):
        import torch
        from paper_2105_11815_gb300 import sharded

        def cb(ptr, count, dtype, stream):
            ext = torch.cuda.ExternalStream(int(stream))
            ext.synchronize()
            t = sharded._tensor_at(ptr, count, dtype, "cuda")
            self.slots[rank] = t.double().cpu()
            self.bar.wait()
            tot = self.slots[0].clone()
            for r in range(1, self.k):
                tot += self.slots[r]
            self.bar.wait()
            with torch.cuda.stream(ext):
                t.copy_(tot.to(device="cuda", dtype=t.dtype))
            ext.synchronize()
        return cb


def _run_rowblock(torch, pkg, mats, bs, opts, d, k):
    from paper_2105_11815_gb300 import sharded
    ts = ThreadSum(k)
    xs = [torch.empty(d, dtype=torch.float64, device="cuda") for _ in range(k)]
    infos, errs = [None] * k, []

    def run(r):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                infos[r] = sharded.solve_rowblock(mats[r][0], bs[r], mats[r][1], opts, xs[r],
                                                  allreduce=ts.callback(r), stream=st)
            st.synchronize()
        except Exception as e:  # surfaced below
            errs.append(e)
            ts.bar.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(k)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return xs, infos


@pytest.mark.parametrize("k,mixed", [(2, False), (3, False), (2, True)])
def test_rowblock_solve_matches_the_one_process_solve(k, mixed):
    torch, pkg = cuda()
    from paper_2105_11815_gb300 import sharded
    n, d = 12000, 150
    A, b, _ = workloads.gaussian_lls(n, d, seed=40 + k)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    opts = pkg.ski_opts_default(m=2 * d, s=2, seed=9, tol=1e-10, tau_r=1e-12, **prec)
    mats, bs = [], []
    for start, cnt in sharded.row_blocks(n, k):
        mats.append((pkg.dense_matrix(At[start:start + cnt]), start))
        bs.append(bt[start:start + cnt])
    xs, infos = _run_rowblock(torch, pkg, mats, bs, opts, d, k)
    x1 = torch.empty(d, dtype=torch.float64, device="cuda")
    i1 = pkg.ski_solve(pkg.dense_matrix(At), bt, opts, x1)
    for r in range(k):
        assert infos[r].status == 0
        assert torch.equal(xs[r], xs[0])                      # the same x on every process
        assert infos[r].iters == infos[0].iters and infos[r].metric == infos[0].metric
    x = xs[0].cpu().numpy()
    assert olsqr.residual_metric_dd(A, b, x) <= 1e-10
    assert rel_fro(x, x1.cpu().numpy()) <= 1e-9
    assert abs(infos[0].iters - i1.iters) <= 2


def test_rowblock_solve_of_a_csr_matrix():
    torch, pkg = cuda()
    from paper_2105_11815_gb300 import sharded
    n, d = 30000, 200
    rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=8, nnz_row=8, heavy_frac=1e-3, heavy_nnz=100)
    A = sp.csr_matrix((v, ci, rp), shape=(n, d))
    opts = pkg.ski_opts_default(m=2 * d, s=2, seed=4, tol=1e-10, tau_r=1e-12)
    mats, bs, keep = [], [], []
    for start, cnt in sharded.row_blocks(n, 2):
        blk = A[start:start + cnt]
        arrs = (to_dev(torch, blk.indptr.astype(np.int64)), to_dev(torch, blk.indices.astype(np.int32)),
                to_dev(torch, blk.data))
        keep.append(arrs)
        mats.append((pkg.csr_matrix(arrs[0], arrs[1], arrs[2], cnt, d), start))
        bs.append(to_dev(torch, b[start:start + cnt]))
    xs, infos = _run_rowblock(torch, pkg, mats, bs, opts, d, 2)
    assert infos[0].status == 0 and torch.equal(xs[0], xs[1])
    x = xs[0].cpu().numpy()
    assert olsqr.residual_metric_dd(A, b, x) <= 1e-10
    assert rel_fro(x, olsqr.lstsq_reference(A, b)) <= 1e-8
