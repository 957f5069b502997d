"""Grouped Step 4 of the batched form (ski_opts.batch_lsqr = 1): the LSQR
iterations of all problems in flight run as one launch per kernel over
(problem, block) work items.  Each problem's kernels compute the same row
blocks in the same order as its own launches (batch_lsqr = 0), so x, R and the
iteration counts agree bit for bit; every solve also passes the acceptance
metric recomputed on the host.  CSR problems in the same batch keep their own
loop."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lsqr as olsqr
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, to_dev

pytestmark = pytest.mark.gpu


def _solve(torch, pkg, mats, bs, shapes, o):
    xs = [torch.empty(d, dtype=torch.float64, device="cuda") for _, d in shapes]
    infos = pkg.ski_solve_batched(mats, bs, o, xs)
    return [x.cpu().numpy() for x in xs], infos


@pytest.mark.parametrize("mixed,streams", [(False, 0), (True, 0), (False, 3)])
def test_grouped_lsqr_matches_each_problems_own_launches(mixed, streams):
    torch, pkg = cuda()
    shapes, As, bs = workloads.ragged_batch_torch(24, 777, "cuda")
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    mats = [pkg.dense_matrix(a) for a in As]
    base = dict(m=-2000, s=1, seed=31, tol=1e-10, tau_r=1e-12, streams=streams, **prec)
    xg, ig = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(batch_lsqr=1, **base))
    xo, io = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(batch_lsqr=0, **base))
    for i, (n, d) in enumerate(shapes):
        assert ig[i].status == 0 and io[i].status == 0, (i, ig[i].status, io[i].status)
        assert ig[i].iters == io[i].iters, (i, ig[i].iters, io[i].iters)
        assert np.array_equal(xg[i], xo[i]), i
        assert olsqr.residual_metric_dd(As[i].cpu().numpy(), bs[i].cpu().numpy(), xg[i]) <= 1e-10


def test_grouped_batch_with_csr_problems():
    torch, pkg = cuda()
    shapes, As, bs = workloads.ragged_batch_torch(6, 99, "cuda")
    mats = [pkg.dense_matrix(a) for a in As]
    keep, host = [], []
    for k in range(2):
        n, d = 6000 + 1000 * k, 80 + 40 * k
        rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=50 + k, nnz_row=8, heavy_frac=1e-3, heavy_nnz=40)
        arrs = (to_dev(torch, rp.astype(np.int64)), to_dev(torch, ci.astype(np.int32)), to_dev(torch, v))
        keep.append(arrs)
        mats.insert(2 * k + 1, pkg.csr_matrix(arrs[0], arrs[1], arrs[2], n, d))
        bs.insert(2 * k + 1, to_dev(torch, b))
        shapes.insert(2 * k + 1, (n, d))
        host.append((2 * k + 1, sp.csr_matrix((v, ci, rp), shape=(n, d)), b))
    base = dict(m=-2000, s=2, seed=8, tol=1e-10, tau_r=1e-12)
    xg, ig = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(batch_lsqr=1, **base))
    xo, io = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(batch_lsqr=0, **base))
    for i in range(len(mats)):
        assert ig[i].status == 0 and ig[i].iters == io[i].iters and np.array_equal(xg[i], xo[i]), i
    for i, A, b in host:
        assert olsqr.residual_metric_dd(A, b, xg[i]) <= 1e-10


def test_grouped_batch_across_every_pass_class():
    # d = 300, 800, 1500, 3000: the four register-blocked classes of the LSQR
    # pass (columns per thread 1, 2, 4 with twice the rows, 8 with prefetch)
    # in one group, against each problem's own launches
    torch, pkg = cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    shapes = [(9000, 300), (10000, 800), (12000, 1500), (14000, 3000)]
    As = [torch.randn(n, d, generator=g, device="cuda", dtype=torch.float64) for n, d in shapes]
    bs = [torch.randn(n, generator=g, device="cuda", dtype=torch.float64) for n, _ in shapes]
    mats = [pkg.dense_matrix(a) for a in As]
    base = dict(m=-2000, s=1, seed=3, tol=1e-10, tau_r=1e-12, streams=4)
    xg, ig = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(batch_lsqr=1, **base))
    xo, io = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(batch_lsqr=0, **base))
    for i in range(len(shapes)):
        assert ig[i].status == 0 and ig[i].iters == io[i].iters and np.array_equal(xg[i], xo[i]), i
        assert olsqr.residual_metric_dd(As[i].cpu().numpy(), bs[i].cpu().numpy(), xg[i]) <= 1e-10


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_with_gram_step2_matches_single_solves(mixed):
    # Step 2 from the Gram matrix in a batch (several problems in flight on
    # their streams): each problem's x, R factor choice and iteration count
    # equal its own ski_solve with the same options, bit for bit
    torch, pkg = cuda()
    shapes, As, bs = workloads.ragged_batch_torch(10, 4242, "cuda")
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    mats = [pkg.dense_matrix(a) for a in As]
    base = dict(s=1, tol=1e-10, tau_r=1e-12, factorization=2, **prec)
    # in a batch, m = -2000 gives each problem m = 2 d, and problem i draws
    # its sketch with seed + i; a single solve takes both itself
    xb, ib = _solve(torch, pkg, mats, bs, shapes, pkg.ski_opts_default(m=-2000, seed=5, streams=4, **base))
    for i, (n, d) in enumerate(shapes):
        x = torch.empty(d, dtype=torch.float64, device="cuda")
        info = pkg.ski_solve(mats[i], bs[i], pkg.ski_opts_default(m=2 * d, seed=5 + i, **base), x)
        assert ib[i].status == 0 and info.status == 0, (i, ib[i].status, info.status)
        assert ib[i].gram == info.gram == 1, (i, ib[i].gram, info.gram)
        assert ib[i].iters == info.iters, (i, ib[i].iters, info.iters)
        assert np.array_equal(xb[i], x.cpu().numpy()), i
        assert olsqr.residual_metric_dd(As[i].cpu().numpy(), bs[i].cpu().numpy(), xb[i]) <= 1e-10
