"""GPU parity of the s-hashing variant T (Def. 7) against the oracle.

The variant draws the s rows of each column with replacement, so one row of A
can be listed twice in one bucket of the library's gather (same row, same or
opposite sign).  Small m makes that frequent; s > m makes it certain.

Tolerances as for s-hashing: draws bit-exact; FP64 sketch <= 1e-12 relative
Frobenius; FP32 <= 1e-5; solves reach ||A^T r|| / (||A||_F ||r||) <= 1e-10
recomputed by the oracle and x within 1e-8 of LAPACK's solution.
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hashing, lsqr as olsqr, sketch as osk, wht as owht
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,s,m,n", [(1, 1, 512, 4096), (2, 3, 4, 10001), (3, 5, 3, 777), (4, 8, 9, 3000),
                                        (5, 2, 40000, 1_000_003), (6, 64, 100, 50)])
def test_variant_draws_bit_exact(seed, s, m, n):
    torch, pkg = cuda()
    idx = torch.empty(n * s, dtype=torch.int32, device="cuda")
    sg = torch.empty(n * s, dtype=torch.int8, device="cuda")
    pkg.ski_hash_variant_indices(seed, s, m, n, idx, sg)
    ri, rs = hashing.variant_table(seed, s, m, n)
    assert np.array_equal(idx.cpu().numpy().reshape(n, s), ri)
    assert np.array_equal(sg.cpu().numpy().reshape(n, s), rs)


def _sketch(torch, pkg, A, b, **kw):
    n, d = A.shape
    o = pkg.ski_opts_default(hash_kind=pkg.SKI_S_HASHING_VARIANT, **kw)
    dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[o.sketch_dtype]
    ncols = d + (b is not None)
    ld = ncols + 3
    SA = torch.full((o.m, ld), float("nan"), dtype=dt, device="cuda")
    pkg.ski_sketch_hash(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b) if b is not None else None, o, SA, ld)
    return SA[:, :ncols].double().cpu().numpy()


@pytest.mark.parametrize("n,d,m,s", [(4096, 256, 512, 1), (3001, 37, 4, 3), (5000, 300, 310, 2), (2000, 40, 3, 5),
                                     (1, 5, 5, 2), (700, 9, 64, 64)])
def test_dense_variant_sketch_fp64(n, d, m, s):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n + d)
    got = _sketch(torch, pkg, A, b, m=m, s=s, seed=11)
    want = osk.sketch_rows(11, s, m, A, b, variant=True)
    assert rel_fro(got, want) <= 1e-12
    # the canonical bucket order makes repeated entries reproducible bit for bit
    assert np.array_equal(got, _sketch(torch, pkg, A, b, m=m, s=s, seed=11))


def test_dense_variant_sketch_equals_explicit_T_times_A():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(600, 12, seed=2)
    T = osk.s_hashing_variant_matrix(5, 3, 8, 600)
    got = _sketch(torch, pkg, A, b, m=8, s=3, seed=5)
    assert rel_fro(got, np.column_stack([T @ A, T @ b])) <= 1e-12


def test_dense_variant_sketch_fp32():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(5000, 70, seed=3)
    got = _sketch(torch, pkg, A, b, m=150, s=3, seed=3, sketch_dtype=pkg.SKI_F32)
    assert rel_fro(got, osk.sketch_rows(3, 3, 150, A, b, variant=True)) <= 1e-5


@pytest.mark.parametrize("m,s", [(600, 2), (6, 4)])
def test_csr_variant_sketch_fp64(m, s):
    torch, pkg = cuda()
    rp, ci, v, b = workloads.csr_heavy_rows(20000, 300, seed=4, nnz_row=8, heavy_frac=0.002, heavy_nnz=200)
    A = sp.csr_matrix((v, ci, rp), shape=(20000, 300))
    o = pkg.ski_opts_default(m=m, s=s, seed=13, hash_kind=pkg.SKI_S_HASHING_VARIANT)
    SA = torch.empty(m, 301, dtype=torch.float64, device="cuda")
    keep = (to_dev(torch, rp), to_dev(torch, ci), to_dev(torch, v), to_dev(torch, b))
    pkg.ski_sketch_hash(pkg.csr_matrix(keep[0], keep[1], keep[2], 20000, 300), keep[3], o, SA, 301)
    assert rel_fro(SA.cpu().numpy(), osk.sketch_rows(13, s, m, A, b, variant=True)) <= 1e-12


@pytest.mark.parametrize("s,m,slab", [(2, 120, 0), (3, 40, 0), (2, 120, 32)])
def test_hrht_variant_sketch_fp64(s, m, slab):
    torch, pkg = cuda()
    A, b = workloads.dense_high_coherence(5000, 50, seed=3)
    got = _sketch(torch, pkg, A, b, m=m, s=s, seed=21, premix=1, n_pad=8192, premix_slab=slab)
    want = owht.hrht_sketch(21, s, m, A, b, 8192, variant=True)
    assert rel_fro(got, want) <= 1e-12


def _solve(torch, pkg, A, b, **kw):
    o = pkg.ski_opts_default(tol=1e-10, tau_r=1e-12, hash_kind=pkg.SKI_S_HASHING_VARIANT, **kw)
    x = torch.empty(A.shape[1], dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, x)
    return x.cpu().numpy(), info


@pytest.mark.parametrize("s,premix,mixed", [(3, 0, 0), (2, 1, 0), (2, 1, 1)])
def test_variant_solve(s, premix, mixed):
    torch, pkg = cuda()
    n, d, m = 12000, 300, 600
    A, b = workloads.dense_high_coherence(n, d, seed=s) if premix else workloads.dense_gaussian(n, d, seed=s)
    kw = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    x, info = _solve(torch, pkg, A, b, m=m, s=s, seed=9, premix=premix, n_pad=16384 if premix else 0, **kw)
    assert info.status == 0 and info.rank == d
    assert olsqr.residual_metric(A, b, x) <= 1e-10
    assert rel_fro(x, olsqr.lstsq_reference(A, b)) <= 1e-8
    if not mixed:
        # same steps in the oracle with the same T: iteration counts agree
        _, oinfo = olsqr.ski_lls(A, b, seed=9, s=s, m=m, premix=bool(premix), n_pad=16384 if premix else None,
                                 tau_r=1e-12, variant=True)
        assert abs(info.iters - oinfo["iters"]) <= 2 + info.restarts * 5


def test_variant_batched_matches_single():
    torch, pkg = cuda()
    shapes = workloads.ragged_batch(5, seed=4, n_lo=500, n_hi=3000, d_lo=8, d_hi=120)
    As, bs = zip(*[workloads.gaussian_lls(n, d, seed=200 + i)[:2] for i, (n, d) in enumerate(shapes)])
    At = [to_dev(torch, A) for A in As]
    bt = [to_dev(torch, b) for b in bs]
    o = pkg.ski_opts_default(m=-2000, s=2, seed=60, tol=1e-10, tau_r=1e-12, hash_kind=pkg.SKI_S_HASHING_VARIANT)
    xs = [torch.empty(A.shape[1], dtype=torch.float64, device="cuda") for A in As]
    infos = pkg.ski_solve_batched([pkg.dense_matrix(a) for a in At], bt, o, xs)
    for i, A in enumerate(As):
        assert infos[i].status == 0
        assert olsqr.residual_metric(A, bs[i], xs[i].cpu().numpy()) <= 1e-10
        oi = copy.copy(o)
        oi.m, oi.seed = 2 * A.shape[1], 60 + i
        xi = torch.empty(A.shape[1], dtype=torch.float64, device="cuda")
        pkg.ski_solve(pkg.dense_matrix(At[i]), bt[i], oi, xi)
        assert torch.equal(xi, xs[i])
