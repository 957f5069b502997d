"""GPU parity of the whole solve (Algorithm 1) against the oracle.

Bar for every solve: ||A^T r|| / (||A||_F ||r||) <= 1e-10 recomputed by the
oracle in FP64 on the returned x, and x within 1e-8 (relative) of LAPACK's
least-squares solution (the solution's own conditioning allows no tighter
bound for kappa ~ 1e3 inputs at this residual).
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adjoint as oadj, lsqr as olsqr
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _solve(torch, pkg, A, b, check=True, **kw):
    At, bt = to_dev(torch, A), to_dev(torch, b)
    d = A.shape[1]
    o = pkg.ski_opts_default(tol=1e-10, tau_r=1e-12, **kw)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x, check=check)
    return x.cpu().numpy(), info


def _assert_solution(A, b, x, tol_x=1e-8):
    assert olsqr.residual_metric(A, b, x) <= 1e-10
    xr = olsqr.lstsq_reference(A, b)
    assert rel_fro(x, xr) <= tol_x


def test_config1_plain_fp64():
    # dense 4096 x 256, 1-hashing, m = 2d = 512, Householder QR, R-preconditioned LSQR
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(4096, 256, seed=20210525)
    x, info = _solve(torch, pkg, A, b, m=512, s=1, seed=1)
    assert info.status == 0 and info.rank == 256
    _assert_solution(A, b, x)
    # same algorithm step by step in the oracle: iteration counts agree
    xo, oinfo = olsqr.ski_lls(A, b, seed=1, s=1, m=512, tau_r=1e-12)
    assert abs(info.iters - oinfo["iters"]) <= 2 + info.restarts * 5
    # the library's own FP64 metric agrees with the oracle's up to summation order
    assert abs(info.metric - olsqr.residual_metric(A, b, x)) <= 0.05 * info.metric + 1e-15


@pytest.mark.parametrize("kind,s,gamma", [("gauss", 1, 2.0), ("gauss", 2, 1.5), ("coh", 1, 3.0), ("coh", 2, 4.0)])
def test_premix_solves(kind, s, gamma):
    torch, pkg = cuda()
    n, d = 12000, 300
    A, b = (workloads.dense_gaussian if kind == "gauss" else workloads.dense_high_coherence)(n, d, seed=s)
    x, info = _solve(torch, pkg, A, b, m=int(gamma * d), s=s, seed=3, premix=1, n_pad=16384)
    assert info.status == 0
    _assert_solution(A, b, x)


def test_csr_solve():
    torch, pkg = cuda()
    n, d = 60000, 400
    rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=6, nnz_row=8, heavy_frac=1e-3, heavy_nnz=200)
    A = sp.csr_matrix((v, ci, rp), shape=(n, d))
    keep = (to_dev(torch, rp), to_dev(torch, ci), to_dev(torch, v), to_dev(torch, b))
    M = pkg.csr_matrix(keep[0], keep[1], keep[2], n, d)
    o = pkg.ski_opts_default(m=2 * d, s=2, seed=4, tol=1e-10, tau_r=1e-12)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(M, keep[3], o, x)
    assert info.status == 0
    xn = x.cpu().numpy()
    assert olsqr.residual_metric(A, b, xn) <= 1e-10
    assert rel_fro(xn, olsqr.lstsq_reference(A, b)) <= 1e-8


@pytest.mark.parametrize("sd,qd", [(1, 1), (2, 1)])
def test_mixed_precision_solve(sd, qd):
    torch, pkg = cuda()
    A, b = workloads.usv(8000, 200, 1e6, seed=2)
    x, info = _solve(torch, pkg, A, b, m=400, s=1, seed=5, premix=1, sketch_dtype=sd, qr_dtype=qd)
    assert info.status == 0
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def test_square_one_hashing_loses_rank_exactly_on_collisions():
    # Example 1: with n = d and s = 1, SA = S A has full rank iff the d columns
    # of S land in distinct rows (probability prod_k (1 - k/m)); otherwise R is
    # singular and the solve reports it.
    from oracle import hashing
    torch, pkg = cuda()
    n = d = 8
    m = 64
    A, b, _ = workloads.gaussian_lls(n, d, seed=7, noise=1e-2)
    seen = set()
    for seed in range(12):
        x, info = _solve(torch, pkg, A, b, check=False, m=m, s=1, seed=seed)
        idx, _ = hashing.hash_table(seed, 1, m, n)
        distinct = np.unique(idx[:, 0]).size == n
        seen.add(distinct)
        assert info.status == (0 if distinct else pkg.STATUS.index("SKI_ESINGULAR"))
    assert seen == {False, True}


@pytest.mark.parametrize("n,d,m,s", [(50, 1, 1, 1), (40, 40, 40, 40), (100, 10, 10, 10), (33, 32, 64, 3)])
def test_edge_shapes(n, d, m, s):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n * d, noise=1e-2)
    x, info = _solve(torch, pkg, A, b, m=m, s=s, seed=2)
    assert info.status == 0
    if n == d:
        assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)
    else:
        _assert_solution(A, b, x, tol_x=1e-7)


def test_early_exit_on_consistent_system():
    torch, pkg = cuda()
    g = np.random.default_rng(0)
    A = g.standard_normal((2000, 50))
    b = A @ g.standard_normal(50)
    x, info = _solve(torch, pkg, A, b, m=100, s=1, seed=1, tau_a=1e-6)
    assert info.early_exit == 1 and info.iters == 0
    assert np.linalg.norm(A @ x - b) <= 1e-6


def test_error_statuses():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(500, 20, seed=1)
    Ad = A.copy()
    Ad[:, 7] = Ad[:, 3]
    _, info = _solve(torch, pkg, Ad, b, check=False, m=40, s=1, seed=1)
    assert info.status == pkg.STATUS.index("SKI_ESINGULAR")
    An = A.copy()
    An[17, 5] = np.nan
    _, info = _solve(torch, pkg, An, b, check=False, m=40, s=1, seed=1)
    assert info.status == pkg.STATUS.index("SKI_ENONFINITE")
    _, info = _solve(torch, pkg, A, b, check=False, m=40, s=1, seed=1, it_max=1)
    assert info.status == pkg.STATUS.index("SKI_ENOCONV")
    with pytest.raises(pkg.SkiError):
        _solve(torch, pkg, A, b, m=10, s=1, seed=1)   # m < d


def test_determinism():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(3000, 100, seed=3)
    x1, _ = _solve(torch, pkg, A, b, m=200, s=2, seed=8, premix=1)
    x2, _ = _solve(torch, pkg, A, b, m=200, s=2, seed=8, premix=1)
    assert np.array_equal(x1, x2)


def test_batched_matches_single():
    torch, pkg = cuda()
    shapes = workloads.ragged_batch(6, seed=9, n_lo=500, n_hi=3000, d_lo=8, d_hi=120)
    As, bs = [], []
    for i, (n, d) in enumerate(shapes):
        A, b, _ = workloads.gaussian_lls(n, d, seed=100 + i)
        As.append(A)
        bs.append(b)
    o = pkg.ski_opts_default(m=-2000, s=1, seed=50, tol=1e-10, tau_r=1e-12)
    At = [to_dev(torch, A) for A in As]
    bt = [to_dev(torch, b) for b in bs]
    xs = [torch.empty(A.shape[1], dtype=torch.float64, device="cuda") for A in As]
    infos = pkg.ski_solve_batched([pkg.dense_matrix(a) for a in At], bt, o, xs)
    for i, (A, b) in enumerate(zip(As, bs)):
        assert infos[i].status == 0
        _assert_solution(A, b, xs[i].cpu().numpy())
        oi = copy.copy(o)
        oi.m = 2 * A.shape[1]
        oi.seed = 50 + i
        xi = torch.empty(A.shape[1], dtype=torch.float64, device="cuda")
        pkg.ski_solve(pkg.dense_matrix(At[i]), bt[i], oi, xi)
        assert torch.equal(xi, xs[i])


def test_adjoint_matches_closed_form_and_finite_differences():
    torch, pkg = cuda()
    from paper_2105_11815_gb300.autograd import lstsq, make_opts
    g = np.random.default_rng(5)
    for trial in range(8):
        A = g.standard_normal((512, 32))
        b = g.standard_normal(512)
        c = g.standard_normal(32)
        At = to_dev(torch, A).requires_grad_(True)
        bt = to_dev(torch, b).requires_grad_(True)
        opts = make_opts(32, gamma=2.0, seed=trial)
        x = lstsq(At, bt, opts)
        L = (x * to_dev(torch, c)).sum()
        L.backward()
        xr = np.linalg.lstsq(A, b, rcond=None)[0]
        dA, db = oadj.lstsq_grad(A, b, xr, c)
        assert rel_fro(At.grad.cpu().numpy(), dA) <= 1e-9
        assert rel_fro(bt.grad.cpu().numpy(), db) <= 1e-9
        if trial < 2:
            EA, eb = g.standard_normal(A.shape), g.standard_normal(b.shape)
            h = 1e-6
            lp = c @ np.linalg.lstsq(A + h * EA, b + h * eb, rcond=None)[0]
            lm = c @ np.linalg.lstsq(A - h * EA, b - h * eb, rcond=None)[0]
            fd = (lp - lm) / (2 * h)
            an = float((At.grad.cpu().numpy() * EA).sum() + bt.grad.cpu().numpy() @ eb)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
