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
    assert info.inv_dtype == pkg.SKI_F32 and info.qr_fallback == 0   # small diagonal ratio: R^{-1} in FP32
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


def _orthogonal_rows(n, d, seed):
    return np.linalg.qr(np.random.default_rng(seed).standard_normal((n, d)))[0]


def _rhs_with_orthogonal_residual(A, seed, Q=None):
    # b = A x_true + e, e orthogonal to range(A) (spanned by the orthonormal Q):
    # x stays O(1), so the FP64 metric's rounding floor u ||A|| ||x|| / ||r||
    # is far below 1e-10
    g = np.random.default_rng(seed)
    Q = np.linalg.qr(A)[0] if Q is None else Q
    e = g.standard_normal(A.shape[0])
    e -= Q @ (Q.T @ e)
    return A @ g.standard_normal(A.shape[1]) + e


def test_fp64_factor_inverse_precision_follows_the_diagonal_ratio():
    # kappa = 1e9: the FP64 factor's diagonal ratio is far above 2^19, so R^{-1}
    # is formed in FP64 from the start
    torch, pkg = cuda()
    A, _ = workloads.usv(4000, 200, 1e9, seed=9)
    b = _rhs_with_orthogonal_residual(A, 4)
    x, info = _solve(torch, pkg, A, b, m=400, s=1, seed=2)
    assert info.status == 0 and info.qr_fallback == 0
    assert info.rdiag_ratio > 2 ** 19 and info.inv_dtype == pkg.SKI_F64
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def kahan_problem(n=4000, d=100, c=0.2, seed=5):
    """A = Q0 K, K the d x d Kahan matrix diag(s^i) (I - c U) with s^2 + c^2 = 1
    and U the strictly upper ones: diagonal ratio s^-(d-1), about 7.5, while
    kappa(K) is about 2e9 -- the diagonal understates kappa by 8 orders.
    b = A x_true + e with e orthogonal to range(Q0)."""
    K = np.diag(np.sqrt(1 - c * c) ** np.arange(d)) @ (np.eye(d) - c * np.triu(np.ones((d, d)), 1))
    Q0 = _orthogonal_rows(n, d, seed)
    A = Q0 @ K
    return A, _rhs_with_orthogonal_residual(A, seed + 1, Q0)


def test_fp64_factor_with_a_misleading_diagonal_still_meets_the_tolerance():
    # The diagonal ratio admits an FP32 inverse, but K's inverse in FP32 is off
    # by more than its own size (||K X - I|| ~ 10), so it cannot precondition.
    # The LSQR budget then sends the solve to the FP64 inverse (qr_fallback = 3)
    # and the solve meets the tolerance.  The report stays consistent: an FP32
    # inverse at the end means no fallback happened.
    torch, pkg = cuda()
    A, b = kahan_problem()
    x, info = _solve(torch, pkg, A, b, m=200, s=1, seed=3)
    assert info.status == 0, (info.status, info.iters, info.qr_fallback)
    assert info.rdiag_ratio < 2 ** 19
    assert info.qr_fallback in (0, 3)
    assert (info.qr_fallback == 3) == (info.inv_dtype == pkg.SKI_F64), (info.qr_fallback, info.inv_dtype)
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def test_mixed_budget_grows_as_the_sketch_shrinks():
    # m = 1.2 d: the larger distortion of the smaller sketch raises the LSQR
    # iteration count for the FP64 and the FP32 factor alike.  The mixed
    # form's budget follows Theorem 10's bound with eps = sqrt(d / m), so the
    # FP32 factor is kept where a fixed 150 iterations would have refactored
    torch, pkg = cuda()
    n, d = 20000, 400
    A, b = workloads.dense_gaussian(n, d, seed=12)
    kw = dict(m=480, s=1, seed=5, premix=1, n_pad=32768)
    x64, i64 = _solve(torch, pkg, A, b, **kw)
    xm, im = _solve(torch, pkg, A, b, sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32, **kw)
    assert i64.status == 0 and im.status == 0
    assert i64.iters > 150
    assert im.qr_fallback == 0, (im.iters, i64.iters)
    assert abs(im.iters - i64.iters) <= 0.1 * i64.iters + 5
    _assert_solution(A, b, xm)
    _assert_solution(A, b, x64)


def test_bf16_sketch_factor_kept_only_when_well_conditioned():
    # A BF16 sketch carries 2^-9 rounding: its FP32 factor preconditions a
    # well-conditioned A (kept) but not kappa = 1e6, where the diagonal ratio
    # sends Steps 1-2 to FP64 at once (qr_fallback = 1) instead of after the
    # LSQR budget (2).  Both solves meet the tolerance.
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(6000, 100, seed=3)
    x, info = _solve(torch, pkg, A, b, m=300, s=1, seed=5, premix=1, sketch_dtype=2, qr_dtype=1)
    assert info.status == 0 and info.qr_fallback == 0
    assert olsqr.residual_metric(A, b, x) <= 1e-10
    A, b = workloads.usv(8000, 200, 1e6, seed=2)
    x, info = _solve(torch, pkg, A, b, m=400, s=1, seed=5, premix=1, sketch_dtype=2, qr_dtype=1)
    assert info.status == 0 and info.qr_fallback == 1 and info.rdiag_ratio > 32
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


def test_widest_dense_problem():
    # d = 8192, the widest dense A the LSQR pass takes (8 x 2 columns per
    # thread of 512); mixed precision keeps the factorisation short
    torch, pkg = cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(8192)
    n, d = 20000, 8192
    At = torch.randn(n, d, generator=g, device="cuda", dtype=torch.float64)
    bt = torch.randn(n, generator=g, device="cuda", dtype=torch.float64)
    o = pkg.ski_opts_default(m=2 * d, s=1, seed=4, tol=1e-10, tau_r=1e-12, sketch_dtype=pkg.SKI_F32,
                             qr_dtype=pkg.SKI_F32)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x)
    assert info.status == 0
    A, b = At.cpu().numpy(), bt.cpu().numpy()
    assert olsqr.residual_metric(A, b, x.cpu().numpy()) <= 1e-10


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
    # results do not depend on the number of problems in flight
    for w in (1, 3, 6):
        ow = copy.copy(o)
        ow.streams = w
        xw = [torch.empty(A.shape[1], dtype=torch.float64, device="cuda") for A in As]
        iw = pkg.ski_solve_batched([pkg.dense_matrix(a) for a in At], bt, ow, xw)
        for i in range(len(As)):
            assert iw[i].status == 0 and iw[i].iters == infos[i].iters
            assert torch.equal(xw[i], xs[i])


@pytest.mark.parametrize("mixed", [False, True])
def test_batched_concurrent_runs_are_identical(mixed):
    # many problems in flight on few streams, repeated: every run must give the
    # same bits (a cross-CTA race on the LSQR scalars once showed up only here;
    # the mixed form runs the FP32 cluster panels and tensor-core GEMMs of
    # several problems at once)
    torch, pkg = cuda()
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    shapes = workloads.ragged_batch(12, seed=19, n_lo=600, n_hi=4000, d_lo=8, d_hi=150)
    At, bt = [], []
    for i, (n, d) in enumerate(shapes):
        A, b, _ = workloads.gaussian_lls(n, d, seed=400 + i)
        At.append(to_dev(torch, A))
        bt.append(to_dev(torch, b))
    mats = [pkg.dense_matrix(a) for a in At]
    ref = None
    for rep in range(8):
        o = pkg.ski_opts_default(m=-2000, s=1, seed=70, tol=1e-10, tau_r=1e-12, streams=(3 if rep % 2 else 5),
                                 **prec)
        xs = [torch.empty(d, dtype=torch.float64, device="cuda") for _, d in shapes]
        infos = pkg.ski_solve_batched(mats, bt, o, xs)
        got = ([x.clone() for x in xs], [i.iters for i in infos])
        if ref is None:
            ref = got
        assert got[1] == ref[1]
        assert all(torch.equal(a, b) for a, b in zip(got[0], ref[0]))


def test_batched_stream_ordering():
    # the batch reads b written by work queued on the caller's stream just
    # before, and the caller's stream sees x after the call
    torch, pkg = cuda()
    As, bs = [], []
    for i in range(5):
        A, b, _ = workloads.gaussian_lls(2000 + 300 * i, 40 + 10 * i, seed=300 + i)
        As.append(A)
        bs.append(b)
    At = [to_dev(torch, A) for A in As]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        bt = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for b in bs]
        torch.cuda._sleep(50_000_000)
        for t, b in zip(bt, bs):
            t.copy_(to_dev(torch, b), non_blocking=True)
        o = pkg.ski_opts_default(m=-2000, s=1, seed=7, tol=1e-10, tau_r=1e-12, streams=4)
        xs = [torch.empty(A.shape[1], dtype=torch.float64, device="cuda") for A in As]
        infos = pkg.ski_solve_batched([pkg.dense_matrix(a) for a in At], bt, o, xs, stream=side)
        ys = [x * 1.0 for x in xs]
    side.synchronize()
    for i, (A, b) in enumerate(zip(As, bs)):
        assert infos[i].status == 0
        _assert_solution(A, b, ys[i].cpu().numpy())


def test_adjoint_batched_matches_single():
    torch, pkg = cuda()
    g = np.random.default_rng(17)
    shapes = [(700, 20), (1500, 64), (512, 32), (2400, 90), (900, 8)]
    At, bt, xs, Rs, gs = [], [], [], [], []
    o = pkg.ski_opts_default(m=-2000, s=1, seed=3, tol=1e-10, tau_r=1e-13, streams=3)
    for i, (n, d) in enumerate(shapes):
        A = g.standard_normal((n, d))
        b = g.standard_normal(n)
        At.append(to_dev(torch, A))
        bt.append(to_dev(torch, b))
        xs.append(torch.empty(d, dtype=torch.float64, device="cuda"))
        Rs.append(torch.empty(d, d, dtype=torch.float64, device="cuda"))
        gs.append(to_dev(torch, g.standard_normal(d)))
    mats = [pkg.dense_matrix(a) for a in At]
    pkg.ski_solve_batched(mats, bt, o, xs, R_outs=Rs)
    dAs = [torch.empty_like(a) for a in At]
    dbs = [torch.empty_like(b) for b in bt]
    infos = pkg.ski_solve_adjoint_batched(mats, bt, xs, Rs, gs, dAs, dbs, o)
    for i, (n, d) in enumerate(shapes):
        assert infos[i].status == 0
        dA1 = torch.empty_like(At[i])
        db1 = torch.empty_like(bt[i])
        pkg.ski_solve_adjoint(mats[i], bt[i], xs[i], Rs[i], d, gs[i], dA1, d, db1, o)
        assert torch.equal(dA1, dAs[i]) and torch.equal(db1, dbs[i])
        A, b = At[i].cpu().numpy(), bt[i].cpu().numpy()
        xr = np.linalg.lstsq(A, b, rcond=None)[0]
        dA, db = oadj.lstsq_grad(A, b, xr, gs[i].cpu().numpy())
        assert rel_fro(dAs[i].cpu().numpy(), dA) <= 1e-9
        assert rel_fro(dbs[i].cpu().numpy(), db) <= 1e-9
    # dA skipped
    dbs2 = [torch.empty_like(b) for b in bt]
    pkg.ski_solve_adjoint_batched(mats, bt, xs, Rs, gs, None, dbs2, o)
    for i in range(len(shapes)):
        assert torch.equal(dbs2[i], dbs[i])


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
        # central finite differences of L along a random direction (EA, eb),
        # on every one of the 8 problems
        EA, eb = g.standard_normal(A.shape), g.standard_normal(b.shape)
        h = 1e-6
        lp = c @ np.linalg.lstsq(A + h * EA, b + h * eb, rcond=None)[0]
        lm = c @ np.linalg.lstsq(A - h * EA, b - h * eb, rcond=None)[0]
        fd = (lp - lm) / (2 * h)
        an = float((At.grad.cpu().numpy() * EA).sum() + bt.grad.cpu().numpy() @ eb)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_lstsq_batched_autograd():
    torch, pkg = cuda()
    from paper_2105_11815_gb300.autograd import lstsq_batched
    g = np.random.default_rng(23)
    shapes = [(512, 32), (800, 16), (640, 48)]
    As = [g.standard_normal(s) for s in shapes]
    bs = [g.standard_normal(s[0]) for s in shapes]
    cs = [g.standard_normal(s[1]) for s in shapes]
    At = [to_dev(torch, A).requires_grad_(True) for A in As]
    bt = [to_dev(torch, b).requires_grad_(True) for b in bs]
    o = pkg.ski_opts_default(m=-2000, s=1, seed=11, tol=1e-10, tau_r=1e-12)
    xs = lstsq_batched(At, bt, o)
    L = sum((x * to_dev(torch, c)).sum() for x, c in zip(xs, cs))
    L.backward()
    for A, b, c, a_t, b_t in zip(As, bs, cs, At, bt):
        xr = np.linalg.lstsq(A, b, rcond=None)[0]
        dA, db = oadj.lstsq_grad(A, b, xr, c)
        assert rel_fro(a_t.grad.cpu().numpy(), dA) <= 1e-9
        assert rel_fro(b_t.grad.cpu().numpy(), db) <= 1e-9


@pytest.mark.parametrize("kappa,qr,expect", [(1e3, 1, 0), (1e5, 3, 1), (1e9, 1, 1), (1e5, 1, 0)])
def test_mixed_precision_fallback(kappa, qr, expect):
    # the FP32 / TF32 factor is kept while kappa(SA) u stays small; past the
    # diagonal-ratio limit Steps 1-2 are redone in FP64 -- either way the
    # FP64 acceptance test holds
    torch, pkg = cuda()
    g = np.random.default_rng(int(np.log10(kappa)) + 10 * qr)
    n, d = 4000, 200
    A, _ = workloads.usv(n, d, kappa, seed=int(np.log10(kappa)))
    # b = A x_true + e with e orthogonal to range(A): x = x_true stays O(1), so
    # the FP64 metric's rounding floor u ||A|| ||x|| / ||r|| is far below 1e-10
    Q = np.linalg.qr(A)[0]
    e = g.standard_normal(n)
    e -= Q @ (Q.T @ e)
    b = A @ g.standard_normal(d) + e
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(m=400, s=1, seed=2, tol=1e-10, tau_r=1e-12, sketch_dtype=pkg.SKI_F32, qr_dtype=qr)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x)
    assert info.status == 0
    # 1: the diagonal ratio triggered it; 2: the LSQR budget did
    assert (info.qr_fallback > 0) == (expect > 0), (info.qr_fallback, info.rdiag_ratio, info.iters)
    assert olsqr.residual_metric(A, b, x.cpu().numpy()) <= 1e-10


# ---------------------------------------------------------------- perturbed back-solve
def test_perturbed_back_solve_matches_the_oracle_on_a_zero_column():
    # Column 5 of A is exactly zero: the sketch's column 5 is zero, r_55 = 0,
    # and the rank rule stops at p = 5.  Without perturb the solve reports the
    # singular factor; with perturb it divides by r_ii + perturb (Ski-LLS-sparse,
    # Section 6).  x_5 is then arbitrary (A's column 5 is zero) while the other
    # entries solve the reduced problem, as in the oracle's perturbed solve.
    from test_oracle_qr_lsqr import zero_column_lls
    torch, pkg = cuda()
    A, b = zero_column_lls()
    keep = np.arange(A.shape[1]) != 5
    _, info = _solve(torch, pkg, A, b, check=False, m=48, s=1, seed=3)
    assert info.status == pkg.STATUS.index("SKI_ESINGULAR") and info.rank == 5
    x, info = _solve(torch, pkg, A, b, m=48, s=1, seed=3, perturb=1e-10)
    assert info.status == 0 and info.rank == 5 and info.inv_dtype == pkg.SKI_F64
    xo, oinfo = olsqr.ski_lls(A, b, seed=3, s=1, m=48, perturb=1e-10)
    assert oinfo["rank"] == 5
    assert rel_fro(x[keep], xo[keep]) <= 1e-9
    xr = np.linalg.lstsq(A[:, keep], b, rcond=None)[0]
    assert rel_fro(x[keep], xr) <= 1e-9
    assert np.isfinite(x[5])
    assert olsqr.residual_metric(A, b, x) <= 1e-10
    assert abs(info.iters - oinfo["iters"]) <= 2 + info.restarts * 5


@pytest.mark.parametrize("premix", [0, 1])
def test_perturbed_back_solve_on_a_repeated_column(premix):
    # Column 7 repeats column 3, so r_77 is rounding noise and the rank rule
    # stops at p = 7.  On a consistent system b = A x_true, Q^T Sb = R x_true
    # has a rounding-level entry 7, x_s = (R + perturb I)^{-1} Q^T Sb stays
    # O(1), and Step 3 already meets tau_a, on the GPU as in the oracle.  (With
    # an inconsistent b that entry is O(||r|| / sqrt(m)), x_3 and x_7 become
    # about 1e7 with opposite signs, and A x cancels to a residual whose FP64
    # rounding is far above 1e-10: the perturbed back-solve is a safeguard,
    # not a solver for rank-deficient problems.)
    torch, pkg = cuda()
    g = np.random.default_rng(44)
    A = g.standard_normal((3000, 40))
    A[:, 7] = A[:, 3]
    b = A @ g.standard_normal(40)
    kw = dict(m=100, s=2, seed=6, perturb=1e-10, tau_a=1e-6)
    if premix:
        kw.update(premix=1, n_pad=4096)
    x, info = _solve(torch, pkg, A, b, **kw)
    assert info.status == 0 and info.rank == 7 and info.early_exit == 1
    xo, oinfo = olsqr.ski_lls(A, b, seed=6, s=2, m=100, perturb=1e-10, tau_a=1e-6, premix=bool(premix),
                              n_pad=4096 if premix else None)
    assert oinfo["rank"] == 7 and oinfo["early_exit"]
    assert np.linalg.norm(A @ x - b) <= 1e-6
    assert np.linalg.norm(A @ xo - b) <= 1e-6


# ---------------------------------------------------------------- wide dynamic range
@pytest.mark.parametrize("premix", [0, 1])
def test_rows_spanning_sixty_decades(premix):
    # Row j of A and b is scaled by 10^e_j, e_j ~ U(-30, 30).  The LSQR pass
    # keeps A as a (hi, lo) float pair after one global power-of-two scale
    # (about 48 significant bits): rows 40 decades below the largest fall
    # under FP32's range there and act as zero in that operator.  The FP64
    # residual and metric see every row, and the warm restarts (iterative
    # refinement against the FP64 residual) must still meet the test.
    torch, pkg = cuda()
    g = np.random.default_rng(77)
    n, d = 20000, 100
    G = g.standard_normal((n, d))
    w = 10.0 ** g.uniform(-30.0, 30.0, n)
    A = w[:, None] * G
    b = w * (G @ g.standard_normal(d) + 1e-3 * g.standard_normal(n))
    kw = dict(m=200, s=1, seed=12)
    if premix:
        kw.update(premix=1, n_pad=32768)
    x, info = _solve(torch, pkg, A, b, **kw)
    assert info.status == 0, (info.status, info.iters, info.restarts)
    assert olsqr.residual_metric(A, b, x) <= 1e-10
