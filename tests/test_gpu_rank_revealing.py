"""Step 2 of Algorithm 1 in its rank-revealing form on the GPU
(ski_opts.factorization = 1): when the plain QR of SA fails the rank rule,
the column-pivoted QR of R gives SA V = Q [R11 R12; 0 0], and Steps 3-5 run
on W = A V1 R11^{-1} (Lemmas 6-8, Theorem 8).

Compared with the oracle's Algorithm 1 with column pivoting of SA itself
(``oracle.lsqr.ski_lls(factorization="qrcp")``; pivoting R picks the same
pivots, pinned on the CPU): the rank p, the pivot set (the columns V1 keeps,
unique for generic inputs), and x, which is unique given that set -- it is
zero outside V1's columns and the least-squares solution of A V1 there.  The
least-squares residual (Theorem 8) and the FP64 acceptance test hold.
"""
import numpy as np
import pytest

from oracle import lsqr as olsqr
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _solve(torch, pkg, A, b, check=True, **kw):
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(tol=1e-10, tau_r=1e-12, **kw)
    x = torch.empty(A.shape[1], dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x, check=check)
    return x.cpu().numpy(), info


def _check_against_oracle(A, b, x, info, oinfo):
    p = oinfo["rank"]
    assert info.rank == p and info.pivoted == 1
    support = set(np.flatnonzero(x).tolist())
    assert support == set(oinfo["piv"][:p].tolist())
    S = np.array(sorted(support))
    xS = np.linalg.lstsq(A[:, S], b, rcond=None)[0]
    assert rel_fro(x[S], xS) <= 1e-8
    assert np.linalg.norm(b - A @ x) == pytest.approx(_ls_residual(A, b, p), rel=1e-10)
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def _ls_residual(A, b, p):
    """||b - U_p U_p^T b||, U_p the leading p left singular vectors of A: the
    least-squares residual of a rank-p A (a pseudo-inverse at its default
    cutoff keeps rounding-level singular values of a product G1 G2 and misses
    it by up to 4e-3 here)."""
    U = np.linalg.svd(A, full_matrices=False)[0][:, :p]
    return np.linalg.norm(b - U @ (U.T @ b))


@pytest.mark.parametrize("n,d,r,m,s,premix", [(3000, 60, 40, 150, 1, 0), (5000, 120, 77, 300, 2, 0),
                                              (4000, 50, 20, 120, 1, 1), (20000, 400, 250, 900, 2, 1)])
def test_low_rank_solve_matches_the_oracle(n, d, r, m, s, premix):
    torch, pkg = cuda()
    A, b = workloads.low_rank_lls(n, d, r, seed=n + d)
    kw = dict(m=m, s=s, seed=r)
    if premix:
        kw.update(premix=1, n_pad=1 << (n - 1).bit_length())
    _, info = _solve(torch, pkg, A, b, check=False, **kw)
    assert info.status == pkg.STATUS.index("SKI_ESINGULAR")      # plain QR stops at the rank rule
    x, info = _solve(torch, pkg, A, b, factorization=1, **kw)
    assert info.status == 0
    xo, oinfo = olsqr.ski_lls(A, b, seed=r, s=s, m=m, premix=bool(premix), n_pad=kw.get("n_pad"),
                              factorization="qrcp")
    assert oinfo["rank"] == r
    _check_against_oracle(A, b, x, info, oinfo)
    assert rel_fro(x, xo) <= 1e-8


def test_full_rank_problem_is_unchanged_by_the_option():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(3000, 80, seed=4)
    x0, i0 = _solve(torch, pkg, A, b, m=160, s=1, seed=2)
    x1, i1 = _solve(torch, pkg, A, b, m=160, s=1, seed=2, factorization=1)
    assert i1.pivoted == 0 and i1.rank == 80
    assert np.array_equal(x0, x1) and i0.iters == i1.iters


def test_zero_and_repeated_columns():
    # column 5 zero, column 9 a copy of column 2: the rank is d - 2 and the
    # pivoted factor keeps one of the two copies (which one is not unique), so
    # x is checked by what is unique: the least-squares residual, a support of
    # p columns that excludes the zero column and holds one copy, and x on that
    # support the least-squares solution there
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(2500, 30, seed=6)
    A = A.copy()
    A[:, 5] = 0.0
    A[:, 9] = A[:, 2]
    x, info = _solve(torch, pkg, A, b, m=90, s=2, seed=4, factorization=1)
    assert info.status == 0 and info.pivoted == 1 and info.rank == 28
    S = np.flatnonzero(x)
    assert len(S) == 28 and 5 not in S and ((2 in S) != (9 in S))
    xS = np.linalg.lstsq(A[:, S], b, rcond=None)[0]
    assert rel_fro(x[S], xS) <= 1e-8
    assert np.linalg.norm(b - A @ x) == pytest.approx(_ls_residual(A, b, 28), rel=1e-10)
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def test_mixed_form_refactors_in_fp64_then_pivots():
    # the FP32 factor of a rank-deficient sketch fails the rank rule, so Steps
    # 1-2 are redone in FP64 (qr_fallback 1) and the FP64 factor is pivoted
    torch, pkg = cuda()
    A, b = workloads.low_rank_lls(6000, 90, 60, seed=12)
    x, info = _solve(torch, pkg, A, b, m=200, s=1, seed=7, premix=1, n_pad=8192, factorization=1,
                     sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32)
    assert info.status == 0 and info.qr_fallback == 1 and info.pivoted == 1 and info.rank == 60
    xo, oinfo = olsqr.ski_lls(A, b, seed=7, s=1, m=200, premix=True, n_pad=8192, factorization="qrcp")
    _check_against_oracle(A, b, x, info, oinfo)


def test_rank_one_and_early_exit():
    # rank 1 (every column a multiple of one vector) and a consistent b: p = 1
    # and Step 3 already meets tau_a
    torch, pkg = cuda()
    g = np.random.default_rng(3)
    u = g.standard_normal(1500)
    A = np.outer(u, g.standard_normal(12))
    b = 2.5 * u
    x, info = _solve(torch, pkg, A, b, m=40, s=1, seed=1, factorization=1, tau_a=1e-8)
    assert info.status == 0 and info.rank == 1 and info.pivoted == 1 and info.early_exit == 1
    assert np.count_nonzero(x) == 1
    assert np.linalg.norm(A @ x - b) <= 1e-8
