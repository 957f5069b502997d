"""Step 2 of Ski-LLS-sparse from a sparse sketch (Section 6;
ski_opts.factorization = 2): SA kept in CSR, R the Cholesky factor of its Gram
matrix SA^T SA, Q^T Sb = R^{-T} SA^T Sb, against the oracle's
``qr.gram_cholesky`` and ``ski_lls(factorization="chol")``; and the fallback to
the Householder QR of the dense sketch when the Cholesky breaks down or a
sketch row is too long for the shared-memory merge."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lsqr as olsqr, qr as oqr, sketch as osk
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _csr(torch, pkg, A):
    A = A.tocsr()
    A.sort_indices()
    arrs = (to_dev(torch, A.indptr.astype(np.int64)), to_dev(torch, A.indices.astype(np.int32)),
            to_dev(torch, A.data.astype(np.float64)))
    return pkg.csr_matrix(arrs[0], arrs[1], arrs[2], A.shape[0], A.shape[1]), arrs


def _solve(torch, pkg, A, b, **kw):
    M, keep = _csr(torch, pkg, A)
    d = A.shape[1]
    o = pkg.ski_opts_default(tol=1e-10, tau_r=1e-12, **kw)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    R = torch.empty(d, d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(M, to_dev(torch, b), o, x, R_out=R)
    return x.cpu().numpy(), R.cpu().numpy(), info


# d = 1300 > 1024: the FP64 Cholesky runs in 512-column panels, the update
# across panels from exact FP16 slice products on the tensor cores
@pytest.mark.parametrize("n,d,s,m", [(20000, 150, 2, 300), (8000, 64, 1, 200), (30000, 300, 3, 700),
                                     (40000, 1300, 2, 2600)])
def test_gram_factor_matches_the_oracle(n, d, s, m):
    torch, pkg = cuda()
    rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=n + d, nnz_row=8, heavy_frac=1e-3, heavy_nnz=min(d, 100))
    A = sp.csr_matrix((v, ci, rp), shape=(n, d))
    x, R, info = _solve(torch, pkg, A, b, m=m, s=s, seed=5, factorization=2)
    assert info.status == 0 and info.gram == 1
    SAb = osk.sketch_rows(5, s, m, A, b)
    Ro = oqr.gram_cholesky(SAb[:, :d])
    assert rel_fro(R, Ro) <= 1e-11
    assert np.allclose(np.tril(R, -1), 0.0)
    xo, oinfo = olsqr.ski_lls(A, b, seed=5, s=s, m=m, factorization="chol")
    assert rel_fro(x, xo) <= 1e-9
    assert abs(info.iters - oinfo["iters"]) <= 1
    assert olsqr.residual_metric(A, b, x) <= 1e-10
    # the same solve through the Householder QR: R agrees up to row signs
    _, Rq, iq = _solve(torch, pkg, A, b, m=m, s=s, seed=5)
    assert iq.gram == 0
    assert rel_fro(np.sign(np.diag(Rq))[:, None] * Rq, R) <= 1e-9


def test_breakdown_falls_back_to_householder():
    # a zero column: the Gram's pivot is 0, the Cholesky reports failure and
    # the Householder QR of the dense sketch is taken (then the perturbed
    # back-solve, since R fails the rank rule)
    torch, pkg = cuda()
    n, d = 6000, 40
    rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=3, nnz_row=6, heavy_frac=0.0, heavy_nnz=0)
    A = sp.csr_matrix((v, ci, rp), shape=(n, d)).tolil()
    A[:, 7] = 0.0
    A = A.tocsr()
    A.eliminate_zeros()
    b = A @ np.random.default_rng(2).standard_normal(d)     # consistent: x_s solves it
    x, R, info = _solve(torch, pkg, A, b, m=120, s=2, seed=9, factorization=2, perturb=1e-8, tau_a=1e-6)
    # rank: the leading diagonal entries that pass the rule stop at column 7
    assert info.status == 0 and info.gram == 0 and info.rank == 7
    assert np.linalg.norm(A @ x - b) <= 1e-6


def test_long_sketch_rows_fall_back():
    # 20000 rows of 50 nonzeros hashed into m = 100 rows: each sketch row
    # gathers ~10000 entries before merging, more than the shared-memory merge
    # takes, so the Householder QR of the dense sketch is used
    torch, pkg = cuda()
    n, d = 20000, 80
    A = sp.random(n, d, density=50 / d, random_state=6, format="csr")
    b = np.random.default_rng(6).standard_normal(n)
    x, R, info = _solve(torch, pkg, A, b, m=100, s=1, seed=1, factorization=2)
    assert info.status == 0 and info.gram == 0
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def _dense_solve(torch, pkg, A, b, check=True, **kw):
    d = A.shape[1]
    o = pkg.ski_opts_default(tol=1e-10, tau_r=1e-12, **kw)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    R = torch.empty(d, d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, x, R_out=R, check=check)
    return x.cpu().numpy(), R.cpu().numpy(), info


@pytest.mark.parametrize("n,d,m,premix", [(6000, 150, 300, 0), (9000, 260, 520, 1), (4000, 33, 70, 0)])
def test_dense_gram_factor_matches_the_oracle(n, d, m, premix):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n + d)
    kw = dict(m=m, s=1, seed=6)
    npad = 1 << (n - 1).bit_length()
    if premix:
        kw.update(premix=1, n_pad=npad)
    x, R, info = _dense_solve(torch, pkg, A, b, factorization=2, **kw)
    assert info.status == 0 and info.gram == 1
    xo, oinfo = olsqr.ski_lls(A, b, seed=6, s=1, m=m, premix=bool(premix), n_pad=npad if premix else None,
                              factorization="chol")
    assert rel_fro(R, oinfo["R"]) <= 1e-11
    assert rel_fro(x, xo) <= 1e-9
    assert abs(info.iters - oinfo["iters"]) <= 1
    assert olsqr.residual_metric(A, b, x) <= 1e-10


@pytest.mark.parametrize("qr", ["f32", "tf32"])
def test_dense_gram_factor_in_fp32(qr):
    # the Gram matrix on the tensor cores and the Cholesky in FP32: R within
    # the FP32 factor's accuracy of the oracle's, and the solve meets 1e-10
    # after as many iterations as the FP64 factor's (TF32: a few more)
    torch, pkg = cuda()
    n, d, m = 20000, 400, 800
    A, b, _ = workloads.gaussian_lls(n, d, seed=8)
    qdt = pkg.SKI_F32 if qr == "f32" else pkg.SKI_TF32
    x, R, info = _dense_solve(torch, pkg, A, b, m=m, s=1, seed=4, factorization=2, sketch_dtype=pkg.SKI_F32,
                              qr_dtype=qdt)
    assert info.status == 0 and info.gram == 1 and info.qr_fallback == 0
    _, oinfo = olsqr.ski_lls(A, b, seed=4, s=1, m=m, factorization="chol")
    assert rel_fro(R, oinfo["R"]) <= (1e-5 if qr == "f32" else 2e-2)
    assert olsqr.residual_metric(A, b, x) <= 1e-10
    if qr == "f32":
        assert abs(info.iters - oinfo["iters"]) <= 2


@pytest.mark.parametrize("kappa,mixed", [(1e6, True), (1e10, False)])
def test_dense_gram_falls_back_when_ill_conditioned(kappa, mixed):
    # kappa(SA)^2 u too large for the Gram matrix's precision: the factor's
    # diagonal ratio passes the limit and Step 2 takes the Householder QR
    torch, pkg = cuda()
    n, d = 12000, 200
    A, b = workloads.usv(n, d, kappa, seed=3)
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    x, R, info = _dense_solve(torch, pkg, A, b, check=False, m=2 * d, s=1, seed=2, factorization=2, **prec)
    assert info.gram == 0
    assert info.status in (0, pkg.STATUS.index("SKI_ENOCONV"))
    # the Householder solve's accuracy.  At kappa = 1e10, |x| ~ 1e9: the
    # FP64 rounding of x alone moves the metric by about 1e-10, so the
    # double-double check allows a few times the acceptance level
    assert olsqr.residual_metric_dd(A, b, x) <= (3e-10 if kappa < 1e8 else 1e-9)


@pytest.mark.parametrize("n,d,m", [(40000, 64, 20000), (3000, 130, 2999)])
def test_dense_fp64_gram_from_slices_matches_the_oracle(n, d, m):
    # the FP64 Gram matrix from exact FP16 slice products on the tensor cores:
    # m = 20000 rows leave 4 bits per slice (14 slices), m = 2999 five (11)
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n + d + m)
    x, R, info = _dense_solve(torch, pkg, A, b, m=m, s=1, seed=8, factorization=2)
    assert info.status == 0 and info.gram == 1
    xo, oinfo = olsqr.ski_lls(A, b, seed=8, s=1, m=m, factorization="chol")
    assert rel_fro(R, oinfo["R"]) <= 1e-12
    assert rel_fro(x, xo) <= 1e-9
    assert olsqr.residual_metric(A, b, x) <= 1e-10


def test_dense_fp64_gram_column_scales():
    # columns 2^-19 .. 2^19 apart (within the rank rule's 1e-12): each column
    # of SA keeps its own exponent in the slices, and the fallback test looks
    # at |SA_j| / r_jj, which such scales leave alone, so the Gram factor is
    # kept although max r_jj / min r_jj is near 2^38; R = R0 D for the column
    # scaling D, R0 the oracle's factor of the unscaled problem
    torch, pkg = cuda()
    n, d, m = 5000, 96, 400
    A, b, _ = workloads.gaussian_lls(n, d, seed=31)
    ex = np.round(np.linspace(-19, 19, d)).astype(int)
    D = np.ldexp(1.0, ex)
    x, R, info = _dense_solve(torch, pkg, A * D, b, m=m, s=1, seed=9, factorization=2)
    assert info.status == 0 and info.gram == 1
    _, oinfo = olsqr.ski_lls(A, b, seed=9, s=1, m=m, factorization="chol")
    assert rel_fro(R / D, oinfo["R"]) <= 1e-12
    assert olsqr.residual_metric(A * D, b, x) <= 1e-10


@pytest.mark.parametrize("mixed", [False, True])
def test_dense_gram_nonfinite_and_singular(mixed):
    # a NaN in A, or two equal columns: the Gram path reports what the
    # Householder path reports (SKI_ENONFINITE, SKI_ESINGULAR)
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(500, 20, seed=1)
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    An = A.copy()
    An[17, 5] = np.nan
    _, _, info = _dense_solve(torch, pkg, An, b, check=False, m=40, s=1, seed=1, factorization=2, **prec)
    assert info.status == pkg.STATUS.index("SKI_ENONFINITE")
    Ad = A.copy()
    Ad[:, 7] = Ad[:, 3]
    _, _, info = _dense_solve(torch, pkg, Ad, b, check=False, m=40, s=1, seed=1, factorization=2, **prec)
    assert info.status == pkg.STATUS.index("SKI_ESINGULAR")


@pytest.mark.parametrize("premix", [0, 1])
def test_dense_fp64_gram_two_level_cholesky(premix):
    # d > 1024: the FP64 Cholesky runs in panels of 512 columns, the update
    # across panels from exact FP16 slice products of the panel's block row
    # (7-bit slices, K = 512) on the tensor cores; R against the oracle's
    # FP64 Gram factor
    torch, pkg = cuda()
    n, d, m = 9000, 1300, 2600
    A, b, _ = workloads.gaussian_lls(n, d, seed=77)
    kw = dict(m=m, s=1, seed=12)
    npad = 16384
    if premix:
        kw.update(premix=1, n_pad=npad)
    x, R, info = _dense_solve(torch, pkg, A, b, factorization=2, **kw)
    assert info.status == 0 and info.gram == 1
    xo, oinfo = olsqr.ski_lls(A, b, seed=12, s=1, m=m, premix=bool(premix), n_pad=npad if premix else None,
                              factorization="chol")
    assert rel_fro(R, oinfo["R"]) <= 1e-12
    assert rel_fro(x, xo) <= 1e-9
    assert abs(info.iters - oinfo["iters"]) <= 1
    assert olsqr.residual_metric(A, b, x) <= 1e-10
