"""GPU parity of the sketch, premix, QR and R^{-1} kernels against the oracle.

Tolerances: hash rows/signs bit-exact; FP64 sketch and premix <= 1e-12
relative Frobenius (the method's FP64 target); FP32 <= 1e-5, BF16 <= 1e-2
(unit roundoff of the storage type times a small growth factor); R <= 1e-12
relative to ||R|| after normalising row signs (Householder signs are arbitrary).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hashing, qr as oqr, sketch as osk, wht as owht
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,s,m,n", [(1, 1, 512, 4096), (2, 2, 7, 10001), (3, 3, 5, 777), (4, 8, 9, 3000),
                                        (5, 2, 40000, 1_000_003), (6, 4, 4, 100)])
def test_hash_indices_bit_exact(seed, s, m, n):
    torch, pkg = cuda()
    idx = torch.empty(n * s, dtype=torch.int32, device="cuda")
    sg = torch.empty(n * s, dtype=torch.int8, device="cuda")
    pkg.ski_hash_indices(seed, s, m, n, idx, sg)
    ri, rs = hashing.hash_table(seed, s, m, n)
    assert np.array_equal(idx.cpu().numpy().reshape(n, s), ri)
    assert np.array_equal(sg.cpu().numpy().reshape(n, s), rs)


def test_premix_signs_bit_exact():
    torch, pkg = cuda()
    D = torch.empty(65537, dtype=torch.int8, device="cuda")
    pkg.ski_premix_signs(20210525, 65537, D)
    assert np.array_equal(D.cpu().numpy(), hashing.premix_signs(20210525, 65537))


def _sketch(torch, pkg, A, b, **kw):
    n, d = A.shape
    At = to_dev(torch, A)
    bt = to_dev(torch, b) if b is not None else None
    o = pkg.ski_opts_default(**kw)
    dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[o.sketch_dtype]
    ncols = d + (b is not None)
    ld = ncols + 3
    SA = torch.full((o.m, ld), float("nan"), dtype=dt, device="cuda")
    pkg.ski_sketch_hash(pkg.dense_matrix(At), bt, o, SA, ld)
    return SA[:, :ncols].double().cpu().numpy()


@pytest.mark.parametrize("n,d,m,s", [(4096, 256, 512, 1), (3001, 37, 100, 3), (5000, 300, 310, 2),
                                     (64, 1, 64, 1), (1, 5, 5, 2)])
def test_dense_sketch_fp64(n, d, m, s):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n + d)
    got = _sketch(torch, pkg, A, b, m=m, s=s, seed=11)
    want = osk.sketch_rows(11, s, m, A, b)
    assert rel_fro(got, want) <= 1e-12


def test_dense_sketch_equals_explicit_S_times_A():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(300, 9, seed=1)
    S = osk.s_hashing_matrix(5, 2, 31, 300)
    got = _sketch(torch, pkg, A, b, m=31, s=2, seed=5)
    assert rel_fro(got[:, :9], S @ A) <= 1e-12
    assert rel_fro(got[:, 9], S @ b) <= 1e-12


def test_dense_sketch_extreme_scales_and_determinism():
    torch, pkg = cuda()
    g = np.random.default_rng(3)
    A = g.standard_normal((2000, 40)) * np.exp(g.uniform(-60, 60, size=(2000, 1)))  # rows span 1e-26..1e26
    got1 = _sketch(torch, pkg, A, None, m=100, s=2, seed=9)
    got2 = _sketch(torch, pkg, A, None, m=100, s=2, seed=9)
    assert np.array_equal(got1, got2)
    want = osk.sketch_rows(9, 2, 100, A)
    # per-entry relative error against the exactly rounded sum magnitude
    assert np.max(np.abs(got1 - want) / (np.abs(want) + 1e-300)) <= 1e-12


@pytest.mark.parametrize("dt,tol", [(1, 1e-5), (2, 1e-2)])
def test_dense_sketch_low_precision(dt, tol):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(4096, 100, seed=2)
    got = _sketch(torch, pkg, A, b, m=256, s=2, seed=3, sketch_dtype=dt)
    assert rel_fro(got, osk.sketch_rows(3, 2, 256, A, b)) <= tol


def test_csr_sketch_fp64():
    torch, pkg = cuda()
    rp, ci, v, b = workloads.csr_heavy_rows(20000, 300, seed=4, nnz_row=8, heavy_frac=0.002, heavy_nnz=200)
    A = sp.csr_matrix((v, ci, rp), shape=(20000, 300))
    o = pkg.ski_opts_default(m=600, s=2, seed=13)
    SA = torch.empty(600, 301, dtype=torch.float64, device="cuda")
    keep = (to_dev(torch, rp), to_dev(torch, ci), to_dev(torch, v))
    M = pkg.csr_matrix(keep[0], keep[1], keep[2], 20000, 300)
    pkg.ski_sketch_hash(M, to_dev(torch, b), o, SA, 301)
    want = osk.sketch_rows(13, 2, 600, A, b)
    assert rel_fro(SA.cpu().numpy(), want) <= 1e-12
    # FP32 output with a padded row stride, and empty rows (5000..5099 dropped)
    keep_rows = np.ones(20000, bool)
    keep_rows[5000:5100] = False
    A2 = sp.csr_matrix(sp.diags(keep_rows.astype(np.float64)) @ A)
    A2.eliminate_zeros()
    A2.sort_indices()
    rp2, ci2, v2 = A2.indptr.astype(np.int64), A2.indices.astype(np.int32), A2.data
    M2 = pkg.csr_matrix(to_dev(torch, rp2), to_dev(torch, ci2), to_dev(torch, v2), 20000, 300)
    o32 = pkg.ski_opts_default(m=600, s=2, seed=13, sketch_dtype=pkg.SKI_F32)
    SA32 = torch.full((600, 305), float("nan"), dtype=torch.float32, device="cuda")
    pkg.ski_sketch_hash(M2, to_dev(torch, b), o32, SA32, 305)
    want2 = osk.sketch_rows(13, 2, 600, A2, b)
    assert rel_fro(SA32[:, :301].double().cpu().numpy(), want2) <= 1e-6


# (40000, 34) and (20000, 34): the TMA-fed first pass (even row stride); odd
# strides take the one-tile-per-CTA kernel
@pytest.mark.parametrize("n,d,npad", [(3000, 7, 4096), (20000, 33, 32768), (1, 3, 1), (2, 2, 2), (700, 5, 1024),
                                      (130000, 3, 262144), (20000, 34, 32768), (40000, 34, 65536),
                                      (40000, 35, 65536)])
def test_premix_fp64(n, d, npad):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(seed=77, n_pad=npad)
    Y = torch.empty(npad, d + 1, dtype=torch.float64, device="cuda")
    pkg.ski_premix(pkg.dense_matrix(At), bt, o, Y, d + 1)
    want = owht.premix(77, np.column_stack([A, b]), npad)
    assert rel_fro(Y.cpu().numpy(), want) <= 1e-12


def test_premix_fp32():
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(5000, 20, seed=5)
    o = pkg.ski_opts_default(seed=1, n_pad=8192, sketch_dtype=pkg.SKI_F32)
    Y = torch.empty(8192, 21, dtype=torch.float32, device="cuda")
    pkg.ski_premix(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, Y, 21)
    assert rel_fro(Y.double().cpu().numpy(), owht.premix(1, np.column_stack([A, b]), 8192)) <= 1e-5


@pytest.mark.parametrize("s", [1, 2])
def test_hrht_sketch_fp64(s):
    torch, pkg = cuda()
    A, b = workloads.dense_high_coherence(5000, 50, seed=3)
    got = _sketch(torch, pkg, A, b, m=120, s=s, seed=21, premix=1, n_pad=8192)
    want = owht.hrht_sketch(21, s, 120, A, b, 8192)
    assert rel_fro(got, want) <= 1e-12


@pytest.mark.parametrize("d,slab,with_b", [(150, 32, True), (150, 64, True), (150, 96, False), (150, 128, True),
                                           (128, 32, True), (31, 32, True), (200, 0, True)])
def test_hrht_sketch_column_slabs(d, slab, with_b):
    # premix and hash gather run slab by slab over the columns; the last slab
    # may be ragged or hold only b
    torch, pkg = cuda()
    A, b = workloads.dense_high_coherence(3000, d, seed=d + slab)
    bb = b if with_b else None
    got = _sketch(torch, pkg, A, bb, m=300, s=2, seed=5, premix=1, n_pad=4096, premix_slab=slab)
    want = owht.hrht_sketch(5, 2, 300, A, bb, 4096)
    assert rel_fro(got, want) <= 1e-12
    got32 = _sketch(torch, pkg, A, bb, m=300, s=2, seed=5, premix=1, n_pad=4096, premix_slab=slab,
                    sketch_dtype=pkg.SKI_F32)
    assert rel_fro(got32, want) <= 1e-5


@pytest.mark.parametrize("kind,s", [("gauss", 2), ("coherent", 1)])
def test_hrht_sketch_full_size_sampled_columns(kind, s):
    # The dense test-set shapes: n = 50000, d = 4000, n_pad = 65536, m = 2d,
    # iid Gaussian and high-coherence (first d rows 1e3 I + N(0, 1e-6)).
    # Checked on sampled columns: column c of S_h H D A is S_h H D A[:, c].
    torch, pkg = cuda()
    n, d, m = 50000, 4000, 8000
    if kind == "gauss":
        A, b = workloads.dense_gaussian(n, d, seed=20210527)
    else:
        A, b = workloads.dense_high_coherence(n, d, seed=20210527)
    got = _sketch(torch, pkg, A, b, m=m, s=s, seed=3, premix=1, n_pad=65536)
    cols = [0, 1, 1234, 2047, 3999, 4000]
    Ab = np.column_stack([A[:, cols[:-1]], b])
    want = owht.hrht_sketch(3, s, m, Ab, None, 65536)
    assert rel_fro(got[:, cols], want) <= 1e-12


# The FP64 premix's last pass stores each column in one shared unit, bounded
# by the sum over the previous pass's tiles of their bounds (high-coherence
# columns, where one tile dominates, keep their precision).  Cases: buckets
# of more than 2^6 rows (the gather renormalises its sums), s = 3, a first
# pass of 5 row bits (not TMA-fed), 9 + 9 row bits (n_pad = 2^18), and three
# passes (n_pad = 2^19: tile families, and all-zero middle-pass tiles in the
# padding).
@pytest.mark.parametrize("n,d,m,s,npad", [(3000, 20, 16, 1, 4096), (3000, 20, 16, 3, 4096), (600, 10, 12, 2, 1024),
                                          (130000, 3, 40, 1, 262144), (300000, 2, 50, 2, 524288),
                                          (5000, 64, 130, 2, 8192)])
def test_hrht_sketch_column_units(n, d, m, s, npad):
    torch, pkg = cuda()
    A, b = workloads.dense_high_coherence(n, d, seed=n + d)
    got = _sketch(torch, pkg, A, b, m=m, s=s, seed=17, premix=1, n_pad=npad)
    again = _sketch(torch, pkg, A, b, m=m, s=s, seed=17, premix=1, n_pad=npad)
    assert np.array_equal(got, again)
    want = owht.hrht_sketch(17, s, m, A, b, npad)
    assert rel_fro(got, want) <= 1e-12


# A NaN or Inf in a column of A makes that column of the premixed result NaN
# (every output row of the column sums it); the other columns are unaffected.
@pytest.mark.parametrize("n,npad,slab", [(3000, 4096, 0), (300, 512, 0), (3000, 4096, 32)])
def test_premix_nonfinite_columns(n, npad, slab):
    torch, pkg = cuda()
    d = 70
    A, b, _ = workloads.gaussian_lls(n, d, seed=n)
    A[17, 3] = np.nan
    A[n - 5, 5] = np.inf
    bad = [3, 5]
    good = [c for c in range(d + 1) if c not in bad]
    got = _sketch(torch, pkg, A, b, m=150, s=2, seed=4, premix=1, n_pad=npad, premix_slab=slab)
    assert np.isnan(got[:, bad]).all()
    want = owht.hrht_sketch(4, 2, 150, A[:, good[:-1]], b, npad)
    assert rel_fro(got[:, good], want) <= 1e-12
    if slab == 0:
        o = pkg.ski_opts_default(seed=77, n_pad=npad)
        Y = torch.empty(npad, d + 1, dtype=torch.float64, device="cuda")
        pkg.ski_premix(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, Y, d + 1)
        Yh = Y.cpu().numpy()
        assert np.isnan(Yh[:, bad]).all()
        assert rel_fro(Yh[:, good], owht.premix(77, np.column_stack([A, b])[:, good], npad)) <= 1e-12


def _signfix(R):
    return np.sign(np.diag(R))[:, None] * R


# FP64 panels of at most 4096 rows run on the 16-CTA cluster kernel, taller
# ones on the cooperative grid-barrier kernel: (5000, 300) is cooperative
# throughout, (4200, 400) switches after its fourth panel.
@pytest.mark.parametrize("m,d,dt", [(512, 256, 0), (1000, 100, 0), (64, 64, 0), (300, 1, 0), (777, 45, 0),
                                    (5000, 300, 0), (4200, 400, 0),
                                    (2000, 300, 1), (2000, 300, 3), (3000, 1000, 1)])
def test_precondition_qr(m, d, dt):
    torch, pkg = cuda()
    g = np.random.default_rng(m + d)
    B = g.standard_normal((m, d + 1))
    tdt = torch.float64 if dt == 0 else torch.float32
    SA = to_dev(torch, B).to(tdt).contiguous()
    R = torch.empty(d, d, dtype=torch.float64, device="cuda")
    qtsb = torch.empty(d, dtype=torch.float64, device="cuda")
    rank = pkg.ski_precondition(m, d, 1, SA, d + 1, dt, R, d, qtsb)
    Ro, C = oqr.householder_qr(B, ncols=d)
    Rg = R.cpu().numpy()
    # FP64: 1e-12.  SKI_TF32, one tensor-core pass (10-bit mantissa): the unit
    # roundoff 2^-10 ~ 1e-3 times a small growth factor over the panels bounds
    # the relative error at 1e-2.  SKI_F32, three passes: FP32 storage and
    # ~2^-21 products, Householder backward error ~ sqrt(d) u per panel -> 2e-5.
    tol = {0: 1e-12, 1: 2e-5, 3: 1e-2}[dt]
    assert rank == d
    assert rel_fro(_signfix(Rg), _signfix(Ro)) <= tol
    sg = np.sign(np.diag(Rg)) * np.sign(np.diag(Ro))
    assert rel_fro(sg * qtsb.cpu().numpy(), C[:, 0]) <= (tol * 10 if dt == 0 else 3 * tol)
    assert np.allclose(np.tril(Rg, -1), 0)


@pytest.mark.parametrize("case", ["scaled_columns", "near_dependent", "tall", "last_panel_short"])
def test_fp32_qr_panel_forms(case):
    # FP32 panels are factored by Cholesky QR twice and Householder
    # reconstruction (two cluster reductions per panel), with columns
    # equilibrated; a panel whose equilibrated Cholesky pivot falls below
    # 2^-24 (condition above ~4e3) takes the column-by-column steps instead.
    # Checked: the backward error ||R^T R - B^T B|| / ||B||^2 at FP32 level in
    # every case; R and Q^T Sb against the oracle at the three-pass FP32
    # tolerance where B is well conditioned; and, where a panel is nearly
    # singular (its FP32 R differs from the FP64 one in the ill-determined
    # direction), that R still preconditions: kappa(B R^{-1}) near 1.
    torch, pkg = cuda()
    g = np.random.default_rng(7)
    m, d = {"scaled_columns": (3000, 200), "near_dependent": (3000, 200), "tall": (12000, 160),
            "last_panel_short": (2500, 77)}[case]
    B = g.standard_normal((m, d + 1))
    if case == "scaled_columns":
        B[:, :d] *= 10.0 ** g.uniform(-5, 0, d)            # equilibration: no fallback needed
    if case == "near_dependent":
        B[:, 37] = B[:, 36] + 1e-6 * g.standard_normal(m)  # panel 1 condition ~1e6: column-by-column
    SA = to_dev(torch, B).to(torch.float32).contiguous()
    R = torch.empty(d, d, dtype=torch.float64, device="cuda")
    qtsb = torch.empty(d, dtype=torch.float64, device="cuda")
    pkg.ski_precondition(m, d, 1, SA, d + 1, pkg.SKI_F32, R, d, qtsb, want_rank=False)
    Bf = SA.double().cpu().numpy()[:, :d]                   # the FP32 input exactly
    Rg = R.cpu().numpy()
    assert np.allclose(np.tril(Rg, -1), 0)
    G = Bf.T @ Bf
    assert np.linalg.norm(Rg.T @ Rg - G) / np.linalg.norm(G) <= 1e-5
    if case == "near_dependent":
        W = np.linalg.solve(Rg.T, Bf.T).T
        assert np.linalg.cond(W) < 2.0
    else:
        Ro, C = oqr.householder_qr(SA.double().cpu().numpy(), ncols=d)
        assert rel_fro(_signfix(Rg), _signfix(Ro)) <= 2e-5
        sg = np.sign(np.diag(Rg)) * np.sign(np.diag(Ro))
        assert rel_fro(sg * qtsb.cpu().numpy(), C[:, 0]) <= 6e-5


def test_fp32_qr_preconditions_ill_conditioned_sketch():
    # R only has to precondition (Theorem 10): kappa(SA R^-1) stays near 1 for
    # the three-pass FP32 QR at kappa(SA) = 1e5, where one TF32 pass does not.
    torch, pkg = cuda()
    g = np.random.default_rng(41)
    m, d = 2000, 200
    U = np.linalg.qr(g.standard_normal((m, d)))[0]
    V = np.linalg.qr(g.standard_normal((d, d)))[0]
    B = (U * (1e5 ** -(np.arange(d) / (d - 1)))) @ V.T
    conds = {}
    for dt in (1, 3):
        SA = to_dev(torch, B).to(torch.float32).contiguous()
        R = torch.empty(d, d, dtype=torch.float64, device="cuda")
        pkg.ski_precondition(m, d, 0, SA, d, dt, R, d, None, want_rank=False)
        W = np.linalg.solve(R.cpu().numpy().T, B.T).T
        conds[dt] = np.linalg.cond(W)
    assert conds[1] < 1.5, conds
    assert conds[3] > 2 * conds[1], conds


@pytest.mark.parametrize("d,dt", [(1, 0), (31, 0), (64, 0), (257, 0), (1000, 0), (500, 1)])
def test_trinv(d, dt):
    torch, pkg = cuda()
    g = np.random.default_rng(d)
    R = np.linalg.qr(g.standard_normal((2 * d + 4, d)), mode="r")  # well conditioned
    Rt = to_dev(torch, R)
    M = torch.empty(d, d, dtype=torch.float64, device="cuda")
    Mt = torch.empty(d, d, dtype=torch.float64, device="cuda")
    pkg.ski_trinv(d, Rt, d, M, Mt, d, dtype=dt)
    Mn = M.cpu().numpy()
    tol = 1e-12 if dt == 0 else 1e-5
    assert np.linalg.norm(Mn @ R - np.eye(d)) / np.sqrt(d) <= tol
    assert np.array_equal(Mt.cpu().numpy(), Mn.T)


def _tf32(x):
    """Round toward zero to the 10-bit mantissa the TF32 tensor cores read."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K,sub", [(128, 32, 32, 0), (200, 300, 100, 0), (257, 64, 1000, 1), (5, 7, 3, 0),
                                       (1000, 256, 32, 1)])
def test_tensor_core_gemm_tf32(M, N, K, sub):
    torch, pkg = cuda()
    g = np.random.default_rng(M + N + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    C0 = g.standard_normal((M, N)).astype(np.float32)
    lda = ldb = (K + 3) // 4 * 4
    Ad = torch.zeros(M, lda, dtype=torch.float32, device="cuda")
    Bd = torch.zeros(N, ldb, dtype=torch.float32, device="cuda")
    Ad[:, :K] = torch.from_numpy(A).cuda()
    Bd[:, :K] = torch.from_numpy(B).cuda()
    Cd = torch.from_numpy(C0).cuda()
    pkg.ski_gemm_tc_f32(M, N, K, Ad, lda, Bd, ldb, Cd, N, subtract=bool(sub))
    D = _tf32(A) @ _tf32(B).T          # exact products of the TF32 operands, FP64 sums
    want = C0 - D if sub else D
    # FP32 accumulation of K products: error <= K * 2^-24 * sum |a||b|
    bound = K * 2.0 ** -23 * (np.abs(_tf32(A)) @ np.abs(_tf32(B)).T) + 1e-6
    assert np.all(np.abs(Cd.cpu().numpy() - want) <= bound)


@pytest.mark.parametrize("M,N,K,sub", [(128, 32, 32, 0), (200, 300, 100, 0), (257, 64, 1000, 1), (5, 7, 3, 0),
                                       (1000, 256, 32, 1), (300, 32, 4000, 0)])
def test_tensor_core_gemm_split_tf32(M, N, K, sub):
    # three TF32 passes: lo*hi + hi*lo + hi*hi against the exact FP64 product
    torch, pkg = cuda()
    g = np.random.default_rng(M * N + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    C0 = g.standard_normal((M, N)).astype(np.float32)
    lda = ldb = (K + 3) // 4 * 4
    Ad = torch.zeros(M, lda, dtype=torch.float32, device="cuda")
    Bd = torch.zeros(N, ldb, dtype=torch.float32, device="cuda")
    Ad[:, :K] = torch.from_numpy(A).cuda()
    Bd[:, :K] = torch.from_numpy(B).cuda()
    Cd = torch.from_numpy(C0).cuda()
    pkg.ski_gemm_tc_f32(M, N, K, Ad, lda, Bd, ldb, Cd, N, subtract=bool(sub), passes=3)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    D = A64 @ B64.T
    want = C0.astype(np.float64) - D if sub else D
    absprod = np.abs(A64) @ np.abs(B64).T
    # per product <= 3 * 2^-22 |a||b| (dropped lo*lo, lo rounded); FP32 sums of
    # K terms <= K * 2^-24 sum |a||b|; the C0 update adds one FP32 rounding
    bound = (3 * 2.0 ** -22 + K * 2.0 ** -24) * absprod + 2.0 ** -23 * np.abs(want) + 1e-6
    err = np.abs(Cd.cpu().numpy() - want)
    assert np.all(err <= bound)
    # and far below one TF32 pass on the same operands
    C1 = torch.from_numpy(C0).cuda()
    pkg.ski_gemm_tc_f32(M, N, K, Ad, lda, Bd, ldb, C1, N, subtract=bool(sub), passes=1)
    err1 = np.abs(C1.cpu().numpy() - want)
    assert np.median(err) * 10 < np.median(err1)
