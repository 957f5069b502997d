"""The Hartley premix F D of Ski-LLS-dense (Section 6, Eq. HR-DHT) and the
sampling sketch S_s of Eq. SR-DHT on the GPU, against the oracle
(``oracle/dht.py``: numpy's FFT route, itself pinned to the explicit F).

Lengths cover every radix of the mixed-radix FFT (4, 2, 3, 5, 7, 11, 13), a
single pass (N = 4), N = 1, and zero-padded lengths (n = 17 -> 18,
n = 1009 -> 1014); the full-size check transforms 50000 x 4000 and compares
sampled columns (the transform acts on each column alone).
"""
import numpy as np
import pytest

from oracle import dht, lsqr as olsqr
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _premix(torch, pkg, A, b, N, dtype, seed=5):
    At, bt = to_dev(torch, A), (to_dev(torch, b) if b is not None else None)
    ncols = A.shape[1] + (b is not None)
    tdt = torch.float64 if dtype == pkg.SKI_F64 else torch.float32
    Y = torch.full((N, ncols + 3), float("nan"), dtype=tdt, device="cuda")
    o = pkg.ski_opts_default(premix=2, n_pad=N, seed=seed, sketch_dtype=dtype)
    pkg.ski_premix(pkg.dense_matrix(At), bt, o, Y, ncols + 3)
    return Y[:, :ncols].double().cpu().numpy()


@pytest.mark.parametrize("n,d,N", [(60, 5, 60), (1000, 7, 1000), (4096, 3, 4096), (2730, 4, 2730), (4, 6, 4),
                                   (1, 2, 1), (17, 3, 18), (1009, 6, 1014), (3000, 2, 2 * 3 * 7 * 11 * 13 * 2)])
def test_dht_premix_matches_the_oracle(n, d, N):
    torch, pkg = cuda()
    g = np.random.default_rng(n + d)
    A, b = g.standard_normal((n, d)), g.standard_normal(n)
    ref = np.column_stack([dht.premix(5, A, N), dht.premix(5, b, N)])
    Y = _premix(torch, pkg, A, b, N, pkg.SKI_F64)
    assert rel_fro(Y, ref) <= 1e-13
    Y32 = _premix(torch, pkg, A, b, N, pkg.SKI_F32)
    assert rel_fro(Y32, ref) <= 2e-6
    # orthogonal: column norms are kept (the padded rows are zero)
    assert np.allclose(np.linalg.norm(Y, axis=0), np.linalg.norm(np.column_stack([A, b]), axis=0), rtol=1e-12)


def test_default_length_and_bad_lengths():
    torch, pkg = cuda()
    A = np.random.default_rng(1).standard_normal((1009, 3))
    At = to_dev(torch, A)
    Y = torch.empty(1014, 3, dtype=torch.float64, device="cuda")
    pkg.ski_premix(pkg.dense_matrix(At), None, pkg.ski_opts_default(premix=2, seed=5), Y, 3)  # n_pad = 0: 1014
    assert rel_fro(Y.cpu().numpy(), dht.premix(5, A, 1014)) <= 1e-13
    for bad in (1010, 1008, 1013):  # not 13-smooth, or below n
        o = pkg.ski_opts_default(premix=2, n_pad=bad, seed=5)
        assert pkg.ski_premix_workspace_size(pkg.dense_matrix(At), 0, o) == 0
        with pytest.raises(pkg.SkiError):
            pkg.ski_premix(pkg.dense_matrix(At), None, o, Y, 3, ws=torch.empty(1 << 20, dtype=torch.uint8,
                                                                             device="cuda"))


@pytest.mark.parametrize("s,dtype", [(1, "f64"), (2, "f64"), (1, "f32")])
def test_hrdht_sketch_matches_the_oracle(s, dtype):
    torch, pkg = cuda()
    n, d, m = 5003, 40, 160
    A, b, _ = workloads.gaussian_lls(n, d, seed=3)
    N = dht.dht_length(n)
    sdt = pkg.SKI_F64 if dtype == "f64" else pkg.SKI_F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    o = pkg.ski_opts_default(premix=2, m=m, s=s, seed=21, sketch_dtype=sdt)
    SA = torch.empty(m, d + 1, dtype=tdt, device="cuda")
    pkg.ski_sketch_hash(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, SA, d + 1)
    ref = dht.hrdht_sketch(21, s, m, A, b, n_h=N)
    assert rel_fro(SA.double().cpu().numpy(), ref) <= (1e-12 if dtype == "f64" else 1e-5)


@pytest.mark.parametrize("premix", [2, 0])
def test_sampling_sketch_matches_the_oracle(premix):
    torch, pkg = cuda()
    n, d, m = 2000, 12, 90
    A, b, _ = workloads.gaussian_lls(n, d, seed=4)
    o = pkg.ski_opts_default(premix=premix, m=m, s=1, seed=33, hash_kind=pkg.SKI_SAMPLING)
    SA = torch.empty(m, d + 1, dtype=torch.float64, device="cuda")
    pkg.ski_sketch_hash(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, SA, d + 1)
    if premix:
        ref = dht.srdht_sketch(33, m, A, b, n_h=dht.dht_length(n))
        assert rel_fro(SA.cpu().numpy(), ref) <= 1e-13
    else:
        from oracle import hashing
        rows = hashing.sample_rows(33, m, n)
        assert np.array_equal(SA.cpu().numpy(), np.column_stack([A, b])[rows])   # a copy of the rows: exact
    # s != 1, CSR, and the Walsh-Hadamard premix are refused with the sampling sketch
    for kw in (dict(s=2), dict(premix=1)):
        bad = pkg.ski_opts_default(m=m, seed=33, hash_kind=pkg.SKI_SAMPLING, **dict(dict(s=1, premix=premix), **kw))
        assert pkg.ski_sketch_workspace_size(pkg.dense_matrix(to_dev(torch, A)), 1, bad) == 0


@pytest.mark.parametrize("n,mixed", [(6000, False), (5003, False), (6000, True)])
def test_solve_with_the_hartley_premix(n, mixed):
    torch, pkg = cuda()
    d, m = 60, 180
    A, b, _ = workloads.gaussian_lls(n, d, seed=n)
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    o = pkg.ski_opts_default(premix=2, m=m, s=1, seed=8, tol=1e-10, tau_r=1e-12, **prec)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, x)
    assert info.status == 0
    xg = x.cpu().numpy()
    assert olsqr.residual_metric(A, b, xg) <= 1e-10
    xo, oinfo = olsqr.ski_lls(A, b, seed=8, s=1, m=m, premix="dht", n_pad=dht.dht_length(n))
    assert rel_fro(xg, xo) <= 1e-8
    if not mixed:
        assert abs(info.iters - oinfo["iters"]) <= 2


def test_sr_dht_solve_of_a_coherent_matrix():
    # Fig. blen_motivation's setting: the sampled sketch of F D A still gives a
    # preconditioner at m = 3d, and the solve reaches the tolerance
    torch, pkg = cuda()
    n, d = 4000, 100
    A = workloads.coherent_dense(n, d)
    b = np.ones(n)
    o = pkg.ski_opts_default(premix=2, m=3 * d, s=1, seed=2, hash_kind=pkg.SKI_SAMPLING, tol=1e-10, tau_r=1e-12)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(to_dev(torch, A)), to_dev(torch, b), o, x)
    assert info.status == 0
    assert olsqr.residual_metric(A, b, x.cpu().numpy()) <= 1e-10


def test_full_size_dht_premix_on_sampled_columns():
    torch, pkg = cuda()
    n, d = 50000, 4000
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    At = torch.randn(n, d, generator=g, device="cuda", dtype=torch.float64)
    bt = torch.ones(n, dtype=torch.float64, device="cuda")
    o = pkg.ski_opts_default(premix=2, seed=19)
    Y = torch.empty(n, d + 1, dtype=torch.float64, device="cuda")
    pkg.ski_premix(pkg.dense_matrix(At), bt, o, Y, d + 1)
    cols = [0, 1, 999, 2048, 3001, 3999]
    ref = dht.premix(19, At[:, cols].cpu().numpy(), n)
    assert rel_fro(Y[:, cols].cpu().numpy(), ref) <= 1e-13
    assert rel_fro(Y[:, d].cpu().numpy(), dht.premix(19, np.ones(n), n)) <= 1e-13
