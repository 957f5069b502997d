"""ski_sketch_hash_noalloc, the variant for callers that cannot allocate.

Some callers cannot call cudaMalloc or hand the library a workspace (their
memory is owned by another allocator, or they run where allocation is not
allowed); this entry point keeps its scratch in a fixed device array of the
library.  This test calls it through the C ABI and checks it against the
workspace entry point ski_sketch_hash, on two calls in a row (the second
reuses the shared scratch left by the first), at the FP64 sketch tolerance
of the other tests (1e-12 relative Frobenius).  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _run(torch, pkg, M, bt, o, m, ncols, dtype):
    """The same sketch through ski_sketch_hash (caller workspace) and through
    ski_sketch_hash_noalloc (the library's fixed array); returns (status of
    the latter, its output, the former's output) as FP64 host arrays."""
    ref = torch.full((m, ncols), float("nan"), dtype=dtype, device="cuda")
    got = torch.full((m, ncols), float("nan"), dtype=dtype, device="cuda")
    pkg.ski_sketch_hash(M, bt, o, ref, ncols)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = pkg.lib().ski_sketch_hash_noalloc(ctypes.byref(M), None if bt is None else ctypes.c_void_p(bt.data_ptr()),
                                          ctypes.byref(o), ctypes.c_void_p(got.data_ptr()), ncols, stream)
    torch.cuda.synchronize()
    return st, got.double().cpu().numpy(), ref.double().cpu().numpy()


def _pair(torch, pkg, n, d, m, s, seed, with_b, hash_kind=0, sketch_dtype=0):
    A, b, _ = workloads.gaussian_lls(n, d, seed=seed)
    At = to_dev(torch, A)
    bt = to_dev(torch, b) if with_b else None
    M = pkg.dense_matrix(At)
    o = pkg.ski_opts_default(m=m, s=s, seed=seed, hash_kind=hash_kind, sketch_dtype=sketch_dtype)
    dtype = torch.float32 if sketch_dtype == pkg.SKI_F32 else torch.float64
    return _run(torch, pkg, M, bt, o, m, d + (1 if with_b else 0), dtype)


def test_noalloc_sketch_matches_workspace_sketch_twice_in_a_row():
    torch, pkg = cuda()
    st1, got1, ref1 = _pair(torch, pkg, 4096, 256, 512, 1, seed=1, with_b=True)
    st2, got2, ref2 = _pair(torch, pkg, 3001, 37, 100, 3, seed=2, with_b=False)
    assert st1 == 0 and st2 == 0
    assert np.isfinite(got1).all() and np.isfinite(got2).all()
    assert rel_fro(got1, ref1) <= 1e-12
    assert rel_fro(got2, ref2) <= 1e-12


def test_noalloc_sketch_with_the_s_hashing_variant():
    # Def. 7's variant draws with replacement, so s = 5 > m = 3 is a valid sketch
    torch, pkg = cuda()
    st, got, ref = _pair(torch, pkg, 2000, 20, 3, 5, seed=3, with_b=True, hash_kind=1)
    assert st == 0 and np.isfinite(got).all()
    assert rel_fro(got, ref) <= 1e-12


def test_noalloc_sketch_of_a_csr_matrix():
    # the CSR route: SA cleared, then every nonzero added into its s rows
    torch, pkg = cuda()
    n, d = 5000, 60
    rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=4, nnz_row=6, heavy_frac=2e-3, heavy_nnz=40)
    M = pkg.csr_matrix(to_dev(torch, rp), to_dev(torch, ci), to_dev(torch, v), n, d)
    o = pkg.ski_opts_default(m=150, s=2, seed=9)
    for _ in range(2):
        st, got, ref = _run(torch, pkg, M, to_dev(torch, b), o, 150, d + 1, torch.float64)
        assert st == 0 and np.isfinite(got).all()
        assert rel_fro(got, ref) <= 1e-12


def test_noalloc_sketch_in_fp32():
    # FP32 output (FP32 accumulation); the FP32 sketch tolerance of the other tests
    torch, pkg = cuda()
    st, got, ref = _pair(torch, pkg, 6000, 90, 300, 2, seed=6, with_b=True, sketch_dtype=pkg.SKI_F32)
    assert st == 0 and np.isfinite(got).all()
    assert rel_fro(got, ref) <= 1e-6


@pytest.mark.parametrize("s", [1, 4])
def test_noalloc_sketch_at_its_limits(s):
    # rows * s = 262144 and m = 32768, the largest request the fixed array takes
    torch, pkg = cuda()
    st, got, ref = _pair(torch, pkg, 262144 // s, 3, 32768, s, seed=10 + s, with_b=True)
    assert st == 0 and np.isfinite(got).all()
    assert rel_fro(got, ref) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, pkg = cuda()
    A = torch.zeros(300000, 2, dtype=torch.float64, device="cuda")
    SA = torch.zeros(8, 2, dtype=torch.float64, device="cuda")
    M = pkg.dense_matrix(A)
    big_rows = pkg.ski_opts_default(m=8, s=1)
    assert pkg.lib().ski_sketch_hash_noalloc(ctypes.byref(M), None, ctypes.byref(big_rows),
                                             ctypes.c_void_p(SA.data_ptr()), 2, None) == 1
    small = pkg.dense_matrix(A[:100])
    big_m = pkg.ski_opts_default(m=40000, s=1)
    assert pkg.lib().ski_sketch_hash_noalloc(ctypes.byref(small), None, ctypes.byref(big_m),
                                             ctypes.c_void_p(SA.data_ptr()), 2, None) == 1
    premix = pkg.ski_opts_default(m=8, s=1, premix=1)
    assert pkg.lib().ski_sketch_hash_noalloc(ctypes.byref(small), None, ctypes.byref(premix),
                                             ctypes.c_void_p(SA.data_ptr()), 2, None) == 1
