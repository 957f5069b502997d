"""Full-size solves in the launch configuration the benchmark times, checked
by properties that hold at any size.  The oracle's step-by-step solve takes
minutes at these sizes, so the acceptance criterion is recomputed on the host
in FP64 from the returned x: ||A^T r|| / (||A||_F ||r||) <= 1e-10 with
r = b - A x (the FP64 acceptance test of Algorithm 1 as the library reads it).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, to_dev

pytestmark = pytest.mark.gpu


def _metric_dense(A, b, x):
    r = b - A @ x
    return np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r))


@pytest.mark.parametrize("mixed", [False, True])
def test_dense_test_set_solve_full_size(mixed):
    # n = 50000, d = 4000, premix to 65536, s = 1, m = 2d (the benchmark's
    # workload), FP64 and the mixed form (FP32 sketch, three-pass TF32 QR)
    torch, pkg = cuda()
    n, d = 50000, 4000
    At, bt = workloads.gaussian_torch(n, d, 20210525, "cuda")
    kw = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    o = pkg.ski_opts_default(m=2 * d, s=1, seed=20210525, premix=1, n_pad=65536, tol=1e-10, tau_r=1e-10, **kw)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x)
    assert info.status == 0 and info.metric <= 1e-10
    if mixed:
        assert info.qr_fallback == 0      # i.i.d. Gaussian: the FP32 factor preconditions
    A = At.cpu().numpy()
    assert _metric_dense(A, bt.cpu().numpy(), x.cpu().numpy()) <= 1e-10


def test_sparse_solve_full_size_mixed():
    # CSR 1e6 x 20000 with 8 nonzeros per row and 0.1% rows of 2000, s = 2,
    # m = 2d, mixed form
    torch, pkg = cuda()
    n, d = 1_000_000, 20000
    rp, ci, v, b = workloads.csr_heavy_rows(n, d, seed=20210525)
    M = pkg.csr_matrix(to_dev(torch, rp), to_dev(torch, ci), to_dev(torch, v), n, d)
    o = pkg.ski_opts_default(m=2 * d, s=2, seed=20210525, tol=1e-10, tau_r=1e-10, sketch_dtype=pkg.SKI_F32,
                             qr_dtype=pkg.SKI_F32)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(M, to_dev(torch, b), o, x)
    assert info.status == 0 and info.metric <= 1e-10
    A = sp.csr_matrix((v, ci, rp), shape=(n, d))
    xh = x.cpu().numpy()
    r = b - A @ xh
    metric = np.linalg.norm(A.T @ r) / (np.sqrt(np.sum(v * v)) * np.linalg.norm(r))
    assert metric <= 1e-10
