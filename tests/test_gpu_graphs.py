"""Launch parameters of Steps 4-5 (ski_opts.graphs, lsqr_pass, lsqr_ctas), the
knobs the autotuner picks, change the work split, not the method.

- Chunks of LSQR and CG iterations replayed as captured CUDA graphs give
  bit-identical results to direct launches (the same kernels in the same order).
- The LSQR pass variants and CTA counts sum in other orders, so they agree to
  rounding: every solve meets the tolerance, and the solutions agree within a
  few units of the conditioning-scaled rounding error.
"""
import numpy as np
import pytest

from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, to_dev

pytestmark = pytest.mark.gpu


def _solve_and_adjoint(torch, pkg, **kw):
    A, b, _ = workloads.gaussian_lls(3000, 120, seed=77)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(m=240, s=1, seed=5, tol=1e-10, tau_r=1e-12, **kw)
    x = torch.empty(120, dtype=torch.float64, device="cuda")
    R = torch.empty(120, 120, dtype=torch.float64, device="cuda")
    info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x, R_out=R)
    g = to_dev(torch, np.random.default_rng(3).standard_normal(120))
    dA, db = torch.empty_like(At), torch.empty_like(bt)
    ai = pkg.ski_solve_adjoint(pkg.dense_matrix(At), bt, x, R, 120, g, dA, 120, db, o)
    return x.cpu().numpy(), db.cpu().numpy(), info, ai


def test_chunk_graphs_match_direct_launches():
    torch, pkg = cuda()
    x0, db0, i0, a0 = _solve_and_adjoint(torch, pkg, graphs=0)
    x1, db1, i1, a1 = _solve_and_adjoint(torch, pkg, graphs=1)
    assert np.array_equal(x0, x1) and np.array_equal(db0, db1)
    assert (i0.iters, a0.iters) == (i1.iters, a1.iters)


@pytest.mark.parametrize("lsqr_pass,lsqr_ctas", [(1, 0), (2, 0), (3, 0), (1, 7), (2, 300), (3, 1), (4, 0), (5, 0), (5, 7), (5, 300)])
def test_lsqr_pass_variants_agree(lsqr_pass, lsqr_ctas):
    torch, pkg = cuda()
    x0, db0, i0, _ = _solve_and_adjoint(torch, pkg)
    x1, db1, i1, a1 = _solve_and_adjoint(torch, pkg, lsqr_pass=lsqr_pass, lsqr_ctas=lsqr_ctas)
    assert i1.status == 0 and i1.metric <= 1e-10
    assert a1.status == 0
    assert np.linalg.norm(x1 - x0) <= 1e-9 * np.linalg.norm(x0)
    assert np.linalg.norm(db1 - db0) <= 1e-8 * np.linalg.norm(db0)
