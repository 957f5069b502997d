"""The sketch-size calibration (the U-curve of the paper's calibration
experiments, Section 7 and Appendices B-C) on the GPU: every grid point is a
real solve that meets the acceptance test, the iteration count falls as gamma
grows (Theorem 10: the distortion shrinks with m), and the chosen point is
the fastest accepted one."""
import pytest

from oracle import lsqr as olsqr
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, to_dev

pytestmark = pytest.mark.gpu


def test_u_curve_on_the_gpu():
    torch, pkg = cuda()
    from paper_2105_11815_gb300 import calibrate as cal
    n, d = 20000, 300
    A, b = workloads.dense_gaussian(n, d, seed=3)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(seed=5, premix=1, n_pad=32768, tol=1e-10, tau_r=1e-10)
    gammas = [1.2, 2.0, 4.0]
    recs = cal.u_curve(pkg.dense_matrix(At), bt, o, gammas, [1, 2], reps=2)
    assert len(recs) == 6
    for r in recs:
        assert r["status"] == 0 and r["metric"] <= 1e-10 and r["ms"] > 0, r
        assert r["m"] == cal.sketch_rows_for(r["gamma"], d, r["s"])
    for s in (1, 2):
        its = [r["iters"] for r in recs if r["s"] == s]
        assert its[0] > its[1] > its[2], its
    best = cal.best(recs)
    assert best["ms"] == min(r["ms"] for r in recs)
    # the solve at the chosen point is the least-squares solution
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    ob = pkg.ski_opts_default(seed=5, premix=1, n_pad=32768, tol=1e-10, tau_r=1e-10, m=best["m"], s=best["s"])
    pkg.ski_solve(pkg.dense_matrix(At), bt, ob, x)
    assert olsqr.residual_metric(A, b, x.cpu().numpy()) <= 1e-10
