"""Failure detection without a GPU fault: a bounded device-side wait that is
made to run out, and host-side status codes for bad inputs."""
import numpy as np
import pytest

from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    torch, pkg = cuda()
    st = pkg.ski_selftest_wait_timeout(100_000)
    assert st == pkg.STATUS.index("SKI_ETIMEOUT")
    # the context is still usable: a sketch runs and matches the oracle
    from oracle import sketch as osk
    A, b, _ = workloads.gaussian_lls(500, 12, seed=3)
    SA = torch.empty(40, 13, dtype=torch.float64, device="cuda")
    At, bt = to_dev(torch, A), to_dev(torch, b)
    pkg.ski_sketch_hash(pkg.dense_matrix(At), bt, pkg.ski_opts_default(m=40, s=2, seed=1), SA, 13)
    assert rel_fro(SA.cpu().numpy(), osk.sketch_rows(1, 2, 40, A, b)) <= 1e-12


def test_persistent_panel_qr_matches_oracle_on_tall_panel():
    # many CTAs per panel (m = 20000 rows): exercises the grid barrier path
    torch, pkg = cuda()
    from oracle import qr as oqr
    g = np.random.default_rng(4)
    m, d = 20000, 70
    B = g.standard_normal((m, d + 1))
    SA = to_dev(torch, B)
    R = torch.empty(d, d, dtype=torch.float64, device="cuda")
    qtsb = torch.empty(d, dtype=torch.float64, device="cuda")
    rank = pkg.ski_precondition(m, d, 1, SA, d + 1, 0, R, d, qtsb)
    Ro, C = oqr.householder_qr(B, ncols=d)
    Rg = R.cpu().numpy()
    sf = np.sign(np.diag(Rg))[:, None]
    so = np.sign(np.diag(Ro))[:, None]
    assert rank == d
    assert rel_fro(sf * Rg, so * Ro) <= 1e-12
