"""The batched form on a ragged batch drawn like the batched workload
(d ~ U{64..1024}, n ~ U{max(2000, 4d)..60000}, A and b i.i.d. N(0,1)), 64
problems in one call: every solve is checked by the oracle's acceptance
metric recomputed on the host, a sample against LAPACK's solution, and the
batched adjoint against the oracle's closed-form gradient."""
import numpy as np
import pytest

from oracle import adjoint as oadj, lsqr as olsqr
from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, rel_fro

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mixed", [False, True])
def test_ragged_batch_of_64(mixed):
    torch, pkg = cuda()
    shapes, As, bs = workloads.ragged_batch_torch(64, 20210525, "cuda")
    prec = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if mixed else {}
    o = pkg.ski_opts_default(m=-2000, s=1, seed=900, tol=1e-10, tau_r=1e-12, **prec)
    mats = [pkg.dense_matrix(a) for a in As]
    xs = [torch.empty(d, dtype=torch.float64, device="cuda") for _, d in shapes]
    Rs = [torch.empty(d, d, dtype=torch.float64, device="cuda") for _, d in shapes]
    infos = pkg.ski_solve_batched(mats, bs, o, xs, R_outs=Rs)
    g = np.random.default_rng(5)
    gs = [torch.from_numpy(g.standard_normal(d)).cuda() for _, d in shapes]
    dAs = [torch.empty_like(a) for a in As]
    dbs = [torch.empty_like(b) for b in bs]
    ainfos = pkg.ski_solve_adjoint_batched(mats, bs, xs, Rs, gs, dAs, dbs, o)
    sample = set(range(0, 64, 16))
    for i, (n, d) in enumerate(shapes):
        assert infos[i].status == 0 and ainfos[i].status == 0, (i, n, d, infos[i].status, ainfos[i].status)
        A, b, x = As[i].cpu().numpy(), bs[i].cpu().numpy(), xs[i].cpu().numpy()
        assert olsqr.residual_metric(A, b, x) <= 1e-10, (i, n, d)
        if i in sample:
            xr = olsqr.lstsq_reference(A, b)
            assert rel_fro(x, xr) <= 1e-8
            dA, db = oadj.lstsq_grad(A, b, xr, gs[i].cpu().numpy())
            assert rel_fro(dAs[i].cpu().numpy(), dA) <= 1e-8
            assert rel_fro(dbs[i].cpu().numpy(), db) <= 1e-8
