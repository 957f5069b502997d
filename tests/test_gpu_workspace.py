"""The workspace is scratch: every entry point must give bit-identical results
whatever the workspace held before the call (zeros, NaNs or another solve's
leftovers).  A read of a scratch word before the kernels write it shows up
here as a difference."""
import numpy as np
import pytest

from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, to_dev

pytestmark = pytest.mark.gpu

FILLS = (0x00, 0xFF, 0x7F)   # zeros, all-ones bytes (NaN doubles), large finite values


def _filled(torch, nbytes, byte):
    return torch.full((max(int(nbytes), 1),), byte, dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("n,d,premix", [(1500, 37, 0), (2999, 120, 0), (700, 8, 0), (3000, 101, 1)])
def test_sketch_independent_of_workspace(n, d, premix):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(m=2 * d + 3, s=2, seed=4, premix=premix)
    mat = pkg.dense_matrix(At)
    nb = pkg.ski_sketch_workspace_size(mat, 1, o)
    outs = []
    for f in FILLS:
        SA = torch.zeros(o.m, d + 1, dtype=torch.float64, device="cuda")
        pkg.ski_sketch_hash(mat, bt, o, SA, d + 1, ws=_filled(torch, nb, f))
        outs.append(SA)
    for y in outs[1:]:
        assert torch.equal(y, outs[0])


@pytest.mark.parametrize("m,d,dt", [(200, 37, 0), (240, 120, 0), (2000, 1001, 0), (240, 120, 1), (2000, 1001, 1)])
def test_precondition_independent_of_workspace(m, d, dt):
    torch, pkg = cuda()
    g = np.random.default_rng(m + d)
    SAh = g.standard_normal((m, d + 1))
    nb = pkg.ski_precondition_workspace_size(m, d, 1, dt)
    outs = []
    for f in FILLS:
        tdt = torch.float64 if dt == 0 else torch.float32
        SA = torch.from_numpy(SAh).to(tdt).cuda()
        R = torch.zeros(d, d, dtype=torch.float64, device="cuda")
        q = torch.zeros(d, dtype=torch.float64, device="cuda")
        pkg.ski_precondition(m, d, 1, SA, d + 1, dt, R, d, q, ws=_filled(torch, nb, f))
        outs.append((R, q))
    for R, q in outs[1:]:
        assert torch.equal(R, outs[0][0]) and torch.equal(q, outs[0][1])


@pytest.mark.parametrize("d,dt", [(37, 0), (120, 0), (1001, 0), (257, 1)])
def test_trinv_independent_of_workspace(d, dt):
    torch, pkg = cuda()
    g = np.random.default_rng(d)
    R = np.triu(g.standard_normal((d, d))) + 4 * np.sqrt(d) * np.eye(d)
    Rt = to_dev(torch, R)
    nb = pkg.ski_trinv_workspace_size(d, dt)
    outs = []
    for f in FILLS:
        M = torch.zeros(d, d, dtype=torch.float64, device="cuda")
        Mt = torch.zeros(d, d, dtype=torch.float64, device="cuda")
        pkg.ski_trinv(d, Rt, d, M, Mt, d, dt, ws=_filled(torch, nb, f))
        outs.append((M, Mt))
    for M, Mt in outs[1:]:
        assert torch.equal(M, outs[0][0]) and torch.equal(Mt, outs[0][1])


@pytest.mark.parametrize("n,d,qr", [(1500, 37, 0), (2999, 120, 0), (700, 8, 0), (2500, 101, 1), (4000, 300, 0)])
def test_solve_independent_of_workspace(n, d, qr):
    torch, pkg = cuda()
    A, b, _ = workloads.gaussian_lls(n, d, seed=n + 1)
    At, bt = to_dev(torch, A), to_dev(torch, b)
    o = pkg.ski_opts_default(m=2 * d, s=1, seed=6, tol=1e-10, tau_r=1e-12, qr_dtype=qr, sketch_dtype=qr)
    mat = pkg.dense_matrix(At)
    nb = pkg.ski_solve_workspace_size(mat, o)
    xs, its = [], []
    for f in FILLS:
        x = torch.zeros(d, dtype=torch.float64, device="cuda")
        info = pkg.ski_solve(mat, bt, o, x, ws=_filled(torch, nb, f))
        xs.append(x)
        its.append(info.iters)
    assert len(set(its)) == 1, its
    for x in xs[1:]:
        assert torch.equal(x, xs[0])
