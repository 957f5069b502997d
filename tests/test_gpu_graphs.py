"""The LSQR and CG chunks replayed as captured CUDA graphs (SKI_CHUNK_GRAPHS=1)
give bit-identical results to direct launches.  The switch is read once per
process, so the graph run happens in a child process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2105_11815_gb300 import workloads
from gpu_util import cuda, to_dev

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, %(root)r); sys.path.insert(0, %(tests)r)
import numpy as np, torch
import paper_2105_11815_gb300 as pkg
from paper_2105_11815_gb300 import workloads
A, b, _ = workloads.gaussian_lls(3000, 120, seed=77)
At, bt = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
o = pkg.ski_opts_default(m=240, s=1, seed=5, tol=1e-10, tau_r=1e-12)
x = torch.empty(120, dtype=torch.float64, device="cuda")
R = torch.empty(120, 120, dtype=torch.float64, device="cuda")
info = pkg.ski_solve(pkg.dense_matrix(At), bt, o, x, R_out=R)
g = torch.from_numpy(np.random.default_rng(3).standard_normal(120)).cuda()
dA, db = torch.empty_like(At), torch.empty_like(bt)
ai = pkg.ski_solve_adjoint(pkg.dense_matrix(At), bt, x, R, 120, g, dA, 120, db, o)
print(json.dumps({"x": x.cpu().numpy().tobytes().hex(), "db": db.cpu().numpy().tobytes().hex(),
                  "iters": int(info.iters), "adj": int(ai.iters)}))
"""


def _run(graphs):
    env = dict(os.environ)
    env["SKI_CHUNK_GRAPHS"] = "1" if graphs else "0"
    code = CHILD % {"root": ROOT, "tests": os.path.join(ROOT, "tests")}
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_chunk_graphs_match_direct_launches():
    cuda()
    a, b = _run(False), _run(True)
    assert a == b
