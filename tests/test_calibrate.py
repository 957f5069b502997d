"""Host logic of the sketch-size calibration (fake solves, no GPU)."""
import math

import paper_2105_11815_gb300 as pkg
from paper_2105_11815_gb300 import calibrate as cal


class _Info:
    def __init__(self, ms, status=0, iters=10):
        self.ms_total, self.status, self.iters = ms, status, iters
        self.restarts = self.qr_fallback = 0
        self.metric = 1e-11
        self.ms_sketch = self.ms_qr = self.ms_trinv = self.ms_lsqr = 0.0


def test_sketch_rows_for():
    assert cal.sketch_rows_for(1.7, 4000, 1) == 6800
    assert cal.sketch_rows_for(1.25, 3, 1) == 4
    assert cal.sketch_rows_for(0.5, 100, 1) == 100     # m >= d (Step 2)
    assert cal.sketch_rows_for(1.0, 2, 5) == 5         # m >= s
    assert cal.sketch_rows_for(2.0, 4000, 2) == 8000   # no rounding up of an exact product


def test_u_curve_times_each_point_and_picks_the_fastest_accepted():
    d = 1000
    A = pkg.ski_matrix(kind=0, n=20000, d=d, ld=d, val=4096)
    o = pkg.ski_opts_default(seed=3)
    calls = []

    def solve(op):
        calls.append((op.m, op.s))
        # QR cost grows with m, LSQR cost falls as the distortion shrinks: a U
        g = op.m / d
        ms = 10.0 * g + 40.0 / math.log(1.0 + g) + (0.5 if op.s == 2 else 0.0) + 0.01 * (len(calls) % 3)
        return _Info(ms, status=1 if (g > 2.9) else 0)
    recs = cal.u_curve(A, None, o, [1.2, 1.7, 2.0, 3.0], [1, 2], reps=3, solve=solve)
    # one warm-up and 3 timed solves per point; a failed solve ends its point
    assert len(recs) == 8 and len(calls) == 6 * 4 + 2 * 2
    assert [(r["s"], r["gamma"]) for r in recs] == [(s, g) for s in (1, 2) for g in (1.2, 1.7, 2.0, 3.0)]
    assert all(r["m"] == cal.sketch_rows_for(r["gamma"], d, r["s"]) for r in recs)
    failed = [r for r in recs if r["gamma"] == 3.0]
    assert all(r["status"] == 1 and r["ms"] is None for r in failed)
    b = cal.best(recs)
    ok = [r for r in recs if r["status"] == 0]
    assert b["ms"] == min(r["ms"] for r in ok) and b["s"] == 1
    # the fastest of the timed repetitions is kept
    g17 = next(r for r in recs if r["gamma"] == 1.7 and r["s"] == 1)
    assert math.isclose(g17["ms"], 17.0 + 40.0 / math.log(2.7), abs_tol=1e-9)
    # the caller's opts are not modified
    assert o.m == 0 and o.s == 1


def test_best_of_nothing_accepted_is_none():
    assert cal.best([{"status": 6, "ms": None, "gamma": 1.0, "s": 1}]) is None
