"""Host logic of the autotuner: the coordinate search, the cache, the problem
signature and the sample choice (fake timers, no GPU)."""
import json
import math

import pytest

import paper_2105_11815_gb300 as pkg
from paper_2105_11815_gb300 import autotune as at


def _opts(**kw):
    o = pkg.ski_opts()
    o.s, o.m, o.it_max = 1, -2000, 10000
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _mats(shapes):
    return [pkg.ski_matrix(kind=0, n=n, d=d, ld=d, val=4096) for n, d in shapes]


def test_coordinate_search_finds_separable_minimum():
    space = {"a": (0, 1, 2, 3), "b": (5, 6, 7)}
    cost = lambda c: (c["a"] - 2) ** 2 + (c["b"] - 7) ** 2 + 1.0
    best, t, trace = at.coordinate_search(cost, space, rounds=2)
    assert best == {"a": 2, "b": 7} and t == 1.0
    # each configuration is timed once
    keys = [tuple(sorted(c.items())) for c, _ in trace]
    assert len(keys) == len(set(keys))


def test_coordinate_search_never_picks_a_failed_run_and_keeps_ties():
    space = {"a": (0, 1, 2)}
    times = {0: 5.0, 1: math.inf, 2: 5.0}
    best, t, _ = at.coordinate_search(lambda c: times[c["a"]], space)
    assert best == {"a": 0} and t == 5.0        # a tie keeps the incumbent (the default)
    best, t, _ = at.coordinate_search(lambda c: {0: math.inf, 1: math.inf, 2: 3.0}[c["a"]], space)
    assert best == {"a": 2}


def test_coordinate_search_second_round_follows_coupling():
    # b's best value depends on a: one sweep is not enough, two are
    space = {"a": (0, 1), "b": (0, 1)}
    cost = {(0, 0): 4.0, (1, 0): 3.0, (0, 1): 5.0, (1, 1): 1.0}
    best, t, _ = at.coordinate_search(lambda c: cost[(c["a"], c["b"])], space, rounds=2)
    assert best == {"a": 1, "b": 1} and t == 1.0


def test_tune_batched_caches_by_signature(tmp_path):
    path = str(tmp_path / "tune.json")
    mats = _mats([(4000, 64), (20000, 300), (60000, 1000)])
    calls = []

    def timer(cfg):
        calls.append(cfg)
        return 1.0 + 0.1 * cfg["lsqr_pass"] + (0.0 if cfg["streams"] == 4 else 0.5) + 0.01 * cfg["lsqr_ctas"] / 76
    o, rec = at.tune_batched(mats, None, None, _opts(), cache_path=path, timer=timer)
    assert rec["config"] == {"lsqr_pass": 1, "lsqr_ctas": 0, "graphs": 0, "streams": 4} and not rec["cached"]
    assert (o.lsqr_pass, o.lsqr_ctas, o.graphs, o.streams) == (1, 0, 0, 4)
    n = len(calls)
    assert n == rec["trials"]
    stored = json.load(open(path))
    assert rec["signature"] in stored
    # same shapes (same buckets): read back, no timing
    mats2 = _mats([(4050, 65), (21000, 310), (61000, 1010)])
    o2, rec2 = at.tune_batched(mats2, None, None, _opts(), cache_path=path, timer=timer)
    assert rec2["cached"] and len(calls) == n and o2.streams == 4
    # the caller's opts are not modified
    base = _opts()
    at.apply(base, {"streams": 16})
    assert base.streams == 0


def test_signature_separates_what_matters():
    mats = _mats([(4000, 64), (20000, 300)])
    s = at.signature(mats, _opts())
    assert s == at.signature(_mats([(4095, 127), (32767, 511)]), _opts())   # same log2 buckets
    assert s != at.signature(_mats([(4000, 64), (20000, 3000)]), _opts())
    assert s != at.signature(mats, _opts(qr_dtype=1))
    assert s != at.signature(mats, _opts(premix=1))
    assert s != at.signature(mats, _opts(hash_kind=1))
    assert s != at.signature(mats, _opts(), "solve")
    csr = [pkg.ski_matrix(kind=1, n=4000, d=64, ld=0, val=4096, rowptr=4096, colidx=4096, nnz=32000)]
    assert json.loads(at.signature(csr, _opts()))["csr"] == 1


def test_sample_indices_keep_the_costliest_and_the_mix():
    costs = [float(c) for c in range(100)]
    idx = at.sample_indices(costs, 10)
    assert len(idx) == 10 and idx == sorted(idx) and len(set(idx)) == 10
    assert set(range(95, 100)) <= set(idx)          # the costliest half of the sample
    assert min(idx) < 20                              # and cheap problems too
    assert at.sample_indices(costs[:4], 10) == [0, 1, 2, 3]
    assert at.sample_indices(costs, 10) == idx       # deterministic


def test_tuned_fields_are_valid_options():
    for f, values in at.SPACE_BATCHED.items():
        assert f in at.FIELDS
        for v in values:
            assert v >= 0
    assert "streams" not in at.SPACE_SOLVE
