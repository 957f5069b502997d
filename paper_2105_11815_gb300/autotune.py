"""Autotuner for the launch parameters of the solve (batched and single).

The library exposes, as ``ski_opts`` fields, the parameters that change how
Steps 4-5 and the batched entry point run but not what they compute:

- ``lsqr_pass``: which kernel runs the dense LSQR pass. 1 is register-blocked
  rows, 2 a TMA-staged row ring, 3 one row per warp, 4 register-blocked rows
  with twice the rows between the two barriers of a row group, 5
  register-blocked rows with the next row group's loads in flight.
- ``lsqr_ctas``: its row tiles, i.e. the number of CTAs. 0 is the library
  default.
- ``graphs``: replay each chunk of iterations as a CUDA graph (1) or launch
  it (0).
- ``streams``: problems in flight in ``ski_solve_batched``.

The best values depend on the problem shapes (n, d, the ragged mix) and on the
GPU, so they are measured rather than modelled. ``tune_batched`` and
``tune_solve`` time candidate settings on the caller's own problems:
- one coordinate at a time, starting from the defaults, for a fixed number of
  rounds;
- each setting timed as the best of ``reps`` runs, after one warm-up run;
- the winner cached in a JSON file under a signature of the problem shapes, so
  a later call with the same signature reads it back without timing.

Every candidate computes the same solution up to rounding. The tuner
therefore checks only the status of each timed run. A setting whose run fails
is never chosen.
"""
import json
import math
import os
import tempfile
import time

import numpy as np

# Candidate values per field, the default first.
SPACE_BATCHED = {
    "lsqr_pass": (1, 2, 3, 4, 5),
    "lsqr_ctas": (0, 19, 38, 76, 304, 608),  # few CTAs: passes of different problems share the SMs
    "graphs": (0, 1),
    "streams": (8, 1, 2, 4, 16),
}
SPACE_SOLVE = {k: v for k, v in SPACE_BATCHED.items() if k != "streams"}
FIELDS = ("lsqr_pass", "lsqr_ctas", "graphs", "streams")


def _bucket(v):
    """Power-of-two bucket of a positive size (the signature's resolution)."""
    return int(math.floor(math.log2(max(1, int(v)))))


def signature(mats, opts, kind="batched"):
    """A string key for the shapes and the options that matter to the timing:
    the number of problems and the log2 buckets of the smallest, median and
    largest n and d, the sketch size rule, s, the premix, the dtypes, and the
    sketching matrix (s-hashing or its variant)."""
    ns = sorted(int(a.n) for a in mats)
    ds = sorted(int(a.d) for a in mats)
    nnz = sorted(int(a.nnz) if int(a.kind) == 1 else 0 for a in mats)

    def q(v):
        return [_bucket(v[0]), _bucket(v[len(v) // 2]), _bucket(v[-1])]
    key = {
        "kind": kind, "count": _bucket(len(mats)), "csr": int(any(int(a.kind) == 1 for a in mats)),
        "n": q(ns), "d": q(ds), "nnz": q(nnz) if nnz[-1] else 0,
        "m": int(opts.m) if int(opts.m) <= 0 else _bucket(int(opts.m)), "s": int(opts.s),
        "premix": int(opts.premix), "sketch": int(opts.sketch_dtype), "qr": int(opts.qr_dtype),
        "hash": int(opts.hash_kind),
    }
    return json.dumps(key, sort_keys=True)


def coordinate_search(evaluate, space, rounds=2, start=None):
    """Minimise evaluate(config) over the product of ``space`` one field at a
    time (fields in the order of ``space``), ``rounds`` sweeps.

    evaluate returns seconds, or math.inf for a failed run.  Ties keep the
    incumbent, so the result is deterministic for a deterministic evaluate.
    Returns (best config, its time, trace of (config, time) in order)."""
    cur = dict(start) if start else {k: v[0] for k, v in space.items()}
    seen = {}
    trace = []

    def ev(cfg):
        key = tuple(sorted(cfg.items()))
        if key not in seen:
            t = evaluate(dict(cfg))
            seen[key] = t
            trace.append((dict(cfg), t))
        return seen[key]

    best = ev(cur)
    for _ in range(rounds):
        changed = False
        for f, values in space.items():
            for v in values:
                if v == cur[f]:
                    continue
                cand = dict(cur)
                cand[f] = v
                t = ev(cand)
                if t < best:
                    best, cur, changed = t, cand, True
        if not changed:
            break
    return cur, best, trace


class Cache:
    """JSON file {signature: {"config": {...}, "seconds": t, "trials": k}}."""

    def __init__(self, path):
        self.path = path
        self.data = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, key):
        rec = self.data.get(key)
        return dict(rec["config"]) if rec else None

    def put(self, key, config, seconds, trials):
        self.data[key] = {"config": dict(config), "seconds": seconds, "trials": trials}
        if not self.path:
            return
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune.")
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def apply(opts, config):
    """A copy of ``opts`` with the tuned fields set."""
    o = type(opts)()
    for name, _ in type(opts)._fields_:
        setattr(o, name, getattr(opts, name))
    for k, v in config.items():
        setattr(o, k, int(v))
    return o


def sample_indices(costs, k):
    """Up to k problem indices: the costliest half, the rest evenly spread
    over the remaining ones (in cost order), so the sample has the batch's mix."""
    order = list(np.argsort(-np.asarray(costs, dtype=np.float64), kind="stable"))
    if k >= len(order):
        return sorted(order)
    top = order[: k // 2]
    rest = order[k // 2:]
    step = len(rest) / float(k - len(top))
    spread = [rest[int(i * step)] for i in range(k - len(top))]
    return sorted(int(i) for i in top + spread)


def _problem_cost(a, m):
    nnz = float(a.nnz) if int(a.kind) == 1 else float(a.n) * float(a.d)
    return 57.0 * nnz + float(m) * float(a.d) ** 2


def _gpu_timer(run, reps):
    """Best of reps wall times of run() (which synchronises), after one warm-up."""
    import torch
    run()
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(reps):
        t0 = time.perf_counter()
        ok = run()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if not ok:
            return math.inf
        best = min(best, t)
    return best


def tune_batched(mats, bs, xs, opts, cache_path=None, sample=16, reps=2, rounds=2, space=None, timer=None):
    """Launch parameters for ski_solve_batched on these problems.

    mats, bs, xs: the batch as passed to ski_solve_batched.  The timed runs
    solve a sample of up to ``sample`` problems (see sample_indices) into
    scratch copies of their x.  timer(config) -> seconds replaces the GPU
    timing (tests).  Returns (tuned opts, record) with record = {"signature",
    "config", "seconds", "trials", "cached"}."""
    space = space or SPACE_BATCHED
    key = signature(mats, opts, "batched")
    cache = Cache(cache_path)
    hit = cache.get(key)
    if hit is not None:
        return apply(opts, hit), {"signature": key, "config": hit, "cached": True}
    if timer is None:
        import paper_2105_11815_gb300 as pkg
        m_of = [int(opts.m) if int(opts.m) > 0 else int(math.ceil(max(1, -int(opts.m) or 2000) / 1000.0 * int(a.d)))
                for a in mats]
        idx = sample_indices([_problem_cost(a, m) for a, m in zip(mats, m_of)], sample)
        sm, sb = [mats[i] for i in idx], [bs[i] for i in idx]
        sx = [xs[i].clone() for i in idx]

        def run_cfg(cfg):
            def run():
                infos = pkg.ski_solve_batched(sm, sb, apply(opts, cfg), sx, check=False)
                return all(int(i.status) == 0 for i in infos)
            return _gpu_timer(run, reps)
        timer = run_cfg
    best, t, trace = coordinate_search(timer, space, rounds=rounds)
    cache.put(key, best, t, len(trace))
    return apply(opts, best), {"signature": key, "config": best, "seconds": t, "trials": len(trace), "cached": False}


def tune_solve(A, b, x, opts, cache_path=None, reps=2, rounds=2, space=None, timer=None):
    """Launch parameters for ski_solve on one problem shape (streams does not
    apply); same contract as tune_batched."""
    space = space or SPACE_SOLVE
    key = signature([A], opts, "solve")
    cache = Cache(cache_path)
    hit = cache.get(key)
    if hit is not None:
        return apply(opts, hit), {"signature": key, "config": hit, "cached": True}
    if timer is None:
        import paper_2105_11815_gb300 as pkg
        xx = x.clone()

        def run_cfg(cfg):
            def run():
                return int(pkg.ski_solve(A, b, apply(opts, cfg), xx, check=False).status) == 0
            return _gpu_timer(run, reps)
        timer = run_cfg
    best, t, trace = coordinate_search(timer, space, rounds=rounds)
    cache.put(key, best, t, len(trace))
    return apply(opts, best), {"signature": key, "config": best, "seconds": t, "trials": len(trace), "cached": False}
