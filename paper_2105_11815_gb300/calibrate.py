"""Runtime calibration of the sketch size m = gamma * d and of the hashing
sparsity s: the U-curve procedure of the paper's calibration experiments
(Section 7 and Appendices B-C), timed on this GPU.

The cost of Steps 1-2 (sketch and QR) grows with m, while the number of LSQR
iterations falls as m grows, because the embedding distortion epsilon shrinks
(Theorem 10 bounds the iterations by (log 2 + |log tau_r|) / |log epsilon|).
The solve time against gamma is therefore U-shaped. Its minimiser depends on
the relative speed of the QR and of the pass over A on the machine. The paper
calibrated on CPUs (gamma = 1.7 for dense problems; m = 1.4 d with s = 2 for
sparse ones). On this GPU the FP64 QR is slow against the pass over A, while
the mixed-precision QR is fast, so the minimiser is measured rather than
taken from those figures.

``u_curve`` solves the caller's problem for each (gamma, s) on a grid and
records each solve's time, iteration count and acceptance metric. ``best``
picks the fastest accepted point. ``python -m paper_2105_11815_gb300.calibrate``
runs the sweep on the seeded synthetic workloads and prints one JSON line per
point, then one for the minimiser.
"""
import argparse
import json
import math


def sketch_rows_for(gamma, d, s):
    """m = ceil(gamma * d), at least d (Step 2 needs m >= d) and at least s."""
    return max(int(math.ceil(gamma * d - 1e-9)), int(d), int(s))


def u_curve(A, b, opts, gammas, ss, reps=2, solve=None):
    """Time the solve of (A, b) for every (gamma, s) in gammas x ss.

    A: a ski_matrix; b: the device right-hand side; opts: a ski_opts whose m
    and s are overwritten per point.  Each point is solved once untimed, then
    ``reps`` times; its time is the fastest ``ms_total`` (the library's own
    CUDA-event time of the whole solve).  solve(opts) -> ski_info replaces the
    GPU solve (tests).  Returns a list of dicts in grid order.
    """
    from . import autotune
    if solve is None:
        import torch
        import paper_2105_11815_gb300 as pkg
        x = torch.empty(int(A.d), dtype=torch.float64, device="cuda")

        def solve(o):
            return pkg.ski_solve(A, b, o, x, check=False)
    out = []
    for s in ss:
        for g in gammas:
            m = sketch_rows_for(g, int(A.d), s)
            o = autotune.apply(opts, {"m": m, "s": int(s)})
            solve(o)
            best_ms, info = math.inf, None
            for _ in range(max(1, reps)):
                inf = solve(o)
                if int(inf.status) != 0:
                    info, best_ms = inf, math.inf
                    break
                if float(inf.ms_total) < best_ms:
                    best_ms, info = float(inf.ms_total), inf
            out.append({
                "gamma": float(g), "s": int(s), "m": m, "status": int(info.status),
                "ms": best_ms if int(info.status) == 0 else None,
                "iters": int(info.iters), "restarts": int(info.restarts), "metric": float(info.metric),
                "ms_sketch": float(info.ms_sketch), "ms_qr": float(info.ms_qr), "ms_trinv": float(info.ms_trinv),
                "ms_lsqr": float(info.ms_lsqr), "qr_fallback": int(info.qr_fallback),
            })
    return out


def best(records):
    """The fastest record whose solve was accepted (status 0), or None."""
    ok = [r for r in records if r["status"] == 0 and r["ms"] is not None]
    return min(ok, key=lambda r: (r["ms"], r["gamma"], r["s"])) if ok else None


def _parse_list(text, conv):
    return [conv(v) for v in text.split(",") if v.strip()]


def main(argv=None):
    ap = argparse.ArgumentParser(description="Runtime U-curve of the sketch size on this GPU")
    ap.add_argument("--kind", choices=("dense", "csr"), default="dense")
    ap.add_argument("--n", type=int, default=50000)
    ap.add_argument("--d", type=int, default=4000)
    ap.add_argument("--premix", type=int, default=1, help="dense only: the Walsh-Hadamard premix (Def. 8)")
    ap.add_argument("--mixed", type=int, default=0, help="1: FP32 sketch and three-pass TF32 QR")
    ap.add_argument("--gammas", default="1.2,1.4,1.7,2,2.5,3")
    ap.add_argument("--ss", default="1,2")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--seed", type=int, default=20210525)
    args = ap.parse_args(argv)

    import torch
    import paper_2105_11815_gb300 as pkg
    from . import workloads
    n, d = args.n, args.d
    kw = dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32) if args.mixed else {}
    keep = []
    if args.kind == "dense":
        A, b = workloads.gaussian_torch(n, d, args.seed, "cuda")
        keep += [A, b]
        M = pkg.dense_matrix(A)
        n_pad = 1 << max(0, (n - 1).bit_length())
        opts = pkg.ski_opts_default(seed=args.seed, premix=args.premix, n_pad=n_pad if args.premix else 0,
                                    tol=1e-10, tau_r=1e-10, **kw)
        label = "dense_%dx%d%s" % (n, d, "_hrht" if args.premix else "")
    else:
        rp, ci, v, bh = workloads.csr_heavy_rows(n, d, seed=args.seed)
        keep += [torch.from_numpy(a).cuda() for a in (rp, ci, v, bh)]
        M = pkg.csr_matrix(keep[0], keep[1], keep[2], n, d)
        b = keep[3]
        opts = pkg.ski_opts_default(seed=args.seed, tol=1e-10, tau_r=1e-10, **kw)
        label = "csr_%dx%d" % (n, d)
    recs = u_curve(M, b, opts, _parse_list(args.gammas, float), _parse_list(args.ss, int), reps=args.reps)
    form = "mixed" if args.mixed else "fp64"
    for r in recs:
        print(json.dumps(dict(workload=label, form=form, **r)))
    print(json.dumps({"workload": label, "form": form, "best": best(recs)}))


if __name__ == "__main__":
    main()
