#!/usr/bin/env python3
"""Benchmark of the Ski-LLS hot path on one GB300 (or N replicas).

One step = Algorithm 1 end to end on the dense least-squares workload of the
paper's dense test set: A = 50000 x 4000 i.i.d. N(0,1), b = ones, randomised
Walsh-Hadamard premix to n_pad = 65536, 1-hashing with m = 2d = 8000, solved
twice -- all-FP64 (sketch, premix, QR, R^{-1} in FP64) and mixed (premix,
sketch, QR, R^{-1} in FP32; LSQR, residuals and scalars in FP64) -- each to
||A^T r|| / (||A||_F ||r||) <= 1e-10.

Headline metric: sketch S*A GB/s of the FP64 path = (bytes of A and b read +
bytes of [SA | Sb] written) / time of the sketch stage (premix + hash), with
the time-to-1e-10 of both solves reported beside it.  Inputs are resident in
HBM and larger than L2 (1.6 GB vs 129 MB), so no flush is needed.

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload (a slice of A's columns) -- the slow reference arm.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sketch S·A GB/s (% HBM peak); LLS time-to-1e-10 residual, mixed vs FP64"

WORKLOADS = {
    # name: (n, d, n_pad, s, gamma, kind)
    "dense_50000x4000_hrht_s1_g2": (50000, 4000, 65536, 1, 2.0, "gauss"),
    "dense_50000x4000_hrht_s2_g2": (50000, 4000, 65536, 2, 2.0, "gauss"),
    "dense_50000x7000_hrht_s1_g2": (50000, 7000, 65536, 1, 2.0, "gauss"),
    "dense_50000x4000_coherent_hrht_s2_g2": (50000, 4000, 65536, 2, 2.0, "coh"),
    "dense_4096x256_s1_m512": (4096, 256, 0, 1, 2.0, "lls"),
    # small case for ncu captures: same kernels, A = 205 MB (larger than L2)
    "dense_50000x512_hrht_s1_g2": (50000, 512, 65536, 1, 2.0, "gauss"),
    # mid case for full ncu captures of the d = 4000 kernel variants (~4.5 GB on the device)
    "dense_32768x3000_hrht_s1_g2": (32768, 3000, 32768, 1, 2.0, "gauss"),
}
DEFAULT = "dense_50000x4000_hrht_s1_g2"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j.get("hbm_gbs", 6800.0), "measured", j
    return 6800.0, "fallback", {}


# FP64 peak from the unit count and clock: 152 SMs x 2 DFMA/clk x 2 flop x
# 2.07 GHz = 1.26 TFLOP/s (a DFMA loop measured 1.00 on this machine).
FP64_PEAK_TFLOPS = 1.26
FP32_PEAK_TFLOPS = 72.0
# DRAM bytes (read + write) of one launch of the hash gather, from ncu
# (profiles/hash_gather_dense_50000x4000.md); None where not captured.
GATHER_TRAFFIC = {"dense_50000x4000_hrht_s1_g2": 2512025088 + 236451840}


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_problem(name, seed):
    from paper_2105_11815_gb300 import workloads
    n, d, npad, s, gamma, kind = WORKLOADS[name]
    if kind == "gauss":
        A, b = workloads.dense_gaussian(n, d, seed)
    elif kind == "coh":
        A, b = workloads.dense_high_coherence(n, d, seed)
    else:
        A, b, _ = workloads.gaussian_lls(n, d, seed)
    return A, b, dict(n=n, d=d, n_pad=npad, s=s, m=int(round(gamma * d)), gamma=gamma, kind=kind)


def sketch_bytes(cfg):
    n, d, m = cfg["n"], cfg["d"], cfg["m"]
    return 8.0 * (n * d + n + m * (d + 1))


def oracle_sample(A, b, cfg, cols, seed):
    """Time the CPU oracle's sketch on A[:, :cols] (the bounded CPU sample)."""
    from oracle import sketch as osk, wht as owht
    Asub = A[:, :cols].copy()
    t0 = time.perf_counter()
    if cfg["n_pad"]:
        owht.hrht_sketch(seed, cfg["s"], cfg["m"], Asub, b, cfg["n_pad"])
    else:
        osk.sketch_rows(seed, cfg["s"], cfg["m"], Asub, b)
    dt = time.perf_counter() - t0
    nbytes = 8.0 * (cfg["n"] * cols + cfg["n"] + cfg["m"] * (cols + 1))
    return nbytes / dt / 1e9, dt


def run_reference(args, name):
    rank, world, _ = dist_init(args.gpus)
    if rank != 0:
        return
    A, b, cfg = make_problem(name, args.seed)
    cols = args.ref_cols
    for _ in range(args.warmup):
        oracle_sample(A, b, cfg, cols, args.seed)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt = oracle_sample(A, b, cfg, cols, args.seed)
        vals.append(v)
        times.append(dt)
    value = statistics.mean(vals)
    sample = "oracle HRHT sketch (numpy FP64) of A[:, :%d] (%d x %d) + b, m=%d, s=%d" % (
        cols, cfg["n"], cols, cfg["m"], cfg["s"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, **cfg},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, name):
    import numpy as np
    import torch

    import paper_2105_11815_gb300 as pkg
    from paper_2105_11815_gb300 import build

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    pkg.lib()
    A, b, cfg = make_problem(name, args.seed + rank)
    n, d, m, s, npad = cfg["n"], cfg["d"], cfg["m"], cfg["s"], cfg["n_pad"]
    At = torch.from_numpy(A).cuda()
    bt = torch.from_numpy(b).cuda()
    Amat = pkg.dense_matrix(At)
    # LSQR stops on Eq. TC-lsqr at tau_r = 1e-10; the FP64 acceptance test
    # ||A^T r|| / (||A||_F ||r||) <= 1e-10 is then checked (warm restart if not)
    common = dict(m=m, s=s, seed=args.seed, premix=1 if npad else 0, n_pad=npad, tol=1e-10, tau_r=1e-10)
    o64 = pkg.ski_opts_default(**common)
    omx = pkg.ski_opts_default(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32, **common)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(pkg.ski_solve_workspace_size(Amat, o64), pkg.ski_solve_workspace_size(Amat, omx)),
                     dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        i64 = pkg.ski_solve(Amat, bt, o64, x, ws=ws)
        imx = pkg.ski_solve(Amat, bt, omx, x, ws=ws)
        return i64, imx

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.ski_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    ev0.record(stream)
    infos = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = pkg.ski_launch_count() - l0
    clk = clocks.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = total_ms / args.steps

    sb = sketch_bytes(cfg)
    sk_ms = max_over_ranks(statistics.mean(i.ms_sketch for i, _ in infos), world)
    value = world * sb / (sk_ms * 1e-3) / 1e9
    hbm, peak_kind, pj = peaks()
    # the hash gather kernel: reads the premixed Y (n_pad x (d+1)) once per nonzero, writes [SA | Sb]
    rows = npad if npad else n
    gather_bytes = 8.0 * (s * rows * (d + 1) + m * (d + 1))
    g_ms = statistics.mean(i.ms_gather for i, _ in infos)
    pm_ms = statistics.mean(i.ms_premix for i, _ in infos)
    premix_bytes = 8.0 * (n * (d + 1) + npad * (d + 1)) if npad else 0.0
    qr_flops = 2.0 * m * (d + 1) ** 2 - 2.0 / 3.0 * d ** 3
    qr64 = statistics.mean(i.ms_qr for i, _ in infos)
    qrmx = statistics.mean(j.ms_qr for _, j in infos)
    # dominant kernel of the step (ncu launch list): the FP64 QR trailing-update
    # GEMM k_gemm<double>, bound by the FP64 pipe.  Its flops, summed over the
    # 32-column panels: W = V^T C and C -= V B' each cost 2 w nct mr.
    gemm_flops = 0.0
    for k0 in range(0, d, 32):
        w = min(32, d - k0)
        gemm_flops += 4.0 * w * ((d + 1) - k0 - w) * (m - k0)
    g64 = statistics.mean(i.ms_qr_gemm for i, _ in infos)
    g32 = statistics.mean(j.ms_qr_gemm for _, j in infos)
    roofline = {"kernel": "k_gemm<double> (FP64 QR trailing update)", "bound": "alu",
                "achieved": gemm_flops / (g64 * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": gemm_flops / (g64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (DFMA loop measured 1.00)",
                "flops_per_step": gemm_flops, "ms_per_step": g64}
    sketch_roofline = {"kernel": "k_sketch_dense_f64acc (hash gather)", "bound": "hbm",
                       "achieved": gather_bytes / (g_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": gather_bytes / (g_ms * 1e-3) / 1e9 / hbm, "traffic": GATHER_TRAFFIC.get(name),
                       "peak_source": peak_kind, "bytes_per_launch": gather_bytes, "ms_per_launch": g_ms}
    tf32_peak = 0.5 * pj.get("bf16_tflops", 1900.0)
    tc_roofline = {"kernel": "k_gemm_tc (TF32 QR trailing update, mixed path)", "bound": "tensor",
                   "achieved": gemm_flops / (g32 * 1e-3) / 1e12, "unit": "TFLOP/s",
                   "peak": tf32_peak, "frac": gemm_flops / (g32 * 1e-3) / 1e12 / tf32_peak,
                   "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 0.5", "ms_per_step": g32}
    stages = {
        "premix_fp64": {"ms": pm_ms, "bound": "hbm", "algorithmic_bytes": premix_bytes,
                        "achieved_gbs": premix_bytes / (pm_ms * 1e-3) / 1e9 if pm_ms > 0 else None},
        "qr_fp64": {"ms": qr64, "bound": "alu", "flops": qr_flops,
                    "achieved_tflops": qr_flops / (qr64 * 1e-3) / 1e12,
                    "peak_tflops": FP64_PEAK_TFLOPS},
        "qr_fp32": {"ms": qrmx, "bound": "alu", "flops": qr_flops,
                    "achieved_tflops": qr_flops / (qrmx * 1e-3) / 1e12, "peak_tflops": FP32_PEAK_TFLOPS},
    }
    lls = {
        "fp64": {"ms": statistics.mean(i.ms_total for i, _ in infos), "iters": infos[-1][0].iters,
                 "metric": max(i.metric for i, _ in infos), "ms_sketch": sk_ms, "ms_qr": qr64,
                 "ms_trinv": statistics.mean(i.ms_trinv for i, _ in infos),
                 "ms_lsqr": statistics.mean(i.ms_lsqr for i, _ in infos)},
        "mixed_fp32": {"ms": statistics.mean(j.ms_total for _, j in infos), "iters": infos[-1][1].iters,
                       "metric": max(j.metric for _, j in infos),
                       "ms_sketch": statistics.mean(j.ms_sketch for _, j in infos), "ms_qr": qrmx,
                       "ms_trinv": statistics.mean(j.ms_trinv for _, j in infos),
                       "ms_lsqr": statistics.mean(j.ms_lsqr for _, j in infos)},
    }

    # end to end through the public API with host buffers: pinned A, b -> device,
    # ski_sketch_hash, [SA | Sb] -> pinned host
    Ah = torch.from_numpy(A).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    SAd = torch.empty(m, d + 1, dtype=torch.float64, device="cuda")
    SAh = torch.empty(m, d + 1, dtype=torch.float64).pin_memory()
    sws = torch.empty(pkg.ski_sketch_workspace_size(Amat, 1, o64), dtype=torch.uint8, device="cuda")

    def e2e_step():
        At.copy_(Ah, non_blocking=True)
        bt.copy_(bh, non_blocking=True)
        pkg.ski_sketch_hash(Amat, bt, o64, SAd, d + 1, ws=sws)
        SAh.copy_(SAd, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    ev0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ev0.elapsed_time(ev1), world) / args.steps
    e2e = {"value": world * sb / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": int(8 * (n * d + n)), "d2h_bytes_per_step": int(8 * m * (d + 1)),
           "ms_per_step": e2e_ms}

    cpu = None
    if rank == 0 and not args.no_cpu:
        vals = [oracle_sample(A, b, cfg, args.ref_cols, args.seed)[0] for _ in range(2)]
        cpu = {"value": statistics.mean(vals), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "oracle HRHT sketch (numpy FP64) of A[:, :%d] + b, same n, n_pad, m, s" % args.ref_cols}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n": n, "d": d, "n_pad": npad, "m": m, "s": s, "gamma": cfg["gamma"],
                       "A": cfg["kind"], "b": "ones" if cfg["kind"] != "lls" else "A x + 1e-3 N(0,1)",
                       "l2": "inputs larger than L2 (A = %.2f GB)" % (8e-9 * n * d),
                       "parallelism": "replicas" if world > 1 else "single"},
            "hbm_frac": value / world / hbm, "roofline": roofline, "sketch_roofline": sketch_roofline,
            "tc_roofline": tc_roofline, "stages": stages, "lls": lls,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=20210525)
    ap.add_argument("--ref-cols", type=int, default=1024)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
