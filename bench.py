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

Outside the timed step the line also carries: the BF16 form of the same
solve; the mixed-precision workload at its own size (A = U diag(sigma) V^T,
200000 x 4000, kappa 1e6 and 1e10), FP64 against mixed; the whole solve end
to end with host buffers; and the oracle timed on the host cores.

--impl reference times the CPU FP64 oracle on the host cores: one oracle
process per core, each on an independent block of A's columns (or whole
problems of the batch) -- the slow reference arm.
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
# each process of the CPU oracle runs one BLAS / OpenMP thread (the paper's
# own timings are sequential); the host cores are used by running one oracle
# process per core on independent parts of the workload.  Set before numpy
# loads its BLAS, and inherited by the oracle's spawned processes.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

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
    # mixed-precision workload: A = U diag(sigma) V^T, kappa 1e6 / 1e10, premix to 262144
    "usv_200000x4000_k1e6_hrht_s1_g2": (200000, 4000, 262144, 1, 2.0, "usv:1e6"),
    "usv_200000x4000_k1e10_hrht_s1_g2": (200000, 4000, 262144, 1, 2.0, "usv:1e10"),
    # sparse workload: CSR, 8 nonzeros per row, 0.1% rows with 2000; s = 2, m = 2d
    "csr_1000000x20000_s2_g2": (1000000, 20000, 0, 2, 2.0, "csr"),
    # ragged batch: 256 problems, d ~ U{64..1024}, n ~ U{max(2000, 4d)..60000}
    "batched_256_ragged_g2": (256, 0, 0, 1, 2.0, "batched"),
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
# DRAM bytes (read + write) per launch, from ncu's dram__bytes_read.sum and
# dram__bytes_write.sum of the current kernels: the whole sketch stage (bucket
# lists, both premix passes, the nonfinite scan, the column-unit bound, the
# hash gather and the NaN post-pass) and the hash gather alone; None where not
# captured.
SKETCH_TRAFFIC = {"dense_50000x4000_hrht_s1_g2": 43264 + 38400 + 429056 + 333056 + 1612551424 + 1555619072 + 7936 +
                  1598208 + 1618771200 + 2050941696 + 2425076480 + 236391168 + 20480}
GATHER_TRAFFIC = {"dense_50000x4000_hrht_s1_g2": 2425076480 + 236391168}
# DRAM bytes (read + write) per step of the FP64 QR trailing-update GEMMs
# (k_gemm<double>): the sum over the 472 launches of one step of ncu's
# dram__bytes_read.sum (27379879168) and dram__bytes_write.sum (6929454592)
# DRAM bytes per step of the grouped FP16 slice-product launches that form
# SA^T SA in the FP64 solve (one ncu capture of the three DRAM/time metrics,
# one pass, full size)
GRAM64_TRAFFIC = {"dense_50000x4000_hrht_s1_g2": 10297787904 + 580307200}
GEMM64_TRAFFIC = {"dense_50000x4000_hrht_s1_g2": 27379879168 + 6929454592}


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


def dist_init(n_gpus, backend=None):
    """Rank, world size and local rank from the launcher's environment.  With
    more than one rank: one process group (NCCL on GPUs, gloo otherwise) used
    only for the barrier and the max-over-ranks of the timings -- the ranks
    are independent replicas, nothing of the data path crosses it."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_problem(name, seed):
    from paper_2105_11815_gb300 import workloads
    n, d, npad, s, gamma, kind = WORKLOADS[name]
    if kind == "gauss":
        A, b = workloads.dense_gaussian(n, d, seed)
    elif kind.startswith("usv:"):
        A, b = workloads.usv_torch(n, d, float(kind[4:]), seed, "cuda")
    elif kind == "coh":
        A, b = workloads.dense_high_coherence(n, d, seed)
    else:
        A, b, _ = workloads.gaussian_lls(n, d, seed)
    return A, b, dict(n=n, d=d, n_pad=npad, s=s, m=int(round(gamma * d)), gamma=gamma, kind=kind)


def sketch_bytes(cfg):
    n, d, m = cfg["n"], cfg["d"], cfg["m"]
    return 8.0 * (n * d + n + m * (d + 1))


def host_cols(A, cols):
    """A[:, :cols] as a host numpy array (A numpy or a device tensor)."""
    if hasattr(A, "detach"):
        return A[:, :cols].cpu().numpy()
    return A[:, :cols].copy()


def host_vec(b):
    return b.cpu().numpy() if hasattr(b, "detach") else b


def host_cores():
    """The host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class HostOracle:
    """The CPU oracle, as it stands, run on every host core: a process pool
    (started with spawn, safe beside CUDA) whose workers each run the oracle on
    one independent part of the workload -- a block of A's columns for the
    sketch (S*A acts on every column alone), whole problems for the batch.
    The inputs are placed once in shared memory; the timed region is the pool's
    map, wall clock, so it includes each worker's attach and dispatch."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.shm = []

    def share(self, arr):
        import numpy as np
        from multiprocessing import shared_memory
        arr = np.ascontiguousarray(arr)
        sh = shared_memory.SharedMemory(create=True, size=max(1, arr.nbytes))
        np.ndarray(arr.shape, dtype=arr.dtype, buffer=sh.buf)[...] = arr
        self.shm.append(sh)
        return (sh.name, arr.shape, arr.dtype.str)

    def run(self, fn, jobs):
        t0 = time.perf_counter()
        out = self.pool.map(fn, jobs, chunksize=1)
        return out, time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()
        for sh in self.shm:
            sh.close()
            sh.unlink()
        self.shm = []


def _attach(ref):
    """A read-only view of an array that HostOracle.share placed in shared memory."""
    import numpy as np
    from multiprocessing import shared_memory
    name, shape, dt = ref
    # the spawned workers share the parent's resource tracker: the segment stays
    # registered once, and the parent unlinks it
    sh = shared_memory.SharedMemory(name=name)
    return sh, np.ndarray(shape, dtype=np.dtype(dt), buffer=sh.buf)


def _oracle_dense_block(job):
    aref, bref, c0, c1, seed, s, m, n_pad = job
    from oracle import sketch as osk, wht as owht
    sha, A = _attach(aref)
    shb, b = _attach(bref) if bref is not None else (None, None)
    Ab = A[:, c0:c1]
    if n_pad:
        owht.hrht_sketch(seed, s, m, Ab, b, n_pad)
    else:
        osk.sketch_rows(seed, s, m, Ab, b)
    del A, Ab, b
    sha.close()
    if shb is not None:
        shb.close()
    return c1 - c0


def dense_oracle_all_cores(ho, aref, bref, cfg, seed):
    """The oracle's sketch of the whole of [A | b], columns split over the host
    cores (b with the first block).  Returns (GB/s, wall s, sample text)."""
    d = cfg["d"]
    chunk = -(-d // ho.cores)
    jobs = [(aref, bref if c0 == 0 else None, c0, min(d, c0 + chunk), seed, cfg["s"], cfg["m"], cfg["n_pad"])
            for c0 in range(0, d, chunk)]
    _, dt = ho.run(_oracle_dense_block, jobs)
    sample = "oracle %s sketch (numpy FP64) of all of A (%d x %d) and b, m=%d, s=%d: %d column blocks of %d on %d " \
             "host processes" % ("HRHT" if cfg["n_pad"] else "s-hashing", cfg["n"], d, cfg["m"], cfg["s"],
                                 len(jobs), chunk, ho.cores)
    return sketch_bytes(cfg) / dt / 1e9, dt, sample


def oracle_sample(A, b, cfg, cols, seed):
    """Time the CPU oracle's sketch on A[:, :cols] (the bounded CPU sample)."""
    from oracle import sketch as osk, wht as owht
    Asub = host_cols(A, cols)
    b = host_vec(b)
    t0 = time.perf_counter()
    if cfg["n_pad"]:
        owht.hrht_sketch(seed, cfg["s"], cfg["m"], Asub, b, cfg["n_pad"])
    else:
        osk.sketch_rows(seed, cfg["s"], cfg["m"], Asub, b)
    dt = time.perf_counter() - t0
    nbytes = 8.0 * (cfg["n"] * cols + cfg["n"] + cfg["m"] * (cols + 1))
    return nbytes / dt / 1e9, dt


def run_reference(args, name):
    rank = int(os.environ.get("RANK", "0"))  # the oracle runs on rank 0 alone: no process group
    if rank != 0:
        return
    A, b, cfg = make_problem(name, args.seed)
    A, b = host_cols(A, cfg["d"]), host_vec(b)
    ho = HostOracle(args.ref_cores or None)
    try:
        aref, bref = ho.share(A), ho.share(b)
        for _ in range(args.warmup):
            dense_oracle_all_cores(ho, aref, bref, cfg, args.seed)
        vals, times = [], []
        sample = ""
        for _ in range(args.steps):
            v, dt, sample = dense_oracle_all_cores(ho, aref, bref, cfg, args.seed)
            vals.append(v)
            times.append(dt)
    finally:
        ho.close()
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, **cfg},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": ho.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_dense(args, A, b, cfg):
    """The oracle's sketch timed on the host: the whole of [A | b] on every
    host core (the reported value), and a column sample on one thread."""
    Ah, bh = host_cols(A, cfg["d"]), host_vec(b)
    ho = HostOracle(args.ref_cores or None)
    try:
        aref, bref = ho.share(Ah), ho.share(bh)
        dense_oracle_all_cores(ho, aref, bref, cfg, args.seed)
        runs = [dense_oracle_all_cores(ho, aref, bref, cfg, args.seed) for _ in range(2)]
    finally:
        ho.close()
    cols = min(args.ref_cols, cfg["d"])
    v1, dt1 = oracle_sample(Ah, bh, cfg, cols, args.seed)
    return {"value": statistics.mean(r[0] for r in runs), "unit": "GB/s", "cores": ho.cores, "kind": "oracle",
            "sample": runs[-1][2], "s_per_run": statistics.mean(r[1] for r in runs),
            "single_thread": {"value": v1, "unit": "GB/s", "cores": 1, "s": dt1,
                              "sample": "oracle %s sketch (numpy FP64) of A[:, :%d] + b, same n, n_pad, m, s" % (
                                  "HRHT" if cfg["n_pad"] else "s-hashing", cols)}}


def usv_solves(pkg, torch, args, n=200000, d=4000, n_pad=262144):
    """The mixed-precision workload at its own size, outside the timed step:
    A = U diag(sigma) V^T (Haar U, V; sigma geometric to kappa), premix to
    262144, s = 1, m = 2d; the all-FP64 solve and the mixed form (FP32 premix
    and sketch, three-pass TF32 QR, FP64 LSQR), each solved once untimed and
    once timed, to the FP64 test 1e-10 (compensated residual).  b = ones at
    kappa = 1e6 and 1e10; at 1e10 that b puts x near 1e11 and the metric of
    any FP64 x near 1e-10 (the solve then ends SKI_ENOCONV with the metric it
    reached), so kappa = 1e10 is also solved with b = A x_true + e, e
    orthogonal to range(A) ("perp"), where x stays O(1).  Times are the
    library's own CUDA-event time of the whole solve."""
    from paper_2105_11815_gb300 import workloads
    out = {}
    for kappa, rhs in ((1e6, "ones"), (1e10, "ones"), (1e10, "perp")):
        A, b = workloads.usv_torch(n, d, kappa, args.seed, "cuda", rhs=rhs)
        M = pkg.dense_matrix(A)
        common = dict(m=2 * d, s=1, seed=args.seed, premix=1, n_pad=n_pad, tol=1e-10, tau_r=1e-10)
        forms = (("fp64", pkg.ski_opts_default(**common)),
                 ("mixed_fp32", pkg.ski_opts_default(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32, **common)),
                 ("fp64_gram", pkg.ski_opts_default(factorization=2, **common)),
                 ("mixed_gram", pkg.ski_opts_default(factorization=2, sketch_dtype=pkg.SKI_F32,
                                                     qr_dtype=pkg.SKI_F32, **common)))
        ws = torch.empty(max(pkg.ski_solve_workspace_size(M, o) for _, o in forms), dtype=torch.uint8, device="cuda")
        x = torch.empty(d, dtype=torch.float64, device="cuda")
        rec = {"b": rhs}
        for lab, o in forms:
            pkg.ski_solve(M, b, o, x, ws=ws, check=False)
            i = pkg.ski_solve(M, b, o, x, ws=ws, check=False)
            rec[lab] = {"ms": i.ms_total, "iters": i.iters, "restarts": i.restarts, "status": i.status,
                        "qr_fallback": i.qr_fallback, "rdiag_ratio": i.rdiag_ratio, "metric": i.metric,
                        "ms_sketch": i.ms_sketch, "ms_qr": i.ms_qr, "ms_trinv": i.ms_trinv, "ms_lsqr": i.ms_lsqr,
                        "gram": i.gram, "timed": False}
        out["kappa_%.0e%s" % (kappa, "" if rhs == "ones" else "_bperp")] = rec
        del A, b, M, ws, x
        torch.cuda.empty_cache()
    return out


def dht_sketch_stages(pkg, Amat, bt, cfg, args, sb):
    """The same sketch with the Hartley premix F D of Eq. HR-DHT (length n, no
    padding at the paper's sizes) instead of H D: one untimed and one timed
    ski_sketch_hash per precision, outside the timed region."""
    import torch
    n, d, m, s = cfg["n"], cfg["d"], cfg["m"], cfg["s"]
    out = {}
    for lab, sdt, tdt in (("fp64", pkg.SKI_F64, torch.float64), ("fp32", pkg.SKI_F32, torch.float32)):
        o = pkg.ski_opts_default(m=m, s=s, seed=args.seed, premix=2, sketch_dtype=sdt)
        ws = torch.empty(pkg.ski_sketch_workspace_size(Amat, 1, o), dtype=torch.uint8, device="cuda")
        SA = torch.empty(m, d + 1, dtype=tdt, device="cuda")
        pkg.ski_sketch_hash(Amat, bt, o, SA, d + 1, ws=ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        pkg.ski_sketch_hash(Amat, bt, o, SA, d + 1, ws=ws)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        bytes_ = sb if sdt == pkg.SKI_F64 else 8.0 * n * (d + 1) + 4.0 * m * (d + 1)
        out["premix_dht_and_hash_%s" % lab] = {
            "ms": ms, "n_h": n, "bound": "alu" if sdt == pkg.SKI_F64 else "hbm", "algorithmic_bytes": bytes_,
            "achieved_gbs": bytes_ / (ms * 1e-3) / 1e9, "timed": False}
        del ws, SA
        torch.cuda.empty_cache()
    return out


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
    At = A if torch.is_tensor(A) else torch.from_numpy(A).cuda()
    bt = b if torch.is_tensor(b) else torch.from_numpy(b).cuda()
    Amat = pkg.dense_matrix(At)
    # LSQR stops on Eq. TC-lsqr at tau_r = 1e-10; the FP64 acceptance test
    # ||A^T r|| / (||A||_F ||r||) <= 1e-10 is then checked (warm restart if not)
    common = dict(m=m, s=s, seed=args.seed, premix=1 if npad else 0, n_pad=npad, tol=1e-10, tau_r=1e-10,
                  premix_slab=args.premix_slab)
    o64 = pkg.ski_opts_default(factorization=args.factorization, **common)
    qmx = pkg.SKI_TF32 if args.qr_mixed == "tf32" else pkg.SKI_F32
    omx = pkg.ski_opts_default(sketch_dtype=pkg.SKI_F32, qr_dtype=qmx, factorization=args.factorization, **common)
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(pkg.ski_solve_workspace_size(Amat, o64), pkg.ski_solve_workspace_size(Amat, omx)),
                     dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        i64 = pkg.ski_solve(Amat, bt, o64, x, ws=ws, check=False)
        imx = pkg.ski_solve(Amat, bt, omx, x, ws=ws, check=False)
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
    # the sketch stage after the bucket lists: with the premix, its passes and
    # the hash gather run slab by slab over the columns (ms_premix covers both);
    # without, the gather alone (ms_gather).  Algorithmic bytes: A and b read
    # once, [SA | Sb] written once -- the intermediates stay in L2.
    g_ms = statistics.mean(i.ms_gather for i, _ in infos)
    pm_ms = statistics.mean(i.ms_premix for i, _ in infos)
    stage_ms = pm_ms + g_ms
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
                "frac": gemm_flops / (g64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": GEMM64_TRAFFIC.get(name),
                "traffic_scope": "bytes per step, summed over the k_gemm<double> QR-update launches of one step",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (DFMA loop measured 1.00)",
                "flops_per_step": gemm_flops, "ms_per_step": g64}
    sketch_roofline = {"kernel": ("premix + hash stage (k_wht_p1_tma, k_wht_fx, k_sketch_qa_f64acc)"
                                  if npad else "k_sketch_dense_f64acc (hash gather)"), "bound": "hbm",
                       "achieved": sb / (stage_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": sb / (stage_ms * 1e-3) / 1e9 / hbm, "traffic": SKETCH_TRAFFIC.get(name),
                       "peak_source": peak_kind, "bytes_per_stage": sb, "ms_per_stage": stage_ms}
    # the hash gather alone (S applied to the premixed rows): reads s * rows *
    # (d + 1) int64 values, writes [SA | Sb]
    rows = npad if npad else n
    gather_bytes = 8.0 * (s * rows * (d + 1) + m * (d + 1))
    hash_roofline = {"kernel": "k_sketch_qa_f64acc (hash gather)" if npad else "k_sketch_dense_f64acc (hash gather)",
                     "bound": "hbm", "achieved": gather_bytes / (g_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": gather_bytes / (g_ms * 1e-3) / 1e9 / hbm, "traffic": GATHER_TRAFFIC.get(name),
                     "peak_source": peak_kind, "bytes_per_launch": gather_bytes, "ms_per_launch": g_ms}
    tf32_peak = 0.5 * pj.get("bf16_tflops", 1900.0)
    # the mixed path's QR runs its products in three TF32 passes: the tensor
    # pipe executes 3x the algorithmic flops counted here
    tc_roofline = {"kernel": "k_gemm_tc<.., SPLIT> (3-pass TF32 QR trailing update, mixed path)", "bound": "tensor",
                   "achieved": gemm_flops / (g32 * 1e-3) / 1e12, "unit": "TFLOP/s",
                   "peak": tf32_peak, "frac": gemm_flops / (g32 * 1e-3) / 1e12 / tf32_peak,
                   "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 0.5", "ms_per_step": g32}
    if args.factorization == 2 and infos[-1][0].gram and infos[-1][1].gram:
        # Step 2 from the Gram matrix in both timed solves: the products are
        # the FP64 form's 66 FP16 slice pairs and the mixed form's 3 TF32
        # passes, m d (d + 1) flops each (the upper triangle of SA^T SA)
        lg = 0
        while (1 << lg) <= m:
            lg += 1
        beta = (24 - lg) // 2
        ns = (54 + beta - 1) // beta
        pairs = sum(min(ns, tt - 1) - max(1, tt - ns) + 1 for tt in range(2, ns + 2))
        gfl = float(m) * d * (d + 1)
        bfp = pj.get("bf16_tflops", 1900.0)
        roofline = {"kernel": "k_gemm_tc<256, 4, 0, 1> (FP64 Gram matrix from FP16 slice products)",
                    "bound": "tensor", "achieved": pairs * gfl / (g64 * 1e-3) / 1e12, "peak": bfp,
                    "unit": "TFLOP/s", "frac": pairs * gfl / (g64 * 1e-3) / 1e12 / bfp,
                    "traffic": GRAM64_TRAFFIC.get(name),
                    "traffic_scope": "bytes per step, summed over the grouped slice-product launches that form "
                                     "SA^T SA",
                    "peak_source": "measured bf16 burst", "pairs": pairs, "flops_per_step": pairs * gfl,
                    "fp64_equivalent_tflops": gfl / (g64 * 1e-3) / 1e12, "ms_per_step": g64}
        tc_roofline = {"kernel": "k_gemm_tc<256, 2, 1> (3-pass TF32 Gram matrix, mixed path)", "bound": "tensor",
                       "achieved": 3 * gfl / (g32 * 1e-3) / 1e12, "unit": "TFLOP/s", "peak": tf32_peak,
                       "frac": 3 * gfl / (g32 * 1e-3) / 1e12 / tf32_peak,
                       "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 0.5", "ms_per_step": g32}
    stages = {
        "premix_and_hash_fp64": {"ms": stage_ms, "bound": "hbm", "algorithmic_bytes": sb,
                                 "achieved_gbs": sb / (stage_ms * 1e-3) / 1e9 if stage_ms > 0 else None},
        "qr_fp64": {"ms": qr64, "bound": "alu", "flops": qr_flops,
                    "achieved_tflops": qr_flops / (qr64 * 1e-3) / 1e12,
                    "peak_tflops": FP64_PEAK_TFLOPS},
        "qr_fp32": {"ms": qrmx, "bound": "alu", "flops": qr_flops,
                    "achieved_tflops": qr_flops / (qrmx * 1e-3) / 1e12, "peak_tflops": FP32_PEAK_TFLOPS},
    }
    if args.factorization == 2:
        # Step 2 from the Gram matrix: G's upper triangle and the Cholesky,
        # FP64-equivalent flops (the FP64 form runs G on the tensor cores)
        s2 = float(m) * d * (d + 1) + d ** 3 / 3.0
        del stages["qr_fp64"], stages["qr_fp32"]
        stages["step2_fp64"] = {"ms": qr64, "method": "gram" if infos[-1][0].gram else "householder (fallback)",
                                "flops": s2, "achieved_tflops": s2 / (qr64 * 1e-3) / 1e12}
        stages["step2_fp32"] = {"ms": qrmx, "method": "gram" if infos[-1][1].gram else "householder (fallback)",
                                "flops": s2, "achieved_tflops": s2 / (qrmx * 1e-3) / 1e12}
    if npad and not args.no_dht:
        stages.update(dht_sketch_stages(pkg, Amat, bt, cfg, args, sb))
    lls = {
        "fp64": {"ms": statistics.mean(i.ms_total for i, _ in infos), "iters": infos[-1][0].iters,
                 "restarts": infos[-1][0].restarts, "status": infos[-1][0].status,
                 "rdiag_ratio": infos[-1][0].rdiag_ratio,
                 "metric": max(i.metric for i, _ in infos), "ms_sketch": sk_ms, "ms_qr": qr64,
                 "ms_trinv": statistics.mean(i.ms_trinv for i, _ in infos),
                 "ms_lsqr": statistics.mean(i.ms_lsqr for i, _ in infos),
                 "factorization": args.factorization, "gram": infos[-1][0].gram,
                 "ms_gram_product": statistics.mean(i.ms_qr_gemm for i, _ in infos) if infos[-1][0].gram else 0.0},
        "mixed_fp32": {"ms": statistics.mean(j.ms_total for _, j in infos), "iters": infos[-1][1].iters,
                       "restarts": infos[-1][1].restarts, "status": infos[-1][1].status,
                       "qr_fallback": infos[-1][1].qr_fallback, "rdiag_ratio": infos[-1][1].rdiag_ratio,
                       "metric": max(j.metric for _, j in infos),
                       "ms_sketch": statistics.mean(j.ms_sketch for _, j in infos), "ms_qr": qrmx,
                       "ms_trinv": statistics.mean(j.ms_trinv for _, j in infos),
                       "ms_lsqr": statistics.mean(j.ms_lsqr for _, j in infos),
                       "factorization": args.factorization, "gram": infos[-1][1].gram,
                       "ms_gram_product": statistics.mean(j.ms_qr_gemm for _, j in infos) if infos[-1][1].gram else 0.0},
    }

    # the BF16 form (BF16 premix and sketch, 3-pass TF32 QR of the BF16 sketch,
    # FP64 LSQR), outside the timed step: its R preconditions only when
    # kappa(SA) 2^-8 is small, else the solve refactors in FP64 (qr_fallback)
    obf = pkg.ski_opts_default(sketch_dtype=pkg.SKI_BF16, qr_dtype=pkg.SKI_F32, **common)
    ib = None
    for _ in range(2):
        ib = pkg.ski_solve(Amat, bt, obf, x, ws=torch.empty(pkg.ski_solve_workspace_size(Amat, obf),
                                                             dtype=torch.uint8, device="cuda"), check=False)
    lls["mixed_bf16"] = {"ms": ib.ms_total, "iters": ib.iters, "restarts": ib.restarts, "status": ib.status,
                         "qr_fallback": ib.qr_fallback, "rdiag_ratio": ib.rdiag_ratio, "metric": ib.metric,
                         "ms_sketch": ib.ms_sketch, "ms_qr": ib.ms_qr, "ms_trinv": ib.ms_trinv,
                         "ms_lsqr": ib.ms_lsqr, "timed": False}
    # Step 2 the other way, outside the timed step (the best of three solves
    # after one untimed): with the Gram matrix in the timed step (the default,
    # factorization = 2: R the Cholesky factor of SA^T SA, the Householder QR
    # past the ratio limit), the Householder QR of SA (Algorithm 1 as printed,
    # factorization = 0), and the other way round
    other = 0 if args.factorization == 2 else 2
    tag = "householder" if other == 0 else "gram"
    for lab, oo in (("fp64_" + tag, pkg.ski_opts_default(factorization=other, **common)),
                    ("mixed_" + tag, pkg.ski_opts_default(factorization=other, sketch_dtype=pkg.SKI_F32,
                                                          qr_dtype=qmx, **common))):
        wsg = torch.empty(pkg.ski_solve_workspace_size(Amat, oo), dtype=torch.uint8, device="cuda")
        runs = [pkg.ski_solve(Amat, bt, oo, x, ws=wsg, check=False) for _ in range(4)][1:]
        ig = min(runs, key=lambda r: r.ms_total)
        lls[lab] = {"ms": ig.ms_total, "iters": ig.iters, "restarts": ig.restarts, "status": ig.status,
                    "gram": ig.gram, "rdiag_ratio": ig.rdiag_ratio, "metric": max(r.metric for r in runs),
                    "ms_sketch": ig.ms_sketch, "ms_qr": ig.ms_qr, "ms_trinv": ig.ms_trinv, "ms_lsqr": ig.ms_lsqr,
                    "ms_gram_product": ig.ms_qr_gemm, "timed": False}
        del wsg
    # the Gram products on the tensor cores, against the measured dense bf16
    # burst (FP16 and BF16 share the nominal rate; TF32 is half of it).
    # Algorithmic flops of SA^T SA's upper triangle: m d (d + 1); the FP64
    # form multiplies 66 pairs of FP16 slices (5-bit slices at m = 8000), the
    # FP32 form three TF32 passes
    bf16_peak = pj.get("bf16_tflops", 1900.0)
    n_pairs = 0
    lg = 0
    while (1 << lg) <= m:
        lg += 1
    beta = (24 - lg) // 2
    ns = (54 + beta - 1) // beta
    for tt in range(2, ns + 2):
        n_pairs += min(ns, tt - 1) - max(1, tt - ns) + 1
    gflop = m * d * (d + 1)
    gram_roofline = {}
    g_fp64 = lls["fp64"] if args.factorization == 2 else lls["fp64_gram"]
    g_mx = lls["mixed_fp32"] if args.factorization == 2 else lls["mixed_gram"]
    if g_fp64["gram"] and g_fp64["ms_gram_product"] > 0:
        t = g_fp64["ms_gram_product"] * 1e-3
        gram_roofline["fp64_slices"] = {
            "kernel": "k_gemm_tc<256, 4, 0, 1> (kind::f16 slice products, FP64 accumulation)", "bound": "tensor",
            "pairs": n_pairs, "slice_bits": beta, "achieved": n_pairs * gflop / t / 1e12,
            "peak": bf16_peak, "unit": "TFLOP/s", "frac": n_pairs * gflop / t / 1e12 / bf16_peak,
            "fp64_equivalent_tflops": gflop / t / 1e12, "peak_source": "measured bf16 burst", "ms": t * 1e3}
    if g_mx["gram"] and g_mx["ms_gram_product"] > 0:
        t = g_mx["ms_gram_product"] * 1e-3
        passes = 3 if args.qr_mixed != "tf32" else 1
        gram_roofline["fp32_3xtf32"] = {
            "kernel": "k_gemm_tc<256, 2, 1> (3-pass TF32 Gram product)" if passes == 3 else
                      "k_gemm_tc<256, 2, 0> (TF32 Gram product)", "bound": "tensor",
            "achieved": passes * gflop / t / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
            "frac": passes * gflop / t / 1e12 / tf32_peak,
            "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 0.5", "ms": t * 1e3}

    # end to end through the public API with host buffers: pinned A, b -> device,
    # ski_sketch_hash, [SA | Sb] -> pinned host
    Ah = (A.cpu() if torch.is_tensor(A) else torch.from_numpy(A)).pin_memory()
    bh = (b.cpu() if torch.is_tensor(b) else torch.from_numpy(b)).pin_memory()
    # the whole solve end to end, outside the timed step: pinned A, b -> device,
    # ski_solve (FP64, then mixed), x -> pinned host
    xh = torch.empty(d, dtype=torch.float64).pin_memory()
    e2e_solve = {"h2d_bytes_per_solve": int(8 * (n * d + n)), "d2h_bytes_per_solve": int(8 * d)}
    for lab, oo in (("fp64", o64), ("mixed_fp32", omx)):
        t_s = []
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            At.copy_(Ah, non_blocking=True)
            bt.copy_(bh, non_blocking=True)
            pkg.ski_solve(Amat, bt, oo, x, ws=ws, check=False)
            xh.copy_(x, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:
                t_s.append(e0.elapsed_time(e1))
        e2e_solve[lab + "_ms"] = statistics.mean(t_s)
    if not args.no_usv and npad:
        lls["usv_200000x4000"] = usv_solves(pkg, torch, args)
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
        cpu = cpu_baseline_dense(args, A, b, cfg)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n": n, "d": d, "n_pad": npad, "m": m, "s": s, "gamma": cfg["gamma"],
                       "mixed_qr": args.qr_mixed, "premix_slab": args.premix_slab,
                       "factorization": args.factorization,
                       "A": cfg["kind"], "b": "ones" if cfg["kind"] != "lls" else "A x + 1e-3 N(0,1)",
                       "l2": "inputs larger than L2 (A = %.2f GB)" % (8e-9 * n * d),
                       "parallelism": "replicas" if world > 1 else "single"},
            "hbm_frac": value / world / hbm, "roofline": roofline, "sketch_roofline": sketch_roofline,
            "hash_roofline": hash_roofline, "tc_roofline": tc_roofline, "gram_roofline": gram_roofline,
            "stages": stages, "lls": lls,
            "e2e": e2e, "e2e_solve": e2e_solve, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- sparse workload
def csr_bytes(n, nnz, m, d):
    """Sketch metric bytes of the CSR path: rowptr, colidx, values and b read,
    [SA | Sb] written."""
    return 8.0 * (n + 1) + 12.0 * nnz + 8.0 * n + 8.0 * m * (d + 1)


def make_csr(name, seed):
    from paper_2105_11815_gb300 import workloads
    n, d, _, s, gamma, _ = WORKLOADS[name]
    rowptr, colidx, val, b = workloads.csr_heavy_rows(n, d, seed)
    return rowptr, colidx, val, b, dict(n=n, d=d, n_pad=0, s=s, m=int(round(gamma * d)), gamma=gamma, kind="csr",
                                        nnz=int(rowptr[-1]))


def csr_oracle_sample(rowptr, colidx, val, b, cfg, cols, seed):
    """Time the oracle's CSR sketch restricted to the columns < cols (all rows)."""
    import numpy as np
    import scipy.sparse as sp
    from oracle import sketch as osk
    n = cfg["n"]
    keep = colidx < cols
    rows = np.repeat(np.arange(n), np.diff(rowptr))[keep]
    A = sp.csr_matrix((val[keep], (rows, colidx[keep])), shape=(n, cols))
    t0 = time.perf_counter()
    osk.sketch_rows(seed, cfg["s"], cfg["m"], A, b)
    dt = time.perf_counter() - t0
    return csr_bytes(n, int(keep.sum()), cfg["m"], cols) / dt / 1e9, dt, int(keep.sum())


def _oracle_csr_block(job):
    rref, cref, vref, bref, c0, c1, n, seed, s, m = job
    import numpy as np
    import scipy.sparse as sp
    from oracle import sketch as osk
    shs = [_attach(r) for r in (rref, cref, vref)]
    (_, rowptr), (_, colidx), (_, val) = shs
    shb, b = _attach(bref) if bref is not None else (None, None)
    keep = (colidx >= c0) & (colidx < c1)
    rows = np.repeat(np.arange(n), np.diff(rowptr))[keep]
    A = sp.csr_matrix((val[keep], (rows, colidx[keep] - c0)), shape=(n, c1 - c0))
    osk.sketch_rows(seed, s, m, A, b)
    nnz = int(keep.sum())
    del rowptr, colidx, val, b, keep, rows, A
    for sh, _ in shs:
        sh.close()
    if shb is not None:
        shb.close()
    return nnz


def csr_oracle_all_cores(ho, refs, cfg, seed):
    """The oracle's CSR sketch of all of [A | b], columns split over the host
    cores (each process builds its column block's CSR, then sketches it)."""
    d = cfg["d"]
    chunk = -(-d // ho.cores)
    rref, cref, vref, bref = refs
    jobs = [(rref, cref, vref, bref if c0 == 0 else None, c0, min(d, c0 + chunk), cfg["n"], seed, cfg["s"], cfg["m"])
            for c0 in range(0, d, chunk)]
    nnzs, dt = ho.run(_oracle_csr_block, jobs)
    sample = ("oracle CSR sketch (numpy FP64) of all of A (%d x %d, %d nonzeros) and b, m=%d, s=%d: %d column blocks "
              "of %d on %d host processes, each also extracting its block" % (cfg["n"], d, sum(nnzs), cfg["m"],
                                                                              cfg["s"], len(jobs), chunk, ho.cores))
    return csr_bytes(cfg["n"], sum(nnzs), cfg["m"], d) / dt / 1e9, dt, sample


def run_reference_csr(args, name):
    rank = int(os.environ.get("RANK", "0"))  # the oracle runs on rank 0 alone: no process group
    if rank != 0:
        return
    rowptr, colidx, val, b, cfg = make_csr(name, args.seed)
    ho = HostOracle(args.ref_cores or None)
    try:
        refs = (ho.share(rowptr), ho.share(colidx), ho.share(val), ho.share(b))
        for _ in range(args.warmup):
            csr_oracle_all_cores(ho, refs, cfg, args.seed)
        vals, times = [], []
        sample = ""
        for _ in range(args.steps):
            v, dt, sample = csr_oracle_all_cores(ho, refs, cfg, args.seed)
            vals.append(v)
            times.append(dt)
    finally:
        ho.close()
    value = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, **cfg},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": ho.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def run_csr(args, name):
    import torch

    import paper_2105_11815_gb300 as pkg
    from paper_2105_11815_gb300 import build

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    pkg.lib()
    rowptr, colidx, val, b, cfg = make_csr(name, args.seed + rank)
    n, d, m, s, nnz = cfg["n"], cfg["d"], cfg["m"], cfg["s"], cfg["nnz"]
    rp, ci, va, bt = (torch.from_numpy(x).cuda() for x in (rowptr, colidx, val, b))
    Amat = pkg.csr_matrix(rp, ci, va, n, d)
    common = dict(m=m, s=s, seed=args.seed, tol=1e-10, tau_r=1e-10)
    o64 = pkg.ski_opts_default(**common)
    omx = pkg.ski_opts_default(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32, **common)
    ogr = pkg.ski_opts_default(factorization=2, **common)  # Step 2 from the sparse sketch's Gram matrix
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(pkg.ski_solve_workspace_size(Amat, o) for o in (o64, omx, ogr)),
                     dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        return pkg.ski_solve(Amat, bt, o64, x, ws=ws), pkg.ski_solve(Amat, bt, omx, x, ws=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.ski_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = pkg.ski_launch_count() - l0
    clk = clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), world) / args.steps
    sb = csr_bytes(n, nnz, m, d)
    sk_ms = max_over_ranks(statistics.mean(i.ms_sketch for i, _ in infos), world)
    value = world * sb / (sk_ms * 1e-3) / 1e9
    hbm, peak_kind, _ = peaks()
    gemm_flops = qr_gemm_flops(m, d)
    g64 = statistics.mean(i.ms_qr_gemm for i, _ in infos)
    roofline = {"kernel": "k_gemm<double> (FP64 QR trailing update)", "bound": "alu",
                "achieved": gemm_flops / (g64 * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": gemm_flops / (g64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz", "ms_per_step": g64}
    g_ms = statistics.mean(i.ms_gather for i, _ in infos)
    sketch_roofline = {"kernel": "k_sketch_csr<double> (CSR hash sketch)", "bound": "hbm",
                       "achieved": sb / (g_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": sb / (g_ms * 1e-3) / 1e9 / hbm, "traffic": None, "peak_source": peak_kind,
                       "bytes_per_launch": sb, "ms_per_launch": g_ms}
    lls = {lab: {"ms": statistics.mean(v.ms_total for v in col), "iters": col[-1].iters,
                 "restarts": col[-1].restarts, "metric": max(v.metric for v in col),
                 "ms_sketch": statistics.mean(v.ms_sketch for v in col),
                 "ms_qr": statistics.mean(v.ms_qr for v in col),
                 "ms_trinv": statistics.mean(v.ms_trinv for v in col),
                 "ms_lsqr": statistics.mean(v.ms_lsqr for v in col)}
           for lab, col in (("fp64", [i for i, _ in infos]), ("mixed_fp32", [j for _, j in infos]))}
    # FP64 with R from the Cholesky factor of the sparse sketch's Gram matrix
    # (factorization 2): one untimed and one timed solve outside the timed region
    pkg.ski_solve(Amat, bt, ogr, x, ws=ws)
    gi = pkg.ski_solve(Amat, bt, ogr, x, ws=ws)
    lls["fp64_gram"] = {"ms": gi.ms_total, "iters": gi.iters, "restarts": gi.restarts, "metric": gi.metric,
                        "status": gi.status, "gram": gi.gram, "ms_sketch": gi.ms_sketch, "ms_qr": gi.ms_qr,
                        "ms_trinv": gi.ms_trinv, "ms_lsqr": gi.ms_lsqr, "timed": False}
    # end to end: pinned CSR arrays and b -> device, ski_sketch_hash, [SA | Sb] -> pinned host
    hs = [torch.from_numpy(x).pin_memory() for x in (rowptr, colidx, val, b)]
    SAd = torch.empty(m, d + 1, dtype=torch.float64, device="cuda")
    SAh = torch.empty(m, d + 1, dtype=torch.float64).pin_memory()
    sws = torch.empty(pkg.ski_sketch_workspace_size(Amat, 1, o64), dtype=torch.uint8, device="cuda")

    def e2e_step():
        for dst, src in zip((rp, ci, va, bt), hs):
            dst.copy_(src, non_blocking=True)
        pkg.ski_sketch_hash(Amat, bt, o64, SAd, d + 1, ws=sws)
        SAh.copy_(SAd, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ev0.elapsed_time(ev1), world) / args.steps
    e2e = {"value": world * sb / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": int(8 * (n + 1) + 12 * nnz + 8 * n), "d2h_bytes_per_step": int(8 * m * (d + 1)),
           "ms_per_step": e2e_ms}
    cpu = None
    if rank == 0 and not args.no_cpu:
        ho = HostOracle(args.ref_cores or None)
        try:
            refs = (ho.share(rowptr), ho.share(colidx), ho.share(val), ho.share(b))
            v, dt, smp = csr_oracle_all_cores(ho, refs, cfg, args.seed)
        finally:
            ho.close()
        v1, dt1, nnz_s = csr_oracle_sample(rowptr, colidx, val, b, cfg, args.ref_cols, args.seed)
        cpu = {"value": v, "unit": "GB/s", "cores": ho.cores, "kind": "oracle", "sample": smp, "s_per_run": dt,
               "single_thread": {"value": v1, "unit": "GB/s", "cores": 1, "s": dt1,
                                 "sample": "oracle CSR sketch (numpy FP64) of the columns < %d (%d nonzeros), all "
                                           "rows" % (args.ref_cols, nnz_s)}}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n": n, "d": d, "nnz": nnz, "m": m, "s": s, "A": "csr_heavy_rows",
                       "b": "ones", "l2": "SA output larger than L2 (%.1f GB)" % (8e-9 * m * (d + 1)),
                       "parallelism": "replicas" if world > 1 else "single"},
            "hbm_frac": value / world / hbm, "roofline": roofline, "sketch_roofline": sketch_roofline,
            "lls": lls, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": int(launches)}),
            flush=True)


# ---------------------------------------------------------------- ragged batch
BATCH_METRIC = "batched LLS problems/s to ||A^T r||/(||A||_F ||r||) <= 1e-10, forward + adjoint backward"


def _oracle_problem(job):
    i, n, d, seed = job
    import numpy as np
    from oracle import adjoint as oadj, lsqr as olsqr
    g = np.random.default_rng((seed, i))
    A = g.standard_normal((n, d))
    b = g.standard_normal(n)
    c = g.standard_normal(d)
    t0 = time.perf_counter()
    x, _ = olsqr.ski_lls(A, b, seed + i, 1, int(2 * d), tau_r=1e-10)
    oadj.lstsq_grad(A, b, x, c)
    return time.perf_counter() - t0


def batch_oracle_all_cores(ho, shapes, seed, count):
    """The oracle's Ski-LLS and adjoint on the first `count` problems of the
    batch, one problem per host process at a time.  The timed region is the
    wall clock of the map; each process draws its problem before its own
    timer starts, so the wall clock also covers those draws."""
    jobs = [(i, n, d, seed) for i, (n, d) in enumerate(shapes[:count])]
    per, dt = ho.run(_oracle_problem, jobs)
    sample = ("oracle Ski-LLS + adjoint (numpy FP64) on the first %d problems of the batch, one per host process "
              "(%d processes); slowest problem %.2f s" % (count, ho.cores, max(per)))
    return count / dt, dt, sample


def run_reference_batched(args, name):
    rank = int(os.environ.get("RANK", "0"))  # the oracle runs on rank 0 alone: no process group
    if rank != 0:
        return
    from paper_2105_11815_gb300 import workloads
    count = WORKLOADS[name][0]
    shapes = workloads.ragged_batch(count, args.seed)
    ho = HostOracle(args.ref_cores or None)
    sample_n = min(count, max(args.ref_problems, ho.cores))
    try:
        for _ in range(args.warmup):
            batch_oracle_all_cores(ho, shapes, args.seed, sample_n)
        vals, times = [], []
        sample = ""
        for _ in range(args.steps):
            v, dt, sample = batch_oracle_all_cores(ho, shapes, args.seed, sample_n)
            vals.append(v)
            times.append(dt)
    finally:
        ho.close()
    value = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": "problems/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "problems": count},
        "cpu_baseline": {"value": value, "unit": "problems/s", "cores": ho.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "problems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def run_batched(args, name):
    import torch

    import paper_2105_11815_gb300 as pkg
    from paper_2105_11815_gb300 import build, workloads

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    pkg.lib()
    count = WORKLOADS[name][0]
    gamma = WORKLOADS[name][4]
    shapes, As, bs = workloads.ragged_batch_torch(count, args.seed + rank, "cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed + 7)
    gs = [torch.randn(d, generator=gen, device="cuda", dtype=torch.float64) for _, d in shapes]
    mats = [pkg.dense_matrix(a) for a in As]
    xs = [torch.empty(d, dtype=torch.float64, device="cuda") for _, d in shapes]
    Rs = [torch.empty(d, d, dtype=torch.float64, device="cuda") for _, d in shapes]
    dAs = [torch.empty_like(a) for a in As]
    dbs = [torch.empty_like(b) for b in bs]
    stream = torch.cuda.current_stream()

    prec = {} if args.batch_precision == "f64" else dict(sketch_dtype=pkg.SKI_F32, qr_dtype=pkg.SKI_F32)

    def opts(streams, batch_lsqr=args.batch_lsqr):
        return pkg.ski_opts_default(m=-int(round(1000 * gamma)), s=1, seed=args.seed, tol=1e-10, tau_r=1e-10,
                                    streams=streams, batch_lsqr=batch_lsqr, factorization=args.factorization, **prec)

    wsz = {}

    def workspace(o):
        k = (o.streams, o.lsqr_ctas, o.batch_lsqr)
        if k not in wsz:
            nb = max(pkg.ski_solve_batched_workspace_size(mats, o),
                     pkg.ski_solve_adjoint_batched_workspace_size(mats, o))
            wsz[k] = torch.empty(nb, dtype=torch.uint8, device="cuda")
        return wsz[k]

    def step(o):
        w = workspace(o)
        t0 = torch.cuda.Event(enable_timing=True)
        t_mid = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        fi = pkg.ski_solve_batched(mats, bs, o, xs, R_outs=Rs, ws=w, check=False)
        t_mid.record(stream)
        bi = pkg.ski_solve_adjoint_batched(mats, bs, xs, Rs, gs, dAs, dbs, o, ws=w, check=False)
        return fi, bi, (t0, t_mid)

    def timed(o, steps, warmup):
        for _ in range(warmup):
            step(o)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [step(o) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = max_over_ranks(e0.elapsed_time(e1), world) / steps
        fwd = statistics.mean(a.elapsed_time(b) for _, _, (a, b) in res)
        return ms, res, fwd

    o_main = opts(args.streams)
    tuned = None
    if args.autotune is not None:
        # launch parameters timed on a sample of this batch (outside the timed
        # region) or read back from the cache file
        from paper_2105_11815_gb300 import autotune
        t_tune = time.perf_counter()
        o_main, rec = autotune.tune_batched(mats, bs, xs, o_main, cache_path=args.autotune or None, sample=16,
                                            reps=1)
        tuned = dict(rec, tuning_s=time.perf_counter() - t_tune)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.ski_launch_count()
    ms_step, res, fwd_ms = timed(o_main, args.steps, args.warmup)
    launches = pkg.ski_launch_count() - l0
    clk = clocks.stop()
    value = world * count / (ms_step * 1e-3)
    fi, bi, _ = res[-1]
    worst = max(i.metric for i in fi)
    iters = [i.iters for i in fi]
    # algorithmic HBM bytes of one step: A read by the sketch, by the residual and
    # split passes (3 reads of A in FP64 + 1 write/read of the float2 copy) and by
    # every LSQR pass (the float2 copy, 8 bytes per element); the adjoint reads A
    # once per CG iteration and twice more, and writes dA
    byt = 0.0
    for (n, d), f, bw in zip(shapes, fi, bi):
        byt += 8.0 * n * d * (1 + 3 + 2 + f.iters + f.restarts * 2)
        byt += 8.0 * n * d * (bw.iters + 3)
    hbm, peak_kind, _ = peaks()
    roofline = {"kernel": "whole batch (A reads of every pass, aggregate)", "bound": "hbm",
                "achieved": byt / (ms_step * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byt / (ms_step * 1e-3) / 1e9 / hbm, "traffic": None, "peak_source": peak_kind,
                "bytes_per_step": byt}
    # sequential form on the same GPU (one problem at a time) and a sweep of the
    # number of problems in flight
    sweep = {}
    for w in args.sweep:
        ms_w, _, fwd_w = timed(opts(w), 1, 1)
        sweep[str(w)] = {"ms_per_step": ms_w, "problems_s": count / (ms_w * 1e-3), "fwd_ms": fwd_w}
    # the other form of Step 4 (per problem or grouped) for comparison
    ms_o, _, fwd_o = timed(opts(args.streams, 1 - args.batch_lsqr), 1, 1)
    sweep["batch_lsqr_%d" % (1 - args.batch_lsqr)] = {"ms_per_step": ms_o, "problems_s": count / (ms_o * 1e-3),
                                                      "fwd_ms": fwd_o}
    # end to end: pinned host A_i, b_i -> device, solve + adjoint, x_i, dA_i, db_i -> host
    Ah = [a.cpu().pin_memory() for a in As]
    bh = [b.cpu().pin_memory() for b in bs]
    xh = [torch.empty(d, dtype=torch.float64).pin_memory() for _, d in shapes]
    dAh = [torch.empty(a.shape, dtype=torch.float64).pin_memory() for a in As]

    def e2e_step():
        for a, h in zip(As, Ah):
            a.copy_(h, non_blocking=True)
        for b, h in zip(bs, bh):
            b.copy_(h, non_blocking=True)
        step(o_main)
        for x, h in zip(xs, xh):
            h.copy_(x, non_blocking=True)
        for a, h in zip(dAs, dAh):
            h.copy_(a, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    nA = sum(n * d for n, d in shapes)
    nb_ = sum(n for n, _ in shapes)
    nd_ = sum(d for _, d in shapes)
    e2e = {"value": world * count / (e2e_ms * 1e-3), "unit": "problems/s",
           "h2d_bytes_per_step": int(8 * (nA + nb_)), "d2h_bytes_per_step": int(8 * (nd_ + nA)),
           "ms_per_step": e2e_ms}
    cpu = None
    if rank == 0 and not args.no_cpu:
        ho = HostOracle(args.ref_cores or None)
        try:
            v, dt, smp = batch_oracle_all_cores(ho, shapes, args.seed, min(count, max(args.ref_problems, ho.cores)))
        finally:
            ho.close()
        cpu = {"value": v, "unit": "problems/s", "cores": ho.cores, "kind": "oracle", "sample": smp, "s_per_run": dt}
    if rank == 0:
        print(json.dumps({
            "metric": BATCH_METRIC, "value": value, "unit": "problems/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "problems": count, "gamma": gamma, "s": 1,
                       "sketch_qr": args.batch_precision,
                       "streams": o_main.streams or "auto", "batch_lsqr": o_main.batch_lsqr,
                       "factorization": args.factorization,
                       "lsqr_pass": o_main.lsqr_pass,
                       "lsqr_ctas": o_main.lsqr_ctas, "graphs": o_main.graphs, "autotune": tuned, "A_bytes": 8 * nA,
                       "l2": "inputs larger than L2 (%.1f GB)" % (8e-9 * nA),
                       "parallelism": "replicas" if world > 1 else "single"},
            "forward_ms": fwd_ms, "backward_ms": ms_step - fwd_ms, "worst_metric": worst,
            "iters": {"min": min(iters), "max": max(iters), "mean": statistics.mean(iters)},
            "restarts": {"max": max(i.restarts for i in fi), "mean": statistics.mean(i.restarts for i in fi)},
            "adjoint_iters": {"min": min(i.iters for i in bi), "max": max(i.iters for i in bi),
                              "mean": statistics.mean(i.iters for i in bi)},
            "statuses": {"forward": {str(k): sum(1 for i in fi if i.status == k) for k in set(i.status for i in fi)},
                         "backward": {str(k): sum(1 for i in bi if i.status == k) for k in set(i.status for i in bi)}},
            "failed": [{"i": k, "n": shapes[k][0], "d": shapes[k][1], "status": int(i.status), "iters": int(i.iters),
                        "restarts": int(i.restarts), "metric": i.metric} for k, i in enumerate(fi) if i.status][:8],
            "roofline": roofline, "streams_sweep": sweep, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": int(launches)}), flush=True)


def run_sketch_sweep(args):
    """The dense test-set sketch cases: d in {4000, 7000}, i.i.d. or high
    coherence, s in {1, 2}, gamma in {1.5, 2, 3, 4}, premix to 65536 (FP64).
    One JSON line per case: ski_sketch_hash on device-resident A, CUDA events
    over `steps` calls after `warmup`."""
    import torch

    import paper_2105_11815_gb300 as pkg
    from paper_2105_11815_gb300 import build, workloads
    build.build()
    pkg.lib()
    n, npad = 50000, 65536
    hbm, peak_kind, _ = peaks()
    stream = torch.cuda.current_stream()
    for d in (4000, 7000):
        for kind in ("gauss", "coh"):
            if kind == "gauss":
                A, b = workloads.gaussian_torch(n, d, args.seed, "cuda")
            else:
                A, b = workloads.dense_high_coherence_torch(n, d, args.seed, "cuda")
            mat = pkg.dense_matrix(A)
            for s in (1, 2):
                for gamma in (1.5, 2.0, 3.0, 4.0):
                    m = int(round(gamma * d))
                    o = pkg.ski_opts_default(m=m, s=s, seed=args.seed, premix=1, n_pad=npad)
                    SA = torch.empty(m, d + 1, dtype=torch.float64, device="cuda")
                    ws = torch.empty(pkg.ski_sketch_workspace_size(mat, 1, o), dtype=torch.uint8, device="cuda")
                    for _ in range(args.warmup):
                        pkg.ski_sketch_hash(mat, b, o, SA, d + 1, ws=ws)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    for _ in range(args.steps):
                        pkg.ski_sketch_hash(mat, b, o, SA, d + 1, ws=ws)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / args.steps
                    byt = 8.0 * (n * d + n + m * (d + 1))
                    print(json.dumps({"metric": "sketch S·A GB/s (premix + hash, FP64)", "value": byt / (ms * 1e-3) / 1e9,
                                      "unit": "GB/s", "ms": ms, "hbm_frac": byt / (ms * 1e-3) / 1e9 / hbm,
                                      "peak_source": peak_kind, "config": {"n": n, "d": d, "A": kind, "s": s,
                                                                           "gamma": gamma, "m": m, "n_pad": npad}}),
                          flush=True)
                    del SA, ws
            del A, b, mat
            torch.cuda.empty_cache()


def qr_gemm_flops(m, d):
    """Flops of the QR trailing-update GEMMs, summed over the 32-column panels:
    W = V^T C and C -= V B' each cost 2 w nct mr."""
    f = 0.0
    for k0 in range(0, d, 32):
        w = min(32, d - k0)
        f += 4.0 * w * ((d + 1) - k0 - w) * (m - k0)
    return f


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=20210525)
    ap.add_argument("--ref-cols", type=int, default=1024, help="one-thread oracle sample: columns of A")
    ap.add_argument("--ref-cores", type=int, default=0, help="host processes of the oracle (0 = every host core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-dht", action="store_true", help="skip the untimed Hartley-premix sketch stages")
    ap.add_argument("--no-usv", action="store_true",
                    help="skip the untimed mixed-precision-workload solves of the default line")
    ap.add_argument("--streams", type=int, default=0, help="batched workload: problems in flight (0 = auto)")
    ap.add_argument("--batch-lsqr", type=int, default=0, choices=(0, 1),
                    help="batched workload: 0 = Step 4 per problem, 1 = grouped over the problems in flight")
    ap.add_argument("--autotune", nargs="?", const="", default=None,
                    help="batched workload: tune the launch parameters first (optional JSON cache path)")
    ap.add_argument("--sweep", type=int, nargs="*", default=[1], help="batched workload: also time these")
    ap.add_argument("--ref-problems", type=int, default=3, help="batched workload: oracle sample size")
    ap.add_argument("--premix-slab", type=int, default=0, help="premix column slab width (0 = full width)")
    ap.add_argument("--factorization", type=int, default=2, choices=(0, 2),
                    help="dense workloads: Step 2 of the timed solves (2 from the Gram matrix SA^T SA, with the "
                         "Householder QR past its ratio limit; 0 the Householder QR); the other runs untimed")
    ap.add_argument("--qr-mixed", default="f32", choices=["f32", "tf32"],
                    help="QR precision of the mixed solve: f32 (three TF32 passes) or tf32 (one)")
    ap.add_argument("--sketch-sweep", action="store_true",
                    help="time the sketch alone on the 32 dense test-set cases (one JSON line each)")
    ap.add_argument("--batch-precision", default="f64", choices=["f64", "mixed"],
                    help="batched workload: sketch and QR in FP64, or FP32 with three TF32 passes "
                         "(LSQR, residuals and the acceptance test stay FP64 either way)")
    args = ap.parse_args()
    if args.sketch_sweep:
        run_sketch_sweep(args)
        return
    kind = WORKLOADS[args.workload][5]
    if args.impl == "reference":
        if kind == "csr":
            run_reference_csr(args, args.workload)
        elif kind == "batched":
            run_reference_batched(args, args.workload)
        else:
            run_reference(args, args.workload)
    elif kind == "csr":
        run_csr(args, args.workload)
    elif kind == "batched":
        run_batched(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
