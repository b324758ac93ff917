#!/usr/bin/env python
"""rand_cholQR benchmark: effective HBM GB/s of the factorization of an m x n FP64 matrix.

Workload (the large single-matrix configuration): m = 2^23 rows, n = 64 columns,
kappa = 1e12, V = U diag(sigma) W^T (seeded, synthetic), CountSketch s1 = 2(n^2+n),
Gaussian sketch s2 = 4n.  One step = one full rand_cholQR call (sketch, Householder R_s,
W = V R_s^{-1}, Gram, Cholesky, Q = W R_c^{-1}, R = R_c R_s) on data resident in HBM.

Metric: effective GB/s = 32 m n / t -- the method's algorithmic traffic (three reads of V
and one write of Q, FP64) over the step time; V is 4.3 GB, far larger than the 129 MB L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 (under torchrun) factors ONE matrix of N m rows, row-sharded over the ranks (Sec. 4.1):
each rank holds m rows, and the step's two cross-shard sums (the s2 x n sketch and the n x n
Gram) are NCCL allreduces.  Per-rank work is fixed (weak scaling); the value is the
whole-job aggregate.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Derived FP64 ALU peak: 2 DFMA/clk/SM (GB300's FP64 units) x 152 SMs x 2.07 GHz x 2 flops.
FP64_ALU_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12



# Roofline model per kernel kind: (bound, algorithmic units per row of V per launch).
# FP64 CUDA-core passes are bound by the FP64 pipe (flops per row); the pair-arithmetic and
# tensor-core passes, and the CountSketch scatter, by HBM (bytes per row: an 8-byte FP64
# or (hi, lo) FP32 pair read per element, plus the write for the solves).

def identity_gap2(G):
    """||G - I||_2 of a small symmetric Gram, on the host (numpy's symmetric eigensolver); inf
    when G is not finite, so that a maximum over results cannot hide a bad one."""
    import numpy as np
    Gh = G.double().cpu().numpy()
    if not np.isfinite(Gh).all():
        return float("inf")
    return float(np.abs(np.linalg.eigvalsh(Gh - np.eye(Gh.shape[0]))).max())

def roofline_model(kind, n):
    return {"trsm": ("alu", n * n), "gram": ("alu", n * (n + 1)),
            "cs_scatter": ("hbm", 8 * n), "trsm_df": ("hbm", 16 * n),
            "gram_df": ("hbm", 8 * n), "gram_tc": ("hbm", 8 * n),
            "trsm_tc": ("hbm", 16 * n), "solve_gram": ("hbm", 16 * n)}.get(kind)


# DRAM bytes per row of V (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture at
# m = 2^20, n = 64 with --set full, divided by m), scaled to a launch by the rows it processes.
# Valid for n = 64 and the kernels as captured (the capture of commit b7e56f9: k_trsm_oz's
# full-width instance, the mean of its two launches, and k_gram_split<64>; of commit adeb14f:
# k_solve_gram, the mean of two launches); a kernel changed since its capture has no entry (its
# traffic is reported as null until it is captured again).
MEASURED_DRAM_BYTES_PER_ROW_N64 = {"trsm_tc": (543.559e6 + 486.409e6) / 1048576,
                                   "gram_tc": (537.007e6 + 3.075e6) / 1048576,
                                   "solve_gram": (537.512e6 + 492.633e6) / 1048576}


# The unit a kernel kind's roofline is taken over, and how many of them one factorization runs:
# a solve is one launch for n <= 64 and three or four block products above, the Gram one launch
# or two (the first 64 columns, then the rest against all).
UNIT_NAME = {"trsm_tc": "solve", "gram_tc": "Gram"}
UNITS_PER_STEP = {"trsm_tc": 2, "gram_tc": 1, "solve_gram": 1, "cs_scatter": 1}


def dominant_roofline(kt, ms_per_step, steps, m, n):
    """The roofline object of the kernel kind with the most device time over `steps` steps
    (kt: {kind: (total ms, launches)}), taken per unit of UNITS_PER_STEP (a solve, a Gram) or
    per launch, with its share of the step."""
    kind, (tot_ms, launches) = max(kt.items(), key=lambda kv: kv[1][0])
    units = UNITS_PER_STEP.get(kind, launches / steps) * steps
    roof = kernel_roofline(kind, tot_ms / units, m, n)
    roof["kernel_share"] = tot_ms / (ms_per_step * steps)
    return roof


def kernel_roofline(kind, avg_ms, m, n):
    model = roofline_model(kind, n)
    if model is None:
        return {"bound": None, "kernel": kind, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None}
    bound, per_row = model
    if bound == "alu":
        achieved = per_row * m / (avg_ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": kind, "achieved": achieved,
                "peak": FP64_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_ALU_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz",
                "algorithmic": f"{per_row} FP64 flops per row x {m} rows per launch"}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    achieved = per_row * m / (avg_ms / 1e3) / 1e9
    traffic = MEASURED_DRAM_BYTES_PER_ROW_N64[kind] * m if (n == 64 and kind in MEASURED_DRAM_BYTES_PER_ROW_N64) else None
    return {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "traffic_source": ("ncu dram bytes per row at m=2^20, n=64, scaled by m" if traffic else
                               "not captured since the kernel last changed"),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
            "algorithmic": f"{per_row} bytes per row x {m} rows per {UNIT_NAME.get(kind, 'launch')}"}

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=2**23)
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--kappa", type=float, default=1e12)
    p.add_argument("--s1", type=int, default=0, help="CountSketch size (default 2 (n^2 + n))")
    p.add_argument("--s2", type=int, default=0, help="Gaussian sketch size (default 4 n)")
    p.add_argument("--prec", default="fp64", choices=["fp64", "f32x2"])
    p.add_argument("--fused", action="store_true",
                   help="n = 64: the first solve and the Gram in one fused launch instead of two")
    p.add_argument("--no-extras", action="store_true",
                   help="skip e2e, baselines, CPU baseline (quick runs)")
    p.add_argument("--no-serve", action="store_true", help="skip the served-stream measurement")
    p.add_argument("--serve-requests", type=int, default=20000,
                   help="requests of the served stream (the configuration's full stream is 20000)")
    p.add_argument("--gen", default="qr", choices=["qr", "gauss"],
                   help="qr: V = U diag(sigma) W^T; gauss: plain N(0,1/m) entries (kappa ~ 1, "
                        "no QR in the generator -- for profiler runs)")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def sketch_sizes(a):
    """(s1, s2) of the run: the method's 2 (n^2 + n) and 4 n unless given."""
    d1, d2 = 2 * (a.n * a.n + a.n), 4 * a.n
    return (a.s1 or d1), (a.s2 or d2)


def workload_name(a):
    s1, s2 = sketch_sizes(a)
    return f"rand_cholQR m={a.m} n={a.n} kappa={a.kappa:g} s1={s1} s2={s2}"


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for i, nm in enumerate(names):
                    if r[5 + i].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, single-threaded, on a bounded row sample
# ---------------------------------------------------------------------------------------
def cpu_baseline(n, kappa, rows, s1, s2):
    import oracle
    import synthetic
    V = synthetic.make_v(rows, n, kappa, seed=0)
    S2 = oracle.gauss_sketch(1, s2, s1)
    t0 = time.perf_counter()
    oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    dt = time.perf_counter() - t0
    return {"value": 32.0 * rows * n / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"rand_cholQR of the first {rows} rows (m={rows}, n={n}, kappa={kappa:g}, "
                      f"same s1/s2), single-threaded FP64 C oracle, {dt:.1f} s"}


def fp64_dgemm_tflops(torch, dev, size=8192, reps=3):
    """Context for the FP64 roof: cuBLAS DGEMM (torch.matmul on FP64, size^3), TFLOP/s by CUDA
    events over `reps` products after one warm-up."""
    a = torch.randn((size, size), dtype=torch.float64, device=dev)
    b = torch.randn((size, size), dtype=torch.float64, device=dev)
    c = a @ b
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        c = a @ b
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * size ** 3 / (ms / 1e3) / 1e12


def cpu_baseline_small():
    """The oracle on the small-matrix configuration (m = 20000, n = 16, kappa = 1e10,
    s1 = 544, s2 = 64): microseconds per call, single thread, the mean of 5 calls."""
    import oracle
    import synthetic
    m, n = 20000, 16
    V = synthetic.make_v(m, n, 1e10, seed=0)
    S2 = oracle.gauss_sketch(1, 64, 544)
    oracle.rand_cholqr(V, 544, 64, seed=0, S2=S2)
    t0 = time.perf_counter()
    for _ in range(5):
        oracle.rand_cholqr(V, 544, 64, seed=0, S2=S2)
    us = (time.perf_counter() - t0) / 5 * 1e6
    return {"value": us, "unit": "us per call", "cores": 1, "kind": "oracle",
            "sample": "rand_cholQR m=20000 n=16 kappa=1e10 s1=544 s2=64, single-threaded FP64 C oracle"}


def cpu_baseline_parallel(n, kappa, rows, s1, s2):
    """The oracle's own routines, unchanged, on every host core: the row-block decomposition
    of Sec. 4.1 (per-block CountSketch with the global row index, trsm and Gram), one thread per
    block (the routines release the interpreter lock), the small steps on one core, the two
    block sums in fixed order.  The same algorithm as the oracle, parallel over row blocks."""
    import threading

    import numpy as np

    import oracle
    import synthetic
    cores = os.cpu_count() or 1
    V = synthetic.make_v(rows, n, kappa, seed=0)
    S2 = oracle.gauss_sketch(1, s2, s1)
    cuts = [rows * k // cores for k in range(cores + 1)]
    blocks = [(cuts[k], cuts[k + 1]) for k in range(cores) if cuts[k + 1] > cuts[k]]
    out = [None] * len(blocks)

    def par(fn):
        ts = [threading.Thread(target=fn, args=(k, a, b)) for k, (a, b) in enumerate(blocks)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()

    t0 = time.perf_counter()

    def sk(k, a, b):
        out[k] = oracle.countsketch_rows(V[a:b], s1, 0, a)
    par(sk)
    W1 = out[0].copy()
    for w in out[1:]:
        W1 += w
    Rs = oracle.hhqr_r(oracle.gemm(S2, W1))
    Ws_blocks = [None] * len(blocks)

    def wg(k, a, b):
        W = oracle.trsm(V[a:b], Rs)
        Ws_blocks[k] = W
        out[k] = oracle.gram(W)
    par(wg)
    G = out[0].copy()
    for g in out[1:]:
        G += g
    Rc = oracle.chol(G)

    def fin(k, a, b):
        out[k] = oracle.trsm(Ws_blocks[k], Rc)
    par(fin)
    oracle.trmm(Rc, Rs)
    dt = time.perf_counter() - t0
    return {"value": 32.0 * rows * n / dt / 1e9, "unit": "GB/s", "cores": len(blocks), "kind": "oracle",
            "sample": f"rand_cholQR of the first {rows} rows (n={n}, kappa={kappa:g}, same s1/s2): the "
                      f"oracle's routines over {len(blocks)} row blocks in {len(blocks)} threads "
                      f"(Sec. 4.1 decomposition), {dt:.2f} s"}


def run_reference(a):
    """--impl reference: the oracle, timed on the host cores, on a bounded sample per step."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    import synthetic
    rows = 1 << 16
    s1, s2 = sketch_sizes(a)
    V = synthetic.make_v(rows, a.n, a.kappa, seed=0)
    S2 = oracle.gauss_sketch(1, s2, s1)
    for _ in range(a.warmup):
        oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    dt = (time.perf_counter() - t0) / a.steps
    value = 32.0 * rows * a.n / dt / 1e9
    line = {"impl": "reference", "metric": "rand_cholQR effective HBM GB/s (m x n FP64)",
            "value": value, "unit": "GB/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample_rows": rows},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {rows} rows of the workload per step"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# Served stream: Poisson arrivals of requests through randqr_submit / randqr_poll
# ---------------------------------------------------------------------------------------
def serve_bench(rq, synthetic, torch, dev, n_req=20000, loads=(0.5, 0.8, 0.95), seed=7):
    """The served stream: requests with m log-uniform in [1e4, 4e6], n uniform in
    {4, 8, 16, 32, 64}, kappa one of 1, 1e4, 1e8, 1e12 with equal odds (one pre-built matrix
    per (n, kappa); a request takes its first m rows).  The sequential plain-FP64 service time of every
    request is measured first; arrivals are then Poisson at each offered load x that capacity,
    through randqr_submit / randqr_poll with 8 slots and a 64 GB budget, in FP64 and with
    max_orth_err = 1e-12 (the caller accepts 1e-12: rand_cholQR may take its reduced-precision
    row passes).  A saturation run (every request submitted at once) gives the served capacity.
    Reports p50/p99 latency and throughput per load, next to a single FIFO server running the
    measured sequential service times on the same arrivals, and the worst ||I - Q^T Q||_2 over a
    sample of each run's results."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ns = [4, 8, 16, 32, 64]
    klev = [1.0, 1e4, 1e8, 1e12]
    pools = {(n, k): synthetic.make_v_torch(4_000_000, n, k, seed=100 + n, device=dev)
             for n in ns for k in klev}
    reqs = []
    for _ in range(n_req):
        m = int(np.exp(rng.uniform(np.log(1e4), np.log(4e6))))
        n = int(rng.choice(ns))
        k = klev[min(3, int(rng.uniform(0, 12) // 3))]
        reqs.append((m, n, k))
    ctx = rq.Context(dev.index or 0)
    qbuf = {}
    for (m, n, k) in sorted(set(reqs), key=lambda r: -r[0] * r[1])[:16]:
        qbuf[(m, n)] = (torch.empty((m, n), dtype=torch.float64, device=dev),
                        torch.empty((n, n), dtype=torch.float64, device=dev))
    for (m, n, k) in sorted(set(reqs), key=lambda r: -r[0] * r[1])[:16]:  # workspaces, sketches
        rq.randqr_factor(pools[(n, k)][:m], seed=0, ctx=ctx, Q=qbuf[(m, n)][0], R=qbuf[(m, n)][1])
    svc = []
    for (m, n, k) in reqs:
        Q = torch.empty((m, n), dtype=torch.float64, device=dev)
        R = torch.empty((n, n), dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        rq.randqr_factor(pools[(n, k)][:m], seed=0, ctx=ctx, Q=Q, R=R)  # waits for the status
        svc.append(time.perf_counter() - t0)
    ctx.close()
    mean_svc = float(np.mean(svc))

    def pct(x, p):
        return float(np.percentile(np.asarray(x) * 1e3, p))

    def run_served(max_orth, arrivals, max_outstanding=None):
        """One pass of the stream; arrivals None: saturation (at most max_outstanding requests
        submitted and not finished at any time, refilled as they finish)."""
        sctx = rq.Context(dev.index or 0)
        rq.randqr_serve_config(sctx, slots=8, hbm_budget_bytes=64 << 30)
        for (m, n, k) in sorted(set(reqs), key=lambda r: -r[0] * r[1])[:16]:
            Q, R = qbuf[(m, n)]
            t, _ = rq.randqr_submit(sctx, pools[(n, k)][:m], Q=Q, R=R, seed=0, max_orth_err=max_orth)
            rq.randqr_wait(sctx, t)
        torch.cuda.synchronize()
        lat, pending, nxt, sample = [], {}, 0, {}
        t0 = time.perf_counter()
        sub_t = {}
        while len(lat) < n_req:
            now = time.perf_counter() - t0
            while nxt < n_req and ((arrivals is None and len(pending) < max_outstanding) or
                                   (arrivals is not None and arrivals[nxt] <= now)):
                m, n, k = reqs[nxt]
                # every request in flight has buffers of its own (freed when it finishes)
                Q = torch.empty((m, n), dtype=torch.float64, device=dev)
                R = torch.empty((n, n), dtype=torch.float64, device=dev)
                if nxt % max(1, n_req // 200) == 0:  # about 200 kept for the accuracy sample
                    sample[nxt] = (Q, R)
                t, _ = rq.randqr_submit(sctx, pools[(n, k)][:m], Q=Q, R=R, seed=0, max_orth_err=max_orth)
                pending[t] = nxt
                sub_t[t] = arrivals[nxt] if arrivals is not None else time.perf_counter() - t0
                nxt += 1
            for t in list(pending):
                st, _ = rq.randqr_poll(sctx, t)
                if st != rq.PENDING:
                    if st != 0:
                        raise rq.RandQRError(st)
                    pending.pop(t)
                    lat.append(time.perf_counter() - t0 - sub_t.pop(t))
            if arrivals is not None and not pending and nxt < n_req:
                time.sleep(max(0.0, min(0.001, arrivals[nxt] - (time.perf_counter() - t0))))
        span = time.perf_counter() - t0
        gaps, first = [], []
        for i, (Q, R) in sample.items():
            G = Q.T @ Q
            gaps.append(identity_gap2(G))
            if len(first) < 3:  # what the first sampled results look like
                first.append({"request": i, "m": Q.shape[0], "n": Q.shape[1], "gap": gaps[-1],
                              "q_fro2": float((Q * Q).sum().item()), "r00": float(R[0, 0].item())})
        sctx.close()
        return {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "throughput_req_s": n_req / span,
                "eff_GBs": bytes_total / span / 1e9, "max_orth_err_2_sampled": max(gaps, default=float("nan")),
                "samples": len(gaps), "samples_not_finite": sum(1 for g in gaps if g == float("inf")),
                "samples_exact": sum(1 for g in gaps if g == 0.0), "first_samples": first}

    bytes_total = sum(32.0 * m * n for (m, n, k) in reqs)
    res = {"requests": n_req, "slots": 8, "budget_bytes": 64 << 30,
           "workload": "m log-uniform [1e4, 4e6], n in {4,8,16,32,64}, kappa in {1,1e4,1e8,1e12}",
           "sequential_fp64": {"mean_service_ms": mean_svc * 1e3, "capacity_req_s": 1.0 / mean_svc},
           "loads": {}}
    for load in loads:
        arr = np.cumsum(np.random.default_rng(seed + int(load * 100)).exponential(mean_svc / load, size=n_req))
        free_at, seq_lat = 0.0, []
        for a_t, sv in zip(arr, svc):
            start = max(a_t, free_at)
            free_at = start + sv
            seq_lat.append(free_at - a_t)
        res["loads"][str(load)] = {
            "rate_per_s": load / mean_svc,
            "sequential_fp64": {"p50_ms": pct(seq_lat, 50), "p99_ms": pct(seq_lat, 99)},
            "served_fp64": run_served(0.0, arr), "served_mixed": run_served(1e-12, arr)}
    res["saturation"] = {"max_outstanding": 32, "served_fp64": run_served(0.0, None, 32),
                         "served_mixed": run_served(1e-12, None, 32)}
    mid = res["loads"].get("0.8") or next(iter(res["loads"].values()))
    res["served_fp64"] = dict(mid["served_fp64"], max_orth_err_2=mid["served_fp64"]["max_orth_err_2_sampled"])
    res["served_mixed"] = dict(mid["served_mixed"], max_orth_err_2=mid["served_mixed"]["max_orth_err_2_sampled"])
    del pools, qbuf
    return res


# ---------------------------------------------------------------------------------------
# Batched: 512 uneven matrices in one autotuned graph launch
# ---------------------------------------------------------------------------------------
def batch_bench(rq, synthetic, torch, dev, count=512, seed=11):
    """m log-uniform in [4096, 262144], n uniform in {8, 16, 32, 64}, kappa log-uniform in
    [1, 1e12] (one 262144-row matrix per (n, kappa decade pair); an item takes its first m
    rows), default sketch sizes per item.  Times graph replays of randqr_factor_batched
    against the same factorizations issued one call after another on one stream."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ns = [8, 16, 32, 64]
    klev = [1.0, 1e3, 1e6, 1e9, 1e12]
    pools = {(n, k): synthetic.make_v_torch(262144, n, k, seed=200 + n, device=dev)
             for n in ns for k in klev}
    shapes = []
    for _ in range(count):
        m = int(np.exp(rng.uniform(np.log(4096), np.log(262144))))
        n = int(rng.choice(ns))
        k = klev[min(4, int(rng.uniform(0, 12) // 2.4))]
        shapes.append((m, n, k))
    Vs = [pools[(n, k)][:m] for (m, n, k) in shapes]
    Qs = [torch.empty((m, n), dtype=torch.float64, device=dev) for (m, n, k) in shapes]
    Rs = [torch.empty((n, n), dtype=torch.float64, device=dev) for (m, n, k) in shapes]
    bytes_total = sum(32.0 * m * n for (m, n, k) in shapes)
    out = {"count": count, "V_bytes": sum(8.0 * m * n for (m, n, k) in shapes),
           "workload": "m log-uniform [4096, 262144], n in {8,16,32,64}, kappa in {1,1e3,1e6,1e9,1e12}"}
    stream = torch.cuda.current_stream()
    for prec, name in ((rq.FP64, "fp64"), (rq.F32X2, "f32x2")):
        ctx = rq.Context(dev.index or 0)
        items = rq.batch_items(Vs, Qs, Rs, seeds=list(range(count)))
        t0 = time.perf_counter()
        sts = rq.randqr_factor_batched(ctx, items, prec=prec)
        plan_s = time.perf_counter() - t0
        if any(s != 0 for s in sts):
            raise RuntimeError(f"batched statuses {set(sts)}")
        lanes, tuned_ms = rq.randqr_batch_plan_info(ctx, items, prec=prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            rq.randqr_factor_batched(ctx, items, prec=prec, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        # the same factorizations, one call after another on one stream
        seq_ctx = rq.Context(dev.index or 0)
        for i, V in enumerate(Vs):
            rq.randqr_factor(V, seed=i, prec=prec, Q=Qs[i], R=Rs[i], ctx=seq_ctx, sync=False)
        torch.cuda.synchronize()
        e0.record(stream)
        for i, V in enumerate(Vs):
            rq.randqr_factor(V, seed=i, prec=prec, Q=Qs[i], R=Rs[i], ctx=seq_ctx, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1)
        rq.randqr_factor_batched(ctx, items, prec=prec)
        worst = 0.0
        for i in range(0, count, 32):
            worst = max(worst, identity_gap2(Qs[i].T @ Qs[i]))
        out[name] = {"ms_per_batch": ms, "eff_GBs": bytes_total / (ms / 1e3) / 1e9,
                     "lanes": lanes, "autotune_ms": tuned_ms, "plan_build_s": plan_s,
                     "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / ms,
                     "max_orth_err_2_sampled": worst}
        seq_ctx.close()
        ctx.close()
    del pools, Vs, Qs, Rs
    return out


# ---------------------------------------------------------------------------------------
# The other single-matrix configurations: small-matrix latency, and the large matrix at the
# other column counts and precisions, each with its accuracy against the FP64 targets.
# ---------------------------------------------------------------------------------------
def small_latency(rq, synthetic, torch, dev, reps=200):
    """m = 20000, n = 16, kappa = 1e10 (s1 = 544, s2 = 64): the matrix is 2.56 MB, L2-resident,
    so the call is latency-bound.  Reports the device time per call (back-to-back on one
    stream, CUDA events) and the host wall time of a call that waits for its status."""
    m, n, kappa = 20000, 16, 1e10
    s1, s2 = 2 * (n * n + n), 4 * n
    V = synthetic.make_v_torch(m, n, kappa, seed=0, device=dev)
    Q = torch.empty_like(V)
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    ctx = rq.Context(dev.index or 0)
    stream = torch.cuda.current_stream()
    for _ in range(10):
        rq.randqr_factor(V, s1, s2, seed=0, Q=Q, R=R, ctx=ctx, sync=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        rq.randqr_factor(V, s1, s2, seed=0, Q=Q, R=R, ctx=ctx, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    dev_us = e0.elapsed_time(e1) / reps * 1e3
    walls = []
    for _ in range(50):
        t0 = time.perf_counter()
        rq.randqr_factor(V, s1, s2, seed=0, Q=Q, R=R, ctx=ctx)  # waits for the status
        walls.append((time.perf_counter() - t0) * 1e6)
    _, _, info = rq.randqr_factor(V, s1, s2, seed=0, Q=Q, R=R, ctx=ctx, accuracy=True)
    ctx.close()
    return {"workload": f"rand_cholQR m={m} n={n} kappa={kappa:g} s1={s1} s2={s2}",
            "device_us_per_call": dev_us, "wall_us_p50": statistics.median(walls),
            "wall_us_min": min(walls), "orth_err_2": info.orth_err2, "resid_rel_F": info.resid_relF}


def large_config(rq, synthetic, torch, dev, m, n, kappa, prec, steps=3):
    """One large single-matrix configuration: ms per step, effective GB/s (32 m n bytes per
    step) and the accuracy the call states about its result."""
    s1, s2 = 2 * (n * n + n), 4 * n
    V = synthetic.make_v_torch(m, n, kappa, seed=1, device=dev)
    Q = torch.empty_like(V)
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    ctx = rq.Context(dev.index or 0)
    stream = torch.cuda.current_stream()
    rq.randqr_factor(V, s1, s2, seed=0, prec=prec, Q=Q, R=R, ctx=ctx, sync=False)
    torch.cuda.synchronize()
    ctx.kernel_times()
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rq.randqr_factor(V, s1, s2, seed=0, prec=prec, Q=Q, R=R, ctx=ctx, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    kt = ctx.kernel_times()
    ms = e0.elapsed_time(e1) / steps
    st, _ = rq.get_status(ctx)
    _, _, info = rq.randqr_factor(V, s1, s2, seed=0, prec=prec, Q=Q, R=R, ctx=ctx, accuracy=True)
    ctx.close()
    del V, Q
    torch.cuda.empty_cache()
    return {"m": m, "n": n, "kappa": kappa, "precision": "fp64" if prec == rq.FP64 else "f32x2",
            "ms_per_step": ms, "value": 32.0 * m * n / (ms / 1e3) / 1e9, "unit": "GB/s", "status": st,
            "orth_err_2": info.orth_err2, "resid_rel_F": info.resid_relF,
            "kernels_ms_per_step": {k: v[0] / steps for k, v in kt.items()}}


def l2_resident_rowpass(rq, synthetic, torch, dev, m=1 << 17, n=64, steps=20):
    """The row-pass kernels on one matrix small enough to stay in L2 between steps (in-place
    factorization, m x n FP64 = 64 MB at the defaults against 129 MB of L2), timed twice: warm
    (nothing else runs between the steps, so the kernels read V from L2) and cold (a 512 MB
    buffer is written between the steps, so they read it from HBM).  Same launches, same sizes:
    equal per-kernel times mean the kernel is bound by its own work, not by its HBM traffic."""
    V0 = synthetic.make_v_torch(m, n, 1e12, seed=3, device=dev)
    V = V0.clone()
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    flush = torch.empty(1 << 26, dtype=torch.float64, device=dev)
    ctx = rq.Context(dev.index or 0)
    s1, s2 = 2 * (n * n + n), 4 * n
    out = {"m": m, "n": n, "bytes_resident": 8 * m * n}
    for mode in ("warm", "cold"):
        for _ in range(3):
            V.copy_(V0)
            rq.randqr_factor(V, s1, s2, seed=0, Q=V, R=R, ctx=ctx, sync=False)
        torch.cuda.synchronize()
        ctx.kernel_times()
        ctx.set_profiling(True)
        for _ in range(steps):  # Q = V in place: the step's working set stays at m n 8 bytes
            if mode == "cold":
                flush.fill_(1.0)
            rq.randqr_factor(V, s1, s2, seed=0, Q=V, R=R, ctx=ctx, sync=False)
        torch.cuda.synchronize()
        ctx.set_profiling(False)
        kt = ctx.kernel_times()
        out[mode + "_kernels_us"] = {k: 1e3 * v[0] / steps for k, v in kt.items()}
    st, _ = rq.get_status(ctx)
    out["status"] = st
    ctx.close()
    del V, V0, flush
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------------
def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_05868_gb300 as rq
    from paper_2309_05868_gb300 import sharded
    import synthetic

    m, n = a.m, a.n
    s1, s2 = sketch_sizes(a)
    prec = rq.FP64 if a.prec == "fp64" else rq.F32X2
    dev = torch.device("cuda", local_rank)
    if world > 1 and a.prec != "fp64":
        raise SystemExit("the row-sharded path (N > 1) runs FP64 row passes only")
    if world > 1 and a.gen == "qr":
        V = synthetic.make_v_block_torch(m, n, a.kappa, rank, world, seed=0, device=dev)
    elif a.gen == "qr":
        V = synthetic.make_v_torch(m, n, a.kappa, seed=rank, device=dev)
    else:
        g = torch.Generator(device=dev)
        g.manual_seed(rank)
        V = torch.randn((m, n), generator=g, device=dev, dtype=torch.float64) / m ** 0.5
    Q = torch.empty_like(V)
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    ctx = rq.Context(local_rank)
    if a.fused:
        ctx.set_fused_first_pass(True)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stages = sharded.DeviceStages(ctx, stream, sync=False)
    allreduce = sharded.dist_allreduce() if world > 1 else None

    def factor_once(Vin, prec_):
        if world > 1:
            _, Rk = sharded.factor_row_sharded(Vin, rank * m, allreduce, s1, s2, seed=0, Q=Q,
                                               stages=stages)
            R.copy_(Rk)
        else:
            rq.randqr_factor(Vin, s1, s2, seed=0, prec=prec_, Q=Q, R=R, ctx=ctx, sync=False)

    def measure(prec_, steps, sample_clocks=False):
        def step():
            factor_once(V, prec_)

        for _ in range(max(a.warmup, 3)):
            step()
        st, info = rq.get_status(ctx)
        if st != 0:
            raise rq.RandQRError(st, info)
        ctx.kernel_times()  # clear
        ctx.set_profiling(True)
        clocks = ClockSampler(local_rank)
        if sample_clocks:
            clocks.start()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if sample_clocks else None
        ms_ = e0.elapsed_time(e1) / steps
        ctx.set_profiling(False)
        kt_ = ctx.kernel_times()
        st, info = rq.get_status(ctx)
        if st != 0:
            raise rq.RandQRError(st, info)
        if world > 1:
            t = torch.tensor([ms_], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms_ = t.item()
        # accuracy of the timed result (whole matrix, checked on the device with torch; the
        # row blocks' Q^T Q and squared norms summed over the ranks)
        G = Q.T @ Q
        sq = torch.stack([torch.linalg.norm(V - Q @ R) ** 2, torch.linalg.norm(V) ** 2])
        if world > 1:
            torch.distributed.all_reduce(G)
            torch.distributed.all_reduce(sq)
        orth = identity_gap2(G)
        resid = (sq[0] / sq[1]).sqrt().item()
        return ms_, kt_, clk, {"orth_err_2": orth, "resid_rel_F": resid}

    ms, kt, clk, acc = measure(prec, a.steps, sample_clocks=True)

    algo_bytes = 32.0 * m * n
    value = algo_bytes * world / (ms / 1e3) / 1e9

    roof = dominant_roofline(kt, ms, a.steps, m, n)

    line = {"metric": "rand_cholQR effective HBM GB/s (m x n FP64)", "value": value,
            "unit": "GB/s", "n_gpus": world, "steps": a.steps, "warmup": max(a.warmup, 3),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.prec == "fp64" else "f32x2",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "m": m, "n": n, "kappa": a.kappa,
                       "s1": s1, "s2": s2, "precision": a.prec,
                       "parallelism": f"row-sharded x{world} (NCCL allreduce of the sketch and Gram)"
                       if world > 1 else "single",
                       "l2": "inputs larger than L2 (V = %.1f GB)" % (8.0 * m * n / 1e9)},
            "roofline": roof, "clocks": clk,
            "gpu_launches": sum(c for _, c in kt.values()),
            "kernels_ms_per_step": {k: v[0] / a.steps for k, v in kt.items()},
            "accuracy": acc}

    # everything past the timed step is context: on one GPU a failure there must not cost
    # the line (with several ranks it ends the run, since the ranks meet in collectives)
    try:
        if not a.no_extras and world == 1:
            # the row-sharded decomposition as logical shards on this GPU (sums in shard order)
            P = 4
            cuts = sharded.even_cuts(m, P)
            Qs = Q

            def logical_step():
                sharded.factor_logical_shards(V, cuts, s1, s2, seed=0, Q=Qs, stages=stages)

            for _ in range(3):
                logical_step()
            torch.cuda.synchronize()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            for _ in range(3):
                logical_step()
            h1.record(stream)
            torch.cuda.synchronize()
            sh_ms = h0.elapsed_time(h1) / 3
            st, info = rq.get_status(ctx)
            line["sharded_logical"] = {"shards": P, "ms_per_step": sh_ms,
                                       "value": algo_bytes / (sh_ms / 1e3) / 1e9, "unit": "GB/s",
                                       "over_unsharded": sh_ms / ms, "status": st}

        if not a.no_extras and world == 1:
            # the paper's multisketch sizes (Sec. 6.2) on the same matrix: a larger sketch GEMM
            p1, p2 = synthetic.paper_multisketch_sizes(n)
            for _ in range(2):
                rq.randqr_factor(V, p1, p2, seed=0, prec=prec, Q=Q, R=R, ctx=ctx, sync=False)
            torch.cuda.synchronize()
            ctx.kernel_times()
            ctx.set_profiling(True)
            p0, pe = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for _ in range(3):
                rq.randqr_factor(V, p1, p2, seed=0, prec=prec, Q=Q, R=R, ctx=ctx, sync=False)
            pe.record(stream)
            torch.cuda.synchronize()
            ctx.set_profiling(False)
            pkt = ctx.kernel_times()
            pms = p0.elapsed_time(pe) / 3
            st, _ = rq.get_status(ctx)
            line["paper_sketch_sizes"] = {"s1": p1, "s2": p2, "ms_per_step": pms, "status": st,
                                          "value": algo_bytes / (pms / 1e3) / 1e9, "unit": "GB/s",
                                          "kernels_ms_per_step": {k: v[0] / 3 for k, v in pkt.items()}}

        if not a.no_extras:
            if world == 1:
                # the other precision of the row passes, on the same matrix
                other = "f32x2" if a.prec == "fp64" else "fp64"
                oprec = rq.F32X2 if other == "f32x2" else rq.FP64
                oms, okt, _, oacc = measure(oprec, a.steps)
                line["modes"] = {other: {"value": algo_bytes / (oms / 1e3) / 1e9, "unit": "GB/s",
                                         "ms_per_step": oms, "accuracy": oacc,
                                         "kernels_ms_per_step": {k: v[0] / a.steps for k, v in okt.items()}}}
                # the first row pass as one fused launch or as two (solve, then the Gram of W)
                ctx.set_fused_first_pass(not a.fused)
                tms, tkt, _, tacc = measure(prec, a.steps)
                ctx.set_fused_first_pass(a.fused)
                line["modes"]["two_pass" if a.fused else "fused_first_pass"] = {
                    "value": algo_bytes / (tms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": tms,
                    "accuracy": tacc, "kernels_ms_per_step": {k: v[0] / a.steps for k, v in tkt.items()}}

            # end to end through the public API: pinned host V in, Q and R back to pinned host,
            # every step.  On one GPU that is the host-buffer call randqr_factor_host (its own
            # upload, factorization in the context's staging area, download); consecutive steps
            # alternate between two contexts on two streams, so step i + 1's upload overlaps step
            # i's factorization and download (the pipeline a caller streaming matrices through the
            # GPU would use).  Row shards (N > 1) copy around the sharded device call the same way.
            Vh = V.cpu().pin_memory()
            ke = max(2, min(a.steps, 6))
            if world == 1:
                Qh = [torch.empty_like(Vh).pin_memory() for _ in range(2)]
                Rh = [torch.empty((n, n), dtype=torch.float64).pin_memory() for _ in range(2)]
                hctx = [ctx, rq.Context(local_rank)]
                hst = [torch.cuda.Stream(device=dev) for _ in range(2)]
                done = [torch.cuda.Event() for _ in range(2)]

                def e2e_step(i):
                    b = i % 2
                    rq.randqr_factor_host(Vh, s1, s2, seed=0, prec=prec, Q=Qh[b], R=Rh[b], ctx=hctx[b],
                                          stream=hst[b], sync=False)
                    done[b].record(hst[b])

                for i in range(2):  # staging areas, workspaces and sketches in place
                    e2e_step(i)
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                for b in range(2):
                    hst[b].wait_event(f0)
                for i in range(ke):
                    e2e_step(i)
                for b in range(2):
                    stream.wait_event(done[b])
                f1.record(stream)
                torch.cuda.synchronize()
                for b in range(2):
                    st_b, _ = rq.get_status(hctx[b], hst[b])
                    if st_b != 0:
                        raise SystemExit(f"randqr_factor_host failed with status {st_b}")
                e2e_ms = f0.elapsed_time(f1) / ke
                del Qh, hctx
                pipeline = ("randqr_factor_host on pinned host buffers; consecutive steps on two "
                            "contexts and streams, so uploads, factorizations and downloads overlap")
            else:
                Qh = torch.empty_like(Vh).pin_memory()
                Rh = torch.empty((n, n), dtype=torch.float64).pin_memory()
                Vd = [torch.empty_like(V) for _ in range(2)]
                Qd = [torch.empty_like(V) for _ in range(2)]
                Rd = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(2)]
                s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
                ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "comp", "out")}

                def e2e_step(i):
                    b = i % 2
                    with torch.cuda.stream(s_in):
                        if i >= 2:
                            s_in.wait_event(ev["comp"][b])  # step i - 2 has read Vd[b]
                        Vd[b].copy_(Vh, non_blocking=True)
                        ev["in"][b].record(s_in)
                    stream.wait_event(ev["in"][b])
                    if i >= 2:
                        stream.wait_event(ev["out"][b])  # step i - 2's download has read Qd[b], Rd[b]
                    _, Rk = sharded.factor_row_sharded(Vd[b], rank * m, allreduce, s1, s2, seed=0, Q=Qd[b],
                                                       stages=stages)
                    Rd[b].copy_(Rk)
                    ev["comp"][b].record(stream)
                    with torch.cuda.stream(s_out):
                        s_out.wait_event(ev["comp"][b])
                        Qh.copy_(Qd[b], non_blocking=True)
                        Rh.copy_(Rd[b], non_blocking=True)
                        ev["out"][b].record(s_out)

                for i in range(2):
                    e2e_step(i)
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                s_in.wait_event(f0)
                for i in range(ke):
                    e2e_step(i)
                stream.wait_event(ev["out"][(ke - 1) % 2])
                stream.wait_event(ev["out"][(ke - 2) % 2])
                f1.record(stream)
                torch.cuda.synchronize()
                e2e_ms = f0.elapsed_time(f1) / ke
                del Qh, Vd, Qd
                pipeline = "upload, sharded factorization and download of consecutive steps overlap (3 streams)"
            if world > 1:
                t = torch.tensor([e2e_ms], device=dev)
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
                e2e_ms = t.item()
            line["e2e"] = {"value": algo_bytes * world / (e2e_ms / 1e3) / 1e9, "unit": "GB/s",
                           "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": 8 * m * n + 8 * n * n,
                           "ms_per_step": e2e_ms, "pipeline": pipeline}
            del Vh

            # GPU baselines on a matrix all three can factor (kappa = 1e4), same size
            Vb = synthetic.make_v_torch(m, n, 1e4, seed=rank + 100, device=dev)
            times = {}
            for name, fn in [("rand_cholqr", lambda: rq.randqr_factor(Vb, s1, s2, seed=0, prec=prec, Q=Q, R=R, ctx=ctx, sync=False)),
                             ("cholqr2", lambda: rq.randqr_cholqr2(Vb, Q=Q, R=R, ctx=ctx, sync=False)),
                             ("shifted_cholqr3", lambda: rq.randqr_shifted_cholqr3(Vb, Q=Q, R=R, ctx=ctx, sync=False))]:
                fn()
                torch.cuda.synchronize()
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                for _ in range(3):
                    fn()
                g1.record(stream)
                torch.cuda.synchronize()
                times[name] = g0.elapsed_time(g1) / 3
                st, _ = rq.get_status(ctx)
                times[name + "_status"] = st
            line["baselines_ms"] = {"kappa": 1e4, **times,
                                    "rand_cholqr_over_cholqr2": times["rand_cholqr"] / times["cholqr2"],
                                    "rand_cholqr_over_shifted_cholqr3": times["rand_cholqr"] / times["shifted_cholqr3"]}
            del Vb
            if world == 1:
                line["small_matrix"] = small_latency(rq, synthetic, torch, dev)
                line["row_pass_l2_resident"] = l2_resident_rowpass(rq, synthetic, torch, dev)
                line["other_configs"] = [large_config(rq, synthetic, torch, dev, 1 << 23, 32, 1e12, rq.FP64)]
                # the headline shape across the conditioning range (accuracy; the timing does not
                # depend on kappa)
                for kap in (1.0, 1e4, 1e8, 1e15):
                    line["other_configs"].append(large_config(rq, synthetic, torch, dev, 1 << 23, 64, kap,
                                                              rq.FP64, steps=1))
                for kap in (1e2, 1e6, 1e10, 1e12):
                    for pr in (rq.FP64, rq.F32X2):
                        line["other_configs"].append(large_config(rq, synthetic, torch, dev, 1 << 23, 128, kap, pr,
                                                                  steps=1))
            if world == 1:
                try:  # context only: a failure here must not cost the line
                    line["fp64_dgemm_tflops"] = fp64_dgemm_tflops(torch, dev)
                except Exception as e:  # noqa: BLE001
                    line["fp64_dgemm_tflops"] = None
                    line["fp64_dgemm_error"] = str(e)[:200]
            if not a.no_serve:
                del Q
                torch.cuda.empty_cache()
                line["serving"] = serve_bench(rq, synthetic, torch, dev, n_req=a.serve_requests)
                torch.cuda.empty_cache()
                line["batched"] = batch_bench(rq, synthetic, torch, dev)
            if rank == 0:
                line["cpu_baseline"] = cpu_baseline(n, a.kappa, 1 << 18, s1, s2)
                line["cpu_baseline_parallel"] = cpu_baseline_parallel(n, a.kappa, 1 << 20, s1, s2)
                line["cpu_baseline_small"] = cpu_baseline_small()
    except Exception as e:  # noqa: BLE001
        if world > 1:
            raise
        line["extras_error"] = f"{type(e).__name__}: {str(e)[:300]}"

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
