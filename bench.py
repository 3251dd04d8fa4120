"""Benchmark of the ANOVA-NFFT matvec (arXiv 2312.00538, Sec. 3) on the 1e6-point workload.

Workload: n = 1,000,000 points, d = 9 N(0,1) features min-max scaled into [-0.2, 0.2], three
3-D windows, sigma = 1, bandwidth N = 32 (oversampled grid 64^3), Kaiser-Bessel cut-off m = 4,
FP32 plan, 1 right-hand side v ~ N(0,1). A step is one full matvec K v = sum_l K_l v (spread,
reduce, FFT/scale/IFFT passes, interpolation, window sum) with v already resident in HBM; the
plan (sort, tables) is built once before timing and reported separately. Between timed steps the
L2 cache is flushed by writing a 512 MiB buffer (the matvec's working set, ~80 MB, fits in L2).

`python bench.py --impl reference` times the FP64 CPU oracle (direct summation) on the host cores
instead, on a bounded row sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ANOVA-NFFT matvec pts/s"
UNIT = "pts/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES_PER_SM = 128     # FP32 FMA units per Blackwell SM
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--sigma", type=float, default=1.0)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="matvec: one problem split by rows over the GPUs (strong scaling) instead of one "
                         "independent problem per GPU")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="matvec", choices=["matvec", "ipm_batch", "serve", "precond_study", "predict",
                                                                   "matvec_batch", "woodbury", "serve5", "matvec64"],
                    help="matvec (default, the headline line) or ipm_batch (independent SVM "
                         "solves, one at a time vs concurrently)")
    ap.add_argument("--count", type=int, default=64, help="ipm_batch: number of problems")
    ap.add_argument("--rank", type=int, default=200, help="woodbury: preconditioner rank")
    ap.add_argument("--err-tol", type=float, default=0.0,
                    help="ipm_batch/serve5: pivoted-Cholesky tolerance (0: the workloads' stated rank 100; "
                         "Table 1: 1e-5)")
    ap.add_argument("--krylov-tol", type=float, default=1e-6,
                    help="ipm_batch/serve5: relative residual of each Newton solve (workload 3's MINRES tol)")
    ap.add_argument("--max-iter", type=int, default=150,
                    help="ipm_batch/serve5: interior point iterations (C = 100 problems take 80-110)")
    ap.add_argument("--rates", default="1,2,5,10,20,50", help="serve5: arrival rates (requests/s)")
    ap.add_argument("--concurrency", type=int, default=8, help="ipm_batch: concurrent solves")
    ap.add_argument("--m-precise", type=int, default=0,
                    help="ipm_batch/serve/serve5: window cut-off of the solver's FP64 plan (0: the library default)")
    ap.add_argument("--m-refine", type=int, default=-1,
                    help="ipm_batch/serve/serve5: window cut-off of the FP64 refinement plan (-1: the library "
                         "default, 0: the FP64 plan serves both)")
    ap.add_argument("--n-max", type=int, default=200_000, help="ipm_batch/serve: largest n")
    ap.add_argument("--rate", type=float, default=1.0,
                    help="serve: mean arrival rate of requests (Poisson, requests/s)")
    ap.add_argument("--budget-gib", type=float, default=64.0, help="serve: device-memory budget")
    ap.add_argument("--tune", action="store_true",
                    help="matvec: build the plan with anova_nfft_plan_tuned (launch-setting search)")
    ap.add_argument("--factors", default="cholesky_greedy,cholesky_rp,nystrom,cholesky_per_window",
                    help="precond_study: comma-separated low-rank factors to compare")
    ap.add_argument("--sizes", default="5000,20000,50000", help="precond_study: training sizes")
    return ap.parse_args()


def workload(n, seed_offset=0):
    from synth import config2, matvec_vectors, SEED_BASE
    cfg = config2(n=n, seed=SEED_BASE + 2 + seed_offset)
    return cfg["X"], cfg["windows"], SEED_BASE + 2 + 100 + seed_offset


def workload_name(n, sigma, nrhs):
    return "anova_nfft_matvec n=%d d=9 windows=3x3D sigma=%g N=32 m=4 nrhs=%d" % (n, sigma, nrhs)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi every 200 ms while running (SM clock, max clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9 or parts[0] != self.gpu:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing
def oracle_rows_per_s(X, W, sigma, v, budget_s, max_rows, seed):
    """Time the FP64 direct-sum oracle on a row sample sized to about budget_s seconds."""
    from oracle import kernel as ok
    from synth import subsample_rows
    n = X.shape[0]
    calib = subsample_rows(n, 16, seed)
    t0 = time.perf_counter()
    ok.anova_matvec(X, W, sigma, v, rows=calib)
    t_row = (time.perf_counter() - t0) / len(calib)
    rows = int(max(16, min(max_rows, budget_s / max(t_row, 1e-9))))
    idx = subsample_rows(n, rows, seed + 1)
    t0 = time.perf_counter()
    ok.anova_matvec(X, W, sigma, v, rows=idx)
    t = time.perf_counter() - t0
    return rows / t, rows, t, ok.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.n
    X, W, vseed = workload(n)
    from synth import matvec_vectors
    v = matvec_vectors(n, 1, vseed)[:, 0]
    # size each step so that warm-up + timed steps take about two minutes (at most 4 s a step)
    rate0, rows0, _, cores = oracle_rows_per_s(X, W, args.sigma, v, 1.0, 20000, 7)
    per_step_s = min(4.0, 120.0 / max(1, args.steps + args.warmup))
    rows = int(max(16, min(20000, per_step_s * rate0)))
    from oracle import kernel as ok
    from synth import subsample_rows
    for i in range(args.warmup):
        ok.anova_matvec(X, W, args.sigma, v, rows=subsample_rows(n, rows, 100 + i))
    times = []
    for i in range(args.steps):
        idx = subsample_rows(n, rows, 1000 + i)
        t0 = time.perf_counter()
        ok.anova_matvec(X, W, args.sigma, v, rows=idx)
        times.append(time.perf_counter() - t0)
    tot = float(np.sum(times))
    value = rows * args.steps / tot
    sample = ("FP64 direct sum of %d sampled output rows over all %d points and 3 windows per step "
              "(a full matvec is n rows; pts/s = rows computed per second)" % (rows, n))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(n, args.sigma, 1), "oracle": "direct summation"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def profile_traffic(kernel_key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None when
    the summary is missing or was taken on a different kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "matvec_n1e6_fp32_traffic.txt")
    try:
        with open(path) as f:
            rec = json.load(f)
        entry = rec[kernel_key]
        src = open(os.path.join(ROOT, entry["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != entry["source_sha256_16"]:
            return None
        return float(entry["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2312_00538_gb300 as ab
    from synth import matvec_vectors

    n, nrhs, sigma = args.n, args.nrhs, args.sigma
    X, W, vseed = workload(n, seed_offset=rank)    # independent problem per rank (weak scaling)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tune_report = None
    if args.tune:
        plan, tune_report = ab.anova_nfft_plan_tuned(X, W, sigma, N=32, m=4, flags=ab.ANOVA_FP32, nrhs=nrhs,
                                                     reps=5, stream=stream)
    else:
        plan = ab.anova_nfft_plan(X, W, sigma, N=32, m=4, flags=ab.ANOVA_FP32, stream=stream)
    torch.cuda.synchronize()
    plan_ms = 1000 * (time.perf_counter() - t0)
    V = matvec_vectors(n, nrhs, vseed)
    v = torch.tensor(np.ascontiguousarray(V.T), dtype=torch.float32, device="cuda")
    if nrhs == 1:
        v = v.reshape(-1)
    Kv = torch.empty_like(v)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        ab.anova_matvec(plan, v, Kv, nrhs)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ab.anova_plan_set_timing(plan, False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for s, e in ev:
        flush.zero_()
        s.record(stream)
        step()
        e.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = float(sum(s.elapsed_time(e) for s, e in ev))
    _, launches = ab.anova_plan_stage_times(plan)
    kv_timed = Kv.detach().cpu().numpy().astype(np.float64).reshape(nrhs, n).T   # result of the last timed step
    # same steps again with per-stage events, for the roofline of the dominant kernel
    ab.anova_plan_set_timing(plan, True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    stage_ms, _ = ab.anova_plan_stage_times(plan)
    ab.anova_plan_set_timing(plan, False)
    clocks = sampler.stop()

    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * n * nrhs / (ms_per_step / 1000.0)

    # ---------------------------------------------------------------- e2e through host buffers
    e2e = None
    if not args.no_e2e:
        vh = torch.empty((nrhs, n), dtype=torch.float32, pin_memory=True)
        vh.copy_(torch.from_numpy(np.ascontiguousarray(V.T).astype(np.float32)))
        kh = torch.empty((nrhs, n), dtype=torch.float32, pin_memory=True)
        for _ in range(2):
            ab.anova_matvec_host(plan, vh, kh, nrhs)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ab.anova_matvec_host(plan, vh, kh, nrhs)
        t_e2e = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        e2e = {"value": world * n * nrhs * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 4 * n * nrhs, "d2h_bytes_per_step": 4 * n * nrhs}

    # ---------------------------------------------------------------- roofline
    peaks, peak_kind = load_peaks()
    P = W.shape[0]
    m = 4
    fma_per_pt = P * (2 * m) ** 3 * nrhs               # multiply-adds per point, one of spread/interp
    dominant = "spread" if stage_ms["spread"] >= stage_ms["interp"] else "interp"
    dom_ms = stage_ms[dominant] / args.steps
    flops = 2.0 * fma_per_pt * n
    fp32_peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops / (dom_ms / 1000.0) / 1e12
    # the committed DRAM counters are for one right-hand side
    traffic = (profile_traffic("k_spread_f32_3d_m4" if dominant == "spread" else "k_interp_f32_3d_m4")
               if nrhs == 1 else None)
    fp32_measured = ab.anova_measure_fp32_peak()
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak_tflops, "traffic": traffic,
                "kernel": "k_%s (FP32, 3-D windows, m=4)" % dominant,
                "peak_source": "derived: %d SMs x %d FP32 FMA/clk x 2 x %.0f MHz" % (
                    SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ),
                "peak_measured": fp32_measured, "frac_of_measured": achieved / fp32_measured,
                "peak_measured_source": "anova_measure_fp32_peak in this run: independent fma.rn.f32x2 "
                                        "chains on every SM, best of 5"}
    alg_bytes = n * (P * 2 * 4 * 3 + 4 * nrhs + 4 * nrhs)   # coords read twice, v read, Kv written
    hbm_gbs = alg_bytes / (ms_per_step / 1000.0) / 1e9
    hbm = {"algorithmic_bytes_per_step": alg_bytes, "achieved_gbs": hbm_gbs,
           "peak_gbs": peaks["hbm_gbs"], "frac": hbm_gbs / peaks["hbm_gbs"],
           "peak_kind": peak_kind}

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's direct FP64 sum on the fixed 5,000-row sample of the workload: timed as the
        # CPU baseline (all host cores, then one core on a smaller sample) and used to state the
        # error of the result the timed steps produced
        from oracle import kernel as ok
        from synth import SEED_BASE, subsample_rows
        sample_seed = SEED_BASE + 2 + 200 + rank
        idx = subsample_rows(n, 5000, sample_seed)
        t0 = time.perf_counter()
        ref = ok.anova_matvec(X, W, sigma, V.astype(np.float64), rows=idx)
        t_all = time.perf_counter() - t0
        cores = ok.num_threads()
        ok.set_num_threads(1)
        try:
            rows1 = min(len(idx), max(16, int(4.0 * len(idx) / max(t_all * cores, 1e-9))))
            t0 = time.perf_counter()
            ok.anova_matvec(X, W, sigma, V[:, :1].astype(np.float64), rows=idx[:rows1])
            t_one = time.perf_counter() - t0
        finally:
            ok.set_num_threads(cores)
        ref = ref.reshape(len(idx), nrhs)
        errs = [float(np.linalg.norm(kv_timed[idx, j] - ref[:, j]) / np.linalg.norm(ref[:, j]))
                for j in range(nrhs)]
        accuracy = {"rel_l2": max(errs), "rel_l2_per_rhs": errs if nrhs > 1 else None,
                    "bar": 1e-4, "rows": int(len(idx)),
                    "against": "FP64 direct sum (oracle) of 5,000 fixed sampled rows (seed %d) over all "
                               "%d points, on the Kv of the last timed step" % (sample_seed, n)}
        cpu = {"value": len(idx) / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 direct sum of %d sampled output rows over all %d points and %d right-hand "
                         "side(s) (%.1f s); pts/s = output rows per second" % (len(idx), n, nrhs, t_all),
               "one_core": {"value": rows1 / t_one, "unit": UNIT, "cores": 1,
                            "sample": "%d of the same rows, 1 right-hand side, one thread (%.1f s)"
                                      % (rows1, t_one)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(n, sigma, nrhs), "global_batch": world * n,
                       "parallelism": "replicas (one independent problem per GPU)" if world > 1 else "single GPU",
                       "l2": "flushed between steps (512 MiB write)", "plan_ms": plan_ms,
                       "plan": ("tuned: %s" % json.dumps(tune_report)) if tune_report else "default settings"},
            "gpu_launches": int(launches),
            "stage_ms_per_step": {k: v2 / args.steps for k, v2 in stage_ms.items()},
            "roofline": roofline,
            "hbm_roofline": hbm,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_shard(args):
    """One workload-2 problem split by rows over the ranks (strong scaling): each rank spreads its
    points into every window's grid (anova_matvec_grids), one all-reduce sums the grids (NCCL;
    nothing to sum at one rank), and each rank finishes the product for its own rows
    (anova_matvec_from_grids: full-grid FFT passes, interpolation, window sum). A step is one such
    matvec of the whole problem; value = n / (max over ranks of the step time)."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2312_00538_gb300 as ab
    from synth import matvec_vectors
    n, sigma = args.n, args.sigma
    X, W, vseed = workload(n)                      # the same problem on every rank
    b0, b1 = rank * n // world, (rank + 1) * n // world
    stream = torch.cuda.current_stream()
    plan = ab.anova_nfft_plan(X[b0:b1], W, sigma, N=32, m=4, flags=ab.ANOVA_FP32, stream=stream)
    v_all = matvec_vectors(n, 1, vseed)[:, 0]
    v = torch.tensor(v_all[b0:b1], dtype=torch.float32, device="cuda")
    kv = torch.empty_like(v)
    gt = ab.anova_plan_grid_size(plan)
    grids = torch.empty(gt, dtype=torch.float32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        ab.anova_matvec_grids(plan, v, grids, 1)
        if world > 1:
            dist.all_reduce(grids)
        ab.anova_matvec_from_grids(plan, grids, kv, 1)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = float(sum(a.elapsed_time(b) for a, b in ev)) / args.steps
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # the rows of this rank against the fused one-plan matvec of the whole problem (one rank) or
    # the oracle's direct sum on sampled rows of this rank (several ranks)
    from oracle import kernel as ok
    from synth import subsample_rows
    idx = subsample_rows(b1 - b0, 500, 11 + rank)
    ref = ok.anova_matvec(X, W, sigma, v_all, rows=b0 + idx)
    got = kv.cpu().numpy().astype(np.float64)[idx]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    if world > 1:
        t = torch.tensor([err], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        err = float(t.item())
    if rank == 0:
        print(json.dumps({
            "metric": METRIC + " (one problem row-sharded over the GPUs)", "value": n / (ms / 1000.0), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(n, sigma, 1), "parallelism": "rows split over %d GPU(s), one "
                       "all-reduce of the %d-value grids per matvec" % (world, gt),
                       "l2": "flushed between steps (512 MiB write)"},
            "accuracy": {"rel_l2": err, "bar": 1e-4, "rows": 500 * world,
                         "against": "FP64 direct sum (oracle) of 500 sampled rows per rank"}}), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_ipm_batch(args):
    """Independent SVM solves of workload 4 (n log-uniform, (C, sigma) grid, rank 100): the plain
    path solves them one after another, the batched path `concurrency` at a time on separate
    streams. Solves/s and the per-solve latency distribution of both; equal results asserted."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config4
    probs = config4(count=args.count, n_hi=args.n_max)
    o = ab.svm_opts_default()
    o.rank = 100
    if args.m_precise:
        o.m_precise = args.m_precise
    if args.m_refine >= 0:
        o.m_refine = args.m_refine
    o.max_iter = args.max_iter
    o.err_tol = args.err_tol
    o.krylov_tol = args.krylov_tol
    tol = 1e-6
    plist = [dict(X=p["X"], y=p["y"], C=p["C"], ell=p["sigma"], windows=p["windows"]) for p in probs]
    torch.cuda.synchronize()
    ab.svm_ipm_solve_batch(plist[:2], tol, opts=o, concurrency=1)      # warm-up
    res = {}
    for mode, conc in (("plain", 1), ("batched", args.concurrency)):
        t0 = time.perf_counter()
        out = ab.svm_ipm_solve_batch(plist, tol, opts=o, concurrency=conc)
        wall = time.perf_counter() - t0
        lat = np.array([r[2]["time_ms"] for r in out])
        if mode == "plain":
            per = [dict(n=int(p["X"].shape[0]), C=p["C"], sigma=p["sigma"], it=r[2]["iterations"],
                        krylov=r[2]["krylov_iterations"], fp64_krylov=r[2]["fp64_krylov_iterations"],
                        rank=r[2]["rank"], ms=round(r[2]["time_ms"], 1), conv=r[2]["converged"])
                   for p, r in zip(probs, out)]
            print(json.dumps({"per_problem_plain": per}), file=sys.stderr, flush=True)
        res[mode] = {"solves_per_s": len(plist) / wall, "wall_s": wall,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "converged": int(sum(r[2]["converged"] for r in out)),
                     "alphas": [r[0] for r in out]}
    same = all(np.array_equal(a, b) for a, b in zip(res["plain"].pop("alphas"), res["batched"].pop("alphas")))
    line = {"metric": "IPM solves/s (workload 4, batched vs plain)", "value": res["batched"]["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "%d SVM problems, n log-uniform [5e3, %d], d=9, C x sigma grid, rank 100, "
                                   "gap 1e-6" % (args.count, args.n_max), "concurrency": args.concurrency,
                       "err_tol": args.err_tol, "krylov_tol": args.krylov_tol, "max_iter": args.max_iter,
                       "m_precise": o.m_precise, "m_refine": o.m_refine},
            "plain": res["plain"], "batched": res["batched"], "results_identical": bool(same),
            "speedup": res["batched"]["solves_per_s"] / res["plain"]["solves_per_s"]}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving loop over workload-4 problems: requests arrive as a seeded Poisson stream at
    `rate` per second and are admitted by the native server (free slot + device-memory budget).
    Reports throughput and the latency (arrival to completion) distribution."""
    import threading
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config4
    probs = config4(count=args.count, n_hi=args.n_max)
    o = ab.svm_opts_default()
    o.rank = 100
    if args.m_precise:
        o.m_precise = args.m_precise
    if args.m_refine >= 0:
        o.m_refine = args.m_refine
    o.max_iter = args.max_iter
    tol = 1e-6
    torch.cuda.synchronize()
    ab.svm_ipm_solve_batch([dict(X=p["X"], y=p["y"], C=p["C"], ell=p["sigma"], windows=p["windows"])
                            for p in probs[:2]], tol, opts=o, concurrency=1)      # warm-up
    gaps = np.random.default_rng(20231201).exponential(1.0 / args.rate, size=len(probs))
    srv = ab.SvmServer(tol, opts=o, slots=args.concurrency,
                       hbm_budget_bytes=int(args.budget_gib * (1 << 30)))
    tickets = []

    def producer():
        t_next = time.perf_counter()
        for p, g in zip(probs, gaps):
            t_next += g
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(p["X"], p["y"], p["C"], ell=p["sigma"], windows=p["windows"]))

    t0 = time.perf_counter()
    th = threading.Thread(target=producer)
    th.start()
    th.join()
    srv.drain()
    wall = time.perf_counter() - t0
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.destroy()
    line = {"metric": "SVM serving: solves/s at Poisson arrivals (workload 4)",
            "value": len(probs) / wall, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "%d SVM problems, n log-uniform [5e3, %d], d=9, C x sigma grid, rank 100, "
                                   "gap 1e-6" % (args.count, args.n_max),
                       "arrival_rate_per_s": args.rate, "slots": args.concurrency,
                       "budget_gib": args.budget_gib},
            "wall_s": wall, "p50_latency_ms": st["p50_latency_ms"], "p99_latency_ms": st["p99_latency_ms"],
            "mean_latency_ms": st["mean_latency_ms"],
            "peak_reserved_gib": st["peak_reserved_bytes"] / (1 << 30),
            "converged": int(sum(r[2]["converged"] for r in outs))}
    print(json.dumps(line), flush=True)
    return 0


def run_serve5(args):
    """Workload 5: Poisson streams of SVM solve requests (n log-uniform in [1e4, n_max], d in
    {6, 9, 12, 15, 18}, (C, sigma) from the workload-4 grid) at each rate, served by the native
    server (slots, 180 GiB budget, backfill) and by the plain one-at-a-time path (the same server
    with one slot, i.e. svm_ipm_solve on each request in arrival order), on the same arrival
    stream. Per rate: solves/s (requests / (last completion - first arrival)) and the latency
    (arrival to completion) distribution of both."""
    import threading
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config5
    o = ab.svm_opts_default()
    o.rank = 100
    if args.m_precise:
        o.m_precise = args.m_precise
    if args.m_refine >= 0:
        o.m_refine = args.m_refine
    o.max_iter = args.max_iter
    o.err_tol = args.err_tol
    o.krylov_tol = args.krylov_tol
    tol = 1e-6
    rates = [float(x) for x in args.rates.split(",")]
    warm = config5(2, 1.0, seed=77, n_hi=20000)
    ab.svm_ipm_solve_batch([dict(X=p["X"], y=p["y"], C=p["C"], ell=p["sigma"], windows=p["windows"]) for p in warm],
                           tol, opts=o, concurrency=1)
    rows = []
    for ri, rate in enumerate(rates):
        reqs = config5(args.count, rate, seed=9000 + ri, n_hi=args.n_max)
        row = {"rate_per_s": rate, "requests": len(reqs),
               "n_mean": float(np.mean([r["X"].shape[0] for r in reqs]))}
        results = {}
        for mode, slots in (("served", args.concurrency), ("sequential", 1)):
            srv = ab.SvmServer(tol, opts=o, slots=slots, hbm_budget_bytes=int(args.budget_gib * (1 << 30)))
            tickets = []

            def producer():
                t0p = time.perf_counter()
                for r in reqs:
                    dt = t0p + r["arrival"] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    tickets.append(srv.submit(r["X"], r["y"], r["C"], ell=r["sigma"], windows=r["windows"]))

            t0 = time.perf_counter()
            th = threading.Thread(target=producer)
            th.start()
            th.join()
            srv.drain()
            wall = time.perf_counter() - t0
            outs = [srv.wait(t) for t in tickets]
            st = srv.stats()
            srv.destroy()
            results[mode] = [o_[0] for o_ in outs]
            row[mode] = {"solves_per_s": len(reqs) / (wall - reqs[0]["arrival"]), "wall_s": wall,
                         "p50_latency_ms": st["p50_latency_ms"], "p99_latency_ms": st["p99_latency_ms"],
                         "mean_latency_ms": st["mean_latency_ms"], "backfilled": st["backfilled"],
                         "peak_reserved_gib": st["peak_reserved_bytes"] / (1 << 30),
                         "converged": int(sum(o_[2]["converged"] for o_ in outs))}
        row["results_identical"] = bool(all(np.array_equal(a, b) for a, b in
                                            zip(results["served"], results["sequential"])))
        row["speedup"] = row["served"]["solves_per_s"] / row["sequential"]["solves_per_s"]
        print(json.dumps(row), file=sys.stderr, flush=True)
        rows.append(row)
    line = {"metric": "SVM serving on workload 5: solves/s and p50/p99 latency vs the plain sequential path",
            "value": float(np.mean([r["served"]["solves_per_s"] for r in rows])), "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "%d requests per rate, n log-uniform [1e4, %d], d in {6,9,12,15,18}, "
                                   "(C, sigma) grid, rank 100, gap 1e-6" % (args.count, args.n_max),
                       "slots": args.concurrency, "budget_gib": args.budget_gib, "err_tol": args.err_tol,
                       "krylov_tol": args.krylov_tol, "max_iter": args.max_iter, "m_precise": o.m_precise,
                       "m_refine": o.m_refine},
            "per_rate": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_precond_study(args):
    """Synthetic analogue of the paper's preconditioner comparison (Sec. 6, the setup-time and
    Krylov-iteration figures): workload-3-like data (8 Gaussian + 4 binary features, tanh teacher,
    5 % flips) at several training sizes; for each low-rank factor (greedy and randomly pivoted
    Cholesky, Nystrom, per-window stacked greedy factors) and rank, the factor's setup time on the FP64 plan and the mean number of
    GMRES iterations per IPM step (the paper's solver), plus the MINRES count for comparison.
    sigma = 0.5 and err_tol = 0, so that every factor reaches the rank asked for."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config3
    all_kinds = {"cholesky_greedy": ab.PCHOL_GREEDY, "cholesky_rp": ab.PCHOL_RANDOM, "nystrom": ab.NYSTROM,
                 "cholesky_per_window": ab.PCHOL_PER_WINDOW, "nystrom_random": ab.NYSTROM_RANDOM}
    kinds = {k: all_kinds[k] for k in args.factors.split(",")}
    rows = []
    for n in (int(v) for v in args.sizes.split(",")):
        cfg = config3(n=n)
        X, y, W = cfg["X"], cfg["y"], cfg["windows"]
        p64 = ab.anova_nfft_plan(X, W, 0.5, N=64, m=6, flags=ab.ANOVA_FP64)
        for rank in (50, 100, 200, 400):
            for name, kind in kinds.items():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lr = ab.lowrank_precond_build(p64, kind, rank, 0.0, seed=7)
                torch.cuda.synchronize()
                setup_ms = 1000 * (time.perf_counter() - t0)
                got_rank, _ = ab.lowrank_info(lr)
                lr.destroy()
                row = {"n_train": n, "rank": rank, "factor": name, "rank_reached": got_rank,
                       "setup_ms": round(setup_ms, 2)}
                for krylov, label in ((ab.SVM_KRYLOV_GMRES, "gmres"), (ab.SVM_KRYLOV_MINRES, "minres")):
                    o = ab.svm_opts_default()
                    o.rank = rank
                    o.precond = kind
                    o.seed = 7
                    o.err_tol = 0.0
                    o.ell = 0.5
                    o.krylov = krylov
                    o.max_iter = 100
                    o.krylov_tol = 1e-6
                    t0 = time.perf_counter()
                    _, _, st, status = ab.svm_ipm_solve(X, y, 10.0, 1e-6, opts=o, windows=W)
                    row[label] = {"ipm_iterations": st["iterations"],
                                  "krylov_per_ipm_step": round(st["krylov_iterations"] / max(1, st["iterations"]), 2),
                                  "solve_s": round(time.perf_counter() - t0, 3), "converged": st["converged"],
                                  "rel_gap": st["rel_gap"]}
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
        p64.destroy()
    print(json.dumps({"metric": "preconditioner study (setup ms, Krylov iterations per IPM step)",
                      "data": "synthetic (workload 3 generator), C = 10, sigma = 0.5, err_tol 0, gap 1e-6",
                      "rows": rows}), flush=True)
    return 0


def run_predict(args):
    """Prediction (targets distinct from the sources, Sec. 6) on the matvec workload's points:
    n sources with weights w, n fresh targets from the same generator. Times, with CUDA events and
    inputs resident, (a) anova_cross_matvec per call, (b) anova_model_create once, and (c)
    anova_model_eval per call; the value is target points per second of (c)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import matvec_vectors
    n = args.n
    Xs, W, vseed = workload(n)
    Xt = workload(n, seed_offset=1)[0]
    w = torch.tensor(matvec_vectors(n, 1, vseed)[:, 0], dtype=torch.float32, device="cuda")
    src = ab.anova_nfft_plan(Xs, W, args.sigma, N=32, m=4)
    tgt = ab.anova_nfft_plan(Xt, W, args.sigma, N=32, m=4)
    f = torch.empty(n, dtype=torch.float32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn, steps):
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    for _ in range(max(3, args.warmup)):
        ab.anova_cross_matvec(src, tgt, w, f)
    cross_ms = timed(lambda: ab.anova_cross_matvec(src, tgt, w, f), args.steps)
    f_cross = f.clone()
    models = []
    create_ms = timed(lambda: models.append(ab.anova_model_create(src, w)), 3)
    model = models[-1]
    for _ in range(max(3, args.warmup)):
        ab.anova_model_eval(model, tgt, f)
    eval_ms = timed(lambda: ab.anova_model_eval(model, tgt, f), args.steps)
    rel = float(torch.linalg.vector_norm((f - f_cross).double()) / torch.linalg.vector_norm(f_cross.double()))
    print(json.dumps({
        "metric": "ANOVA-NFFT prediction (targets != sources) target points/s", "value": n / (eval_ms / 1e3),
        "unit": "target_points/s", "ms_per_step": eval_ms, "steps": args.steps, "higher_is_better": True,
        "data": "synthetic", "dtype": "f32",
        "config": {"workload": "prediction n_source=%d n_target=%d d=9 windows=3x3D sigma=%g N=32 m=4"
                               % (n, n, args.sigma), "l2": "flushed between steps (512 MiB write)"},
        "cross_matvec_ms": cross_ms, "model_create_ms": create_ms, "model_eval_ms": eval_ms,
        "model_vs_cross_rel_l2": rel}), flush=True)
    return 0


def run_matvec_batch(args):
    """Matvecs of `count` independent problems of uneven size (workload-4 sizes and sigma grid,
    three 3-D windows, FP32): one after another on one stream, against one CUDA graph with a
    branch per problem (anova_matvec_batch_*). Inputs resident, L2 flushed between steps; the
    value is points of all problems per second through the graph."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config4
    probs = config4(count=args.count, n_hi=args.n_max)
    stream = torch.cuda.current_stream()
    plans, vs, kvs = [], [], []
    for q in probs:
        p = ab.anova_nfft_plan(q["X"], q["windows"], q["sigma"], N=32, m=4, stream=stream)
        v = torch.randn(q["X"].shape[0], device="cuda")
        plans.append(p), vs.append(v), kvs.append(torch.empty_like(v))
    total = sum(q["X"].shape[0] for q in probs)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    batch = ab.anova_matvec_batch_create(plans, vs, kvs, stream=stream)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / args.steps

    def sequential():
        for p, v, k in zip(plans, vs, kvs):
            ab.anova_matvec(p, v, k, 1)

    seq_ms = timed(sequential)
    graph_ms = timed(batch.run)
    print(json.dumps({
        "metric": "ANOVA-NFFT matvecs of independent problems, points/s", "value": total / (graph_ms / 1e3),
        "unit": "pts/s", "ms_per_step": graph_ms, "steps": args.steps, "higher_is_better": True,
        "data": "synthetic", "dtype": "f32",
        "config": {"workload": "%d problems, n log-uniform [5e3, %d] (total %d points), d=9, windows=3x3D, "
                               "sigma grid, N=32, m=4" % (len(probs), args.n_max, total),
                   "l2": "flushed between steps (512 MiB write)"},
        "sequential_ms": seq_ms, "graph_ms": graph_ms, "speedup": seq_ms / graph_ms}), flush=True)
    return 0


def run_matvec64(args):
    """The FP64 plan's matvec (the precise path: N = 64, m = 6 unless --m-precise) on workload 3's
    points (n = 1e5, four 3-D windows), one RHS, inputs resident, L2 flushed between steps; CUDA
    events on the plan's stream, per-stage times from a second timed pass."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config3, matvec_vectors, SEED_BASE
    cfg = config3()
    X, W = cfg["X"], cfg["windows"]
    n = X.shape[0]
    m = args.m_precise or 6
    plan = ab.anova_nfft_plan(X, W, 1.0, N=64, m=m, flags=ab.ANOVA_FP64)
    v = torch.tensor(matvec_vectors(n, 1, SEED_BASE + 64)[:, 0], dtype=torch.float64, device="cuda")
    kv = torch.empty_like(v)
    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
    for _ in range(max(1, args.warmup)):
        flush.zero_()
        ab.anova_matvec(plan, v, kv, 1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    st = torch.cuda.current_stream()
    for a, b in ev:
        flush.zero_()
        a.record(st)
        ab.anova_matvec(plan, v, kv, 1)
        b.record(st)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ab.anova_plan_set_timing(plan, True)
    for _ in range(args.steps):
        flush.zero_()
        ab.anova_matvec(plan, v, kv, 1)
    stages, _ = ab.anova_plan_stage_times(plan)
    line = {"metric": "ANOVA-NFFT FP64 matvec pts/s (workload 3 points)", "value": n / (ms / 1e3), "unit": "pts/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64 (spread and interpolation sums in FP32 pairs)", "data": "synthetic",
            "config": {"workload": "FP64 plan, n=%d, d=12, four 3-D windows, N=64, m=%d, 1 RHS" % (n, m),
                       "l2": "flushed between steps"},
            "stage_ms_per_step": {k: t / args.steps for k, t in stages.items()}}
    print(json.dumps(line), flush=True)
    return 0


def run_woodbury(args):
    """The Woodbury core M = I + L^T Theta^-1 L (Sec. 5) at workload-3 size (n = 1e5, rank 200):
    lowrank_precond_set_theta on the FP64 pipe against the exact-slice tensor-core path, Theta^-1
    spread over 1e-2 .. 1e8. Each call is timed with the host clock around the synchronous call
    (both include the Cholesky factor, its inverse and the Schur value)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    from synth import config3
    cfg = config3()
    n, rank = cfg["X"].shape[0], args.rank
    plan = ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0, N=64, m=6, flags=ab.ANOVA_FP64)
    t0 = time.perf_counter()
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, rank, 0.0)
    torch.cuda.synchronize()
    build_ms = 1000 * (time.perf_counter() - t0)
    rng = np.random.default_rng(5)
    theta = torch.tensor(1.0 / 10.0 ** rng.uniform(-2, 8, n), dtype=torch.float64, device="cuda")
    y = torch.tensor(cfg["y"], dtype=torch.float64, device="cuda")
    res, cores = {}, {}
    for name, path in (("fp64_pipe", ab.LOWRANK_CORE_SIMT), ("tensor_cores", ab.LOWRANK_CORE_TENSOR)):
        ab.lowrank_set_core_path(lr, path)
        for _ in range(max(3, args.warmup)):
            ab.lowrank_precond_set_theta(lr, theta, y)
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ab.lowrank_precond_set_theta(lr, theta, y)
            ts.append(1000 * (time.perf_counter() - t0))
        M = torch.empty((rank, rank), dtype=torch.float64, device="cuda")
        ab.lowrank_core(lr, M)
        cores[name] = M.cpu().numpy()
        res[name] = {"set_theta_ms": float(np.median(ts)), "min_ms": float(np.min(ts))}
    diff = float(np.linalg.norm(cores["tensor_cores"] - cores["fp64_pipe"]) / np.linalg.norm(cores["fp64_pipe"]))
    line = {"metric": "Woodbury core set_theta ms (workload 3: n=1e5, rank %d)" % rank,
            "value": res["tensor_cores"]["set_theta_ms"], "unit": "ms", "n_gpus": 1, "higher_is_better": False,
            "dtype": "bf16 slices -> FP64", "data": "synthetic",
            "config": {"workload": "Woodbury core M = I + L^T Theta^-1 L, n=%d, rank %d, Theta^-1 in [1e-2, 1e8]"
                                   % (n, rank), "build_ms": build_ms},
            "fp64_pipe": res["fp64_pipe"], "tensor_cores": res["tensor_cores"],
            "speedup": res["fp64_pipe"]["set_theta_ms"] / res["tensor_cores"]["set_theta_ms"],
            "rel_frobenius_difference": diff}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ipm_batch":
        return run_ipm_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "precond_study":
        return run_precond_study(args)
    if args.workload == "predict":
        return run_predict(args)
    if args.workload == "matvec_batch":
        return run_matvec_batch(args)
    if args.workload == "woodbury":
        return run_woodbury(args)
    if args.workload == "matvec64":
        return run_matvec64(args)
    if args.workload == "serve5":
        return run_serve5(args)
    if args.shard:
        return run_shard(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
