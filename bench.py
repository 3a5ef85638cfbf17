"""Benchmark of GB300 k-means++ D^2 seeding (one JSON line on rank 0).

A step is one whole seeding (all K passes and K-1 draws) of the named
workload, through the library's C ABI, with the points already resident in
HBM.  L2 is flushed (a 512 MiB buffer is written) between timed steps, and
each step is timed with CUDA events on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--dtype f32|bf16|fp8] [--forms bf16,fp8|none]
                  [--shard replicas|points] [--impl kpp|reference]

Workloads: the seeding workloads (default gmm-N2e7-d128-K2048-t3, the
largest single-GPU one: 2e7 x 128, K = 2048; an FP32 run also times the same
data stored as BF16 and FP8, --forms), ``batch-512`` (kpp_seed_batched over
512 uneven problems), ``lloyd-<seeding workload>`` (one Lloyd iteration from
that workload's k-means++ seeds; the assignment is also timed alone for its
tensor roofline) and ``kmpar-<seeding workload>`` (one whole k-means||
initialisation, ell = --ell-mult x K, --rounds rounds; its nearest-candidate
search timed alone for the roofline).

Under torchrun (N > 1): for a single problem every rank seeds its own
replica of the workload (its own Philox stream: weak scaling), or, with
``--shard points``, the ranks split one problem by rows and exchange two
small messages per pass over NCCL (strong scaling); for the 512-problem
batch the problems are split between the ranks with no collective on the
data path (strong scaling).  Timing is barrier-bracketed and the max over
ranks is reported.

``--impl reference`` times the FP64 CPU oracle (the correctness reference,
not a GPU code; multi-threaded over the host cores for the seeding
workloads) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-means++ seeding ms & N·K·d/s; HBM GB/s vs peak; BF16/batched vs FP32"
UNIT = "N*K*d/s"
DEFAULT_WORKLOAD = "gmm-N2e7-d128-K2048-t3"
BATCH_WORKLOAD = "batch-512"
LLOYD_PREFIX = "lloyd-"  # e.g. lloyd-gmm-N1e7-d64-K1024: one Lloyd iteration from the seeds
KMPAR_PREFIX = "kmpar-"  # e.g. kmpar-gmm-N1e6-d32-K256: k-means|| (ell = 2K, 5 rounds)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "fp8"])
    ap.add_argument("--impl", default="kpp", choices=["kpp", "reference"])
    ap.add_argument("--form", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--smem-cache", type=int, default=0)
    ap.add_argument("--alternate", type=int, default=0)
    ap.add_argument("--l2-policy", type=int, default=0)
    ap.add_argument("--min-rows", type=int, default=0)
    ap.add_argument("--forms", default="bf16,fp8",
                    help="FP32 runs: precision forms of the same data timed beside it "
                         "(comma list, or 'none')")
    ap.add_argument("--form-steps", type=int, default=3,
                    help="timed steps of each precision form beside the FP32 run")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "points"],
                    help="N > 1 and one seeding workload: every rank seeds its own replica "
                         "(weak scaling), or one problem is split by rows over the ranks "
                         "(strong scaling)")
    ap.add_argument("--no-read-peaks", action="store_true",
                    help="skip the live pure-read bandwidth measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity-sample", action="store_true",
                    help="skip the sampled D^2 check of the timed seeding")
    ap.add_argument("--no-phi", action="store_true")
    ap.add_argument("--no-sequential", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (it runs, untimed, unless a knob is given)")
    ap.add_argument("--tune-passes", type=int, default=0)
    ap.add_argument("--phi-seeds", type=int, default=0,
                    help="precision forms: also compare mean phi over this many draw seeds")
    ap.add_argument("--n-points", type=int, default=0,
                    help="a smaller instance of the workload's recipe (profiling)")
    ap.add_argument("--k-seeds", type=int, default=0)
    ap.add_argument("--ell-mult", type=float, default=2.0, help="k-means||: ell = this x K")
    ap.add_argument("--rounds", type=int, default=5, help="k-means||: oversampling rounds")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# The sources each kernel is compiled from (device code and the host code
# that plans and launches it): an ncu figure stays valid while these are
# unchanged.
KERNEL_SOURCES = {
    "persistent": ["kpp_device.cuh", "kpp_pass.cuh", "kpp_persistent.cuh", "kpp_persistent.cu",
                   "kpp_persistent_f32.cu", "kpp_persistent_bf16.cu", "kpp_persistent_fp8.cu"],
    "streamed": ["kpp_device.cuh", "kpp_pass.cuh", "kpp_streamed.cu"],
    "batched": ["kpp_device.cuh", "kpp_pass.cuh", "kpp_persistent.cuh", "kpp_batched.cuh",
                "kpp_batched.cu", "kpp_batched_f32.cu", "kpp_batched_bf16.cu",
                "kpp_batched_fp8.cu"],
}


def kernel_source_hash(kind: str = "persistent"):
    """SHA-256 over one kernel's CUDA sources (to tell whether a committed ncu
    traffic figure still describes the kernel being run)."""
    import hashlib

    h = hashlib.sha256()
    files = [os.path.join(ROOT, "paper_1908_02136_gb300", "csrc", f) for f in KERNEL_SOURCES[kind]]
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def plan_signature(plan: dict) -> str:
    """The launch shape an ncu figure was taken with."""
    keys = ("form", "grid", "lanes_per_row", "d2_in_smem", "rows_per_cta", "cached_rows_per_cta")
    return " ".join(f"{k}={plan[k]}" for k in keys)


def _profile_fields(path: str, names) -> dict:
    try:
        txt = open(path).read()
    except OSError:
        return {}
    fields = {}
    for line in txt.splitlines():
        if ":" in line and line.split(":", 1)[0] in names:
            k, v = line.split(":", 1)
            fields[k] = v.strip()
    return fields


def profiled_traffic(kind: str, workload: str, dtype: str, plan: dict, passes: int = 1):
    """DRAM bytes per launch from the committed ncu summary of this kernel on
    this workload (its per-pass figure times the passes of one launch), or
    None if there is none, its launch shape differs or its sources changed
    since."""
    path = os.path.join(ROOT, "profiles", f"{kind}_kernel_{workload}_{dtype}.md")
    f = _profile_fields(path, ("traffic_bytes_per_pass", "traffic_bytes_per_launch",
                               "kernel_source_sha256", "plan_signature"))
    if f.get("kernel_source_sha256") != kernel_source_hash(kind):
        return None
    if f.get("plan_signature") != plan_signature(plan):
        return None
    try:
        if "traffic_bytes_per_pass" in f:
            return int(float(f["traffic_bytes_per_pass"]) * passes)
        return int(f["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def profiled_batch_traffic():
    """DRAM bytes of one step of the batch workload (all waves) from the
    committed ncu summary, or None if absent or the sources changed since."""
    path = os.path.join(ROOT, "profiles", f"batched_kernel_{BATCH_WORKLOAD}_f32.md")
    f = _profile_fields(path, ("traffic_bytes_per_step", "kernel_source_sha256"))
    if f.get("kernel_source_sha256") != kernel_source_hash("batched"):
        return None
    try:
        return int(f["traffic_bytes_per_step"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# GB300 HBM3e bandwidth as specified (the denominators above are measured).
NOMINAL_HBM_GBS = 8000.0


def cpu_info():
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return os.cpu_count(), model


def _reference_line(args, world, metric, value, ms, config, sample):
    cores, model = cpu_info()
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host_cores": cores, "cpu": model},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference_other(args, world):
    """The reference arm of the batch, Lloyd and k-means|| workloads: the
    oracle's routine for that step on a bounded sample, N*K*d per second."""
    import numpy as np

    import oracle
    from paper_1908_02136_gb300 import datagen

    steps = max(1, args.steps)
    if args.workload == BATCH_WORKLOAD:
        probs, budget = [], 0.0
        for pr in datagen.batch_table():
            if budget + pr.N * pr.K * pr.d > 2e9:
                continue
            probs.append(pr)
            budget += pr.N * pr.K * pr.d
        data = [(pr, datagen.batch_problem_points(pr)) for pr in probs]
        times = []
        for s_ in range(args.warmup + steps):
            t0 = time.perf_counter()
            for pr, x in data:
                oracle.seed(x, pr.K, 1, pr.p)
            if s_ >= args.warmup:
                times.append(time.perf_counter() - t0)
        dt = sum(times) / len(times)
        _reference_line(args, world, METRIC, budget / dt, 1e3 * dt,
                        {"workload": BATCH_WORKLOAD, "problems": len(probs)},
                        f"{len(probs)} of the 512 problems (N*K*d <= 2e9 in total), "
                        "one oracle seeding each per step (serial FP64)")
        return
    lloyd = args.workload.startswith(LLOYD_PREFIX)
    wl = datagen.WORKLOADS[args.workload[len(LLOYD_PREFIX if lloyd else KMPAR_PREFIX):]]
    N, d, K = wl.N, wl.d, wl.K
    if lloyd:
        n_s = int(max(K, min(N, 3e9 / (K * d))))
    else:
        ell, R = args.ell_mult * K, args.rounds
        n_s = int(min(N, max(4 * K, 3e9 / (ell * R * d))))
    x = datagen.gmm(n_s, d, wl.n_comp, wl.data_seed, wl.mean_box, wl.sigma, wl.weights,
                    wl.outlier_frac, wl.outlier_center)
    C = x[:K].astype(np.float64)
    times = []
    for s_ in range(args.warmup + steps):
        t0 = time.perf_counter()
        if lloyd:
            oracle.lloyd_step(x, C)
        else:
            oracle.kmeans_par(x, K, ell, R, wl.draw_seed, 0, cand_cap=n_s)
        if s_ >= args.warmup:
            times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    if lloyd:
        metric = "k-means Lloyd iteration N*K*d/s (after k-means++ seeding)"
        sample = (f"one Lloyd step of the first {n_s} of {N} points from {K} centres "
                  "(the sample's first points) per step (serial FP64)")
    else:
        metric = "k-means|| initialisation N*K*d/s (oversampling + weighted recluster)"
        sample = (f"k-means|| on {n_s} of {N} points (same K, ell, rounds) per step "
                  "(serial FP64)")
    _reference_line(args, world, metric, n_s * K * d / dt, 1e3 * dt,
                    {"workload": args.workload, "N": N, "d": d, "K": K, "sample_points": n_s},
                    sample)


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores
    (the multi-threaded seeding oracle for the seeding workloads)."""
    from paper_1908_02136_gb300 import datagen

    if rank != 0:
        return
    if (args.workload == BATCH_WORKLOAD or args.workload.startswith(LLOYD_PREFIX)
            or args.workload.startswith(KMPAR_PREFIX)):
        run_reference_other(args, world)
        return
    wl = datagen.WORKLOADS[args.workload]
    import oracle

    # the workload's recipe on at most 2*10^6 points (numpy draws the larger
    # workloads too slowly for a bench run)
    x = datagen.workload_points(wl) if wl.N <= 2_000_000 else datagen.gmm(
        min(wl.N, 2_000_000), wl.d, wl.n_comp, wl.data_seed, wl.mean_box, wl.sigma, wl.weights,
        wl.outlier_frac, wl.outlier_center)
    N = x.shape[0]
    cores, model = cpu_info()
    # passes per step sized so that warm-up and timed steps take about two minutes
    t0 = time.perf_counter()
    oracle.seed_mt(x, min(2, wl.K), wl.draw_seed, 0, threads=cores)
    per_pass = (time.perf_counter() - t0) / min(2, wl.K)
    budget = max(0.5, 120.0 / max(1, args.steps + args.warmup))
    K_s = int(max(1, min(wl.K, budget / max(per_pass, 1e-9))))
    for _ in range(args.warmup):
        oracle.seed_mt(x, K_s, wl.draw_seed, 0, threads=cores)
    times, threads = [], cores
    for s in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.seed_mt(x, K_s, wl.draw_seed, s, threads=cores)
        times.append(time.perf_counter() - t0)
        threads = r["threads"]
    ms = 1e3 * sum(times) / len(times)
    value = N * K_s * wl.d / (sum(times) / len(times))
    sample = (f"{N} of {wl.N} points x {wl.d} dims (the workload's recipe), {K_s} of {wl.K} "
              f"passes per step (multi-threaded FP64 oracle, {threads} threads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name, "N": N, "d": wl.d, "K": wl.K,
                                        "dtype": "f32", "passes_per_step": K_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "host_cores": cores, "cpu": model},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batch(args, rank, world, dev, pg, barrier):
    """The 512-problem batch: one kpp_seed_batched call per step, against the
    same problems seeded one kpp_seed call after another (the plain path).
    With N > 1 ranks the problems are split between the ranks (longest
    processing time first, no collective on the data path): strong scaling
    of the fixed 512-problem workload."""
    import ctypes

    import numpy as np
    import torch

    import paper_1908_02136_gb300 as kpp
    from paper_1908_02136_gb300 import datagen, multi

    full = datagen.batch_table()
    shards = multi.shard_problems([pr.N * pr.K * pr.d for pr in full], world)
    table = [full[i] for i in shards[rank]]
    xs = [torch.from_numpy(datagen.batch_problem_points(pr)).to(dev) for pr in table]
    Ks = [pr.K for pr in table]
    streams = [pr.p for pr in table]
    seeds = [1] * len(table)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    nkd_all = float(sum(pr.N * pr.K * pr.d for pr in full))
    alg_bytes_all = float(sum(pr.N * pr.K * pr.d * 4 for pr in full))
    alg_bytes = float(sum(pr.N * pr.K * pr.d * 4 for pr in table))
    n_waves = len({pr.d for pr in table})
    with torch.cuda.stream(stream):
        outs, ws = kpp.seed_batched(xs, Ks, seeds, streams, check=True)
        sh = ctypes.c_void_p(stream.cuda_stream)
        arr = (kpp.Problem * len(table))()
        for i, (x, K) in enumerate(zip(xs, Ks)):
            idx, d2, phi = outs[i]
            arr[i].points, arr[i].row_scales = x.data_ptr(), None
            arr[i].N, arr[i].d, arr[i].K = x.shape[0], x.shape[1], K
            arr[i].seed, arr[i].stream_id = 1, streams[i]
            arr[i].indices_out, arr[i].d2_out, arr[i].phi_out = (idx.data_ptr(), d2.data_ptr(),
                                                                 phi.data_ptr())

        def launch():
            st = kpp.kpp_seed_batched(arr, len(table), kpp.F32, ws.data_ptr(), ws.numel(), sh)
            if st != kpp.OK:
                raise kpp.KppError(st, "kpp_seed_batched")

        for _ in range(args.warmup):
            flush.fill_(1)
            launch()
        st = kpp.kpp_read_status(ws.data_ptr(), sh)
        if st != kpp.OK:
            raise kpp.KppError(st, "warmup")
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize(dev)
        barrier()
        sampler = ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
        sampler.start()
        time.sleep(0.3)
        for s_ in range(args.steps):
            flush.fill_(s_ & 0xFF)
            starts[s_].record(stream)
            launch()
            ends[s_].record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        barrier()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        # the plain path: one kpp_seed per problem, back to back
        seq_ms = None
        if not args.no_sequential:
            wss = [kpp.workspace_for(x.shape[0], x.shape[1], K, kpp.F32, dev)
                   for x, K in zip(xs, Ks)]
            o2 = [(torch.empty(K, dtype=torch.int64, device=dev),
                   torch.empty(x.shape[0], dtype=torch.float32, device=dev),
                   torch.empty(1, dtype=torch.float64, device=dev)) for x, K in zip(xs, Ks)]

            def seq():
                for i, (x, K) in enumerate(zip(xs, Ks)):
                    st = kpp.kpp_seed(x.data_ptr(), None, x.shape[0], x.shape[1], K, kpp.F32, 1,
                                      streams[i], None, 0, o2[i][0].data_ptr(),
                                      o2[i][1].data_ptr(), o2[i][2].data_ptr(), wss[i].data_ptr(),
                                      wss[i].numel(), sh)
                    if st != kpp.OK:
                        raise kpp.KppError(st, "kpp_seed")

            seq()
            torch.cuda.synchronize(dev)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(2)
            a_.record(stream)
            seq()
            b_.record(stream)
            torch.cuda.synchronize(dev)
            seq_ms = a_.elapsed_time(b_)
    total_ms = multi.max_over_ranks(sum(step_ms), pg, dev)
    if seq_ms is not None:
        seq_ms = multi.max_over_ranks(seq_ms, pg, dev)
    ms = total_ms / args.steps
    for (idx, d2, phi), pr in zip(outs, table):
        ih = idx.cpu().numpy()
        assert np.all((ih >= 0) & (ih < pr.N)) and len(set(ih.tolist())) == pr.K
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    # the slowest rank's own bytes over its own time would flatter; the
    # roofline is per GPU: this rank's bytes over the job's step time
    achieved = alg_bytes / (ms / 1e3) / 1e9
    traffic = profiled_batch_traffic() if world == 1 else None
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": nkd_all * args.steps / (total_ms / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "problems": len(full), "sum_NKd": nkd_all,
                       "problems_on_rank0": len(table), "form": "batched",
                       "parallelism": f"problems split over {world} ranks (LPT)",
                       "l2": "flushed between steps (512 MiB write)",
                       "plain_sequential_ms": seq_ms,
                       "batched_speedup_vs_plain": (seq_ms / ms) if seq_ms else None},
            "clocks": clocks, "e2e": None,
            # one cooperative launch per distinct d (wave) per step
            "gpu_launches": args.steps * n_waves,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "batched_kernel (all waves of one step)",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "algorithmic_bytes_all_ranks": alg_bytes_all},
            "cpu_baseline": None,
        }), flush=True)


def phi_over_seeds(kpp, x, pts, scales, code, K, seed0, stream_id, R, stream, dev):
    """Mean seeding cost over R draw seeds, precision form vs FP32: the form's
    seeds scored on the original FP32 points (replayed through the FP32 path)
    against FP32 seeding with the same draw seeds; means with 95 % intervals
    and the paired relative difference."""
    import torch

    form, fp32 = [], []
    with torch.cuda.stream(stream):
        for r in range(R):
            sd = seed0 + 1000 + r
            idx, _, _ = kpp.seed(pts, K, sd, stream_id, dtype=code, row_scales=scales, check=True)
            _, _, p_form = kpp.seed(x, K, sd, stream_id, forced=idx.clone(), check=True)
            _, _, p32 = kpp.seed(x, K, sd, stream_id, check=True)
            form.append(float(p_form.item()))
            fp32.append(float(p32.item()))
    torch.cuda.synchronize(dev)

    def summary(v):
        m = statistics.fmean(v)
        half = 1.96 * statistics.stdev(v) / math.sqrt(len(v))
        return {"mean": m, "ci95": half}

    rel = [(a - b) / b for a, b in zip(form, fp32)]
    sf, s32, sr = summary(form), summary(fp32), summary(rel)
    return {"seeds": R, "phi_form_on_fp32_points": sf, "phi_fp32": s32,
            "rel_diff_of_means": (sf["mean"] - s32["mean"]) / s32["mean"],
            "paired_rel_diff": sr,
            "means_agree_within_ci": abs(sf["mean"] - s32["mean"]) <= sf["ci95"] + s32["ci95"]}


def run_lloyd(args, rank, world, dev, pg, barrier):
    """One Lloyd iteration (assignment on the tensor cores + update) on a
    seeding workload's points, from that workload's k-means++ seeds: each
    step is kpp_lloyd_step from the same seeds; the assignment alone is also
    timed (kpp_lloyd_assign) for its tensor roofline."""
    import ctypes

    import numpy as np
    import torch

    import paper_1908_02136_gb300 as kpp
    from paper_1908_02136_gb300 import datagen, multi

    wl = datagen.WORKLOADS[args.workload[len(LLOYD_PREFIX):]]
    if args.n_points or args.k_seeds:  # a smaller instance of the same recipe (profiling)
        import dataclasses

        n_, k_ = args.n_points or wl.N, args.k_seeds or wl.K
        wl = dataclasses.replace(wl, N=n_, K=k_, name=f"{wl.name}@N{n_}K{k_}")
    x = datagen.workload_points(wl, dev)
    N, d, K = wl.N, wl.d, wl.K
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        idx, _, _ = kpp.seed(x, K, wl.draw_seed, multi.replica_stream(0, rank))
        C = x[idx].contiguous()
        ll = kpp.Lloyd(x, K)
        labels = torch.empty(N, dtype=torch.int32, device=dev)
        d2 = torch.empty(N, dtype=torch.float32, device=dev)
        C2 = torch.empty_like(C)
        counts = torch.empty(K, dtype=torch.int64, device=dev)
        phi = torch.empty(1, dtype=torch.float64, device=dev)
        sh = ctypes.c_void_p(stream.cuda_stream)

        def step():
            st = kpp.kpp_lloyd_step(x.data_ptr(), N, d, C.data_ptr(), K, labels.data_ptr(),
                                    d2.data_ptr(), C2.data_ptr(), counts.data_ptr(),
                                    phi.data_ptr(), ll.ws.data_ptr(), ll.ws.numel(), sh)
            if st != kpp.OK:
                raise kpp.KppError(st, "kpp_lloyd_step")

        def assign():
            st = kpp.kpp_lloyd_assign(C.data_ptr(), N, d, K, labels.data_ptr(), ll.ws.data_ptr(),
                                      ll.ws.numel(), sh)
            if st != kpp.OK:
                raise kpp.KppError(st, "kpp_lloyd_assign")

        def timed(fn, steps):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            for a_, b_ in ev:
                flush.fill_(3)
                a_.record(stream)
                fn()
                b_.record(stream)
            torch.cuda.synchronize(dev)
            return [a_.elapsed_time(b_) for a_, b_ in ev]

        for _ in range(args.warmup):
            flush.fill_(1)
            step()
        st = kpp.kpp_read_status(ll.ws.data_ptr(), sh)
        if st != kpp.OK:
            raise kpp.KppError(st, "warmup")
        torch.cuda.synchronize(dev)
        barrier()
        sampler = ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
        sampler.start()
        time.sleep(0.3)
        step_ms = timed(step, args.steps)
        assign_ms = timed(assign, args.steps)
        clocks = sampler.stop()
        barrier()
        st = kpp.kpp_read_status(ll.ws.data_ptr(), sh)
        if st != kpp.OK:
            raise kpp.KppError(st, "timed steps")
    total_ms = multi.max_over_ranks(sum(step_ms), pg, dev)
    ms = total_ms / args.steps
    a_ms = statistics.fmean(assign_ms)
    nkd = float(N) * K * d
    dp = 64 if d <= 64 else 128
    kpad = (K + 127) // 128 * 128
    tensor_flops = 3 * 2.0 * N * kpad * dp  # hi.hi + hi.lo + lo.hi, padded tiles
    peaks = measured_peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    achieved = tensor_flops / (a_ms / 1e3) / 1e12
    # bounded CPU sample: the oracle's Lloyd step on the first points
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        n_s = max(1, min(N, int(3e9 / (K * d))))
        xs = x[:n_s].cpu().numpy()
        t0 = time.perf_counter()
        oracle.lloyd_step(xs, C.double().cpu().numpy())
        dt = time.perf_counter() - t0
        cores, model = cpu_info()
        cpu = {"value": n_s * K * d / dt, "unit": "N*K*d/s", "cores": 1, "kind": "oracle",
               "sample": f"{n_s} of {N} points, all {K} centres, one Lloyd step (serial FP64)",
               "host_cores": cores, "cpu": model}
    if rank == 0:
        print(json.dumps({
            "metric": "k-means Lloyd iteration N*K*d/s (after k-means++ seeding)",
            "value": nkd * world * args.steps / (total_ms / 1e3), "unit": "N*K*d/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "d": d, "K": K,
                       "assignment": "tcgen05 BF16 split (hi.hi + hi.lo + lo.hi), FP32 accumulate, "
                                     "CTA pairs (cta_group::2, 256 x 256 tiles)",
                       "assign_ms": a_ms, "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (512 MiB write)",
                       "phi": float(phi.item())},
            "clocks": clocks, "e2e": None, "gpu_launches": 5 * args.steps,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "lloyd_assign_pair_kernel",
                         "tensor_flops_per_launch": tensor_flops,
                         "algorithmic_flops_per_launch": 2.0 * nkd,
                         "peak_source": "measured bf16 (burst)" if peaks else "fallback"},
            "cpu_baseline": cpu,
        }), flush=True)


def run_kmpar(args, rank, world, dev, pg, barrier):
    """k-means|| (kpp_kmeans_par) on a seeding workload's points: each step
    is one whole initialisation (c_0, the oversampling rounds, the weights,
    the weighted k-means++ recluster).  Its dominant kernel on the large
    workloads is the tensor-core nearest-candidate search, timed alone
    (kpp_lloyd_assign at K = ell candidates) for the roofline."""
    import ctypes

    import torch

    import paper_1908_02136_gb300 as kpp
    from paper_1908_02136_gb300 import datagen, multi

    wl = datagen.WORKLOADS[args.workload[len(KMPAR_PREFIX):]]
    x = datagen.workload_points(wl, dev)
    N, d, K = wl.N, wl.d, wl.K
    ell, R = args.ell_mult * K, args.rounds
    cap = min(N, kpp.kmeans_par_cap(ell, R))
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    seed, sid = wl.draw_seed, multi.replica_stream(0, rank)
    with torch.cuda.stream(stream):
        ws = torch.empty(kpp.kpp_kmeans_par_workspace_size(N, d, cap), dtype=torch.uint8,
                         device=dev)

        def step():
            return kpp.kmeans_par(x, K, seed, sid, ell=ell, rounds=R, cand_cap=cap, workspace=ws)

        for _ in range(args.warmup):
            flush.fill_(1)
            r = step()
        n_cand = int(r["cand"].numel())
        torch.cuda.synchronize(dev)
        barrier()
        sampler = ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
        sampler.start()
        time.sleep(0.3)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a_, b_ in ev:
            flush.fill_(3)
            a_.record(stream)
            r = step()
            b_.record(stream)
        torch.cuda.synchronize(dev)
        # the dominant kernel alone: nearest of ell candidates for every point
        ke = min(N, 4096, int(round(ell)))
        ll = kpp.Lloyd(x, ke)
        C = x[r["cand"][:ke]].contiguous() if n_cand >= ke else x[:ke].contiguous()
        lab = torch.empty(N, dtype=torch.int32, device=dev)
        sh = ctypes.c_void_p(stream.cuda_stream)
        aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a_, b_ in aev:
            flush.fill_(3)
            a_.record(stream)
            st = kpp.kpp_lloyd_assign(C.data_ptr(), N, d, ke, lab.data_ptr(), ll.ws.data_ptr(),
                                      ll.ws.numel(), sh)
            b_.record(stream)
            if st != kpp.OK:
                raise kpp.KppError(st, "kpp_lloyd_assign")
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        barrier()
        st = kpp.kpp_read_status(ll.ws.data_ptr(), sh)
        if st != kpp.OK:
            raise kpp.KppError(st, "kpp_lloyd_assign (device)")
    step_ms = [a_.elapsed_time(b_) for a_, b_ in ev]
    a_ms = statistics.fmean(a_.elapsed_time(b_) for a_, b_ in aev)
    total_ms = multi.max_over_ranks(sum(step_ms), pg, dev)
    ms = total_ms / args.steps
    nkd = float(N) * K * d
    dp = 64 if d <= 64 else 128
    kpad = (ke + 127) // 128 * 128
    tensor_flops = 3 * 2.0 * N * kpad * dp
    peaks = measured_peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    achieved = tensor_flops / (a_ms / 1e3) / 1e12
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        # about 1.2e10 FP64 distance terms: N_s x (ell x rounds) x d
        n_s = int(min(N, max(4 * K, 1.2e10 / (ell * R * d))))
        xs = x[:n_s].cpu().numpy()
        t0 = time.perf_counter()
        o = oracle.kmeans_par(xs, K, ell, R, seed, sid, cand_cap=min(n_s, cap))
        dt = time.perf_counter() - t0
        cores, model = cpu_info()
        cpu = {"value": n_s * K * d / dt, "unit": "N*K*d/s", "cores": 1, "kind": "oracle",
               "sample": f"k-means|| on the first {n_s} of {N} points (same K, ell, rounds), "
                         f"{len(o['cand'])} candidates, serial FP64",
               "seconds": dt, "host_cores": cores, "cpu": model}
    if rank == 0:
        launches = 7 + 8 * R  # prepare, c_0, phi; 8 per round; weights, transpose, recluster, out
        print(json.dumps({
            "metric": "k-means|| initialisation N*K*d/s (oversampling + weighted recluster)",
            "value": nkd * world * args.steps / (total_ms / 1e3), "unit": "N*K*d/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "d": d, "K": K, "ell": ell,
                       "rounds": R, "candidates": n_cand, "status": int(r["status"]),
                       "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (512 MiB write)",
                       "phi_after_rounds": float(r["phi"].item()),
                       "assign_ms_at_ell": a_ms},
            "clocks": clocks, "e2e": None, "gpu_launches": launches * args.steps,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "lloyd_assign_pair_kernel",
                         "launch": f"kpp_lloyd_assign, N={N}, K={ke} candidates",
                         "tensor_flops_per_launch": tensor_flops,
                         "peak_source": "measured bf16 (burst)" if peaks else "fallback"},
            "cpu_baseline": cpu,
        }), flush=True)


def l2_bytes(dev) -> int:
    import torch

    try:
        return int(torch.cuda.get_device_properties(dev).L2_cache_size)
    except (AttributeError, RuntimeError):
        return 126 << 20


def read_peaks(kpp, dev):
    """Pure-read bandwidth of this GPU measured live (kpp_measure_read): HBM
    over a 4 GiB buffer, L2 over 64 MiB read 64 times after a warming sweep."""
    import torch

    out = {}
    try:
        out["hbm_read_gbs"] = kpp.measure_read_gbs(4 << 30, 8, dev)
        out["l2_read_gbs"] = kpp.measure_read_gbs(64 << 20, 64, dev)
    except (kpp.KppError, RuntimeError) as e:
        out["error"] = str(e)
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    return out


def roofline_for(plan, form_name, N, d, K, eb, has_scales, ms_per_step, wl_name, dtype, dev,
                 peaks_live):
    """Roofline of the dominant kernel of one seeding (the persistent kernel,
    one launch per seeding, or the streamed pass kernel, K launches).

    Algorithmic bytes per pass = the points (N*d*b, plus 4N for FP8 scales),
    plus the 8N bytes of D^2 read and written where D^2 lives in global memory
    (streamed form; persistent form without room for D^2 in shared memory).
    The bound is L2 when that working set fits the L2 (the persistent form
    keeps it there with an evict-last policy), HBM otherwise; `peak` is the
    measured copy bandwidth of MEASURED_PEAKS.json for HBM and the live
    L2 read rate for L2, with the live pure-read rates reported beside."""
    peaks = measured_peaks()
    hbm_copy = peaks["hbm_gbs"] if peaks else 6800.0
    launches = plan["launches"]
    per_launch_ms = ms_per_step / launches
    passes_per_launch = K // launches
    point_bytes = N * d * eb + (4 * N if has_scales else 0)
    d2_global = form_name in ("streamed", "recompute") or not plan["d2_in_smem"]
    d2_bytes = 8 * N if d2_global else 0
    per_pass = point_bytes + d2_bytes
    alg_bytes = passes_per_launch * per_pass
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    working_set = point_bytes + (4 * N if d2_global else 0)
    l2 = l2_bytes(dev)
    in_l2 = working_set <= l2
    traffic = (profiled_traffic(form_name, wl_name, dtype, plan, passes_per_launch)
               if form_name in KERNEL_SOURCES else None)
    if in_l2 and "l2_read_gbs" in peaks_live:
        bound, peak, src = "l2", peaks_live["l2_read_gbs"], "measured live: L2 read (kpp_measure_read)"
    else:
        bound, peak = "hbm", hbm_copy
        src = "measured copy (MEASURED_PEAKS.json)" if peaks else "fallback"
    r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "traffic": traffic, "peak_source": src,
         "kernel": f"{form_name}_kernel", "algorithmic_bytes_per_launch": alg_bytes,
         "algorithmic_bytes_per_pass": per_pass, "points_bytes_per_pass": point_bytes,
         "us_per_pass": 1e3 * per_launch_ms / passes_per_launch,
         "working_set_bytes": working_set, "l2_bytes": l2,
         "hbm_copy_gbs": hbm_copy, "frac_of_hbm_copy": achieved / hbm_copy,
         "nominal_hbm_gbs": NOMINAL_HBM_GBS, "frac_of_nominal_hbm": achieved / NOMINAL_HBM_GBS}
    if "hbm_read_gbs" in peaks_live:
        r["hbm_read_gbs"] = peaks_live["hbm_read_gbs"]
        r["frac_of_hbm_read"] = achieved / peaks_live["hbm_read_gbs"]
    if "l2_read_gbs" in peaks_live:
        r["l2_read_gbs"] = peaks_live["l2_read_gbs"]
    if traffic is not None:
        r["traffic_over_algorithmic"] = traffic / alg_bytes
    return r


def run_seeding(args, rank, world, local, dev, pg, barrier):
    """One problem of a seeding workload: the FP32 (or --dtype) seeding timed
    over --steps, then -- for an FP32 run -- the same data stored as BF16 and
    FP8 (--forms), each timed on fewer steps, with the cost distortion of its
    seeds; the end-to-end time through kpp_seed_host; the roofline of the
    dominant kernel; and the multi-threaded FP64 oracle as the CPU baseline."""
    import ctypes

    import numpy as np
    import torch

    import paper_1908_02136_gb300 as kpp
    from paper_1908_02136_gb300 import datagen, multi

    wl = datagen.WORKLOADS[args.workload]
    if args.n_points or args.k_seeds:
        import dataclasses

        n_, k_ = args.n_points or wl.N, args.k_seeds or wl.K
        wl = dataclasses.replace(wl, N=n_, K=k_, name=f"{wl.name}@N{n_}K{k_}")
    x_np = datagen.workload_points(wl) if wl.N <= 2_000_000 else None
    x = torch.from_numpy(x_np).to(dev) if x_np is not None else datagen.workload_points(wl, dev)
    N, d, K = wl.N, wl.d, wl.K
    peaks_live = read_peaks(kpp, dev) if not args.no_read_peaks else {}
    opts = kpp.Options()
    opts.form = args.form
    opts.lanes_per_row = args.lanes
    opts.ctas_per_sm = args.ctas_per_sm
    opts.smem_cache = args.smem_cache
    opts.alternate = args.alternate
    opts.l2_policy = args.l2_policy
    opts.min_rows_per_cta = args.min_rows
    knobs = (args.form, args.lanes, args.ctas_per_sm, args.smem_cache, args.alternate,
             args.l2_policy, args.min_rows)
    stream = torch.cuda.Stream(dev)
    sh = ctypes.c_void_p(stream.cuda_stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    seed = wl.draw_seed
    stream_id = multi.replica_stream(0, rank)
    codes = {"f32": kpp.F32, "bf16": kpp.BF16, "fp8": kpp.FP8_E4M3}
    ebytes = {"f32": 4, "bf16": 2, "fp8": 1}

    def store(dtype):
        """The points as stored for `dtype`; quantisation (S0) timed apart."""
        if dtype == "f32":
            return x, None, 0.0
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a_.record(stream)
            q = kpp.quantize(x, dtype)
            b_.record(stream)
        torch.cuda.synchronize(dev)
        pts_, sc_ = (q, None) if dtype == "bf16" else q
        return pts_, sc_, a_.elapsed_time(b_)

    def time_form(dtype, pts, scales, steps, warmup):
        """Tunes (untimed), then times `steps` seedings with CUDA events on the
        launching stream, L2 flushed between them, clocks sampled."""
        code = codes[dtype]
        tuned = None
        if not args.no_tune and not any(knobs):
            t0 = time.time()
            try:
                best, tms = kpp.tune(pts, K, dtype=code, row_scales=scales,
                                     passes=args.tune_passes)
                tuned = {"options": {k: v for k, v in best.items() if v}, "ms_per_pass": tms,
                         "seconds": round(time.time() - t0, 2)}
            except kpp.KppError as e:
                tuned = {"error": str(e)}
        with torch.cuda.device(dev):
            pst, plan = kpp.kpp_describe(N, d, K, code, opts)
        if pst != kpp.OK:
            raise kpp.KppError(pst, "kpp_describe")
        plan = plan.as_dict()
        ws = kpp.workspace_for(N, d, K, code, dev, opts)
        idx = torch.empty(K, dtype=torch.int64, device=dev)
        d2 = torch.empty(N, dtype=torch.float32, device=dev)
        phi = torch.empty(1, dtype=torch.float64, device=dev)

        def launch():
            st = kpp.kpp_seed(pts.data_ptr(), None if scales is None else scales.data_ptr(), N,
                              d, K, code, seed, stream_id, None, 0, idx.data_ptr(),
                              d2.data_ptr(), phi.data_ptr(), ws.data_ptr(), ws.numel(), sh, opts)
            if st != kpp.OK:
                raise kpp.KppError(st, "kpp_seed")

        with torch.cuda.stream(stream):
            for _ in range(warmup):
                flush.fill_(1)
                launch()
            st = kpp.kpp_read_status(ws.data_ptr(), sh)
            if st != kpp.OK:
                raise kpp.KppError(st, "warmup")
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
            torch.cuda.synchronize(dev)
            barrier()
            torch.cuda.synchronize(dev)
            sampler = ClockSampler(local)
            sampler.start()
            time.sleep(0.3)  # let the sampler take a first sample
            for s_ in range(steps):
                flush.fill_(s_ & 0xFF)  # L2 flush between steps, outside the events
                starts[s_].record(stream)
                launch()
                ends[s_].record(stream)
            torch.cuda.synchronize(dev)
            clocks = sampler.stop()
            barrier()
            st = kpp.kpp_read_status(ws.data_ptr(), sh)
            if st != kpp.OK:
                raise kpp.KppError(st, "timed steps")
        step_ms = [a_.elapsed_time(b_) for a_, b_ in zip(starts, ends)]
        total_ms = multi.max_over_ranks(sum(step_ms), pg, dev)
        # cheap invariants of the timed result (full parity lives in tests/)
        idx_h = idx.cpu().numpy()
        assert np.all((idx_h >= 0) & (idx_h < N)) and len(set(idx_h.tolist())) == K
        assert float(d2[idx].abs().max()) == 0.0
        form_name = {kpp.FORM_STREAMED: "streamed", kpp.FORM_PERSISTENT: "persistent",
                     kpp.FORM_RECOMPUTE: "recompute", kpp.FORM_SMALL: "small"}[plan["form"]]
        return {"idx": idx, "d2": d2, "phi": phi, "ws": ws, "plan": plan, "form": form_name,
                "tuned": tuned, "ms": total_ms / steps, "step_ms": step_ms,
                "clocks": clocks, "steps": steps}

    def phi_gate(dtype, r):
        """Cost distortion of a precision form's seeds: its own phi (its sum of
        D^2 on its stored points) against the FP64-summed cost of the same
        seeds on the original FP32 points (the FP32 path replayed on its
        indices), and that cost against an FP32 seeding with the same draws."""
        with torch.cuda.stream(stream):
            phi_form = float(r["phi"].item())
            _, _, phi_orig = kpp.seed(x, K, seed, stream_id, forced=r["idx"].clone(), check=True)
            _, _, phi32 = kpp.seed(x, K, seed, stream_id, check=True)
            torch.cuda.synchronize(dev)
        phi_orig, phi32 = float(phi_orig.item()), float(phi32.item())
        g = {"phi_form_own": phi_form, "phi_of_form_seeds_on_fp32_points": phi_orig,
             "phi_rel_diff": abs(phi_form - phi_orig) / phi_orig,
             "phi_gate_1e-3": abs(phi_form - phi_orig) <= 1e-3 * phi_orig,
             "phi_fp32_same_seed": phi32, "phi_vs_fp32_run": (phi_orig - phi32) / phi32}
        if args.phi_seeds > 1:
            g["over_seeds"] = phi_over_seeds(kpp, x, r["pts"], r["scales"], codes[dtype], K,
                                             wl.draw_seed, stream_id, args.phi_seeds, stream, dev)
        return g

    dtype = args.dtype
    pts, scales, q_ms = store(dtype)
    main_r = time_form(dtype, pts, scales, args.steps, args.warmup)
    main_r["pts"], main_r["scales"] = pts, scales
    ms_per_step = main_r["ms"]
    nkd = float(N) * K * d
    value = nkd * world / (ms_per_step / 1e3)
    roofline = roofline_for(main_r["plan"], main_r["form"], N, d, K, ebytes[dtype],
                            scales is not None, ms_per_step, wl.name, dtype, dev, peaks_live)
    precision = None
    if dtype != "f32" and not args.no_phi:
        precision = phi_gate(dtype, main_r)
        precision["quantize_ms"] = q_ms
    parity = None if args.no_parity_sample else sampled_parity(main_r, pts, scales, dtype, N, K,
                                                               seed, stream_id)

    # precision forms of the same data beside the FP32 headline
    forms_block = None
    forms = [] if (dtype != "f32" or args.forms in ("", "none")) else args.forms.split(",")
    if forms:
        forms_block = {}
        for fd in forms:
            fpts, fsc, fq_ms = store(fd)
            fr = time_form(fd, fpts, fsc, max(1, min(args.steps, args.form_steps)),
                           max(1, min(args.warmup, 2)))
            fr["pts"], fr["scales"] = fpts, fsc
            froof = roofline_for(fr["plan"], fr["form"], N, d, K, ebytes[fd], fsc is not None,
                                 fr["ms"], wl.name, fd, dev, peaks_live)
            entry = {"ms_per_seeding": fr["ms"], "value": nkd * world / (fr["ms"] / 1e3),
                     "speedup_vs_f32": ms_per_step / fr["ms"], "steps": fr["steps"],
                     "quantize_ms": fq_ms, "form": fr["form"], "plan": fr["plan"],
                     "autotuner": fr["tuned"], "clocks": fr["clocks"],
                     "gpu_launches": fr["plan"]["launches"] * fr["steps"],
                     "roofline": {k: froof[k] for k in
                                  ("bound", "achieved", "peak", "frac", "traffic",
                                   "traffic_over_algorithmic", "frac_of_hbm_read",
                                   "frac_of_nominal_hbm", "us_per_pass",
                                   "algorithmic_bytes_per_pass")
                                  if k in froof}}
            if not args.no_phi:
                entry["phi"] = phi_gate(fd, fr)
            forms_block[fd] = entry
            del fpts, fsc, fr
            torch.cuda.empty_cache()

    # e2e: host points (pinned) -> C ABI -> host results, wall clock incl. copies
    e2e = None
    if not args.no_e2e:
        xh = pts.cpu().pin_memory()
        sh_host = None if scales is None else scales.cpu().pin_memory()
        hidx, hd2, hphi, st, bufs = kpp.seed_host(xh, K, seed, stream_id, dtype=dtype,
                                                  row_scales_host=sh_host, device=dev, opts=opts)
        e2e_steps = max(1, min(args.steps, 5 if N * d * ebytes[dtype] < (1 << 30) else 3))
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            hidx, hd2, hphi, st, bufs = kpp.seed_host(xh, K, seed, stream_id, dtype=dtype,
                                                      row_scales_host=sh_host, device=dev,
                                                      opts=opts, buffers=bufs)
            if st != kpp.OK:
                raise kpp.KppError(st, "kpp_seed_host")
        e2e_s = multi.max_over_ranks(time.perf_counter() - t0, pg, dev)
        h2d = N * d * ebytes[dtype] + (4 * N if scales is not None else 0)
        d2h = 8 * K + 4 * N + 8
        e2e = {"value": nkd * world * e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * e2e_s / e2e_steps, "steps": e2e_steps}
        del xh, sh_host, bufs

    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        stored = x_np if dtype == "f32" else (
            pts.cpu().numpy().view(np.uint16) if dtype == "bf16" else pts.cpu().numpy())
        if stored is None:
            stored = x.cpu().numpy()
        sc_np = None if scales is None else scales.cpu().numpy()
        cpu_baseline = oracle_baseline(stored, sc_np, K, seed, stream_id)

    if rank == 0:
        plan = main_r["plan"]
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic",
            "config": {"workload": wl.name, "N": N, "d": d, "K": K, "storage": dtype,
                       "form": main_r["form"], "plan": plan, "autotuner": main_r["tuned"],
                       "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (512 MiB write)",
                       "step_ms_min": min(main_r["step_ms"]),
                       "step_ms_max": max(main_r["step_ms"])},
            "clocks": main_r["clocks"], "e2e": e2e,
            "gpu_launches": plan["launches"] * args.steps,
            "precision": precision, "forms": forms_block, "parity_sample": parity,
            "read_peaks": peaks_live,
            "roofline": roofline, "cpu_baseline": cpu_baseline,
        }), flush=True)


def run_sharded_seeding(args, rank, world, local, dev, pg, barrier):
    """--shard points: ONE problem of the workload split by rows over the
    ranks (contiguous ranges, Algorithm 2's partition), each rank seeding its
    range with kpp_shard_* and exchanging, per pass, the D^2 totals
    (all-gather) and the new centre's row (sum all-reduce) over NCCL.  A step
    is one whole seeding of the problem; strong scaling of the fixed problem."""
    import torch

    import paper_1908_02136_gb300 as kpp
    from paper_1908_02136_gb300 import datagen, multi

    wl = datagen.WORKLOADS[args.workload]
    if args.n_points or args.k_seeds:
        import dataclasses

        n_, k_ = args.n_points or wl.N, args.k_seeds or wl.K
        wl = dataclasses.replace(wl, N=n_, K=k_, name=f"{wl.name}@N{n_}K{k_}")
    N, d, K = wl.N, wl.d, wl.K
    lo, hi = multi.shard_rows(N, world)[rank]
    x = (torch.from_numpy(datagen.workload_points(wl)).to(dev) if N <= 2_000_000
         else datagen.workload_points(wl, dev))
    mine = x[lo:hi].clone()  # this rank's rows only
    del x
    torch.cuda.empty_cache()
    comm = multi.ProcessGroupComm(pg) if pg is not None else multi.InProcessComm()
    shard = kpp.PointShard(mine, lo, N, K, wl.draw_seed, 0, rank, world)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.fill_(1)
        multi.seed_sharded([shard], comm, K)
    torch.cuda.synchronize(dev)
    st = shard.status()
    if st != kpp.OK:
        raise kpp.KppError(st, "sharded warmup")
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        starts[s_].record(stream)
        multi.seed_sharded([shard], comm, K)
        ends[s_].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = multi.max_over_ranks(sum(step_ms), pg, dev)
    ms = total_ms / args.steps
    idx = shard.idx.cpu().numpy()
    assert (idx >= 0).all() and (idx < N).all() and len(set(idx.tolist())) == K
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    per_pass = (hi - lo) * d * 4 + 8 * (hi - lo)  # this rank's points and D^2
    achieved = per_pass * K / (ms / 1e3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": float(N) * K * d / (ms / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "N": N, "d": d, "K": K, "form": "sharded",
                       "parallelism": f"points split over {world} ranks (contiguous rows)",
                       "rows_on_rank0": hi - lo,
                       "l2": "flushed between steps (512 MiB write)"},
            "clocks": clocks, "e2e": None,
            # per pass: the pass, the pick (not after the last), plus the first seed and phi
            "gpu_launches": args.steps * (2 * K + 1),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "streamed pass kernel (per rank)",
                         "algorithmic_bytes_per_pass_rank0": per_pass},
            "cpu_baseline": None,
        }), flush=True)


def sampled_parity(r, pts, scales, dtype, N, K, seed, stream_id, n_rows: int = 2000):
    """Checks of the timed seeding's own output that any size allows (plain
    FP64 numpy on a sample, not the oracle): the indices are distinct and in
    range, D^2 is 0 at every chosen point, and the D^2 of `n_rows` sampled
    rows equals, within 1e-5 relative, the FP64 minimum of the squared
    distances from the stored values to all K chosen centres."""
    import numpy as np
    import torch

    idx = r["idx"].cpu().numpy()
    d2 = r["d2"]
    rng = np.random.default_rng(12345)
    rows = np.sort(rng.choice(N, min(N, n_rows), replace=False))

    def decode(sel):
        t = torch.as_tensor(sel, device=pts.device)
        if dtype == "f32":
            return pts[t].double().cpu().numpy()
        if dtype == "bf16":
            return pts[t].view(torch.bfloat16).double().cpu().numpy()
        q = pts[t].view(torch.float8_e4m3fn).double()
        return (q * scales[t].double()[:, None]).cpu().numpy()

    xs, cs = decode(rows), decode(idx)
    best = np.full(rows.size, np.inf)
    for k0 in range(0, K, 128):
        diff = xs[:, None, :] - cs[None, k0:k0 + 128, :]
        best = np.minimum(best, np.einsum("ijk,ijk->ij", diff, diff).min(axis=1))
    got = d2[torch.as_tensor(rows, device=d2.device)].double().cpu().numpy()
    zero = best == 0.0
    rel = np.abs(got[~zero] - best[~zero]) / best[~zero]
    ok_zero = bool(np.all(got[zero] == 0.0))
    chosen_zero = bool(float(d2[r["idx"]].abs().max()) == 0.0)
    return {"rows": int(rows.size), "max_rel_d2_err": float(rel.max()) if rel.size else 0.0,
            "d2_tolerance": 1e-5, "zero_where_expected": ok_zero,
            "chosen_points_zero": chosen_zero,
            "distinct_in_range": bool(len(set(idx.tolist())) == K and (idx >= 0).all()
                                      and (idx < N).all()),
            "ok": bool((rel.max() if rel.size else 0.0) <= 1e-5 and ok_zero and chosen_zero)}


def oracle_baseline(stored, scales, K, seed, stream_id, budget_s: float = 15.0):
    """The multi-threaded FP64 oracle on all host cores, on the workload's
    stored points, for as many of the K passes as fit about `budget_s`
    seconds (calibrated on a 2-pass run); N*K*d per second."""
    import oracle

    N, d = stored.shape
    cores, model = cpu_info()
    t0 = time.perf_counter()
    r = oracle.seed_mt(stored, min(2, K), seed, stream_id, scales=scales, threads=cores)
    per_pass = (time.perf_counter() - t0) / min(2, K)
    K_s = int(max(1, min(K, budget_s / max(per_pass, 1e-9))))
    t0 = time.perf_counter()
    r = oracle.seed_mt(stored, K_s, seed, stream_id, scales=scales, threads=cores)
    dt = time.perf_counter() - t0
    import hashlib

    import numpy as np

    # the exact bytes the oracle read (and the GPU path was given)
    digest = hashlib.sha256(memoryview(np.ascontiguousarray(stored)).cast("B")).hexdigest()
    return {"value": N * K_s * d / dt, "unit": UNIT, "cores": r["threads"], "kind": "oracle",
            "sample": f"full workload data ({N} x {d}), first {K_s} of {K} passes, "
                      f"multi-threaded FP64 oracle on {r['threads']} threads ({dt:.1f} s)",
            "host_cores": cores, "cpu": model, "seconds": dt,
            "data_sha256": digest}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import paper_1908_02136_gb300 as kpp
    from paper_1908_02136_gb300 import datagen, multi

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    if args.workload == BATCH_WORKLOAD:
        run_batch(args, rank, world, dev, pg, barrier)
        return
    if args.workload.startswith(LLOYD_PREFIX):
        run_lloyd(args, rank, world, dev, pg, barrier)
        return
    if args.workload.startswith(KMPAR_PREFIX):
        run_kmpar(args, rank, world, dev, pg, barrier)
        return
    if args.shard == "points":
        run_sharded_seeding(args, rank, world, local, dev, pg, barrier)
    else:
        run_seeding(args, rank, world, local, dev, pg, barrier)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
