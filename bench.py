"""Benchmark of the black-box FMM matvec (phi = K_hat sigma) on GB300.

Default workload ("uniform-1M-p5-d5"): N = 1,048,576 points uniform in the
unit cube, kernel 1/r, Chebyshev order p = 5, uniform octree of depth 5, one
right-hand side, sigma ~ U(-1, 1) -- the N = 1M 1/r configuration at the
depth that is fastest here (depth 6 is timed too, under "depth6").  Other
named workloads (--workload): uniform-1M-p5-d6, clustered-2M-exp0.3-p6-d6,
jittered-500k-exp0.2-p5-d5-rhs64, uniform-4k-p4-d3 (see workloads.py).

A step is one full matvec (gather, P2M/M2M/compress, M2L, L2L/decompress,
L2P, P2P, combine) with inputs resident in HBM.  L2 is flushed between timed
steps by writing a 512 MB buffer (the working set is smaller than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload NAME] [--precision fp16x3|tf32x3|bf16x3|tf32|fp32]
                    [--interp chebyshev|uniform] [--near auto|ordered|symmetric]

Prints one JSON line (rank 0).  Under torchrun every rank runs an
independent replica of the workload (the matvec is single-GPU: replicas
only) and value counts all ranks' work over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1903_02153_gb300 import workloads as W  # noqa: E402

METRIC = ("N=1M 1/r matvec ms & N^2/s at rel err<=1e-5 vs plain GPU form; serve p50/p99 ms")
KERNEL_NAMES = {1: "1/r", 2: "1/r^2", 3: "exp(-r/ell)", 4: "exp(-(r/ell)^2)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform-1M-p5-d5", choices=sorted(W.CONFIGS))
    ap.add_argument("--precision", default="fp16x3")
    ap.add_argument("--interp", default="chebyshev", choices=["chebyshev", "uniform"],
                    help="uniform: equally spaced nodes with the Fourier-domain M2L (FP32)")
    ap.add_argument("--svd-eps", type=float, default=1e-6)
    ap.add_argument("--near", default="auto", choices=["auto", "ordered", "symmetric", "box"],
                    help="near-field form: symmetric = each neighbour leaf pair once (symmetric kernels), "
                         "ordered = every target leaf its own pairs, box = ordered with a work item per "
                         "level-(D-1) box, auto = measured by the autotuner; a fixed form keeps the "
                         "tuner's other choices (a profiler run "
                         "pins the form the plain run chose, since the tuner's timings under it mislead)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-depth6", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-precision-forms", action="store_true",
                    help="skip the 2M clustered exp(-r/0.3) p = 6 workload in every M2L arithmetic form")
    ap.add_argument("--serving", type=int, default=200,
                    help="timed requests of the Poisson serving stream (p50/p99 latency, throughput); 0 = skip")
    return ap.parse_args()


def serving(args, torch):
    """Continuous-batching request loop on a Poisson stream (workloads.
    serving_stream with a pool of 12 resident plans): mixed N (log-uniform
    10k..500k, uniform/clustered), kernels, p in {4,5,6}, nrhs in {1,8,32}.
    1. warm-up: every plan of the pool is built and run once per nrhs value;
    2. capacity: a closed burst of requests from the stream, all submitted at
       once (the server batches and overlaps them); capacity = requests / time;
    3. timed: open-loop Poisson arrivals at 0.6 x that capacity; latency is
       submit -> result on the host (pinned-memory transfers included)."""
    from paper_1903_02153_gb300 import serve as S
    npool, burst = 12, 48
    reqs = W.serving_stream(burst + args.serving, n_hi=500_000, plans=npool)
    pts_cache = {}

    def point_source(key):
        kind, n, seed, kid, ell, p, depth = key
        if (kind, n, seed) not in pts_cache:
            pts_cache[(kind, n, seed)] = W.make_points(kind, n, seed)
        return pts_cache[(kind, n, seed)], kid, ell, p, depth

    def key_of(d):
        return (d["kind"], d["n"], d["point_seed"], d["kernel"], d["ell"], d["p"], d["depth"])

    def make(d, nrhs=None):
        nrhs = d["nrhs"] if nrhs is None else nrhs
        sig = W.uniform_sigma(d["n"], nrhs, seed=d["sigma_seed"]).astype(np.float32)
        return S.Request(key_of(d), sig.reshape(d["n"], nrhs))

    ex = S.GpuExecutor(point_source, precision=args.precision, svd_eps=args.svd_eps, slots=4,
                       domain=(W.UNIT_LO, W.UNIT_SIDE))
    srv = S.Server(ex, device_budget_bytes=96 << 30, slots=4, max_batch_nrhs=32).start()
    t0 = time.perf_counter()
    pool = {}
    for d in reqs:
        pool.setdefault(key_of(d), d)
    for d in pool.values():
        for nrhs in (1, 8, 32):
            srv.submit(make(d, nrhs)).wait(600)
    warm_s = time.perf_counter() - t0
    builds0 = srv.builds
    t0 = time.perf_counter()
    hs = [srv.submit(make(d)) for d in reqs[:burst]]
    for h in hs:
        h.wait(600)
    capacity = burst / (time.perf_counter() - t0)
    rate = 0.6 * capacity
    timed = []
    t_start = time.perf_counter()
    t_next = t_start
    for d in reqs[burst:]:
        t_next += d["gap"] / rate
        while time.perf_counter() < t_next:
            time.sleep(50e-6)
        timed.append(srv.submit(make(d)))
    for r in timed:
        r.wait(600)
    wall = max(r.t_done for r in timed) - t_start
    srv.stop()
    ok = [r for r in timed if r.error is None]
    lat = np.array([r.latency for r in ok])
    return {"requests": len(timed), "failed": len(timed) - len(ok), "resident_plans": len(pool),
            "warmup_s_incl_plan_builds": warm_s, "plan_builds_after_warmup": srv.builds - builds0,
            "capacity_req_per_s": capacity, "arrival_rate_per_s": rate,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "throughput_N2nrhs_per_s": sum(float(r.n) ** 2 * r.nrhs for r in ok) / wall,
            "requests_per_s": len(ok) / wall, "mean_batch": float(np.mean([r.batch_size for r in ok])),
            "mix": "12 resident plans: N log-uniform 10k..500k, uniform/clustered, K in {1/r, 1/r^2, "
                   "exp(-r), exp(-r^2)}, p in {4,5,6}; nrhs in {1,8,32}; Poisson arrivals at 0.6 x the "
                   "closed-burst capacity; 4 slots; max batch 32 columns"}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window": "last 1 s of warm-up + stage timing + timed steps"}


def workload(name):
    c = dict(W.CONFIGS[name])
    c["name"] = name
    pts = W.make_points(c["kind"], c["n"])
    sig = W.make_sigma(c["kind"], c["n"], c["nrhs"]).astype(np.float32)
    if sig.ndim == 1:
        sig = sig[:, None]
    return c, pts, np.asfortranarray(sig)


def describe(c):
    return ("%s: N=%d %s points, K=%s (ell=%g), p=%d, depth %d, %d RHS"
            % (c["name"], c["n"], c["kind"], KERNEL_NAMES[c["kernel"]], c["ell"], c["p"], c["depth"], c["nrhs"]))


def tuning_summary(bb, plan, nrhs):
    """The plan's launch choices for nrhs (after the autotuner ran)."""
    t = bb.bbfmm_get_tuning(plan.handle, nrhs)
    if t.near_mode == bb.NEAR_MODES["symmetric"]:
        near = "symmetric pairs"
    else:
        near = "ordered, a work item per level-(D-1) box" if t.near_box else "ordered"
    return {"near_field": near, "m2l_tile": int(t.m2l_tile), "m2l_stages": int(t.m2l_stages),
            "leaf_gemm": bool(t.leaf_gemm), "measured": bool(t.measured)}


def make_plan(bb, torch, dev, pts, c, depth, precision, eps, interp="chebyshev", near="auto"):
    """A plan of workload c; near "box" (the ordered form by level-(D-1) box)
    runs the tuning sweep and then fixes the near-field form."""
    mode = {"box": "ordered"}.get(near, near)
    plan = bb.Plan(torch.from_numpy(pts).to(dev), c["kernel"], c["p"], depth, ell=c["ell"], precision=precision,
                   svd_eps=eps, domain=(W.UNIT_LO, W.UNIT_SIDE), max_nrhs=c["nrhs"], interp=interp, near_mode=mode)
    if near == "box":
        bb.bbfmm_autotune(plan.handle, c["nrhs"])
        t = bb.bbfmm_get_tuning(plan.handle, c["nrhs"])
        bb.bbfmm_set_tuning(plan.handle, c["nrhs"], mode, t.m2l_tile, t.m2l_stages, near_box=True,
                            leaf_gemm=bool(t.leaf_gemm))
    return plan


def time_plan(bb, torch, dev, pts, sig_dev, c, depth, precision, eps, flush, stream, nsteps=5, interp="chebyshev",
              near="auto"):
    """Mean device time of nsteps matvecs (L2 flushed before each)."""
    plan = make_plan(bb, torch, dev, pts, c, depth, precision, eps, interp, near)
    phi = torch.empty_like(sig_dev)
    for _ in range(3):
        bb.bbfmm_matvec(plan.handle, sig_dev, phi, c["nrhs"], stream)
    ts = []
    for _ in range(nsteps):
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bb.bbfmm_matvec(plan.handle, sig_dev, phi, c["nrhs"], stream)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    info = plan.info()
    tuning = tuning_summary(bb, plan, c["nrhs"])
    out = phi.cpu().numpy().astype(np.float64)
    # per-stage device times (L2 flushed), for this form's M2L roofline
    bb.bbfmm_set_timing(plan.handle, True)
    stage = np.zeros(8)
    for _ in range(3):
        flush.fill_(4.0)
        bb.bbfmm_matvec(plan.handle, sig_dev, phi, c["nrhs"], stream)
        torch.cuda.synchronize()
        stage += bb.bbfmm_stage_times(plan.handle)
    stage /= 3
    plan.close()
    ms = float(np.mean(ts))
    return ({"depth": depth, "m2l_precision": precision, "near_field": tuning["near_field"], "tuning": tuning,
             "ms_per_step": ms,
             "value": float(c["n"]) ** 2 * c["nrhs"] / (ms / 1e3),
             "near_symmetric": int(info.near_symmetric), "close_pairs": int(info.close_pairs),
             "stages_ms": {k: float(v) for k, v in zip(bb.STAGES, stage)}, "_info": info},
            out.T if out.ndim == 2 else out[:, None])


# DRAM traffic per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)
# is recorded in this file with a digest of the sources the kernel was built
# from; a figure counts only while the kernel's sources still have that
# digest (otherwise the kernel changed since the capture and traffic is null)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_uniform1M_p5.txt")
KERNEL_SOURCES = {"k_m2l_tc": ["m2l_tc.cu", "tc_ptx.cuh"],
                  "k_p2p_sym": ["p2p_kernels.cuh", "p2p.cu"], "k_p2p": ["p2p_kernels.cuh", "p2p.cu"]}


def source_digest(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1903_02153_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload, precision):
    """Bytes per launch from the traffic file, or None when the kernel's
    sources changed since the capture (or nothing was captured for it)."""
    if kernel not in KERNEL_SOURCES or not os.path.exists(TRAFFIC_FILE):
        return None
    want = source_digest(kernel)
    with open(TRAFFIC_FILE) as fh:
        for line in fh:
            f = line.split()
            if len(f) >= 5 and not line.startswith("#") and f[:3] == [kernel, workload, precision] and f[3] == want:
                return int(f[4])
    return None


def roofline(precision, info, nrhs, m2l_ms, clocks, torch, dev, workload=None, interp="chebyshev", p=5):
    peaks, kind = measured_peaks()
    if interp == "uniform":
        # Fourier-domain M2L: per interaction pair and kept frequency one
        # complex multiply-add (8 flops) on the FP32 pipe; the per-box DFTs are
        # not counted (they are ~5 % of the pairs' work at p = 5)
        nf = 2 * p - 1
        nw = nf * nf * p
        flops = 8.0 * info.m2l_pairs * nw * nrhs
        f_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * 128 * 2 * f_mhz * 1e6 / 1e12
        achieved = flops / (m2l_ms / 1e3) / 1e12
        return {"kernel": "k_fft_fwd + k_fft_m2l + k_fft_inv (all levels)", "bound": "alu", "peak": peak,
                "peak_source": "FP32 FMA: %d SMs x 128 lanes x 2 flop x median SM clock %.0f MHz" % (sms, f_mhz),
                "achieved": achieved, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "work": "8 flops x %d interaction pairs x %d frequencies x %d RHS" % (info.m2l_pairs, nw, nrhs)}
    passes = {"fp32": 1, "tf32": 1, "tf32x3": 3, "bf16x3": 3, "fp16x3": 3}[precision]
    flops = 2.0 * info.m2l_pairs * info.rank * info.rank * passes * nrhs
    achieved = flops / (m2l_ms / 1e3) / 1e12
    if precision == "fp32":
        f_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * 128 * 2 * f_mhz * 1e6 / 1e12
        r = {"kernel": "k_m2l_fp32 (all levels)", "bound": "alu", "peak": peak,
             "peak_source": "FP32 FMA: %d SMs x 128 lanes x 2 flop x median SM clock %.0f MHz" % (sms, f_mhz)}
    elif precision in ("tf32", "tf32x3"):
        r = {"kernel": "k_m2l_tc (all levels)", "bound": "tensor", "peak": peaks["bf16_tflops"] * 1.1 / 2.25,
             "peak_source": "%s bf16 %.0f TF/s x nominal tf32/bf16 ratio 1.1/2.25" % (kind, peaks["bf16_tflops"])}
    else:
        r = {"kernel": "k_m2l_tc (all levels)", "bound": "tensor", "peak": peaks["bf16_tflops"],
             "peak_source": "%s bf16 dense %.0f TF/s (fp16 runs at the same rate)" % (kind, peaks["bf16_tflops"])}
    r.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / r["peak"],
              "traffic": measured_traffic("k_m2l_tc", workload, precision) if precision != "fp32" else None,
              "work": "2 r^2 flops x %d interaction pairs x %d pass(es) x %d RHS, r = %d"
                      % (info.m2l_pairs, passes, nrhs, info.rank)})
    return r


MUFU_PER_EVAL = {1: 1, 2: 1, 3: 2, 4: 1}   # rsqrt; rcp; rsqrt + ex2; ex2


def stage_rooflines(info, c, nrhs, stage, precision, clocks, torch, dev, m2l, ms_step):
    """Each stage's algorithmic work over its CUDA-event time (stage timing
    runs the stages one after another, so each time is that stage alone),
    against the bound of that stage, and the overall fraction sum(ideal stage
    times) / the timed matvec (ms_step: stages overlapped as in production).
      upward / downward: FP32 flops of P2M (2 N p^3), compression and
        decompression (2 p^3 r per box and level), M2M / L2L (8 children x 3
        passes x p^4 FMAs per parent), L2P (2 N p^3), against the FP32 FMA
        peak (SMs x 128 lanes x 2 x clock);
      m2l: the tensor-core roofline above;
      p2p: kernel evaluations (ordered pairs, or about half with the
        symmetric form) against the MUFU bound (SMs x 16 per clock / MUFU ops
        per evaluation) and, beside it, the FP32 pipe at ~7 FP32 ops per
        evaluation (3 differences, 3 FMAs for r^2, 1 FMA into the sum);
      gather / combine: bytes moved against the measured HBM bandwidth."""
    peaks, kind = measured_peaks()
    f_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32 = sms * 128 * 2 * f_mhz * 1e6            # flop/s
    N, p, D, r = float(c["n"]), c["p"], c["depth"], info.rank
    p3 = p ** 3
    boxes = sum(8 ** l for l in range(2, D + 1))
    parents = sum(8 ** l for l in range(2, D))
    up_flops = nrhs * (2 * N * p3 + 2.0 * p3 * r * boxes + parents * 2.0 * 8 * 3 * p ** 4)
    down_flops = nrhs * (2.0 * p3 * r * boxes + parents * 2.0 * 8 * 3 * p ** 4 + 2 * N * p3)
    mufu = sms * 16 * f_mhz * 1e6 / MUFU_PER_EVAL.get(c["kernel"], 1)
    evals = float(info.p2p_evals) * nrhs
    slots = 13 * 4 * N if (info.near_symmetric and nrhs == 1) else 0.0
    gather_b = 4 * N * (1 + 2 * nrhs) + (4 * N * nrhs if nrhs > 1 else 0)
    combine_b = 4 * N * (1 + 3 * nrhs) + slots
    hbm = peaks["hbm_gbs"] * 1e9
    ms = {k: float(v) for k, v in zip(["gather", "upward", "m2l", "downward", "l2p", "p2p", "combine", "total"],
                                      stage)}

    def ent(work, t_ms, peak, unit, scale, bound, what):
        ach = work / (t_ms / 1e3) if t_ms > 0 else 0.0
        return {"bound": bound, "achieved": ach / scale, "peak": peak / scale, "unit": unit,
                "frac": ach / peak, "ms": t_ms, "ideal_ms": 1e3 * work / peak, "work": what}

    out = {
        "upward": ent(up_flops, ms["upward"], fp32, "TFLOP/s", 1e12, "alu",
                      "%.3g FP32 flops (P2M, M2M, compression)" % up_flops),
        "downward": ent(down_flops, ms["downward"], fp32, "TFLOP/s", 1e12, "alu",
                        "%.3g FP32 flops (decompression, L2L, L2P)" % down_flops),
        "p2p": ent(evals, ms["p2p"], mufu, "Geval/s", 1e9, "mufu",
                   "%d kernel evaluations (%d ordered pairs) x %d RHS, %d MUFU op(s) each"
                   % (info.p2p_evals, info.p2p_pairs, nrhs, MUFU_PER_EVAL.get(c["kernel"], 1))),
        "gather": ent(gather_b, ms["gather"], hbm, "GB/s", 1e9, "hbm", "%d bytes" % gather_b),
        "combine": ent(combine_b, ms["combine"], hbm, "GB/s", 1e9, "hbm", "%d bytes" % combine_b),
    }
    out["p2p"]["frac_of_fp32_pipe"] = evals * 7 / (ms["p2p"] / 1e3) / fp32 if ms["p2p"] > 0 else 0.0
    m2l_ideal = m2l["frac"] * ms["m2l"]     # work / peak = achieved x time / peak
    out["m2l"] = {"bound": m2l["bound"], "achieved": m2l["achieved"], "peak": m2l["peak"], "unit": m2l["unit"],
                  "frac": m2l["frac"], "ms": ms["m2l"], "ideal_ms": m2l_ideal}
    ideal = sum(v["ideal_ms"] for v in out.values())
    out["overall"] = {"ideal_ms": ideal, "ms": ms_step, "stages_serialized_ms": ms["total"],
                      "frac": ideal / ms_step if ms_step else 0.0,
                      "peaks": "%s HBM %.0f GB/s, bf16 %.0f TF/s; FP32 and MUFU from %d SMs at %.0f MHz"
                               % (kind, peaks["hbm_gbs"], peaks["bf16_tflops"], sms, f_mhz)}
    return out


def slowest_rank(x, dist, dev):
    """x of the slowest rank (all-reduce MAX over the group; every rank gets
    it); x itself without a group.  dev: the tensor's device for the
    collective (CUDA for NCCL, CPU for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank runs the same workload)."""
    return world * float(units_per_rank) / float(seconds)


def run_ours(args, rank, world, local):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1903_02153_gb300 import bbfmm as bb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    interp = args.interp
    precision = args.precision if interp == "chebyshev" else "fp32"
    c, pts, sig_host = workload(args.workload)
    n, nrhs, depth = c["n"], c["nrhs"], c["depth"]
    plan = make_plan(bb, torch, dev, pts, c, depth, precision, args.svd_eps, interp, args.near)
    sigma = torch.from_numpy(np.ascontiguousarray(sig_host.T)).to(dev)   # (nrhs, n): column-major n x nrhs
    phi = torch.empty_like(sigma)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        bb.bbfmm_matvec(plan.handle, sigma, phi, nrhs, stream)

    # clocks are sampled every 100 ms from the last second of warm-up through
    # the timed steps (the timed region alone can be shorter than a period)
    with ClockSampler(local) as clk:
        t_end = time.perf_counter() + 1.0
        k = 0
        while k < max(args.warmup, 3) or time.perf_counter() < t_end:
            step()
            k += 1
            if k % 16 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        # the launch choices the autotuner made on the first matvec
        info = plan.info()
        tuning = tuning_summary(bb, plan, nrhs)
        # per-stage device times (CUDA events inside the library, on its streams)
        bb.bbfmm_set_timing(plan.handle, True)
        stage = np.zeros(8)
        for _ in range(3):
            flush.fill_(1.0)
            step()
            torch.cuda.synchronize()
            stage += bb.bbfmm_stage_times(plan.handle)
        stage /= 3
        bb.bbfmm_set_timing(plan.handle, False)
        # timed steps
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        t_wall0 = time.perf_counter()
        # an NVTX range around the timed steps, so that a profiler can take
        # exactly these launches (ncu --nvtx --nvtx-include "bench_timed/")
        torch.cuda.nvtx.range_push("bench_timed")
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if dist is not None:
        dist.barrier()
    ms = slowest_rank(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)]), dist, dev)
    status = bb.bbfmm_status(plan.handle)
    # the library's kernels per step: the kernel nodes of the graph the timed steps replayed
    launches = bb.bbfmm_matvec_launches(plan.handle, nrhs)

    # end to end through the C ABI with host buffers (pinned), copies timed
    sig_pin = torch.from_numpy(np.ascontiguousarray(sig_host.T)).pin_memory()
    phi_pin = torch.empty(nrhs, n, dtype=torch.float32).pin_memory()
    for _ in range(3):
        bb.bbfmm_matvec(plan.handle, sig_pin, phi_pin, nrhs, stream)
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bb.bbfmm_matvec(plan.handle, sig_pin, phi_pin, nrhs, stream)   # synchronizes
        e2e.append(time.perf_counter() - t0)
    e2e_s = slowest_rank(np.mean(e2e), dist, dev)

    phi_main = phi_pin.numpy().T.astype(np.float64)
    acc = accuracy_check(pts, sig_host, phi_main, c, nodes=interp) if rank == 0 else None
    extra = {}
    if rank == 0 and not args.no_depth6 and args.workload == "uniform-1M-p5-d5":
        d6, phi6 = time_plan(bb, torch, dev, pts, sigma, c, 6, precision, args.svd_eps, flush, stream,
                             interp=interp, near=args.near)
        d6["accuracy"] = accuracy_check(pts, sig_host, phi6, dict(c, depth=6), nodes=interp)
        d6info = d6.pop("_info")
        # the depth-6 M2L against the same peak (its DRAM traffic while the kernel sources match the capture)
        d6["m2l_roofline"] = roofline(precision, d6info, nrhs, d6["stages_ms"]["m2l"], {"sm_mhz": None}, torch, dev,
                                      "uniform-1M-p5-d6", interp, c["p"])
        extra["depth6"] = d6
    if rank == 0 and precision != "fp32" and not args.no_plain:
        # the plain form: FP32 M2L and the ordered near field, its own
        # accuracy, and how far the mixed form's result is from it
        plain, phi_plain = time_plan(bb, torch, dev, pts, sigma, c, depth, "fp32", args.svd_eps, flush, stream,
                                     near="ordered")
        plain["speedup_of_this_form"] = plain["ms_per_step"] / ms
        plain["accuracy"] = accuracy_check(pts, sig_host, phi_plain, c, nodes=interp)
        plain["rel_diff_mixed_vs_plain"] = float(np.linalg.norm(phi_main - phi_plain) / np.linalg.norm(phi_plain))
        pinfo = plain.pop("_info")
        # (FP32 FMA peak at the maximum SM clock: the timed region's clocks are sampled above)
        plain["m2l_roofline"] = roofline("fp32", pinfo, nrhs, plain["stages_ms"]["m2l"], {"sm_mhz": None},
                                         torch, dev, args.workload)
        extra["plain_fp32_form"] = plain

    clocks = clk.summary()
    m2l_roof = roofline(precision, info, nrhs, float(stage[2]), clocks, torch, dev, args.workload, interp, c["p"])
    N = float(n)
    unit = "N^2/s" if nrhs == 1 else "N^2*nrhs/s"
    out = {
        "metric": METRIC, "value": job_rate(world, N * N * nrhs, ms / 1e3), "unit": unit, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(c), "n": n, "kernel": KERNEL_NAMES[c["kernel"]], "ell": c["ell"],
                   "p": c["p"], "depth": depth, "nrhs": nrhs, "interp": interp, "m2l_precision": precision,
                   "near_field": tuning["near_field"], "tuning": tuning,
                   "close_pairs_fp64": int(info.close_pairs),
                   "svd_rank": info.rank,
                   "svd_eps": args.svd_eps, "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": "replicas"},
        "stages_ms": {k: float(v) for k, v in zip(bb.STAGES, stage)},
        "roofline": m2l_roof,
        "rooflines": stage_rooflines(info, c, nrhs, stage, precision, clocks, torch, dev, m2l_roof, ms)
        if interp == "chebyshev" else None,
        "e2e": {"value": job_rate(world, N * N * nrhs, e2e_s), "unit": unit, "ms": e2e_s * 1e3,
                "h2d_bytes_per_step": 4 * n * nrhs, "d2h_bytes_per_step": 4 * n * nrhs},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "device_status": status,
        "wall_s_timed_region": t_wall,
        "accuracy": acc,
    }
    out.update(extra)
    if rank == 0 and args.serving > 0:
        out["serving"] = serving(args, torch)
    if rank == 0 and not args.no_precision_forms and args.workload == "uniform-1M-p5-d5" and interp == "chebyshev":
        out["precision_forms"] = precision_forms(bb, torch, dev, flush, stream)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pts, sig_host, c)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return out if rank == 0 else None


def accuracy_check(pts, sig, phi, c, nsample=256, ncols=4, nodes="chebyshev"):
    """Sampled targets against the oracle bbFMM (uncompressed M2L, FP64, same
    node set) and exact direct-sum rows, on the first ncols right-hand sides."""
    from oracle import oracle
    idx = np.sort(np.random.default_rng(99).choice(pts.shape[0], nsample, replace=False))
    s64 = sig[:, :ncols].astype(np.float64)
    ref = oracle.bbfmm(pts, s64, c["kernel"], c["p"], c["depth"], ell=c["ell"], lo=W.UNIT_LO, side=W.UNIT_SIDE,
                       sample=idx, nodes=nodes)
    direct = oracle.direct(pts[idx], pts, s64, c["kernel"], c["ell"])
    got = phi[idx, :ncols]
    return {"sample": nsample, "columns": int(min(ncols, sig.shape[1])),
            "rel_err_vs_oracle_fmm": oracle.rel_err(got, ref),
            "oracle_err_vs_direct": oracle.rel_err(ref, direct),
            "gpu_err_vs_direct": oracle.rel_err(got, direct)}


def precision_forms(bb, torch, dev, flush, stream, eps=1e-7, nsample=512):
    """The precision-form workload (2,000,000 clustered points, exp(-r/0.3),
    p = 6, depth 6, one RHS): the M2L in each arithmetic form the library
    has, each timed (L2 flushed) and its error reported against the FP64
    oracle FMM and the direct sum on the same sampled targets."""
    from oracle import oracle
    c, pts, sig = workload("clustered-2M-exp0.3-p6-d6")
    idx = np.sort(np.random.default_rng(98).choice(c["n"], nsample, replace=False))
    s64 = sig[:, 0].astype(np.float64)
    ref = oracle.bbfmm(pts, s64, c["kernel"], c["p"], c["depth"], ell=c["ell"], lo=W.UNIT_LO, side=W.UNIT_SIDE,
                       sample=idx)
    direct = oracle.direct(pts[idx], pts, s64, c["kernel"], c["ell"])
    e_or = oracle.rel_err(ref, direct)
    sig_dev = torch.from_numpy(np.ascontiguousarray(sig.T)).to(dev)
    out = {"workload": describe(c), "svd_eps": eps, "sample": nsample, "oracle_err_vs_direct": e_or, "forms": {}}
    for prec in ("fp32", "tf32", "tf32x3", "bf16x3", "fp16x3"):
        r, phi = time_plan(bb, torch, dev, pts, sig_dev, c, c["depth"], prec, eps, flush, stream, nsteps=5)
        r.pop("_info")
        got = phi[idx, 0]
        e1, e2 = oracle.rel_err(got, ref), oracle.rel_err(got, direct)
        r.update({"rel_err_vs_oracle_fmm": e1, "gpu_err_vs_direct": e2, "gate1": e1 <= 1e-5,
                  "gate2": e2 <= 1.1 * e_or})
        out["forms"][prec] = r
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(pts, sig, c, min_s=10.0, max_runs=8):
    """The FP64 oracle, as it stands, on the host cores: whole matvecs of the
    workload (upward pass, uncompressed M2L on every level, downward pass,
    near field, all targets), repeated until min_s seconds have passed."""
    from oracle import oracle
    s64 = sig.astype(np.float64)
    walls, stages = [], np.zeros(4)
    t_all = time.perf_counter()
    while len(walls) < max_runs and (not walls or time.perf_counter() - t_all < min_s):
        t0 = time.perf_counter()
        _, tm = oracle.bbfmm(pts, s64, c["kernel"], c["p"], c["depth"], ell=c["ell"], lo=W.UNIT_LO,
                             side=W.UNIT_SIDE, times=True)
        walls.append(time.perf_counter() - t0)
        stages += tm
    t = float(np.mean(walls))
    unit = "N^2/s" if c["nrhs"] == 1 else "N^2*nrhs/s"
    return {"value": float(c["n"]) ** 2 * c["nrhs"] / t, "unit": unit, "cores": oracle.num_threads(),
            "nproc": os.cpu_count(), "cpu_model": cpu_model(), "kind": "oracle", "matvec_s": t,
            "stage_s": {k: float(v) / len(walls) for k, v in zip(["upward", "m2l", "downward", "near"], stages)},
            "sample": "%d whole FP64 matvec(s) of the workload (every target, uncompressed M2L), mean wall time"
                      % len(walls)}


def run_reference(args, rank, world):
    """The reference arm is the FP64 oracle: each step one whole matvec of the
    same workload on the host cores (a few seconds on 16 cores)."""
    if rank != 0:
        return None
    c, pts, sig = workload(args.workload)
    per = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(pts, sig, c, min_s=0.0, max_runs=1)
        if k >= args.warmup:
            per.append(r)
    est = float(np.mean([r["matvec_s"] for r in per]))
    value = float(c["n"]) ** 2 * c["nrhs"] / est
    unit = per[0]["unit"]
    return {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": est * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": describe(c), "n": c["n"], "p": c["p"], "depth": c["depth"], "nrhs": c["nrhs"]},
            "cpu_baseline": {"value": value, "unit": unit, "cores": per[0]["cores"], "nproc": per[0]["nproc"],
                             "cpu_model": per[0]["cpu_model"], "kind": "oracle",
                             "sample": "one whole FP64 matvec of the workload per step (every target, "
                                       "uncompressed M2L)"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    out = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world, local)
    if out is not None and rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
