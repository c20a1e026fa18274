"""Benchmark of one black-box FMM matvec (phi = K_hat sigma) on GB300.

Workload (default): N = 1,048,576 points uniform in the unit cube, kernel 1/r,
Chebyshev order p = 5, uniform octree of depth 5, one right-hand side,
sigma ~ U(-1, 1): the N = 1M 1/r configuration, at the depth that is fastest
on this GPU (depth 6 is measured too and reported under "depth6").

A step is one full matvec (gather, P2M/M2M/compress, M2L, L2L/decompress,
L2P, P2P, combine) with inputs resident in HBM.  L2 is flushed between
timed steps by writing a 512 MB buffer (the working set is smaller than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--precision fp32|tf32x3] [--depth D]

Prints one JSON line (rank 0).  With torchrun each rank runs an independent
replica of the same workload (the matvec is single-GPU; replicas only).
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
SM_COUNT_NOMINAL = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None)
    ap.add_argument("--depth", type=int, default=5)
    ap.add_argument("--svd-eps", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-depth6", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

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
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
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
                "samples": len(sm)}


def m2l_flops_per_rhs(info, passes):
    return 2.0 * info.m2l_pairs * info.rank * info.rank * passes


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
    precision = args.precision or "fp16x3"
    name = "uniform-1M-p5-d%d" % args.depth
    c = dict(W.CONFIGS["uniform-1M-p5-d6"], depth=args.depth)
    n, p, depth = c["n"], c["p"], c["depth"]
    pts = W.uniform_points(n)
    sig_host = W.uniform_sigma(n).astype(np.float32)
    plan = bb.Plan(torch.from_numpy(pts).to(dev), c["kernel"], p, depth, precision=precision,
                   svd_eps=args.svd_eps, domain=(W.UNIT_LO, W.UNIT_SIDE))
    info = plan.info()
    sigma = torch.from_numpy(sig_host).to(dev)
    phi = torch.empty_like(sigma)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        bb.bbfmm_matvec(plan.handle, sigma, phi, 1, stream)

    # clocks are sampled (every 100 ms) from the last second of warm-up through
    # the timed steps: the timed region alone is shorter than one sample period
    with ClockSampler(local) as clk:
        t_end = time.perf_counter() + 1.0
        k = 0
        while k < max(args.warmup, 3) or time.perf_counter() < t_end:
            step()
            k += 1
            if k % 16 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()

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
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms = float(np.mean(step_ms))
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the C ABI with host buffers (pinned), copies timed
    sig_pin = torch.from_numpy(sig_host).pin_memory()
    phi_pin = torch.empty(n, dtype=torch.float32).pin_memory()
    for _ in range(3):
        bb.bbfmm_matvec(plan.handle, sig_pin, phi_pin, 1, stream)
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bb.bbfmm_matvec(plan.handle, sig_pin, phi_pin, 1, stream)   # synchronizes
        e2e.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e))

    # accuracy of this run against the oracle on sampled targets
    acc = None
    if rank == 0:
        acc = accuracy_check(pts, sig_host, phi_pin.numpy().astype(np.float64), c)

    depth6 = None
    if rank == 0 and not args.no_depth6 and args.depth != 6:
        depth6 = other_depth(bb, torch, dev, pts, sigma, c, 6, precision, flush, stream, args.svd_eps)
    # the plain FP32 GPU form (M2L on the CUDA cores) on the same workload
    plain = None
    if rank == 0 and precision != "fp32":
        plain = other_depth(bb, torch, dev, pts, sigma, c, args.depth, "fp32", flush, stream, args.svd_eps)
        plain["speedup_of_this_form"] = plain["ms_per_step"] / ms

    peaks, peak_kind = measured_peaks()
    clocks = clk.summary()
    N = float(n)
    value = world * N * N / (ms / 1e3)
    passes = {"fp32": 1, "tf32": 1, "tf32x3": 3, "bf16x3": 3, "fp16x3": 3}[precision]
    m2l_ms = float(stage[2])
    p2p_ms = float(stage[5])
    m2l_fl = m2l_flops_per_rhs(info, passes)
    if precision == "fp32":
        f_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        props = torch.cuda.get_device_properties(dev)
        peak = props.multi_processor_count * 128 * 2 * f_mhz * 1e6 / 1e12
        roof = {"kernel": "k_m2l_fp32 (all levels)", "bound": "alu", "achieved": m2l_fl / (m2l_ms / 1e3) / 1e12,
                "peak": peak, "unit": "TFLOP/s",
                "peak_source": "FP32 FMA: %d SMs x 128 lanes x 2 flop x median SM clock %.0f MHz"
                               % (props.multi_processor_count, f_mhz),
                "traffic": None}
    elif precision in ("tf32", "tf32x3"):
        tf32 = peaks["bf16_tflops"] * (1.1 / 2.25)
        roof = {"kernel": "k_m2l_tc (all levels)", "bound": "tensor",
                "achieved": m2l_fl / (m2l_ms / 1e3) / 1e12, "peak": tf32, "unit": "TFLOP/s",
                "peak_source": "%s bf16 %.0f TF/s x nominal tf32/bf16 ratio 1.1/2.25" % (peak_kind,
                                                                                     peaks["bf16_tflops"]),
                "traffic": None}
    else:   # FP16 / BF16 operands run at the 16-bit dense rate
        roof = {"kernel": "k_m2l_tc (all levels)", "bound": "tensor",
                "achieved": m2l_fl / (m2l_ms / 1e3) / 1e12, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                "peak_source": "%s bf16 dense %.0f TF/s (fp16 runs at the same rate)" % (peak_kind,
                                                                                      peaks["bf16_tflops"]),
                "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # gather, P2P, P2M, M2M, compress, M2L (one launch on the tensor cores,
    # one per level in FP32), L2L, decompress, L2P, combine
    m2l_launches = depth - 1 if precision == "fp32" else 1
    launches_per_step = 2 + 1 + (depth - 2) + (depth - 1) + m2l_launches + (depth - 2) + (depth - 1) + 1 + 1
    out = {
        "metric": METRIC, "value": value, "unit": "N^2/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s: N=%d uniform unit cube, 1/r, p=%d, depth %d, 1 RHS, sigma~U(-1,1)"
                               % (name, n, p, depth), "n": n, "kernel": "1/r", "p": p, "depth": depth,
                   "nrhs": 1, "m2l_precision": precision, "svd_rank": info.rank, "svd_eps": args.svd_eps,
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": "replicas"},
        "stages_ms": {k: float(v) for k, v in zip(bb.STAGES, stage)},
        "roofline": roof,
        "e2e": {"value": world * N * N / e2e_s, "unit": "N^2/s", "ms": e2e_s * 1e3,
                "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
        "accuracy": acc,
    }
    if depth6 is not None:
        out["depth6"] = depth6
    if plain is not None:
        out["plain_fp32_form"] = plain
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pts, sig_host, c)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return out if rank == 0 else None


def other_depth(bb, torch, dev, pts, sigma, c, depth, precision, flush, stream, eps):
    """Mean device time of 5 matvecs of another configuration (L2 flushed)."""
    plan = bb.Plan(torch.from_numpy(pts).to(dev), c["kernel"], c["p"], depth, precision=precision,
                   svd_eps=eps, domain=(W.UNIT_LO, W.UNIT_SIDE))
    phi = torch.empty_like(sigma)
    for _ in range(3):
        bb.bbfmm_matvec(plan.handle, sigma, phi, 1, stream)
    ts = []
    for k in range(5):
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bb.bbfmm_matvec(plan.handle, sigma, phi, 1, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    plan.close()
    ms = float(np.mean(ts))
    return {"depth": depth, "m2l_precision": precision, "ms_per_step": ms,
            "value": float(c["n"]) ** 2 / (ms / 1e3)}


def accuracy_check(pts, sig, phi, c, nsample=256):
    from oracle import oracle
    idx = np.sort(np.random.default_rng(99).choice(pts.shape[0], nsample, replace=False))
    s64 = sig.astype(np.float64)
    ref = oracle.bbfmm(pts, s64, c["kernel"], c["p"], c["depth"], lo=W.UNIT_LO, side=W.UNIT_SIDE,
                       sample=idx)
    direct = oracle.direct(pts[idx], pts, s64, c["kernel"])
    return {"sample": nsample, "rel_err_vs_oracle_fmm": oracle.rel_err(phi[idx], ref),
            "oracle_err_vs_direct": oracle.rel_err(ref, direct),
            "gpu_err_vs_direct": oracle.rel_err(phi[idx], direct)}


def cpu_baseline(pts, sig, c, target_s=15.0):
    """The FP64 oracle, as it stands, on the host cores: the full upward pass
    plus the far field, downward pass and near field for a sample of target
    leaves, extrapolated to all leaves by the sampled fraction."""
    from oracle import oracle
    n = pts.shape[0]
    s64 = sig.astype(np.float64)
    rng = np.random.default_rng(7)
    nsample = 64
    while True:
        idx = np.sort(rng.choice(n, nsample, replace=False))
        t0 = time.perf_counter()
        _, tm = oracle.bbfmm(pts, s64, c["kernel"], c["p"], c["depth"], lo=W.UNIT_LO, side=W.UNIT_SIDE,
                             sample=idx, times=True)
        wall = time.perf_counter() - t0
        if wall > target_s / 4 or nsample >= 8192:
            break
        nsample *= 4
    # leaves touched by the sample
    cells = oracle.leaf_cells(pts[idx], W.UNIT_LO, W.UNIT_SIDE, c["depth"])
    nleaf_s = len({tuple(v) for v in cells})
    nleaf = 8 ** c["depth"]
    t_full = tm[0] + (tm[1] + tm[2] + tm[3]) * (nleaf / nleaf_s)
    return {"value": float(n) ** 2 / t_full, "unit": "N^2/s", "cores": oracle.num_threads(),
            "kind": "oracle", "est_matvec_s": t_full,
            "sample": "full upward pass + far/downward/near field for %d random targets in %d of %d leaves "
                      "(%.1f s measured), extrapolated by leaf fraction" % (nsample, nleaf_s, nleaf, wall)}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step a bounded sample of the same
    workload on the host cores."""
    if rank != 0:
        return None
    c = dict(W.CONFIGS["uniform-1M-p5-d6"], depth=args.depth)
    n = c["n"]
    pts = W.uniform_points(n)
    sig = W.uniform_sigma(n).astype(np.float32)
    per = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(pts, sig, c, target_s=4.0)
        if k >= args.warmup:
            per.append(r)
    est = float(np.mean([r["est_matvec_s"] for r in per]))
    value = float(n) ** 2 / est
    return {"metric": METRIC, "value": value, "unit": "N^2/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": est * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "uniform-1M-p5-d%d: N=%d uniform unit cube, 1/r, p=5, depth %d, 1 RHS"
                                   % (args.depth, n, args.depth), "n": n, "p": 5, "depth": args.depth},
            "cpu_baseline": {"value": value, "unit": "N^2/s", "cores": per[0]["cores"], "kind": "oracle",
                             "sample": per[0]["sample"]},
            "e2e": {"value": value, "unit": "N^2/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if out is not None and rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
