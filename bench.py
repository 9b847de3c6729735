"""Benchmark of the QIHT hot path on one GB300 (or N replicas under torchrun).

Workload (the large single solve): Gaussian Phi 8192 x 32768 with entries
N(0, 1/m), x with s = 256 nonzeros +-U(0.5, 1.5), y = Phi x + noise at 30 dB,
Phi and y quantized to b bits (default 8), 300 QIHT iterations.

One step = the whole hot path on one input: max |Phi|, max |y|, three stochastic
quantizations (Q1, Q2 of Phi, Q(y)) and the 300-iteration solve (one CUDA graph).
value   = iterations per second over the timed steps (inputs resident in HBM).
e2e     = the same metric with Phi and y copied from pinned host memory and x,
          the support and the report copied back, inside the timed region.
roofline: the gradient kernel g = Q1^T r (one pass over the codes of Q1), timed
          alone with CUDA events on its stream with the solver's launch plan;
          algorithmic bytes = m n b / 8 + 4 m + 4 n per launch.
cpu_baseline / --impl reference: the CPU oracle (plain FP64 C, OpenMP over the
          host cores) on one bounded sample (the first 2048 rows of the same matrix,
          200 iterations), extrapolated to the full step.

Under torchrun with N > 1 ranks, every rank solves its own independent instance
(replicas; no collective in the data path) and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

M, N, S, ITERS = 8192, 32768, 256, 300
METRIC = "NIHT iterations/s"
UNIT = "iterations/s"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gemv_t_traffic.txt")
# iterations per execution of the solver graph's loop body (the library's default)
BODY_UNROLL = int(os.environ.get("QIHT_UNROLL", "8"))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--bits", type=int, default=8)
    ap.add_argument("--bits-y", type=int, default=None, help="width of the observation's codes (default: --bits)")
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--m", type=int, default=M)
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--s", type=int, default=S)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-widths", action="store_true", help="skip the gradient kernel at the other code widths")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched measurements (many right-hand sides; many problems) of the default line")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the brief runs of the other workloads (interferometry, MRI operator form, Phi on the "
                         "fly, fresh realizations, unrolled) in the default line")
    ap.add_argument("--gemv-launches", type=int, default=200)
    ap.add_argument("--workload", choices=["single", "interferometry", "mri", "batched", "multi", "fresh", "unrolled", "fly",
                                           "mri_op"],
                    default="single",
                    help="single: the large single solve (default); batched: 512 independent problems in one "
                         "launch; multi: 1024 right-hand sides sharing the large matrix (tensor-core gradient)")
    ap.add_argument("--nprob", type=int, default=512)
    ap.add_argument("--nrhs", type=int, default=1024)
    ap.add_argument("--plain-sample", type=int, default=16)
    ap.add_argument("--bits-factor", type=int, default=12, help="mri_op: bits of the quantized transform factor")
    ap.add_argument("--mri-grid", type=int, default=128,
                    help="mri_op: image side N (128, or the paper's 512, where s = 4096 and no dense matrix is formed)")
    ap.add_argument("--fp8", action="store_true",
                    help="multi: the FP8 (e4m3) gradient product, residual as three e4m3 terms (2- and 4-bit codes)")
    ap.add_argument("--eager", action="store_true",
                    help="launch the solver's kernels one by one instead of one graph (for kernel profilers, "
                         "which do not see the kernels of graphs with conditional nodes)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def config(args, world):
    if args.workload == "mri":
        return {"workload": f"MRI-shaped single solve: radial k-space samples (a third of a 128x128 grid) of the "
                            f"orthonormal 2D DFT of a 2D Haar synthesis, stacked real {args.m}x{args.n}, synthetic "
                            f"head image with its s={args.s} largest Haar coefficients, 30 dB, Phi quantized to "
                            f"{args.bits} bits, y to {args.bits_y or args.bits} bits, {args.iters} iterations",
                "m": args.m, "n": args.n, "s": args.s, "bits_phi": args.bits, "bits_y": args.bits_y or args.bits,
                "iters_per_step": args.iters, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                "l2": "Q1 codes %.0f MiB per iteration; L2 flushed between timed steps by the quantization "
                      "of Phi (%.0f MiB of FP32 read)" % (args.m * args.n * args.bits / 8 / 2**20,
                                                          args.m * args.n * 4 / 2**20),
                "step": "max|Phi|, max|y|, quantize Q1, Q2, Q(y), one solve (one graph launch)"}
    if args.workload == "interferometry":
        return {"workload": f"interferometry-shaped single solve: 48 antennas uniform in a 1 km disk, "
                            f"Phi_kp = exp(-2 pi i (u_k l_p + v_k m_p)) over 2256 baselines x 128x128 pixels, "
                            f"stacked real {args.m}x{args.n}, 50 log-normal point sources, 20 dB, s={args.s}, "
                            f"Phi quantized to {args.bits} bits, y to {args.bits_y or args.bits} bits, {args.iters} iterations",
                "m": args.m, "n": args.n, "s": args.s, "bits_phi": args.bits, "bits_y": args.bits_y or args.bits,
                "iters_per_step": args.iters, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                "l2": "Q1 codes %.0f MiB per iteration; L2 flushed between timed steps by the quantization "
                      "of Phi (%.0f MiB of FP32 read)" % (args.m * args.n * args.bits / 8 / 2**20,
                                                          args.m * args.n * 4 / 2**20),
                "step": "max|Phi|, max|y|, quantize Q1, Q2, Q(y), one solve (one graph launch)"}
    return {"workload": f"large single solve: Gaussian Phi {args.m}x{args.n} N(0,1/m), s={args.s}, "
                        f"x=+-U(0.5,1.5), 30 dB, Phi quantized to {args.bits} bits, y to {args.bits_y or args.bits} bits, "
                        f"{args.iters} iterations",
            "m": args.m, "n": args.n, "s": args.s, "bits_phi": args.bits, "bits_y": args.bits_y or args.bits,
            "iters_per_step": args.iters, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2: Q1 codes %.0f MiB streamed every iteration" %
                  (args.m * args.n * args.bits / 8 / 2**20),
            "step": "max|Phi|, max|y|, quantize Q1, Q2, Q(y), 300-iteration solve (one graph launch)"}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
SAMPLE_ROWS, SAMPLE_ITERS = 2048, 200


def cpu_model() -> str:
    """The host CPU's model name (x86 'model name', or the Arm implementer/part pair)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(p, bits, iters_total, rows=SAMPLE_ROWS, iters=SAMPLE_ITERS, threads=None):
    """The CPU oracle (FP64 C, OpenMP over the host cores) on a bounded sample of the workload:
    the first `rows` rows (same n, s), its three quantizations and `iters` iterations. The
    quantization and the per-iteration work scale linearly with m, so the step time of the full
    problem is estimated as (m / rows) x (quantize time + iters_total x per-iteration time).
    Both CPU figures of the bench (the reference arm and the cpu_baseline of our line) use this
    one sample definition."""
    import oracle
    nproc = os.cpu_count() or 1
    oracle.set_threads(threads or nproc)
    used = oracle.get_threads()
    sub_phi = np.ascontiguousarray(p.phi[:rows])
    sub_y = np.ascontiguousarray(p.y[:rows])
    t0 = time.perf_counter()
    c1, sphi = oracle.quantize(sub_phi, bits, 0, 0)
    c2, _ = oracle.quantize(sub_phi, bits, 0, 1, sphi)
    cy, sy = oracle.quantize(sub_y, bits, 0, 2)
    A1 = oracle.dequantize(c1, bits, sphi)
    A2 = oracle.dequantize(c2, bits, sphi)
    yq = oracle.dequantize(cy, bits, sy)
    t1 = time.perf_counter()
    oracle.niht(A1, A2, yq, p.s, iters)
    t2 = time.perf_counter()
    scale = p.m / rows
    t_quant = (t1 - t0) * scale
    t_iter = (t2 - t1) / iters * scale
    step = t_quant + iters_total * t_iter
    return {"value": iters_total / step, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"first {rows} of {p.m} rows (n={p.n}, s={p.s}): quantize Q1,Q2,Q(y) + {iters} "
                      f"iterations, FP64 C with OpenMP on {used} threads; the full step's time is extrapolated "
                      f"from the sample by m/{rows} = {scale:g}",
            "extrapolated": True, "nproc": nproc, "cpu_model": cpu_model(),
            "sample_seconds": round(t2 - t0, 3), "est_step_seconds": round(step, 3)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    p = synth.large_noisy(seed=0, m=args.m, n=args.n, s=args.s)
    for _ in range(args.warmup):
        oracle_sample(p, args.bits, args.iters, rows=256, iters=2)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = oracle_sample(p, args.bits, args.iters)
        vals.append(last["est_step_seconds"])
    wall = time.perf_counter() - t0
    step = statistics.mean(vals)
    value = args.iters / step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"], "extrapolated": True, "nproc": last["nproc"],
                             "cpu_model": last["cpu_model"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "each step times the bounded sample (not the full problem); ms_per_step is the full "
                    "step's time extrapolated from it",
            "wall_seconds": round(wall, 2)}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"qiht_clocks_{os.getpid()}.csv")
        self.uuid = uuid

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def start_clocks(dev):
    """nvidia-smi clock sampling of this GPU, started before a timed region."""
    import torch
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = Clocks(uuid)
    clk.start()
    time.sleep(0.3)
    return clk


def traffic_for_kernel(bits, m, n):
    """DRAM bytes per launch of the gradient kernel from the committed ncu summary
    (profiles/gemv_t_traffic.txt), only while the kernel source is unchanged since
    the capture and for the captured shape."""
    try:
        d = {}
        for line in open(TRAFFIC_FILE):
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                d[k] = v
        src = open(os.path.join(ROOT, "paper_1802_04907_gb300", "csrc", "gemv.cu"), "rb").read()
        if d.get("gemv_cu_sha1") != hashlib.sha1(src).hexdigest():
            return None
        v = d.get(f"bits{bits}_m{m}_n{n}")
        return int(v) if v is not None else None
    except Exception:
        return None


def replica_throughput(ms_local: float, units_local: float, reduce_max, reduce_sum):
    """Whole-job throughput of independent replicas (one per rank, no collective in the data
    path): the units every rank processed, summed, over the slowest rank's time. reduce_max /
    reduce_sum combine a float over the ranks (identity on one rank)."""
    ms_max = reduce_max(ms_local)
    units = reduce_sum(units_local)
    return units / (ms_max / 1e3), ms_max


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1802_04907_gb300 as q

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    if args.workload == "interferometry":
        p = synth.interferometry(seed=rank)
        args.m, args.n, args.s = p.phi.shape[0], p.phi.shape[1], p.s
    elif args.workload == "mri":
        p = synth.mri(seed=rank)
        args.m, args.n, args.s = p.phi.shape[0], p.phi.shape[1], p.s
    else:
        p = synth.large_noisy(seed=rank, m=args.m, n=args.n, s=args.s)
    phi_h = torch.from_numpy(p.phi).pin_memory()
    y_h = torch.from_numpy(p.y).pin_memory()
    phi = phi_h.to(dev)
    y = y_h.to(dev)
    bits = args.bits
    bits_y = args.bits_y or bits
    codes = q.quantize_problem(phi, y, bits, bits_y, seed=rank)
    solver = q.Solver(args.m, args.n, args.s, args.iters, device=dev, eager=args.eager)

    def step():
        q.quantize_problem(phi, y, bits, bits_y, seed=rank, out=codes)
        solver(*codes)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    rep0 = solver.read_report()
    assert rep0.status == q.OK, rep0

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = Clocks(uuid)
    clk.start()
    time.sleep(0.3)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.stop()
    rep = solver.read_report()
    iters_done = rep.iters_run
    xg = solver.x.double().cpu().numpy()
    rel_err = float(np.linalg.norm(xg - p.x_true) / np.linalg.norm(p.x_true))

    def reduce_with(op):
        def f(v):
            t = torch.tensor([v], dtype=torch.float64, device=dev)
            if world > 1:
                dist.all_reduce(t, op=op)
            return float(t.item())
        return f

    value, ms_max = replica_throughput(ms, args.steps * iters_done, reduce_with(dist.ReduceOp.MAX),
                                       reduce_with(dist.ReduceOp.SUM))

    # solve only (quantization excluded), same buffers
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        solver(*codes)
    ev1.record(stream)
    barrier()
    solve_ms = ev0.elapsed_time(ev1) / args.steps

    # gradient kernel alone: average launch duration with CUDA events on its stream
    q1 = codes[0]
    r = (torch.randn(args.m, device=dev) * 0.01).float()
    rmax = r.abs().max().reshape(1).contiguous()
    g = torch.empty(args.n, dtype=torch.float32, device=dev)
    for _ in range(5):
        q.gemv_t_prescaled(q1, r, rmax, g, stream=stream)
    barrier()
    nl = args.gemv_launches
    ev0.record(stream)
    for _ in range(nl):
        q.gemv_t_prescaled(q1, r, rmax, g, stream=stream)
    ev1.record(stream)
    barrier()
    gemv_ms = ev0.elapsed_time(ev1) / nl
    alg_bytes = args.m * args.n * bits / 8 + 4 * args.m + 4 * args.n
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (gemv_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_for_kernel(bits, args.m, args.n), "kernel": "k_gemv_t (g = Q1^T r)",
                "avg_launch_us": gemv_ms * 1e3, "algorithmic_bytes_per_launch": alg_bytes,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                else "fallback 6.8 TB/s"}
    # the same gradient kernel at the other code widths of the workload (b in {2, 4, 8}): the
    # codes of the same Phi quantized to b bits, timed alone the same way
    by_bits = {}
    if args.workload == "single" and not args.no_widths:
        for b in (8, 4, 2):
            if b == bits:
                by_bits[str(b)] = {k: roofline[k] for k in ("achieved", "frac", "avg_launch_us",
                                                             "algorithmic_bytes_per_launch", "traffic")}
                continue
            qb, _ = q.quantize_pair(phi, b, 11, q.STREAM_Q1, q.STREAM_Q2)
            for _ in range(5):
                q.gemv_t_prescaled(qb, r, rmax, g, stream=stream)
            barrier()
            ev0.record(stream)
            for _ in range(nl):
                q.gemv_t_prescaled(qb, r, rmax, g, stream=stream)
            ev1.record(stream)
            barrier()
            ms_b = ev0.elapsed_time(ev1) / nl
            alg_b = args.m * args.n * b / 8 + 4 * args.m + 4 * args.n
            ach_b = alg_b / (ms_b / 1e3) / 1e9
            by_bits[str(b)] = {"achieved": ach_b, "frac": ach_b / peak, "avg_launch_us": ms_b * 1e3,
                               "algorithmic_bytes_per_launch": alg_b, "traffic": traffic_for_kernel(b, args.m, args.n)}
            del qb
        roofline["by_bits"] = by_bits
    if args.m * args.n * bits / 8 < 100 * 2**20:
        roofline["note"] = ("the Q1 codes (%.0f MiB) fit in the 129 MB L2: repeated gradient launches read them "
                            "mostly from L2, so the fraction of the HBM peak can exceed 1"
                            % (args.m * args.n * bits / 8 / 2**20))

    # end to end: host buffers in, host results out, through the public API. Every step
    # copies its Phi and y from pinned host memory and reads x, the support and the report
    # back; the inputs are double-buffered on the device, so the copy of step k+1 (on a
    # copy stream) overlaps the quantization and solve of step k.
    e2e = None
    if not args.no_e2e:
        x_h = torch.empty(args.n, dtype=torch.float32).pin_memory()
        sup_h = torch.empty(args.s, dtype=torch.int32).pin_memory()
        rep_h = torch.empty(q.REPORT_BYTES, dtype=torch.uint8).pin_memory()
        slots = [(phi, y), (torch.empty_like(phi), torch.empty_like(y))]
        copy_stream = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        consumed = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_run(k_steps):
            with torch.cuda.stream(copy_stream):
                slots[0][0].copy_(phi_h, non_blocking=True)
                slots[0][1].copy_(y_h, non_blocking=True)
                copied[0].record(copy_stream)
            for k in range(k_steps):
                a, b = k % 2, (k + 1) % 2
                if k + 1 < k_steps:
                    with torch.cuda.stream(copy_stream):
                        if k >= 1:
                            copy_stream.wait_event(consumed[b])
                        slots[b][0].copy_(phi_h, non_blocking=True)
                        slots[b][1].copy_(y_h, non_blocking=True)
                        copied[b].record(copy_stream)
                stream.wait_event(copied[a])
                q.quantize_problem(slots[a][0], slots[a][1], bits, bits_y, seed=rank, out=codes)
                consumed[a].record(stream)
                solver(*codes)
                x_h.copy_(solver.x, non_blocking=True)
                sup_h.copy_(solver.support, non_blocking=True)
                rep_h.copy_(solver.report, non_blocking=True)

        e2e_run(2)
        barrier()
        ev0.record(stream)
        e2e_run(args.steps)
        ev1.record(stream)
        barrier()
        e_ms = ev0.elapsed_time(ev1)
        te = torch.tensor([e_ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * args.steps * iters_done / (float(te.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(p.phi.nbytes + p.y.nbytes),
               "d2h_bytes_per_step": int(4 * args.n + 4 * args.s + q.REPORT_BYTES),
               "pipelining": "inputs double-buffered: the copy of step k+1 overlaps step k"}

    # kernels launched per step: 2 max-abs + 3 quantize, 3 in the solver's set-up, then per
    # iteration the persistent iteration kernel and the gradient kernel (shrinks stay inside);
    # the graph runs its loop body (BODY_UNROLL iterations) whole, the kernels after the
    # last iteration return at once
    unroll = 1 if args.eager else BODY_UNROLL
    launches_per_step = 5 + 3 + 2 * unroll * -(-iters_done // unroll)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the bounded sample that the reference arm times too: 200 iterations on the first
        # 2048 rows, on all host cores
        cpu = oracle_sample(p, bits, args.iters, rows=min(SAMPLE_ROWS, p.m))
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "extrapolated", "nproc",
                                   "cpu_model")}

    # the metric's second half: batched vs plain solves/s at equal error, measured in this run
    batched = None
    if rank == 0 and world == 1 and args.workload == "single" and not args.no_batched:
        del phi_h, y_h
        batched = batched_summary(args)
    others = None
    if rank == 0 and world == 1 and args.workload == "single" and not args.no_others:
        others = others_summary(args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": f"u{bits}", "data": "synthetic",
                "config": config(args, world), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": args.steps * launches_per_step,
                "solve_only": {"ms_per_solve": solve_ms, "iters_per_s": iters_done / (solve_ms / 1e3),
                               "us_per_iter": solve_ms * 1e3 / max(iters_done, 1)},
                "arith": "codes x 24-bit fixed-point residual via dp4a, exact int accumulation; FP32 vectors; "
                         "FP64 step size and norms",
                "rel_err_x": rel_err,
                "report": {"iters_run": rep.iters_run, "backtracks": rep.backtracks,
                           "support_changes": rep.support_changes, "resid_norm2": rep.resid_norm2,
                           "full_selects": rep.full_selects,
                           "iteration_phases_us": [round(v, 2) for v in rep.phase_us[:7]]},
                "driver": "eager launches" if args.eager else "one CUDA graph per solve"}
        if batched is not None:
            line["batched"] = batched
        if others is not None:
            line["other_workloads"] = others
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched workload: many independent problems of uneven size in one launch
# ---------------------------------------------------------------------------
def batched_summary(args):
    """Both batched workloads for the default line (the many-right-hand-side solve one timed launch
    after one warm-up, the many-problem launch three after three):
    many right-hand sides sharing the large Phi (1024 x s=256, 8-bit, 300 iterations; the
    gradients as one tensor-core product) and many independent problems of uneven size (512,
    4-bit, 100 iterations, one persistent launch), each against plain single solves at equal
    error."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup = 1, 1
    a.m, a.n, a.s, a.bits, a.iters = M, N, S, 8, ITERS
    t0 = time.perf_counter()
    mu = run_multi(a, emit=False)
    t1 = time.perf_counter()
    b = copy.copy(a)
    b.steps, b.warmup = 3, 3                          # ~65 ms a launch: steady state for a few tenths of a second
    ba = run_batched(b, emit=False)
    t2 = time.perf_counter()
    keep_m = ("value", "unit", "ms_per_step", "plain", "speedup_vs_plain", "equal_error", "roofline", "clocks",
              "statuses", "config")
    keep_b = ("value", "unit", "ms_per_step", "plain", "speedup_vs_plain", "equal_error", "roofline", "clocks",
              "statuses", "config")
    return {"multi_rhs": {**{k: mu[k] for k in keep_m if k in mu}, "wall_s": round(t1 - t0, 1)},
            "many_problems": {**{k: ba[k] for k in keep_b if k in ba}, "wall_s": round(t2 - t1, 1)}}


def quick_solves(p, bits_phi, bits_y, iters, steps, dev):
    """it/s of qiht_niht_solve (cached graph) on problem p, CUDA events over `steps` solves after a
    warm-up one, with the relative error of x against the truth and the product timed alone."""
    import torch

    import paper_1802_04907_gb300 as q

    phi = torch.from_numpy(p.phi).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    q1, q2, qy = q.quantize_problem(phi, y, bits_phi, bits_y, 5)
    sv = q.Solver(p.m, p.n, p.s, iters, device=dev)
    sv(q1, q2, qy)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        sv(q1, q2, qy)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    rep = sv.read_report()
    xt = torch.from_numpy(p.x_true).to(dev, torch.float32)
    err = float(torch.linalg.norm(sv.x - xt) / torch.linalg.norm(xt))
    r = torch.randn(p.m, device=dev)
    rmax = r.abs().max().reshape(1)
    g = torch.empty(p.n, device=dev)
    for _ in range(5):
        q.gemv_t_prescaled(q1, r, rmax, g)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(100):
        q.gemv_t_prescaled(q1, r, rmax, g)
    ev1.record()
    torch.cuda.synchronize()
    us = ev0.elapsed_time(ev1) / 100 * 1e3
    del phi, y, q1, q2, qy
    return {"iterations_per_s": rep.iters_run / (ms / 1e3), "ms_per_solve": ms, "rel_err": err,
            "backtracks": rep.backtracks, "gemv_t_us": us}


def others_summary(args):
    """The other workloads, briefly, for the default line (so that a run of the default bench
    records them): the interferometry-shaped solve at 8/8 and 2/8 bits, the MRI operator form
    (with the dense 8-bit composite beside it), Phi on the fly, fresh realizations of the large
    matrix, and the unrolled forward + adjoint."""
    import copy

    import torch

    import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    t0 = time.perf_counter()
    p = synth.interferometry(seed=0)
    intf = {}
    for bp, by in ((8, 8), (2, 8)):
        r = quick_solves(p, bp, by, ITERS, 3, dev)
        by_ = p.m * p.n * bp / 8 + 4 * p.m + 4 * p.n
        r["gemv_t_hbm_frac"] = by_ / (r["gemv_t_us"] * 1e-6) / 1e9 / hbm
        intf[f"{bp}/{by}"] = r
    out["interferometry_4512x16384_s64_300it"] = {**intf, "wall_s": round(time.perf_counter() - t0, 1)}
    del p
    keep = ("value", "unit", "ms_per_step", "ms_per_iteration", "rel_err", "status", "config")
    for name, fn, extra in (("mri_operator_form", run_mri_op, ("dense_8bit_composite", "operator_application_us")),
                            ("phi_on_the_fly", run_fly, ("stored_fp32_phi", "gradient_product")),
                            ("fresh_realizations", run_fresh, ("fixed_quantizations",)),
                            ("unrolled_forward_adjoint", run_unrolled, ())):
        a = copy.copy(args)
        a.steps, a.warmup, a.iters = 3, 3, ITERS
        a.bits, a.bits_y = 8, None
        a.m, a.n, a.s = M, N, S
        t0 = time.perf_counter()
        ln = fn(a, emit=False)
        torch.cuda.empty_cache()
        rf = ln.get("roofline") or {}
        out[name] = {**{k: ln[k] for k in keep + extra if k in ln},
                     "roofline": {k: rf[k] for k in ("bound", "frac", "avg_launch_us", "kernel") if k in rf},
                     "wall_s": round(time.perf_counter() - t0, 1)}
    return out


def run_batched(args, emit=True):
    """512 Gaussian problems, m ~ U[128, 2048], n = 4m, s ~ U[8, 128], x with N(0,1) nonzeros,
    noiseless, 4-bit Phi and y, 100 iterations each, generated on the device from seeds.
    value = solves/s of one qiht_niht_solve_batched launch; the same problems solved one by one
    with qiht_niht_solve (cached graphs) give the plain rate; both median recovery errors are
    reported (equal error)."""
    import torch

    import paper_1802_04907_gb300 as q

    dev = torch.device("cuda", torch.cuda.current_device())
    bits, iters, nprob = 4, 100, args.nprob
    rng = np.random.Generator(np.random.PCG64(2024))
    gen = torch.Generator(device=dev)
    probs, truths = [], []
    total_codes = 0
    for i in range(nprob):
        m = int(rng.integers(128, 2049))
        n = 4 * m
        s = int(rng.integers(8, 129))
        gen.manual_seed(1_000_003 * i + 17)
        phi = torch.randn(m, n, generator=gen, device=dev, dtype=torch.float32) / float(np.sqrt(m))
        sup = torch.randperm(n, generator=gen, device=dev)[:s]
        x = torch.zeros(n, device=dev, dtype=torch.float32)
        x[sup] = torch.randn(s, generator=gen, device=dev, dtype=torch.float32)
        y = (phi.double() @ x.double()).float()
        q1, q2, qy = q.quantize_problem(phi, y, bits, bits, seed=i)
        del phi
        probs.append((q1, q2, qy, s))
        truths.append(x)
        total_codes += q1.nbytes
    torch.cuda.synchronize()

    def rel_err(xs):
        e = [float(torch.linalg.norm(xs[i] - truths[i]) / torch.linalg.norm(truths[i])) for i in range(nprob)]
        return float(np.median(e))

    for _ in range(max(1, args.warmup)):
        res = q.niht_solve_batched(probs, iters)
    torch.cuda.synchronize()
    clk = start_clocks(torch.device("cuda", torch.cuda.current_device()))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        res = q.niht_solve_batched(probs, iters)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = clk.stop()
    reps = res.all_reports()
    it_done = sum(r.iters_run for r in reps)
    err_b = rel_err(res.x)
    # plain: one qiht_niht_solve per problem (graphs cached by the first pass)
    solvers = [q.Solver(pr[0].rows, pr[0].cols, pr[3], iters, device=dev) for pr in probs]
    for sv, pr in zip(solvers, probs):
        sv(*pr[:3])
    torch.cuda.synchronize()
    ev0.record()
    for sv, pr in zip(solvers, probs):
        sv(*pr[:3])
    ev1.record()
    torch.cuda.synchronize()
    ms_plain = ev0.elapsed_time(ev1)
    err_p = rel_err([sv.x for sv in solvers])
    peak, peak_kind = load_peaks()
    # algorithmic bytes: every iteration streams Q1 once (plus the support columns of Q2)
    alg = sum(it * pr[0].nbytes for it, pr in zip([r.iters_run for r in reps], probs))
    achieved = alg / (ms / 1e3) / 1e9
    line = {"metric": "batched solves/s", "value": nprob / (ms / 1e3), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u4", "data": "synthetic",
            "config": {"workload": f"{nprob} independent Gaussian problems, m~U[128,2048], n=4m, s~U[8,128], "
                                   f"N(0,1) nonzeros, noiseless, 4-bit, {iters} iterations each",
                       "codes_bytes_per_iteration": int(total_codes)},
            "iterations_per_s": it_done / (ms / 1e3),
            "plain": {"solves_per_s": nprob / (ms_plain / 1e3), "ms": ms_plain,
                      "how": "qiht_niht_solve per problem, graphs cached"},
            "speedup_vs_plain": ms_plain / ms,
            "equal_error": {"batched_median_rel_err": err_b, "plain_median_rel_err": err_p},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "note": "Q1 code bytes streamed per iteration over the launch time"},
            "statuses": {str(k): sum(1 for r in reps if r.status == k) for k in sorted({r.status for r in reps})}}
    line["clocks"] = clocks
    if emit:
        print(json.dumps(line))
    return line


def run_multi(args, emit=True):
    """nrhs right-hand sides sharing the large Gaussian matrix (8192 x 32768, N(0, 1/m)), each
    x_k with s = 256 N(0,1) nonzeros at a uniform support, y_k = Phi x_k + noise at 30 dB, Phi
    and y_k quantized to 8 bits, 300 iterations each; inputs generated on the device from seeds.
    value = solves/s of qiht_niht_solve_multi; a sample of the right-hand sides solved one by one
    with qiht_niht_solve gives the plain rate; median recovery errors of both are reported (equal
    error). The roofline is the tensor-core gradient product timed alone (residual split + GEMM)
    against the measured dense bf16 rate (f16 and bf16 run at the same rate)."""
    import torch

    import paper_1802_04907_gb300 as q

    dev = torch.device("cuda", torch.cuda.current_device())
    m, n, s, bits, iters, nrhs = args.m, args.n, args.s, args.bits, args.iters, args.nrhs
    fp8 = bool(getattr(args, "fp8", False))
    gen = torch.Generator(device=dev)
    gen.manual_seed(4242)
    phi = torch.randn(m, n, generator=gen, device=dev, dtype=torch.float32) / float(np.sqrt(m))
    X = torch.zeros(nrhs, n, device=dev, dtype=torch.float32)
    for k in range(nrhs):
        sup = torch.randperm(n, generator=gen, device=dev)[:s]
        X[k, sup] = torch.randn(s, generator=gen, device=dev, dtype=torch.float32)
    Yc = (X @ phi.t()).contiguous()                     # nrhs x m, FP32
    sig = torch.sqrt((Yc.double() ** 2).sum(dim=1) / (m * 10.0 ** 3.0)).float()
    Y = (Yc + sig[:, None] * torch.randn(nrhs, m, generator=gen, device=dev, dtype=torch.float32)).contiguous()
    q1, q2 = q.quantize_pair(phi, bits, 7, q.STREAM_Q1, q.STREAM_Q2)
    ys = [q.quantize(Y[k], bits, 7, q.STREAM_Y) for k in range(nrhs)]
    del phi, Yc
    torch.cuda.synchronize()
    ws = q._ws(q.lib().qiht_solve_multi_workspace_size(m, n, s, nrhs), dev)
    out = (torch.empty(nrhs, n, device=dev), torch.empty(nrhs, s, dtype=torch.int32, device=dev),
           torch.zeros(nrhs, q.REPORT_BYTES, dtype=torch.uint8, device=dev))
    for _ in range(max(1, args.warmup)):
        res = q.niht_solve_multi(q1, q2, ys, s, iters, workspace=ws, out=out, fp8=fp8)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    clocks.start()
    time.sleep(0.3)
    ev0.record()
    for _ in range(args.steps):
        res = q.niht_solve_multi(q1, q2, ys, s, iters, workspace=ws, out=out, fp8=fp8)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    reps = res.all_reports()

    def rel(xs, idx):
        return [float(torch.linalg.norm(xs[i] - X[k]) / torch.linalg.norm(X[k])) for i, k in enumerate(idx)]

    err_m = rel(res.x, range(nrhs))
    # plain: a sample of the right-hand sides through qiht_niht_solve (graph cached by a first pass)
    sample = list(range(0, nrhs, max(1, nrhs // args.plain_sample)))[: args.plain_sample]
    sv = q.Solver(m, n, s, iters, device=dev)
    sv(q1, q2, ys[sample[0]])
    torch.cuda.synchronize()
    xs_plain = []
    t_plain = 0.0
    for k in sample:
        ev0.record()
        sv(q1, q2, ys[k])
        ev1.record()
        torch.cuda.synchronize()
        t_plain += ev0.elapsed_time(ev1)
        xs_plain.append(sv.x.clone())
    err_p = rel(xs_plain, sample)
    # the gradient product alone: residual split + tcgen05 GEMM over all right-hand sides
    R = torch.randn(nrhs, m, generator=gen, device=dev, dtype=torch.float32)
    G = torch.empty(nrhs, n, device=dev)
    wsg = q._ws(q.lib().qiht_gemv_t_multi_workspace_size(m, nrhs), dev)
    for _ in range(3):
        q.gemv_t_multi(q1, R, G, workspace=wsg, fp8=fp8)
    torch.cuda.synchronize()
    reps_g = 10
    ev0.record()
    for _ in range(reps_g):
        q.gemv_t_multi(q1, R, G, workspace=wsg, fp8=fp8)
    ev1.record()
    torch.cuda.synchronize()
    gemm_us = ev0.elapsed_time(ev1) / reps_g * 1e3
    flops = 2.0 * m * n * nrhs
    tflops = flops / (gemm_us * 1e-6) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops", 1900.0)) * (2.0 if fp8 else 1.0)
    launches = 3 + 2 * iters                          # init, GEMMs, step kernels, final (the step splits the residual)
    # the GEMM's last partial wave split in two K halves adds a kernel that zeroes those tiles of G
    # before each GEMM (same rule as the library: 256 x 256 tiles, one CTA per SM)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ntiles = (-(-n // 256)) * (-(-nrhs // 256))
    tail = ntiles % nsm
    if ntiles > nsm and 0 < tail and 2 * tail <= nsm:
        launches += iters
    line = {"metric": "multi-RHS solves/s", "value": nrhs / (ms / 1e3), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"u{bits}" + ("+e4m3" if fp8 else ""),
            "data": "synthetic",
            "config": {"workload": f"{nrhs} right-hand sides sharing Gaussian Phi {m}x{n} N(0,1/m), s={s} "
                                   f"N(0,1) nonzeros each, 30 dB, {bits}-bit Phi and y, {iters} iterations",
                       "nrhs": nrhs, "m": m, "n": n, "s": s, "bits": bits, "iters_per_step": iters,
                       "l2": "inputs larger than L2: Q1 codes 256 MiB read by every gradient product"},
            "iterations_per_s": sum(r.iters_run for r in reps) / (ms / 1e3),
            "ms_per_iteration_all_rhs": ms / max(1, iters),
            "plain": {"solves_per_s": len(sample) / (t_plain / 1e3), "ms_per_solve": t_plain / len(sample),
                      "sample": len(sample), "how": "qiht_niht_solve per right-hand side, graph cached"},
            "speedup_vs_plain": (nrhs / (ms / 1e3)) / (len(sample) / (t_plain / 1e3)),
            "equal_error": {"multi_median_rel_err": float(np.median(err_m)),
                            "multi_median_rel_err_on_sample": float(np.median([err_m[k] for k in sample])),
                            "plain_median_rel_err_on_sample": float(np.median(err_p))},
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "traffic": None,
                         "kernel": ("k_mrhs_gemm (G = Q1^T R, e4m3 tcgen05 kind::f8f6f4, three residual terms)"
                                    if fp8 else "k_mrhs_gemm (G = Q1^T R, f16 tcgen05, hi + lo parts)"),
                         "avg_launch_us": gemm_us, "algorithmic_flops_per_launch": flops,
                         "note": ("2 m n nrhs flops (R counted once; the three e4m3 terms triple the MMA work); "
                                  "timed with the residual split; peak: measured dense bf16 burst x 2 (the nominal "
                                  "fp8/bf16 ratio)") if fp8 else
                                 ("2 m n nrhs flops (R counted once; the hi and lo parts double the MMA work); "
                                  "timed with the residual split; peak: measured dense bf16 burst (f16 rate equal)")},
            "gpu_launches": launches * args.steps,
            "clocks": clk,
            "statuses": {str(k): sum(1 for r in reps if r.status == k) for k in sorted({r.status for r in reps})},
            "per_rhs_mean": {"iterations": float(np.mean([r.iters_run for r in reps])),
                             "backtracks": float(np.mean([r.backtracks for r in reps])),
                             "support_changes": float(np.mean([r.support_changes for r in reps])),
                             "ranked_selections": float(np.mean([r.full_selects for r in reps]))}}
    if emit:
        print(json.dumps(line))
    return line


def run_fresh(args, emit=True):
    """The large single solve with fresh realizations of Q(Phi) and Q(y) in every iteration
    (Algorithm 2 as written): 8192 x 32768, s = 256, 30 dB, 8-bit, --iters iterations (default
    here 60). value = iterations/s of qiht_niht_solve_fresh (Phi resident in HBM; every iteration
    re-quantizes it twice). The fixed-quantization solve of the same problem is timed beside it."""
    import torch

    import paper_1802_04907_gb300 as q

    dev = torch.device("cuda", torch.cuda.current_device())
    m, n, s, bits = args.m, args.n, args.s, args.bits
    iters = args.iters if args.iters != ITERS else 60
    gen = torch.Generator(device=dev)
    gen.manual_seed(99)
    phi = torch.randn(m, n, generator=gen, device=dev, dtype=torch.float32) / float(np.sqrt(m))
    sup = torch.randperm(n, generator=gen, device=dev)[:s]
    xt = torch.zeros(n, device=dev)
    xt[sup] = (torch.rand(s, generator=gen, device=dev) + 0.5) * torch.sign(torch.randn(s, generator=gen, device=dev))
    yc = phi @ xt
    y = yc + torch.sqrt((yc.double() ** 2).sum() / (m * 1e3)).float() * torch.randn(m, generator=gen, device=dev)
    for _ in range(max(1, args.warmup)):
        sv = q.niht_solve_fresh(phi, y, bits, bits, 5, s, iters)
    torch.cuda.synchronize()
    clk = start_clocks(torch.device("cuda", torch.cuda.current_device()))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        sv = q.niht_solve_fresh(phi, y, bits, bits, 5, s, iters)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = clk.stop()
    rep = sv.read_report()
    err = float(torch.linalg.norm(sv.x - xt) / torch.linalg.norm(xt))
    q1, q2, qy = q.quantize_problem(phi, y, bits, bits, 5)
    fx = q.Solver(m, n, s, iters, device=dev)
    fx(q1, q2, qy)
    torch.cuda.synchronize()
    ev0.record()
    fx(q1, q2, qy)
    ev1.record()
    torch.cuda.synchronize()
    ms_fx = ev0.elapsed_time(ev1)
    err_fx = float(torch.linalg.norm(fx.x - xt) / torch.linalg.norm(xt))
    line = {"metric": "NIHT iterations/s (fresh realizations)", "value": rep.iters_run / (ms / 1e3),
            "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"u{bits}",
            "data": "synthetic",
            "config": {"workload": f"single solve {m}x{n}, s={s}, +-U(0.5,1.5), 30 dB, {bits}-bit, {iters} iterations, "
                                   "fresh Q(Phi) x2 and Q(y) per iteration",
                       "l2": "inputs larger than L2: Phi FP32 1 GiB read by every re-quantization"},
            "ms_per_iteration": ms / max(1, rep.iters_run),
            "fixed_quantizations": {"iterations_per_s": iters / (ms_fx / 1e3), "rel_err": err_fx},
            "rel_err": err, "status": rep.status, "gpu_launches": None}
    line["clocks"] = clocks
    if emit:
        print(json.dumps(line))
    return line


def run_fly(args, emit=True):
    """Phi computed on the fly (Section IV-C) for the gridded interferometry matrix: 48 antennas
    (2256 baselines, 4512 stacked rows), 128 x 128 sky (16384 columns), 50 sources, s = 64, 20 dB,
    --bits for Phi and y, --iters iterations (default here 60). value = iterations/s of Algorithm 2
    with both realizations of Q(Phi) drawn from the operator in every iteration
    (qiht_niht_solve_fresh_fly: no copy of Phi, FP32 or codes of all realizations, is held). Beside
    it: the same solve from the stored FP32 matrix, and the fused generate + quantize + GEMV^T
    against the GEMV^T of stored codes at 8, 4 and 2 bits. The roofline is the fused product's
    instruction issue (bound "alu")."""
    import torch

    import paper_1802_04907_gb300 as q
    import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    bits = args.bits
    iters = args.iters if args.iters != ITERS else 60
    p = synth.interferometry_gridded(48, 128, n_src=50, s=64, snr_db=20.0, seed=0)
    m, n, s = p.m, p.n, p.s
    op = q.FlyOp(torch.from_numpy(np.ascontiguousarray(p.meta["uv"], dtype=np.int32)).to(dev),
                 torch.from_numpy(p.meta["table"]).to(dev), p.meta["grid"])
    y = torch.from_numpy(p.y).to(dev)
    xt = torch.from_numpy(p.x_true).to(dev, torch.float32)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            out = fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps, out

    clk = start_clocks(dev)
    torch.cuda.synchronize()
    ms, sv = timed(lambda: q.niht_solve_fresh_fly(op, y, bits, bits, 5, s, iters), args.steps)
    clocks = clk.stop()
    rep = sv.read_report()
    err = float(torch.linalg.norm(sv.x - xt) / torch.linalg.norm(xt))
    phi = torch.from_numpy(p.phi).to(dev)
    ms_st, st = timed(lambda: q.niht_solve_fresh(phi, y, bits, bits, 5, s, iters), max(1, args.steps // 2))
    same = bool(torch.equal(st.x, sv.x) and torch.equal(st.support, sv.support))
    # the gradient product alone: fused on the fly against stored codes (max |r| given to both)
    r = torch.from_numpy(synth.random_floats(m, seed=3, scale=0.3)).to(dev)
    g = torch.empty(n, device=dev)
    sc = torch.empty(1, device=dev)
    rmax = torch.abs(r).max().reshape(1)
    prod = {}
    for b in (8, 4, 2):
        us_fly = timed(lambda: q.gemv_t_fly(op, b, 1, 0, r, g, scale=sc), 100)[0] * 1e3
        Q = q.fly_quantize(op, b, 1, 0)
        us_st = timed(lambda: q.gemv_t_prescaled(Q, r, rmax, g), 100)[0] * 1e3
        us_qp = timed(lambda: q.fly_quantize(op, b, 1, 0, 1), 20)[0] * 1e3
        prod[f"bits{b}"] = {"fused_on_the_fly_us": us_fly, "stored_codes_us": us_st,
                            "two_realizations_from_operator_us": us_qp}
    us_qp_fp32 = timed(lambda: q.quantize_pair(phi, bits, 1, 0, 1), 20)[0] * 1e3
    # roofline of the fused product: algorithmic operations per entry (Philox4x32-10: 10 rounds of
    # two wide multiplies and two three-input XORs per four entries = 10; phase index 1.5; table
    # read 1; code 3; multiply-accumulate 1) against the issue rate of 152 SMs x 4 schedulers x
    # 32 lanes at the maximum SM clock
    ops = 16.5 * m * n
    us_f = prod[f"bits{bits}"]["fused_on_the_fly_us"]
    peak = 152 * 4 * 32 * 2.07e9 / 1e12
    achieved = ops / (us_f * 1e-6) / 1e12
    line = {"metric": "NIHT iterations/s (fresh realizations, Phi on the fly)", "value": rep.iters_run / (ms / 1e3),
            "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"u{bits}",
            "data": "synthetic",
            "config": {"workload": f"gridded interferometry {m}x{n} (48 antennas, 128x128 sky), 50 sources, s={s}, "
                                   f"20 dB, {bits}-bit Phi and y, {iters} iterations, fresh Q(Phi) x2 and Q(y) per "
                                   "iteration drawn from the operator",
                       "m": m, "n": n, "s": s, "bits": bits, "iters_per_step": iters,
                       "l2": "no matrix is read: the operator is 9 KB of baselines and a 1 KB table"},
            "ms_per_iteration": ms / max(1, rep.iters_run), "rel_err": err, "status": rep.status,
            "stored_fp32_phi": {"iterations_per_s": iters / (ms_st / 1e3), "identical_results": same,
                                "quantize_two_realizations_us": us_qp_fp32},
            "gradient_product": prod,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": f"k_fly_gemv_t (generate + quantize + Q^T r, {bits}-bit codes)",
                         "avg_launch_us": us_f, "algorithmic_ops_per_launch": ops,
                         "note": "16.5 lane operations per entry (Philox 10, phase index 1.5, table read 1, code 3, "
                                 "multiply-accumulate 1); peak = 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz "
                                 "(the maximum SM clock), the issue limit"},
            "gpu_launches": None, "clocks": clocks}
    if emit:
        print(json.dumps(line))
    return line


def run_mri_op(args, emit=True):
    """The MRI operator form (Section IV-B): Phi = S (A (x) A) on the 128 x 128 head-like phantom
    (a third of k-space on radial lines, 11364 stacked rows, 16384 Haar coefficients), s = 512,
    30 dB, the 1D transform A = F_1 H^T quantized to --bits-factor bits (default 12, the paper's
    transform width), k-space to --bits-y (default 8), --iters iterations (default here 100).
    value = iterations/s of qiht_niht_solve_separable (dense transforms of the image, never an
    m x n matrix). Beside it: the dense materialized composite at 8 bits (the fixed-codes
    solver), whose recovery is limited by that quantization."""
    import torch

    import paper_1802_04907_gb300 as q
    import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    iters = args.iters if args.iters != ITERS else 100
    bf = args.bits_factor
    by = args.bits_y or 8
    N0 = getattr(args, "mri_grid", 128)
    dense = N0 <= 128
    p = synth.mri(N0, s=512 if N0 <= 128 else 4096, snr_db=30.0, seed=0, materialize=dense)
    N, s = p.meta["grid"], p.s
    op = q.SepOp(torch.from_numpy(p.meta["factor"]).to(dev), torch.from_numpy(p.meta["mask"]).to(dev))
    y = torch.from_numpy(p.y).to(dev)
    xt = torch.from_numpy(p.x_true).to(dev, torch.float32)
    for _ in range(max(1, args.warmup)):
        sv = q.niht_solve_separable(op, y, bf, by, 5, s, iters)
    torch.cuda.synchronize()
    clk = start_clocks(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        sv = q.niht_solve_separable(op, y, bf, by, 5, s, iters)
    ev1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    rep = sv.read_report()
    err = float(torch.linalg.norm(sv.x - xt) / torch.linalg.norm(xt))
    # the materialized composite at 8 bits through the fixed-codes solver, for the recovery
    dense_line = None
    if dense:
        phi = torch.from_numpy(p.phi).to(dev)
        q1, q2, qy = q.quantize_problem(phi, y, 8, by, 5)
        fx = q.Solver(p.m, p.n, s, iters, device=dev)
        fx(q1, q2, qy)
        torch.cuda.synchronize()
        ev0.record()
        fx(q1, q2, qy)
        ev1.record()
        torch.cuda.synchronize()
        ms_fx = ev0.elapsed_time(ev1)
        err_fx = float(torch.linalg.norm(fx.x - xt) / torch.linalg.norm(xt))
        dense_line = {"iterations_per_s": iters / (ms_fx / 1e3), "rel_err": err_fx}
        del phi, q1, q2, qy, fx
    # one operator application: 6 N^3 multiply-adds (two GEMMs) and the gather or scatter
    _, fh, _ = q.sep_quantize_factor(op, bf, 5, 0)
    xv = torch.randn(op.cols, device=dev)
    rv = torch.randn(op.rows, device=dev)
    for _ in range(5):
        q.sep_apply(op, fh, xv)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(200):
        q.sep_apply(op, fh, xv)
    ev1.record()
    torch.cuda.synchronize()
    us_f = ev0.elapsed_time(ev1) / 200 * 1e3
    ev0.record()
    for _ in range(200):
        q.sep_apply(op, fh, rv, adjoint=True)
    ev1.record()
    torch.cuda.synchronize()
    us_a = ev0.elapsed_time(ev1) / 200 * 1e3
    flops = 12.0 * N**3
    peak = 152 * 128 * 2 * 2.07e9 / 1e12                  # FP32 FMA: 128 lanes per SM per clock
    line = {"metric": "NIHT iterations/s (MRI operator form)", "value": rep.iters_run / (ms / 1e3),
            "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"f32 products, u{bf} factor",
            "data": "synthetic",
            "config": {"workload": f"MRI operator form: {N}x{N} head phantom, radial third of k-space ({p.m} stacked "
                                   f"rows), {p.n} Haar coefficients, s={s}, 30 dB, {bf}-bit transform factor, "
                                   f"{by}-bit k-space, {iters} iterations",
                       "N": N, "m": p.m, "n": p.n, "s": s, "bits_factor": bf, "bits_y": by, "iters_per_step": iters,
                       "l2": "operator state (two 256x128 factors, 2N x 2N products) fits L2"},
            "ms_per_iteration": ms / max(1, rep.iters_run), "rel_err": err, "status": rep.status,
            "backtracks": rep.backtracks,
            "dense_8bit_composite": dense_line if dense_line is not None else "not formed: the dense m x n matrix "
                                    "of this size would not fit",
            "operator_application_us": {"forward": us_f, "adjoint": us_a},
            "roofline": {"bound": "alu", "achieved": flops / (us_f * 1e-6) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (us_f * 1e-6) / 1e12 / peak, "traffic": None,
                         "kernel": "k_sgemm (forward application: two FP32 GEMMs and the gather)",
                         "avg_launch_us": us_f, "algorithmic_flops_per_launch": flops,
                         "note": "12 N^3 flops per application; peak = FP32 FMA of 152 SMs x 128 lanes x 2.07 GHz; "
                                 "at N = 128 an application is a few small launches (latency-bound)"},
            "gpu_launches": None, "clocks": clocks}
    if emit:
        print(json.dumps(line))
    return line


def run_unrolled(args, emit=True):
    """Differentiation workload: 64 problems, Gaussian Phi 2048 x 8192 N(0, 1/m), s = 64 N(0,1)
    nonzeros, per-row complex gain |g| ~ U(0.9, 1.1), arg g ~ U(-0.1, 0.1), y = [Re g; Im g] Phi x
    + noise at 30 dB (not quantized), 4-bit codes of Phi, K = 50 unrolled iterations, loss
    ||x_K - x_true||^2. value = problems per second of one forward + backward (gradients in y and
    the gain), sqrt(K) checkpoints; inputs generated on the device from seeds."""
    import torch

    import paper_1802_04907_gb300 as q

    dev = torch.device("cuda", torch.cuda.current_device())
    P, m, n, s, K, bits = 64, 2048, 8192, 64, 50, 4
    gen = torch.Generator(device=dev)
    gen.manual_seed(31)
    Q1s, Q2s, ys, gas, gbs, xts = [], [], [], [], [], []
    for p in range(P):
        phi = torch.randn(m, n, generator=gen, device=dev) / float(np.sqrt(m))
        x = torch.zeros(n, device=dev)
        x[torch.randperm(n, generator=gen, device=dev)[:s]] = torch.randn(s, generator=gen, device=dev)
        mag = 0.9 + 0.2 * torch.rand(m, generator=gen, device=dev)
        ph = -0.1 + 0.2 * torch.rand(m, generator=gen, device=dev)
        a, b = mag * torch.cos(ph), mag * torch.sin(ph)
        px = phi @ x
        clean = torch.cat([a * px, b * px])
        sig = torch.sqrt((clean.double() ** 2).sum() / (2 * m * 1e3)).float()
        ys.append(clean + sig * torch.randn(2 * m, generator=gen, device=dev))
        q1, q2 = q.quantize_pair(phi, bits, 1000 + p, q.STREAM_Q1, q.STREAM_Q2)
        Q1s.append(q1)
        Q2s.append(q2)
        gas.append(a)
        gbs.append(b)
        xts.append(x)
        del phi
    Y, GA, GB, XT = (torch.stack(t).contiguous() for t in (ys, gas, gbs, xts))
    op = q.Unrolled(Q1s, Q2s, s, K)
    torch.cuda.synchronize()

    def step():
        X = op.forward(Y, GA, GB)
        return X, op.backward(Y, GA, GB, 2.0 * (X - XT))

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    clk = start_clocks(torch.device("cuda", torch.cuda.current_device()))
    torch.cuda.synchronize()
    ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t_fwd = t_all = 0.0
    for _ in range(args.steps):
        ev0.record()
        X = op.forward(Y, GA, GB)
        ev1.record()
        op.backward(Y, GA, GB, 2.0 * (X - XT))
        ev2.record()
        torch.cuda.synchronize()
        t_fwd += ev0.elapsed_time(ev1)
        t_all += ev0.elapsed_time(ev2)
    ms = t_all / args.steps
    clocks = clk.stop()
    loss = float(((X - XT) ** 2).sum())
    rel = float(torch.linalg.norm(X - XT) / torch.linalg.norm(XT))
    codes = sum(qq.nbytes for qq in Q1s) + sum(qq.nbytes for qq in Q2s)
    # dense products per forward + backward: K forward, K recomputed, K adjoint (A^T v over all n)
    passes = 3 * K
    # launches of this library per step: forward = init, planes, K x (product, step), output;
    # backward = per checkpoint segment one planes kernel, then K x 2 recomputed, K x 2 adjoint
    c = math.isqrt(K - 1) + 1 if K > 1 else 1
    ud_launches = args.steps * ((3 + 2 * K) + (-(-K // c) + 4 * K))
    achieved = passes * (codes / 2) / (ms / 1e3) / 1e9
    peak, _ = load_peaks()
    line = {"metric": "unrolled forward+backward problems/s", "value": P / (ms / 1e3), "unit": "problems/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"u{bits}", "data": "synthetic",
            "config": {"workload": f"{P} problems, Gaussian Phi {m}x{n}, s={s}, per-row complex gain, 30 dB, "
                                   f"{bits}-bit codes, K={K} unrolled iterations, sqrt(K) checkpoints, gradients "
                                   "in y and the gain",
                       "P": P, "m": m, "n": n, "s": s, "K": K, "bits": bits},
            "ms_forward": t_fwd / args.steps, "ms_forward_backward": ms, "loss": loss, "rel_err_xK": rel,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "note": "3K dense code passes (forward, recomputation, adjoint) over the step time; "
                                 "the per-problem step kernels are not counted"},
            "clocks": clocks, "gpu_launches": ud_launches}
    if emit:
        print(json.dumps(line))
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "multi":
        run_multi(args)
    elif args.workload == "fly":
        run_fly(args)
    elif args.workload == "mri_op":
        run_mri_op(args)
    elif args.workload == "fresh":
        run_fresh(args)
    elif args.workload == "unrolled":
        run_unrolled(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
