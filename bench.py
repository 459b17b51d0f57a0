"""Benchmark of the plain-LRSTV ADMM iteration (arXiv 2204.12879, Algorithm 1)
on GB300.

One step = one whole denoise of the 200x200x80 Pavia-shaped synthetic cube
(6 endmembers, 40 Voronoi cells, mixed Gaussian / impulse / stripe /
dead-line noise): lrstv_init, then its 50 ADMM iterations (steps 1-7 each:
L/T_z stencil, 3-D DFT Z-solve, fused F/S/multiplier update, t-SVT of the
three gradient tensors), so every timed window covers whole penalty
schedules whatever --steps and --warmup are.  Each E-step's Jacobi SVDs start
from the previous E-step's singular vectors (LRSTV_FLAG_WARM_START;
--jacobi-start cold starts every one from the identity).  value = ADMM
iterations per second over all ranks; cubes/s = steps / time.  The timed
pass runs without the library's per-launch profiler; a second, profiled pass
of the same denoise gives the per-kernel table and the roofline.  The FP32
FMA and tensor-pipe peaks of the roofline fractions are measured in the same
run by the library's throughput probes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (one cube per rank, no
collective on the data path); only the timing barrier and the max over ranks
cross ranks.  --impl reference times the FP64 CPU oracle on the host cores
(a bounded number of single ADMM iterations of the same cube; its line's
steps is the number it timed).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "c1": {"recipe": "c1", "seed": 1, "iters": 20,
           "desc": "32x32x16 synthetic cube, 4 endmembers, 12 Voronoi cells, Gaussian 0.1 + 10% impulse, 20 ADMM iterations"},
    "c2": {"recipe": "c2", "seed": 2, "iters": 50,
           "desc": "200x200x80 Pavia-shaped synthetic cube, 6 endmembers, 40 Voronoi cells, mixed noise (Gaussian U[0.1,0.2] per band, 20% impulse, stripes on 30% and dead lines on 10% of bands), 50 ADMM iterations"},
    "c3": {"recipe": "c3", "seed": 3, "iters": 60,
           "desc": "256x256x191 Washington-DC-shaped synthetic cube, 8 endmembers, mixed noise, 60 ADMM iterations"},
}
BATCH = {"count": 64, "seed": 4, "iters": 50,
         "desc": "batch of 64 uneven synthetic cubes drawn by seed from 64x64x31, 128x128x64, 145x145x220 (Indian Pines shape) and 200x200x80, each with Gaussian U[0.05,0.2] and impulse U[0,0.3] noise, 50 ADMM iterations, one persistent Jacobi launch per step"}
METRIC = "ADMM iterations/s (plain LRSTV, FP32, 1e-4 max-abs vs FP64 oracle)"
UNIT = "iter/s"
METRIC_TUCKER = "ADMM iterations/s (full TDLRSTV, Tucker L-update, FP32)"
METRIC_BF16X3 = "ADMM iterations/s (plain LRSTV, mixed precision: 3xBF16 tensor-core GEMMs)"
METRIC_BATCH = "cube-ADMM-iterations/s (batched plain LRSTV, FP32)"
UNIT_BATCH = "cube-iter/s"
METRIC_UNROLL = "unrolled-LRSTV training steps/s (forward + backward + update, FP32)"
UNIT_UNROLL = "step/s"
FP32_LANES_PER_SM = 128
# kernels a plan runs on its side stream (lrstv_iterate: the next iteration's
# L-update and Z-solve, the Tucker update), overlapped with the E-step
SIDE_STREAM_KERNELS = ("l_tz", "r2c_z", "cgemm_z", "c2r_z", "tucker")


# ------------------------------------------------------------ multi-rank ---
def dist_env():
    """(rank, world, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank denoises its own cube: a distinct seed per rank."""
    return base_seed + 1000 * rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while the
    timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
                 "200", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()

    def summary(self):
        if not self.rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in self.rows]
        mx = [num(r[2]) for r in self.rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(self.rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------ roofline ---
def gemm_precision(args, wl_name):
    """Split precision of the tensor-core GEMMs: the mixed-precision workload
    (256x256x191) runs 3xBF16 unless told otherwise, the others 3xTF32."""
    if args.precision != "auto":
        return args.precision
    return "bf16x3" if wl_name == "c3" else "tf32x3"


def tucker_ranks(args, shape):
    """Multilinear ranks of the full TDLRSTV L-update (--tucker R3): r1 =
    0.8 n1, r2 = 0.8 n2 (Section IV-D), r3 given; None for plain LRSTV."""
    if not args.tucker:
        return None
    n1, n2, n3 = shape
    return (max(1, round(0.8 * n1)), max(1, round(0.8 * n2)), min(args.tucker, n3))


def metric_for(args, wl_name):
    """The metric of a single-cube workload's line, the same for both arms."""
    if args.tucker:
        return METRIC_TUCKER
    if gemm_precision(args, wl_name) == "bf16x3":
        return METRIC_BF16X3
    return METRIC


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_work(name, shape):
    """Algorithmic work of one launch of each kernel: ('hbm', bytes) or
    ('alu', flops); FP32 cubes are 4N bytes, half spectra 8 h n1 n2 bytes."""
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    P = n1 * n2
    h = n3 // 2 + 1
    nr, nc = max(n1, n2), min(n1, n2)
    spec = 8 * h * P
    if name == "l_tz":      # reads Y S Z G1 G2 F[3] G3[3], writes L T_z
        return "hbm", 13 * 4 * N
    if name == "fs_dual":   # reads Y L Z S G1 G2 E[3] G3[3] G4[3] ... writes F[3] S G1 G2 G3[3]
        return "hbm", 23 * 4 * N
    if name == "r2c_z":
        return "hbm", 4 * N + spec
    if name == "c2r_z":
        return "hbm", spec + 4 * N
    if name == "r2c_e":
        return "hbm", 6 * 4 * N + 3 * spec
    if name == "c2r_e":
        return "hbm", 3 * spec + 12 * 4 * N
    if name == "cgemm_z":   # average of the 4 spatial passes: 8 flops per complex MAC
        return "alu", 8 * P * h * (n1 + n2) // 2
    if name == "cgemm_e":
        return "alu", 8 * nr * nc * nc * 3 * h
    if name == "warm_e":    # per E-step: V V^H, (V V^H) V, A V per slice; the NS update and
        # sigma / V diag g launches are HBM-light; this is the per-launch average over 5 launches
        return "alu", 8 * 3 * h * (2 * nc ** 3 + nr * nc * nc) // 5
    return None, 0


def jacobi_flops(prof, shape):
    """FP32 flops of the Jacobi launches as the kernel does the work: 8 nr per
    examined column pair (the inner product w_p^H w_q; the squared norms are
    tracked through the rotations) and 18 (nr + nc) per rotated pair (phase,
    two complex scaled sums on W's and V's rows)."""
    n1, n2, _ = shape
    nr, nc = max(n1, n2), min(n1, n2)
    return 8.0 * nr * prof.jacobi_pairs + 18.0 * (nr + nc) * prof.jacobi_rotations


def jacobi_textbook_flops(prof, shape):
    """The same launches at the usual count of a complex one-sided Jacobi
    sweep, about 30 n^3 flops a slice (n = nc; pairs, their inner products and
    rotations of W and V), times the sweep-slices the launches ran (pairs
    examined / (nc (nc - 1) / 2))."""
    n1, n2, _ = shape
    nc = min(n1, n2)
    sweep_slices = prof.jacobi_pairs / max(nc * (nc - 1) / 2, 1)
    return 30.0 * nc ** 3 * sweep_slices


def derived_peaks(pk, pk_kind, probes, sm_count):
    """The roofs the line's fractions use.  FP32 FMA and TF32 come from this
    run's probes when they ran (the larger of the scalar and paired FMA
    rates); otherwise FP32 is derived from the device's SM count, 128 FP32
    lanes, 2 flops per FMA and sm_max_mhz, and TF32 is half the BF16 figure
    (the nominal ratio).  BF16 is MEASURED_PEAKS.json's cuBLAS figure."""
    out = {"sm_count": sm_count, "bf16": pk["bf16_tflops"],
           "bf16_source": f"bf16_tflops of MEASURED_PEAKS.json (cuBLAS, {pk_kind})"}
    if probes:
        unit = max(("fp32_fma", "fp32_fma2"), key=lambda u: probes[u]["tflops"])
        ck = probes[unit]["clocks"] or {}
        out["fp32"] = probes[unit]["tflops"]
        out["fp32_source"] = (f"measured in this run: lrstv_peak_probe {unit} on {sm_count} SMs, "
                              f"median SM clock {ck.get('sm_mhz')} MHz, reasons {ck.get('reasons')}")
        ck = probes["tf32_mma"]["clocks"] or {}
        out["tf32"] = probes["tf32_mma"]["tflops"]
        out["tf32_source"] = (f"measured in this run: lrstv_peak_probe tf32_mma (tcgen05 kind::tf32, "
                              f"128x256x8), median SM clock {ck.get('sm_mhz')} MHz, "
                              f"reasons {ck.get('reasons')}")
        out["probes"] = probes
    else:
        mhz = pk.get("sm_max_mhz", 2070.0)
        out["fp32"] = sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        out["fp32_source"] = (f"derived (probes not run): {sm_count} SMs x {FP32_LANES_PER_SM} "
                              f"lanes x 2 x {mhz} MHz")
        out["tf32"] = 0.5 * pk["bf16_tflops"]
        out["tf32_source"] = "derived (probes not run): half the BF16 figure, the nominal ratio"
    return out


def tensor_fracs(kernels, shape, precision, peak):
    """Tensor-pipe fraction of each tensor-core GEMM kernel on the main
    stream: the split's three products at 8 real flops per complex
    multiply-add (24 per complex MAC in the pipe) over the launch's average
    time, against the measured peak of the split's operand type (TF32 or
    BF16).  The side stream's GEMMs (the Z-solve's) are left out: their
    in-region times include waiting for SMs (their serialised times are in the
    ncu launch list)."""
    roof = peak["bf16"] if precision == "bf16x3" else peak["tf32"]
    out = {}
    for name in ("cgemm_e",):
        if name not in kernels:
            continue
        useful = kernel_work(name, shape)[1]
        s = kernels[name]["ms_per_launch"] / 1e3
        pipe = 3 * useful / s / 1e12
        out[name] = {"pipe_tflops": pipe, "peak": roof, "frac": pipe / roof,
                     "useful_tflops": useful / s / 1e12}
    return out


def stage_bounds(kernels, shape, iterations, precision, jacobi_flops_total, pk, peak):
    """Each stage's algorithmic work per iteration at its own roof, in ms:
    HBM bytes at the measured bandwidth for the stencil and threshold
    kernels; max(FP32 ALU, HBM) for the mode-3 DFTs (4 flops per
    real-by-complex product); three products per complex multiply-add at the
    split's tensor rate (BF16, or TF32) for the tensor-core GEMMs; the
    Jacobi's device-counted flops at the FP32 peak.  kernels is the
    per-kernel table ({name: {"launches", ...}}) of a pass that covered
    `iterations` iterations.  Stages without a stated bound are listed."""
    n1, n2, n3 = shape
    P, h = n1 * n2, n3 // 2 + 1
    hbm = pk["hbm_gbs"] * 1e9
    fp32 = peak["fp32"] * 1e12
    tensor = (peak["bf16"] if precision == "bf16x3" else peak["tf32"]) * 1e12
    per, unbounded = {}, []
    for name, v in kernels.items():
        per_it = v["launches"] / iterations
        if name == "jacobi":
            sec = jacobi_flops_total / iterations / fp32
        elif name in ("cgemm_z", "cgemm_e", "warm_e"):
            sec = 3 * kernel_work(name, shape)[1] * per_it / tensor
        elif name in ("r2c_z", "c2r_z", "r2c_e", "c2r_e"):
            flops = 4 * n3 * h * P * (3 if name.endswith("_e") else 1)
            sec = max(flops / fp32, kernel_work(name, shape)[1] / hbm) * per_it
        else:
            kind, work = kernel_work(name, shape)
            if kind != "hbm":
                unbounded.append(name)
                continue
            sec = work * per_it / hbm
        per[name] = sec * 1e3
    return {"ms_per_iteration": per, "sum_ms": sum(per.values()), "without_bound": unbounded}


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(workload, {}).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2204_12879_gb300", "csrc", rec["source"])
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return rec["dram_bytes_per_launch"] if digest == rec["source_sha256"] else None


# ---------------------------------------------------------------- arms ---
def make_input(wl, rank):
    import numpy as np
    from synthetic import RECIPES, make_cube
    r = RECIPES[wl["recipe"]]
    clean, noisy = make_cube(r, replica_seed(wl["seed"], rank))
    return r.shape, clean, noisy.astype(np.float32)


def measure_peaks(clock_gpu):
    """FP32 FMA and tensor-pipe throughput measured on this device by the
    library's probes (lrstv_peak_probe), each with the SM clocks sampled while
    it runs.  Returns {unit: {"tflops", "ms", "clocks"}}."""
    from paper_2204_12879_gb300 import lrstv
    work = {"fp32_fma": 13_000_000, "fp32_fma2": 6_500_000, "tf32_mma": 5_500_000,
            "bf16_mma": 5_500_000}
    out = {}
    for unit, w in work.items():
        cs = ClockSampler(clock_gpu)
        cs.start()
        tf, ms = lrstv.lrstv_peak_probe(unit, w)
        if ms < 300.0:  # long enough for the 200 ms clock samples
            tf, ms = lrstv.lrstv_peak_probe(unit, int(w * 400.0 / max(ms, 1.0)))
        out[unit] = {"tflops": tf, "ms": ms, "clocks": cs.stop()}
    return out


def clock_gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(vis) if vis.isdigit() else local


def run_ours(args, wl_name):
    import numpy as np
    import torch

    from paper_2204_12879_gb300 import builder, lrstv
    from synthetic import flat, mpsnr

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        builder.build()
    barrier(world)
    lrstv.load()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count

    wl = WORKLOADS[wl_name]
    shape, clean, Y = make_input(wl, rank)
    n1, n2, n3 = shape
    iters = wl["iters"]
    flags = lrstv.FLAG_WARM_START if args.jacobi_start == "warm" else 0
    precision = gemm_precision(args, wl_name)
    if precision == "bf16x3":
        flags |= lrstv.FLAG_BF16X3
    if args.dft == "simt":
        flags |= lrstv.FLAG_SIMT_DFT
    if args.jacobi_schedule == "slice":
        flags |= lrstv.FLAG_JACOBI_PER_SLICE
    if args.jacobi_panel == 16:
        flags |= lrstv.FLAG_JACOBI_PANEL16
    if args.jacobi_order == "fixed":
        flags |= lrstv.FLAG_JACOBI_FIXED_ORDER
    params = lrstv.Params.make(n1, n2, max_iter=iters, flags=flags)
    plan = lrstv.Plan(n1, n2, n3, params)
    ranks = tucker_ranks(args, (n1, n2, n3))
    if ranks:
        plan.set_tucker(ranks)
    y_dev = torch.from_numpy(flat(Y)).cuda()
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    gpu = clock_gpu_index(local)

    def denoise():
        # one step: a whole denoise of the cube (lrstv_init, then every
        # iteration of it in one lrstv_iterate call, so that the library can
        # overlap each iteration's L/Z steps with the previous E-step)
        plan.init(y_dev)
        plan.iterate(iters)

    pk_meas = measure_peaks(gpu) if rank == 0 and not args.no_peaks else None
    for _ in range(args.warmup):
        denoise()
    torch.cuda.synchronize()

    # timed pass: the library's profiler is off (no per-launch events, no
    # device work counters)
    clocks = ClockSampler(gpu)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t0, t1 = ev(), ev()
    t0.record(stream)
    for _ in range(args.steps):
        denoise()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    stats = plan.stats()
    ms_max = max_over_ranks(ms, world, device=torch.device("cuda", local))

    # profiled pass of the same work (whole denoises): per-launch CUDA events
    # on the launching streams and the Jacobi's work counters, for the
    # per-kernel table, the roofline and the stage bounds
    n_prof = min(args.steps, 2)
    plan.profile_enable(True)
    p0, p1 = ev(), ev()
    p0.record(stream)
    for _ in range(n_prof):
        denoise()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    prof = plan.profile_read()
    plan.profile_enable(False)

    # end to end through the host-buffer call, the same K steps: each is one
    # lrstv_plan_run_host (H2D of Y, a whole denoise, D2H of X and S)
    yh = torch.from_numpy(flat(Y)).pin_memory()
    xh = torch.empty_like(yh).pin_memory()
    sh = torch.empty_like(yh).pin_memory()
    plan.run_host(yh, xh, sh)  # untimed warm-up call
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(args.steps):
        plan.run_host(yh, xh, sh)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e = max_over_ranks(e0.elapsed_time(e1), world, device=torch.device("cuda", local))
    X = xh.numpy().astype(np.float64).reshape(shape, order="F")
    quality = {"mpsnr_db": round(mpsnr(X, clean), 3),
               "noisy_mpsnr_db": round(mpsnr(Y, clean), 3)}
    plan.close()
    if precision == "bf16x3":
        # the same denoise with FP32-accurate (3xTF32) GEMMs, the path held to
        # 1e-4 of the FP64 oracle: the mixed-precision error at full size
        ref_params = lrstv.Params.make(n1, n2, max_iter=iters, flags=flags & ~lrstv.FLAG_BF16X3)
        with lrstv.Plan(n1, n2, n3, ref_params) as ref_plan:
            if ranks:
                ref_plan.set_tucker(ranks)
            ref_plan.run_host(yh, xh, sh)
        Xr = xh.numpy().astype(np.float64).reshape(shape, order="F")
        quality["vs_tf32x3"] = {"max_abs": float(np.max(np.abs(X - Xr))),
                                "mpsnr_db": round(mpsnr(Xr, clean), 3),
                                "d_mpsnr_db": float(mpsnr(X, clean) - mpsnr(Xr, clean))}

    if rank != 0:
        return None
    pk, pk_kind = peaks()
    peak = derived_peaks(pk, pk_kind, pk_meas, sm_count)
    kernels = {}
    for k in range(16):
        if prof.launches[k]:
            kernels[lrstv.kernel_name(k)] = {"launches": prof.launches[k],
                                             "ms_per_launch": prof.ms[k] / prof.launches[k],
                                             "share": prof.ms[k] / max(sum(prof.ms), 1e-9)}
    prof_iters = n_prof * iters
    # The Jacobi is the dominant kernel: 78% of the serialised launch list of
    # this workload (profiles/launches_c2_200x200x80.md), and the E-step's
    # critical path.  The side stream's kernels (the next iteration's L-update
    # and Z-solve, the Tucker update, the early Newton-Schulz products) wait
    # there for the SMs that the Jacobi holds, so their in-region times include
    # that wait and would overstate them.
    dom = "jacobi" if "jacobi" in kernels else max(
        kernels, key=lambda n: kernels[n]["ms_per_launch"] * kernels[n]["launches"])
    for name in SIDE_STREAM_KERNELS:
        if name in kernels:
            kernels[name]["side_stream"] = True
    avg_s = kernels[dom]["ms_per_launch"] / 1e3
    if dom == "jacobi":
        flops = jacobi_flops(prof, shape) / prof.launches[6]
        textbook = jacobi_textbook_flops(prof, shape) / prof.launches[6]
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak["fp32"],
                "unit": "TFLOP/s", "peak_source": peak["fp32_source"],
                "work": "the kernel's own: 8 nr flops per examined column pair, 18 (nr + nc) per "
                        "rotated pair, counted on the device",
                "achieved_textbook": textbook / avg_s / 1e12,
                "frac_textbook": textbook / avg_s / 1e12 / peak["fp32"]}
    else:
        bound, work = kernel_work(dom, shape)
        if bound == "hbm":
            roof = {"bound": "hbm", "achieved": work / avg_s / 1e9, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({pk_kind})"}
        else:
            roof = {"bound": "alu", "achieved": work / avg_s / 1e12, "peak": peak["fp32"],
                    "unit": "TFLOP/s", "peak_source": peak["fp32_source"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dom
    roof["measured"] = (f"launch durations from the library's CUDA events on the launching "
                        f"streams over a profiled pass of {n_prof} whole denoise(s) run right "
                        f"after the timed pass (the timed pass runs without them)")
    roof["traffic"] = traffic_for(dom, wl_name)
    bounds = stage_bounds(kernels, shape, prof_iters, precision, jacobi_flops(prof, shape), pk,
                          peak)
    bounds["iteration_ms"] = ms_max / (args.steps * iters)
    bounds["frac"] = bounds["sum_ms"] / bounds["iteration_ms"]
    value = world * args.steps * iters / (ms_max / 1e3)
    metric = metric_for(args, wl_name)
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == "tf32x3" else "f32 (GEMMs 3xbf16)", "data": "synthetic",
        "config": {"workload": wl["desc"], "shape": list(shape),
                   "step": f"one whole denoise of the cube: lrstv_init + {iters} ADMM iterations",
                   "iters_per_cube": iters, "cubes_per_s": world * args.steps / (ms_max / 1e3),
                   "parallelism": "replicas" if world > 1 else "single",
                   "jacobi_start": args.jacobi_start,
                   "gemm_precision": precision,
                   "mode3_dft": "tensor cores" if args.dft == "tc" else "SIMT direct sums",
                   "jacobi_schedule": ("task graph: panel-pair tasks of every slice on all SMs"
                                       if args.jacobi_schedule == "tasks" else "one CTA per slice"),
                   "jacobi_panel": args.jacobi_panel,
                   "jacobi_order": ("columns by norm, largest first, each sweep"
                                    if args.jacobi_order == "sorted" else "stored order"),
                   "l_update": ("Tucker projection, one HOOI sweep per iteration, ranks %s" % (ranks,)
                                if ranks else "plain (full Tucker ranks)"),
                   "l2": "working set (18 state cubes + spectra, ~330 MB) exceeds the 129 MB L2",
                   "timed_pass": "profiler off"},
        "roofline": roof,
        "tensor_roofline": tensor_fracs(kernels, shape, precision, peak),
        "peaks": peak,
        "stage_bounds": bounds,
        "kernels": kernels,
        "profiled_pass": {"denoises": n_prof, "ms_per_iteration": ms_prof / prof_iters,
                          "overhead_vs_timed": (ms_prof / prof_iters) / (ms / (args.steps * iters))},
        "gpu_launches": int(sum(prof.launches)) * args.steps // n_prof,
        "jacobi": {"max_sweeps_last": stats.jacobi_max_sweeps,
                   "unconverged_last": stats.jacobi_unconverged,
                   "pairs_per_denoise": prof.jacobi_pairs // n_prof,
                   "rotations_per_denoise": prof.jacobi_rotations // n_prof},
        "e2e": {"value": world * args.steps * iters / (e2e / 1e3), "unit": UNIT,
                "ms_per_step": e2e / args.steps, "h2d_bytes_per_step": 4 * n1 * n2 * n3,
                "d2h_bytes_per_step": 8 * n1 * n2 * n3,
                "step": f"one lrstv_plan_run_host call: copy Y in, {iters} iterations, copy X and S out"},
        "quality": quality,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(wl, Y, budget_s=args.cpu_budget, ranks=ranks)
    return line


def run_batch(args):
    """The batched form: all cubes advance one ADMM iteration per step (one
    persistent Jacobi launch over every Fourier slice of every cube); value =
    cube-iterations per second.  The same cubes run one plan at a time for a
    few iterations give the unbatched comparison."""
    import numpy as np
    import torch

    from paper_2204_12879_gb300 import builder, lrstv
    from synthetic import batch_recipes, flat, make_cube

    builder.build()
    recs = batch_recipes(BATCH["count"], BATCH["seed"])
    shapes = [r.shape for r in recs]
    Ys = [torch.from_numpy(flat(make_cube(r, 5000 + i)[1])).cuda() for i, r in enumerate(recs)]
    flags = lrstv.FLAG_WARM_START if args.jacobi_start == "warm" else 0
    if args.jacobi_order == "fixed":
        flags |= lrstv.FLAG_JACOBI_FIXED_ORDER
    params = [lrstv.Params.make(sh[0], sh[1], max_iter=BATCH["iters"], flags=flags)
              for sh in shapes]
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with lrstv.Batch(shapes, params) as b:
        b.init(Ys)
        done = 0
        for _ in range(args.warmup):
            b.iterate(1)
            done += 1
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        first = done
        t0, t1 = ev(), ev()
        t0.record(stream)
        for _ in range(args.steps):  # the profiler is off in the timed pass
            if done >= BATCH["iters"]:
                b.init(Ys)
                done = 0
            b.iterate(1)
            done += 1
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        clk = clocks.stop()
        unconv = sum(b.plan(i).stats().jacobi_unconverged for i in range(len(shapes)))
        # profiled pass over the same iterations of the denoise, for the
        # persistent Jacobi's share (cube 0's profile) and the launches of a
        # step (every group's launches are in the profile of its first cube)
        ngroups, _ = b.groups()
        b.init(Ys)
        for _ in range(first):
            b.iterate(1)
        plans = [b.plan(i) for i in range(len(shapes))]
        for p in plans:
            p.profile_enable(True)
        p0 = plans[0]
        q0, q1 = ev(), ev()
        q0.record(stream)
        done = first
        for _ in range(args.steps):
            if done >= BATCH["iters"]:
                b.init(Ys)
                done = 0
            b.iterate(1)
            done += 1
        q1.record(stream)
        torch.cuda.synchronize()
        ms_prof = q0.elapsed_time(q1)
        prof = p0.profile_read()
        spans = sum(sum(p.profile_read().launches) for p in plans)
        for p in plans:
            p.profile_enable(False)
    # unbatched comparison: the same cubes, one plan after another, over the
    # iterations right after the batch's warm-up (the first iterations, whose
    # thresholds cut every singular value, run no Jacobi sweep)
    single_ms = 0.0
    k_single = 3
    for i, sh in enumerate(shapes):
        with lrstv.Plan(*sh, params[i]) as pl:
            pl.init(Ys[i])
            pl.iterate(args.warmup)
            a, c = ev(), ev()
            a.record(stream)
            pl.iterate(k_single)
            c.record(stream)
            torch.cuda.synchronize()
            single_ms += a.elapsed_time(c) / k_single
    n = len(shapes)
    value = n * args.steps / (ms / 1e3)
    slices = sum(3 * (sh[2] // 2 + 1) for sh in shapes)
    return {
        "metric": METRIC_BATCH, "value": value,
        "unit": UNIT_BATCH, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH["desc"], "cubes": n,
                   "shapes": {f"{a}x{b_}x{c}": shapes.count((a, b_, c)) for (a, b_, c) in sorted(set(shapes))},
                   "fourier_slices_per_step": slices, "cubes_per_s": value / BATCH["iters"],
                   "jacobi_start": args.jacobi_start,
                   "groups": ngroups},
        "gpu_launches": int(spans),
        "launches_per_step": {"profiled": spans / args.steps, "groups": ngroups,
                              "note": "one launch per kernel and group of equal shape and "
                                      "parameters, one persistent Jacobi launch; the profiler "
                                      "brackets the DFT, GEMM, stencil and Jacobi launches"},
        "jacobi_persistent": {"launches": prof.launches[6],
                              "ms_per_launch": prof.ms[6] / max(prof.launches[6], 1),
                              "share_of_step": prof.ms[6] / max(ms_prof, 1e-9),
                              "unconverged_slices": unconv,
                              "measured": "a profiled pass over the same iterations, after the timed one"},
        "window": f"iterations {first}..{first + args.steps - 1} of each 50-iteration denoise (re-initialised at 50)",
        "unbatched": {"ms_per_step": single_ms, "speedup_of_batch": single_ms / (ms / args.steps)},
        "clocks": clk,
    }


UNROLL = {"batch": 8, "iters": 10, "pool": 2000, "seed": 5,
          "desc": "unrolled plain LRSTV, 10 iterations with 40 learnable scalars (tau, alpha, lambda, mu per iteration), batch 8 of 64x64x31 synthetic pairs (4 endmembers, 12 Voronoi cells, Gaussian 0.1 + 10% impulse), MSE to the clean cube, Adam on the log-scalars, warm-started Jacobi"}


def run_unroll(args):
    """The differentiable unrolled form: one step = forward (10 iterations,
    iterates kept; SVD factors kept, or recomputed in the backward pass with
    --unroll-factors recompute) + backward (hand-written adjoint) + an Adam
    update of the 40 log-scalars, on the next batch of 8 pairs from a pool
    resident in HBM.  value = training steps per second."""
    import numpy as np
    import torch

    from paper_2204_12879_gb300 import builder
    from paper_2204_12879_gb300.unrolled import UnrolledLRSTV
    from synthetic import RECIPES, make_cube

    builder.build()
    rec = RECIPES["c5"]
    n1, n2, n3 = rec.shape
    B, K = UNROLL["batch"], UNROLL["iters"]
    pairs = [make_cube(rec, 70000 + i) for i in range(UNROLL["pool"])]
    to_dev = lambda cubes: torch.from_numpy(np.ascontiguousarray(
        np.stack([c.astype(np.float32).transpose(2, 1, 0) for c in cubes]))).cuda()
    clean = to_dev([c for c, _ in pairs])
    noisy = to_dev([y for _, y in pairs])
    nb = UNROLL["pool"] // B
    from paper_2204_12879_gb300 import lrstv
    recompute = args.unroll_factors == "recompute"
    model = UnrolledLRSTV(n1, n2, n3, batch=B, iters=K, flags=lrstv.FLAG_WARM_START | (
        lrstv.FLAG_UNROLL_RECOMPUTE if recompute else 0))
    opt = torch.optim.Adam(model.parameters(), lr=0.02)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(i, marks=None):
        sl = slice((i % nb) * B, (i % nb + 1) * B)
        opt.zero_grad(set_to_none=True)
        X = model(noisy[sl])
        loss = ((X - clean[sl]) ** 2).mean()
        if marks is not None:
            marks[0].record(stream)
        loss.backward()
        opt.step()
        return loss

    losses = []
    for i in range(args.warmup):
        losses.append(float(step(i)))
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0, t1 = ev(), ev()
    mids = [ev() for _ in range(args.steps)]
    starts = [ev() for _ in range(args.steps)]
    ends = [ev() for _ in range(args.steps)]
    t0.record(stream)
    last = None
    for i in range(args.steps):
        starts[i].record(stream)
        last = step(args.warmup + i, marks=[mids[i]])
        ends[i].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    fwd = sum(starts[i].elapsed_time(mids[i]) for i in range(args.steps)) / args.steps
    bwd = sum(mids[i].elapsed_time(ends[i]) for i in range(args.steps)) / args.steps
    unconv, gerr = model.handle.stats()
    value = args.steps / (ms / 1e3)
    return {
        "metric": METRIC_UNROLL,
        "value": value, "unit": UNIT_UNROLL, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": UNROLL["desc"], "shape": [n1, n2, n3], "batch": B,
                   "unrolled_iters": K, "learnable_scalars": 4 * K,
                   "svd_factors": ("recomputed in the backward pass" if recompute
                                   else "kept from the forward pass"),
                   "pool": f"{UNROLL['pool']} pairs resident in HBM, cycled",
                   "cubes_per_s": value * B, "cube_iterations_per_s": value * B * K},
        "phases": {"forward_ms": fwd, "backward_and_update_ms": bwd,
                   "arena_bytes": model.handle.nbytes},
        "loss": {"first_warmup": losses[0] if losses else None, "last": float(last)},
        "unconverged_slices": unconv, "gemm_errors": gerr,
        "clocks": clk,
    }


def oracle_baseline(wl, Y, budget_s=25.0, max_iters=None, ranks=None):
    """Times the FP64 oracle (as it stands) on the same cube: whole ADMM
    iterations from the initial state until the time budget is spent; with
    ranks, the full TDLRSTV iteration (Tucker L-update of oracle/tucker.py)."""
    import numpy as np

    import oracle
    r = Y.shape
    params = oracle.Params(n1=r[0], n2=r[1])
    if ranks:
        from oracle import tucker
        st = tucker.TuckerState(oracle, Y.astype(np.float64), params, ranks)
    else:
        st = oracle.State(Y.astype(np.float64), params)
    done, t = 0, 0.0
    while (t < budget_s or done == 0) and (max_iters is None or done < max_iters):
        a = time.perf_counter()
        st.iterate(1)
        t += time.perf_counter() - a
        done += 1
    what = "TDLRSTV iteration(s), Tucker ranks %s," % (ranks,) if ranks else "ADMM iteration(s)"
    return {"value": done / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} {what} of the {r[0]}x{r[1]}x{r[2]} cube from its initial state ({t:.1f} s)"}


def _reference_line(args, world, metric, unit, cb, config, steps):
    """The reference arm's line: `steps` is the number of units actually
    timed (a bounded sample), each one step of the line; the FP64 CPU oracle
    has nothing to warm up (no caches to fill, no compilation), so none is
    run and warmup is 0."""
    config = dict(config, warmup_note="the CPU oracle runs no warm-up step")
    return {
        "impl": "reference", "metric": metric, "value": cb["value"], "unit": unit,
        "n_gpus": world, "steps": steps, "warmup": 0,
        "ms_per_step": 1e3 / cb["value"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def _reference_batch(args, world):
    """The FP64 oracle on the batch's cubes (the GPU arm's recipes and seeds):
    one ADMM iteration of each cube from its initial state, in batch order,
    until the time budget is spent; cube-iterations per second."""
    import numpy as np

    import oracle
    from synthetic import batch_recipes, make_cube
    recs = batch_recipes(BATCH["count"], BATCH["seed"])
    budget = args.cpu_budget * 4
    done, t = 0, 0.0
    for i, r in enumerate(recs):
        if done and t >= budget:
            break
        Y = make_cube(r, 5000 + i)[1].astype(np.float32).astype(np.float64)
        st = oracle.State(Y, oracle.Params(n1=r.shape[0], n2=r.shape[1]))
        a = time.perf_counter()
        st.iterate(1)
        t += time.perf_counter() - a
        done += 1
    cb = {"value": done / t, "unit": UNIT_BATCH, "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"one ADMM iteration of each of the first {done} of the batch's "
                    f"{len(recs)} cubes, from their initial states ({t:.1f} s)"}
    return _reference_line(args, world, METRIC_BATCH, UNIT_BATCH, cb,
                           {"workload": BATCH["desc"], "cubes_timed": done,
                            "step": "one ADMM iteration of one cube",
                            "note": "FP64 CPU oracle on the host cores, one cube after another"},
                           done)


def _reference_unroll(args, world):
    """The FP64 reference of the unrolled iteration and its hand-derived
    adjoint (oracle/adjoint.py) on the GPU arm's pairs: forward with the
    iterates kept and backward to the 40 scalars, one pair after another
    until the time budget is spent.  A training step is a batch of pairs (the
    update of 40 scalars is negligible): steps/s = pairs/s / batch."""
    import numpy as np

    from oracle import adjoint
    from synthetic import RECIPES, make_cube
    rec = RECIPES["c5"]
    n1, n2, n3 = rec.shape
    B, K = UNROLL["batch"], UNROLL["iters"]
    # the solver's default scalars: tau, alpha, lambda = 1 / sqrt(n1 n2), mu_k = 1e-2 1.5^k
    thetas = np.array([[1e-3, 0.2, 1.0 / np.sqrt(n1 * n2), min(1e-2 * 1.5 ** k, 1e6)]
                       for k in range(K)])
    budget = args.cpu_budget * 4
    done, t = 0, 0.0
    while done == 0 or (t < budget and done < UNROLL["pool"]):
        clean, noisy = make_cube(rec, 70000 + done)
        c = clean.astype(np.float32).astype(np.float64)
        y = noisy.astype(np.float32).astype(np.float64)
        a = time.perf_counter()
        adjoint.unrolled_loss_grad(y, c, thetas)
        t += time.perf_counter() - a
        done += 1
    value = done / t / B
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cb = {"value": value, "unit": UNIT_UNROLL, "cores": cores, "kind": "oracle",
          "sample": f"forward and backward of {done} pair(s) of {n1}x{n2}x{n3}, {K} iterations "
                    f"each ({t:.1f} s; numpy FP64, LAPACK threads up to the {cores} cores)"}
    return _reference_line(args, world, METRIC_UNROLL, UNIT_UNROLL, cb,
                           {"workload": UNROLL["desc"], "pairs_timed": done,
                            "step": f"forward and backward of {B} pairs (one training step)",
                            "note": "FP64 CPU reference of the unrolled iteration and its adjoint"},
                           max(1, done // B))


def run_reference(args, wl_name):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    if wl_name == "c4":
        return _reference_batch(args, world)
    if wl_name == "c5":
        return _reference_unroll(args, world)
    wl = WORKLOADS[wl_name]
    shape, clean, Y = make_input(wl, 0)
    ranks = tucker_ranks(args, shape)
    cb = oracle_baseline(wl, Y, budget_s=args.cpu_budget * 4, max_iters=max(args.steps, 1),
                         ranks=ranks)
    steps_run = int(cb["sample"].split()[0])
    config = {"workload": wl["desc"], "shape": list(shape), "iters_per_cube": wl["iters"],
              "step": (f"one ADMM iteration of the cube from its initial state (a bounded "
                       f"sample of the {wl['iters']}-iteration denoise the GPU arm's step runs)"),
              "note": "FP64 CPU oracle on the host cores; the metric (iterations/s) is the GPU arm's"}
    if ranks:
        config["tucker_ranks"] = list(ranks)
    return _reference_line(args, world, metric_for(args, wl_name), UNIT, cb, config, steps_run)


def run_micro(args):
    """One standalone operator, for kernel captures: `tsvt` runs lrstv_tsvt on
    a seeded random cube of --shape three times and prints its last time."""
    import numpy as np
    import torch

    from paper_2204_12879_gb300 import builder, lrstv
    builder.build()
    shape = tuple(int(x) for x in args.shape.split(","))
    N = shape[0] * shape[1] * shape[2]
    A = torch.from_numpy(np.random.default_rng(0).standard_normal(N).astype(np.float32)).cuda()
    sweeps, ms = 0, 0.0
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        out = lrstv.lrstv_tsvt(A, shape, 1.0)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e)
    _, sweeps = lrstv.lrstv_tsvt(A, shape, 1.0, out=out, sweeps=True)
    print(json.dumps({"micro": "tsvt", "shape": list(shape), "t": 1.0, "ms": ms,
                      "sweeps": sweeps, "slices": shape[2] // 2 + 1}))


def run_sweep_profile(args):
    """One warm-started denoise of the workload, printing after every ADMM
    iteration the distribution of the Jacobi's per-slice sweep counts (all
    slices of an E-step run concurrently, one CTA each, so the slowest slice
    sets the E-step's time)."""
    import numpy as np
    import torch

    from paper_2204_12879_gb300 import builder, lrstv
    from synthetic import flat

    builder.build()
    lrstv.load()
    wl = WORKLOADS[args.workload]
    shape, _, Y = make_input(wl, 0)
    n1, n2, n3 = shape
    y = torch.from_numpy(flat(Y)).cuda()
    flags = lrstv.FLAG_WARM_START if args.jacobi_start == "warm" else 0
    if args.jacobi_order == "fixed":
        flags |= lrstv.FLAG_JACOBI_FIXED_ORDER
    with lrstv.Plan(n1, n2, n3, lrstv.Params.make(n1, n2, max_iter=wl["iters"], flags=flags)) as pl:
        if args.tucker:
            pl.set_tucker((max(1, round(0.8 * n1)), max(1, round(0.8 * n2)), min(args.tucker, n3)))
        pl.init(y)
        for it in range(wl["iters"]):
            pl.iterate(1)
            sw = np.abs(pl.slice_sweeps())
            torch.cuda.synchronize()
            print(json.dumps({"iteration": it, "max": int(sw.max()), "median": float(np.median(sw)),
                              "mean": round(float(sw.mean()), 3),
                              "slowest_slice": [int(v) for v in np.unravel_index(sw.argmax(), sw.shape)],
                              "histogram": np.bincount(sw.ravel()).tolist()}), flush=True)


def build_parser():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed steps; a step of c1-c3 is one whole denoise of the cube")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["c4", "c5"], default="c2",
                    help="c4 = the batch of 64 uneven cubes, c5 = the unrolled, "
                         "differentiable form (training steps)")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle time for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the FP32 / tensor-pipe throughput probes (peaks then derived)")
    ap.add_argument("--jacobi-start", choices=["cold", "warm"], default="warm",
                    help="start each E-step's Jacobi SVDs from the identity or from the "
                         "previous E-step's singular vectors (LRSTV_FLAG_WARM_START)")
    ap.add_argument("--tucker", type=int, default=0, metavar="R3",
                    help="full TDLRSTV: Tucker L-update with ranks (0.8 n1, 0.8 n2, R3)")
    ap.add_argument("--precision", choices=["auto", "tf32x3", "bf16x3"], default="auto",
                    help="tensor-core GEMM split: 3xTF32 (FP32-accurate) or 3xBF16 "
                         "(LRSTV_FLAG_BF16X3); auto = 3xBF16 for c3 only")
    ap.add_argument("--dft", choices=["tc", "simt"], default="tc",
                    help="mode-3 DFT engine: the tensor-core pipeline or the SIMT direct sums "
                         "(LRSTV_FLAG_SIMT_DFT)")
    ap.add_argument("--jacobi-schedule", choices=["tasks", "slice"], default="tasks",
                    help="the Jacobi's task-graph schedule over all SMs, or one CTA per slice "
                         "(LRSTV_FLAG_JACOBI_PER_SLICE)")
    ap.add_argument("--jacobi-panel", type=int, choices=[32, 16], default=32,
                    help="the Jacobi's column panel width: 32 (16-warp CTAs) or 16 (8-warp CTAs, "
                         "two to an SM; LRSTV_FLAG_JACOBI_PANEL16)")
    ap.add_argument("--jacobi-order", choices=["sorted", "fixed"], default="sorted",
                    help="the Jacobi orders each sweep's columns by norm, largest first, or "
                         "keeps their stored order (LRSTV_FLAG_JACOBI_FIXED_ORDER)")
    ap.add_argument("--unroll-factors", choices=["keep", "recompute"], default="keep",
                    help="c5: keep every iteration's SVD factors from the forward pass, or "
                         "recompute them in the backward pass (LRSTV_FLAG_UNROLL_RECOMPUTE)")
    ap.add_argument("--micro", choices=["tsvt"], default=None,
                    help="time one standalone operator instead of the iteration")
    ap.add_argument("--shape", default="200,200,16", help="n1,n2,n3 for --micro")
    ap.add_argument("--sweep-profile", action="store_true",
                    help="print the per-slice Jacobi sweep distribution of every iteration of one "
                         "denoise (c1-c3) instead of timing")
    return ap


def main(argv=None):
    ap = build_parser()
    args = ap.parse_args(argv)
    if args.micro:
        run_micro(args)
        return
    if args.sweep_profile:
        run_sweep_profile(args)
        return
    if args.workload == "c4" and args.impl == "ours":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.workload == "c5" and args.impl == "ours":
        print(json.dumps(run_unroll(args)), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    line = (run_reference if args.impl == "reference" else run_ours)(args, args.workload)
    if line is not None:
        print(json.dumps(line), flush=True)
    _, world, _ = dist_env()
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
