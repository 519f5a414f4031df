"""Benchmark of the SE(2,N) inpainting hot path on GB300.

One step = one whole inpaint of the 512x512, N=32 workload (seeded
piecewise-smooth image, 80 % random mask plus 4-px bars every 32 px,
beta = 0.25, 10 restoration intervals of 500 Crank-Nicolson steps, T = 2 per
interval): orientation, lift, the 2-D DFT, 10 x diffusion, 9 x (inverse
DFT, static restoration, forward DFT), inverse DFT, projection, all through
se2n_inpaint with the inputs resident in HBM. By default each interval's
500 steps are applied as one precomputed S-step propagator per class of
frequencies, built inside every timed inpaint, and each interval runs as
one column pass (DFT along y, propagators, inverse DFT) and one row pass
(real DFTs along x around the restoration) (--diffusion propagator);
--diffusion steps runs the fused step-by-step kernel between cuFFT
transforms instead, and the default line reports that path too.

Metric: Mathieu updates per second over the whole inpaint time (value),
counting the frequencies the path integrates: the lifted volume is real, so
the H x (W/2 + 1) frequencies of the Hermitian half carry the whole
spectrum, and updates = 512 * 257 * 32 * 500 * 10 per inpaint (on the
propagator path these are equivalent updates: each interval's 500 steps
are applied as one precomputed map). The count over all M^2 frequencies
that the method's own formulation integrates is reported beside it
(m2_updates_per_s). Plus ms per inpaint (the first figure of the line), the FP32 error against the FP64 oracle, the roofline of the
dominant kernel (the column pass against the measured copy rate, with the
row pass and the propagator build beside it; or the step kernel, FP32 ALU
bound, whose flops are those of the frequencies it integrates, the
Hermitian half 512 x 257 of the spectrum), the end-to-end number from host
buffers (se2n_inpaint_host) and the oracle's CPU rate.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload 512|dr|batch|surrogate|unet-forward] [--diffusion propagator|steps]
Multi-GPU (torchrun): every rank inpaints its own image (replicas, weak
scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Mathieu updates/s (M²·N·steps); ms per 512² N=32 inpaint, err vs FP64"
UNIT = "updates/s"
FLOPS_PER_UPDATE = 22          # per complex angle per CN step: 2 x (1 add + 5 FMA)
GOLDEN = os.path.join(ROOT, "tests", "golden", "curves_noise_512_N32.npz")
L2_FLUSH_BYTES = 256 << 20
SM_COUNT, FP32_LANES_PER_SM = 152, 128


def _workload():
    return synth.workload_512()


def integrated_updates(H, W, N, steps, rounds):
    """Crank-Nicolson updates of one inpaint over the frequencies the path
    integrates: the Hermitian half, H x (W/2 + 1) frequencies, N angles,
    `steps` steps in each of `rounds` intervals."""
    return H * (W // 2 + 1) * N * steps * rounds


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


GOLDEN_DYNAMIC = os.path.join(ROOT, "tests", "golden", "curves_noise_512_N32_dynamic.npz")
GOLDEN_GUARD0 = os.path.join(ROOT, "tests", "golden", "curves_noise_512_N32_guard0.npz")
GOLDEN_N30 = os.path.join(ROOT, "tests", "golden", "curves_noise_512_N30.npz")
SENSITIVITY_N30 = os.path.join(ROOT, "tests", "golden", "sensitivity_512_N30.json")
SENSITIVITY = os.path.join(ROOT, "tests", "golden", "sensitivity_512_N32.json")


def fp32_sensitivity(path=SENSITIVITY):
    """The FP64 oracle's sensitivity to FP32 rounding on the 512x512 workload
    (written by tests/golden/make_sensitivity.py), or None."""
    try:
        s = json.load(open(path))
    except (OSError, ValueError):
        return None
    out = {k: s[k]["max_abs_over_max_f"] for k in ("storage_full", "perturb_full", "fp32_full", "fp32_half")}
    out["s32"] = max(out["fp32_half"], out["fp32_full"])
    return out


def _config(w, extra=None, dynamic=False):
    cfg = {
        "workload": f"curves_noise_512_N32{'_dynamic' if dynamic else ''}: {w.H}x{w.W} image, N={w.N}, "
                    f"beta={w.beta}, {w.rounds} restoration intervals x {w.steps} CN steps, T={w.T}, eps={w.eps}, "
                    "80% random mask + 4-px bars every 32 px"
                    + (", dynamic restoration (Section 5.3)" if dynamic else ""),
        "updates_per_step": integrated_updates(w.H, w.W, w.N, w.steps, w.rounds),
        "updates_basis": "H x (W/2 + 1) frequencies (the Hermitian half the path integrates) x N x steps x "
                         "intervals; the method's M^2 count is m2_updates_per_step",
        "m2_updates_per_step": w.updates(),
        "l2": "flushed between timed steps (256 MiB write)",
        "parallelism": "replicas",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"se2n_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines()]
        except OSError:
            return None
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = [float(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        load = [s for s in sm if s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

KERNEL_SOURCES = {"diffuse": ("diffuse_impl.cuh", "diffuse_x2.cuh", "diffuse.cu"),
                  "prop_build": ("propagator.cu", "prop_classes.cuh", "diffuse_x2.cuh", "diffuse_impl.cuh"),
                  "col_prop": ("colprop.cu", "bulk_copy.cuh", "rowdft.cuh", "smem_fft.cuh", "prop_classes.cuh", "diffuse_x2.cuh"),
                  "row_pass": ("rowfft.cu", "smem_fft.cuh", "restore.cuh"),
                  "prop_build_wide": ("propagator.cu", "prop_classes.cuh", "diffuse_x2.cuh", "diffuse_impl.cuh"),
                  "prop_apply_tiled": ("propagator.cu", "prop_classes.cuh", "diffuse_x2.cuh", "diffuse_impl.cuh")}
TRAFFIC_FILES = {"diffuse": "diffuse_traffic.json", "prop_build": "prop_build_traffic.json",
                 "col_prop": "col_prop_traffic.json", "row_pass": "row_pass_traffic.json",
                 "prop_build_wide": "prop_build_wide_traffic.json",
                 "prop_apply_tiled": "prop_apply_tiled_traffic.json"}


def kernel_source_hash(kind="diffuse"):
    """Hash of a kernel's source files: a stored DRAM-traffic figure is only
    valid for the exact kernel it was captured on."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_1304_2062_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_record(kind):
    """The committed ncu traffic record of the kernel, or None if it was taken
    on a different kernel source."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", TRAFFIC_FILES[kind])))
    except (OSError, ValueError):
        return None
    return rec if rec.get("kernel_source_hash") == kernel_source_hash(kind) else None


def stored_traffic(kind="diffuse"):
    """DRAM bytes per launch of the kernel from the committed ncu summary, or
    None if it was taken on a different kernel source."""
    rec = stored_record(kind)
    return rec.get("dram_bytes_per_launch") if rec else None


def propagator_gemm_flops(classes, N, S):
    """FP32 flops of building the S-step propagators and the products a class:
    every op of the library's powering program but its copies is one
    N x N x N product (2 N^3 flops); the O(N^2) solves of the first step are
    not counted."""
    from paper_1304_2062_gb300 import se2n
    ops, _ = se2n.se2n_prop_chain(S)
    products = sum(o != se2n.PROP_COPY for o in ops)
    return classes * products * 2 * N ** 3, products


def propagator_classes(H, W, half=True):
    """Classes of frequencies that share one propagator: row slots s in
    [0, H/4] (rows s, H/2 - s, and H/2 + s, H - s reversed) times column
    pairs l and (W/2 - l) (Hermitian half: l <= W/2)."""
    row_slots = H // 4 + 1
    cols = W // 4 + 1 if half else W // 4 + 1 + (3 * W) // 4 - W // 2
    return row_slots * cols


def propagator_build_items(H, W, half=True):
    """Classes the build computes: on square planes (Hermitian half) a class
    and its transpose share one build, so n (n + 1) / 2 of the n x n slot
    pairs; otherwise every class."""
    if half and H == W:
        n = W // 4 + 1
        return n * (n + 1) // 2
    return propagator_classes(H, W, half)


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_items, rank, world):
    """Independent images dealt to ranks round-robin: every image goes to
    exactly one rank, and rank loads differ by at most one image."""
    return list(range(rank, n_items, world))


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1304_2062_gb300 import se2n

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = _workload()
    f32 = w.f.astype(np.float32)
    stream = torch.cuda.Stream(dev)
    plan = se2n.se2n_plan_create(w.H, w.W, w.N, 0, stream)
    dynamic = args.workload == "dr"
    prop = args.diffusion == "propagator"
    flags = se2n.SE2N_DIFFUSE_PROPAGATOR if prop else 0
    prm = se2n.se2n_params_default(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps,
                                   sigma_smooth=w.sigma, dynamic=int(dynamic), diffuse_flags=flags)
    f_d = torch.tensor(f32, device=dev)
    m_d = torch.tensor(w.mask, device=dev)
    vol = torch.empty((w.N, w.H, w.W), dtype=torch.complex64, device=dev)
    out = torch.empty((w.H, w.W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        # every step builds its propagators again: the timed inpaint is one
        # whole problem, nothing carried over from the previous step
        if prop:
            se2n.se2n_plan_drop_propagators(plan)
        se2n.se2n_inpaint(plan, f_d, m_d, None, prm, vol, out)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local_rank) as clocks:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        # the same K steps again with the plan's stage events on (a CUDA event
        # pair around every launch of a stage, on the plan's stream): the
        # kernels' launch times for the rooflines. The events cost about 0.1 ms
        # an inpaint, so the steps above, whose time is the result, run
        # without them.
        se2n.se2n_plan_profile(plan, True)
        for i in range(args.steps):
            flush.zero_()
            step()
        torch.cuda.synchronize(dev)
        prof = se2n.se2n_plan_profile_read(plan, reset=True)
        se2n.se2n_plan_profile(plan, False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / args.steps
    upd = integrated_updates(w.H, w.W, w.N, w.steps, w.rounds)
    value = world * upd * args.steps / (total_ms / 1e3)

    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    peak_basis = "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (derived, not measured)"
    # the path integrates the Hermitian half of the spectrum: H x (W/2 + 1) frequencies
    updates_per_launch = w.H * (w.W // 2 + 1) * w.N * w.steps
    if prop:
        # every interval is one column pass (DFT along y, propagators, inverse
        # DFT along y) and one row pass (inverse real DFT along x, restoration,
        # forward real DFT along x); the propagators are built once. The
        # column passes take the largest share of the inpaint.
        c_ms, c_calls = prof["diffuse"]
        c_s = c_ms / c_calls / 1e3
        r_ms, r_calls = prof["fft"]
        r_s = r_ms / r_calls / 1e3
        b_ms, b_calls = prof["propagator"]
        b_s = b_ms / b_calls / 1e3
        classes = propagator_classes(w.H, w.W)
        wc = w.W // 2 + 1
        spec_bytes = 8 * wc * w.H * w.N
        # the method's bytes: the half spectrum in and out, and every class's
        # propagator once as its N (N + 1) / 2 distinct entries (the kernel
        # reads the stored rows, 4 N^2 bytes a class: stored_bytes_per_launch)
        col_bytes = 2 * spec_bytes + 4 * (w.N * (w.N + 1) // 2) * classes
        col_stored_bytes = 2 * spec_bytes + 4 * w.N * w.N * classes
        row_bytes = 2 * spec_bytes + 6 * w.H * w.W
        col_flops = 2 * wc * w.N * 5 * w.H * int(math.log2(w.H)) + 4 * w.N * w.N * w.H * wc
        items = propagator_build_items(w.H, w.W)
        flops, products = propagator_gemm_flops(items, w.N, w.steps)
        # the symmetric build (N = 16, 32) computes the 10 upper-triangle 8 x 8
        # tiles of the 16 of every product and mirrors them
        exec_flops = flops * 10 // 16 if w.N in (16, 32) else flops
        hbm = _peaks().get("hbm_gbs")
        hbm_basis = "MEASURED_PEAKS.json hbm_gbs (copy, burst)"
        roofline = {"bound": "hbm", "achieved": round(col_bytes / c_s / 1e9, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(col_bytes / c_s / 1e9 / hbm, 4) if hbm else None,
                    "traffic": args.traffic if args.traffic is not None else stored_traffic("col_prop"),
                    "kernel": f"k_col_tma<{w.N},{w.H}> (column pass: DFT along y, x <- x + D_S x, inverse DFT; "
                              "whole columns in shared memory, bulk copies in and out, one persistent block an SM)",
                    "bytes_per_launch": col_bytes,
                    "bytes_basis": "one read and one write of the row-transformed half spectrum (8 (W/2+1) H N "
                                   "bytes each) + every class's symmetric propagator once, as its N (N + 1) / 2 "
                                   "distinct entries (4 N (N + 1) / 2 bytes a class)",
                    "stored_bytes_per_launch": col_stored_bytes,
                    "stored_basis": "the propagators as the kernel reads them, full rows (4 N^2 bytes a class)",
                    "avg_launch_ms": round(c_s * 1e3, 4), "peak_basis": hbm_basis,
                    "flops_per_launch": col_flops,
                    "flops_basis": "2 (W/2+1) N complex DFTs of length H at 5 H log2 H + 4 N^2 a frequency",
                    "frac_of_fp32_peak": round(col_flops / c_s / 1e12 / peak, 4),
                    "row_pass": {"kernel": f"k_row<{w.N},{w.W}> (inverse real DFT along x, restoration, forward "
                                           "real DFT; one block a row)", "bound": "hbm",
                                 "avg_launch_ms": round(r_s * 1e3, 4), "bytes_per_launch": row_bytes,
                                 "bytes_basis": "one read and one write of the half spectrum + f, mask, bins",
                                 "achieved_gbs": round(row_bytes / r_s / 1e9, 1), "peak_gbs": hbm,
                                 "frac": round(row_bytes / r_s / 1e9 / hbm, 4) if hbm else None,
                                 "traffic": stored_traffic("row_pass")},
                    "build": {"kernel": f"k_prop_build_sym<{w.N}> ({items} of the {classes} classes computed, each "
                                        "also stored permuted for its transpose; FP32 symmetric products; on a side "
                                        "stream, overlapping the orientation and the first row pass)",
                              "bound": "alu",
                              "avg_launch_ms": round(b_s * 1e3, 4),
                              "flops_basis": "executed flops: classes built x products x 2 N^3 x 10/16 (the symmetric "
                              "kernel computes the 10 upper-triangle 8x8 tiles of 16 and mirrors them), "
                              f"S = {w.steps}: {products} products (se2n_prop_chain's program; binary powering "
                              f"takes {w.steps.bit_length() - 1 + bin(w.steps).count('1') - 1})",
                              "flops_per_launch": exec_flops,
                              "full_product_flops_per_launch": flops,
                              "achieved_tflops": round(exec_flops / b_s / 1e12, 3), "peak_tflops": round(peak, 3),
                              "frac": round(exec_flops / b_s / 1e12 / peak, 4), "peak_basis": peak_basis,
                              "frac_full_product_equivalent": round(flops / b_s / 1e12 / peak, 4),
                              "traffic": stored_traffic("prop_build")},
                    "frequencies_integrated": "Hermitian half, H x (W/2 + 1)"}
    else:
        d_ms, d_calls = prof["diffuse"]
        d_avg_s = d_ms / d_calls / 1e3
        achieved = FLOPS_PER_UPDATE * updates_per_launch / d_avg_s / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4),
                    "traffic": args.traffic if args.traffic is not None else stored_traffic(),
                    "kernel": "k_diffuse_x2<32,2,false> (packed FP32 pairs, truncated corner correction)",
                    "flops_per_update": FLOPS_PER_UPDATE, "updates_per_launch": updates_per_launch,
                    "avg_launch_ms": round(d_avg_s * 1e3, 4), "peak_basis": peak_basis,
                    "diffuse_updates_per_s": updates_per_launch / d_avg_s,
                    "hbm_gbs_of_diffuse": round(16 * w.H * (w.W // 2 + 1) * w.N / d_avg_s / 1e9, 1),
                    "frequencies_integrated": "Hermitian half, H x (W/2 + 1)"}
    stages = {k: {"ms_per_step": round(v[0] / args.steps, 4), "calls_per_step": v[1] / args.steps}
              for k, v in prof.items() if k != "kernels"}
    launches = int(prof["kernels"])

    cfg = _config(w, {"diffusion": "S-step propagators built every inpaint (SE2N_DIFFUSE_PROPAGATOR)" if prop
                      else "step by step, the fused Crank-Nicolson kernel"}, dynamic=dynamic)
    result = {"metric": METRIC, "ms_per_inpaint": round(ms_per_step, 4), "value": value, "unit": UNIT,
              "m2_updates_per_s": world * w.updates() * args.steps / (total_ms / 1e3),
              "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
              "roofline": roofline, "gpu_launches": launches, "stages_ms": stages,
              "stage_timing": "stages_ms and the rooflines' launch times come from the same K steps run again with "
                              "the plan's stage events on (CUDA events around each launch, plan stream); the timed "
                              "steps run without them (they add about 0.1 ms an inpaint)"}
    if prop:
        # the other two ways to run the same inpaint, on the same plan and inputs:
        # propagators kept from the previous call (serving one beta dt and S),
        # and the step-by-step kernel with its own roofline
        with torch.cuda.stream(stream):
            def timed3(fn):
                evs = []
                for _ in range(3):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    b.record(stream)
                    evs.append((a, b))
                torch.cuda.synchronize(dev)
                return sum(a.elapsed_time(b) for a, b in evs) / 3
            se2n.se2n_inpaint(plan, f_d, m_d, None, prm, vol, out)
            kept = timed3(lambda: se2n.se2n_inpaint(plan, f_d, m_d, None, prm, vol, out))
            # the passes' launch times from three more, with stage events on
            se2n.se2n_plan_profile(plan, True)
            timed3(lambda: se2n.se2n_inpaint(plan, f_d, m_d, None, prm, vol, out))
            kprof = se2n.se2n_plan_profile_read(plan, reset=True)
            se2n.se2n_plan_profile(plan, False)
            prm_s = se2n.se2n_params_default(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps,
                                             sigma_smooth=w.sigma, dynamic=int(dynamic))
            se2n.se2n_inpaint(plan, f_d, m_d, None, prm_s, vol, out)
            torch.cuda.synchronize(dev)
            se2n.se2n_plan_profile(plan, True)
            stepwise = timed3(lambda: se2n.se2n_inpaint(plan, f_d, m_d, None, prm_s, vol, out))
            sprof = se2n.se2n_plan_profile_read(plan, reset=True)
            se2n.se2n_plan_profile(plan, False)
        sd_s = sprof["diffuse"][0] / sprof["diffuse"][1] / 1e3
        s_ach = FLOPS_PER_UPDATE * updates_per_launch / sd_s / 1e12
        result["propagators_kept"] = {"ms_per_step": round(kept, 4), "value": world * upd / (kept / 1e3)}
        # the row and column passes timed where nothing runs beside them (in the
        # timed inpaints the build overlaps the orientation and the first row pass)
        c_s = kprof["diffuse"][0] / kprof["diffuse"][1] / 1e3
        r_s = kprof["fft"][0] / kprof["fft"][1] / 1e3
        hbm = roofline["peak"]
        col_bytes, row_bytes = roofline["bytes_per_launch"], roofline["row_pass"]["bytes_per_launch"]
        roofline.update({"achieved": round(col_bytes / c_s / 1e9, 1), "avg_launch_ms": round(c_s * 1e3, 4),
                         "frac": round(col_bytes / c_s / 1e9 / hbm, 4) if hbm else None,
                         "frac_of_fp32_peak": round(roofline["flops_per_launch"] / c_s / 1e12 / peak, 4),
                         "timed_on": "the inpaints that reuse the propagators (CUDA events around each launch)"})
        roofline["row_pass"].update({"avg_launch_ms": round(r_s * 1e3, 4),
                                     "achieved_gbs": round(row_bytes / r_s / 1e9, 1),
                                     "frac": round(row_bytes / r_s / 1e9 / hbm, 4) if hbm else None,
                                     "timed_on": "the inpaints that reuse the propagators; the average over all "
                                                 "row passes of an inpaint (lift and projection included)"})
        result["step_by_step"] = {
            "ms_per_step": round(stepwise, 4), "value": world * upd / (stepwise / 1e3),
            "roofline": {"bound": "alu", "kernel": "k_diffuse_x2<32,2,false>", "avg_launch_ms": round(sd_s * 1e3, 4),
                         "achieved": round(s_ach, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                         "frac": round(s_ach / peak, 4), "traffic": stored_traffic(),
                         "flops_per_update": FLOPS_PER_UPDATE, "updates_per_launch": updates_per_launch}}
    if dynamic:
        # with propagators the image value h and its argmax angle come from a
        # row pass (counted with the row passes); the growth kernel reads h,
        # the argmax and the set and updates set, references and bins: about
        # 16 bytes a pixel. Step by step, the growth step also reads the real
        # volume once (4 N bytes a pixel) for the maximum.
        dr_ms, dr_calls = prof["dr"]
        per_px = 16 if prop else 4 * w.N + 16
        dr_s = dr_ms / dr_calls / 1e3
        result["dynamic_restoration"] = {
            "growth_steps_per_inpaint": dr_calls / args.steps,
            "ms_per_growth_step": round(dr_s * 1e3, 4),
            "algorithmic_bytes_per_growth_step": per_px * w.H * w.W,
            "hbm_gbs": round(per_px * w.H * w.W / dr_s / 1e9, 1),
            "bytes_basis": ("16 bytes a pixel (h 4, argmax 1, set in and out 2, reference and bin read and "
                            "written 10); h and the argmax come from a row pass") if prop else
                           "4 N bytes a pixel (the real volume, read once) + 16 (h, argmax, set, reference)"}
    result["clocks"] = clocks.summary()

    # end to end from pinned host buffers through se2n_inpaint_host
    f_h = torch.tensor(f32).pin_memory()
    m_h = torch.tensor(w.mask).pin_memory()
    o_h = torch.empty((w.H, w.W), dtype=torch.float32).pin_memory()
    for _ in range(2):
        se2n.se2n_inpaint_host(plan, f_h.data_ptr(), m_h.data_ptr(), prm, o_h.data_ptr())
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        if prop:
            se2n.se2n_plan_drop_propagators(plan)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        se2n.se2n_inpaint_host(plan, f_h.data_ptr(), m_h.data_ptr(), prm, o_h.data_ptr())
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = statistics.median(e2e_ms)
    result["e2e"] = {"value": world * upd / (e2e_step / 1e3), "unit": UNIT,
                     "ms_per_step": e2e_step, "h2d_bytes_per_step": f32.nbytes + w.mask.nbytes,
                     "d2h_bytes_per_step": o_h.numel() * 4, "api": "se2n_inpaint_host (pinned host buffers)"}

    # error of this result against the FP64 oracle (stored reference, same inputs)
    golden = GOLDEN_DYNAMIC if dynamic else GOLDEN
    sens = fp32_sensitivity()
    if rank == 0 and os.path.exists(golden):
        g = np.load(golden)
        b_d = torch.tensor(g["bins"], device=dev)
        with torch.cuda.stream(stream):
            se2n.se2n_inpaint(plan, f_d, m_d, b_d, prm, vol, out)
            own = torch.empty_like(b_d)
            se2n.se2n_orient(plan, f_d, m_d, w.sigma, 1e-4, own)
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy().astype(np.float64)
        ref = g["out"].astype(np.float64)
        result["err_vs_fp64"] = {
            "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_over_max_f": float(np.abs(got - ref).max() / np.abs(w.f).max()),
            "bins": "oracle's (FP64) bins given to both sides",
            "own_bin_mismatches": int((own.cpu().numpy() != g["bins"]).sum()),
            "oracle_seconds_for_this_result": float(g["oracle_seconds"][0])}
        if sens:
            result["err_vs_fp64"]["bound"] = {
                "max_abs_over_max_f": 4.0 * sens["s32"],
                "basis": "4 x S32, S32 = the largest change of the FP64 oracle's own result when its transforms run "
                         "in FP32 and its volume is stored in FP32 (tests/golden/sensitivity_512_N32.json: "
                         f"{sens['fp32_half']:.2e} on the Hermitian half, {sens['fp32_full']:.2e} on the full "
                         f"spectrum; FP32 storage alone {sens['storage_full']:.2e})",
                "within": result["err_vs_fp64"]["max_abs_over_max_f"] <= 4.0 * sens["s32"]}
        if not dynamic and os.path.exists(GOLDEN_GUARD0):
            # the paper's restoration rule as printed (no relative guard)
            g0 = np.load(GOLDEN_GUARD0)
            prm0 = se2n.se2n_params_default(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps,
                                            sigma_smooth=w.sigma, diffuse_flags=flags, guard=0.0)
            with torch.cuda.stream(stream):
                se2n.se2n_inpaint(plan, f_d, m_d, torch.tensor(g0["bins"], device=dev), prm0, vol, out)
            torch.cuda.synchronize(dev)
            got0 = out.cpu().numpy().astype(np.float64)
            ref0 = g0["out"].astype(np.float64)
            result["err_vs_fp64"]["guard0"] = {
                "rel_l2": float(np.linalg.norm(got0 - ref0) / np.linalg.norm(ref0)),
                "max_abs_over_max_f": float(np.abs(got0 - ref0).max() / np.abs(w.f).max()),
                "rule": "sigma at every good pixel with h(t_i) > 0 (guard 0), against the oracle's guard-0 result"}

    if rank == 0 and prop and not dynamic:
        result["paper_angle_count"] = paper_angle_count(w, dev, stream, flush)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, dynamic=dynamic)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return result


def paper_angle_count(w, dev, stream, flush):
    """The same 512x512 inpaint with the paper's N = 30 angles (propagators
    built every inpaint, the row and column passes with the 30 angles in 32
    slots): ms per inpaint over 5 flushed runs and the error against the
    FP64 oracle's stored N = 30 result."""
    import torch

    from paper_1304_2062_gb300 import se2n
    w30 = synth.workload_512(N=30)
    f32 = w30.f.astype(np.float32)
    plan = se2n.se2n_plan_create(w30.H, w30.W, 30, 0, stream)
    f_d = torch.tensor(f32, device=dev)
    m_d = torch.tensor(w30.mask, device=dev)
    vol = torch.empty((30, w30.H, w30.W), dtype=torch.complex64, device=dev)
    out = torch.empty((w30.H, w30.W), dtype=torch.float32, device=dev)
    prm = se2n.se2n_params_default(N=30, beta=w30.beta, T=w30.T, steps=w30.steps, rounds=w30.rounds, eps=w30.eps,
                                   sigma_smooth=w30.sigma, diffuse_flags=se2n.SE2N_DIFFUSE_PROPAGATOR)
    res = {"N": 30, "workload": "the same image, mask and parameters with N = 30"}
    with torch.cuda.stream(stream):
        for _ in range(3):
            se2n.se2n_plan_drop_propagators(plan)
            se2n.se2n_inpaint(plan, f_d, m_d, None, prm, vol, out)
        ms = []
        for _ in range(5):
            flush.zero_()
            se2n.se2n_plan_drop_propagators(plan)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            se2n.se2n_inpaint(plan, f_d, m_d, None, prm, vol, out)
            b.record(stream)
            ms.append((a, b))
        torch.cuda.synchronize(dev)
    res["ms_per_inpaint"] = round(sum(a.elapsed_time(b) for a, b in ms) / len(ms), 4)
    res["timing"] = "CUDA events, L2 flushed and the propagators rebuilt before each of 5 inpaints"
    if os.path.exists(GOLDEN_N30):
        g = np.load(GOLDEN_N30)
        with torch.cuda.stream(stream):
            se2n.se2n_inpaint(plan, f_d, m_d, torch.tensor(g["bins"], device=dev), prm, vol, out)
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy().astype(np.float64)
        ref = g["out"].astype(np.float64)
        err = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
               "max_abs_over_max_f": float(np.abs(got - ref).max() / np.abs(w30.f).max())}
        sens = fp32_sensitivity(SENSITIVITY_N30)
        if sens:
            err["bound"] = {"max_abs_over_max_f": 4.0 * sens["s32"],
                            "basis": "4 x S32 of tests/golden/sensitivity_512_N30.json",
                            "within": err["max_abs_over_max_f"] <= 4.0 * sens["s32"]}
        res["err_vs_fp64"] = err
    plan.close()
    return res


# ----------------------------------------------------------------------------
# the 2048x2048, N=64 workload
# ----------------------------------------------------------------------------

GOLDEN_2048 = os.path.join(ROOT, "tests", "golden", "lines_patches_2048_N64.npz")


def run_2048(args, rank, world, local_rank):
    """2048x2048 lines-plus-texture image, N=64 (a 2 GiB complex64 volume),
    85 % of the pixels corrupted, one interval of 1000 Crank-Nicolson steps:
    the main run (beta = 0.25, T = 50) timed as the line's value, and the
    stiff run (beta = 10, T = 1000: beta dt = 10, split diagonal, with and
    without the FP64 Sherman-Morrison correction) beside it. Each step is one
    whole inpaint through se2n_inpaint (orientation, lift, transforms,
    diffusion, inverse, projection). Errors: the projected image against the
    FP64 oracle's stored result at every 4th row and column, and the
    diffused spectrum of the main run against the oracle's integration of a
    seeded sample of its frequencies (all 64 angles each)."""
    import torch

    from paper_1304_2062_gb300 import se2n

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(dev)
    w = synth.workload_2048(side=args.side)
    ws = synth.workload_2048(stress=True, side=args.side)
    f32 = w.f.astype(np.float32)
    plan = se2n.se2n_plan_create(w.H, w.W, w.N, 0, stream)
    prop = args.diffusion == "propagator"
    flags = se2n.SE2N_DIFFUSE_PROPAGATOR if prop else 0

    def params(wk, fl):
        return se2n.se2n_params_default(N=wk.N, beta=wk.beta, T=wk.T, steps=wk.steps, rounds=wk.rounds, eps=wk.eps,
                                        sigma_smooth=wk.sigma, diffuse_flags=fl)
    prm = params(w, flags)
    f_d = torch.tensor(f32, device=dev)
    m_d = torch.tensor(w.mask, device=dev)
    vol = torch.empty((w.N, w.H, w.W), dtype=torch.complex64, device=dev)
    out = torch.empty((w.H, w.W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(p):
        if prop:
            se2n.se2n_plan_drop_propagators(plan)
        se2n.se2n_inpaint(plan, f_d, m_d, None, p, vol, out)

    def timed(p, k, warm):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                step(p)
            torch.cuda.synchronize(dev)
            if dist:
                dist.barrier()
            evs = []
            for _ in range(k):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step(p)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, dev) / k

    with ClockSampler(local_rank) as clocks:
        ms = timed(prm, args.steps, args.warmup)
    # the kernels' launch times from the same steps with the stage events on
    se2n.se2n_plan_profile(plan, True)
    timed(prm, max(1, min(args.steps, 3)), 0)
    prof = se2n.se2n_plan_profile_read(plan, reset=True)
    se2n.se2n_plan_profile(plan, False)
    launches = prof["kernels"] / max(1, min(args.steps, 3))
    upd = integrated_updates(w.H, w.W, w.N, w.steps, w.rounds)
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    d_ms, d_calls = prof["diffuse"]
    d_s = d_ms / d_calls / 1e3
    if prop:
        b_ms, b_calls = prof["propagator"]
        b_s = b_ms / b_calls / 1e3
        items = propagator_build_items(w.H, w.W)
        flops, products = propagator_gemm_flops(items, w.N, w.steps)
        # the symmetric build computes the 36 upper-triangle 8 x 8 tiles of the
        # 64 of every N = 64 product and mirrors them
        exec_flops = flops * 36 // 64
        # DRAM traffic from a one-launch capture of a smaller square plane of
        # the same workload, scaled to this launch by the classes built (the
        # build) and by the method's bytes (the apply)
        rec_b, rec_a = stored_record("prop_build_wide"), stored_record("prop_apply_tiled")
        b_traffic = round(rec_b["dram_bytes_per_launch"] * items / rec_b["classes_built"]) if rec_b else None
        roofline = {"bound": "alu",
                    "kernel": f"k_prop_build_symw<{w.N}> ({items} classes computed, row slot <= column slot; a "
                              "transposed class applies its transpose's rows; FP32 symmetric products)",
                    "achieved": round(exec_flops / b_s / 1e12, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                    "frac": round(exec_flops / b_s / 1e12 / peak, 4), "traffic": b_traffic,
                    "traffic_basis": (f"ncu on {rec_b['workload']} ({rec_b['dram_bytes_per_launch']} bytes, "
                                      f"{rec_b['classes_built']} classes) x classes built") if rec_b else None,
                    "avg_launch_ms": round(b_s * 1e3, 4), "flops_per_launch": exec_flops,
                    "flops_basis": f"executed flops: classes x {products} products x 2 N^3 x 36/64 (the upper-triangle "
                                   "8x8 tiles)",
                    "full_product_flops_per_launch": flops,
                    "frac_full_product_equivalent": round(flops / b_s / 1e12 / peak, 4),
                    "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (derived, not measured)",
                    "apply_avg_launch_ms": round(d_s * 1e3, 4)}
        # the separate apply on the Hermitian half, tile by tile: the half
        # spectrum in and out, and every built class's N x N rows once (a
        # transposed class reads its transpose's rows, from L2 when the
        # super-tile order works)
        wc = w.W // 2 + 1
        a_bytes = 2 * 8 * w.N * w.H * wc + 4 * w.N * w.N * items
        hbm = _peaks().get("hbm_gbs")
        roofline["apply"] = {"kernel": f"k_prop_apply_tiled<{w.N}>", "bound": "hbm", "avg_launch_ms": round(d_s * 1e3, 4),
                             "bytes_per_launch": a_bytes,
                             "traffic": round(rec_a["dram_bytes_per_launch"] * a_bytes / rec_a["method_bytes"])
                             if rec_a else None,
                             "traffic_basis": (f"ncu on {rec_a['workload']} ({rec_a['dram_bytes_per_launch']} bytes for "
                                               f"{rec_a['method_bytes']} method's bytes) x method's bytes")
                             if rec_a else None,
                             "bytes_basis": "8 N H (W/2 + 1) bytes in and out + 4 N^2 bytes a built class",
                             "achieved": round(a_bytes / d_s / 1e9, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(a_bytes / d_s / 1e9 / hbm, 4) if hbm else None,
                             "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy, burst)"}
    else:
        achieved = FLOPS_PER_UPDATE * upd / d_s / 1e12
        roofline = {"bound": "alu", "kernel": f"k_diffuse_x2<{w.N},4,...> (packed FP32 pairs)",
                    "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4), "traffic": None, "flops_per_update": FLOPS_PER_UPDATE,
                    "updates_per_launch": upd, "avg_launch_ms": round(d_s * 1e3, 4),
                    "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (derived, not measured)",
                    "hbm_gbs_of_diffuse": round(16 * w.H * (w.W // 2 + 1) * w.N / d_s / 1e9, 1)}
    stages = {k: {"ms_per_step": round(v[0] / max(1, min(args.steps, 3)), 4)} for k, v in prof.items()
              if k != "kernels" and v[1] > 0}

    # the other diffusion on the same inpaint, for comparison
    other = params(w, 0 if prop else se2n.SE2N_DIFFUSE_PROPAGATOR)
    other_ms = timed(other, 2, 1)
    # the stiff run: split diagonal (beta T > 8), FP32 and FP64 corrections
    stiff = {}
    for name, fl in (("fp32_correction", 0), ("fp64_correction", se2n.SE2N_DIFFUSE_SM_FP64)):
        stiff[name] = {"ms_per_inpaint": round(timed(params(ws, fl), 2, 1), 4)}

    result = {"metric": METRIC, "ms_per_inpaint": round(ms, 4), "value": world * upd / (ms / 1e3), "unit": UNIT,
              "m2_updates_per_s": world * w.updates() / (ms / 1e3), "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": {"workload": f"{w.name}: {w.H}x{w.W} lines plus textured patches, N=64, 85% "
                                     "random mask, beta=0.25, T=50, one interval of 1000 CN steps",
                         "updates_per_step": upd, "m2_updates_per_step": w.updates(),
                         "diffusion": "S-step propagators (separate apply)" if prop else
                                      "step by step, the fused Crank-Nicolson kernel",
                         "l2": "flushed between timed steps (256 MiB write); the 2 GiB volume exceeds L2",
                         "parallelism": "replicas"},
              "roofline": roofline, "stages_ms": stages, "gpu_launches": int(round(launches)),
              ("step_by_step" if prop else "propagators"): {"ms_per_inpaint": round(other_ms, 4),
                                                            "value": world * upd / (other_ms / 1e3)},
              "stiff_run": {"workload": "beta=10, T=1000, 1000 steps (beta dt = 10), split diagonal", **stiff},
              "clocks": clocks.summary()}

    # errors against the FP64 oracle
    if rank == 0:
        import oracle
        err = {}
        bins_main = oracle.orient(f32.astype(np.float64), w.mask, w.N)["bins"]
        b_d = torch.tensor(bins_main, device=dev)
        if os.path.exists(GOLDEN_2048) and w.H == 2048:
            g = np.load(GOLDEN_2048)
            st = int(g["stride"][0])
            for name, wk, fl in (("main", w, flags), ("stiff_fp32", ws, 0), ("stiff_fp64", ws, se2n.SE2N_DIFFUSE_SM_FP64)):
                key = "main_out" if name == "main" else "stress_out"
                if key not in g:
                    continue
                with torch.cuda.stream(stream):
                    se2n.se2n_inpaint(plan, f_d, m_d, b_d, params(wk, fl), vol, out)
                torch.cuda.synchronize(dev)
                got = out.cpu().numpy()[::st, ::st].astype(np.float64)
                ref = g[key].astype(np.float64)
                err[name] = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                             "max_abs_over_max_f": float(np.abs(got - ref).max() / np.abs(w.f).max()),
                             "compared": f"every {st}th row and column of the projected image"}
        # the diffused spectrum of the main run at a seeded sample of frequencies
        with torch.cuda.stream(stream):
            se2n.se2n_lift(plan, f_d, m_d, b_d, vol)
            se2n.se2n_forward(plan, vol)
        torch.cuda.synchronize(dev)
        rng = np.random.default_rng(2048)
        freqs = np.sort(rng.choice(w.H * w.W, size=4096, replace=False))
        v0 = vol.reshape(w.N, -1)[:, torch.tensor(freqs, device=dev)].cpu().numpy()
        with torch.cuda.stream(stream):
            se2n.se2n_diffuse(plan, vol, w.beta, w.T, w.steps, flags)
        torch.cuda.synchronize(dev)
        v1 = vol.reshape(w.N, -1)[:, torch.tensor(freqs, device=dev)].cpu().numpy()
        # the oracle integrates the sampled frequencies' systems in place on
        # the full-size index space (the symbols follow from H, W and k, l)
        full = np.zeros((w.N, w.H, w.W), np.complex128)
        full.reshape(w.N, -1)[:, freqs] = v0
        t0 = time.perf_counter()
        ref = oracle.diffuse(full, w.beta, w.T, w.steps, freqs=freqs).reshape(w.N, -1)[:, freqs]
        err["spectrum_sampled"] = {
            "rel_l2": float(np.linalg.norm(v1 - ref) / np.linalg.norm(ref)),
            "frequencies": int(freqs.size), "oracle_seconds": round(time.perf_counter() - t0, 2),
            "note": "the GPU's own lifted and transformed spectrum, diffused by both sides"}
        result["err_vs_fp64"] = err
    plan.close()
    if dist:
        dist.destroy_process_group()
    return result


# ----------------------------------------------------------------------------
# the oracle as CPU baseline / reference arm
# ----------------------------------------------------------------------------

def _oracle_sample(w, steps, rounds, dynamic=False, nthreads=None):
    """The oracle's whole inpaint of the workload's image with `rounds`
    intervals of `steps` steps (same dt), on `nthreads` threads (all host
    cores by default). Returns (updates, seconds), updates counted like our
    arm's value (the Hermitian half; the oracle itself integrates all M^2
    frequencies, so per such update it does twice the work)."""
    import oracle
    p = oracle.Params(N=w.N, beta=w.beta, T=w.T / w.rounds * rounds, steps=steps, rounds=rounds, eps=w.eps,
                      dynamic=int(dynamic))
    f = w.f.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    oracle.inpaint(f, w.mask, p, nthreads=nthreads or os.cpu_count())
    dt = time.perf_counter() - t0
    return integrated_updates(w.H, w.W, w.N, steps, rounds), dt


def cpu_baseline(w, steps=75, rounds=2, dynamic=False):
    """The oracle as it stands on this host: a bounded sample of the workload
    on all cores, a smaller one on one core, and the time of the full run
    that wrote the stored reference result."""
    cores = os.cpu_count()
    upd, dt = _oracle_sample(w, steps, rounds, dynamic, nthreads=cores)
    s1 = max(steps // 4, 5)
    upd1, dt1 = _oracle_sample(w, s1, rounds, dynamic, nthreads=1)
    _oracle_sample(w, 1, 1, dynamic, nthreads=cores)  # the OpenMP thread count back to all cores
    golden = GOLDEN_DYNAMIC if dynamic else GOLDEN
    full = None
    if os.path.exists(golden):
        g = np.load(golden)
        full = {"seconds": round(float(g["oracle_seconds"][0]), 2),
                "run": f"the FP64 oracle's complete {w.rounds} x {w.steps}-step inpaint that wrote "
                       f"tests/golden/{os.path.basename(golden)} (tests/golden/make_references.py, 8-core x86 host)",
                "value": integrated_updates(w.H, w.W, w.N, w.steps, w.rounds) / float(g["oracle_seconds"][0])}
    return {"value": upd / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"the FP64 oracle's whole inpaint of the same 512x512 N=32 image with {rounds} intervals "
                      f"x {steps} CN steps ({upd:.3g} updates counted like value, {dt:.1f} s)"
                      + (", dynamic restoration" if dynamic else "")
                      + ", all host cores (OpenMP over frequencies, numpy FFTs)",
            "one_core": {"value": upd1 / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"{rounds} intervals x {s1} CN steps ({upd1:.3g} updates, {dt1:.1f} s), one "
                                   "OpenMP thread"},
            "full_run_stored": full,
            "build": "gcc -O3 -fopenmp (portable flags: the same source and results on x86_64 and aarch64)"}


def run_batch(args, rank, world, local_rank):
    """256 seeded images of uneven size (128..1024) and N (16, 32, 64): the
    whole method through one graph-captured batch with one persistent
    diffusion launch, against one se2n_inpaint per image. Images are dealt
    to ranks round-robin (weak scaling)."""
    import torch

    from paper_1304_2062_gb300 import se2n

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    allw = synth.workload_batch()
    mine = [allw[i] for i in shard(len(allw), rank, world)]
    stream = torch.cuda.Stream(dev)
    w0 = allw[0]
    prop = args.diffusion == "propagator"
    prm = se2n.se2n_params_default(beta=w0.beta, T=w0.T, steps=w0.steps, rounds=w0.rounds, eps=w0.eps,
                                   diffuse_flags=se2n.SE2N_DIFFUSE_PROPAGATOR if prop else 0)
    imgs = []
    for w in mine:
        imgs.append((torch.tensor(w.f.astype(np.float32), device=dev), torch.tensor(w.mask, device=dev),
                     torch.zeros((w.H, w.W), dtype=torch.float32, device=dev), w.N))
    t0 = time.perf_counter()
    batch = se2n.se2n_batch_create(imgs, prm, 0, se2n.SE2N_BATCH_AUTOTUNE, stream)
    create_s = time.perf_counter() - t0
    info = se2n.se2n_batch_get_info(batch)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # updates over the frequencies integrated (the Hermitian half of every
    # image's spectrum); the library's count over all M^2 is updates_per_run
    updates = sum(integrated_updates(w.H, w.W, w.N, w.steps, w.rounds) for w in mine)

    def timed(fn, k):
        evs = []
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn(batch)
            torch.cuda.synchronize(dev)
            if dist:
                dist.barrier()
            for _ in range(k):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn(batch)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, dev) / k

    with ClockSampler(local_rank) as clocks:
        ms = timed(se2n.se2n_batch_run, args.steps)
    ms_per_image = timed(se2n.se2n_batch_run_per_image, max(1, min(args.steps, 3)))
    ms_diff = timed(se2n.se2n_batch_run_diffusion, max(1, min(args.steps, 5)))

    # end to end: every image's f and mask from pinned host memory into the
    # batch's device inputs, one graph launch, every output back to pinned host
    host_in = [(torch.from_numpy(w.f.astype(np.float32)).pin_memory(), torch.from_numpy(w.mask).pin_memory())
               for w in mine]
    host_out = [torch.empty((w.H, w.W), dtype=torch.float32).pin_memory() for w in mine]

    def e2e_once():
        with torch.cuda.stream(stream):
            for (hf, hm), (df, dm, _, _) in zip(host_in, imgs):
                df.copy_(hf, non_blocking=True)
                dm.copy_(hm, non_blocking=True)
            se2n.se2n_batch_run(batch)
            for ho, (_, _, do, _) in zip(host_out, imgs):
                ho.copy_(do, non_blocking=True)
        stream.synchronize()

    for _ in range(max(1, args.warmup)):
        e2e_once()
    if dist:
        dist.barrier()
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_once()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    ms_e2e = max_over_ranks(statistics.median(e2e_ms), dist, dev)
    h2d = sum(hf.nbytes + hm.nbytes for hf, hm in host_in)
    d2h = sum(ho.nbytes for ho in host_out)
    # the persistent launch integrates the Hermitian half of the spectra of the
    # images it keeps (all of them step by step; with propagators, the shapes
    # the batch left to it), one interval
    half_updates = info["step_updates"]
    achieved = FLOPS_PER_UPDATE * half_updates / (ms_diff / 1e3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    batch.close()
    if dist:
        dist.destroy_process_group()
    total_updates = updates * world
    return {"metric": METRIC, "value": total_updates / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of 256 seeded images, sides from {128,256,384,512,768,1024}, N U{16,32,64}, "
                                   "60-90% corrupted, beta=0.25, T=2, 100 CN steps, 1 interval",
                       "images_this_rank": len(mine), "updates_per_step": total_updates,
                       "updates_basis": "H x (W/2 + 1) frequencies (the Hermitian half) x N x steps, summed over "
                                        "the images; m2_updates_per_step counts all H x W",
                       "m2_updates_per_step": info["updates_per_run"] * world,
                       "diffusion": ("S-step propagators for the shapes where they are estimated cheaper "
                                     f"({info['prop_images']} images; {info['fused_images']} of them, the "
                                     "shapes the row and column passes cover (N = 16, 30, 32), whole inpaints on "
                                     "them, the others with the separate apply), the persistent step kernel for "
                                     "the rest")
                       if prop else "the persistent step-by-step kernel for every image",
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"},
            "per_image_launches": {"ms_per_step": ms_per_image, "value": total_updates / (ms_per_image / 1e3),
                                   "speedup_of_batched": ms_per_image / ms},
            "roofline": ({"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                          "frac": round(achieved / peak, 4), "traffic": None, "kernel": "k_diffuse_batch",
                          "avg_launch_ms": round(ms_diff, 3)} if half_updates > 0 else
                         {"bound": None, "kernel": None,
                          "note": "every image is integrated by propagators (the persistent step kernel has no "
                                  "work): the rooflines of the build, the row and column passes and the separate "
                                  "apply are those of the 512 and 2048 workloads"}),
            "e2e": {"value": total_updates / (ms_e2e / 1e3), "unit": UNIT, "ms_per_step": ms_e2e,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "se2n_batch_run on device inputs refreshed from pinned host buffers"},
            "autotune": info, "create_s": create_s, "clocks": clocks.summary(),
            "gpu_launches": len(mine) * 6 + w0.rounds * 1}


# ----------------------------------------------------------------------------
# learned surrogate
# ----------------------------------------------------------------------------

SURR_METRIC = "surrogate inpaints/s (256x256, batch 64, method fallback at known-pixel RMS > 2e-2)"
SURR_UNIT = "images/s"
SURR_BATCH = 64
SURR_THRESHOLD = 2e-2
SURR_LAUNCHES_PER_CALL = 20
# (input channels used, output channels, level) of the 14 3x3 convolutions;
# the first layer reads 2 real channels (f, mask) of its 8-channel input
SURR_CONVS = [(2, 32, 0), (32, 32, 0), (32, 64, 1), (64, 64, 1), (64, 128, 2), (128, 128, 2), (128, 256, 3),
              (256, 256, 3), (384, 128, 2), (128, 128, 2), (192, 64, 1), (64, 64, 1), (96, 32, 0), (32, 32, 0)]


def surrogate_flops(H, W):
    """Algorithmic conv flops of one forward pass of one H x W image
    (2 x 9 x Cin x Cout per output pixel, plus the 1x1 head)."""
    fl = sum(2 * 9 * cin * cout * (H >> lvl) * (W >> lvl) for cin, cout, lvl in SURR_CONVS)
    return fl + 2 * 32 * H * W


def surrogate_train_flops(H, W):
    """Forward + data gradient (not for the first layer) + weight gradient."""
    first = 2 * 9 * 2 * 32 * H * W
    f = surrogate_flops(H, W)
    return 3 * f - first


def _surrogate_chunk(job):
    first, count = job
    return first, synth.surrogate_examples(first, count)


def _psnr(a, b):
    return float(10 * np.log10(1.0 / max(np.mean((np.asarray(a, np.float64) - b) ** 2), 1e-30)))


def run_surrogate(args, rank, world, local_rank):
    """The learned surrogate end to end: 20000 seeded 256x256 pairs
    (corrupted image, method-inpainted image) made by the GPU method, the
    network trained on them by the library's own kernels, then timed
    inference of batches of 64 with the method as fallback, against the
    method on the same images. Reports PSNR against the clean images and
    against the method's output on 512 held-out images."""
    import multiprocessing as mp

    pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
    import torch

    from paper_1304_2062_gb300 import se2n

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    H = W = synth.SURROGATE_SIDE
    mp_ = synth.surrogate_method_params()
    N = mp_["N"]
    stream = torch.cuda.Stream(dev)
    plan = se2n.se2n_plan_create(H, W, N, 0, stream)
    prm = se2n.se2n_params_default(reinject=1, **mp_)
    vol = torch.empty((N, H, W), dtype=torch.complex64, device=dev)

    def make_set(first, count):
        F = torch.empty((count, H, W), dtype=torch.float32, device=dev)
        M = torch.empty((count, H, W), dtype=torch.uint8, device=dev)
        T = torch.empty((count, H, W), dtype=torch.float32, device=dev)
        C = []
        per = max(64, count // (4 * (os.cpu_count() or 1)))
        jobs = [(s, min(per, first + count - s)) for s in range(first, first + count, per)]
        gpu_ms = 0.0
        for s, (clean, mask) in pool.imap(_surrogate_chunk, jobs):
            i0, n = s - first, clean.shape[0]
            with torch.cuda.stream(stream):
                F[i0:i0 + n].copy_(torch.from_numpy(clean * mask))
                M[i0:i0 + n].copy_(torch.from_numpy(mask))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for j in range(i0, i0 + n):
                    se2n.se2n_inpaint(plan, F[j], M[j], None, prm, vol, T[j])
                b.record(stream)
            b.synchronize()
            gpu_ms += a.elapsed_time(b)
            C.append(clean)
        return F, M, T, np.concatenate(C), gpu_ms

    t0 = time.perf_counter()
    first, count = synth.SURROGATE_TRAIN_SEEDS
    count = args.train_pairs or count
    Ftr, Mtr, Ttr, _, gen_ms = make_set(first, count)
    gen_s = time.perf_counter() - t0
    vfirst, vcount = synth.SURROGATE_VAL_SEEDS
    Fv, Mv, Tv, Cv, _ = make_set(vfirst, vcount)
    pool.close()

    # training: Adam, cosine-decayed learning rate, blocks of 32 consecutive
    # (independently seeded) examples in a fresh random order every epoch
    u = se2n.se2n_unet_create(SURR_BATCH, H, W, stream)
    se2n.se2n_unet_init(u, 7)
    tb = 32
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(0)
    starts = []

    def next_start():
        if not starts:
            starts.extend(rng.permutation(np.arange(0, count - tb + 1, tb)).tolist())
        return starts.pop()

    lr0, lr_min, warm = 1e-3, 1e-5, 200

    def train(nsteps, total, done):
        for k in range(nsteps):
            s = next_start()
            i = done + k
            x = i / max(total, 1)
            lr = lr_min + 0.5 * (lr0 - lr_min) * (1 + np.cos(np.pi * min(x, 1.0)))
            lr *= min(1.0, (i + 1) / warm)
            se2n.se2n_unet_train_step(u, Ftr[s], Mtr[s], Ttr[s], tb, float(lr), loss)

    with torch.cuda.stream(stream):
        # time 30 steps of the warm-up ramp to size the run to the time budget
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        train(10, 10 ** 9, 0)
        a.record(stream)
        train(20, 10 ** 9, 10)
        b.record(stream)
        b.synchronize()
        ms_step = a.elapsed_time(b) / 20
        total = max(300, int(args.train_seconds * 1e3 / ms_step))
        t1 = time.perf_counter()
        losses = []
        done = 30
        while done < total:
            n = min(500, total - done)
            train(n, total, done)
            done += n
            losses.append(float(loss.item()))
        torch.cuda.synchronize(dev)
        train_s = time.perf_counter() - t1

    # validation: network alone, network with fallback, method
    net = torch.empty_like(Tv)
    sur = torch.empty_like(Tv)
    resid = np.zeros(vcount, np.float32)
    fallbacks = 0
    with torch.cuda.stream(stream):
        for s in range(0, vcount, SURR_BATCH):
            n = min(SURR_BATCH, vcount - s)
            se2n.se2n_unet_forward(u, Fv[s:s + n], Mv[s:s + n], n, net[s:s + n])
            r = np.zeros(n, np.float32)
            fallbacks += se2n.se2n_surrogate_inpaint(u, plan, prm, Fv[s:s + n], Mv[s:s + n], n, SURR_THRESHOLD, vol,
                                                     sur[s:s + n], r)
            resid[s:s + n] = r
        torch.cuda.synchronize(dev)
    net_h, sur_h, meth_h = net.cpu().numpy(), sur.cpu().numpy(), Tv.cpu().numpy()
    f_h = Fv.cpu().numpy()
    quality = {
        "validation_images": vcount,
        "psnr_vs_clean_db": {"surrogate_with_fallback": _psnr(sur_h, Cv), "network_alone": _psnr(net_h, Cv),
                             "method": _psnr(meth_h, Cv), "zero_filled_input": _psnr(f_h, Cv)},
        "psnr_vs_method_db": {"surrogate_with_fallback": _psnr(sur_h, meth_h), "network_alone": _psnr(net_h, meth_h),
                              "zero_filled_input": _psnr(f_h, meth_h)},
        "fallbacks": int(fallbacks), "threshold": SURR_THRESHOLD,
        "known_pixel_rms": {"median": float(np.median(resid)), "max": float(resid.max())},
    }

    # timed: surrogate inference of batches of 64 (held-out images), fallback included
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    nb = vcount // SURR_BATCH

    def batch(i):
        s = (i % nb) * SURR_BATCH
        return s, s + SURR_BATCH

    def timed(fn, k):
        with torch.cuda.stream(stream):
            for i in range(args.warmup):
                fn(i)
            torch.cuda.synchronize(dev)
            if dist:
                dist.barrier()
            evs = []
            for i in range(k):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn(i)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, dev) / k

    nf = []

    def surrogate_step(i):
        s, e = batch(i)
        nf.append(se2n.se2n_surrogate_inpaint(u, plan, prm, Fv[s:e], Mv[s:e], SURR_BATCH, SURR_THRESHOLD, vol,
                                             sur[s:e], None))

    def forward_step(i):
        s, e = batch(i)
        se2n.se2n_unet_forward(u, Fv[s:e], Mv[s:e], SURR_BATCH, net[s:e])

    def method_step(i):
        s, e = batch(i)
        for j in range(s, e):
            se2n.se2n_inpaint(plan, Fv[j], Mv[j], None, prm, vol, Tv[j])

    # the method by S-step propagators (row and column passes): the plan
    # builds them on the first image and keeps them for the rest
    prm_p = se2n.se2n_params_default(reinject=1, diffuse_flags=se2n.SE2N_DIFFUSE_PROPAGATOR, **mp_)

    def method_prop_step(i):
        s, e = batch(i)
        for j in range(s, e):
            se2n.se2n_inpaint(plan, Fv[j], Mv[j], None, prm_p, vol, Tv[j])

    se2n.se2n_plan_profile(plan, True)
    with ClockSampler(local_rank) as clocks:
        ms = timed(surrogate_step, args.steps)
    method_kernels = int(se2n.se2n_plan_profile_read(plan, reset=True)["kernels"])
    se2n.se2n_plan_profile(plan, False)
    nf_timed = int(sum(nf[-args.steps:]))
    kernels_per_fallback = method_kernels / max(1, sum(nf))
    ms_fwd = timed(forward_step, max(3, min(args.steps, 10)))
    ms_method = timed(method_step, max(3, min(args.steps, 5)))
    se2n.se2n_inpaint(plan, Fv[0], Mv[0], None, prm_p, vol, Tv[0])  # builds the propagators
    ms_method_prop = timed(method_prop_step, max(3, min(args.steps, 5)))
    fl = surrogate_flops(H, W) * SURR_BATCH
    peaks = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = fl / (ms_fwd / 1e3) / 1e12
    train_tflops = surrogate_train_flops(H, W) * tb / (ms_step / 1e3) / 1e12

    # end to end: pinned host inputs in, result out, every step
    fh = torch.from_numpy(f_h[:SURR_BATCH].copy()).pin_memory()
    mh = torch.from_numpy(Mv[:SURR_BATCH].cpu().numpy()).pin_memory()
    oh = torch.empty((SURR_BATCH, H, W), dtype=torch.float32).pin_memory()
    Fd, Md, Od = torch.empty_like(Fv[:SURR_BATCH]), torch.empty_like(Mv[:SURR_BATCH]), torch.empty_like(Tv[:SURR_BATCH])

    def e2e_step(i):
        Fd.copy_(fh, non_blocking=True)
        Md.copy_(mh, non_blocking=True)
        se2n.se2n_surrogate_inpaint(u, plan, prm, Fd, Md, SURR_BATCH, SURR_THRESHOLD, vol, Od, None)
        oh.copy_(Od, non_blocking=True)

    ms_e2e = timed(e2e_step, max(3, min(args.steps, 10)))
    u.close()
    plan.close()
    if dist:
        dist.destroy_process_group()
    res = {"metric": SURR_METRIC, "value": world * SURR_BATCH / (ms / 1e3), "unit": SURR_UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (FP32 accumulate)", "data": "synthetic",
           "config": {"workload": f"surrogate_lines_circles_256: {count} training pairs (seeds {first}..), "
                                  f"{vcount} held-out (seeds {vfirst}..), 50% random masks, targets from the GPU "
                                  f"method (N={N}, beta={mp_['beta']}, T={mp_['T']}, {mp_['steps']} steps, "
                                  "known pixels re-injected); 4-level U-Net 32-64-128-256",
                      "batch": SURR_BATCH, "l2": "flushed between timed steps (256 MiB write)",
                      "parallelism": "replicas"},
           "method_same_images": {"ms_per_step": ms_method, "value": world * SURR_BATCH / (ms_method / 1e3),
                                  "api": "se2n_inpaint per image, step by step", "speedup_of_surrogate": ms_method / ms},
           "method_same_images_propagators": {
               "ms_per_step": ms_method_prop, "value": world * SURR_BATCH / (ms_method_prop / 1e3),
               "api": "se2n_inpaint per image, S-step propagators kept by the plan (row and column passes)",
               "speedup_of_surrogate": ms_method_prop / ms},
           "quality": quality,
           "roofline": {"bound": "tensor", "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "kernel": "se2n_unet_forward: 13 tcgen05 convolutions (TMA) + first layer on CUDA cores",
                        "flops_per_launch": fl, "avg_launch_ms": round(ms_fwd, 4),
                        "peak_basis": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json bf16_tflops)"},
           "training": {"pairs": count, "batch": tb, "steps": done, "seconds": round(train_s, 2),
                        "lr": f"Adam, linear warm-up over {warm} steps to {lr0}, cosine to {lr_min}",
                        "ms_per_step": round(ms_step, 3), "tflops": round(train_tflops, 2),
                        "loss_every_500_steps": [float(f"{v:.3g}") for v in losses],
                        "pair_generation_s": round(gen_s, 2), "method_gpu_s_for_pairs": round(gen_ms / 1e3, 2)},
           "e2e": {"value": world * SURR_BATCH / (ms_e2e / 1e3), "unit": SURR_UNIT, "ms_per_step": ms_e2e,
                   "h2d_bytes_per_step": int(fh.numel() * 4 + mh.numel()), "d2h_bytes_per_step": int(oh.numel() * 4),
                   "api": "pinned host copies + se2n_surrogate_inpaint"},
           "clocks": clocks.summary(),
           # per surrogate call: input packing, 3 pools, 14 convolutions, head, residual; plus the
           # method's kernels for the images that fell back (counted by the plan)
           "gpu_launches": SURR_LAUNCHES_PER_CALL * args.steps + int(round(kernels_per_fallback * nf_timed)),
           "fallbacks_in_timed_region": nf_timed}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = surrogate_cpu_baseline()
    return res


def run_unet_forward(args, rank, world, local_rank):
    """The network's inference kernels alone: batches of 64 seeded 256x256
    inputs (the surrogate workload's images and masks) through
    se2n_unet_forward, initialised weights (the kernels' cost does not depend
    on their values). Roofline: the forward's algorithmic conv flops against
    the measured dense bf16 peak."""
    import torch

    from paper_1304_2062_gb300 import se2n

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    H = W = synth.SURROGATE_SIDE
    clean, mask = synth.surrogate_examples(synth.SURROGATE_VAL_SEEDS[0] + 64 * rank, SURR_BATCH)
    stream = torch.cuda.Stream(dev)
    F = torch.tensor(clean * mask, device=dev)
    M = torch.tensor(mask, device=dev)
    out = torch.empty((SURR_BATCH, H, W), dtype=torch.float32, device=dev)
    u = se2n.se2n_unet_create(SURR_BATCH, H, W, stream)
    se2n.se2n_unet_init(u, 7)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            se2n.se2n_unet_forward(u, F, M, SURR_BATCH, out)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        evs = []
        with ClockSampler(local_rank) as clocks:
            for _ in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                se2n.se2n_unet_forward(u, F, M, SURR_BATCH, out)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, dev) / args.steps
    u.close()
    if dist:
        dist.destroy_process_group()
    fl = surrogate_flops(H, W) * SURR_BATCH
    peak = _peaks().get("bf16_tflops", 1890.1)
    achieved = fl / (ms / 1e3) / 1e12
    res = {"metric": "surrogate network forward images/s (256x256, batch 64)", "value": world * SURR_BATCH / (ms / 1e3),
           "unit": SURR_UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (FP32 accumulate)",
           "data": "synthetic", "config": {"workload": "unet_forward_256_b64: 64 seeded lines-and-circles images, "
                                                      "50% masks, 4-level U-Net 32-64-128-256",
                                           "l2": "flushed between timed steps (256 MiB write)",
                                           "parallelism": "replicas"},
           "roofline": {"bound": "tensor", "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "kernel": "se2n_unet_forward: 13 tcgen05 convolutions (TMA) + first layer on CUDA cores",
                        "flops_per_launch": fl, "avg_launch_ms": round(ms, 4),
                        "peak_basis": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json bf16_tflops)"},
           "clocks": clocks.summary(), "gpu_launches": 20 * args.steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = unet_cpu_baseline()
    return res


def unet_cpu_baseline():
    """The FP64 reference network (oracle/unet.py) forward on one image."""
    from oracle import unet as ou
    clean, mask = synth.surrogate_example(synth.SURROGATE_VAL_SEEDS[0])
    p = ou.he_params(7)
    t0 = time.perf_counter()
    ou.forward(p, (clean * mask)[None], mask[None])
    dt = time.perf_counter() - t0
    return {"value": 1 / dt, "unit": SURR_UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the FP64 reference network's forward of one 256x256 image ({dt:.1f} s, numpy)"}


def surrogate_cpu_baseline(n=8):
    """The FP64 oracle's method on n held-out surrogate images (images/s)."""
    import oracle
    first = synth.SURROGATE_VAL_SEEDS[0]
    p = oracle.Params(reinject=1, **synth.surrogate_method_params())
    t0 = time.perf_counter()
    for i in range(n):
        clean, mask = synth.surrogate_example(first + i)
        oracle.inpaint(clean * mask, mask, p)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": SURR_UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the FP64 oracle's method (the surrogate's fallback and teacher) on {n} held-out 256x256 "
                      f"images, {dt:.1f} s, all host cores"}


def _reference_line(args, world, metric, unit, value, ms, cfg, sample):
    return {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, rank, world):
    """The oracle as the reference arm, on the same workload, metric and unit
    as our arm, each step a bounded sample of it (rank 0 only)."""
    if rank != 0:
        return None
    import oracle
    if args.workload == "surrogate":
        first = synth.SURROGATE_VAL_SEEDS[0]
        p = oracle.Params(reinject=1, **synth.surrogate_method_params())
        per = 2

        def one(k):
            for i in range(per):
                clean, mask = synth.surrogate_example(first + (k * per + i) % synth.SURROGATE_VAL_SEEDS[1])
                oracle.inpaint(clean * mask, mask, p)
        for k in range(args.warmup):
            one(k)
        times = []
        for k in range(args.steps):
            t0 = time.perf_counter()
            one(k)
            times.append(time.perf_counter() - t0)
        total = sum(times)
        value = per * args.steps / total
        return _reference_line(args, world, SURR_METRIC, SURR_UNIT, value, total / args.steps * 1e3,
                               {"workload": "surrogate_lines_circles_256 (held-out images)",
                                "reference_sample": f"{per} images per step"},
                               f"each step: the FP64 oracle's method on {per} held-out 256x256 images (the surrogate's "
                               "teacher and fallback), all host cores")
    if args.workload == "batch":
        allw = synth.workload_batch()
        steps = 10

        def one(k):
            w = allw[k % len(allw)]
            pp = oracle.Params(N=w.N, beta=w.beta, T=w.T * steps / w.steps, steps=steps, rounds=1, eps=w.eps)
            t0 = time.perf_counter()
            oracle.inpaint(w.f, w.mask, pp)
            return integrated_updates(w.H, w.W, w.N, steps, 1), time.perf_counter() - t0
        for k in range(args.warmup):
            one(k)
        upd, total = 0, 0.0
        for k in range(args.steps):
            u_, dt = one(args.warmup + k)
            upd += u_
            total += dt
        return _reference_line(args, world, METRIC, UNIT, upd / total, total / args.steps * 1e3,
                               {"workload": "batch of 256 seeded images (sampled one per step)",
                                "reference_sample": f"one batch image per step, {steps} CN steps"},
                               f"each step: the FP64 oracle's inpaint of the next image of the batch with {steps} "
                               "CN steps (same dt), all host cores")
    w = _workload()
    dynamic = args.workload == "dr"
    # with dynamic restoration two intervals, so that the sample holds a growth step
    steps, rounds = (10, 2) if dynamic else (20, 1)
    for _ in range(args.warmup):
        _oracle_sample(w, steps, rounds, dynamic)
    times, upd = [], 0
    for _ in range(args.steps):
        upd, dt = _oracle_sample(w, steps, rounds, dynamic)
        times.append(dt)
    total = sum(times)
    value = upd * args.steps / total
    sample = (f"each step: the FP64 oracle's inpaint of the 512x512 N=32 image with {rounds} interval(s) x {steps} "
              f"CN steps ({upd:.3g} updates counted like our arm's value){', dynamic restoration' if dynamic else ''}, "
              f"all host cores ({cpu_model()})")
    return _reference_line(args, world, METRIC, UNIT, value, total / args.steps * 1e3,
                           _config(w, {"reference_sample": f"{rounds} x {steps} steps per step"}, dynamic=dynamic),
                           sample)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["512", "dr", "2048", "batch", "surrogate", "unet-forward"], default="512",
                    help="512: the 512x512 N=32 10x500-step inpaint (default); dr: the same with dynamic "
                         "restoration; 2048: the 2048x2048 N=64 1000-step inpaint (and its beta dt = 10 run); "
                         "batch: 256 uneven images; surrogate: train the U-Net on method pairs, "
                         "time its inference with fallback")
    ap.add_argument("--diffusion", choices=["propagator", "steps"], default=None,
                    help="512 / dr / 2048: integrate each interval by S-step propagators built every inpaint (default) "
                         "or step by step with the fused Crank-Nicolson kernel")
    ap.add_argument("--side", type=int, default=2048,
                    help="2048: the same workload on a side x side image, a smaller case for profiling (the "
                         "stored FP64 result it is compared with is for 2048 only)")
    ap.add_argument("--train-seconds", type=float, default=150.0, help="surrogate training time budget")
    ap.add_argument("--train-pairs", type=int, default=0, help="surrogate training pairs (0: all 20000)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per diffusion launch from an ncu capture of the current kernel")
    args = ap.parse_args()
    if args.diffusion is None:
        args.diffusion = "propagator"
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif args.workload == "batch":
        res = run_batch(args, rank, world, local_rank)
    elif args.workload == "2048":
        res = run_2048(args, rank, world, local_rank)
    elif args.workload == "surrogate":
        res = run_surrogate(args, rank, world, local_rank)
    elif args.workload == "unet-forward":
        res = run_unet_forward(args, rank, world, local_rank)
    else:
        res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
