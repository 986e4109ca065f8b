#!/usr/bin/env python
"""Benchmark of the B-spline interpolation path on GB300.

One step = the whole path on one batch: prefilter + inverse real 3D FFT of a
512^3 3-component Kolmogorov-spectrum field into quintic (order 6) B-spline
coefficients, then locate/bin/sort 2^24 clustered particles and evaluate u
and grad u at each of them, issued as one bspline_eval call (the particle
sort runs on a second stream beside the transform; the evaluation waits for
both).  Metric: particles/s (whole job over all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank holds a replica of the
field and evaluates its own 2^24 particles: the path has no exchange step
(weak scaling, no collective on the data path).

--impl reference times the CPU FP64 oracle (numpy) on this machine's host
cores on a bounded sample of the same workload and prints the same JSON line
with "impl": "reference".
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
sys.path.insert(0, ROOT)

METRIC = "particles/s for u+grad-u (quintic B-spline, 512^3), FP32 vs FP64 form, % HBM peak"
UNIT = "particles/s"
WORKLOAD_NAME = "throughput512"
STAGES = ["fft_x", "fft_yz", "bin", "scan", "scatter", "gather", "gather_direct"]
ERR_SAMPLE = 1500          # particles at which each form's outputs are compared with the oracle
ERR_SAMPLE_SEED = 42


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


_OVERRIDE = {}


# ----------------------------------------------------------------------------- ranks (N > 1)

def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time: the job is done when every replica is (all_reduce MAX)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, P: int, steps: int, ms_total: float) -> float:
    """Whole-job particles/s: every rank evaluates its own P particles per step (weak scaling)."""
    return world * P * steps / (ms_total / 1e3)


def rank_particle_seed(wl: dict, rank: int) -> int:
    """Each rank draws its own particle shard from the same recipe."""
    return wl["particle_seed"] + rank


def workload():
    """The benchmark workload; --N/--P shrink it for profiling captures only (not bench values)."""
    from paper_1201_4060_gb300 import synth
    wl = dict(synth.WORKLOADS[WORKLOAD_NAME])
    wl.update(_OVERRIDE)
    return wl


def config_block(wl, dtype, world):
    return {
        "workload": f"{wl['N']}^3 x 3-component Kolmogorov field, order-{wl['order']} (quintic) B-spline, "
                    f"{wl['P']} clustered particles per GPU, u + grad u, {dtype} coefficients",
        "N": wl["N"], "order": wl["order"], "particles_per_gpu": wl["P"], "coeff_dtype": dtype,
        "particles": "clustered: 60% uniform, 40% Gaussian clumps sigma=0.1 around 64 centres",
        "step": "one bspline_eval call: prefilter+inverse real FFT beside the bin+counting sort (second stream), then weights+stencil contraction",
        "parallelism": f"replicas x{world} (particle shard per GPU, no collective)",
        "l2": "no flush: inputs larger than L2 (u_hat 1.62 GB, coefficients 1.61 GB, positions 0.40 GB)",
    }


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons in a background thread."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.samples = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        window = "timed region"
        if not inside:
            inside = [s for s in self.samples if t0 - 0.3 <= s[0] <= t1 + 0.3]
            window = "timed region +-0.3 s (region shorter than the sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [num(s[1][1]) for s in inside if num(s[1][1]) is not None]
        smax = [num(s[1][2]) for s in inside if num(s[1][2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i in range(4) if s[1][5 + i].lower() == "active"})
        pw = [num(s[1][3]) for s in inside if num(s[1][3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inside), "window": window,
                "power_w_median": statistics.median(pw) if pw else None}


# ----------------------------------------------------------------------------- algorithmic bytes

def algorithmic_bytes(stage: str, N: int, P: int, dtype: str, order: int = 6) -> float:
    """Bytes a kernel must move at minimum (each input read once, each output written once)."""
    H = N // 2 + 1
    cplx = 16 if dtype == "f64" else 8
    elem = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
    outb = 8 if dtype == "f64" else 4
    tb = 8 if dtype == "f64" else 4
    spec = 3 * N * N * H * cplx
    coef = 3 * N ** 3 * elem
    bx = 8 if dtype == "f64" else 16             # brick extents (x = z); y is 12 up to order 6 in FP32
    by = 8 if (dtype == "f64" or order > 6) else 12
    nb = (-(-N // bx)) ** 2 * (-(-N // by))
    rec = 16 if tb == 4 else 32                  # first node + t per axis (the stored record adds padding)
    return {
        "fft_x": 2 * spec,                       # read u_hat, write the x-transformed spectrum
        "fft_yz": spec + coef,                   # read that spectrum, write coefficients (ring stays in L2)
        "bin": P * 24,                           # positions in (per-brick counts stay in L2)
        "scan": 4 * 4 * (nb + 1),
        "scatter": P * 24 + P * (rec + 4),       # positions in again; sorted record and original index out
        "gather": coef + P * (rec + 4) + P * 12 * outb,    # coefficients once, sorted records, u and grad out
        "gather_direct": 4 * nb,                 # per-brick counts (its particles are counted in "gather")
    }[stage]


def kernel_source_sha(stage: str) -> str:
    files = {"gather": ["particles.cuh"], "gather_direct": ["particles.cuh"], "bin": ["particles.cu"],
             "scan": ["particles.cu"],
             "scatter": ["particles.cu"], "fft_x": ["fft.cu", "fft_core.cuh"],
             "fft_yz": ["fft.cu", "fft_core.cuh"]}[stage]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1201_4060_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(stage: str, dtype: str, N: int, order: int):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    sha = kernel_source_sha(stage)
    key = f"{stage}:{dtype}:N{N}:o{order}"
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == key and parts[1] == sha:
                return float(parts[2])
    return None


# ----------------------------------------------------------------------------- our arm

def dense_field_on_gpu(F, dtype_torch, device):
    import torch
    N = F.N
    uh = torch.zeros((3, N, N, N // 2 + 1), dtype=dtype_torch, device=device)
    idx = torch.from_numpy(F.idx).to(device)
    vals = torch.from_numpy(F.val).to(device=device, dtype=dtype_torch)
    uh[:, idx[:, 0], idx[:, 1], idx[:, 2]] = vals
    return uh


def run_form(B, wl, F, x, dtype, steps, warmup, device, timed_stages=True, sample=None, band=0):
    """Time `steps` whole-path steps with one plan of coefficient type dtype (band > 0: the plan is told
    that modes beyond |k_i| <= band are zero); returns (ms/step, stage dict, non-finite count, outputs at
    the sampled particle indices (host FP64 arrays) or None)."""
    import torch
    plan = B.Plan(wl["N"], wl["order"], dtype)
    if band:
        plan.set_band(band)
    uh = dense_field_on_gpu(F, plan.uhat_dtype, device)
    coef = plan.empty_coeffs()
    P = x.shape[0]
    u = torch.empty((P, 3), dtype=plan.out_dtype, device=device)
    g = torch.empty((P, 3, 3), dtype=plan.out_dtype, device=device)
    stream = torch.cuda.current_stream()

    def step():
        plan.eval(uh, x, coef, u, g)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if timed_stages:
        plan.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stages = plan.stage_times() if timed_stages else {}
    nonfinite = plan.status()
    plan.set_timing(False)
    sampled = None
    if sample is not None:
        sampled = (u[sample].double().cpu().numpy(), g[sample].double().cpu().numpy())
    del uh, coef, u, g
    plan.close()
    torch.cuda.empty_cache()
    return ms / steps, stages, nonfinite, sampled


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    from paper_1201_4060_gb300 import _build, synth
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    from paper_1201_4060_gb300 import bspline as B

    wl = workload()
    N, order, P = wl["N"], wl["order"], wl["P"]
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    xs = synth.clustered_particles(P, seed=rank_particle_seed(wl, rank))
    x = torch.from_numpy(xs).to(device)

    # ---- headline: FP32 coefficients (--dtype: another form, for profiling captures), whole path, K steps
    hd = args.dtype
    plan = B.Plan(N, order, hd)
    uh = dense_field_on_gpu(F, plan.uhat_dtype, device)
    coef = plan.empty_coeffs()
    u = torch.empty((P, 3), dtype=plan.out_dtype, device=device)
    g = torch.empty((P, 3, 3), dtype=plan.out_dtype, device=device)
    stream = torch.cuda.current_stream()

    def step():
        plan.eval(uh, x, coef, u, g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    plan.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if world > 1:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    time.sleep(0.2)
    sampler.stop()
    clocks = sampler.summary(t0, t1)
    stages = plan.stage_times()
    nonfinite = plan.status()
    plan.set_timing(False)
    ms_total = max_over_ranks(ms_total, world, device)
    value = job_throughput(world, P, args.steps, ms_total)
    launches = sum(n for (_, n) in stages.values())

    # ---- roofline of the dominant kernel (largest share of the timed region)
    pk = peaks()
    dom = max(STAGES, key=lambda s: stages[s][0])
    dom_ms = stages[dom][0] / max(stages[dom][1], 1)
    abytes = algorithmic_bytes(dom, N, P, hd, order)
    achieved = abytes / (dom_ms / 1e3) / 1e9
    traffic = measured_traffic(dom, hd, N, order)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "peak_source": pk["source"] + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic, "algorithmic_bytes": abytes, "avg_launch_ms": dom_ms,
                "traffic_source": ("profiles/traffic.txt: DRAM bytes of one launch of this kernel on this workload "
                                   "from a one-pass ncu capture, taken on the same kernel source (hash "
                                   f"{kernel_source_sha(dom)}); not measured in this run" if traffic is not None
                                   else "none for the current kernel source")}
    # the gather's arithmetic: Table 1 multiply-adds per particle against the FP32 FMA pipe
    from_table1 = 6 * order ** 3 + 15 * order ** 2 + 12 * order
    g_ms = stages["gather"][0] / max(stages["gather"][1], 1)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    fma_peak = sms * 128 * pk["sm_max_mhz"] * 1e6
    fma_rate = P * from_table1 / (g_ms / 1e3)
    g_bytes = algorithmic_bytes("gather", N, P, hd, order)
    gather = {"avg_launch_ms": g_ms, "achieved_gbs": g_bytes / (g_ms / 1e3) / 1e9,
              "hbm_frac": g_bytes / (g_ms / 1e3) / 1e9 / pk["hbm_gbs"],
              "fma_per_particle_table1": from_table1, "fma_rate_tfma": fma_rate / 1e12,
              "fma_peak_tfma_at_max_clock": fma_peak / 1e12, "alu_frac_at_max_clock": fma_rate / fma_peak,
              "particles_per_s": P / (g_ms / 1e3),
              # the bound that binds: shared-memory reads of the stencil (3 n^3 FP32 values per particle)
              # against 128 bytes per clock per SM at the maximum clock
              "smem_bytes_per_particle": 3 * order ** 3 * 4,
              "smem_gbs": P * 3 * order ** 3 * 4 / (g_ms / 1e3) / 1e9,
              "smem_peak_gbs_at_max_clock": sms * 128 * pk["sm_max_mhz"] * 1e6 / 1e9,
              "smem_frac_at_max_clock": P * 3 * order ** 3 * 4 / (g_ms / 1e3) / (sms * 128 * pk["sm_max_mhz"] * 1e6),
              "traffic": measured_traffic("gather", hd, N, order)}
    stages_ms = {s: {"total_ms": stages[s][0], "launches": stages[s][1],
                     "share": stages[s][0] / max(sum(v[0] for v in stages.values()), 1e-30)} for s in STAGES}
    # outputs at a fixed sample of particles, for the error against the oracle (computed after the run)
    sample_idx = np.sort(np.random.default_rng(ERR_SAMPLE_SEED).choice(P, ERR_SAMPLE, replace=False))
    sample_t = torch.from_numpy(sample_idx).to(device)
    sampled = {"f32": (u[sample_t].double().cpu().numpy(), g[sample_t].double().cpu().numpy())}
    del uh, coef, u, g
    plan.close()
    torch.cuda.empty_cache()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": hd,
           "data": f"synthetic: Kolmogorov-spectrum field (seed {wl['field_seed']}), clustered particles "
                   f"(seed {wl['particle_seed']} + rank); no dataset",
           "config": config_block(wl, hd, world), "roofline": roofline, "gather": gather,
           "stages_ms": stages_ms, "gpu_launches": launches, "clocks": clocks, "nonfinite_positions": nonfinite}

    # ---- other coefficient forms and the end-to-end number (rank 0 only at N = 1)
    if world == 1 and not args.quick and hd == "f32":
        forms = {"f32": {"particles_per_s": value, "ms_per_step": ms_total / args.steps}}
        ks = max(3, min(args.steps, 20))
        ms_bf, st_bf, _, sampled["bf16"] = run_form(B, wl, F, x, "bf16", ks, 2, device, sample=sample_t)
        gb = st_bf["gather"][0] / max(st_bf["gather"][1], 1)
        forms["bf16"] = {"particles_per_s": P / (ms_bf / 1e3), "ms_per_step": ms_bf, "gather_ms": gb,
                         "gather_hbm_frac": algorithmic_bytes("gather", N, P, "bf16", order) / (gb / 1e3) / 1e9 /
                         pk["hbm_gbs"]}
        ms_64, st_64, _, sampled["f64"] = run_form(B, wl, F, x, "f64", 2, 1, device, sample=sample_t)
        g64 = st_64["gather"][0] / max(st_64["gather"][1], 1)
        forms["f64"] = {"particles_per_s": P / (ms_64 / 1e3), "ms_per_step": ms_64, "gather_ms": g64,
                        "fft_ms": sum(st_64[s][0] / max(st_64[s][1], 1) for s in ("fft_x", "fft_yz"))}
        forms["f32"]["gather_ms"] = g_ms
        if not args.no_cpu_baseline:
            errs = form_errors(sampled, sample_idx)
            for k, v in errs["forms"].items():
                forms[k]["err_vs_oracle"] = v
            forms["f32"]["e_trunc"] = errs["e_trunc"]
            forms["f32"]["e_prec_below_e_trunc"] = errs["e_prec_below_e_trunc"]
        out["forms"] = forms
        out["e2e"] = run_e2e(B, wl, F, xs, device, steps=24)
        out["band"] = run_band(B, wl, F, x, xs, device, ks, sample_t, sampled["f32"])
        orders, o_sampled, o_idx = run_orders(B, device)
        if not args.no_cpu_baseline:
            oe = orders_errors(o_sampled, o_idx)
            for row in orders["rows"]:
                e = oe[f"o{row['order']}_{row['dtype']}"]
                row["err_vs_oracle"] = e["err"]
                row["e_trunc"] = e["e_trunc"]
                if row["dtype"] == "f32":
                    row["e_prec_below_e_trunc"] = e["e_prec_below_e_trunc"]
        out["orders256"] = orders
        out["transform"] = run_transform(B, wl, F, device)
        out["adjoint"] = run_adjoint(B, device)
        out["batch"] = run_batch(B, device)
        out["sparse"] = run_sparse(B, wl, F, device)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(samples=1 << 17)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_adjoint(B, device, steps=10, warmup=3):
    """Adjoint (differentiation) workload: 256^3 Kolmogorov field, cubic B-spline, 2^22 uniform particles,
    N(0, 1) cotangents on u and grad u.  One step = one bspline_spread_adjoint call producing g_u_hat (through
    the spread onto the coefficients and the transposed transform) and g_x, after zeroing g_coeffs."""
    import torch
    from paper_1201_4060_gb300 import synth
    wl = synth.WORKLOADS["adjoint256"]
    N, order, P = wl["N"], wl["order"], wl["P"]
    plan = B.Plan(N, order, "f32")
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    uh = dense_field_on_gpu(F, plan.uhat_dtype, device)
    coef = plan.coeffs(uh)
    x = torch.from_numpy(synth.make_particles(wl["particles"], P, wl["particle_seed"], N)).to(device)
    gu_h, gg_h = synth.cotangents(P, wl["particle_seed"] + 1)
    gu = torch.from_numpy(gu_h).float().to(device)
    gg = torch.from_numpy(gg_h).float().to(device)
    g_coef = torch.zeros((3, N, N, N), dtype=torch.float32, device=device)
    g_uh = torch.empty((3, N, N, N // 2 + 1), dtype=torch.complex64, device=device)
    g_x = torch.empty((P, 3), dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream()
    plan._stream(stream)

    def step():
        g_coef.zero_()
        rc = B.bspline_spread_adjoint(plan.handle, coef.data_ptr(), x.data_ptr(), P, gu.data_ptr(), gg.data_ptr(),
                                      g_coef.data_ptr(), g_uh.data_ptr(), g_x.data_ptr())
        if rc != B.OK:
            raise B.BSplineError(rc, "bspline_spread_adjoint")

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    plan.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = plan.stage_times()
    plan.set_timing(False)
    names = ["bin", "scan", "scatter", "spread", "grad_x", "adj_fft"]
    stages = {s: st[s][0] / max(st[s][1], 1) for s in names}
    # the same steps with the deterministic (fixed-point) spread
    plan.set_deterministic(True)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    plan.set_timing(True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_det = e0.elapsed_time(e1) / steps
    st_det = plan.stage_times()
    plan.set_timing(False)
    plan.set_deterministic(False)
    rec = 16
    coef_b, spec_b = 3 * N ** 3 * 4, 3 * N * N * (N // 2 + 1) * 8
    hp = ((N // 2 + 1) + 7) // 8 * 8
    work_b = 3 * N * N * hp * 8
    abytes = {"spread": P * (rec + 4) + P * 48 + 2 * coef_b,          # records, cotangents, g_coef += (read + write)
              "grad_x": coef_b + P * (rec + 4) + P * 48 + P * 24,     # coefficients once, records, cotangents, g_x
              "adj_fft": coef_b + work_b + 2 * work_b + work_b + spec_b}  # z: read g_coef, write; y: rw; x: r, write
    pk = peaks()
    out = {"workload": f"{N}^3 x 3-component Kolmogorov field (seed {wl['field_seed']}), order-{order} B-spline, "
                       f"{P} uniform particles (seed {wl['particle_seed']}), N(0,1) cotangents on u and grad u "
                       f"(seed {wl['particle_seed'] + 1}), f32 coefficients, f64 positions",
           "particles_per_s": P / (ms / 1e3), "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "step": "g_coeffs zeroed, bin+sort, spread onto coefficients, position gradients, transposed transform",
           "stages_ms": stages,
           "deterministic": {"ms_per_step": ms_det, "particles_per_s": P / (ms_det / 1e3),
                             "spread_ms": st_det["spread"][0] / max(st_det["spread"][1], 1),
                             "how": "bspline_plan_set_deterministic: fixed-point sums, bit-identical per call"},
           "hbm_frac": {s: abytes[s] / (stages[s] / 1e3) / 1e9 / pk["hbm_gbs"] for s in abytes if stages[s] > 0}}
    del uh, coef, x, gu, gg, g_coef, g_uh, g_x
    plan.close()
    torch.cuda.empty_cache()
    return out


def run_orders(B, device, reps=10, sample=ERR_SAMPLE):
    """Config of the orders: 256^3 Kolmogorov field, orders 2/4/6/8, 10^6 uniform particles sorted by cell,
    FP32 and FP64 coefficients.  Per order and form: the evaluation (bspline_interp on built coefficients)
    as given (the library sorts), and with BSPLINE_INTERP_SORTED on the same particles put in the plan's
    brick order (bspline_sort_order, outside the timed region); and the transform alone.  Returns the
    block and the sampled outputs (for the errors against the oracle)."""
    import numpy as np
    import torch
    from paper_1201_4060_gb300 import synth
    wl = synth.WORKLOADS["orders256"]
    N, P = wl["N"], wl["P"]
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    xs = synth.make_particles(wl["particles"], P, wl["particle_seed"], N)
    x = torch.from_numpy(xs).to(device)
    sample_idx = np.sort(np.random.default_rng(ERR_SAMPLE_SEED).choice(P, sample, replace=False))
    st = torch.from_numpy(sample_idx).to(device)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows, sampled = [], {}
    for order in wl["order"]:
        for dtype in ("f32", "f64"):
            plan = B.Plan(N, order, dtype)
            uh = dense_field_on_gpu(F, plan.uhat_dtype, device)
            coef = plan.empty_coeffs()
            t_coef = timed(lambda: plan.coeffs(uh, coef))
            u = torch.empty((P, 3), dtype=plan.out_dtype, device=device)
            g = torch.empty((P, 3, 3), dtype=plan.out_dtype, device=device)
            t_given = timed(lambda: plan.interp(coef, x, u, g))
            sampled[f"o{order}_{dtype}"] = (u[st].double().cpu().numpy(), g[st].double().cpu().numpy())
            perm = plan.sort_order(x).long()
            xp = x[perm].contiguous()
            t_sorted = timed(lambda: plan.interp(coef, xp, u, g, sorted=True))
            # the flagged call's outputs come in the brick order: compare them at the same particles
            inv = torch.empty_like(perm)
            inv[perm] = torch.arange(P, device=device)
            ok = torch.equal(u[inv[st]].double(), torch.from_numpy(sampled[f"o{order}_{dtype}"][0]).to(device))
            rows.append({"order": order, "dtype": dtype, "coeffs_ms": t_coef, "interp_ms": t_given,
                         "particles_per_s": P / (t_given / 1e3), "interp_sorted_flag_ms": t_sorted,
                         "particles_per_s_sorted_flag": P / (t_sorted / 1e3), "sorted_flag_same_u": bool(ok)})
            del uh, coef, u, g, perm, xp, inv
            plan.close()
            torch.cuda.empty_cache()
    out = {"workload": f"{N}^3 Kolmogorov field (seed {wl['field_seed']}), orders {list(wl['order'])}, {P} uniform "
                       f"particles sorted by cell (seed {wl['particle_seed']}), u + grad u",
           "step": "bspline_interp on built coefficients (A3-A6); coeffs_ms = bspline_coeffs (A1-A2) alone",
           "rows": rows, "reps": reps}
    return out, sampled, sample_idx


def run_transform(B, wl, F, device, reps=10):
    """The coefficient transform (prefilter + inverse real 3D FFT, A1-A2) at the headline size: the
    library's two kernels (bspline_coeffs, FP32) beside cuFFT's C2R (torch.fft.irfftn, a timing
    comparator only) preceded by the prefilter as a separate elementwise multiply, on the same half
    spectrum.  HBM fractions count one read of the spectrum and one write of the coefficients."""
    import numpy as np
    import torch
    N, order = wl["N"], wl["order"]
    plan = B.Plan(N, order, "f32")
    uh = dense_field_on_gpu(F, plan.uhat_dtype, device)
    coef = plan.empty_coeffs()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ours = timed(lambda: plan.coeffs(uh, coef))
    rc, c = B.bspline_prefilter_values(N, order, B.PREFILTER_INTERP)
    c = torch.tensor(c, dtype=torch.float32, device=device)
    cxyz = c[:, None, None] * c[None, :, None] * c[None, None, :N // 2 + 1]
    tmp = torch.empty_like(uh)
    res_box = {}

    def cufft():
        torch.mul(uh, cxyz, out=tmp)
        res_box["out"] = torch.fft.irfftn(tmp, s=(N, N, N), dim=(1, 2, 3), norm="forward")

    def cufft_only():
        res_box["out"] = torch.fft.irfftn(tmp, s=(N, N, N), dim=(1, 2, 3), norm="forward")

    t_mul_fft = timed(cufft)
    t_fft = timed(cufft_only)
    out = res_box.pop("out")
    same = float((out - coef).abs().max() / coef.abs().max())
    pk = peaks()
    spec = 3 * N * N * (N // 2 + 1) * 8
    cb = 3 * N ** 3 * 4
    res = {"workload": f"{N}^3 x 3 half spectrum (complex64) -> FP32 coefficients, order {order} prefilter",
           "ours_ms": ours, "ours_hbm_frac": (spec + cb) / (ours / 1e3) / 1e9 / pk["hbm_gbs"],
           "cufft_c2r_plus_multiply_ms": t_mul_fft, "cufft_c2r_only_ms": t_fft,
           "cufft_c2r_hbm_frac": (spec + cb) / (t_fft / 1e3) / 1e9 / pk["hbm_gbs"],
           "ours_vs_cufft_with_multiply": t_mul_fft / ours,
           "max_rel_diff_vs_cufft": same,
           "note": "cuFFT via torch.fft.irfftn is a timing comparator only; the path never calls it"}
    del uh, coef, out, tmp, cxyz
    plan.close()
    torch.cuda.empty_cache()
    return res


def run_sparse(B, wl, F, device, reps=5):
    """The gather split on sparse particle sets (same 512^3 quintic field, FP32): per-call interpolation time
    with every brick staged, with the automatic split, and with the split bspline_plan_autotune picks."""
    import numpy as np
    import torch
    from paper_1201_4060_gb300 import synth
    N, order = wl["N"], wl["order"]
    plan = B.Plan(N, order, "f32")
    coef = plan.coeffs(dense_field_on_gpu(F, plan.uhat_dtype, device))
    out = {"workload": f"{N}^3 field of the headline, order {order}, f32 coefficients, uniform particles (seed 11)",
           "cases": []}

    def timed(x, u, g):
        for _ in range(2):
            plan.interp(coef, x, u, g)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.interp(coef, x, u, g)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for lp in (18, 20):
        P = 1 << lp
        x = torch.from_numpy(synth.uniform_particles(P, seed=11)).to(device)
        u = torch.empty((P, 3), device=device)
        g = torch.empty((P, 3, 3), device=device)
        plan.set_gather_split(0)
        staged = timed(x, u, g)
        plan.set_gather_split(B.GATHER_SPLIT_AUTO)
        auto = timed(x, u, g)
        split, _ = plan.autotune(coef, x, u, g)
        tuned = timed(x, u, g)
        out["cases"].append({"particles": P, "particles_per_brick": P / (-(-N // 16)) ** 2 / (-(-N // 12)),
                             "interp_ms_all_staged": staged, "interp_ms_auto": auto, "autotuned_split": split,
                             "interp_ms_autotuned": tuned, "particles_per_s_autotuned": P / (tuned / 1e3)})
        del x, u, g
    plan.close()
    del coef
    torch.cuda.empty_cache()
    return out


def run_batch(B, device, steps=10, warmup=3):
    """64 independent small fields (grids 32..192 including 3 * 2^k, log-uniform 1e3..1e6 particles each),
    cubic, FP32: the whole batch replayed as one CUDA graph launch (streams chosen by the autotuner), and
    the same work as eager per-field calls for comparison.  One step = every field once."""
    import torch
    from paper_1201_4060_gb300 import synth
    wl = synth.WORKLOADS["batch64"]
    spec = synth.batch_workload(wl["nfields"], wl["field_seed"], wl["particle_seed"])
    order = wl["order"]
    plans, uh, co, xs, ou, og = [], [], [], [], [], []
    for f in spec:
        plan = B.Plan(f["N"], order, "f32")
        F = synth.kolmogorov_field(f["N"], seed=f["field_seed"])
        plans.append(plan)
        uh.append(dense_field_on_gpu(F, plan.uhat_dtype, device))
        co.append(plan.empty_coeffs())
        xs.append(torch.from_numpy(synth.uniform_particles(f["P"], seed=f["particle_seed"])).to(device))
        ou.append(torch.empty((f["P"], 3), dtype=torch.float32, device=device))
        og.append(torch.empty((f["P"], 3, 3), dtype=torch.float32, device=device))
    total = sum(f["P"] for f in spec)
    stream = torch.cuda.current_stream()
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=4)
    k, _ = batch.autotune(stream)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_graph = timed(lambda: batch.launch(stream))
    cfg = batch.config()
    status, nonfinite = batch.status()

    def eager():
        for i in range(len(plans)):
            plans[i].coeffs(uh[i], co[i])
            plans[i].interp(co[i], xs[i], ou[i], og[i])

    ms_eager = timed(eager)
    # the same batch with every plan told its field's band (the generator's |k| <= N/3): the grouped
    # transforms skip the zero modes (same bits as the full path, tested)
    for i, f in enumerate(spec):
        plans[i].set_band(f["N"] // 3)
    batch.capture(uh, co, xs, ou, og, streams=k)
    ms_band = timed(lambda: batch.launch(stream))
    grids = sorted(set(f["N"] for f in spec))
    out = {"workload": f"{len(spec)} fields, grids {grids} (field i: grid {list(synth.BATCH_GRIDS)}[i mod 6], "
                       f"seed {wl['field_seed']} + i), order-{order} B-spline, f32 coefficients, uniform particles "
                       f"log-uniform 1e3..1e6 per field (seed {wl['particle_seed']}), {total} in all",
           "particles": total, "particles_per_s": total / (ms_graph / 1e3), "ms_per_batch": ms_graph,
           "graph_streams": k, "graph_launches_per_batch": 1, "kernel_launches_per_batch": cfg["kernel_nodes"],
           "particle_side": ("one persistent queue kernel (count, scan, placement and gather tasks of every field)"
                             if cfg["queue"] else "per-field kernels"),
           "queue_brick_y": cfg["brick_y"], "queue_item_particles": cfg["item_particles"],
           "status": status, "nonfinite": nonfinite,
           "eager_ms_per_batch": ms_eager, "eager_particles_per_s": total / (ms_eager / 1e3),
           "band_ms_per_batch": ms_band, "band_particles_per_s": total / (ms_band / 1e3),
           "steps": steps, "warmup": warmup}
    batch.close()
    for p in plans:
        p.close()
    del uh, co, xs, ou, og
    torch.cuda.empty_cache()
    return out


def run_band(B, wl, F, x, xs, device, steps, sample_t, full_sampled):
    """The same workload on plans told that the field is band-limited (bspline_plan_set_band with the
    generator's |k| <= N/3, the 2/3-rule dealiasing of pseudo-spectral codes): the transform skips the
    zero modes and bspline_run_host copies only the band box.  The outputs must be the full path's bits;
    reported beside the headline, which takes every mode of the spectrum."""
    import numpy as np
    N, P = wl["N"], wl["P"]
    K = N // 3
    ms, st, _, samp = run_form(B, wl, F, x, "f32", steps, 2, device, sample=sample_t, band=K)
    same = bool(np.array_equal(samp[0], full_sampled[0]) and np.array_equal(samp[1], full_sampled[1]))
    return {"kmax": K, "input": f"modes with |kx|, |ky|, kz <= {K} (the field generator's band, |k| <= N/3)",
            "particles_per_s": P / (ms / 1e3), "ms_per_step": ms,
            "fft_x_ms": st["fft_x"][0] / max(st["fft_x"][1], 1), "fft_yz_ms": st["fft_yz"][0] / max(st["fft_yz"][1], 1),
            "gather_ms": st["gather"][0] / max(st["gather"][1], 1),
            "sampled_outputs_equal_full_path": same,
            "e2e": run_e2e(B, wl, F, xs, device, steps=24, band=K)}


def e2e_h2d_bytes(N: int, P: int, band: int = 0) -> int:
    """Host-to-device bytes of one end-to-end step: the complex64 half spectrum [3][N][N][N/2+1] (with a band K,
    only the box kx, ky in [0, K] and [N - K, N), kz in [0, K] that bspline_run_host copies) and the FP64
    positions [P][3]."""
    modes = 3 * (2 * band + 1) ** 2 * (band + 1) if band else 3 * N * N * (N // 2 + 1)
    return modes * 8 + P * 3 * 8


def run_e2e(B, wl, F, xs, device, steps, band=0):
    """Same metric through the host-buffer API: every step copies u_hat and the positions from pinned
    host memory to the device and u and grad u back, all inside the timed region.  Steps alternate
    between two plans on two streams (bspline_run_host_async, then bspline_wait before a plan is
    reused), so one step's result copy overlaps the next step's input copy, as a caller streaming
    steps would run them; the value is a whole sequence over its step count, the median of three
    sequences.  A single
    synchronous bspline_run_host call is timed as well, for reference."""
    import numpy as np
    import torch
    N, order, P = wl["N"], wl["order"], wl["P"]
    plans = [B.Plan(N, order, "f32") for _ in range(2)]
    for p in plans:
        if band:
            p.set_band(band)                             # only the band box of u_hat crosses the host link
    streams = [torch.cuda.Stream(device) for _ in range(2)]
    uh = torch.from_numpy(F.dense(np.complex64)).pin_memory()
    xh = torch.from_numpy(xs).pin_memory()
    outs = [(torch.empty((P, 3), dtype=torch.float32).pin_memory(),
             torch.empty((P, 3, 3), dtype=torch.float32).pin_memory()) for _ in range(2)]
    for i in range(2):                                   # first calls allocate the plans' device buffers
        plans[i].run_host(uh, xh, *outs[i], stream=streams[i])
    t = time.perf_counter()
    plans[0].run_host(uh, xh, *outs[0], stream=streams[0])
    single = time.perf_counter() - t
    # three sequences of `steps` steps, their median: the host link is shared with the host's other work,
    # and single sequences have varied between runs from 10.7 to 17.7 ms per step at 512^3 / 2^24
    seqs = []
    for _ in range(3):
        t0 = time.perf_counter()
        for k in range(steps):
            i = k % 2
            plans[i].wait()                              # its previous step is done: buffers free
            plans[i].run_host(uh, xh, *outs[i], stream=streams[i], wait=False)
        for p in plans:
            p.wait()
        seqs.append((time.perf_counter() - t0) / steps)
    t = statistics.median(seqs)
    for p in plans:
        p.close()
    h2d = e2e_h2d_bytes(N, P, band)
    d2h = outs[0][0].numel() * 4 + outs[0][1].numel() * 4
    del uh, xh, outs
    torch.cuda.empty_cache()
    return {"value": P / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": t * 1e3, "steps": steps, "sequences_ms_per_step": [s * 1e3 for s in seqs],
            "single_call_ms": single * 1e3,
            "api": "bspline_run_host_async + bspline_wait on two alternating plans (pinned host buffers)"}


# ----------------------------------------------------------------------------- oracle (CPU)
# The oracle runs only here, in child processes (single-threaded numpy each): the CPU baseline (one core,
# and every host core as separate processes), and the error of each form's sampled outputs against it.

ORACLE_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _component_half(F, c):
    import numpy as np
    N = F.N
    half = np.zeros((1, N, N, N // 2 + 1), np.complex128)
    half[0, F.idx[:, 0], F.idx[:, 1], F.idx[:, 2]] = F.val[c]
    return half


def cpu_worker(mode: str, samples: int, steps: int = 1, warmup: int = 0) -> dict:
    """Runs in a child process with single-threaded numpy: times the oracle on a bounded sample."""
    import numpy as np
    from oracle import bspline_oracle as O
    from paper_1201_4060_gb300 import synth
    wl = workload()
    N, order, P = wl["N"], wl["order"], wl["P"]
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    # coefficient build of one component at full size (the three components are identical work)
    half = _component_half(F, 0)
    t = time.perf_counter()
    c = O.coefficients(half, order)
    t_coef1 = time.perf_counter() - t
    cb = np.broadcast_to(c, (3, N, N, N))
    x = synth.clustered_particles(P, seed=wl["particle_seed"])
    rng = np.random.default_rng(0)
    g_times = []
    for i in range(warmup + steps):
        sel = x[rng.integers(0, P, samples)]
        t = time.perf_counter()
        O.evaluate(cb, sel, order)
        dt = time.perf_counter() - t
        if i >= warmup:
            g_times.append(dt)
    t_g = statistics.mean(g_times)
    t_step = 3 * t_coef1 + t_g * (P / samples)
    return {"t_coef_one_component_s": t_coef1, "t_gather_sample_s": t_g, "gather_sample": samples,
            "t_step_est_s": t_step, "per_step_est_s": [3 * t_coef1 + tg * (P / samples) for tg in g_times]}


# --- every host core: one process per core (spawned), the coefficients in shared memory

def _pool_init():
    for k, v in ORACLE_ENV.items():
        os.environ[k] = v


def _pool_noop(_):
    import numpy  # noqa: F401  (imports paid before the timed region)
    from oracle import bspline_oracle  # noqa: F401
    return os.getpid()


def _pool_build(args):
    """One component's coefficients (prefilter + inverse real FFT, oracle) into the shared array."""
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import bspline_oracle as O
    shm_half, shm_coef, c, N, order = args
    h = shared_memory.SharedMemory(name=shm_half)
    k = shared_memory.SharedMemory(name=shm_coef)
    try:
        half = np.ndarray((3, N, N, N // 2 + 1), np.complex128, buffer=h.buf)
        coef = np.ndarray((3, N, N, N), np.float64, buffer=k.buf)
        coef[c] = O.coefficients(half[c:c + 1], order)[0]
        del half, coef
    finally:
        h.close()
        k.close()
    return c


def _pool_eval(args):
    """u and grad u of one chunk of the sample (oracle), from the shared coefficients."""
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import bspline_oracle as O
    shm_coef, N, order, xs = args
    k = shared_memory.SharedMemory(name=shm_coef)
    try:
        coef = np.ndarray((3, N, N, N), np.float64, buffer=k.buf)
        u, g = O.evaluate(coef, xs, order)
        del coef
    finally:
        k.close()
    return float(np.abs(u).sum() + np.abs(g).sum())


def cpu_worker_all_cores(samples: int, steps: int = 1, warmup: int = 0) -> dict:
    """The oracle on every host core: the three components' coefficient builds in parallel processes
    (once), then per step u / grad u of a fresh sample of particles split over one process per core;
    wall-clock per stage, each step's estimate = coefficient build + the sample scaled to every particle."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    from paper_1201_4060_gb300 import synth
    wl = workload()
    N, order, P = wl["N"], wl["order"], wl["P"]
    cores = os.cpu_count() or 1
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    x = synth.clustered_particles(P, seed=wl["particle_seed"])
    rng = np.random.default_rng(0)
    hb = 3 * N * N * (N // 2 + 1) * 16
    cbytes = 3 * N ** 3 * 8
    sh = shared_memory.SharedMemory(create=True, size=hb)
    sk = shared_memory.SharedMemory(create=True, size=cbytes)
    try:
        half = np.ndarray((3, N, N, N // 2 + 1), np.complex128, buffer=sh.buf)
        half[...] = F.dense()
        del half
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_pool_init) as pool:
            pool.map(_pool_noop, range(cores))
            t = time.perf_counter()
            pool.map(_pool_build, [(sh.name, sk.name, c, N, order) for c in range(3)])
            t_coef = time.perf_counter() - t
            g_times = []
            for i in range(warmup + steps):
                chunks = np.array_split(x[rng.integers(0, P, samples)], cores)
                t = time.perf_counter()
                pool.map(_pool_eval, [(sk.name, N, order, ch) for ch in chunks], chunksize=1)
                if i >= warmup:
                    g_times.append(time.perf_counter() - t)
    finally:
        sh.close()
        sh.unlink()
        sk.close()
        sk.unlink()
    t_g = statistics.mean(g_times)
    return {"cores": cores, "t_coef_s": t_coef, "t_gather_sample_s": t_g, "gather_sample": samples,
            "t_step_est_s": t_coef + t_g * (P / samples),
            "per_step_est_s": [t_coef + tg * (P / samples) for tg in g_times]}


def cpu_worker_errors(path: str) -> dict:
    """Errors of each form's sampled outputs against the oracle (FP64): normwise max and RMS, per quantity,
    against the oracle of the exact FP64 spectrum and (FP32 / BF16 forms, which take a complex64
    spectrum) of that rounded input; the method's truncation error E_trunc (Section 5, Eqs. l2-error /
    l2-error-der, closed form over the field's modes) beside the FP32 form's E_prec."""
    import math as m
    import numpy as np
    from oracle import bspline_oracle as O
    from paper_1201_4060_gb300 import synth
    wl = workload()
    N, order = wl["N"], wl["order"]
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    d = np.load(path)
    xs = d["x"]

    def oracle_at(field):
        ou = np.empty((xs.shape[0], 3))
        og = np.empty((xs.shape[0], 3, 3))
        for c in range(3):
            coef_c = O.coefficients(_component_half(field, c), order)[0]
            uc, gc = O.evaluate(np.broadcast_to(coef_c, (3, N, N, N)), xs, order)
            ou[:, c] = uc[:, 0]
            og[:, c, :] = gc[:, 0, :]
            del coef_c
        return ou, og

    def errs(u, g, ou, og):
        return {"u_normwise": float(np.abs(u - ou).max() / np.abs(ou).max()),
                "grad_normwise": float(np.abs(g - og).max() / np.abs(og).max()),
                "u_rms_rel": float(m.sqrt(np.mean((u - ou) ** 2) / np.mean(ou ** 2))),
                "grad_rms_rel": float(m.sqrt(np.mean((g - og) ** 2) / np.mean(og ** 2)))}

    exact = oracle_at(F)
    rounded = oracle_at(F.rounded(np.complex64))
    out = {"forms": {}}
    for form in ("f32", "bf16", "f64"):
        if f"{form}_u" not in d:
            continue
        u, g = d[f"{form}_u"], d[f"{form}_g"]
        e = {"vs_exact_input": errs(u, g, *exact), "sample": int(xs.shape[0])}
        if form != "f64":
            e["vs_complex64_input"] = errs(u, g, *rounded)
        out["forms"][form] = e
    mse_u, mse_g = O.l2_error_field(N, F.idx, F.val, order)
    ou, og = exact
    tr = {"u": m.sqrt(mse_u.sum() / 3.0 / np.mean(ou ** 2)), "grad": m.sqrt(mse_g.sum() / 9.0 / np.mean(og ** 2))}
    out["e_trunc"] = {"u_rms_rel": tr["u"], "grad_rms_rel": tr["grad"],
                      "how": "closed form of Section 5 (l2-error, l2-error-der) over the field's modes"}
    if "f32" in out["forms"]:
        ep = out["forms"]["f32"]["vs_exact_input"]
        out["e_prec_below_e_trunc"] = bool(ep["u_rms_rel"] < tr["u"] and ep["grad_rms_rel"] < tr["grad"])
    return out


def _spawn_worker(mode, samples, steps=1, warmup=0, extra=()):
    env = dict(os.environ, **ORACLE_ENV)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", mode, "--samples", str(samples),
           "--steps", str(steps), "--warmup", str(warmup), *extra]
    for k, v in _OVERRIDE.items():
        cmd += [f"--{k}", str(v)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle worker failed:\n{r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def form_errors(sampled: dict, sample_idx) -> dict:
    """Each form's error at the sampled particles, against the oracle run in a child process."""
    import tempfile
    import numpy as np
    from paper_1201_4060_gb300 import synth
    wl = workload()
    x = synth.clustered_particles(wl["P"], seed=wl["particle_seed"])[sample_idx]
    arrays = {"x": x}
    for k, (u, g) in sampled.items():
        arrays[f"{k}_u"] = u
        arrays[f"{k}_g"] = g
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sampled.npz")
        np.savez(path, **arrays)
        return _spawn_worker("errors", 0, extra=("--in", path))


def cpu_worker_orders_errors(path: str) -> dict:
    """Per order and form of the orders block: the sampled outputs' error against the oracle (FP64, on the
    exact spectrum), E_prec (RMS) beside E_trunc (closed form of Section 5) per order."""
    import math as m
    import numpy as np
    from oracle import bspline_oracle as O
    from paper_1201_4060_gb300 import synth
    wl = synth.WORKLOADS["orders256"]
    N, P = wl["N"], wl["P"]
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    d = np.load(path)
    xs = synth.make_particles(wl["particles"], P, wl["particle_seed"], N)[d["idx"]]
    half = F.dense()
    out = {}
    for order in wl["order"]:
        ou, og = O.evaluate(O.coefficients(half, order), xs, order)
        mse_u, mse_g = O.l2_error_field(N, F.idx, F.val, order)
        tr_u = m.sqrt(mse_u.sum() / 3.0 / np.mean(ou ** 2))
        tr_g = m.sqrt(mse_g.sum() / 9.0 / np.mean(og ** 2))
        for dtype in ("f32", "f64"):
            u, g = d[f"o{order}_{dtype}_u"], d[f"o{order}_{dtype}_g"]
            err = {"u_normwise": float(np.abs(u - ou).max() / np.abs(ou).max()),
                   "grad_normwise": float(np.abs(g - og).max() / np.abs(og).max()),
                   "u_rms_rel": float(m.sqrt(np.mean((u - ou) ** 2) / np.mean(ou ** 2))),
                   "grad_rms_rel": float(m.sqrt(np.mean((g - og) ** 2) / np.mean(og ** 2)))}
            out[f"o{order}_{dtype}"] = {"err": err, "e_trunc": {"u_rms_rel": tr_u, "grad_rms_rel": tr_g},
                                        "e_prec_below_e_trunc": bool(err["u_rms_rel"] < tr_u and
                                                                     err["grad_rms_rel"] < tr_g)}
    return out


def orders_errors(sampled: dict, sample_idx) -> dict:
    import tempfile
    import numpy as np
    arrays = {"idx": sample_idx}
    for k, (u, g) in sampled.items():
        arrays[f"{k}_u"] = u
        arrays[f"{k}_g"] = g
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "orders.npz")
        np.savez(path, **arrays)
        return _spawn_worker("orders-errors", 0, extra=("--in", path))


def cpu_baseline(samples: int) -> dict:
    wl = workload()
    one = _spawn_worker("baseline", samples)
    allc = _spawn_worker("baseline-all", samples * 16)
    cores = allc["cores"]
    model = cpu_model()
    return {"value": wl["P"] / allc["t_step_est_s"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": f"numpy FP64 oracle, {cores} single-threaded processes ({model}): the 3 components' "
                      f"coefficient builds at full {wl['N']}^3 in parallel ({allc['t_coef_s']:.2f} s) + u/grad u "
                      f"at {samples * 16} of the {wl['P']} particles split over {cores} processes "
                      f"({allc['t_gather_sample_s']:.2f} s, x{wl['P'] / (samples * 16):g})",
            "t_step_est_s": allc["t_step_est_s"],
            "cores_all": {"value": wl["P"] / allc["t_step_est_s"], "cores": cores, **allc},
            "cores_1": {"value": wl["P"] / one["t_step_est_s"], "cores": 1,
                        "sample": f"one thread: coefficient build of one of the 3 components at full {wl['N']}^3 "
                                  f"(x3) + u/grad u at {samples} of the {wl['P']} particles "
                                  f"(x{wl['P'] // samples}); {one['t_coef_one_component_s']:.2f} s + "
                                  f"{one['t_gather_sample_s']:.2f} s measured",
                        **one}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    wl = workload()
    samples = 1 << 17
    w = _spawn_worker("baseline-all", samples, steps=args.steps, warmup=args.warmup)
    per = w["per_step_est_s"]
    t_step = statistics.mean(per)
    value = wl["P"] / t_step
    cores = w["cores"]
    sample = (f"numpy FP64 oracle on {cores} single-threaded processes ({cpu_model()}): the 3 components' "
              f"coefficient builds at full {wl['N']}^3 in parallel, timed once ({w['t_coef_s']:.2f} s, counted in "
              f"every step) + per step u/grad u at {samples} random particles of {wl['P']} split over the "
              f"processes (x{wl['P'] / samples:g})")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (same recipe and seeds)",
           "config": config_block(wl, "f64 (oracle)", world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_part(args) -> dict:
    """One secondary block alone on cuda:0 (for ncu captures of its kernels)."""
    import torch
    from paper_1201_4060_gb300 import _build, synth
    _build.build()
    from paper_1201_4060_gb300 import bspline as B
    device = torch.device("cuda", 0)
    if args.part == "adjoint":
        return run_adjoint(B, device, steps=args.steps, warmup=args.warmup)
    if args.part == "batch":
        return run_batch(B, device, steps=args.steps, warmup=args.warmup)
    if args.part == "orders":
        return run_orders(B, device)[0]
    wl = workload()
    F = synth.kolmogorov_field(wl["N"], seed=wl["field_seed"])
    return run_transform(B, wl, F, device)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="headline only (no other forms, no e2e)")
    ap.add_argument("--dtype", choices=["f32", "bf16", "f64"], default="f32",
                    help="coefficient type of the timed step (f32 is the benchmark; others for profiling captures)")
    ap.add_argument("--part", choices=["adjoint", "batch", "orders", "transform"], default=None,
                    help="run one secondary block alone and print it (profiling captures; not a bench line)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--samples", type=int, default=4096, help=argparse.SUPPRESS)
    ap.add_argument("--in", dest="input", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--N", type=int, default=None, help="grid size override (profiling captures only)")
    ap.add_argument("--P", type=int, default=None, help="particle count override (profiling captures only)")
    args = ap.parse_args()
    if args.N:
        _OVERRIDE["N"] = args.N
    if args.P:
        _OVERRIDE["P"] = args.P
    if args.cpu_worker == "baseline-all":
        print(json.dumps(cpu_worker_all_cores(args.samples, args.steps, args.warmup)))
        return
    if args.cpu_worker == "errors":
        print(json.dumps(cpu_worker_errors(args.input)))
        return
    if args.cpu_worker == "orders-errors":
        print(json.dumps(cpu_worker_orders_errors(args.input)))
        return
    if args.cpu_worker:
        print(json.dumps(cpu_worker(args.cpu_worker, args.samples, args.steps, args.warmup)))
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.part:
        print(json.dumps(run_part(args)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
