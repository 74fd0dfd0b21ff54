#!/usr/bin/env python3
"""Benchmark of the DFS spectral-interpolation step (type-2 NUFFT) on GB300.

One step = set_points (fold + bin the departure points) + execute (all fields:
deconvolve/pad + theta FFT pass + phi FFT pass + interpolation) on one batch of
synthetic input already resident in HBM.  The default workload is the
2048 x 1024 grid with three fields (h, u, v) in FP32 with FP64 coordinate
folding (2,097,152 departure points).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

With N > 1 the script runs under torch.distributed.run, one replica per GPU
(the interpolation of independent members shards with no exchange: weak scaling).
``--impl reference`` times the FP64 direct-sum oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NUFFT interp points·fields/s at stated error; HBM roofline frac; p50/p99 lat"
UNIT = "point-fields/s"
L2_FLUSH_BYTES = 512 << 20          # written between timed steps (L2 is 126 MB)

WORKLOADS = {
    "c3_2048x1024_f32": ("f32", "c3"),
    "c3pr_2048x1024_f32": ("f32", "c3pr"),
    "c3grid_2048x1024_f32": ("f32", "c3grid"),
    "c3sl_2048x1024_f32": ("f32", "c3sl"),
    "c3lag_2048x1024_f32": ("f32", "c3lag"),
    "c3lag_2048x1024_f64": ("f64", "c3lag"),
    "c3gl_2048x1024_f32": ("f32", "c3gl"),
    "c4_ensemble_f32": ("f32", "c4"),
    "c3_2048x1024_f64": ("f64", "c3"),
    "c2_512x256_f64": ("f64", "c2"),
    "c2_512x256_f32": ("f32", "c2"),
    "c1_64x32_f64": ("f64", "c1"),
}
DEFAULT_WORKLOAD = "c3_2048x1024_f32"


def make_workload(name):
    from paper_2605_01313_gb300 import synth
    dtype, kind = WORKLOADS[name]
    if kind == "c4":
        return synth.workload_c4()
    if kind == "c3":
        return synth.workload_c3(dtype)
    if kind == "c3grid":
        # the C3 departure points; the fields (h, u, v) of the tilted steady zonal
        # flow given by their samples on the arrival grid (the whole step)
        wl = synth.workload_c3(dtype)
        alpha = math.pi / 2 - 0.05
        lon_a, colat_a = synth.grid0_points(wl.n_lon, wl.n_lat)
        h, u, v = synth.zonal_flow_values(lon_a, colat_a, alpha)
        wl.grid = np.stack([h, u, v]).reshape(3, wl.n_lat, wl.n_lon)
        wl.parity = [1, -1, -1]
        wl.coeffs = np.stack(synth.zonal_flow_coeffs(wl.n_lon, wl.n_lat, alpha))
        wl.name = "c3grid_%dx%d_%s" % (wl.n_lon, wl.n_lat, dtype)
        return wl
    if kind == "c3sl":
        # the whole semi-Lagrangian interpolation step of the tilted steady zonal
        # flow (TC2 of Sec. 6, 1800 s): departure points from the Eq. 2.4 terms on
        # the arrival grid, (h, u, v) from their arrival-grid samples carried
        # there, the wind rotated back to the arrival frame
        wl = synth.workload_c3(dtype)
        alpha = math.pi / 2 - 0.05
        dt = 1800.0
        lon_a, colat_a = synth.grid0_points(wl.n_lon, wl.n_lat)
        h, u, v = synth.zonal_flow_values(lon_a, colat_a, alpha)
        wl.grid = np.stack([h, u, v]).reshape(3, wl.n_lat, wl.n_lon)
        wl.parity = [1, -1, -1]
        wl.coeffs = np.stack(synth.zonal_flow_coeffs(wl.n_lon, wl.n_lat, alpha))
        w, wa = synth.zonal_flow_settls_terms(lon_a, colat_a, alpha, dt)
        wl.sl = {"w": w.reshape(2, wl.n_lat, wl.n_lon), "wa": wa.reshape(2, wl.n_lat, wl.n_lon),
                 "dt_over_a": dt / synth.EARTH_RADIUS, "iterations": 3}
        wl.lon, wl.colat = lon_a, colat_a       # arrival points; departures come from the step
        wl.name = "c3sl_%dx%d_%s" % (wl.n_lon, wl.n_lat, dtype)
        return wl
    if kind == "c3gl":
        # the C3 departure points; the fields (h, u, v) of the tilted steady zonal
        # flow sampled on a Gauss-Legendre latitude grid (the spherical-harmonic
        # model's grid, Sec. 3 and 5): coefficients by the latitude solve each step
        wl = synth.workload_c3(dtype)
        alpha = math.pi / 2 - 0.05
        wl.parity = [1, -1, -1]
        wl.coeffs = np.stack(synth.zonal_flow_coeffs(wl.n_lon, wl.n_lat, alpha))

        def sampler(colat, wl=wl, alpha=alpha):
            cc, ll = np.meshgrid(colat, np.arange(wl.n_lon) * 2 * math.pi / wl.n_lon,
                                 indexing="ij")
            h, u, v = synth.zonal_flow_values(ll.ravel(), cc.ravel(), alpha)
            return np.stack([h, u, v]).reshape(3, wl.n_lat, wl.n_lon)
        wl.gauss = sampler
        wl.grid = np.zeros((3, wl.n_lat, wl.n_lon))       # replaced once the plan's nodes exist
        wl.name = "c3gl_%dx%d_%s" % (wl.n_lon, wl.n_lat, dtype)
        return wl
    if kind == "c3lag":
        # the C3 spectra and departure points, the fields given by their samples on
        # the arrival grid: the spectral step (grid -> coefficients -> NUFFT) timed,
        # and beside it the cubic and quintic Lagrange interpolation of the same
        # samples (the paper's baseline), with the error of all three
        wl = synth.workload_c3(dtype)
        wl.grid = synth.coeffs_to_grid_samples(wl.coeffs, wl.n_lon, wl.n_lat)
        wl.parity = [1, -1, -1]
        wl.lag = (3, 5)
        wl.name = "c3lag_%dx%d_%s" % (wl.n_lon, wl.n_lat, dtype)
        return wl
    if kind == "c3pr":
        # the C3 points; fields given as partial-regularity coefficients (Sec. 4),
        # truncated as in the paper (N = J - 2, M = J - 1)
        wl = synth.workload_c3(dtype)
        rng = np.random.default_rng(33)
        J = wl.n_lat
        wl.pr = np.stack([synth.random_pr_spectrum(rng, J - 1, J - 2, 3.0) for _ in range(3)])
        wl.coeffs = None                  # complex form only for the oracle legs
        wl.name = "c3pr_%dx%d_%s" % (wl.n_lon, wl.n_lat, dtype)
        return wl
    if kind == "c2":
        return synth.workload_c2(dtype)
    return synth.workload_c1()


# ------------------------------------------------------------------ helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.lines = []
        self.proc = None
        self.gpu_id = gpu_id
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
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
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def stage_bytes(prm, n_fields, n_points, rows):
    """Algorithmic HBM bytes per launch of each stage (one execute of all fields):
    what each stage must read and write once.  A real-field plan reads the
    coefficient columns m >= 0 (plus the Nyquist column) and keeps N1/2 + 1
    theta-pass columns; the fine grid holds the real part only."""
    cs = 16 if prm["dtype"] == 0 else 8
    rs = cs // 2
    N1, N2, n1 = prm["N1"], prm["N2"], prm["n1"]
    F, P = n_fields, n_points
    herm = prm.get("flags", 0) & 1
    cin = N1 // 2 + 2 if herm else N1            # coefficient columns read
    tc = N1 // 2 + 1 if herm else N1             # theta-pass columns
    rec = 8 + 2 * rs + 4                       # sorted record: base int2, offsets, index
    return {
        "set_points": P * (16 + 4) + P * (16 + 4) + P * rec,
        "theta_pass": F * (N2 * cin * cs + rows * tc * cs) + 8 * (N1 + N2),
        "phi_pass": F * (rows * tc * cs + rows * n1 * rs),     # writes the real part only
        "interp": F * (rows * n1 * rs + P * rs) + P * rec,
    }


def model_bytes(prm, n_fields, n_points):
    """Bytes of the reference traffic model of one step: a complex oversampled
    grid, two-pass pruned FFT and one interpolation pass, per field
    N1 N2 c (1 + 2 sigma + 2 sigma^2) + 16 P / F + s_out P (13 N1 N2 c at sigma 2)."""
    cs = 16 if prm["dtype"] == 0 else 8
    rs = cs // 2
    sg = prm.get("sigma", 2) or 2
    per_field = prm["N1"] * prm["N2"] * cs * (1 + 2 * sg + 2 * sg * sg) + rs * n_points
    return n_fields * per_field + 16 * n_points


def interp_flops(prm, n_fields, n_points):
    """Algorithmic flops of one interpolation launch: per point, the w x w real
    tap sum and the w-row combination for every field (2 w (w + 1) each) plus
    the 2 w kernel weights by degree-w Horner polynomials (4 w^2)."""
    w = prm["w"]
    return n_fields * n_points * 2 * w * (w + 1) + n_points * 4 * w * w


def df32_interp_ops(prm, n_fields, n_points):
    """FP32 arithmetic instructions (FADD, FMUL, FFMA: one each) of one
    double-single interpolation launch (FP64 plans, k_interp_df), counted from
    its operations: TwoSum 6, TwoProduct 2, a double-single product 7 (with its
    fast renormalisation), sum 11, Horner step 15, Dot2 step 12.  Per point: the
    x and y weights, each (w + 1) / 2 mirror pairs of an even and an odd Horner
    chain (w - 1 steps together), one product s o and the two sums, plus u = s^2
    for each axis; per point and field, w stencil rows of w Dot2 steps, each row
    then renormalised (3) and added by one more Dot2 step."""
    w = prm["w"]
    pairs = (w + 1) // 2
    weights = pairs * ((w - 1) * 15 + 7 + 2 * 11) + 7
    rows = w * (12 * w + 3 + 12)
    return n_points * (2 * weights + n_fields * rows)


def fft_flops(prm, n_fields, rows, stage):
    """Algorithmic flops of one FFT pass, 5 L log2 L a complex transform of
    length L: the theta pass transforms the coefficient columns (N1/2 + 1 of a
    real-field plan, else N1) at length n2; the phi pass the needed rows at
    length n1 / 2 (its complex-to-real form)."""
    if stage == "theta_pass":
        cols = prm["N1"] // 2 + 1 if prm["flags"] & 1 else prm["N1"]
        L = prm["n2"]
        return n_fields * cols * 5.0 * L * math.log2(L)
    L = prm["n1"] // 2
    return n_fields * rows * 5.0 * L * math.log2(L)


def profile_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if the kernel's source is unchanged since the capture."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        text = open(os.path.join(pdir, fn)).read()
        meta = dict(re.findall(r"^- (\w+): `?([^`\n]+)`?$", text, flags=re.M))
        if meta.get("stage") != kernel or meta.get("workload") != workload:
            continue
        src = meta.get("source_file")
        if not src or "dram_bytes_per_launch" not in meta:
            continue
        path = os.path.join(ROOT, src)
        if not os.path.exists(path):
            continue
        h = hashlib.sha1(open(path, "rb").read()).hexdigest()
        if h != meta.get("source_sha1"):
            return None
        try:
            return float(meta["dram_bytes_per_launch"])
        except ValueError:
            return None
    return None


def set_points_launches(prm):
    """Kernels one set_points launches: one fold for unsorted points; else
    fold+count, the in-bin row prefix, the two bin-scan passes and the
    scatter."""
    return 1 if prm["flags"] & 2 else 5


def max_over_ranks(x, ws, device="cpu"):
    """Largest value of x over the ranks of the default process group (x itself
    for one rank).  NCCL needs a CUDA device; gloo runs on the CPU."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ws, units_per_rank_step, steps, max_total_ms):
    """Whole-job throughput: every rank processes its own replica of the
    workload; the job's time is the slowest rank's."""
    return ws * units_per_rank_step * steps / (max_total_ms * 1e-3)


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = make_workload(args.workload)
    line = measure(args, args.workload, wl, ws, rank, dev, serving=True)
    if args.workload == DEFAULT_WORKLOAD and not args.no_fp64:
        # the same workload with an FP64 plan at tol 1e-12 (the paper's precision)
        from paper_2605_01313_gb300 import synth
        wl64 = synth.Workload("c3_2048x1024_f64", wl.n_lon, wl.n_lat, wl.coeffs, wl.lon,
                              wl.colat, 1e-12, "f64", sample=wl.sample)
        rec = measure(args, "c3_2048x1024_f64", wl64, ws, rank, dev, serving=False,
                      cpu_seconds=args.cpu_seconds / 2)
        if line is not None:
            line["fp64"] = {k: rec[k] for k in FP64_KEYS if k in rec}
    if args.workload == DEFAULT_WORKLOAD and not args.no_ensemble:
        # the batched form: 64 members of four grid sizes in one graph launch a step
        rec = measure_ensemble(args, "c4_ensemble_f32", ws, rank, dev,
                               cpu_seconds=args.cpu_seconds / 4)
        if line is not None:
            line["ensemble"] = {k: rec[k] for k in ENSEMBLE_KEYS if k in rec}
    if line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# keys of the nested ensemble record of the default run
ENSEMBLE_KEYS = ("metric", "value", "unit", "ms_per_step", "p50_ms", "p99_ms", "steps", "warmup",
                 "dtype", "config", "roofline", "gpu_launches", "persistent", "e2e", "error",
                 "clocks")

# keys of the nested FP64 record of the default run
FP64_KEYS = ("metric", "value", "unit", "ms_per_step", "p50_ms", "p99_ms", "steps", "warmup",
             "dtype", "config", "roofline", "roofline_step", "stages", "gpu_launches", "e2e",
             "error", "clocks")


def measure(args, name, wl, ws, rank, dev, serving, cpu_seconds=None):
    """Time one workload (warm-up, K timed steps, stage times, end to end through
    the host-buffer entry points, roofline, oracle error); returns the JSON
    line's dict on rank 0, None on the other ranks."""
    import torch
    from paper_2605_01313_gb300 import Plan, nufft

    pr_in = getattr(wl, "pr", None) is not None
    grid_in = getattr(wl, "grid", None) is not None
    sl = getattr(wl, "sl", None)
    F, P = (wl.pr.shape[0] if pr_in else wl.n_fields), wl.n_points
    cd = torch.complex128 if wl.dtype == "f64" else torch.complex64
    rd = torch.float64 if wl.dtype == "f64" else torch.float32
    lon = torch.from_numpy(wl.lon).to(dev)
    colat = torch.from_numpy(wl.colat).to(dev)
    if grid_in:
        coeffs = torch.from_numpy(wl.grid).to(rd).to(dev)
    else:
        coeffs = torch.from_numpy(wl.pr if pr_in else wl.coeffs).to(cd).to(dev)
    out = torch.empty((F, P), dtype=rd, device=dev)
    if sl is not None:
        w_t = torch.from_numpy(sl["w"]).to(rd).to(dev).contiguous()
        wa_t = torch.from_numpy(sl["wa"]).to(rd).to(dev).contiguous()
        pq_t = torch.empty((2, P), dtype=rd, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    gauss = getattr(wl, "gauss", None)
    opts = nufft.Options.make(real_fields=not args.general, keep_order=args.keep_order,
                              gauss=gauss is not None)
    t_plan = time.perf_counter()
    plan = Plan(wl.n_lon, wl.n_lat, wl.tol, wl.dtype, F, stream=stream, options=opts)
    t_plan = time.perf_counter() - t_plan
    prm = plan.params
    if gauss is not None:         # samples at the plan's Gauss-Legendre latitudes
        wl.grid = gauss(plan.latitudes())
        coeffs = torch.from_numpy(wl.grid).to(rd).to(dev)

    def step(evs=None):
        if sl is not None:        # departure points of Eq. 2.4 into the point buffers
            if evs:
                evs[0].record(stream)
            nufft.departure_points(w_t, sl["dt_over_a"], sl["iterations"], wa_t, stream,
                                   lon_out=lon, colat_out=colat, pq_out=pq_t)
            if evs:
                evs[1].record(stream)
        plan.set_points(lon, colat)
        if pr_in:
            plan.execute_pr(coeffs, out)
        elif grid_in:
            plan.interpolate_grid(coeffs, wl.parity, out)
        else:
            plan.execute(coeffs, out)
        if sl is not None:        # the wind to the arrival frame, in place
            if evs:
                evs[2].record(stream)
            nufft.rotate_to_arrival(wl.n_lon, wl.n_lat, None, None, out[1], out[2],
                                    u_a=out[1], v_a=out[2], stream=stream, pq=pq_t)
            if evs:
                evs[3].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)
    stats = nufft.dfsnufft_plan_point_stats(plan._h)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler(("GPU-" + str(uuid)) if uuid else None)
    nufft.dfsnufft_plan_enable_timing(plan._h, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sl_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)]
             for _ in range(args.steps)] if sl is not None else None
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    for i in range(args.steps):
        flush.fill_(i & 255)                  # untimed: evicts L2 between timed steps
        ev[i][0].record(stream)
        step(sl_ev[i] if sl_ev else None)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    stage = nufft.dfsnufft_plan_read_timing(plan._h)
    nufft.dfsnufft_plan_enable_timing(plan._h, False)
    total_ms = max_over_ranks(total_ms, ws, dev)
    value = weak_scaling_value(ws, F * P, args.steps, total_ms)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_lon, h_colat = pin(wl.lon), pin(wl.colat)
    if sl is not None:
        h_w = pin(sl["w"].astype(np.float64 if wl.dtype == "f64" else np.float32))
        h_wa = pin(sl["wa"].astype(np.float64 if wl.dtype == "f64" else np.float32))
    if grid_in:
        h_coef = pin(wl.grid.astype(np.float64 if wl.dtype == "f64" else np.float32))
    else:
        h_coef = pin((wl.pr if pr_in else wl.coeffs).astype(
            np.complex128 if wl.dtype == "f64" else np.complex64))
    h_out = torch.empty((F, P), dtype=rd).pin_memory().numpy()
    e2e_steps = max(3, args.steps)

    def e2e_step():
        if not (pr_in or grid_in):
            # new points and coefficients from host arrays, values back: the
            # library's joint call (copies and passes scheduled together)
            plan.execute_points_host(h_lon, h_colat, h_coef, h_out)
            return
        # the host-buffer entry points take complex coefficients: partial-
        # regularity and grid input go through pinned copies around the call
        if sl is None:
            lon.copy_(torch.from_numpy(h_lon), non_blocking=True)
            colat.copy_(torch.from_numpy(h_colat), non_blocking=True)
        else:                 # the points come from the step itself
            w_t.copy_(torch.from_numpy(h_w), non_blocking=True)
            wa_t.copy_(torch.from_numpy(h_wa), non_blocking=True)
        coeffs.copy_(torch.from_numpy(h_coef), non_blocking=True)
        step()
        torch.from_numpy(h_out).copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)

    for _ in range(2):
        e2e_step()
    e2e_ms = []
    for _ in range(e2e_steps):
        flush.fill_(3)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = max_over_ranks(sum(e2e_ms), ws, dev)
    e2e_value = weak_scaling_value(ws, F * P, e2e_steps, e2e_total)
    if not (pr_in or grid_in):
        # the bytes the host-buffer entry points copy (a real-field plan stages
        # only the coefficient columns its theta pass reads)
        cb = nufft.dfsnufft_plan_host_copy_bytes(plan._h)
        h2d, d2h = cb["points_h2d"] + cb["coeffs_h2d"], cb["values_d2h"]
    else:
        h2d = (2 * 8 * P if sl is None else h_w.nbytes + h_wa.nbytes) + h_coef.nbytes
        d2h = h_out.nbytes
    assert np.array_equal(h_out, out.cpu().numpy()), "host and device paths disagree"

    comparator = None
    if getattr(wl, "lag", None):
        # the Lagrange interpolation of the same arrival-grid samples at the same
        # points, timed the same way (L2 flushed before each run)
        comparator, lag_vals = {}, {}
        for order in wl.lag:
            lo = torch.empty((F, P), dtype=rd, device=dev)
            for _ in range(3):
                nufft.lagrange_interp(coeffs, wl.parity, lon, colat, order, out=lo, stream=stream)
            times = []
            for i in range(args.steps):
                flush.fill_(i & 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                nufft.lagrange_interp(coeffs, wl.parity, lon, colat, order, out=lo, stream=stream)
                e1.record(stream)
                times.append((e0, e1))
            torch.cuda.synchronize(dev)
            ms = float(np.mean([a.elapsed_time(b) for a, b in times]))
            comparator["lagrange%d" % order] = {"ms": ms, "value": F * P / (ms * 1e-3),
                                                "unit": UNIT}
            lag_vals["lagrange%d" % order] = lo.cpu().numpy()
        comparator["spectral"] = {"ms": total_ms / args.steps,
                                  "value": F * P / (total_ms / args.steps * 1e-3), "unit": UNIT}

    if rank != 0:
        plan.destroy()
        return None

    # ---- roofline of the dominant kernel
    pk, pk_kind = peaks()
    per_stage_ms = {k: (v[0] / v[1] if v[1] else None) for k, v in stage.items()}
    sbytes = stage_bytes(prm, F, P, stats["rows_needed"])
    if pr_in:       # the theta pass reads the partial-regularity arrays instead
        cs = 16 if prm["dtype"] == 0 else 8
        N1, N2 = prm["N1"], prm["N2"]
        sbytes["theta_pass"] += F * (wl.pr.shape[1] * wl.pr.shape[2] - N2 * (N1 // 2 + 2)) * cs
    dom = max(("theta_pass", "phi_pass", "interp", "set_points"),
              key=lambda k: per_stage_ms[k] or 0.0)
    dom_ms = per_stage_ms[dom]
    if wl.dtype == "f64" and dom == "interp" and not (prm["flags"] & 2):
        # FP64 plans interpolate in double-single arithmetic on the FP32 units:
        # the stage's FP32 instructions (df32_interp_ops) against the FP32 pipe's
        # instruction rate, measured live by the FMA probe (FLOP/s / 2)
        fma32 = nufft.dfsnufft_probe_fma_rate("f32", 20.0)
        ops = df32_interp_ops(prm, F, P)
        achieved = ops / (dom_ms * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": fma32 / 2e12,
                "unit": "T FP32-instructions/s", "frac": achieved / (fma32 / 2e12),
                "ops_per_launch": ops,
                "peak_source": "measured FP32 FMA rate / 2 (dfsnufft_probe_fma_rate, "
                               "one FFMA instruction = 2 FLOP)",
                "traffic": profile_traffic(dom, name),
                "hbm": {"achieved": sbytes[dom] / (dom_ms * 1e-3) / 1e9,
                        "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": sbytes[dom] / (dom_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}}
    else:
        achieved = sbytes[dom] / (dom_ms * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                "peak_source": "%s hbm_gbs" % pk_kind,
                "traffic": profile_traffic(dom, name)}
    stages_out = {}
    for k in per_stage_ms:
        ms = per_stage_ms[k]
        stages_out[k] = {"ms": ms, "bytes": sbytes[k],
                         "gbs": (sbytes[k] / (ms * 1e-3) / 1e9) if ms else None}
    # whole step against HBM: this path's own algorithmic bytes, and the
    # reference traffic model's (effective bandwidth)
    step_s = total_ms / args.steps * 1e-3
    own = sum(sbytes.values())
    mod = model_bytes(prm, F, P)
    roof_step = {"bound": "hbm", "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "own_bytes": own, "own_achieved": own / step_s / 1e9,
                 "own_frac": own / step_s / 1e9 / pk["hbm_gbs"],
                 "model_bytes": mod, "model_achieved": mod / step_s / 1e9,
                 "model_frac": mod / step_s / 1e9 / pk["hbm_gbs"],
                 "model": "13 N1 N2 c + 16 P / F + s_out P per field (complex grid, sigma 2)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # FP64 plans compute in double-single (pairs of FP32, 48-bit significands)
        # on the FP32 units, FP64 kept for the folding and the factors' set-up
        "dtype": "df32" if wl.dtype == "f64" else wl.dtype, "data": "synthetic",
        "config": {"workload": name, "grid": "%dx%d" % (wl.n_lon, wl.n_lat),
                   "modes": "%dx%d" % (2 * wl.n_lat, wl.n_lon), "fields": F, "points": P,
                   "tol": wl.tol, "w": prm["w"], "fine": "%dx%d" % (prm["n2"], prm["n1"]),
                   "rows_needed": stats["rows_needed"], "l2": "flushed between steps (512 MiB write)",
                   "real_fields": bool(prm["flags"] & 1), "keep_order": bool(prm["flags"] & 2),
                   "tile": [prm["tile_x"], prm["tile_y"]],
                   "sigma": prm["sigma"],
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roof,
        "roofline_step": roof_step,
        "stages": stages_out,
        # set_points (set_points_launches); theta pass, phi pass, interpolation;
        # grid input: the two forward passes (Gauss-Legendre: longitude pass,
        # latitude solve, coefficient mapping; the FP32 solve is our tcgen05
        # kernel, the FP64 one cuBLAS DGEMM, not counted); FP64 plans in
        # double-single: the exponent reductions of the coefficients (and samples)
        "gpu_launches": (set_points_launches(prm) + 3
                         + ((3 if gauss is not None and wl.dtype == "f32" else 2)
                            if grid_in else 0)
                         + (2 if sl is not None else 0)
                         + ((1 + (1 if grid_in and gauss is None else 0))
                            if wl.dtype == "f64" and not prm["flags"] & 2 else 0))
                        * args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_total / e2e_steps},
        "clocks": clocks,
    }
    if pr_in:
        line["config"]["input"] = "partial-regularity DFS coefficients (Sec. 4), M = %d, N = %d" % (
            wl.pr.shape[1] - 1, wl.pr.shape[2] - 1)
    if sl is not None:
        rs = 4 if wl.dtype == "f32" else 8
        dep_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in sl_ev]))
        rot_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in sl_ev]))
        dep_b, rot_b = (6 * rs + 16) * P, 6 * rs * P     # + p, q written / read
        stages_out["departure_points"] = {"ms": dep_ms, "bytes": dep_b,
                                          "gbs": dep_b / (dep_ms * 1e-3) / 1e9,
                                          "iterations": sl["iterations"]}
        stages_out["rotate_to_arrival"] = {"ms": rot_ms, "bytes": rot_b,
                                           "gbs": rot_b / (rot_ms * 1e-3) / 1e9}
    if grid_in:
        line["config"]["input"] = ("samples of the tilted steady zonal flow (h, u, v) on the "
                                   "arrival grid; coefficients computed on the GPU each step")
        if sl is not None:
            line["config"]["input"] += ("; departure points of Eq. 2.4 (TC2 flow, dt 1800 s, "
                                        "%d iterations) and the wind rotated to the arrival "
                                        "frame each step" % sl["iterations"])
        # the forward transform has no stage timer of its own: the step minus the stages
        line["stages"]["grid_to_coeffs"] = {
            "ms": line["ms_per_step"] - sum(v["ms"] for v in stages_out.values()),
            "note": "step time minus the timed stages"}
    if ws == 1 and not args.no_cpu_baseline:
        if pr_in:
            # the oracle's own route: partial-regularity -> standard -> complex
            import oracle
            cs_ = []
            for f in range(F):
                fc, fs = oracle.pr_to_std(np.ascontiguousarray(wl.pr[f].real.T),
                                          np.ascontiguousarray(wl.pr[f].imag.T))
                cs_.append(oracle.complex_from_cossin(fc, fs, wl.n_lon, wl.n_lat))
            wl.coeffs = np.stack(cs_)
        line["cpu_baseline"], line["error"] = cpu_baseline(
            wl, out.cpu().numpy(), cpu_seconds or args.cpu_seconds,
            lag_vals if comparator else None)
    if gauss is not None:
        line["config"]["input"] = ("samples of the tilted steady zonal flow (h, u, v) on the "
                                   "Gauss-Legendre grid; coefficients by the latitude solve "
                                   "each step")
        line["config"]["plan_seconds"] = t_plan
    if comparator:
        line["comparator"] = comparator
        line["config"]["input"] = ("samples of the C3 spectra on the arrival grid; the step "
                                   "computes coefficients and evaluates them at the departure "
                                   "points; comparator: Lagrange interpolation of the same "
                                   "samples")
    plan.destroy()
    if serving and ws == 1 and args.serve_seconds > 0:
        line["serving"] = serving_sweep(dev, [100, 500, 1000, 2000, 5000], args.serve_seconds)
    return line


def oracle_values(wl, s):
    """The oracle's values of the workload's fields at its sampled points s.  For
    the whole semi-Lagrangian step: the oracle's departure points of those
    arrival points first, the wind rotated to the arrival frame after."""
    import oracle
    sl = getattr(wl, "sl", None)
    if sl is None:
        return oracle.evaluate(wl.coeffs, wl.lon[s], wl.colat[s]).real
    from oracle import departure as dep
    rnd = (lambda a: a.astype(np.float32).astype(np.float64)) if wl.dtype == "f32" else \
        (lambda a: a)
    lon_d, colat_d = dep.departure_points(rnd(sl["w"]), rnd(sl["wa"]), sl["dt_over_a"],
                                          sl["iterations"], index=s)
    vals = oracle.evaluate(wl.coeffs, lon_d, colat_d).real
    la, ca = dep.arrival_points(wl.n_lon, wl.n_lat)
    u, v = dep.rotate_to_arrival(vals[1], vals[2], la[s], ca[s], lon_d, colat_d)
    return np.stack([vals[0], u, v])


def _oracle_sample_size(wl, seconds):
    probe = wl.sample[:4]
    t0 = time.perf_counter()
    oracle_values(wl, probe)
    per_point = (time.perf_counter() - t0) / probe.size
    return int(max(8, min(wl.sample.size, seconds / max(per_point, 1e-9))))


def cpu_baseline(wl, gpu_vals, seconds, others=None):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload's checked points; also the GPU error on that sample (and that of
    the other value arrays in ``others``, by name)."""
    import oracle
    n = _oracle_sample_size(wl, seconds)
    s = wl.sample[:n]
    t0 = time.perf_counter()
    ref = oracle_values(wl, s)
    dt = time.perf_counter() - t0
    err = [oracle.rel_linf(gpu_vals[f][s], ref[f]) for f in range(wl.n_fields)]
    what = ("departure points (NumPy), FP64 direct sum, rotation"
            if getattr(wl, "sl", None) is not None else "FP64 direct sum")
    base = {"value": n * wl.n_fields / dt, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": "%d of the workload's seeded check points x %d fields, %s"
                      % (n, wl.n_fields, what)}
    bound = 1e-11 if wl.dtype == "f64" else 2e-5
    out = {"rel_linf_per_field": err, "bound": bound, "ok": max(err) <= bound,
           "points_checked": int(n)}
    for name, vals in (others or {}).items():
        out[name] = [oracle.rel_linf(vals[f][s], ref[f]) for f in range(wl.n_fields)]
    return base, out


# ------------------------------------------------------------------ ensemble and serving

def run_ensemble(args):
    """64 members on four grids, three FP32 fields each: one CUDA graph per step."""
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    line = measure_ensemble(args, args.workload, ws, rank, dev, args.cpu_seconds)
    if line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_ensemble(args, name, ws, rank, dev, cpu_seconds):
    """The ensemble step of workload ``name`` (the fork/join graph and the
    persistent launch), timed on every rank; the line on rank 0, else None."""
    import torch
    from paper_2605_01313_gb300 import nufft

    members = make_workload(name)
    groups, pts, cfs, outs, host_in, host_out = [], [], [], [], [], []
    by_size = {}
    for wl in members:
        by_size.setdefault((wl.n_lon, wl.n_lat), []).append(wl)
    total_pf = 0
    for (n_lon, n_lat), wls in sorted(by_size.items()):
        groups.append((len(wls), n_lon, n_lat))
        lon = np.concatenate([w.lon for w in wls])
        colat = np.concatenate([w.colat for w in wls])
        coef = np.stack([w.coeffs for w in wls]).astype(np.complex64)
        pts.append((torch.from_numpy(lon).to(dev), torch.from_numpy(colat).to(dev),
                    [w.n_points for w in wls]))
        cfs.append(torch.from_numpy(coef).to(dev))
        outs.append(torch.empty(3 * lon.size, dtype=torch.float32, device=dev))
        host_in.append(tuple(torch.from_numpy(a).pin_memory() for a in (lon, colat, coef)))
        host_out.append(torch.empty(3 * lon.size, dtype=torch.float32).pin_memory())
        total_pf += 3 * lon.size
    stream = torch.cuda.current_stream(dev)
    # bin size, oversampling and kernel width per grid size from the autotuner
    from paper_2605_01313_gb300 import autotune
    t_tune = time.perf_counter()
    opts, tuned = [], []
    for gi, (m, n_lon, n_lat) in enumerate(groups):
        best, cands = autotune.tune(n_lon, n_lat, pts[gi][0], pts[gi][1], pts[gi][2], cfs[gi],
                                    tol=1e-6, dtype="f32", n_fields=3,
                                    real_fields=not args.general, path=None)
        opts.append(best)
        ch = [c for c in cands if c["opts"] == best.as_dict()][0]
        tuned.append({"grid": "%dx%d" % (n_lon, n_lat), "tile": [ch["params"]["tile_x"],
                      ch["params"]["tile_y"]], "sigma": ch["params"]["sigma"],
                      "w": ch["params"]["w"], "keep_order": bool(ch["params"]["flags"] & 2),
                      "tuner_ms": ch["ms"], "tuner_err": ch["err"],
                      "candidates": len(cands)})
    t_tune = time.perf_counter() - t_tune
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)

    def time_ensemble(ens):
        for _ in range(args.warmup):
            flush.fill_(1)
            ens.run(pts, cfs, outs)
        ens.check()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sampler = ClockSampler(("GPU-" + str(uuid)) if uuid else None)
        torch.cuda.synchronize(dev)
        sampler.start()
        for i in range(args.steps):
            flush.fill_(i & 255)
            ev[i][0].record(stream)
            ens.run(pts, cfs, outs)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        ens.check()
        return [a.elapsed_time(b) for a, b in ev], clocks

    # the same step as one persistent launch (transform and interpolation of all
    # groups from one device work queue): with the tuned options where that
    # form takes them, else with each grid's default options
    import oracle
    persistent = None
    pers_opts, pers_note = opts, "autotuned options"
    try:
        pens = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3, stream=stream,
                              options=pers_opts, persistent=True)
    except nufft.DfsError:
        pers_opts = [nufft.Options.make(real_fields=not args.general) for _ in groups]
        pers_note = "default options (the tuned ones include a kind the persistent form does not take)"
        pens = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3, stream=stream,
                              options=pers_opts, persistent=True)
    p_ms, _ = time_ensemble(pens)
    p_err = {}
    for gi, (m, n_lon, n_lat) in enumerate(groups):
        wl = by_size[(n_lon, n_lat)][0]
        vals = outs[gi][:3 * wl.n_points].view(3, wl.n_points).cpu().numpy()
        s_ = wl.sample[:32]
        ref = oracle.evaluate(wl.coeffs, wl.lon[s_], wl.colat[s_])
        p_err["%dx%d" % (n_lon, n_lat)] = max(oracle.rel_linf(vals[f][s_], ref[f].real)
                                              for f in range(3))
    p_total = max_over_ranks(sum(p_ms), ws, dev)
    persistent = {"ms_per_step": p_total / args.steps,
                  "value": weak_scaling_value(ws, total_pf, args.steps, p_total), "unit": UNIT,
                  "options": pers_note,
                  "gpu_launches_per_step": sum(
                      set_points_launches(nufft.dfsnufft_plan_get_params(pens.plan_handle(gi)))
                      for gi in range(len(groups))) + 1,
                  "error": {"rel_linf_first_member_32_points": p_err, "bound": 2e-5,
                            "ok": max(p_err.values()) <= 2e-5}}
    pens.destroy()

    ens = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3, stream=stream, options=opts)
    step_ms, clocks = time_ensemble(ens)
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    value = weak_scaling_value(ws, total_pf, args.steps, total_ms)
    # end to end: pinned host inputs in, values out, inside the timed region
    e2e_ms = []
    for i in range(max(3, min(args.steps, 8))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for g in range(len(groups)):
            pts[g][0].copy_(host_in[g][0], non_blocking=True)
            pts[g][1].copy_(host_in[g][1], non_blocking=True)
            cfs[g].copy_(host_in[g][2], non_blocking=True)
        ens.run(pts, cfs, outs)
        for g in range(len(groups)):
            host_out[g].copy_(outs[g], non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(sum(t.numel() * t.element_size() for t in hi) for hi in host_in)
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    # algorithmic bytes of every stage of every group, one step
    step_bytes = 0
    sp_launches = []
    for gi, (m, n_lon, n_lat) in enumerate(groups):
        prm = nufft.dfsnufft_plan_get_params(ens.plan_handle(gi))
        sp_launches.append(set_points_launches(prm))
        st = nufft.dfsnufft_plan_point_stats(ens.plan_handle(gi))
        step_bytes += sum(stage_bytes(prm, 3 * m, sum(pts[gi][2]), st["rows_needed"]).values())
    pk, pk_kind = peaks()
    achieved = step_bytes / (total_ms / args.steps * 1e-3) / 1e9
    if rank != 0:
        ens.destroy()
        return None
    # accuracy: the first member of every group against the oracle on its
    # seeded check points (and the oracle's own rate on them)
    errs, o_pf, o_s = {}, 0, 0.0
    for gi, (m, n_lon, n_lat) in enumerate(groups):
        wl = by_size[(n_lon, n_lat)][0]
        vals = outs[gi][:3 * wl.n_points].view(3, wl.n_points).cpu().numpy()
        n = min(wl.sample.size, _oracle_sample_size(wl, cpu_seconds / len(groups)))
        s_ = wl.sample[:n]
        t0 = time.perf_counter()
        ref = oracle.evaluate(wl.coeffs, wl.lon[s_], wl.colat[s_])
        o_s += time.perf_counter() - t0
        o_pf += 3 * n
        errs["%dx%d" % (n_lon, n_lat)] = max(oracle.rel_linf(vals[f][s_], ref[f].real)
                                             for f in range(3))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": name,
                   "groups": ["%dx(%dx%d)" % g for g in groups], "fields": 3,
                   "members": sum(g[0] for g in groups), "point_fields": total_pf, "tol": 1e-6,
                   "graph": "one CUDA graph launch per step (fork/join over group streams)",
                   "real_fields": not args.general, "autotuned": tuned,
                   "tune_seconds": t_tune,
                   "l2": "flushed between steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": {"kernel": "whole step (all stages, all groups)", "bound": "hbm",
                     "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "peak_source": "%s hbm_gbs" % pk_kind,
                     "traffic": None},
        # per group: set_points (set_points_launches), theta, phi, interpolation
        "gpu_launches": sum(sp_launches[gi] + 3 for gi in range(len(groups))) * args.steps,
        "persistent": persistent,
        "e2e": {"value": total_pf / (np.mean(e2e_ms) * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(np.mean(e2e_ms))},
        "clocks": clocks,
        "error": {"rel_linf_first_member": errs, "bound": 2e-5,
                  "ok": max(errs.values()) <= 2e-5},
        "cpu_baseline": {"value": o_pf / o_s, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": "seeded check points of the first member of each grid, "
                                   "3 fields, FP64 direct sum (%d point-fields)" % o_pf},
    }
    ens.destroy()
    return line


def serving_sweep(dev, rates, seconds, budget_gb=120):
    """Poisson request streams (grid uniform over five sizes, three FP32 fields,
    inputs resident on the device) through the continuous-batching server, and
    the same requests per call through FP64 plans."""
    import torch
    from paper_2605_01313_gb300 import Plan, synth
    from paper_2605_01313_gb300.serve import Server, poisson_run
    reqs, reqs64 = [], []
    for gi, (n_lon, n_lat) in enumerate(synth.SERVE_GRIDS):
        for j in range(2):
            wl = synth.workload_member(5 + 10 * gi + j, n_lon, n_lat, "f32", n_sample=8)
            base = {"n_lon": n_lon, "n_lat": n_lat, "pf": 3 * wl.n_points,
                    "lon": torch.from_numpy(wl.lon).to(dev),
                    "colat": torch.from_numpy(wl.colat).to(dev)}
            r = dict(base, coeffs=torch.from_numpy(wl.coeffs).to(torch.complex64).to(dev),
                     values=torch.empty((3, wl.n_points), dtype=torch.float32, device=dev))
            reqs.append(r)
            reqs64.append(dict(base, coeffs=torch.from_numpy(wl.coeffs).to(dev),
                               values=torch.empty((3, wl.n_points), dtype=torch.float64,
                                                  device=dev)))
    order = np.random.default_rng(55).permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    reqs64 = [reqs64[i] for i in order]
    from paper_2605_01313_gb300.nufft import Options
    srv = Server(tol=1e-6, dtype="f32", n_fields=3, hbm_budget=int(budget_gb) << 30, max_batch=8,
                 options=Options.make(real_fields=True))
    out = []
    for k, rate in enumerate(rates):
        # warm-up at this rate: the server creates a slot (a batched plan and its
        # buffers) the first time the concurrency calls for one, a one-time
        # cost kept out of the steady-state latencies; the slot counts before
        # and after the measured run show whether one was still created in it
        poisson_run(srv, reqs, rate, max(0.5, seconds / 2), seed=100 + k)
        slots0 = srv.stats()["slots"]
        lat, pf, wall, n = poisson_run(srv, reqs, rate, seconds, seed=10 + k)
        out.append({"rate": rate, "requests": n, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                    "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "max_ms": float(np.max(lat) * 1e3),
                    "value": pf / wall, "slots": [slots0, srv.stats()["slots"]]})
    stats = srv.stats()
    srv.close()
    # FP64, one request at a time (plans cached per grid)
    plans = {}
    stream = torch.cuda.current_stream(dev)
    for r in reqs64:
        key = (r["n_lon"], r["n_lat"])
        if key not in plans:
            plans[key] = Plan(r["n_lon"], r["n_lat"], 1e-12, "f64", 3, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pf64, n64 = 0, 0
    while time.perf_counter() - t0 < seconds:
        r = reqs64[n64 % len(reqs64)]
        p = plans[(r["n_lon"], r["n_lat"])]
        p.set_points(r["lon"], r["colat"])
        p.execute(r["coeffs"], r["values"])
        torch.cuda.synchronize(dev)
        pf64 += r["pf"]
        n64 += 1
    fp64 = {"value": pf64 / (time.perf_counter() - t0), "requests": n64, "tol": 1e-12}
    for p in plans.values():
        p.destroy()
    return {"unit": UNIT, "dtype": "f32", "tol": 1e-6, "budget_gb": budget_gb, "max_batch": 8,
            "grids": ["%dx%d" % g for g in synth.SERVE_GRIDS], "sweep": out,
            "batches": stats["batches"], "requests_batched": stats["members"],
            "slots": stats["slots"], "fp64_per_call": fp64}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    wls = make_workload(args.workload)
    if not isinstance(wls, list):
        wls = [wls]
    for w in wls:
        if getattr(w, "pr", None) is not None and w.coeffs is None:
            # partial-regularity input: the oracle's map to complex coefficients
            w.coeffs = np.stack([oracle.complex_from_cossin(
                *oracle.pr_to_std(np.ascontiguousarray(p_.real.T), np.ascontiguousarray(p_.imag.T)),
                w.n_lon, w.n_lat) for p_ in w.pr])
    wl = wls[-1]
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    # points per step, spread over the members (largest grid sets the cost)
    n = max(len(wls), _oracle_sample_size(wl, per_step))
    times = []
    pf = 0
    for i in range(args.warmup + args.steps):
        t_step = 0.0
        pf_step = 0
        for j, w in enumerate(wls):
            k = n // len(wls) + (1 if j < n % len(wls) else 0)
            if k == 0:
                continue
            s = w.sample[(i * k) % w.sample.size:][:k]
            if s.size < k:
                s = w.sample[:k]
            t0 = time.perf_counter()
            oracle_values(w, s)
            t_step += time.perf_counter() - t0
            pf_step += s.size * w.n_fields
        if i >= args.warmup:
            times.append(t_step)
            pf += pf_step
    total = sum(times)
    value = pf / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": "%dx%d" % (wl.n_lon, wl.n_lat),
                   "members": len(wls), "fields": wl.n_fields, "points": wl.n_points},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": "%d points x %d fields per step, FP64 direct sum"
                                   % (n, wl.n_fields)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="leave the 64-member ensemble record out of the default run")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the nested FP64 record of the default workload")
    ap.add_argument("--keep-order", action="store_true",
                    help="evaluate the points unsorted, in their grid order")
    ap.add_argument("--general", action="store_true",
                    help="general plans (no real-field symmetry) instead of real-field plans")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="seconds per rate of the serving sweep in the default run (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, _, _ = dist_env()
    if args.gpus > 1 and ws == 1 and "LOCAL_RANK" not in os.environ:
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               "--nproc-per-node", str(args.gpus), "--master-addr", "127.0.0.1",
               "--master-port", "29533"] + sys.argv
        sys.exit(subprocess.call(cmd))
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2605_01313_gb300 import build
        build.build()
        if WORKLOADS[args.workload][1] == "c4":
            run_ensemble(args)
        else:
            run_ours(args)


if __name__ == "__main__":
    main()
