#!/usr/bin/env python3
"""Benchmark of the finite-frequency traveltime tomography hot path on GB300.

Workload (default ``slices3d``, the largest single-GPU configuration): the 256-element ring
of radius 100 mm stepped to 16 z positions 4 mm apart (pairs only within a slice, 522240
pairs), three frequency bands (0.6 / 1.0 / 1.4 MHz, sigma 0.2 MHz, one 4096-sample Phi table
each, cut-off 3 periods), 1566720 rows, 256 x 256 x 96 voxels at 0.75 mm, 12 random
ellipsoidal inclusions, data = J dc + N(0, 5 ns), 20 CGLS iterations with relative damping
1e-3 replayed from a CUDA graph. ``--workload ring256`` runs the single-ring configuration
(32640 pairs, 200 x 200 x 40 voxels at 1 mm, 30 iterations). Synthetic, seeded inputs (the
paper's lab dataset is not available).

One step = one damped least-squares solve (fft_cg_solve) on resident data: (n_iter + 1)
applications each of J and J^T, every entry rebuilt on the fly. The Phi tables and the culled
geometry are built once before timing (their build time is reported as ``setup_ms``). The
metric is in-support pair-voxel evaluations per second (J and J^T together); the roofline is
that of the J^T kernel against the FP32 issue rate of the chip.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun each rank runs its own replica (the path has no exchange step on one
acquisition per GPU); rank 0 prints one JSON line.
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
from typing import Optional

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "J & J^T pair-voxel evals/s (in-support), ms per CG iter, % FP32 roofline, err vs FP64 oracle"
UNIT = "eval/s"
# FP32 lane operations of one in-support evaluation in the canonical (textbook detour) count:
# 6 FADD (difference vectors), 6 (squared norms), 2 (R = R^2 rsqrt), 3 (scaled detour),
# 2 (index, fraction), 2 (lerp), 1 (rsqrt product), 1 (times Phi), 1 (accumulate).
OPS_PER_EVAL = 24
FP32_LANES_PER_SM_CLK = 128
# DRAM bytes (read + write) of one J^T (the apply kernel and its slot reduction, as timed) per
# workload, from ncu captures of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum); a workload without a capture of the current build reports null.
APPLY_TRAFFIC_BYTES = {
    # plain-band apply 3910192640 + 149975552, sharp-band apply 5340387840 + 374120960,
    # jt_reduce 342418176 + 6821632
    "slices3d": 10123916800,
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    """(world size, rank, local rank) from the launcher's environment; with more than one rank
    a process group: NCCL over the GPUs, or gloo where no CUDA device is visible (the host
    side of the replica logic, tested on CPU)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """The largest of the ranks' values (step times: the job is as slow as its slowest rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- CPU oracle legs

def oracle_leg(w, n_rows: int, n_vox: int, d_gpu, r_host, g_gpu, seed: int = 0, phi: str = "table",
               trig_terms: int = 0):
    """The FP64 oracle on a bounded sample of the workload: J on n_rows random rows (timed:
    in-support evals/s on the host cores) and J^T on n_vox random voxels. Returns the
    cpu_baseline record and the relative L2 errors of the GPU's J and J^T on the sample."""
    import oracle
    og = oracle.Geometry.from_workload(w, phi=phi, n_terms=trig_terms)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(og.M, n_rows, replace=False)).astype(np.int64)
    vox = np.sort(rng.choice(og.V, n_vox, replace=False)).astype(np.int64)
    units = og.count_support(rows)
    m = wl.model_for(w)
    t0 = time.perf_counter()
    d_ref = og.J(m, rows)
    secs = time.perf_counter() - t0
    g_ref = og.JT(r_host, vox)
    cpu = {"value": units / secs, "unit": UNIT, "cores": oracle.n_threads(), "kind": "oracle",
           "sample": f"FP64 oracle J on {n_rows} random rows of {w.name} ({units} in-support evals, {secs:.1f} s)"}
    err = {"J_rel_l2": float(np.linalg.norm(d_gpu[rows] - d_ref) / np.linalg.norm(d_ref)),
           "JT_rel_l2": float(np.linalg.norm(g_gpu[vox] - g_ref) / np.linalg.norm(g_ref)),
           "sample": f"J on the {n_rows} oracle rows, J^T on {n_vox} random voxels"}
    return cpu, err


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    w = wl.by_name(args.workload)
    og = oracle.Geometry.from_workload(w)
    m = wl.model_for(w)
    rng = np.random.default_rng(123)
    n_rows = args.ref_rows
    samples = [np.sort(rng.choice(og.M, n_rows, replace=False)).astype(np.int64)
               for _ in range(args.warmup + args.steps)]
    units = [og.count_support(r) for r in samples]
    times = []
    for i, rows in enumerate(samples):
        t0 = time.perf_counter()
        og.J(m, rows)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append((dt, units[i]))
    tot_t = sum(t for t, _ in times)
    tot_u = sum(u for _, u in times)
    value = tot_u / tot_t
    sample = f"FP64 oracle J on {n_rows} random rows of {w.name} per step ({tot_u // max(len(times), 1)} in-support evals)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded ring-array workload)",
        "config": {"workload": w.name, "pairs": og.M, "voxels": og.V, "l2": "inputs resident, CPU"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.n_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- PSF batch

def run_psf(args, ws, rank, local):
    """Batched Hessian PSFs on the slice-by-slice geometry: 128 seeded spikes x 3 nested ring
    subsets (every 4th / 2nd / every element) = 384 PSFs, BF16 tensor-core path against the
    FP32 CUDA-core path (per PSF: column J e_k then J^T restricted to the rows it touches)."""
    import torch
    import paper_1908_03302_gb300 as fg
    torch.cuda.set_device(local)
    w = wl.by_name(args.psf_geometry)
    tables = [fg.Table(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max) for b in w.bands]
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, tables,
                      band_of_row=w.band_of_row if len(w.bands) > 1 else None)
    spikes = wl.random_voxels(w.grid, args.psf_spikes, 8)
    subsets = wl.ring_subsets(n_slices=16 if w.name == "slices3d" else 1, n_bands=len(w.bands))
    n_psf = len(spikes) * len(subsets)
    out_tc = torch.empty(n_psf * geo.V, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    for _ in range(args.warmup):
        geo.psf_batch(spikes, subsets, mode=1, out=out_tc)
    tc_ms = [timed(lambda: geo.psf_batch(spikes, subsets, mode=1, out=out_tc)) for _ in range(args.steps)]
    # tensor-core work of one batch: MMA flops (2 x generated J entries x MMA width) against the
    # measured sustained BF16 rate, and the rate at which J entries are generated
    pk, pk_kind = peaks()
    mma_flops = float(geo.info().psf_tc_mma_flops)
    tc_s = statistics.mean(tc_ms) * 1e-3
    peak_tc = float(pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1700.0)
    tensor = {"mma_tflops": mma_flops / tc_s / 1e12, "peak_tflops": peak_tc,
              "peak_basis": f"bf16 sustained ({pk_kind})", "frac": mma_flops / tc_s / 1e12 / peak_tc,
              "mma_flops_per_batch": mma_flops}
    # what bounds the batch is generating the J tiles in FP32: generated entries per second of
    # the whole call against the canonical FP32 issue rate of one evaluation (the J / J^T peak)
    entries = float(geo.info().psf_tc_entries)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = float(pk.get("sm_max_mhz") or 2070.0)
    peak_evals = sm_count * FP32_LANES_PER_SM_CLK * sm_max * 1e6 / OPS_PER_EVAL
    generation = {"bound": "alu", "achieved": entries / tc_s / 1e9, "peak": peak_evals / 1e9, "unit": "Geval/s",
                  "frac": entries / tc_s / peak_evals, "traffic": None,
                  "kernel": "psf_tc_kernel (J tiles generated in FP32, BF16 MMA), whole fft_psf_batch call",
                  "entries_per_batch": entries,
                  "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM_CLK} FP32 lanes x {sm_max:.0f} MHz "
                                f"({pk_kind}) / {OPS_PER_EVAL} ops per eval"}
    if args.psf_tc_only:
        if rank == 0:
            print(json.dumps({"psf_tc_ms": tc_ms, "geometry": w.name, "spikes": len(spikes), "tensor": tensor,
                              "roofline": generation}), flush=True)
        return 0
    # FP32 path on a slice of the spikes (same per-PSF cost), scaled to the whole batch
    k32 = min(len(spikes), args.psf_fp32_spikes)
    out_fp = torch.empty(k32 * len(subsets) * geo.V, device="cuda", dtype=torch.float32)
    fp_ms = timed(lambda: geo.psf_batch(spikes[:k32], subsets, mode=0, out=out_fp))
    # the FP32 path with four columns per J^T (columns in spike-major order)
    out_fp4 = torch.empty_like(out_fp)
    fp4_ms = timed(lambda: geo.psf_batch(spikes[:k32], subsets, mode=2, out=out_fp4))
    tc = out_tc.view(len(subsets), len(spikes), geo.V)
    fp = out_fp.view(len(subsets), k32, geo.V)
    fp4 = out_fp4.view(len(subsets), k32, geo.V)
    diff = []
    for sb in range(len(subsets)):
        for k in range(k32):
            nrm = float(fp[sb, k].double().norm())
            if nrm > 0:
                diff.append(float((tc[sb, k].double() - fp[sb, k].double()).norm()) / nrm)
    # CPU baseline leg: the FP64 oracle on sampled voxels of a few PSFs (timed, and the same
    # values give the sampled error of both GPU paths)
    errs_tc, errs_fp, errs_fp4, cpu = [], [], [], None
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        og = oracle.Geometry.from_workload(w)
        rng = np.random.default_rng(12)
        secs, n_vals = 0.0, 0
        for k in range(min(2, k32)):
            vk = int(spikes[k])
            i, j, z = vk % w.grid.nx, (vk // w.grid.nx) % w.grid.ny, vk // (w.grid.nx * w.grid.ny)
            near = []
            for _ in range(256):
                di, dj, dz = rng.integers(-20, 21, 3)
                ii, jj, zz = min(max(i + di, 0), w.grid.nx - 1), min(max(j + dj, 0), w.grid.ny - 1), \
                    min(max(z + dz, 0), w.grid.nz - 1)
                near.append((zz * w.grid.ny + jj) * w.grid.nx + ii)
            vox = np.unique(np.array(near, dtype=np.int64))
            for sb in (0, 2):
                t0 = time.perf_counter()
                ref = og.psf(np.array([vk]), [subsets[sb]], vox)[0, 0]
                secs += time.perf_counter() - t0
                n_vals += len(vox)
                n = np.linalg.norm(ref)
                vt = torch.as_tensor(vox, device="cuda")
                errs_tc.append(float(np.linalg.norm(tc[sb, k][vt].double().cpu().numpy() - ref) / n))
                errs_fp.append(float(np.linalg.norm(fp[sb, k][vt].double().cpu().numpy() - ref) / n))
                errs_fp4.append(float(np.linalg.norm(fp4[sb, k][vt].double().cpu().numpy() - ref) / n))
        cpu = {"value": 1e3 * secs / n_vals * n_psf * geo.V, "unit": "ms", "cores": oracle.n_threads(),
               "kind": "oracle",
               "sample": f"FP64 oracle PSF values at {n_vals} voxels (2 spikes x subsets {{64, 256}}, within 20 "
                         f"voxels of the spike) in {secs:.1f} s, scaled linearly to {n_psf} PSFs x {geo.V} voxels"}
    fp_full_ms = fp_ms * len(spikes) / k32
    fp4_full_ms = fp4_ms * len(spikes) / k32
    tc_avg = statistics.mean(tc_ms)
    info = geo.info()
    line = {
        "metric": "batched Hessian PSFs: ms per batch (BF16 tensor cores vs FP32), PSF rel-L2 vs FP64 oracle",
        "value": tc_avg, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tc_avg, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 x bf16 -> f32 (tensor cores); f32 generation",
        "data": "synthetic (seeded slice-by-slice ring geometry, seeded spikes)",
        "config": {"workload": "psf3d" if w.name == "slices3d" else "psf-" + w.name, "pairs": geo.M, "voxels": geo.V, "spikes": len(spikes),
                   "subsets": [int(len(sb)) for sb in subsets], "psfs": n_psf,
                   "support_evals_per_apply": int(info.support_evals)},
        "fp32_path_ms_per_batch": fp_full_ms, "fp32_path_measured": f"{k32} spikes x 3 subsets, scaled",
        "speedup_tc_vs_fp32": fp_full_ms / tc_avg,
        "fp32_batched_path_ms_per_batch": fp4_full_ms,
        "fp32_batched_path": "four columns per J^T (fft_psf_batch mode 2), same spikes, scaled",
        "speedup_tc_vs_fp32_batched": fp4_full_ms / tc_avg,
        "tensor": tensor,
        "roofline": generation,
        "tc_vs_fp32_rel_l2_max": max(diff) if diff else None,
        "err_vs_fp64_oracle": {"tc_rel_l2_max": max(errs_tc), "fp32_rel_l2_max": max(errs_fp),
                               "fp32_batched_rel_l2_max": max(errs_fp4),
                               "sample": "2 spikes x subsets {64, 256}, <=256 voxels within 20 of the spike"}
        if errs_tc else None,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- elevation spacing

def fwhm(profile: np.ndarray, h: float, centre: int) -> Optional[float]:
    """Full width at half maximum (m) of a PSF profile around its peak at index `centre`, by
    linear interpolation between samples; None if it does not fall to half on both sides."""
    p = np.asarray(profile, dtype=np.float64)
    half = 0.5 * p[centre]
    if not half > 0:
        return None
    edges = []
    for step in (-1, 1):
        i = centre
        while 0 <= i + step < len(p) and p[i + step] > half:
            i += step
        if not 0 <= i + step < len(p):
            return None
        a, b = p[i], p[i + step]
        edges.append(i + step * (a - half) / (a - b))
    return abs(edges[1] - edges[0]) * h


def run_spacing(args, ws, rank, local):
    """Resolution against elevation spacing (Sec. III-C): Hessian PSFs H e_k = J^T J e_k with all
    rows of a 256-element ring stacked at 3 mm (11 elevations) or 8 mm (7 elevations), for spikes
    at x = 0, 20, 40, 60 mm on the mid plane; reports per PSF the peak, the vertical and
    horizontal half-maximum widths through the spike and the deepest negative lobe (the
    trade-offs) relative to the peak, and the GPU time of each batch (FP32 path)."""
    import torch
    import paper_1908_03302_gb300 as fg
    torch.cuda.set_device(local)
    xs_mm = (0, 20, 40, 60)
    res = {}
    for spacing, npos in ((3e-3, 11), (8e-3, 7)):
        w = wl.elevation_stack(spacing, npos)
        g = w.grid
        tables = [fg.Table(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max) for b in w.bands]
        geo = fg.Geometry(w.tx, w.row_pairs(), g, w.c0, tables)
        ic, kc = (g.nx - 1) // 2, (g.nz - 1) // 2
        spikes = [(kc * g.ny + ic) * g.nx + ic + int(round(x * 1e-3 / g.h)) for x in xs_mm]
        rows = np.arange(geo.M, dtype=np.int32)
        out = torch.empty(len(spikes) * geo.V, device="cuda", dtype=torch.float32)
        geo.psf_batch(spikes, [rows], mode=0, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        geo.psf_batch(spikes, [rows], mode=0, out=out)
        b.record()
        torch.cuda.synchronize()
        psf = out.view(len(spikes), g.nz, g.ny, g.nx).double().cpu().numpy()
        entry = {"elevations": npos, "rows": geo.M, "ms": a.elapsed_time(b), "psfs": []}
        for x, v in zip(xs_mm, spikes):
            i = v % g.nx
            vert = psf[xs_mm.index(x), :, ic, i]
            horz = psf[xs_mm.index(x), kc, ic, :]
            fz, fx = fwhm(vert, g.h, kc), fwhm(horz, g.h, i)
            # trade-offs: the deepest negative lobe relative to the peak, along z and along x
            entry["psfs"].append({"x_mm": x, "peak": float(vert[kc]),
                                  "fwhm_z_mm": None if fz is None else 1e3 * fz,
                                  "fwhm_x_mm": None if fx is None else 1e3 * fx,
                                  "neg_lobe_z": float(max(0.0, -vert.min()) / vert[kc]),
                                  "neg_lobe_x": float(max(0.0, -horz.min()) / horz[i])})
        res[f"{spacing * 1e3:.0f}mm"] = entry
    if rank == 0:
        print(json.dumps({"metric": "PSF widths and trade-offs for 3 mm vs 8 mm elevation spacing",
                          "value": res["3mm"]["ms"] + res["8mm"]["ms"], "unit": "ms",
                          "higher_is_better": False, "n_gpus": ws, "dtype": "f32",
                          "data": "synthetic (seeded ring stacks, unit spikes)",
                          "config": {"workload": "elevation spacing", "grid": "141 x 141 x 33 @ 1 mm",
                                     "ring": "256 elements, 100 mm", "band": "1 MHz, sigma 0.4 MHz"},
                          "spacing": res}), flush=True)
    return 0


# --------------------------------------------------------------------------- low-rank resolution

def run_lowrank(args, ws, rank, local):
    """Low-rank posterior covariance and resolution (Sec. II-D) on ring256: the k dominant
    eigenpairs of H = J^T J / sigma^2 (sigma = 25 ns, the paper's cross-correlation accuracy)
    by randomized subspace iteration, then the diagonals of the low-rank posterior covariance
    and resolution matrix (alpha relative to the mean diagonal of H)."""
    import torch
    import paper_1908_03302_gb300 as fg
    torch.cuda.set_device(local)
    w = wl.by_name("ring256")
    tables = [fg.Table(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max) for b in w.bands]
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, tables)
    k, ell, q, sigma = args.lowrank_k, args.lowrank_k + 16, 1, 2.5e-8
    omega = torch.as_tensor(np.ascontiguousarray(wl.gaussian_block(geo.V, ell, 41).T), dtype=torch.float32,
                            device="cuda")
    geo.hessian_lowrank(omega[:8], 4, 0, sigma)          # warm-up (graphs, attributes, caches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, vecs = geo.hessian_lowrank(omega, k, q, sigma)
    t1 = time.perf_counter()
    alpha = 1e-3 * geo.frob2() / sigma ** 2 / geo.V
    post, res = geo.lowrank_diag(vecs, lam, alpha)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    n_apply = (q + 2) * ell
    if rank == 0:
        r = res.double()
        print(json.dumps({"metric": "low-rank posterior / resolution: seconds for k eigenpairs of H",
                          "value": t1 - t0, "unit": "s", "higher_is_better": False, "n_gpus": ws,
                          "dtype": "f32 (FP64 Gram, host FP64 Rayleigh-Ritz)",
                          "data": "synthetic (ring256 geometry, seeded Gaussian start block)",
                          "config": {"workload": "ring256 low-rank", "k": k, "ell": ell, "power_iterations": q,
                                     "sigma_s": sigma, "alpha_rel": 1e-3},
                          "H_applications": n_apply, "ms_per_H_application": 1e3 * (t1 - t0) / n_apply,
                          "diag_seconds": t2 - t1,
                          "eigenvalues": {"first": float(lam[0]), "k_th": float(lam[-1]),
                                          "decay_k_over_1": float(lam[-1] / lam[0])},
                          "resolution_diag": {"max": float(r.max()), "mean": float(r.mean())}}), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm

def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:   # NVTX is only a marker for profilers
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="slices3d",
                    choices=["ring32", "ring256", "ring256_3band", "slices3d", "psf3d", "spacing", "lowrank"])
    ap.add_argument("--lowrank-k", type=int, default=64)
    ap.add_argument("--psf-spikes", type=int, default=128)
    ap.add_argument("--psf-fp32-spikes", type=int, default=8)
    ap.add_argument("--psf-geometry", default="slices3d", choices=["slices3d", "ring256", "ring256_3band"])
    ap.add_argument("--psf-tc-only", action="store_true", help="time only the tensor-core path (profiling)")
    ap.add_argument("--dt-mode", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default work decomposition")
    ap.add_argument("--ref-rows", type=int, default=1024)
    ap.add_argument("--cpu-rows", type=int, default=4096)
    ap.add_argument("--phi", default="table", choices=["table", "trig"],
                    help="Phi representation: sampled table (default) or sine series")
    ap.add_argument("--trig-terms", type=int, default=0, help="sine-series terms (0: automatic)")
    ap.add_argument("--mode", default="solve", choices=["solve", "apply", "batch"],
                    help="apply: only build the geometry and run --steps J^T and J applications "
                         "(a short program for ncu captures; prints timings, not the bench line)")
    args = ap.parse_args()

    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "psf3d":
        return run_psf(args, ws, rank, local)
    if args.workload == "spacing":
        return run_spacing(args, ws, rank, local)
    if args.workload == "lowrank":
        return run_lowrank(args, ws, rank, local)

    import torch
    import paper_1908_03302_gb300 as fg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = wl.by_name(args.workload)

    # ---- setup (not part of a step): tables, geometry, data
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.phi == "trig":
        tables = [fg.TrigTable(b.f_center_hz, b.f_sigma_hz, b.dt_max, args.trig_terms) for b in w.bands]
    else:
        tables = [fg.Table(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max) for b in w.bands]
    t1 = time.perf_counter()
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, tables,
                      band_of_row=w.band_of_row if len(w.bands) > 1 else None, dt_mode=args.dt_mode)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # work decomposition picked by timing candidates on the device (set-up, not a step)
    tuning = geo.autotune() if not args.no_autotune else None
    t3 = time.perf_counter()
    info = geo.info()
    support = int(info.support_evals)
    m_true = torch.as_tensor(wl.model_for(w), dtype=torch.float32, device=dev)
    noise = torch.as_tensor(wl.noise(geo.M, w.noise_seed), dtype=torch.float32, device=dev)
    d = geo.J(m_true) + noise
    m = torch.zeros(geo.V, dtype=torch.float32, device=dev)
    geo.frob2()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()
    n_iter = w.cg_iters
    evals_per_step = 2 * (n_iter + 1) * support
    launches_per_step = 8 + 10 * n_iter

    def step(mbuf):
        mbuf.zero_()
        geo.cg_solve(d, w.lambda_rel, n_iter, m=mbuf, check_status=False)   # asynchronous

    if args.mode == "apply":
        r0 = torch.randn(geo.M, device=dev, dtype=torch.float32) * 1e-8
        g0 = torch.empty(geo.V, device=dev, dtype=torch.float32)
        for i in range(args.warmup + args.steps):
            nvtx_push("apply")   # lets a profiler skip the autotuner's launches of the same kernels
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            geo.JT(r0, out=g0)
            b.record(stream)
            c, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c.record(stream)
            geo.J(m_true, out=d)
            e.record(stream)
            torch.cuda.synchronize()
            nvtx_pop()
            if rank == 0:
                print(json.dumps({"apply": i, "ms_JT": a.elapsed_time(b), "ms_J": c.elapsed_time(e),
                                  "support": support, "evaluated": int(info.evaluated_evals),
                                  "entries": int(info.n_entries), "items": int(info.n_items)}), flush=True)
        return 0
    if args.mode == "batch":
        # four-column J^T and J (one group), the Hessian columns of the low-rank solver
        D4 = torch.randn((4, geo.M), device=dev, dtype=torch.float32) * 1e-8
        M4 = torch.randn((4, geo.V), device=dev, dtype=torch.float32)
        G4 = torch.empty((4, geo.V), device=dev, dtype=torch.float32)
        Q4 = torch.empty((4, geo.M), device=dev, dtype=torch.float32)
        for i in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            geo.JT_batch(D4, out=G4)
            b.record(stream)
            c.record(stream)
            geo.J_batch(M4, out=Q4)
            e.record(stream)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"batch": i, "columns": 4, "ms_JT4": a.elapsed_time(b), "ms_J4": c.elapsed_time(e),
                                  "support": support}), flush=True)
        return 0

    for _ in range(args.warmup):
        step(m)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step(m)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    geo.cg_status()   # raises if a solve broke down
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), ws)

    # ---- dominant kernel: J^T (and J) applications timed alone on the launching stream
    reps = 10
    r = torch.randn(geo.M, device=dev, dtype=torch.float32) * 1e-8
    gbuf = torch.empty(geo.V, device=dev, dtype=torch.float32)
    dbuf = torch.empty(geo.M, device=dev, dtype=torch.float32)
    jt_ms, j_ms = [], []
    for i in range(reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        geo.JT(r, out=gbuf)
        b.record(stream)
        c, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c.record(stream)
        geo.J(m_true, out=dbuf)
        e.record(stream)
        torch.cuda.synchronize()
        jt_ms.append(a.elapsed_time(b))
        j_ms.append(c.elapsed_time(e))
    # the 2-D approximation (Eq. forward_2D) on the same geometry: the plane map and the
    # kernel integrated over the grid's layers (single-ring workloads only)
    j2_ms, jt2_ms = [], []
    m2 = torch.randn(geo.V2, device=dev, dtype=torch.float32)
    g2 = torch.empty(geo.V2, device=dev, dtype=torch.float32)
    for i in range(3 if len(np.unique(w.tx[:, 2])) == 1 else 0):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        geo.J2d(m2, out=dbuf)
        b.record(stream)
        c.record(stream)
        geo.JT2d(r, out=g2)
        e.record(stream)
        torch.cuda.synchronize()
        j2_ms.append(a.elapsed_time(b))
        jt2_ms.append(c.elapsed_time(e))
    clocks = sampler.stop()

    # ---- end to end through the public API with host buffers
    d_host = d.cpu().pin_memory()
    m_host = torch.empty(geo.V, dtype=torch.float32).pin_memory()
    d_dev = torch.empty_like(d)
    m_dev = torch.empty_like(m)
    e2e_ms = []
    step_avg_ms = total_ms / args.steps
    n_e2e = max(2, min(args.steps, 5 if step_avg_ms < 5000 else 3))
    for i in range(n_e2e):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        d_dev.copy_(d_host, non_blocking=True)
        m_dev.zero_()
        geo.cg_solve(d_dev, w.lambda_rel, n_iter, m=m_dev, check_status=False)
        m_host.copy_(m_dev, non_blocking=True)
        geo.cg_status()
        e2e_ms.append(1e3 * (time.perf_counter() - t_a))
    e2e_total = max_over_ranks(sum(e2e_ms) / len(e2e_ms), ws)

    # ---- CPU baseline leg (rank 0): the FP64 oracle on sampled rows (J, timed) and voxels
    #      (J^T); the same outputs give the sampled error of the GPU results
    err = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dj = geo.J(m_true).double().cpu().numpy()
        gj = geo.JT(r).double().cpu().numpy()
        cpu, err = oracle_leg(w, args.cpu_rows, 1024, dj, r.double().cpu().numpy(), gj, phi=args.phi,
                              trig_terms=args.trig_terms)

    if rank != 0:
        return 0
    pk, pk_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    sm_max = float(pk.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    # canonical FP32 operations per evaluation: the 24-op table mix; with the sine series the
    # 4-op lookup becomes 16 ops (sin, cos, argument, cut) plus 2 per term of the recurrence
    n_terms = int(info.phi_terms)
    ops = OPS_PER_EVAL if n_terms == 0 else OPS_PER_EVAL - 4 + 16 + 2 * n_terms
    peak_evals = sm_count * FP32_LANES_PER_SM_CLK * sm_max * 1e6 / ops
    jt_avg = statistics.mean(jt_ms) * 1e-3
    j_avg = statistics.mean(j_ms) * 1e-3
    achieved = support / jt_avg
    value = ws * evals_per_step * args.steps / (total_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ring-array workload; FP32 kernels, FP64 CG scalars)",
        "config": {"workload": w.name, "pairs": geo.M, "voxels": geo.V, "cg_iters": n_iter,
                   "support_evals_per_apply": support, "evaluated_evals_per_apply": int(info.evaluated_evals),
                   "dt_mode": ["stable", "naive", "fp64"][args.dt_mode],
                   "phi": "table (4096 samples)" if n_terms == 0 else f"sine series ({n_terms} terms)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "ms_per_cg_iter": total_ms / args.steps / n_iter,
        "ms_per_J": 1e3 * j_avg, "ms_per_JT": 1e3 * jt_avg,
        "J_evals_per_s": support / j_avg, "JT_evals_per_s": support / jt_avg,
        "J_dense_equiv_per_s": geo.M * geo.V / j_avg, "JT_dense_equiv_per_s": geo.M * geo.V / jt_avg,
        "ms_per_J2d": statistics.mean(j2_ms) if j2_ms else None,
        "ms_per_JT2d": statistics.mean(jt2_ms) if jt2_ms else None,
        "setup_ms": {"table": 1e3 * (t1 - t0), "geometry_and_cull": 1e3 * (t2 - t1), "autotune": 1e3 * (t3 - t2)},
        "autotune": tuning,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_evals / 1e9, "unit": "Geval/s",
                     "frac": achieved / peak_evals,
                     "traffic": APPLY_TRAFFIC_BYTES.get(w.name) if (args.dt_mode == 0 and n_terms == 0) else None,
                     "kernel": "apply_kernel (J^T) + jt_reduce",
                     "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM_CLK} FP32 lanes x {sm_max:.0f} MHz "
                                   f"({pk_kind}) / {ops} ops per eval"},
        "err_vs_fp64_oracle": err,
        "cpu_baseline": cpu,
        "e2e": {"value": ws * evals_per_step / (e2e_total * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 4 * geo.M, "d2h_bytes_per_step": 4 * geo.V,
                "ms_per_step": e2e_total, "steps": n_e2e},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
