#!/usr/bin/env python3
"""Benchmark of the PSF-matching hot path: PSF-matched Mpix/s (solve + convolve + variance).

One step is one batch of full-chip subtractions through the C ABI (``psfm_batch_subtract``;
``--single`` uses one ``psfm_subtract`` per step): for every chip, stamp extraction, basis
convolution and Gram per stamp, normalisation, the solve with the iterative stamp rejection,
r_bad, then the spatially varying convolution of the whole chip, the per-patch variance
propagation, the mask propagation and the covariance pseudo-matrix.  The default batch is 4
distinct 4846 x 4868 chips (seeds 2..5) in flight on 4 streams, replayed from a CUDA graph.
Inputs (472 MB per chip) are resident in HBM and larger than L2.

Prints one JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle on bounded
cut-outs of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PSF-matched Mpix/s (solve+convolve+variance), batched mixed vs plain FP32"
WORKLOAD = dict(
    workload="full_chip_4846x4868_moffat_S2_49terms_300stamps",
    W=4846, H=4868, basis_sigma=(0.8, 1.6, 3.2), degrees=(6, 4, 2), kernel=31,
    spatial_order=2, stamps=300, grid=(15, 20), seed=2)
# DRAM bytes (read + write) of one k_conv_image launch on the full-chip workload, from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as it stands.
CONV_TRAFFIC_FULL_CHIP = 236.24064e6 + 75.099904e6
SM_COUNT = 152
FP32_LANES_PER_SM = 128
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3, "f32x2": 4, "bf16x6": 5}
PRECISION_NOTE = {
    "f32x2": "stamp design+Gram double-float (FP32 pairs), normal equations double-float "
             "Cholesky + FP64 refinement, FP32 image/variance",
    "fp64": "stamp design+Gram FP64, double-float Cholesky + FP64 refinement, FP32 image/variance",
    "fp32": "stamp design+Gram FP32 (plain), FP32 image/variance",
    "tf32": "FP32 stamp design, Gram on tensor cores (TF32), FP32 image/variance",
    "bf16x3": "FP32 stamp design, Gram on tensor cores (BF16x3), FP32 image/variance",
    "bf16x6": "stamp design double-float, Gram (sqrt(w) C)^T (sqrt(w) C) on the tcgen05 tensor "
              "cores from seven exact BF16 slices with exact per-level integer sums (bases of "
              "more than 64 augmented columns: double-float Gram), double-float Cholesky + FP64 "
              "refinement, FP32 image/variance"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--chips", type=int, default=4, help="full chips per step (batched)")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--single", action="store_true", help="one psfm_subtract per step, no batch")
    ap.add_argument("--exposure", action="store_true",
                    help="60 uneven chips of one exposure (GPU-generated inputs)")
    ap.add_argument("--small", action="store_true", help="512x512 plain-method workload")
    ap.add_argument("--stack", action="store_true", help="16-warp 6000x6000 stacking workload")
    ap.add_argument("--precision", default="bf16x6", choices=list(PRECISION))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the unbatched and plain FP32 comparison arms")
    ap.add_argument("--no-tune", action="store_true",
                    help="default image-convolution launch shape (no autotuning)")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the exposure and stacking sub-results")
    return ap.parse_args()


def chip_specs(precision, small=False):
    from paper_1901_09999_gb300 import psfm as P
    from paper_1901_09999_gb300 import synth
    prec = PRECISION[precision]
    if small:
        return (P.basis_spec((0.7, 1.5, 3.0), (4, 2, 2), 10, 0),
                P.config(badmask=synth.BADMASK, precision=prec))
    return (P.basis_spec(WORKLOAD["basis_sigma"], WORKLOAD["degrees"], 15, 2),
            P.config(badmask=synth.BADMASK, grid_nx=15, grid_ny=20, precision=prec))


def _gen_chip(args):
    seed, small = args
    sys.path.insert(0, ROOT)
    from paper_1901_09999_gb300 import synth
    f = synth.small_gaussian_field(seed) if small else synth.full_chip_field(seed)
    return f.sci, f.ref, f.var_sci, f.var_ref, f.mask_sci, f.mask_ref


def gen_chips(n, small):
    """Generate n seeded chips in parallel worker processes (spawned before any CUDA use)."""
    seeds = [(WORKLOAD["seed"] + i, small) for i in range(n)]
    if n == 1:
        return [_gen_chip(seeds[0])]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(n, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_chip, seeds)


def flops_per_pixel(b):
    """Algorithmic work per output pixel: image = separable passes plus per-pixel coefficient
    polynomials, 2w(N_H + N_b) + 2N_b(N_s + 1); variance = direct w^2 taps, 2w^2."""
    from paper_1901_09999_gb300 import psfm as P
    w = 2 * b.half_width + 1
    nb, ns = P.basis_size(b), P.spatial_size(b)
    nh = sum(b.degree[g] + 1 for g in range(b.n_gauss))
    return 2 * w * (nh + nb) + 2 * nb * (ns + 1), 2 * w * w


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # the raw samples go to PSFM_CLOCKS_DIR (default: the system temporary directory)
        d = os.environ.get("PSFM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"psfm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.f = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-i", str(self.index),
                                          "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.f is not None:
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle

# Samples the FP64 oracle is timed on (a baseline, not a target):
#  * "small": the 512 x 512 plain-method workload in full (30 stamps, S = 0, 27 terms);
#  * "chip_block": a block of 4 x 3 subregions of the full chip's real 15 x 20 grid (each
#    subregion 323 x 243 px, so 12 stamps and about 0.95 Mpix, plus the 30 px footprint margin
#    on every side), with the full-chip basis (S = 2, 49 terms); its stamps per pixel are those
#    of the chip, so the chip's rate follows linearly.
BLOCK_GRID = (4, 3)
BLOCK_MARGIN = 30   # stamp half width + kernel half width


def chip_block(chip, k, W=None, H=None):
    """Block k (row-major over the 15 / 4 x 20 / 3 blocks of the grid) of a full chip given as
    the 6 host arrays (sci, ref, var_sci, var_ref, mask_sci, mask_ref)."""
    H, W = chip[0].shape
    gx, gy = WORKLOAD["grid"]
    bx, by = BLOCK_GRID
    nbx = gx // bx
    i, j = k % nbx, (k // nbx) % (gy // by)
    x0, x1 = (i * bx * W) // gx, ((i + 1) * bx * W) // gx
    y0, y1 = (j * by * H) // gy, ((j + 1) * by * H) // gy
    xa, xb = max(0, x0 - BLOCK_MARGIN), min(W, x1 + BLOCK_MARGIN)
    ya, yb = max(0, y0 - BLOCK_MARGIN), min(H, y1 + BLOCK_MARGIN)
    return tuple(np.ascontiguousarray(a[ya:yb, xa:xb]) for a in chip)


def write_oracle_inputs(path, kind, chip=None, k=0):
    """Save one oracle sample: the small workload (seed 1 + k), or block k of a full chip
    (generated from the workload's seed unless given as the 6 host arrays)."""
    from paper_1901_09999_gb300 import synth
    if kind == "small":
        f = synth.small_gaussian_field(1 + k)
        arrs = (f.sci, f.ref, f.var_sci, f.var_ref, f.mask_sci, f.mask_ref)
    else:
        if chip is None:
            f = synth.full_chip_field(WORKLOAD["seed"])
            chip = (f.sci, f.ref, f.var_sci, f.var_ref, f.mask_sci, f.mask_ref)
        arrs = chip_block(chip, k)
    np.savez(path, kind=kind, I2=arrs[0], I1=arrs[1], V2=arrs[2], V1=arrs[3], m2=arrs[4],
             m1=arrs[5])


def oracle_sample(path):
    """Time the FP64 oracle's whole path (extraction, solve with the rejection loop, convolve,
    variance, mask, covariance pseudo-matrix) on one saved sample; returns (Mpix, seconds)."""
    from oracle import psfm_oracle as O
    from paper_1901_09999_gb300 import synth
    z = np.load(path)
    kind = str(z["kind"])
    I1, I2, V1, V2, m1, m2 = (z[k] for k in ("I1", "I2", "V1", "V2", "m1", "m2"))
    if kind == "small":
        ob = O.Basis((0.7, 1.5, 3.0), (4, 2, 2), 10, 0)
        oc = O.Config(badmask=synth.BADMASK)
    else:
        ob = O.Basis(WORKLOAD["basis_sigma"], WORKLOAD["degrees"], 15, 2)
        oc = O.Config(grid_nx=BLOCK_GRID[0], grid_ny=BLOCK_GRID[1], badmask=synth.BADMASK)
    t = time.perf_counter()
    sol = O.solve_kernel(I1, I2, V1, V2, m1, m2, ob, oc)
    O.convolve_image(I1, m1, sol, oc.badmask, I2)
    O.variance_image(V1, m1, sol, oc.badmask, 64, V2=V2)
    O.mask_image(m1, sol, oc, m2)
    O.pseudo_matrix(sol, oc)
    dt = time.perf_counter() - t
    return I1.size / 1e6, dt


def run_oracle_parallel(reps, paths):
    """Run the oracle sample ``reps`` times in one single-threaded process per path, all
    concurrently; returns (per-process [(Mpix, s)] lists, wall seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    t = time.perf_counter()
    procs = []
    for path in paths:
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "r=[bench.oracle_sample(%r) for _ in range(%d)]; print(json.dumps(r))"
                % (ROOT, path, reps))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    res = []
    for pr in procs:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return res, time.perf_counter() - t


def oracle_rate(res):
    """Aggregate throughput of concurrent processes: sum of each one's Mpix / busy seconds."""
    return sum(sum(a for a, _ in r) / sum(b for _, b in r) for r in res)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_paths(d, kind, n, chip=None):
    paths = []
    for k in range(n):
        p = os.path.join(d, f"oracle_{kind}_{k}.npz")
        write_oracle_inputs(p, kind, chip, k)
        paths.append(p)
    return paths


def cpu_baseline(cores, chip=None):
    """The oracle on the host cores: the small workload in full and a block of the full chip,
    each single-threaded (one process) and on every core (one single-threaded process per core,
    each on its own sample).  The headline value is the full-chip block on every core."""
    rows = []
    with tempfile.TemporaryDirectory() as d:
        for kind, what in (("small", "512x512 plain-method workload in full (30 stamps, S=0, "
                                     "27 terms)"),
                           ("chip_block", "4x3-subregion block of the 4846x4868 chip's real "
                                          "15x20 grid (12 stamps, ~1.0 Mpix with the 30 px "
                                          "margin, S=2, 49 terms), scaled linearly to the "
                                          "chip")):
            paths = oracle_paths(d, kind, cores, chip)
            single, w1 = run_oracle_parallel(1, paths[:1])
            allc, wn = run_oracle_parallel(1, paths)
            busy = sum(b for r in allc for _, b in r)
            rows.append({"sample": kind, "what": what, "mpix_per_sample": single[0][0][0],
                         "single_thread": oracle_rate(single), "all_cores": oracle_rate(allc),
                         "processes": len(paths), "cpu_s": round(busy, 1),
                         "wall_s": round(w1 + wn, 1)})
    head = rows[1]
    return {"value": head["all_cores"], "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "single_thread": head["single_thread"], "cpu_model": cpu_model(), "nproc": cores,
            "sample": f"FP64 numpy oracle, whole path (extraction, solve with rejection, convolve, "
                      f"variance, mask, pseudo-matrix); value = {head['what']}, one "
                      f"single-threaded process per core ({cores}), each on its own block",
            "rows": rows}


def reference_arm(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores, on blocks of the
    full-chip workload (each step: one 4 x 3-subregion block of the real 15 x 20 grid in each of
    one single-threaded process per core)."""
    cores = host_cores()
    with tempfile.TemporaryDirectory() as d:
        paths = oracle_paths(d, "chip_block", cores)
        for _ in range(args.warmup):
            run_oracle_parallel(1, paths)
        res, wall = run_oracle_parallel(args.steps, paths)
    val = oracle_rate(res)
    busy = sum(b for r in res for _, b in r)
    mpix = res[0][0][0]
    sample = (f"{args.steps} step(s); per step one 4x3-subregion block (~{mpix:.2f} Mpix with "
              f"margin, 12 stamps) of the full chip's 15x20 grid in each of {cores} "
              f"single-threaded processes; {busy:.1f} CPU-s")
    print(json.dumps({
        "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference", "device": f"host cores only ({cores}); the GPUs of the launch idle",
        "config": dict(WORKLOAD, sample=sample),
        "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ----------------------------------------------------------------------------- GPU arm

def exposure_chips(dev, seed=4, n=60, precision="f32x2"):
    """60 chips of uneven sizes, PSF FWHM 3-8 px, masked 1-20 %, S = 1..3, 49-70 terms, basis
    widths by the paper's ISIS prescription scaled by the chip's worse seeing (GPU-generated)."""
    from paper_1901_09999_gb300 import psfm as P
    from paper_1901_09999_gb300 import synth
    chips, bases = [], []
    for c in synth.exposure_chips(seed, n):
        fmax = max(c["fwhm_ref"], c["fwhm_sci"])
        sig = synth.isis_prescription_sigmas(fmax)
        h = int(np.ceil(4.7 * sig[-1]))
        chips.append(synth.torch_chip_pair(c["seed"], c["W"], c["H"], c["fwhm_ref"],
                                           c["fwhm_sci"], c["mask_frac"], dev))
        bases.append(P.basis_spec(sig, c["degrees"], h, c["spatial_order"]))
    cfg = P.config(badmask=synth.BADMASK, grid_nx=12, grid_ny=12, precision=PRECISION[precision])
    return chips, bases, cfg


STACK = dict(workload="stack_16_warps_6000x6000_target_fwhm7.5_S1", warps=16, size=6000,
             sources=6000, target_fwhm=7.5, spatial_order=1, grid=(12, 12), seed=5)


def stack_result(dev, args, steps, warmup, stream):
    """Config 5: PSF-homogenised stack of 16 warps of one 6000 x 6000 skycell (psfm_stack: each
    warp matched to a Gaussian target of FWHM 7.5 px, convolved with its variance, mask and
    pseudo-matrix, then the inverse-variance weighted coadd).  Mpix/s counts input pixels.
    Returns a result dict (value, ms_per_step, config, launches, stage times)."""
    import torch
    from paper_1901_09999_gb300 import psfm as P
    from paper_1901_09999_gb300 import synth
    n, size = STACK["warps"], STACK["size"]
    warps, src = synth.torch_skycell_warps(STACK["seed"], n, size, STACK["sources"], dev)
    sig = synth.isis_prescription_sigmas(STACK["target_fwhm"])
    h = int(np.ceil(4.7 * sig[-1]))
    b = P.basis_spec(sig, (6, 4, 2), h, STACK["spatial_order"])
    cfg = P.config(badmask=synth.BADMASK, grid_nx=STACK["grid"][0], grid_ny=STACK["grid"][1],
                   precision=PRECISION[args.precision])
    imgs = [w["image"] for w in warps]
    vars_ = [w["var"] for w in warps]
    masks = [w["mask"] for w in warps]
    shape = P.psfm_shape(size, size, size)
    if not args.no_tune:
        autotune([b], [(size, size)], stream)
    ws = torch.empty(P.psfm_workspace_size(P.OP_STACK, shape, b, cfg, len(src)), dtype=torch.uint8,
                     device=dev)

    def step():
        return P.psfm_stack(imgs, vars_, masks, [src] * n, STACK["target_fwhm"], [b] * n, cfg,
                            workspace=ws, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            out = step()
        torch.cuda.synchronize()
        l0 = P.psfm_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            out = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = P.psfm_launch_count() - l0
        P.psfm_profile_enable(True)
        step()
        torch.cuda.synchronize()
        prof = P.psfm_profile_read()
        P.psfm_profile_enable(False)
    cnt = out[3].cpu().numpy()
    conv_ms, conv_n, _ = prof.get("conv_image", (float("nan"), 1, 1))
    f_img, _ = flops_per_pixel(b)
    res = {"value": n * size * size / 1e6 * steps / (ms / 1e3), "unit": "Mpix/s",
           "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
           "config": dict(STACK, h=h, basis_sigma=list(sig), degrees=[6, 4, 2],
                          precision=args.precision, counts="input pixels",
                          output_mpix=size * size / 1e6, coverage_mean=float(cnt.mean()),
                          l2="inputs larger than L2"),
           "gpu_launches": launches, "conv_image_ms": conv_ms / conv_n,
           "conv_image_tflops": size * size * f_img / (conv_ms / conv_n / 1e3) / 1e12,
           "stages_ms": {k: v[0] for k, v in prof.items()}}
    del warps, imgs, vars_, masks, ws, out
    return res


def exposure_result(dev, args, steps, warmup, stream):
    """Config 4: one exposure of 60 uneven chips in one batch (graph replay); returns a result
    dict (value, ms_per_step, config, launches)."""
    import torch
    from paper_1901_09999_gb300 import psfm as P
    chips, bases, cfg = exposure_chips(dev, precision=args.precision)
    mpix = sum(c["img"].numel() for c in chips) / 1e6
    if not args.no_tune:
        autotune(bases, [(c["img"].shape[1], c["img"].shape[0]) for c in chips], stream)
    batch = P.Batch(chips, bases, cfg, n_streams=args.streams, want_cov=True)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            batch.run(stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            batch.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sols = batch.solutions(stream)
    res = {"value": mpix * steps / (ms / 1e3), "unit": "Mpix/s", "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup,
           "config": {"workload": "exposure_60_uneven_chips_S1-3_49-70terms", "chips": len(chips),
                      "mpix": mpix, "precision": args.precision,
                      "batching": f"{len(chips)} chips on {args.streams} streams, CUDA graph "
                                  "replay"},
           "gpu_launches": batch.kernel_count() * steps,
           "stamps_used_min": min(s_.n_used for s_ in sols)}
    batch.close()
    del chips, batch
    return res


def run_stack(args, world, local):
    """--stack: the stacking workload as the bench line."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1901_09999_gb300 import build
    build.build()
    stream = torch.cuda.Stream()
    with ClockSampler(local) as clk:
        r = stack_result(dev, args, args.steps, max(3, args.warmup), stream)
    print(json.dumps({
        "metric": METRIC, "value": r["value"], "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": r["warmup"], "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": r["config"], "gpu_launches": r["gpu_launches"],
        "clocks": clk.summary(), "stages_ms": r["stages_ms"]}))
    return 0


def autotune(bases, sizes, stream):
    """Tunes the image convolution's launch shape (tile height, planes per chunk) for every
    distinct basis class of the workload on a synthetic image of that class's size (the
    largest chip of the class: larger than L2, as the real inputs are, so that the staging of
    each tile from HBM is part of what is timed), unless the library's table has it already
    (loaded from PSFM_TUNE_CACHE when set).  Returns the table entries used and the seconds
    spent."""
    from paper_1901_09999_gb300 import psfm as P
    t0 = time.perf_counter()
    cache = os.environ.get("PSFM_TUNE_CACHE")
    if cache and os.path.exists(cache):
        try:
            P.tune_load(cache)
        except Exception:
            pass
    have = {(e["half_width"], e["spatial_order"], tuple(e["degree"])) for e in P.tune_entries()}
    classes = {}
    for b, (w, h) in zip(bases, sizes):
        key = (b.half_width, b.spatial_order, tuple(b.degree[:b.n_gauss]))
        cw, ch = classes.get(key, (0, 0, None))[:2]
        classes[key] = (max(cw, w), max(ch, h), b)
    for key, (w, h, b) in classes.items():
        if key not in have:
            P.tune_conv(b, w, h, stream)
    if cache:
        try:
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            P.tune_save(cache)
        except Exception:
            pass
    used = [e for e in P.tune_entries()
            if (e["half_width"], e["spatial_order"], tuple(e["degree"])) in classes]
    return used, time.perf_counter() - t0


def fp32_peak_probe(dev, stream, sms):
    """Measured FP32 FMA throughput (TFLOP/s) of the library's probe kernel: 8 blocks of 256
    threads per SM, 8 independent chains per thread; best of 3 launches after one warm-up."""
    import torch
    from paper_1901_09999_gb300 import psfm as P
    best = 0.0
    with torch.cuda.stream(stream):
        P.fma_probe(sms * 8, 4000, stream)
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl, _ = P.fma_probe(sms * 8, 40000, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def max_over_ranks(ms, world, device=None):
    """Slowest rank's time of the timed region (every rank holds the same work: replicas)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(px_per_step, world, steps, ms):
    """Whole-job Mpix/s: the pixels every rank processed over the slowest rank's time."""
    return px_per_step * world * steps / 1e6 / (ms / 1e3)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return 0

    if args.stack:
        return run_stack(args, world, local)

    nchips = 1 if args.single else args.chips
    host_chips = None
    if not args.exposure:
        # numpy generation in spawned workers before the first CUDA call
        host_chips = gen_chips(nchips, args.small)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1901_09999_gb300 import build
    build.build()
    from paper_1901_09999_gb300 import psfm as P

    def put(a):
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    if args.exposure:
        chips, bases, cfg = exposure_chips(dev, precision=args.precision)
        workload = dict(workload="exposure_60_uneven_chips_S1-3_49-70terms", chips=len(chips),
                        mpix=sum(c["img"].numel() for c in chips) / 1e6)
    else:
        b, cfg = chip_specs(args.precision, args.small)
        chips = [dict(img=put(c[0]), ref=put(c[1]), var_img=put(c[2]), var_ref=put(c[3]),
                      mask_img=put(c[4]), mask_ref=put(c[5])) for c in host_chips]
        bases = [b] * len(chips)
        workload = (dict(WORKLOAD) if not args.small else
                    {"workload": "small_512x512_gaussian_S0_27terms"})
        workload.update(chips_per_step=len(chips),
                        seeds=[WORKLOAD["seed"] + i for i in range(len(chips))])
    oracle_chip = host_chips[0] if (host_chips and not args.small) else None
    del host_chips
    px_per_step = sum(c["img"].numel() for c in chips)
    stream = torch.cuda.Stream()
    tuning, tuning_s = (None, 0.0)
    if not args.no_tune:
        tuning, tuning_s = autotune(bases, [(c["img"].shape[1], c["img"].shape[0]) for c in chips],
                                    stream)

    if args.single:
        c0 = chips[0]
        outs = dict(out=torch.empty_like(c0["img"]), out_var=torch.empty_like(c0["img"]),
                    out_mask=torch.empty_like(c0["mask_img"]))
        shape = P.psfm_shape(c0["img"].shape[1], c0["img"].shape[0], c0["img"].stride(0))
        ws = torch.empty(P.psfm_workspace_size(P.OP_SUBTRACT, shape, bases[0], cfg),
                         dtype=torch.uint8, device=dev)

        def step():
            P.psfm_subtract(c0["img"], c0["ref"], c0["var_img"], c0["var_ref"], c0["mask_img"],
                            c0["mask_ref"], bases[0], cfg, workspace=ws, stream=stream, **outs)
        batch = None
    else:
        batch = P.Batch(chips, bases, cfg, n_streams=args.streams, want_cov=True)

        def step():
            batch.run(stream)

    sols = None
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        if batch is not None:
            sols = batch.solutions(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        l0 = P.psfm_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if batch is not None:
            sols = batch.solutions(stream)
            launches = batch.kernel_count() * args.steps
        else:
            launches = P.psfm_launch_count() - l0
    ms = max_over_ranks(ms, world, dev)
    value = job_throughput(px_per_step, world, args.steps, ms)

    # roofline of the dominant kernel, timed with the library's CUDA events on its stream in a
    # separate (non-graph, unshared) subtraction of chip 0 right after the timed region
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else 2070.0
    c0, b0 = chips[0], bases[0]
    P.psfm_profile_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(2):
            P.psfm_subtract(c0["img"], c0["ref"], c0["var_img"], c0["var_ref"], c0["mask_img"],
                            c0["mask_ref"], b0, cfg, stream=stream)
    torch.cuda.synchronize()
    prof = P.psfm_profile_read()
    P.psfm_profile_enable(False)
    f_img, f_var = flops_per_pixel(b0)
    npx0 = c0["img"].numel()
    conv_ms, conv_n, _ = prof.get("conv_image", (float("nan"), 1, 1))
    var_ms, var_n, _ = prof.get("variance", (float("nan"), 1, 1))
    peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    probe = fp32_peak_probe(dev, stream, sms)
    achieved = npx0 * f_img / (conv_ms / conv_n / 1e3) / 1e12
    step_flops = sum(c["img"].numel() * sum(flops_per_pixel(b)) for c, b in zip(chips, bases))
    step_tflops = step_flops / (ms / args.steps / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": (CONV_TRAFFIC_FULL_CHIP if (not args.small and not args.exposure)
                            else None),
                "kernel": "k_conv_image", "kernel_ms": conv_ms / conv_n,
                "algorithmic_flop_per_px": f_img,
                "peak_note": f"FP32 FMA: {sms} SMs (device properties) x 128 lanes x 2 flop x "
                             f"{sm_mhz:.0f} MHz (median SM clock sampled in the timed region)",
                "peak_probe": probe, "frac_of_probe": achieved / probe,
                "variance_kernel": {"achieved": npx0 * f_var / (var_ms / var_n / 1e3) / 1e12,
                                    "ms": var_ms / var_n},
                "step": {"flop_per_px": f_img + f_var, "achieved": step_tflops,
                         "frac": step_tflops / peak,
                         "what": "image + variance algorithmic flops of every chip of a step / "
                                 "ms_per_step (the solve side counted as overhead)"}}
    stages = {k: v[0] / v[2] for k, v in prof.items()}

    # comparison arms on the same chips: (1) batching: one unbatched psfm_subtract per chip at
    # the same precision; (2) precision: the same batch with FP32 stamp design and Gram (the
    # plain FP32 path; its normal equations are not numerically positive definite, so it takes
    # the FP64 LU fallback, and it misses the parity tolerances)
    comparisons = None
    if not args.no_plain and not args.single:
        def time_arm(fn, n):
            with torch.cuda.stream(stream):
                fn()
                torch.cuda.synchronize()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                for _ in range(n):
                    fn()
                a1.record(stream)
                torch.cuda.synchronize()
            return a0.elapsed_time(a1) / n

        outs1 = [dict(out=P._like(c["img"]), out_var=P._like(c["img"]),
                      out_mask=P._like(c["mask_img"])) for c in chips]
        ws1 = torch.empty(max(P.psfm_workspace_size(
            P.OP_SUBTRACT, P.psfm_shape(c["img"].shape[1], c["img"].shape[0], c["img"].stride(0)),
            b, cfg) for c, b in zip(chips, bases)), dtype=torch.uint8, device=dev)

        def unbatched():
            for c, b, o in zip(chips, bases, outs1):
                P.psfm_subtract(c["img"], c["ref"], c["var_img"], c["var_ref"], c["mask_img"],
                                c["mask_ref"], b, cfg, workspace=ws1, stream=stream, **o)

        n3 = max(1, min(3, args.steps))
        ums = time_arm(unbatched, n3)
        del outs1, ws1
        _, cfg32 = chip_specs("fp32", args.small)
        batch32 = P.Batch(chips, bases, cfg32, n_streams=args.streams, want_cov=True)
        pms = time_arm(lambda: batch32.run(stream), n3)
        batch32.close()
        del batch32
        # the other accurate mode: the double-float Gram when timing the tensor-core one, and
        # the other way round
        other = "f32x2" if args.precision != "f32x2" else "bf16x6"
        _, cfgo = chip_specs(other, args.small)
        batcho = P.Batch(chips, bases, cfgo, n_streams=args.streams, want_cov=True)
        tms = time_arm(lambda: batcho.run(stream), n3)
        batcho.close()
        del batcho
        comparisons = {
            "unbatched_same_precision": {
                "value": px_per_step / 1e6 / (ums / 1e3), "unit": "Mpix/s", "ms_per_step": ums,
                "what": f"same chips, one psfm_subtract each ({args.precision}), no streams or "
                        "graph"},
            "batched_plain_fp32": {
                "value": px_per_step / 1e6 / (pms / 1e3), "unit": "Mpix/s", "ms_per_step": pms,
                "what": "same batch (streams + graph), FP32 stamp design and Gram; fails the "
                        "parity tolerances (FP32 normal equations; FP64 LU fallback)"},
            "batched_over_unbatched": ums / (ms / args.steps),
            "this_precision_over_plain_fp32": pms / (ms / args.steps)}
        comparisons[f"batched_{other}"] = {
            "value": px_per_step / 1e6 / (tms / 1e3), "unit": "Mpix/s", "ms_per_step": tms,
            "what": ("same batch, stamp Gram in double-float on the FP32 pipes (meets the "
                     "parity tolerances)") if other == "f32x2" else
                    ("same batch, stamp Gram on the tensor cores from exact BF16 split products "
                     "(meets the parity tolerances)")}

    e2e = None
    if not args.no_e2e and not args.exposure:
        keys = ("img", "ref", "var_img", "var_ref", "mask_img", "mask_ref")
        h_in = [[c[k].cpu().pin_memory() for k in keys] for c in chips]
        bi = sum(t.numel() * t.element_size() for hs in h_in for t in hs)
        if batch is not None:
            # two device buffer sets, each with its own batch graph: while one step computes,
            # the copy stream uploads the next step's inputs into the other set and reads the
            # previous step's outputs back
            chips2 = [{k: torch.empty_like(c[k]) for k in keys} for c in chips]
            batch2 = P.Batch(chips2, bases, cfg, n_streams=args.streams, want_cov=True)
            sets = [(chips, batch), (chips2, batch2)]
            h_out = [[[torch.empty(t.shape, dtype=t.dtype).pin_memory()
                       for t in (b.diff[i], b.diff_var[i], b.diff_mask[i])]
                      for i in range(len(chips))] for _, b in sets]
            bo = sum(t.numel() * t.element_size() for hs in h_out[0] for t in hs)
            # host-to-device and device-to-host copies on streams of their own, so that the two
            # directions of the link run at the same time
            up = torch.cuda.Stream()
            down = torch.cuda.Stream()
            ev_up = [torch.cuda.Event(), torch.cuda.Event()]
            ev_comp = [torch.cuda.Event(), torch.cuda.Event()]
            ev_down = [torch.cuda.Event(), torch.cuda.Event()]

            def upload(si):
                for c, hs in zip(sets[si][0], h_in):
                    for k, hh in zip(keys, hs):
                        c[k].copy_(hh, non_blocking=True)
                ev_up[si].record(up)

            def download(si):
                b = sets[si][1]
                for i, hs in enumerate(h_out[si]):
                    for hh, d in zip(hs, (b.diff[i], b.diff_var[i], b.diff_mask[i])):
                        hh.copy_(d, non_blocking=True)
                ev_down[si].record(down)

            def e2e_run(n, start_event=None):
                with torch.cuda.stream(up):
                    if start_event is not None:
                        up.wait_event(start_event)
                    upload(0)
                for k in range(n):
                    si = k % 2
                    stream.wait_event(ev_up[si])
                    if k >= 2:  # this set's outputs of two steps ago have been read back
                        stream.wait_event(ev_down[si])
                    sets[si][1].run(stream)
                    ev_comp[si].record(stream)
                    if k + 1 < n:
                        with torch.cuda.stream(up):
                            if k >= 1:  # the other set's inputs are free once its step is done
                                up.wait_event(ev_comp[1 - si])
                            upload(1 - si)
                    with torch.cuda.stream(down):
                        down.wait_event(ev_comp[si])
                        download(si)
                stream.wait_event(ev_down[(n - 1) % 2])

            e2e_run(2)  # captures the second graph
            torch.cuda.synchronize()
            n2 = max(2, args.steps)
            e0.record(stream)
            e2e_run(n2, e0)
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms = e0.elapsed_time(e1)
            batch2.close()
            del chips2
        else:
            d_out = [(outs["out"], outs["out_var"], outs["out_mask"])]
            h_out = [[torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in o] for o in d_out]
            bo = sum(t.numel() * t.element_size() for hs in h_out for t in hs)

            def e2e_step():
                for c, hs in zip(chips, h_in):
                    for k, hh in zip(keys, hs):
                        c[k].copy_(hh, non_blocking=True)
                step()
                for hs, ds in zip(h_out, d_out):
                    for hh, d in zip(hs, ds):
                        hh.copy_(d, non_blocking=True)

            with torch.cuda.stream(stream):
                e2e_step()
                torch.cuda.synchronize()
                n2 = max(2, args.steps // 2)
                e0.record(stream)
                for _ in range(n2):
                    e2e_step()
                e1.record(stream)
                torch.cuda.synchronize()
            e2e_ms = e0.elapsed_time(e1)
        e2e = {"value": px_per_step * n2 / 1e6 / (e2e_ms / 1e3), "unit": "Mpix/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "overlap": "copies of one step overlap the compute of the next (two buffer sets; "
                          "uploads and read-backs on separate streams)"
                          if batch is not None else "none"}

    # the batching and stacking workloads as sub-results of the same run (their own steps)
    subs = {}
    if not args.no_sub and not args.small and not args.exposure and not args.single:
        if batch is not None:
            batch.close()
            batch = None
        del chips
        torch.cuda.empty_cache()
        for name, fn in (("exposure", exposure_result), ("stack", stack_result)):
            try:
                subs[name] = fn(dev, args, 3, 2, stream)
            except Exception as e:  # reported, not fatal for the headline
                subs[name] = {"error": str(e)[-300:]}
            torch.cuda.empty_cache()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(host_cores(), oracle_chip)
        except Exception as e:  # the oracle is a reported baseline only
            cpu = {"error": str(e)[-300:]}
    sol_info = None
    if sols is not None:
        sol_info = [{"n_used": s_.n_used, "n_iter": s_.n_iter, "b0": s_.b0, "r_bad": s_.r_bad}
                    for s_ in sols[:4]]
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload, l2="inputs larger than L2 (472 MB per chip), no flush",
                       precision=PRECISION_NOTE[args.precision],
                       batching=("none" if args.single else
                                 f"{nchips} chips on {args.streams} streams, CUDA graph replay"),
                       parallelism=f"replicas x{world}"),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "comparisons": comparisons, "sub_results": subs or None,
        "tuning": {"entries": tuning, "seconds": tuning_s,
                   "what": "image-convolution launch shape per basis class, chosen by the "
                           "library's autotuner (psfm_tune_conv) before the timed region"},
        "clocks": clocks, "single_chip_stages_ms": stages, "solutions": sol_info,
    }
    print(json.dumps(line))
    if batch is not None:
        batch.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
