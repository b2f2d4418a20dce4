#!/usr/bin/env python3
"""Benchmark of the PSF-matching hot path: PSF-matched Mpix/s (solve + convolve + variance).

One step is one full subtraction of the full-chip workload through the C ABI call
``psfm_subtract``: stamp extraction, basis convolution and Gram per stamp, normalisation,
the FP64 solve with the iterative stamp rejection, r_bad, then the spatially varying
convolution of the whole chip, the per-patch variance propagation, the mask propagation and
the covariance pseudo-matrix.  Inputs (4846 x 4868 float32 images, variances and uint16
masks; about 472 MB) are resident in HBM and larger than L2.

Prints one JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle on bounded
cut-outs of the same workload instead.
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
sys.path.insert(0, ROOT)

METRIC = "PSF-matched Mpix/s (solve+convolve+variance), batched mixed vs plain FP32"
WORKLOAD = dict(
    workload="full_chip_4846x4868_moffat_S2_49terms_300stamps",
    W=4846, H=4868, basis_sigma=(0.8, 1.6, 3.2), degrees=(6, 4, 2), kernel=31,
    spatial_order=2, stamps=300, grid=(15, 20), seed=2)
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--small", action="store_true", help="512x512 plain-method workload")
    ap.add_argument("--precision", default="f32x2", choices=["fp64", "f32x2", "fp32"],
                    help="arithmetic of the stamp design blocks and Gram matrices")
    return ap.parse_args()


PRECISION = {"fp64": 0, "fp32": 1, "f32x2": 4}


def workload_specs(small, precision="f32x2"):
    from paper_1901_09999_gb300 import psfm as P
    from paper_1901_09999_gb300 import synth
    prec = PRECISION[precision]
    if small:
        b = P.basis_spec((0.7, 1.5, 3.0), (4, 2, 2), 10, 0)
        c = P.config(badmask=synth.BADMASK, precision=prec)
    else:
        b = P.basis_spec(WORKLOAD["basis_sigma"], WORKLOAD["degrees"], 15, 2)
        c = P.config(badmask=synth.BADMASK, grid_nx=15, grid_ny=20, precision=prec)
    return b, c


def make_field(small, seed):
    from paper_1901_09999_gb300 import synth
    if small:
        return synth.small_gaussian_field(seed)
    return synth.full_chip_field(seed)


def flops_per_pixel(b):
    """Algorithmic work per output pixel (image: separable passes plus coefficient
    evaluation; variance: direct w^2 taps)."""
    from paper_1901_09999_gb300 import psfm as P
    w = 2 * b.half_width + 1
    nb = P.basis_size(b)
    ns = P.spatial_size(b)
    nh = sum(b.degree[g] + 1 for g in range(b.n_gauss))
    return 2 * w * (nh + nb) + 2 * nb * (ns + 1), 2 * w * w


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
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

_ORACLE_INPUTS = None


def oracle_inputs():
    """A 288 x 288 cut-out around the centre of the full-chip workload (generated once)."""
    global _ORACLE_INPUTS
    if _ORACLE_INPUTS is None:
        from paper_1901_09999_gb300 import synth
        f = synth.full_chip_field(WORKLOAD["seed"])
        n = 288
        y0, x0 = (f.shape[0] - n) // 2, (f.shape[1] - n) // 2
        cut = lambda a: np.ascontiguousarray(a[y0:y0 + n, x0:x0 + n])
        _ORACLE_INPUTS = tuple(map(cut, (f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci)))
    return _ORACLE_INPUTS


def oracle_sample():
    """Time the FP64 oracle (solve + convolve + variance + mask + covariance) on the cut-out
    with the full-chip basis (S = 2, 49 terms) and a 2 x 2 stamp grid."""
    from oracle import psfm_oracle as O
    from paper_1901_09999_gb300 import synth
    I1, I2, V1, V2, m1, m2 = oracle_inputs()
    n = I1.shape[0]
    ob = O.Basis(WORKLOAD["basis_sigma"], WORKLOAD["degrees"], 15, 2)
    oc = O.Config(grid_nx=2, grid_ny=2, badmask=synth.BADMASK)
    t = time.perf_counter()
    sol = O.solve_kernel(I1, I2, V1, V2, m1, m2, ob, oc)
    O.convolve_image(I1, m1, sol, oc.badmask, I2)
    O.variance_image(V1, m1, sol, oc.badmask, 64, V2=V2)
    O.mask_image(m1, sol, oc, m2)
    O.pseudo_matrix(sol, oc)
    dt = time.perf_counter() - t
    return n * n / 1e6, dt


def run_oracle_subprocess(reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; r=[bench.oracle_sample() for _ in range(%d)];"
            "print(json.dumps(r))" % (ROOT, reps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         cwd=ROOT, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(reps=1):
    r = run_oracle_subprocess(reps)
    mpix = sum(a for a, _ in r)
    sec = sum(b for _, b in r)
    return {"value": mpix / sec, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(r)} x 288x288 cut-out of the full-chip workload (S=2, 49 terms, "
                      f"2x2 stamp grid), solve+convolve+variance+mask+covariance, FP64 numpy, "
                      f"single-threaded BLAS, {sec:.1f} s"}


# ----------------------------------------------------------------------------- main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            run_oracle_subprocess(1)
        r = run_oracle_subprocess(args.steps)
        mpix = sum(a for a, _ in r)
        sec = sum(b for _, b in r)
        val = mpix / sec
        print(json.dumps({
            "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * sec / len(r), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(WORKLOAD, sample="288x288 cut-out per step"),
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(r)} x 288x288 cut-outs, {sec:.1f} s"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1901_09999_gb300 import build
    build.build()
    from paper_1901_09999_gb300 import psfm as P

    b, c = workload_specs(args.small, args.precision)
    field = make_field(args.small, WORKLOAD["seed"] + rank)
    H, W = field.shape

    def put(a):
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    t_img, t_ref = put(field.sci), put(field.ref)
    t_vi, t_vr = put(field.var_sci), put(field.var_ref)
    t_mi, t_mr = put(field.mask_sci), put(field.mask_ref)
    out = torch.empty_like(t_img)
    out_var = torch.empty_like(t_img)
    out_mask = torch.empty_like(t_mi)
    shape = P.psfm_shape(W, H, W)
    need = P.psfm_workspace_size(P.OP_SUBTRACT, shape, b, c)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return P.psfm_subtract(t_img, t_ref, t_vi, t_vr, t_mi, t_mr, b, c, out=out, out_var=out_var,
                               out_mask=out_mask, workspace=ws, stream=stream)

    for _ in range(max(3, args.warmup)):
        sol = step()[4]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    launches0 = P.psfm_launch_count()
    P.psfm_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            sol = step()[4]
        e1.record(stream)
        torch.cuda.synchronize()
    prof = P.psfm_profile_read()
    P.psfm_profile_enable(False)
    launches = P.psfm_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    mpix_total = W * H * world * args.steps / 1e6
    value = mpix_total / (ms / 1e3)

    # roofline of the dominant kernel (the spatially varying image convolution)
    f_img, f_var = flops_per_pixel(b)
    stages = {k: v for k, v in prof.items()}
    conv_ms, conv_n, _ = stages.get("conv_image", (float("nan"), 1, 1))
    var_ms, var_n, _ = stages.get("variance", (float("nan"), 1, 1))
    peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    achieved = W * H * f_img / (conv_ms / conv_n / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None, "kernel": "k_conv_image",
                "kernel_ms": conv_ms / conv_n,
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)",
                "variance_kernel": {"achieved": W * H * f_var / (var_ms / var_n / 1e3) / 1e12,
                                    "ms": var_ms / var_n}}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda t: t.cpu().pin_memory()
        h_in = [pin(t) for t in (t_img, t_ref, t_vi, t_vr, t_mi, t_mr)]
        h_out = [torch.empty(out.shape, dtype=out.dtype).pin_memory(),
                 torch.empty(out.shape, dtype=out.dtype).pin_memory(),
                 torch.empty(out_mask.shape, dtype=out_mask.dtype).pin_memory()]
        d_in = [t_img, t_ref, t_vi, t_vr, t_mi, t_mr]
        bi = sum(t.numel() * t.element_size() for t in h_in)
        bo = sum(t.numel() * t.element_size() for t in h_out)

        def e2e_step():
            for d, h in zip(d_in, h_in):
                d.copy_(h, non_blocking=True)
            step()
            for h, d in zip(h_out, (out, out_var, out_mask)):
                h.copy_(d, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        n2 = max(2, args.steps // 2)
        e0.record(stream)
        for _ in range(n2):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": W * H * n2 / 1e6 / (e0.elapsed_time(e1) / 1e3), "unit": "Mpix/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(8)
        except Exception as e:  # the oracle is a reported baseline only
            cpu = {"error": str(e)[-300:]}
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD if not args.small else {"workload": "small_512x512_gaussian_S0_27terms"},
                       l2="inputs (472 MB) larger than L2, no flush",
                       precision=f"stamp design+Gram {args.precision}, FP64 normal equations, FP32 image/variance passes",
                       parallelism=f"replicas x{world}"),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(), "stages_ms": {k: v[0] / args.steps for k, v in stages.items()},
        "solution": {"n_used": sol.n_used, "n_iter": sol.n_iter, "b0": sol.b0, "r_bad": sol.r_bad},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
