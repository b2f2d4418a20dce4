"""Shared helpers of the GPU parity tests: seeded workloads, device upload, oracle mirrors of
the C-ABI basis / config structures, and the comparison metrics with their tolerances."""
import numpy as np

from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

# Per-pixel image tolerance: 1e-3 of the local noise sigma (sqrt of the output variance).
IMG_TOL_SIGMA = 1e-3
# Variance map: FP32 kernel realisation and 31^2-tap FP32 sums against FP64.
VAR_RTOL = 2e-5
# Pseudo-matrix: FP64 on both sides.
COV_ATOL = 1e-10
# Pseudo-matrix of a difference: the combination weights are mean variances taken from the
# FP32 variance maps (relative error ~1e-7).
COV_DIFF_ATOL = 1e-6


def device():
    import torch
    from paper_1901_09999_gb300 import build
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    build.build()
    P.load()
    return torch.device("cuda:0")


def upload(field, dev, pad=0):
    """Field -> dict of CUDA tensors; ``pad`` extra columns give a row pitch > width."""
    import torch

    def put(a, dtype=None):
        H, W = a.shape
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        t = torch.zeros((H, W + pad), dtype=torch.from_numpy(a[:1, :1]).dtype, device=dev)
        t[:, :W] = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        return t[:, :W]

    return dict(ref=put(field.ref), sci=put(field.sci), var_ref=put(field.var_ref),
                var_sci=put(field.var_sci), mask_ref=put(field.mask_ref),
                mask_sci=put(field.mask_sci))


def host(t):
    a = t.cpu().numpy()
    return a.view(np.uint16) if a.dtype == np.int16 else a


def specs(sigma, degree, h, S, **cfg):
    """The same basis / config for the C ABI and the oracle."""
    b = P.basis_spec(sigma, degree, h, S)
    c = P.config(**cfg)
    ob = O.Basis(tuple(sigma), tuple(degree), h, S)
    oc = O.Config(grid_nx=c.grid_nx, grid_ny=c.grid_ny,
                  stamp_half=None if c.stamp_half < 0 else c.stamp_half,
                  thresh_nsigma=c.thresh_nsigma, reject_nsigma=c.reject_nsigma,
                  soften_alpha=c.soften_alpha, bad_frac=c.bad_frac, max_iter=c.max_iter,
                  var_tile=c.var_tile, cov_grid=c.cov_grid,
                  norm_mode="joint" if c.norm_mode == P.NORM_JOINT else "separate",
                  badmask=c.badmask, conv_bad=c.conv_bad, conv_poor=c.conv_poor,
                  max_cand=c.max_cand, dual=bool(c.dual), penalty=c.penalty)
    return b, c, ob, oc


def oracle_solution_from_gpu(sol: P.Solution, ob, W, H):
    """The oracle's Solution holding a GPU solution's coefficients (both kernels' terms when
    the solution has 2 N_b N_s of them: the dual kernel)."""
    n = len(O.basis_terms(ob)) * len(O.spatial_terms(ob.S))
    dual = sol.ncoef == 2 * n
    coeff = np.concatenate([sol.coeff[:sol.ncoef], [sol.d0]])
    return O.Solution(sol.b0, coeff, sol.d0, ob, W, H, dual=dual)


def gpu_solution_from_oracle(osol: O.Solution, r_bad):
    n = osol.a.size
    return P.Solution.from_values(osol.b0, osol.d0, osol.coeff[:n], r_bad)


def kernel_rel_err(sol_a: O.Solution, sol_b: O.Solution, points):
    """max over points of ||K_a - K_b||_2 / ||K_b||_2 of the realised kernels."""
    e = 0.0
    for x, y in points:
        Ka, Kb = O.realise_kernel(sol_a, x, y), O.realise_kernel(sol_b, x, y)
        e = max(e, float(np.linalg.norm(Ka - Kb) / np.linalg.norm(Kb)))
    return e


def coeff_rel_err(a, b):
    """Normwise relative error of coefficient vectors."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))
