"""Full-size parity on the 4846 x 4868 chip (seed 2) in the launch configuration the benchmark
times (a batch of chips on priority stream pairs, replayed from a CUDA graph), against the FP64
oracle's solution stored in tests/golden/full_chip_seed2_oracle.npz (written by
tests/golden/make_full_chip_solution.py, which calls only the oracle):

* stamp candidates, statuses, iteration count and r_bad bit-exact; b0 and the realised kernel
  within tolerance;
* the difference image, its variance and its mask at sampled pixels, each evaluated by the
  oracle one pixel at a time with the stored solution;
* the pseudo-matrix of the difference against the oracle's pseudo-matrix of the convolution,
  combined with the delta of the unconvolved image (Sec. 4.4).

Then the precision study: the same chip through every solve precision, each result's error
against the oracle reported (coefficients, realised kernel, difference image, variance) with
the recovered fluxes of the 50 injected transients."""
import os

import numpy as np
import pytest

from gpu_common import IMG_TOL_SIGMA, VAR_RTOL, coeff_rel_err, device, host, kernel_rel_err, \
    oracle_solution_from_gpu
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "full_chip_seed2_oracle.npz")
KERNEL_RTOL = 1e-6
COEFF_RTOL = 1e-6
B0_RTOL = 1e-9
N_SAMPLES = 240


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def chip():
    g = np.load(GOLDEN)
    f = synth.full_chip_field(int(g["seed"]))
    ob = O.Basis(tuple(g["basis_sigma"]), tuple(int(d) for d in g["degrees"]), int(g["h"]),
                 int(g["S"]))
    oc = O.Config(grid_nx=int(g["grid"][0]), grid_ny=int(g["grid"][1]), badmask=synth.BADMASK)
    H, W = f.shape
    osol = O.Solution(float(g["b0"]), g["coeff"], float(g["d0"]), ob, W, H)
    # sampled output pixels: corners, edges, and seeded uniform positions
    rng = np.random.default_rng(11)
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, 0), (0, H // 2),
           (W - 1, H // 2), (W // 2, H - 1), (W // 2, H // 2)]
    pts += [(int(x), int(y)) for x, y in zip(rng.integers(0, W, N_SAMPLES),
                                             rng.integers(0, H, N_SAMPLES))]
    rb = int(g["r_bad"])
    exp = []
    for x, y in pts:
        o = O.convolve_pixel(f.ref, f.mask_ref, osol, oc.badmask, x, y)
        v = O.variance_pixel(f.var_ref, f.mask_ref, osol, oc.badmask, x, y, oc.var_tile,
                             V2=f.var_sci)
        m = O.mask_pixel(f.mask_ref, osol, oc, x, y, f.mask_sci, rb)
        exp.append((float(f.sci[y, x]) - o, v, m))
    return dict(f=f, g=g, ob=ob, oc=oc, osol=osol, pts=pts, exp=exp)


def _upload(f, dev):
    import torch

    def put(a):
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    return dict(img=put(f.sci), ref=put(f.ref), var_img=put(f.var_sci), var_ref=put(f.var_ref),
                mask_img=put(f.mask_sci), mask_ref=put(f.mask_ref))


def _specs(g, precision):
    b = P.basis_spec(tuple(g["basis_sigma"]), tuple(int(d) for d in g["degrees"]), int(g["h"]),
                     int(g["S"]))
    c = P.config(badmask=synth.BADMASK, grid_nx=int(g["grid"][0]), grid_ny=int(g["grid"][1]),
                 precision=precision)
    return b, c


def _sampled(D, V, M, pts):
    d, v, m = host(D), host(V), host(M)
    return [(float(d[y, x]), float(v[y, x]), int(m[y, x])) for x, y in pts]


def _image_errors(got, exp):
    """max |D - D_oracle| / sigma, max |V - V_oracle| / V_oracle over the samples; masks."""
    de = max(abs(a[0] - b[0]) / np.sqrt(b[1]) for a, b in zip(got, exp))
    ve = max(abs(a[1] - b[1]) / b[1] for a, b in zip(got, exp))
    me = sum(a[2] != b[2] for a, b in zip(got, exp))
    return de, ve, me


def test_full_chip_batch_matches_oracle(dev, chip):
    import torch
    f, g, ob = chip["f"], chip["g"], chip["ob"]
    b, c = _specs(g, P.PREC_F32X2)
    # two copies of the chip in one batch, as in the timed configuration (concurrent chips)
    chips = [_upload(f, dev), _upload(f, dev)]
    batch = P.Batch(chips, [b, b], c, n_streams=4, want_cov=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.run(s)   # captures the graph and runs it
        batch.run(s)   # replays it
        sols = batch.solutions(s)
    H, W = f.shape
    pts9 = [(x, y) for x in (0, W // 2, W - 1) for y in (0, H // 2, H - 1)]
    for i, sol in enumerate(sols):
        cand, stat, chi2 = sol.candidates()
        assert np.array_equal(cand, g["cand"])
        assert np.array_equal(stat, g["status"])
        assert sol.n_iter == int(g["n_iter"]) and sol.n_used == int(g["n_used"])
        assert abs(sol.b0 - float(g["b0"])) <= B0_RTOL * abs(float(g["b0"]))
        assert sol.r_bad == int(g["r_bad"])
        ke = kernel_rel_err(oracle_solution_from_gpu(sol, ob, W, H), chip["osol"], pts9)
        assert ke <= KERNEL_RTOL, ke
        got = _sampled(batch.diff[i], batch.diff_var[i], batch.diff_mask[i], chip["pts"])
        de, ve, me = _image_errors(got, chip["exp"])
        assert de <= IMG_TOL_SIGMA, de
        assert ve <= VAR_RTOL, ve
        assert me == 0
        # quality diagnostics against the oracle's solution and chi^2 statistics
        used = g["chi2"][g["status"] == O.STATUS_USED]
        oq = O.quality(chip["osol"], int(g["n_used"]), float(used.mean()), float(used.std()))
        q = sol.quality()
        for k in ("kernel_sum", "mom_x", "mom_y", "mom_xx", "mom_yy", "deconv_max"):
            assert abs(q[k] - oq[k]) <= 1e-6 * max(1.0, abs(oq[k])), k
        assert abs(q["chi2_mean"] - float(used.mean())) <= 1e-4 * float(used.mean())
        assert q["flags"] == oq["flags"]
        ce = coeff_rel_err(sol.coeff[:g["coeff"].size - 1], g["coeff"][:-1])
        print(f"[coeff] full chip, copy {i}: normwise coefficient error {ce:.3e}, "
              f"kernel {ke:.3e}")
        assert ce <= COEFF_RTOL, ce
    # difference pseudo-matrix = (w1 P_conv + w2 delta) / (w1 + w2) (Sec. 4.4)
    Pc = O.pseudo_matrix(chip["osol"], chip["oc"])
    Pd = batch.cov[0].cpu().numpy()
    assert Pd.shape == Pc.shape
    cidx = (Pc.shape[0] - 1) // 2
    off = np.ones(Pc.shape, bool)
    off[cidx, cidx] = False
    k = float(np.sum(Pd[off] * Pc[off]) / np.sum(Pc[off] ** 2))
    assert 0.0 < k < 1.0
    combo = k * Pc
    combo[cidx, cidx] = 1.0
    assert np.max(np.abs(Pd - combo)) <= 1e-6
    # the two copies agree exactly: every sum behind the pseudo-matrix runs in a fixed order
    assert np.array_equal(batch.cov[1].cpu().numpy(), Pd)
    batch.close()


def _transient_flux(D, V, M, f, radius=20):
    """Aperture sums of the difference image at the injected transients (Sec. 4.5-style
    photometry on D), skipping apertures that touch CONV.BAD or masked pixels."""
    d, v, m = host(D).astype(np.float64), host(V).astype(np.float64), host(M)
    out = []
    yy, xx = np.mgrid[-radius:radius + 1, -radius:radius + 1]
    ap = xx * xx + yy * yy <= radius * radius
    for x0, y0, fl in f.manifest["transients"]:
        xi, yi = int(round(x0)), int(round(y0))
        sl = (slice(yi - radius, yi + radius + 1), slice(xi - radius, xi + radius + 1))
        if (m[sl][ap] & (synth.BADMASK | (1 << 14))).any():
            continue
        out.append((float(d[sl][ap].sum()), float(np.sqrt(v[sl][ap].sum())), float(fl)))
    return np.array(out)


def test_precision_study_full_chip(dev, chip):
    """Every solve precision on the full chip; errors against the oracle are reported (run with
    -s to see the table).  Only the accurate modes are held to the parity tolerances."""
    f, g, ob = chip["f"], chip["g"], chip["ob"]
    t = _upload(f, dev)
    H, W = f.shape
    pts9 = [(x, y) for x in (0, W // 2, W - 1) for y in (0, H // 2, H - 1)]
    a_or = chip["osol"].a.ravel()
    rows = []
    for name, prec in (("f32x2", P.PREC_F32X2), ("bf16x6", P.PREC_BF16X6),
                       ("fp64", P.PREC_FP64), ("fp32", P.PREC_FP32), ("bf16x3", P.PREC_BF16X3),
                       ("tf32", P.PREC_TF32)):
        b, c = _specs(g, prec)
        try:
            D, V, M, cov, sol = P.psfm_subtract(t["img"], t["ref"], t["var_img"], t["var_ref"],
                                                t["mask_img"], t["mask_ref"], b, c)
        except P.PsfmError as e:
            rows.append((name, f"status {e.code}"))
            continue
        cand, stat, _ = sol.candidates()
        same = bool(np.array_equal(stat, g["status"]) and np.array_equal(cand, g["cand"]))
        ke = kernel_rel_err(oracle_solution_from_gpu(sol, ob, W, H), chip["osol"], pts9)
        ce = float(np.max(np.abs(sol.coeff[:a_or.size] - a_or)) / np.max(np.abs(a_or)))
        de, ve, me = _image_errors(_sampled(D, V, M, chip["pts"]), chip["exp"])
        tr = _transient_flux(D, V, M, f)
        ratio = float(np.median(tr[:, 0] / tr[:, 2]))
        zrms = float(np.sqrt(np.mean(((tr[:, 0] - tr[:, 2]) / tr[:, 1]) ** 2)))
        rows.append((name, same, sol.n_used, ke, ce, de, ve, me, len(tr), ratio, zrms))
        if prec in (P.PREC_F32X2, P.PREC_FP64, P.PREC_BF16X6):
            assert same and ke <= KERNEL_RTOL and de <= IMG_TOL_SIGMA and ve <= VAR_RTOL
            assert coeff_rel_err(sol.coeff[:a_or.size], a_or) <= COEFF_RTOL
        assert np.isfinite(ke) and np.isfinite(de)
    print("\nmode    stamps=oracle n_used kernel_L2  coeff_inf  D/sigma   V_rel    mask "
          "n_tr flux_ratio z_rms")
    for r in rows:
        if len(r) == 2:
            print(f"{r[0]:7s} {r[1]}")
        else:
            print(f"{r[0]:7s} {str(r[1]):13s} {r[2]:6d} {r[3]:.3e}  {r[4]:.3e}  {r[5]:.2e}  "
                  f"{r[6]:.2e} {r[7]:4d} {r[8]:4d} {r[9]:.4f}     {r[10]:.3f}")
