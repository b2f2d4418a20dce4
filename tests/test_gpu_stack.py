"""GPU parity of the PSF-homogenised stack (psfm_stack through the C ABI, Sec. 5.1-5.2) against
the FP64 oracle: per-input kernel solves against the rendered target, the coverage count and
output mask bit-exact, the weighted image, variance and pseudo-matrix within tolerance."""
import numpy as np
import pytest

from gpu_common import COV_DIFF_ATOL, VAR_RTOL, device, host, kernel_rel_err, \
    oracle_solution_from_gpu, specs
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu

# Realised kernels: as for a single solve (the target is rendered in FP64, source by source in
# the given order, and rounded once on both sides).
KERNEL_RTOL = 1e-6
# Stacked image: 1e-3 of the local noise sigma, as for a single convolved image.
IMG_TOL_SIGMA = 1e-3


@pytest.fixture(scope="module")
def dev():
    return device()


def _warps(seed, n, size, n_stars):
    return synth.skycell_warps(seed, n, size, n_stars, gap_range=(100, 200),
                               block_range=(10, 50), masked_range=(0.03, 0.15))


def _put(a, dev):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_F32X2])
@pytest.mark.parametrize("S", [0, 1])
def test_stack_matches_oracle(dev, prec, S):
    warps, src = _warps(7, 3, 320, 150)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, S, badmask=synth.BADMASK, grid_nx=4,
                         grid_ny=4, precision=prec)
    tf = 1.15 * max(w["fwhm"] for w in warps)
    img, var, msk, cnt, cov, sols = P.psfm_stack(
        [_put(w["image"], dev) for w in warps], [_put(w["var"], dev) for w in warps],
        [_put(w["mask"], dev) for w in warps], [src] * len(warps), tf, [b] * len(warps), c)
    oimg, ovar, omsk, ocnt, ocov, osols = O.stack(warps, src, tf, [ob] * len(warps), oc)
    H, W = oimg.shape
    pts = [(x, y) for x in (0, W // 2, W - 1) for y in (0, H // 2, H - 1)]
    for sol, osol in zip(sols, osols):
        cand, stat, _ = sol.candidates()
        assert np.array_equal(cand, osol.cand)
        assert np.array_equal(stat, osol.status)
        assert sol.n_used == osol.n_used and sol.n_iter == osol.n_iter
        assert kernel_rel_err(oracle_solution_from_gpu(sol, ob, W, H), osol, pts) <= KERNEL_RTOL
        assert sol.r_bad == O.r_bad(osol)
    assert np.array_equal(host(cnt), ocnt)
    assert np.array_equal(host(msk), omsk)
    g_img, g_var = host(img).astype(np.float64), host(var).astype(np.float64)
    cov_ok = ocnt > 0
    assert cov_ok.mean() > 0.5 and (ocnt == len(warps)).any()
    tol = IMG_TOL_SIGMA * np.sqrt(ovar[cov_ok])
    assert np.all(np.abs(g_img[cov_ok] - oimg[cov_ok]) <= tol)
    assert np.allclose(g_var[cov_ok], ovar[cov_ok], rtol=VAR_RTOL, atol=0)
    assert np.all(g_img[~cov_ok] == 0) and np.all(g_var[~cov_ok] == 0)
    assert np.allclose(host(cov), ocov, rtol=0, atol=COV_DIFF_ATOL)


def test_stack_single_input_equals_its_convolution(dev):
    """One input: the stack is that input convolved with its kernel (weights cancel), and its
    variance the propagated variance; pixels without coverage carry the no-data bit."""
    warps, src = _warps(11, 1, 256, 100)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK, grid_nx=3,
                         grid_ny=3, precision=P.PREC_F32X2)
    tf = 1.15 * warps[0]["fwhm"]
    img, var, msk, cnt, cov, sols = P.psfm_stack(
        [_put(warps[0]["image"], dev)], [_put(warps[0]["var"], dev)],
        [_put(warps[0]["mask"], dev)], [src], tf, [b], c)
    osol = oracle_solution_from_gpu(sols[0], ob, 256, 256)
    ref = O.convolve_image(warps[0]["image"], warps[0]["mask"], osol, oc.badmask)
    vref = O.variance_image(warps[0]["var"], warps[0]["mask"], osol, oc.badmask, oc.var_tile)
    ok = host(cnt) == 1
    assert ok.any() and np.array_equal(host(msk) == c.nodata, ~ok)
    g = host(img).astype(np.float64)
    assert np.all(np.abs(g[ok] - ref[ok]) <= IMG_TOL_SIGMA * np.sqrt(vref[ok]))
    assert np.allclose(host(var)[ok], vref[ok], rtol=VAR_RTOL)


def _copies(n, spike=None):
    warps, src = synth.skycell_warps(21, 1, 160, 80, gap_range=(60, 120), block_range=(8, 30),
                                     masked_range=(0.02, 0.08))
    out = []
    for i in range(n):
        w = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in warps[0].items()}
        if spike is not None and i == spike[0]:
            w["image"][spike[2], spike[1]] += spike[3]
        out.append(w)
    return out, src


def _check_planes(got, exp, tol_sigma=IMG_TOL_SIGMA):
    img, var, msk, cnt = [host(t) for t in got]
    oimg, ovar, omsk, ocnt = exp
    assert np.array_equal(cnt, ocnt)
    assert np.array_equal(msk, omsk)
    ok = ocnt > 0
    assert np.all(np.abs(img[ok] - oimg[ok]) <= tol_sigma * np.sqrt(ovar[ok]))
    assert np.allclose(var[ok], ovar[ok], rtol=VAR_RTOL, atol=0)


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_F32X2])
def test_stack_full_spike_matches_oracle(dev, prec):
    """Three copies of a warp, one with a planted spike: the spike's input is rejected around it
    and only there, in both the convolved and the unconvolved stack, as in the oracle."""
    x, y = 80, 80
    warps, src = _copies(3, spike=(1, x, y, 20000.0))
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (2, 2, 2), 8, 0, badmask=synth.BADMASK, grid_nx=2,
                         grid_ny=2, precision=prec)
    tf = 1.15 * warps[0]["fwhm"]
    r = P.psfm_stack_full([_put(w["image"], dev) for w in warps],
                          [_put(w["var"], dev) for w in warps],
                          [_put(w["mask"], dev) for w in warps], [src] * 3, tf, [b] * 3, c)
    o = O.stack_full(warps, src, tf, [ob] * 3, oc)
    assert r["rejected"] == o["rejected"]
    assert r["rejected"][1] > 0 and r["rejected"][0] == 0 and r["rejected"][2] == 0
    _check_planes(r["conv"], o["conv"])
    _check_planes(r["unconv"], o["unconv"])
    assert np.allclose(host(r["cov"]), o["pm"], rtol=0, atol=COV_DIFF_ATOL)


def test_stack_full_uneven_warps_agree_with_oracle(dev):
    """Uneven warps (different PSFs and masks).  Outlier decisions are compared bit for bit;
    a decision may differ only where the oracle's margin |I'_i - m| - n sqrt(V'_i + alpha |m|)
    lies within what the parity tolerances allow (1e-3 sigma on every convolved value that
    enters I'_i and the median m, 2e-5 on V'_i): such pixels are counted as fragile.  Coverage
    may then differ only within r_bad of a fragile pixel, and the stacks agree everywhere else."""
    warps, src = _warps(7, 3, 320, 150)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 1, badmask=synth.BADMASK, grid_nx=4,
                         grid_ny=4, precision=P.PREC_F32X2)
    tf = 1.15 * max(w["fwhm"] for w in warps)
    clip = 5.0
    r = P.psfm_stack_full([_put(w["image"], dev) for w in warps],
                          [_put(w["var"], dev) for w in warps],
                          [_put(w["mask"], dev) for w in warps], [src] * 3, tf, [b] * 3, c,
                          clip_nsigma=clip)
    o = O.stack_full(warps, src, tf, [ob] * 3, oc, clip_nsigma=clip)
    bits = host(r["outliers"]).view(np.uint32)
    # largest local noise among the usable convolved inputs: bounds the error of the median
    sig_max = np.zeros(bits.shape)
    for O1, V1, ok1 in o["pass1"]:
        sig_max = np.maximum(sig_max, np.where(ok1, np.sqrt(np.maximum(V1, 0.0)), 0.0))
    fragile_any = np.zeros(bits.shape, bool)
    n_fragile = 0
    for i, (out, margin, (O1, V1, ok1)) in enumerate(zip(o["outliers"], o["margins"],
                                                          o["pass1"])):
        g = (bits >> i & 1).astype(bool)
        diff = g != out
        tol = 2 * IMG_TOL_SIGMA * sig_max + clip * np.sqrt(np.maximum(V1, 0.0)) * 1e-4
        assert not np.any(diff & ~np.isfinite(margin)), "decision on an untested pixel"
        assert np.all(np.abs(margin[diff]) <= tol[diff]), np.abs(margin[diff]).max()
        n_fragile += int(diff.sum())
        fragile_any |= diff
        assert abs(r["rejected"][i] - o["rejected"][i]) <= int(diff.sum())
    print(f"fragile outlier decisions: {n_fragile} of {bits.size * 3} tests")
    rb = max(O.r_bad(s_) for s_ in o["sols"])
    near = np.zeros_like(fragile_any)
    H, W = near.shape
    for y, x in zip(*np.nonzero(fragile_any)):
        near[max(0, y - rb):y + rb + 1, max(0, x - rb):x + rb + 1] = True
    for key in ("conv", "unconv"):
        img, var, msk, cnt = [host(t) for t in r[key]]
        oimg, ovar, omsk, ocnt = o[key]
        assert np.all((cnt == ocnt) | near), key
        same = (cnt == ocnt) & (ocnt > 0) & ~near
        assert same.sum() >= 0.95 * (ocnt > 0).sum()
        assert np.all(np.abs(img[same] - oimg[same]) <= IMG_TOL_SIGMA * np.sqrt(ovar[same]))
        assert np.allclose(var[same], ovar[same], rtol=VAR_RTOL, atol=0)
