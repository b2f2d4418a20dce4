"""GPU parity of the apply path (psfm_convolve through the C ABI) against the FP64 oracle:
image (Eq. 12), variance (Eq. 13, per-patch kernels), mask (Sec. 3.4) and pseudo-matrix
(Eq. 10-11, Sec. 4.3-4.4), given the same solution on both sides."""
import numpy as np
import pytest

from gpu_common import (COV_ATOL, COV_DIFF_ATOL, IMG_TOL_SIGMA, VAR_RTOL, device, gpu_solution_from_oracle,
                        host, specs, upload)
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


def _random_solution(ob, W, H, seed, b0=1.05, d0=2.5):
    rng = np.random.default_rng(seed)
    nb, ns = len(O.basis_terms(ob)), len(O.spatial_terms(ob.S))
    a = rng.normal(0, 0.05, (nb, ns))
    a[0, 0] = 0.6
    return O.Solution(b0, np.concatenate([a.ravel(), [d0]]), d0, ob, W, H)


def _compare(f, osol, oc, D, V, M, cov, C1=None, C2=None, check_cov=True):
    oD, oV, oM, oP = O.subtract(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, osol,
                                oc, C1=C1, C2=C2)
    sig = np.sqrt(np.maximum(oV, 1e-30))
    err = np.abs(host(D) - oD) / sig
    assert float(err.max()) <= IMG_TOL_SIGMA, float(err.max())
    vrel = np.abs(host(V) - oV) / np.maximum(np.abs(oV), 1e-30)
    assert float(vrel.max()) <= VAR_RTOL, float(vrel.max())
    assert np.array_equal(host(M), oM)
    if check_cov:
        assert cov.shape == oP.shape
        assert float(np.abs(cov.cpu().numpy() - oP).max()) <= COV_DIFF_ATOL
    return float(err.max()), float(vrel.max())


def test_difference_small_field_given_solution(dev):
    f = synth.small_gaussian_field(1)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    rb = O.r_bad(osol, oc.bad_frac)
    t = upload(f, dev, pad=7)
    D, V, M, cov = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c,
                                   gpu_solution_from_oracle(osol, rb), img=t["sci"],
                                   var_img=t["var_sci"], mask_img=t["mask_sci"])
    _compare(f, osol, oc, D, V, M, cov)


@pytest.mark.parametrize("W,H,h,S,deg", [(157, 211, 7, 2, (3, 2, 1)), (64, 65, 3, 1, (2,)),
                                         (300, 97, 12, 3, (4, 2)), (33, 200, 15, 0, (6, 4, 2)),
                                         (101, 130, 24, 1, (2, 1)), (40, 37, 1, 0, (1,)),
                                         (96, 140, 15, 2, (8, 4)), (70, 90, 24, 1, (6,))])
def test_ragged_spatially_varying(dev, W, H, h, S, deg):
    """Odd sizes that leave partial tiles in x and y, every spatial order, h from 1 to the
    largest supported (24).  The last two cases hold more horizontal planes of one Gaussian
    than the image convolution keeps in shared memory at once (9 planes at h = 15, 7 at
    h = 24), so their degrees are processed in two groups."""
    f = synth.small_gaussian_field(W + H, size=H, width=W, n_stars=max(5, W * H // 1500),
                                   bad_col_frac=0.02)
    sig = (0.9, 1.8, 3.1)[:len(deg)]
    b, c, ob, oc = specs(sig, deg, h, S, badmask=synth.BADMASK, cov_grid=3)
    osol = _random_solution(ob, W, H, seed=W)
    rb = O.r_bad(osol, oc.bad_frac)
    t = upload(f, dev)
    D, V, M, cov = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c,
                                   gpu_solution_from_oracle(osol, rb), img=t["sci"],
                                   var_img=t["var_sci"], mask_img=t["mask_sci"])
    _compare(f, osol, oc, D, V, M, cov)
    # convolve-only mode (no science image): K (x) I1 + d0, V', m1 | flags; a caller-chosen
    # r_bad different from the kernel's own is honoured
    rb2 = min(2, h) if rb != min(2, h) else 0
    O2, V2, M2, cov2 = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c,
                                       gpu_solution_from_oracle(osol, rb2))
    oO = O.convolve_image(f.ref, f.mask_ref, osol, oc.badmask)
    oV = O.variance_image(f.var_ref, f.mask_ref, osol, oc.badmask, oc.var_tile)
    oM = O.mask_image(f.mask_ref, osol, oc, rb=rb2)
    sig_o = np.sqrt(np.maximum(oV + f.var_ref, 1e-30))
    assert float((np.abs(host(O2) - oO) / sig_o).max()) <= IMG_TOL_SIGMA
    assert np.array_equal(host(M2), oM)
    assert float(np.abs(cov2.cpu().numpy() - O.pseudo_matrix(osol, oc)).max()) <= COV_ATOL


def test_correlated_input_noise(dev):
    """A non-white input pseudo-matrix changes the per-patch covariance factor (Sec. 4.3-4.4)
    and the output pseudo-matrix."""
    import torch
    f = synth.small_gaussian_field(3, size=128, n_stars=20)
    b, c, ob, oc = specs((0.8, 2.0), (2, 2), 6, 1, badmask=synth.BADMASK, cov_grid=2)
    osol = _random_solution(ob, 128, 128, seed=5)
    C1 = np.array([[0.0, 0.05, 0.0], [0.1, 1.0, 0.1], [0.0, 0.05, 0.0]])
    C2 = np.zeros((5, 5))
    C2[2, 2], C2[2, 1], C2[2, 3] = 1.0, 0.2, 0.2
    t = upload(f, dev)
    D, V, M, cov = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c,
                                   gpu_solution_from_oracle(osol, 1), img=t["sci"],
                                   var_img=t["var_sci"], mask_img=t["mask_sci"],
                                   cov_ref=torch.from_numpy(C1).to(dev),
                                   cov_img=torch.from_numpy(C2).to(dev))
    _compare(f, osol, oc, D, V, M, cov, C1=C1, C2=C2)


def test_identity_kernel(dev):
    """b0 = 1, all other terms 0: the convolved image is I1 (masked pixels 0), V' = V1."""
    f = synth.small_gaussian_field(4, size=96, n_stars=10)
    b, c, ob, oc = specs((1.0, 2.0), (2, 2), 5, 1, badmask=synth.BADMASK)
    n = P.basis_size(b) * P.spatial_size(b)
    sol = P.Solution.from_values(1.0, 0.0, np.zeros(n), 0)
    t = upload(f, dev)
    O_, V_, M_, cov = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c, sol)
    ok = (f.mask_ref & synth.BADMASK) == 0
    assert np.array_equal(host(O_)[ok], f.ref[ok])
    assert np.allclose(host(V_)[ok], f.var_ref[ok], rtol=1e-6)
    cc = cov.cpu().numpy()
    assert cc[cc.shape[0] // 2, cc.shape[0] // 2] == 1.0 and abs(cc.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("ty", [64, 128])
@pytest.mark.parametrize("W,H,h,S,deg", [(157, 211, 7, 2, (3, 2, 1)), (96, 300, 15, 2, (8, 4)),
                                         (70, 90, 24, 1, (6,)), (45, 260, 1, 3, (2,))])
def test_every_launch_shape_matches_oracle(dev, ty, W, H, h, S, deg):
    """Both tile heights the autotuner may choose (64 and 128 output rows), forced through the
    tuning table, give the same image as the oracle on ragged sizes."""
    f = synth.small_gaussian_field(W * H, size=H, width=W, n_stars=max(5, W * H // 1500),
                                   bad_col_frac=0.02)
    sig = (0.9, 1.8, 3.1)[:len(deg)]
    b, c, ob, oc = specs(sig, deg, h, S, badmask=synth.BADMASK, cov_grid=3)
    osol = _random_solution(ob, W, H, seed=H)
    rb = O.r_bad(osol, oc.bad_frac)
    t = upload(f, dev, pad=5)
    P.tune_clear()
    P.tune_set({"half_width": h, "spatial_order": S, "degree": list(deg), "tile_rows": ty,
                "plane_chunk": 4})
    try:
        D, V, M, cov = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c,
                                       gpu_solution_from_oracle(osol, rb), img=t["sci"],
                                       var_img=t["var_sci"], mask_img=t["mask_sci"])
    finally:
        P.tune_clear()
    _compare(f, osol, oc, D, V, M, cov)


def test_autotuner_picks_a_legal_shape(dev):
    """psfm_tune_conv times the legal shapes of a basis class and stores the fastest; the
    convolution then runs with it and still matches the oracle."""
    W, H = 400, 300
    f = synth.small_gaussian_field(3, size=H, width=W, n_stars=100)
    b, c, ob, oc = specs((0.8, 1.6, 3.2), (6, 4, 2), 15, 2, badmask=synth.BADMASK)
    P.tune_clear()
    e = P.tune_conv(b, W, H)
    assert e["tile_rows"] in (64, 128) and e["plane_chunk"] == 4 and e["ms"] > 0
    assert P.tune_entries() == [e]
    osol = _random_solution(ob, W, H, seed=5)
    rb = O.r_bad(osol, oc.bad_frac)
    t = upload(f, dev)
    try:
        D, V, M, cov = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c,
                                       gpu_solution_from_oracle(osol, rb), img=t["sci"],
                                       var_img=t["var_sci"], mask_img=t["mask_sci"])
    finally:
        P.tune_clear()
    _compare(f, osol, oc, D, V, M, cov)
