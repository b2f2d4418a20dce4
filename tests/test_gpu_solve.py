"""GPU parity of the kernel solve (psfm_solve_kernel / psfm_subtract through the C ABI)
against the FP64 oracle: stamp candidates, rejection decisions and statuses bit-exact;
normalisation, coefficients and realised kernels within tolerance; error codes."""
import numpy as np
import pytest

from gpu_common import (IMG_TOL_SIGMA, VAR_RTOL, coeff_rel_err, device, host, kernel_rel_err,
                        oracle_solution_from_gpu, specs, upload)
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu

# Realised-kernel agreement (normwise, at sample points) and b0: the stamp design blocks are
# FP32 on the GPU, so the solution differs from the FP64 oracle by the FP32 perturbation of
# the normal equations amplified by their condition number.
KERNEL_RTOL = 1e-6
B0_RTOL = 1e-9
# Kernel coefficients (normwise relative): the tolerance the method is held to.
COEFF_RTOL = 1e-6
# The accurate solve modes: FP64; double-float (FP32 pairs) on the FP32 pipes; double-float
# design with the Gram on the tensor cores from exact BF16 split products.
PRECISIONS = [P.PREC_FP64, P.PREC_F32X2, P.PREC_BF16X6]


@pytest.fixture(scope="module")
def dev():
    return device()


def _check_solution(sol, osol, ob, W, H):
    cand, stat, chi2 = sol.candidates()
    assert np.array_equal(cand, osol.cand)
    assert np.array_equal(stat, osol.status)
    assert sol.n_iter == osol.n_iter and sol.n_used == osol.n_used
    both = ~np.isnan(osol.chi2)
    assert np.array_equal(np.isnan(chi2), np.isnan(osol.chi2))
    assert np.allclose(chi2[both], osol.chi2[both], rtol=1e-4)
    assert abs(sol.b0 - osol.b0) <= B0_RTOL * abs(osol.b0)
    gsol = oracle_solution_from_gpu(sol, ob, W, H)
    pts = [(x, y) for x in (0, W // 2, W - 1) for y in (0, H // 2, H - 1)]
    ke = kernel_rel_err(gsol, osol, pts)
    assert ke <= KERNEL_RTOL, ke
    assert sol.r_bad == O.r_bad(osol)
    # quality diagnostics (Sec. 3.7) of the GPU solution, recomputed by the oracle
    q = sol.quality()
    oq = O.quality(gsol, sol.n_used, sol.chi2_mean, sol.chi2_rms)
    for k in ("kernel_sum", "mom_x", "mom_y", "mom_xx", "mom_yy", "mom_xy", "deconv_max"):
        assert abs(q[k] - oq[k]) <= 1e-10 * max(1.0, abs(oq[k])), k
    assert q["flags"] == oq["flags"]
    ce = coeff_rel_err(sol.coeff[:osol.a.size], osol.a.ravel())
    print(f"[coeff] normwise coefficient error {ce:.3e}, realised-kernel error {ke:.3e}")
    assert ce <= COEFF_RTOL, ce
    return ke, ce


@pytest.mark.parametrize("prec", PRECISIONS)
def test_solve_small_field_with_extractor(dev, prec):
    f = synth.small_gaussian_field(1)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK, precision=prec)
    t = upload(f, dev, pad=3)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b, c)
    ocand, med = O.extract_candidates(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref,
                                      f.mask_sci, ob, oc)
    assert np.float32(sol.median) == med
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc,
                          ocand)
    _check_solution(sol, osol, ob, 512, 512)


def test_wide_basis_in_split_product_mode_takes_the_double_float_gram(dev):
    """A basis with more than 64 augmented columns (degrees 6, 6, 2: 62 terms, 65 columns) in
    PREC_BF16X6 solves with the double-float Gram: the same kernels as PREC_F32X2, so the same
    bits."""
    f = synth.small_gaussian_field(1)
    t = upload(f, dev, pad=3)
    sols = []
    for prec in (P.PREC_BF16X6, P.PREC_F32X2):
        b, c, ob, oc = specs((0.7, 1.5, 3.0), (6, 6, 2), 10, 0, badmask=synth.BADMASK,
                             precision=prec)
        assert P.basis_size(b) == 62
        sols.append(P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"],
                                        t["mask_sci"], t["mask_ref"], b, c))
    a, f32 = sols
    assert np.array_equal(a.coeff, f32.coeff)
    assert a.b0 == f32.b0 and a.n_iter == f32.n_iter and a.n_used == f32.n_used


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("mode", ["separate", "joint"])
def test_solve_spatial_order_2_with_rejection(dev, mode, prec):
    """Spatially varying PSF, S = 2; a cosmic ray planted in the science image makes the
    rejection loop remove and replace a stamp."""
    f = synth.small_gaussian_field(9, size=384, n_stars=260, fwhm_ref=3.5, fwhm_sci=5.0)
    sci = f.sci.copy()
    b, c, ob, oc = specs((0.8, 1.6, 3.0), (4, 2, 2), 8, 2, badmask=synth.BADMASK, grid_nx=5,
                         grid_ny=4, norm_mode=P.NORM_JOINT if mode == "joint" else P.NORM_SEPARATE,
                         precision=prec)
    ocand, _ = O.extract_candidates(f.ref, sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    hit = next(r for r in range(ocand.shape[0]) if ocand[r, 1, 0] >= 0)
    x, y = ocand[hit, 0]
    sci[y + 2, x - 1] += 5000.0
    f.sci = sci
    t = upload(f, dev)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b, c)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    assert osol.status[hit, 0] == O.STATUS_REJECTED
    _check_solution(sol, osol, ob, 384, 384)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_caller_stamps(dev, prec):
    f = synth.small_gaussian_field(2, size=256, n_stars=80)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (2, 2, 2), 7, 1, badmask=synth.BADMASK, precision=prec)
    ocand, _ = O.extract_candidates(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci,
                                    ob, O.Config(grid_nx=4, grid_ny=4, badmask=synth.BADMASK))
    stamps = [tuple(xy) for xy in ocand[:, 0] if xy[0] >= 0]
    t = upload(f, dev)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b, c, stamps=stamps)
    cand = np.array([[s] for s in stamps], np.int32)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc, cand)
    _check_solution(sol, osol, ob, 256, 256)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_solve_largest_half_width(dev, prec):
    """The largest supported kernel half width (h = 24, 49 x 49 kernel) with the extractor."""
    f = synth.small_gaussian_field(21, size=400, n_stars=120, bad_col_frac=0.002)
    b, c, ob, oc = specs((1.0, 2.5), (2, 1), 24, 1, badmask=synth.BADMASK, grid_nx=2,
                         grid_ny=2, precision=prec)
    t = upload(f, dev)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b, c)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    _check_solution(sol, osol, ob, 400, 400)


def test_half_bright_field(dev):
    """Half of the field on a much brighter background: most of that half lies above the
    detection threshold (the median sits between the halves), so the detection lists a large
    share of the image; stamps and the solution still match the oracle."""
    f = synth.small_gaussian_field(5, size=256, n_stars=80, bad_col_frac=0.005)
    for a in (f.ref, f.sci, f.var_ref, f.var_sci):
        a[:, 128:] += 4000.0
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (2, 2, 1), 8, 1, badmask=synth.BADMASK, grid_nx=3,
                         grid_ny=3, precision=P.PREC_F32X2)
    t = upload(f, dev)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b, c)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    _check_solution(sol, osol, ob, 256, 256)


def test_subtract_end_to_end_small(dev):
    f = synth.small_gaussian_field(1)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK)
    t = upload(f, dev)
    D, V, M, cov, sol = P.psfm_subtract(t["sci"], t["ref"], t["var_sci"], t["var_ref"],
                                        t["mask_sci"], t["mask_ref"], b, c)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    _check_solution(sol, osol, ob, 512, 512)
    oD, oV, oM, oP = O.subtract(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, osol,
                                oc)
    sig = np.sqrt(oV)
    assert float((np.abs(host(D) - oD) / sig).max()) <= IMG_TOL_SIGMA
    assert float((np.abs(host(V) - oV) / oV).max()) <= VAR_RTOL
    assert np.array_equal(host(M), oM)
    assert float(np.abs(cov.cpu().numpy() - oP).max()) <= 1e-6


def test_too_few_stamps_and_bad_arguments(dev):
    f = synth.small_gaussian_field(3, size=128, n_stars=2)
    b, c, ob, oc = specs((1.0,), (2,), 5, 0, badmask=synth.BADMASK)
    t = upload(f, dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                            t["mask_ref"], b, c)
    assert e.value.code == 2
    with pytest.raises(P.PsfmError) as e:
        P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                            t["mask_ref"], b, c, stamps=[(500, 5), (6, 6), (7, 7)])
    assert e.value.code == 1
    # fully masked image: no background pixels
    f.mask_ref[:] = synth.MASK_BAD
    t = upload(f, dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                            t["mask_ref"], b, c)
    assert e.value.code == 2
    # the library still works after the errors
    f2 = synth.small_gaussian_field(1)
    b2, c2, ob2, oc2 = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK)
    t2 = upload(f2, dev)
    sol = P.psfm_solve_kernel(t2["sci"], t2["ref"], t2["var_sci"], t2["var_ref"], t2["mask_sci"],
                              t2["mask_ref"], b2, c2)
    assert sol.n_used >= 3


@pytest.mark.parametrize("prec", PRECISIONS)
def test_duplicate_gaussian_basis_is_singular(dev, prec):
    """A basis that lists the same Gaussian twice has duplicate design columns: the Cholesky
    meets a pivot inside the singular band and the solve returns PSFM_ERR_SINGULAR, as the
    oracle reports; the library works afterwards."""
    f = synth.small_gaussian_field(1, size=192, n_stars=60)
    b, c, ob, oc = specs((1.5, 1.5), (1, 1), 6, 0, badmask=synth.BADMASK, grid_nx=3, grid_ny=3,
                         max_iter=1, precision=prec)
    with pytest.raises(O.OracleError, match="singular"):
        O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    t = upload(f, dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                            t["mask_ref"], b, c)
    assert e.value.code == 3
    b2, c2, ob2, oc2 = specs((1.5, 2.5), (1, 1), 6, 0, badmask=synth.BADMASK, grid_nx=3,
                             grid_ny=3, max_iter=1, precision=prec)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b2, c2)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob2, oc2)
    _check_solution(sol, osol, ob2, 192, 192)


def test_nonfinite_unmasked_pixel(dev):
    f = synth.small_gaussian_field(1)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK)
    f.sci[100, 100] = np.nan
    f.mask_sci[100, 100] = 0
    f.mask_ref[100, 100] = 0
    t = upload(f, dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                            t["mask_ref"], b, c)
    assert e.value.code == 4


def test_fp32_design_mode_reports_its_error(dev):
    """PREC_FP32 (FP32 design blocks) is a fast approximate mode: it must keep the stamp
    selection and b0, while its kernel error against the FP64 definition is only reported
    (it is set by the conditioning of the normal equations times FP32 rounding)."""
    f = synth.small_gaussian_field(1)
    b, c, ob, oc = specs((0.7, 1.5, 3.0), (4, 2, 2), 10, 0, badmask=synth.BADMASK,
                         precision=P.PREC_FP32)
    t = upload(f, dev)
    sol = P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                              t["mask_ref"], b, c)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    cand, stat, _ = sol.candidates()
    assert np.array_equal(cand, osol.cand)
    assert abs(sol.b0 - osol.b0) <= B0_RTOL * abs(osol.b0)
    gsol = oracle_solution_from_gpu(sol, ob, 512, 512)
    ke = kernel_rel_err(gsol, osol, [(256, 256), (0, 0), (511, 511)])
    print(f"PREC_FP32 realised-kernel error vs FP64 oracle: {ke:.3e}")
    assert ke < 0.1
