"""GPU parity of the dual-kernel subtraction (Eq. 2 with c_i != 0 and the penalty of Sec. 2)
against the FP64 oracle, on a pair whose PSFs are elongated in orthogonal directions: stamp
selection and rejection bit-exact, both realised kernels K1 and K2 = delta - sum c_k B_k within
tolerance, the difference image, its variance and mask, and the pseudo-matrix."""
import numpy as np
import pytest

from gpu_common import IMG_TOL_SIGMA, VAR_RTOL, device, host, oracle_solution_from_gpu, specs, \
    upload
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu

KERNEL_RTOL = 1e-6
B0_RTOL = 1e-9


@pytest.fixture(scope="module")
def dev():
    return device()


def _kernel_err(a, b, pts, realise):
    return max(float(np.linalg.norm(realise(a, x, y) - realise(b, x, y)) /
                     np.linalg.norm(realise(b, x, y))) for x, y in pts)


def _with_masks(f, seed):
    """Masked blocks and scattered bad pixels in both images (different places), so that the
    design columns of the science image see its own mask."""
    rng = np.random.default_rng(seed)
    bit = np.uint16(synth.BADMASK & -synth.BADMASK)
    H, W = f.shape
    for m in (f.mask_ref, f.mask_sci):
        for _ in range(6):
            x, y = rng.integers(0, W - 12), rng.integers(0, H - 12)
            m[y:y + rng.integers(2, 12), x:x + rng.integers(2, 12)] |= bit
        hit = rng.random((H, W)) < 2e-4
        m[hit] |= bit
    return f


@pytest.mark.parametrize("S,norm,masked", [(0, P.NORM_SEPARATE, False),
                                           (1, P.NORM_SEPARATE, False),
                                           (1, P.NORM_SEPARATE, True),
                                           (0, P.NORM_JOINT, True)])
def test_dual_subtract_matches_oracle(dev, S, norm, masked):
    f = synth.elongated_pair(8, 256, 120)
    if masked:
        f = _with_masks(f, 17)
    b, c, ob, oc = specs((0.8, 1.6, 3.0), (4, 2, 2), 8, S, badmask=synth.BADMASK, grid_nx=3,
                         grid_ny=3, precision=P.PREC_F32X2, dual=1, penalty=0.01,
                         norm_mode=norm)
    t = upload(f, dev, pad=5)
    D, V, M, cov, sol = P.psfm_subtract(t["sci"], t["ref"], t["var_sci"], t["var_ref"],
                                        t["mask_sci"], t["mask_ref"], b, c)
    osol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc)
    cand, stat, chi2 = sol.candidates()
    assert np.array_equal(cand, osol.cand) and np.array_equal(stat, osol.status)
    assert sol.n_iter == osol.n_iter and sol.n_used == osol.n_used
    assert abs(sol.b0 - osol.b0) <= B0_RTOL * abs(osol.b0)
    H, W = f.shape
    pts = [(x, y) for x in (0, W // 2, W - 1) for y in (0, H // 2, H - 1)]
    gsol = oracle_solution_from_gpu(sol, ob, W, H)
    assert gsol.dual
    assert _kernel_err(gsol, osol, pts, O.realise_kernel) <= KERNEL_RTOL
    assert _kernel_err(gsol, osol, pts, O.realise_kernel2) <= KERNEL_RTOL
    assert sol.r_bad == O.r_bad(osol)
    oD, oV, oM, oP = O.subtract(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, osol,
                                oc)
    assert np.array_equal(host(M), oM)
    g = host(D).astype(np.float64)
    assert np.all(np.abs(g - oD) <= IMG_TOL_SIGMA * np.sqrt(oV))
    assert np.allclose(host(V), oV, rtol=VAR_RTOL, atol=0)
    assert np.allclose(cov.cpu().numpy(), oP, rtol=0, atol=1e-6)


def _moments(K):
    q = O.kernel_quality(K)
    return q["mom_xx"], q["mom_yy"]


def test_dual_avoids_deconvolution_on_orthogonal_elongations(dev):
    """Reference elongated along x, science along y (Sec. 2: the case the dual kernel is for).
    The single kernel must deconvolve along x (negative second moment, flagged by the quality
    cuts of Sec. 3.7); both dual kernels widen the PSF (positive second moments, K1 along y and
    K2 along x), and the largest normalised residual in the interior drops."""
    f = synth.elongated_pair(8, 256, 120)
    t = upload(f, dev)
    H, W = f.shape
    zmax = {}
    for dual in (0, 1):
        b, c, ob, _ = specs((0.8, 1.6, 3.0), (4, 2, 2), 8, 0, badmask=synth.BADMASK, grid_nx=3,
                            grid_ny=3, precision=P.PREC_F32X2, dual=dual)
        D, V, M, _, sol = P.psfm_subtract(t["sci"], t["ref"], t["var_sci"], t["var_ref"],
                                          t["mask_sci"], t["mask_ref"], b, c, want_cov=False)
        z = (host(D).astype(np.float64) / np.sqrt(host(V).astype(np.float64)))[16:-16, 16:-16]
        zmax[dual] = float(np.abs(z).max())
        q = sol.quality()
        gsol = oracle_solution_from_gpu(sol, ob, W, H)
        if not dual:
            assert q["mom_xx"] < 0 and q["flags"] & P.QUALITY_MOMENT2
            continue
        uu1, vv1 = _moments(O.realise_kernel(gsol, (W - 1) / 2, (H - 1) / 2))
        uu2, vv2 = _moments(O.realise_kernel2(gsol, (W - 1) / 2, (H - 1) / 2))
        assert min(uu1, vv1, uu2, vv2) > 0
        assert vv1 > uu1 and uu2 > vv2
        assert abs(q["mom_xx"] - uu1) <= 1e-6 * abs(uu1) and not q["flags"] & P.QUALITY_MOMENT2
    assert zmax[1] < zmax[0]


def test_dual_requires_double_float(dev):
    f = synth.elongated_pair(9, 128, 40)
    b, c, _, _ = specs((0.8, 1.6), (2, 2), 6, 0, badmask=synth.BADMASK, grid_nx=2, grid_ny=2,
                       precision=P.PREC_FP64, dual=1)
    t = upload(f, dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_solve_kernel(t["sci"], t["ref"], t["var_sci"], t["var_ref"], t["mask_sci"],
                            t["mask_ref"], b, c)
    assert e.value.code == 9


def test_dual_batch_matches_single_calls(dev):
    """The batch API with the dual kernel gives the same results as psfm_subtract per chip."""
    import torch
    fields = [synth.elongated_pair(8, 256, 120), synth.elongated_pair(10, 200, 90)]
    chips = []
    for f in fields:
        t = upload(f, dev)
        chips.append(dict(img=t["sci"], ref=t["ref"], var_img=t["var_sci"], var_ref=t["var_ref"],
                          mask_img=t["mask_sci"], mask_ref=t["mask_ref"]))
    b = P.basis_spec((0.8, 1.6, 3.0), (4, 2, 2), 8, 1)
    c = P.config(badmask=synth.BADMASK, grid_nx=3, grid_ny=3, precision=P.PREC_F32X2, dual=1)
    ref = [P.psfm_subtract(ch["img"], ch["ref"], ch["var_img"], ch["var_ref"], ch["mask_img"],
                           ch["mask_ref"], b, c) for ch in chips]
    batch = P.Batch(chips, [b, b], c, n_streams=2, want_cov=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.run(s)
        batch.run(s)
        sols = batch.solutions(s)
    for i, (D, V, M, cov, sol) in enumerate(ref):
        assert np.array_equal(host(batch.diff[i]), host(D))
        assert np.array_equal(host(batch.diff_var[i]), host(V))
        assert np.array_equal(host(batch.diff_mask[i]), host(M))
        assert np.allclose(batch.cov[i].cpu().numpy(), cov.cpu().numpy(), rtol=1e-12, atol=1e-15)
        assert np.array_equal(sols[i].coeff, sol.coeff) and sols[i].b0 == sol.b0
    batch.close()


def test_dual_unsupported_paths(dev):
    """The workspace-free convolution and the stacks refuse the dual kernel."""
    f = synth.elongated_pair(8, 128, 40)
    t = upload(f, dev)
    b = P.basis_spec((0.8, 1.6), (2, 2), 6, 0)
    c = P.config(badmask=synth.BADMASK, grid_nx=2, grid_ny=2, precision=P.PREC_F32X2, dual=1)
    n = P.basis_size(b) * P.spatial_size(b) * 2
    sol = P.Solution.from_values(1.0, 0.0, np.zeros(n), 1)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_convolve_noalloc(t["ref"], t["var_ref"], t["mask_ref"], b, c, sol, img=t["sci"],
                                var_img=t["var_sci"], mask_img=t["mask_sci"])
    assert e.value.code == 9
    import torch
    src = np.array([[40.0, 40.0, 1000.0], [90.0, 70.0, 2000.0]])
    img = t["sci"].contiguous()
    var = t["var_sci"].contiguous()
    msk = t["mask_sci"].contiguous()
    with pytest.raises(P.PsfmError) as e:
        P.psfm_stack([img], [var], [msk], [src], 6.0, [b], c)
    assert e.value.code == 9
    assert torch.cuda.is_available()
