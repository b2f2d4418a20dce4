"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, a library
routine in a special case, brute force on tiny inputs, an invariant, or a statistical
property of the paper's noise model (Sec. 4.5).  None of them needs a GPU.
"""
import math

import numpy as np
import pytest
from scipy import signal

from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import synth


def gaussian_density(h, sigma):
    u = np.arange(-h, h + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    return np.exp(-(U * U + V * V) / (2 * sigma * sigma)) / (2 * math.pi * sigma * sigma)


def isolated_stars(W, H, spacing, margin, seed=0, flux=(2e4, 8e4)):
    rng = np.random.default_rng(seed)
    out = []
    for y in range(margin, H - margin + 1, spacing):
        for x in range(margin, W - margin + 1, spacing):
            out.append((x + rng.uniform(-0.5, 0.5), y + rng.uniform(-0.5, 0.5),
                        rng.uniform(*flux)))
    return out


# ---------------------------------------------------------------- basis (Eq. 7, Sec. 2)

@pytest.mark.parametrize("degrees,nb", [((4, 2, 2), 27), ((6, 4, 2), 49), ((8, 4, 2), 66)])
def test_basis_count_zero_sum_and_norm(degrees, nb):
    basis = O.Basis((0.8, 1.6, 3.2), degrees, 12)
    B, s, psi = O.basis_kernels(basis)
    assert B.shape == (nb, 25, 25)
    assert np.max(np.abs(B.reshape(nb, -1).sum(1))) < 1e-13          # zero sum, every term
    h = basis.h
    for k, (g, p, q) in enumerate(O.basis_terms(basis)):
        Bp = B[k].copy()
        Bp[h, h] += s[k]
        assert abs(np.sum(Bp * Bp) - 1.0) < 1e-12                     # unit L2 before zero-summing
        # parity of u^p v^q: mirror in u flips sign for odd p, mirror in v for odd q
        assert np.allclose(Bp[:, ::-1], (-1) ** p * Bp, atol=1e-15)
        assert np.allclose(Bp[::-1, :], (-1) ** q * Bp, atol=1e-15)
        if p % 2 or q % 2:
            assert s[k] == 0.0
        else:
            assert s[k] > 0.0
        # the Gaussian decays (garbled sign of Eq. 7 read as exp(-r^2/2s^2))
        assert abs(Bp[0, 0]) < abs(Bp).max()


def test_spatial_terms_order():
    assert O.spatial_terms(0) == [(0, 0)]
    assert O.spatial_terms(2) == [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 0)]
    assert len(O.spatial_terms(3)) == 10
    g = O.spatial_values(0, 99, 100, 100, 1)
    assert np.allclose(g, [1.0, 1.0, -1.0])            # xt = -1, yt = +1


# ---------------------------------------------------------------- Eq. 12, direct sums

def test_direct_conv_matches_scipy():
    rng = np.random.default_rng(3)
    img = rng.normal(size=(37, 53))
    K = rng.normal(size=(7, 7))                         # asymmetric: catches a flipped kernel
    ref = signal.convolve2d(img, K, mode="same", boundary="fill")
    assert np.allclose(O.direct_conv2d(img, K), ref, atol=1e-12)
    for x, y in [(0, 0), (52, 36), (10, 20), (3, 35)]:
        assert abs(O.conv_pixel(img, K, x, y) - ref[y, x]) < 1e-12


def test_design_matrix_columns_are_library_convolutions():
    f = synth.small_gaussian_field(5, size=96, n_stars=12, bad_col_frac=0.03)
    basis = O.Basis((0.7, 1.5), (2, 1), 5, 1)
    cfg = O.Config(badmask=synth.BADMASK, stamp_half=4)
    B, _, _ = O.basis_kernels(basis)
    st = O.stamp_data(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, 40, 51,
                      basis, cfg)
    R = np.where(f.mask_ref & synth.BADMASK, 0.0, f.ref.astype(np.float64))
    for k in range(B.shape[0]):
        full = signal.convolve2d(R, B[k], mode="same")
        ref = full[51 - 4:51 + 5, 40 - 4:40 + 5].ravel()
        assert np.allclose(st.C[:, k], ref, rtol=1e-12, atol=1e-9)
    assert np.allclose(st.g, [1, 2 * 51 / 95 - 1, 2 * 40 / 95 - 1])


def test_spatially_varying_convolution_is_per_pixel_library_convolution():
    f = synth.small_gaussian_field(6, size=64, n_stars=10, bad_col_frac=0.03)
    basis = O.Basis((0.9, 2.0), (2, 1), 4, 2)
    nb, ns = len(O.basis_terms(basis)), len(O.spatial_terms(2))
    rng = np.random.default_rng(1)
    sol = O.Solution(1.1, np.concatenate([rng.normal(0, 0.05, nb * ns), [3.0]]), 3.0, basis, 64, 64)
    out = O.convolve_image(f.ref, f.mask_ref, sol, synth.BADMASK)
    R = np.where(f.mask_ref & synth.BADMASK, 0.0, f.ref.astype(np.float64))
    for x, y in [(0, 0), (63, 63), (31, 7), (12, 50), (60, 2)]:
        K = O.realise_kernel(sol, x, y)
        lib = signal.convolve2d(R, K, mode="same")[y, x] + 3.0
        assert abs(out[y, x] - lib) < 1e-8 * max(1.0, abs(lib))
        assert abs(O.convolve_pixel(f.ref, f.mask_ref, sol, synth.BADMASK, x, y) - lib) < 1e-8 * abs(lib)


# ---------------------------------------------------------------- solve (Eq. 3-6, Sec. 3.2)

def test_two_gaussians_recover_the_difference_gaussian():
    """Matching two Gaussian PSFs sigma1 < sigma2 gives K = f G(sqrt(sigma2^2 - sigma1^2))."""
    s1, s2 = synth.fwhm_to_sigma(4.0), synth.fwhm_to_sigma(5.5)
    sk = math.sqrt(s2 * s2 - s1 * s1)
    f = 1.37
    stars = isolated_stars(200, 200, 60, 40)
    fld = synth.gaussian_pair(200, 200, stars, s1, s2, flux_ratio=f, sky=0.0)
    basis = O.Basis((sk, 0.8, 3.0), (0, 2, 2), 10, 0)
    h = basis.h
    expect = f * gaussian_density(h, sk)
    cand = np.array([[[int(round(x)), int(round(y))]] for x, y, _ in stars], np.int32)
    for mode in ("separate", "joint"):
        cfg = O.Config(norm_mode=mode, max_iter=1, badmask=synth.BADMASK)
        sol = O.solve_kernel(fld.ref, fld.sci, fld.var_ref, fld.var_sci, fld.mask_ref,
                             fld.mask_sci, basis, cfg, cand)
        K = O.realise_kernel(sol, 100, 100)
        # truncation at h = 10 leaves ~1e-9 of the Gaussian's mass outside the kernel; the
        # float32 rounding of the rendered images (~6e-8 relative) sets the floor here
        assert np.max(np.abs(K - expect)) / expect.max() < 1e-5, mode
        assert abs(sol.b0 - f) < 1e-6
        assert np.max(np.abs(sol.a[1:])) < 1e-5
        assert abs(sol.d0) < 1e-5


def test_kernel_sum_is_the_flux_ratio():
    s1, s2 = 1.5, 2.3
    stars = isolated_stars(180, 180, 60, 30, seed=2)
    for f in (0.6, 2.5):
        fld = synth.gaussian_pair(180, 180, stars, s1, s2, flux_ratio=f, sky=100.0)
        cand = np.array([[[int(round(x)), int(round(y))]] for x, y, _ in stars], np.int32)
        # SEPARATE (Sec. 3.2) fixes b0 from footprint sums: exact for any basis.  JOINT fits b0
        # with the kernel terms, exact only when the basis spans the matching kernel (otherwise
        # the even terms trade against b0: the ring residuals Sec. 3.2 warns about).
        for mode, basis in (("separate", O.Basis((0.7, 1.5, 3.0), (4, 2, 2), 10, 0)),
                            ("joint", O.Basis((math.sqrt(s2 * s2 - s1 * s1), 0.7), (0, 2), 10, 0))):
            cfg = O.Config(norm_mode=mode, max_iter=1, badmask=synth.BADMASK)
            sol = O.solve_kernel(fld.ref, fld.sci, fld.var_ref, fld.var_sci, fld.mask_ref,
                                 fld.mask_sci, basis, cfg, cand)
            K = O.realise_kernel(sol, 90, 90)
            assert abs(K.sum() - sol.b0) < 1e-12 * f
            assert abs(sol.b0 - f) < 1e-6 * f, (mode, sol.b0)
            # background: sky * f - f * sky = 0 differential
            assert abs(sol.d0) < 1e-4


def test_identity_when_images_are_equal():
    fld = synth.small_gaussian_field(7, size=160, n_stars=40)
    basis = O.Basis((0.7, 1.5, 3.0), (4, 2, 2), 8, 1)
    cfg = O.Config(grid_nx=3, grid_ny=3, badmask=synth.BADMASK, max_iter=2)
    sol = O.solve_kernel(fld.ref, fld.ref, fld.var_ref, fld.var_ref, fld.mask_ref, fld.mask_ref,
                         basis, cfg)
    assert abs(sol.b0 - 1.0) < 1e-12
    assert np.max(np.abs(sol.a)) < 1e-10
    assert abs(sol.d0) < 1e-9
    D = O.convolve_image(fld.ref, fld.mask_ref, sol, cfg.badmask, fld.ref)
    ok = (fld.mask_ref & cfg.badmask) == 0
    assert np.max(np.abs(D[ok])) < 1e-6
    Vp = O.variance_image(fld.var_ref, fld.mask_ref, sol, cfg.badmask, 64)
    assert np.allclose(Vp[ok], fld.var_ref[ok], rtol=1e-9)
    assert O.r_bad(sol) == 0
    P = O.pseudo_matrix(sol, cfg)
    c = P.shape[0] // 2
    assert abs(P[c, c] - 1) < 1e-12 and abs(P.sum() - 1.0) < 1e-9


def _tiny_problem(seed):
    fld = synth.small_gaussian_field(seed, size=80, n_stars=30, fwhm_ref=2.5, fwhm_sci=3.2)
    basis = O.Basis((1.0,), (2,), 3, 1)
    cfg = O.Config(stamp_half=2, badmask=synth.BADMASK, max_iter=1)
    rng = np.random.default_rng(seed)
    pts = [(int(x), int(y)) for x, y in zip(rng.integers(6, 74, 10), rng.integers(6, 74, 10))]
    return fld, basis, cfg, pts


def test_normal_solve_singular_band():
    """The normal-equation solve against closed forms: for M = [[1, 1 - e], [1 - e, 1]] the
    second Cholesky pivot is 1 - (1 - e)^2 ~ 2e.  Above the singular band the solution is the
    exact inverse applied to v; inside it (and for an exact duplicate) the system is singular;
    an indefinite matrix beyond the band is solved by LU as the plain inverse."""
    v = np.array([1.0, 2.0])
    for e in (1e-3, 1e-8):
        M = np.array([[1.0, 1.0 - e], [1.0 - e, 1.0]])
        det = 1.0 - (1.0 - e) ** 2
        exact = np.array([v[0] - (1 - e) * v[1], v[1] - (1 - e) * v[0]]) / det
        assert np.allclose(O.solve_normal(M, v), exact, rtol=1e-6)
    for e in (1e-13, 0.0):
        M = np.array([[1.0, 1.0 - e], [1.0 - e, 1.0]])
        with pytest.raises(O.OracleError, match="singular"):
            O.solve_normal(M, v)
    M = np.array([[1.0, 2.0], [2.0, 1.0]])   # eigenvalues 3 and -1
    assert np.allclose(O.solve_normal(M, v), np.array([1.0, 0.0]), atol=1e-15)
    assert O._first_bad_pivot(np.array([[4.0, 2.0], [2.0, 3.0]])) is None


def test_duplicate_gaussian_basis_is_singular():
    """A basis that lists the same Gaussian twice has duplicate design columns: the normal
    equations are singular and the solve reports it."""
    f = synth.small_gaussian_field(1, size=192, n_stars=60)
    basis = O.Basis((1.5, 1.5), (1, 1), 6, 0)
    cfg = O.Config(grid_nx=3, grid_ny=3, badmask=synth.BADMASK, max_iter=1)
    with pytest.raises(O.OracleError, match="singular"):
        O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, basis, cfg)
    ok = O.Basis((1.5, 2.5), (1, 1), 6, 0)
    sol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ok, cfg)
    assert np.all(np.isfinite(sol.a))


def test_joint_solve_equals_svd_least_squares():
    """Gram + Cholesky equals an SVD least-squares solve of the stacked weighted design."""
    fld, basis, cfg, pts = _tiny_problem(11)
    cfg.norm_mode = "joint"
    sts = [O.stamp_data(fld.ref, fld.sci, fld.var_ref, fld.var_sci, fld.mask_ref, fld.mask_sci,
                        x, y, basis, cfg) for x, y in pts]
    b0, a, d0 = O.solve_from_stamps(sts, basis, cfg)
    rows, rhs = [], []
    for st in sts:
        for p in range(st.C.shape[0]):
            if not st.ok[p]:
                continue
            wt = 1.0 / math.sqrt(st.var[p])
            row = [st.R[p]] + [st.C[p, k] * st.g[s] for k in range(st.C.shape[1])
                               for s in range(len(st.g))] + [1.0]
            rows.append(np.array(row) * wt)
            rhs.append(st.I2[p] * wt)
    x, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    got = np.concatenate([[b0], a, [d0]])
    assert np.allclose(got, x, rtol=1e-7, atol=1e-9 * np.abs(x).max())


def test_separate_normalisation_is_unweighted_footprint_regression():
    fld, basis, cfg, pts = _tiny_problem(12)
    sts = [O.stamp_data(fld.ref, fld.sci, fld.var_ref, fld.var_sci, fld.mask_ref, fld.mask_sci,
                        x, y, basis, cfg) for x, y in pts]
    b0, a, d0 = O.solve_from_stamps(sts, basis, cfg)
    # brute force: footprint sums recomputed directly from the images
    n = 2 * (2 + 3) + 1
    F1, F2, N = [], [], []
    bad = ((fld.mask_ref | fld.mask_sci) & synth.BADMASK) != 0
    R = np.where(fld.mask_ref & synth.BADMASK, 0.0, fld.ref.astype(np.float64))
    for x, y in pts:
        sl = (slice(max(0, y - 5), y + 6), slice(max(0, x - 5), x + 6))
        good = ~bad[sl]
        F1.append(R[sl][good].sum())
        F2.append(fld.sci[sl].astype(np.float64)[good].sum())
        N.append(good.sum())
    (bb, dd), *_ = np.linalg.lstsq(np.stack([F1, N], 1), np.array(F2), rcond=None)
    assert abs(b0 - bb) < 1e-10 * abs(bb) and abs(d0 - dd) < 1e-7 * max(1, abs(dd))
    # the kernel terms: SVD least squares on the reduced problem
    rows, rhs = [], []
    for st in sts:
        for p in np.nonzero(st.ok)[0]:
            wt = 1.0 / math.sqrt(st.var[p])
            rows.append(np.outer(st.C[p], st.g).ravel() * wt)
            rhs.append((st.I2[p] - b0 * st.R[p] - d0) * wt)
    x, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    assert np.allclose(a, x, rtol=1e-7, atol=1e-9 * np.abs(x).max())


# ---------------------------------------------------------------- variance, covariance (Sec. 4)

def _fixed_solution(W, H, S=0, seed=0):
    basis = O.Basis((0.9, 1.8, 3.0), (2, 2, 0), 7, S)
    nb, ns = len(O.basis_terms(basis)), len(O.spatial_terms(S))
    rng = np.random.default_rng(seed)
    a = rng.normal(0, 0.1, (nb, ns))
    a[0, 0] = 0.8
    return O.Solution(1.0, np.concatenate([a.ravel(), [0.0]]), 0.0, basis, W, H)


def test_variance_of_constant_kernel_is_sigma2_sum_k2():
    W = H = 96
    sol = _fixed_solution(W, H)
    K = O.realise_kernel(sol, 0, 0)
    V = np.full((H, W), 4.0, np.float32)
    Vp = O.variance_image(V, np.zeros((H, W), np.uint16), sol, 0xFF, 64)
    h = sol.basis.h
    assert np.allclose(Vp[h:-h, h:-h], 4.0 * np.sum(K * K), rtol=1e-12)
    # empirical: convolved white noise of variance 4 has variance 4 sum K^2 (Eq. 13)
    noise = synth.white_noise(9, 600, 600, 2.0)
    out = O.direct_conv2d(noise, K)[h:-h, h:-h]
    expect = 4.0 * np.sum(K * K)
    # correlated samples: ~(600/ (2w))^2 independent patches, bound generously
    assert abs(out.var() / expect - 1.0) < 0.05


def test_pseudo_matrix_of_white_noise():
    sol = _fixed_solution(64, 64)
    K = O.realise_kernel(sol, 0, 0)
    P = O.pseudo_conv(K, np.ones((1, 1)))
    assert np.allclose(P, signal.correlate2d(K, K, mode="full"), atol=1e-14)
    # with a correlated input, K * C * K is a convolution followed by a correlation
    rng = np.random.default_rng(4)
    C = rng.normal(size=(5, 5))
    C = C + C[::-1, ::-1]
    P2 = O.pseudo_conv(K, C)
    ref = signal.correlate2d(signal.convolve2d(K, C, mode="full"), K, mode="full")
    assert P2.shape == (2 * K.shape[0] + 5 - 2,) * 2
    assert np.allclose(P2, ref, atol=1e-12)
    # averaged & normalised pseudo-matrix: centre 1, sum (sum K)^2 / sum K^2
    cfg = O.Config()
    Pm = O.pseudo_matrix(sol, cfg)
    c = Pm.shape[0] // 2
    assert abs(Pm[c, c] - 1.0) < 1e-14
    assert abs(Pm.sum() - K.sum() ** 2 / np.sum(K * K)) < 1e-10
    # empirical lag covariances of convolved white noise
    noise = synth.white_noise(10, 700, 700, 1.0)
    out = O.direct_conv2d(noise, K)[10:-10, 10:-10]
    out = out - out.mean()
    var = out.var()
    for dx, dy in [(1, 0), (0, 1), (1, 1), (2, 0), (-1, 2)]:
        a = out[max(0, dy):out.shape[0] + min(0, dy), max(0, dx):out.shape[1] + min(0, dx)]
        b = out[max(0, -dy):out.shape[0] + min(0, -dy), max(0, -dx):out.shape[1] + min(0, -dx)]
        emp = float(np.mean(a * b)) / var
        assert abs(emp - Pm[c + dy, c + dx]) < 0.03


def test_covariance_factor():
    sol = _fixed_solution(64, 64)
    K = O.realise_kernel(sol, 0, 0)
    assert abs(O.covariance_factor(K, np.ones((1, 1))) - 1.0) < 1e-14
    C = np.array([[0.0, 0.1, 0.0], [0.2, 1.0, 0.2], [0.0, 0.1, 0.0]])
    P = O.pseudo_conv(K, C)
    c = P.shape[0] // 2
    assert abs(O.covariance_factor(K, C) - P[c, c] / np.sum(K * K)) < 1e-12


def test_noise_model_matched_filter_photometry():
    """Sec. 4.5: after convolving a difference image with a matched filter, flux / sqrt(expected
    variance) from the variance map plus pseudo-matrix has unit standard deviation (the paper
    reports 0.98 +- 0.03, always within 6%)."""
    W = H = 400
    sol = _fixed_solution(W, H)
    cfg = O.Config(cov_grid=2)
    n1 = synth.white_noise(21, W, H, 3.0)
    n2 = synth.white_noise(22, W, H, 2.0)
    V1 = np.full((H, W), 9.0)
    V2 = np.full((H, W), 4.0)
    m = np.zeros((H, W), np.uint16)
    D, VD, M, P = O.subtract(n1, n2, V1, V2, m, m, sol, cfg)
    G = gaussian_density(6, 1.8)
    G /= G.sum()
    flux = O.direct_conv2d(D, G)
    # expected variance of sum_a G(a) D(x-a): V_D * sum_a sum_b G(a) G(b) P(a - b)
    PG = O.pseudo_conv(G, P)
    c = PG.shape[0] // 2
    expect = VD * PG[c, c]
    ratio = (flux / np.sqrt(expect))[30:-30, 30:-30]
    assert abs(ratio.std() - 1.0) < 0.06


# ---------------------------------------------------------------- masks (Sec. 3.4)

def test_mask_matches_brute_force():
    rng = np.random.default_rng(5)
    H, W = 23, 31
    m1 = synth.random_mask(1, W, H, 0.03)
    m2 = synth.random_mask(2, W, H, 0.05, bit=synth.MASK_SAT)
    sol = _fixed_solution(W, H)
    cfg = O.Config()
    h = sol.basis.h
    for rb in (0, 2, h):
        got = O.mask_image(m1, sol, cfg, m2, rb=rb)
        for y in range(H):
            for x in range(W):
                dmin = None
                for yy in range(y - h, y + h + 1):
                    for xx in range(x - h, x + h + 1):
                        off = not (0 <= yy < H and 0 <= xx < W)
                        if off or (m1[yy, xx] & cfg.badmask):
                            d = max(abs(yy - y), abs(xx - x))
                            dmin = d if dmin is None else min(dmin, d)
                exp = int(m1[y, x]) | int(m2[y, x])
                if dmin is not None and dmin <= rb:
                    exp |= O.CONV_BAD
                elif dmin is not None:
                    exp |= O.CONV_POOR
                assert got[y, x] == exp


def test_r_bad_for_separable_gaussian_kernel():
    """For K = b0 delta + a G - a s delta chosen as a pure Gaussian, K^2 is separable and the
    energy inside the box of radius r is (sum_{|u|<=r} G(u)^2)^2 (x-profile squared)."""
    basis = O.Basis((2.2,), (0,), 9, 0)
    B, s, psi = O.basis_kernels(basis)
    a0 = 0.7
    sol = O.Solution(a0 * s[0], np.array([a0, 0.0]), 0.0, basis, 50, 50)
    K = O.realise_kernel(sol, 25, 25)
    u = np.arange(-9, 10)
    g2 = np.exp(-u * u / (2 * 2.2 ** 2)) ** 2
    tot = g2.sum() ** 2
    expect = next(r for r in range(10) if 1 - (g2[np.abs(u) <= r].sum() ** 2) / tot <= 0.2)
    assert np.allclose(K, a0 * psi[0] * np.outer(np.sqrt(g2), np.sqrt(g2)), atol=1e-15)
    assert O.r_bad(sol, 0.2) == expect


# ---------------------------------------------------------------- stamps (Sec. 3.3, 3.6)

def test_selection_on_a_hand_built_field():
    W, H = 120, 80
    basis = O.Basis((1.0,), (0,), 4, 0)
    cfg = O.Config(grid_nx=2, grid_ny=1, stamp_half=3, badmask=synth.BADMASK, max_cand=3)
    img = np.full((H, W), 100.0, np.float32)
    var = np.full((H, W), 100.0, np.float32)      # sigma = 10 per image -> sqrt(200) on the sum
    m = np.zeros((H, W), np.uint16)

    def peak(x, y, v):
        img[y, x] = 100.0 + v

    peak(20, 20, 300)     # region 0: bright
    peak(40, 50, 500)     # region 0: brighter
    peak(45, 50, 500)     # region 0: equal value, larger index -> after (40, 50)
    peak(6, 40, 900)      # region 0: too close to the edge (footprint radius 3 + 4 = 7 > 6)
    peak(25, 60, 1000)    # region 0: footprint hits a masked pixel
    m[66, 28] = synth.MASK_BAD
    peak(100, 30, 30)     # region 1: below 5 sigma (2 * 30 = 60 < 5 * sqrt(400) = 100)
    peak(90, 40, 400)     # region 1
    peak(91, 40, 400)     # region 1: tie with a neighbour -> lower index (90, 40) wins
    cand, med = O.extract_candidates(img, img, var, var, m, m, basis, cfg)
    assert med == np.float32(200.0)
    assert cand[0].tolist() == [[40, 50], [45, 50], [20, 20]]
    assert cand[1].tolist() == [[90, 40], [-1, -1], [-1, -1]]


def test_rejection_removes_the_stamp_with_an_injected_cosmic_ray():
    s1, s2 = 1.6, 2.2
    stars = isolated_stars(300, 240, 60, 30, seed=8, flux=(3e4, 6e4))
    fld = synth.gaussian_pair(300, 240, stars, s1, s2, sky=200.0)
    rng = np.random.default_rng(8)
    ref = rng.poisson(fld.ref).astype(np.float32)
    sci = rng.poisson(fld.sci).astype(np.float32)
    cand = np.array([[[int(round(x)), int(round(y))], [-1, -1]] for x, y, _ in stars], np.int32)
    hit = 7
    cx, cy = cand[hit, 0]
    cand[hit, 1] = (cx, cy)           # replacement candidate: the same star (clean after repair)
    sci_cr = sci.copy()
    sci_cr[cy + 3, cx - 2] += 4000.0  # cosmic ray inside the stamp of region `hit`
    basis = O.Basis((0.7, 1.5, 3.0), (2, 2, 2), 8, 0)
    cfg = O.Config(grid_nx=len(stars), grid_ny=1, badmask=synth.BADMASK, max_iter=5)
    sol = O.solve_kernel(ref, sci_cr, ref, sci_cr, fld.mask_ref, fld.mask_sci, basis, cfg, cand)
    rejected = [tuple(x) for x in np.argwhere(sol.status == O.STATUS_REJECTED)]
    assert (hit, 0) in rejected
    assert sol.status[hit, 1] in (O.STATUS_USED, O.STATUS_REJECTED)
    assert sol.history[0]["rejected"][0] == (hit, 0)


def test_spatially_varying_kernel_maps_the_local_psfs():
    """Science sigma varies linearly in x.  The kernel realised at x maps the reference PSF onto
    the local science PSF, K(x) (x) G(sigma1) = G(sigma2(x)), within the basis / polynomial
    approximation error: 2nd-order spatial terms follow the variation that a constant kernel
    cannot.  (The kernel itself is fixed only up to frequencies the reference PSF removes, so
    it is the mapped PSF that is compared.)"""
    W, H = 360, 240
    s1 = 1.5
    sig2 = lambda x: 2.0 + 0.6 * x / (W - 1)
    stars = isolated_stars(W, H, 48, 24, seed=9)
    fld = synth.gaussian_pair(W, H, stars, s1, sig2)
    cand = np.array([[[int(round(x)), int(round(y))]] for x, y, _ in stars], np.int32)
    cfg = O.Config(badmask=synth.BADMASK, max_iter=1)
    errs = {}
    for S in (0, 2):
        basis = O.Basis((0.8, 1.6, 3.0), (4, 2, 2), 10, S)
        sol = O.solve_kernel(fld.ref, fld.sci, fld.var_ref, fld.var_sci, fld.mask_ref,
                             fld.mask_sci, basis, cfg, cand)
        errs[S] = []
        for x in (60, 180, 300):
            K = O.realise_kernel(sol, x, 120)
            got = signal.convolve2d(gaussian_density(15, s1), K, mode="full")
            exp = gaussian_density(25, sig2(x))
            errs[S].append(np.linalg.norm(got - exp) / np.linalg.norm(exp))
    assert max(errs[2]) < 2e-3
    assert max(errs[0]) > 2e-2


# ---------------------------------------------------------------- stacking (Sec. 5.1)

def test_render_target_flux():
    T = O.render_target(80, 80, [(40.2, 39.7, 1000.0)], 7.5)
    assert abs(T.sum() - 1000.0) < 1e-6 * 1000


def _coadd_inputs():
    """Two stack inputs that the matching leaves unchanged (kernel = delta exactly): each
    warp is the target itself, plus, far from every source and stamp footprint, a smooth
    pattern below the detection threshold that differs between the warps.  The warps carry
    constant, different variances and different masked blocks, so the pixels are covered by
    two inputs, by one, or by none."""
    W = H = 96
    src = [(20.3, 14.6, 4e4), (31.7, 29.2, 6e4), (19.4, 47.8, 5e4), (33.1, 63.3, 3e4),
           (21.8, 80.1, 7e4)]
    fwhm = 7.5
    T = O.render_target(W, H, src, fwhm).astype(np.float32)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    sig2 = (4.0, 9.0)
    warps = []
    for i, s2 in enumerate(sig2):
        pat = np.where(xx >= 72, (1.5 if i == 0 else -1.2) * math.sqrt(s2) *
                       np.sin(0.21 * xx + 0.13 * (i + 1) * yy) ** 2, 0.0)
        img = (T.astype(np.float64) + pat).astype(np.float32)
        m = np.zeros((H, W), np.uint16)
        if i == 0:
            m[10:20, 75:85] = synth.MASK_BAD
            m[40:44, 70:96] = synth.MASK_BAD
        else:
            m[15:30, 80:90] = synth.MASK_BAD
            m[40:44, 70:96] = synth.MASK_BAD
        warps.append(dict(image=img, var=np.full((H, W), s2, np.float32), mask=m, fwhm=5.0))
    basis = O.Basis((1.0, 2.0), (2, 1), 5, 0)
    cfg = O.Config(grid_nx=2, grid_ny=3, badmask=synth.BADMASK)
    return warps, src, fwhm, basis, cfg, sig2


def test_stack_coadd_is_the_minimum_variance_combination():
    """Sec. 5.1-5.2: the coadd of inputs with constant noise sigma_i^2 that match the target
    exactly is the minimum-variance combination sum(I_i / sigma_i^2) / sum(1 / sigma_i^2) over
    the inputs that cover a pixel, with variance 1 / sum(1 / sigma_i^2).  Weights equal to the
    mean variance (instead of its inverse) or plain averaging fail both."""
    warps, src, fwhm, basis, cfg, sig2 = _coadd_inputs()
    img, var, msk, cnt, P, sols = O.stack(warps, src, fwhm, [basis] * 2, cfg)
    for sol in sols:   # the matching kernel is the delta
        assert abs(sol.b0 - 1.0) < 1e-9 and np.max(np.abs(sol.a)) < 1e-9
        assert O.r_bad(sol) == 0
    use = [(w["mask"].astype(np.int64) & synth.BADMASK) == 0 for w in warps]
    inv = [np.where(u, 1.0 / s2, 0.0) for u, s2 in zip(use, sig2)]
    num = sum(iv * w["image"].astype(np.float64) for iv, w in zip(inv, warps))
    den = sum(inv)
    n = sum(u.astype(np.int32) for u in use)
    assert np.array_equal(cnt, n)
    assert (n == 2).any() and (n == 1).any() and (n == 0).any()
    assert np.array_equal(msk, np.where(n == 0, 1, 0).astype(np.uint16))
    cov = n > 0
    exp_img = num[cov] / den[cov]
    assert np.max(np.abs(img[cov] - exp_img)) <= 1e-8 * np.max(np.abs(exp_img))
    assert np.allclose(var[cov], 1.0 / den[cov], rtol=1e-10, atol=0)
    # the perturbed pixels covered twice are where the weighting shows
    two = (n == 2) & (np.abs(warps[0]["image"] - warps[1]["image"]) > 0.5)
    assert two.sum() > 100
    assert np.all(img[~cov] == 0) and np.all(var[~cov] == 0)
    assert np.allclose(P, O.embed_centre(np.ones((1, 1)), P.shape[0]), atol=1e-9)


def test_combined_pseudo_matrix_of_a_weighted_sum():
    """Sec. 4.4 add rule for a weighted coadd S = sum w_i X_i of independent noise images,
    X_i = K_i (x) white noise of variance s_i^2: the covariance of S at lag D is
    sum w_i^2 s_i^2 (K_i * K_i)(D) (library correlation), so its pseudo-matrix is the
    average of the inputs' pseudo-matrices with weights w_i^2 mean(V_i), V_i = s_i^2 sum K_i^2
    being the inputs' variance maps."""
    u = np.arange(-6, 7, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    K1 = np.exp(-(U * U + V * V) / (2 * 1.3 ** 2))
    K2 = np.exp(-((U - 0.7) ** 2 / (2 * 2.1 ** 2) + V * V / (2 * 1.1 ** 2)))
    K2 /= K2.sum() / 1.7
    s2 = (3.0, 11.0)
    Vm = [s2[0] * np.sum(K1 * K1), s2[1] * np.sum(K2 * K2)]
    wts = [0.7, 0.2]   # any coadd weights (inverse-variance ones make w_i^2 mean(V_i) = w_i)
    cov = sum(w * w * s * signal.correlate2d(K, K, mode="full")
              for w, s, K in zip(wts, s2, (K1, K2)))
    c = (cov.shape[0] - 1) // 2
    expected = cov / cov[c, c]
    Ps = []
    for K in (K1, K2):
        P = O.pseudo_conv(K, np.ones((1, 1)))
        Ps.append(P / P[(P.shape[0] - 1) // 2, (P.shape[0] - 1) // 2])
    got = O.combine_pseudo(Ps, [w * w * v for w, v in zip(wts, Vm)])
    assert got.shape == expected.shape
    assert np.allclose(got, expected, rtol=0, atol=1e-14)
    # a plain average of the pseudo-matrices, weights w_i or weights mean(V_i) would differ
    for bad in ([1.0, 1.0], wts, Vm):
        assert np.max(np.abs(O.combine_pseudo(Ps, bad) - expected)) > 1e-3


def test_per_pixel_forms_match_whole_image_forms():
    """The one-pixel forms used for sampled full-size parity equal the whole-image forms
    (Eq. 12 image, Eq. 13 variance with per-tile kernels, Sec. 3.4 masks), including edges,
    masks, ragged tiles and a spatially varying kernel."""
    W, H = 83, 70
    sol = _fixed_solution(W, H, S=1, seed=3)
    rng = np.random.default_rng(4)
    V = rng.uniform(1.0, 9.0, (H, W)).astype(np.float32)
    V2 = rng.uniform(1.0, 9.0, (H, W)).astype(np.float32)
    m = np.zeros((H, W), np.uint16)
    m[rng.random((H, W)) < 0.01] = 1
    m2 = np.zeros((H, W), np.uint16)
    m2[5, 7] = 4
    cfg = O.Config(badmask=0xFF)
    Vimg = O.variance_image(V, m, sol, 0xFF, 32, V2=V2)
    Mimg = O.mask_image(m, sol, cfg, m2)
    Oimg = O.convolve_image(V, m, sol, 0xFF)
    for y in range(0, H, 3):
        for x in range(0, W, 4):
            assert abs(O.convolve_pixel(V, m, sol, 0xFF, x, y) - Oimg[y, x]) <= \
                1e-12 * np.abs(V).max()
            assert abs(O.variance_pixel(V, m, sol, 0xFF, x, y, 32, V2=V2) - Vimg[y, x]) <= \
                1e-12 * Vimg[y, x]
            assert O.mask_pixel(m, sol, cfg, x, y, m2) == Mimg[y, x]


# ---------------------------------------------------------------- quality (Sec. 3.7)

def test_kernel_quality_closed_forms():
    h = 10
    u = np.arange(-h, h + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    # a normalised Gaussian: zero first moments, second moments sigma^2 (continuous limit),
    # enclosed sum never above the total
    sig = 1.5
    G = np.exp(-(U * U + V * V) / (2 * sig * sig))
    q = O.kernel_quality(3.0 * G / G.sum())
    assert abs(q["kernel_sum"] - 3.0) < 1e-12
    assert abs(q["mom_x"]) < 1e-14 and abs(q["mom_y"]) < 1e-14 and abs(q["mom_xy"]) < 1e-14
    assert abs(q["mom_xx"] - sig * sig) < 1e-9 and abs(q["mom_yy"] - sig * sig) < 1e-9
    assert 1.0 - 1e-9 < q["deconv_max"] <= 1.0
    # a delta shifted by (2, -1): first moments (2, -1), no spread
    D = np.zeros((2 * h + 1, 2 * h + 1))
    D[h - 1, h + 2] = 1.0
    q = O.kernel_quality(D)
    assert (q["mom_x"], q["mom_y"], q["mom_xx"], q["mom_yy"]) == (2.0, -1.0, 0.0, 0.0)
    # a sharpening kernel 2 delta - G (sum 1): negative second moments, central excess
    S = -G / G.sum()
    S[h, h] += 2.0
    q = O.kernel_quality(S)
    assert abs(q["mom_xx"] + sig * sig) < 1e-9
    assert abs(q["deconv_max"] - (2.0 - G[h, h] / G.sum())) < 1e-12


def test_quality_flags_follow_the_recommended_cuts():
    sol = _fixed_solution(64, 64)
    q = O.quality(sol, 10, 0.2, 0.1)
    base = q["flags"]
    assert O.quality(sol, 2, 0.2, 0.1)["flags"] == base | O.QUALITY_FEW_STAMPS
    assert O.quality(sol, 10, 0.6, 0.1)["flags"] == base | O.QUALITY_MEAN_DEV
    assert O.quality(sol, 10, 0.2, 0.31)["flags"] == base | O.QUALITY_RMS_DEV


# ------------------------------------------- stacking with outlier rejection (Sec. 5.1)

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


def test_stack_full_of_identical_inputs_rejects_nothing():
    warps, src = _copies(3)
    ob = O.Basis((0.7, 1.5, 3.0), (2, 2, 2), 8, 0)
    oc = O.Config(grid_nx=2, grid_ny=2, badmask=synth.BADMASK)
    tf = 1.15 * warps[0]["fwhm"]
    r = O.stack_full(warps, src, tf, [ob] * 3, oc)
    assert r["rejected"] == [0, 0, 0]
    img, var, msk, cnt, _, _ = O.stack(warps, src, tf, [ob] * 3, oc)
    assert np.array_equal(r["conv"][3], cnt) and np.array_equal(r["conv"][2], msk)
    assert np.allclose(r["conv"][0], img, rtol=1e-13, atol=1e-9)
    # unconvolved stack of equal inputs: the input itself where unmasked, variance / 3
    ok = (warps[0]["mask"].astype(np.int64) & synth.BADMASK) == 0
    uimg, uvar, _, ucnt = r["unconv"]
    assert np.array_equal(ucnt, np.where(ok, 3, 0))
    assert np.allclose(uimg[ok], warps[0]["image"][ok], rtol=1e-12)
    assert np.allclose(uvar[ok], warps[0]["var"][ok].astype(np.float64) / 3.0, rtol=1e-12)


def test_stack_full_rejects_a_planted_spike_in_its_input_only():
    x, y, amp = 80, 80, 20000.0
    warps, src = _copies(3, spike=(1, x, y, amp))
    ob = O.Basis((0.7, 1.5, 3.0), (2, 2, 2), 8, 0)
    oc = O.Config(grid_nx=2, grid_ny=2, badmask=synth.BADMASK)
    r = O.stack_full(warps, src, 1.15 * warps[0]["fwhm"], [ob] * 3, oc)
    assert r["rejected"][0] == 0 and r["rejected"][2] == 0 and r["rejected"][1] > 0
    # the spiked input is out of both stacks around the spike; the others are equal there
    assert r["conv"][3][y, x] == 2 and r["unconv"][3][y, x] == 2
    assert abs(r["unconv"][0][y, x] - warps[0]["image"][y, x]) < 1e-9 * abs(warps[0]["image"][y, x])


# ---------------------------------------------------------------- binning (Sec. 4.3)

def test_bin_image_white_noise_and_flux():
    rng = np.random.default_rng(3)
    img = rng.normal(10.0, 2.0, (60, 61)).astype(np.float32)
    var = np.full((60, 61), 4.0, np.float32)
    m = np.zeros((60, 61), np.uint16)
    m[7, 9] = 1
    Ib, Vb, Mb, Pb = O.bin_image(img, var, m, 4, 0xFF)
    assert Ib.shape == (15, 15)
    ok = m == 0
    assert abs(Ib.sum() - np.where(ok, img, 0.0)[:60, :60].astype(np.float64).sum()) < 1e-9
    # white noise: variance of a 4x4 sum is 16 sigma^2, no covariance between blocks
    assert Vb[0, 0] == 64.0 and Vb[1, 2] == 60.0 and Mb[1, 2] == 1
    assert Pb.shape == (1, 1) and Pb[0, 0] == 1.0


def test_bin_image_correlated_noise_matches_empirical():
    """Noise convolved with K has pseudo-matrix (K * K) / sum K^2 (Sec. 4.3); after 2x2
    binning the empirical variance of the block sums and their lag-1 covariance match the
    binned variance map and pseudo-matrix."""
    K = np.array([[0.0, 0.1, 0.0], [0.1, 0.6, 0.3], [0.0, 0.2, 0.0]])
    C = O.pseudo_conv(K, np.ones((1, 1)))
    C = C / C[(C.shape[0] - 1) // 2, (C.shape[0] - 1) // 2]
    noise = synth.white_noise(17, 1200, 1200, 1.0)
    conv = O.direct_conv2d(noise, K)[8:-8, 8:-8]
    s2 = float(np.sum(K * K))
    n = conv.shape[0] // 2 * 2
    conv = conv[:n, :n]
    Ib, Vb, Mb, Pb = O.bin_image(conv, np.full(conv.shape, s2), np.zeros(conv.shape, np.uint16),
                                 2, 0xFF, C)
    emp_var = float(Ib.var())
    assert abs(emp_var - float(Vb.mean())) < 0.03 * emp_var
    c = (Pb.shape[0] - 1) // 2
    emp_cov = float(np.mean((Ib[:, 1:] - Ib.mean()) * (Ib[:, :-1] - Ib.mean())))
    assert abs(emp_cov / emp_var - Pb[c, c + 1]) < 0.03


# ---------------------------------------------------------------- dual kernel (Eq. 2)

def test_dual_normal_equations_equal_ridge_least_squares():
    """Dual-kernel normal equations with the penalty (Eq. 5-6 with P_i on the diagonal) equal
    the least-squares solution of the stacked weighted design augmented by sqrt(Phi p_i) rows."""
    f = synth.elongated_pair(5, 64, 12, noise=True)
    ob = O.Basis((1.0, 2.0), (1, 0), 3, 0)
    oc = O.Config(badmask=synth.BADMASK, dual=True, penalty=0.05)
    sts = [O.stamp_data(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, x, y, ob, oc)
           for x, y in ((16, 16), (40, 20), (30, 45))]
    b0, d0 = O.solve_normalisation(sts)
    M, v = O.normal_equations(sts, ob, "separate", b0, d0, oc.penalty)
    rows, rhs = [], []
    for st in sts:
        w = np.sqrt(np.where(st.ok, 1.0 / st.var, 0.0))
        rows.append(O.design_rows(st, 1) * w[:, None])
        rhs.append((st.I2 - b0 * st.R - d0) * w)
    A = np.concatenate(rows)
    p = np.tile(O.penalty_terms(ob), 2)
    phi = oc.penalty * float(np.trace(A.T @ A)) / float(p.sum())
    A = np.concatenate([A, np.diag(np.sqrt(phi * p))])
    y = np.concatenate(rhs + [np.zeros(p.size)])
    ref, *_ = np.linalg.lstsq(A, y, rcond=None)
    assert np.allclose(np.linalg.solve(M, v), ref, rtol=1e-8, atol=1e-12)


def test_penalty_of_gaussian_terms_closed_form():
    """p_k = sum (u^2 + v^2)^2 k_k^2 with k_k of unit L2 norm: k_k^2 is a Gaussian weight of
    per-axis variance s^2 = sigma^2 / 2 times the polynomial squared, so for the (p, q) = (0, 0)
    term p = E[r^4] = 8 s^4 = 2 sigma^4, and for (1, 0) p = E[r^4 u^2] / E[u^2] = 24 s^4 =
    6 sigma^4 (Gaussian moments E u^2 = s^2, E u^4 = 3 s^4, E u^6 = 15 s^6).  The lattice sums
    equal the integrals to ~1e-6 relative for sigma = 1.5 and h = 8 sigma."""
    sig = 1.5
    ob = O.Basis((sig,), (1,), 12, 0)
    terms = O.basis_terms(ob)
    pk = O.penalty_terms(ob)
    for term, k in (((0, 0, 0), 2.0), ((0, 1, 0), 6.0), ((0, 0, 1), 6.0)):
        assert abs(pk[terms.index(term)] - k * sig ** 4) <= 1e-5 * k * sig ** 4, term


def test_dual_identical_images_give_zero_kernels():
    f = synth.elongated_pair(6, 96, 30)
    ob = O.Basis((1.0, 2.0), (2, 0), 5, 0)
    oc = O.Config(grid_nx=2, grid_ny=2, badmask=synth.BADMASK, dual=True)
    sol = O.solve_kernel(f.ref, f.ref, f.var_ref, f.var_ref, f.mask_ref, f.mask_ref, ob, oc)
    assert abs(sol.b0 - 1.0) < 1e-12 and abs(sol.d0) < 1e-9
    assert np.max(np.abs(sol.coeff)) < 1e-9


def test_dual_variance_of_white_noise_is_sum_of_both_kernels():
    """V_D = sigma1^2 sum K1^2 + sigma2^2 sum K2^2 for white inputs and constant kernels."""
    f = synth.elongated_pair(7, 64, 10)
    ob = O.Basis((1.0, 2.0), (2, 0), 5, 0)
    nb = len(O.basis_terms(ob))
    rng = np.random.default_rng(1)
    coeff = np.concatenate([rng.normal(0, 0.1, nb), rng.normal(0, 0.1, nb), [3.0]])
    sol = O.Solution(0.9, coeff, 3.0, ob, 64, 64, dual=True)
    V1 = np.full((64, 64), 4.0, np.float32)
    V2 = np.full((64, 64), 9.0, np.float32)
    m = np.zeros((64, 64), np.uint16)
    Vd = O.variance_image(V1, m, sol, 0xFF, 64, V2=V2, m2=m)
    K1, K2 = O.realise_kernel(sol, 0, 0), O.realise_kernel2(sol, 0, 0)
    expect = 4.0 * np.sum(K1 * K1) + 9.0 * np.sum(K2 * K2)
    assert np.allclose(Vd[5:-5, 5:-5], expect, rtol=1e-12)


def test_dual_kernel_matches_orthogonal_elongations_better():
    """PSFs elongated in orthogonal directions: convolving both images (Eq. 2) leaves smaller
    stamp residuals than convolving the reference alone, which would need deconvolution."""
    f = synth.elongated_pair(8, 192, 90)
    ob = O.Basis((0.8, 1.6, 3.0), (4, 2, 2), 8, 0)
    single = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob,
                            O.Config(grid_nx=3, grid_ny=3, badmask=synth.BADMASK))
    dual = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob,
                          O.Config(grid_nx=3, grid_ny=3, badmask=synth.BADMASK, dual=True))
    assert dual.chi2_mean < single.chi2_mean


# ---------------------------------------------------------------- envelope PSF (Sec. 5.1)

def test_envelope_of_gaussians_is_the_widest():
    """Circular Gaussians with a common peak: the pixel-wise maximum is the widest one, which
    the Gaussian fit reproduces exactly (zero residual)."""
    for models in ([(4.0, 4.0, 0.0, 3.0), (6.2, 6.2, 0.0, 3.0), (5.0, 5.0, 0.0, 3.0)],
                   [(3.5, 3.5, 0.0, 2.0)]):
        top = max(m[0] for m in models)
        assert abs(O.envelope_fwhm(models) - top) <= 2e-7 * top


def test_envelope_circularises_elliptical_inputs():
    """An elliptical input enters as the circular profile of FWHM sqrt(major * minor)."""
    assert abs(O.envelope_fwhm([(6.0, 4.0, 0.0, 3.0)]) - math.sqrt(24.0)) <= 1e-7


def test_envelope_order_and_duplicates():
    m1, m2, m3 = (4.0, 4.5, 0.3, 3.0), (6.0, 5.0, 0.8, 2.5), (5.5, 5.5, 1.0, 4.0)
    ref = O.envelope_fwhm([m1, m2, m3], radius=20)
    assert abs(O.envelope_fwhm([m3, m1, m2], radius=20) - ref) <= 1e-9 * ref
    assert abs(O.envelope_fwhm([m2, m3, m1, m2], radius=20) - ref) <= 1e-9 * ref


def test_envelope_moffat_limit_is_gaussian():
    """Moffat(beta) tends to the Gaussian of the same FWHM as beta grows."""
    assert abs(O.envelope_fwhm([(5.0, 5.0, 1.0, 1e5)]) - 5.0) <= 1e-3


def test_envelope_fit_equals_two_parameter_least_squares():
    """Eliminating the amplitude gives the same fit as a direct two-parameter least squares
    (scipy) on the realised envelope."""
    from scipy.optimize import least_squares
    models = [(4.0, 4.5, 0.3, 3.0), (6.0, 5.0, 0.8, 2.5)]
    R = 18
    u = np.arange(-R, R + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    r2 = U * U + V * V
    E = np.max([O.psf_profile_circular(r2, math.sqrt(a * b), f, be) for a, b, f, be in models], 0)
    fit = least_squares(lambda p: (p[0] * np.exp(-0.5 * r2 / p[1] ** 2) - E).ravel(), [1.0, 2.0],
                        xtol=1e-14, ftol=1e-14, gtol=1e-14)
    k = 2.0 * math.sqrt(2.0 * math.log(2.0))
    assert abs(O.envelope_fwhm(models, radius=R) - k * abs(fit.x[1])) <= 1e-6 * k * fit.x[1]


# ---------------------------------------------------------------- pseudo-matrix resampling

def _gauss_pseudo(w, sig):
    r = (w - 1) // 2
    u = np.arange(-r, r + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    return np.exp(-(U * U + V * V) / (4.0 * sig * sig))


def test_resample_pseudo_identity_and_white():
    C = _gauss_pseudo(21, 2.0)
    assert np.allclose(O.resample_pseudo(C, 1.0), C, rtol=0, atol=1e-15)
    d = np.zeros((9, 9))
    d[4, 4] = 1.0
    for s in (0.6, 1.7, 3.0):
        out = O.resample_pseudo(d, s)
        c = (out.shape[0] - 1) // 2
        assert out[c, c] == 1.0 and np.count_nonzero(out) == 1


def test_resample_pseudo_integer_scale_is_subsampling():
    """An integer scale b samples the input at lags b D exactly (no interpolation); the off-centre
    entries then carry the input's off-centre total."""
    C = _gauss_pseudo(31, 3.0)
    for b in (2, 3, 5):
        out = O.resample_pseudo(C, float(b))
        r = (out.shape[0] - 1) // 2
        sub = C[15 - r * b:15 + r * b + 1:b, 15 - r * b:15 + r * b + 1:b].copy()
        off = np.ones(sub.shape, bool)
        off[r, r] = False
        sub[off] *= (C.sum() - 1.0) / sub[off].sum()
        assert np.allclose(out, sub, rtol=1e-13, atol=0)


def test_resample_pseudo_interpolation_matches_library():
    """Before the off-centre rescaling, the values are scipy's linear grid interpolation (zero
    outside); afterwards the centre is the input's and the off-centre total is the input's."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(3)
    C = _gauss_pseudo(25, 2.5) * (1 + 0.05 * rng.standard_normal((25, 25)))
    C = 0.5 * (C + C[::-1, ::-1])
    C[12, 12] = 1.0
    for s in (0.65, 1.4, 2.3):
        out = O.resample_pseudo(C, s)
        r = (out.shape[0] - 1) // 2
        g = np.arange(25, dtype=np.float64)
        f = RegularGridInterpolator((g, g), C, method="linear", bounds_error=False, fill_value=0.0)
        D = np.arange(-r, r + 1) * s + 12
        Y, X = np.meshgrid(D, D, indexing="ij")
        ref = f(np.stack([Y.ravel(), X.ravel()], 1)).reshape(out.shape)
        off = np.ones(out.shape, bool)
        off[r, r] = False
        ref[off] *= (C.sum() - C[12, 12]) / ref[off].sum()
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-15)
        assert out[r, r] == C[12, 12]
        assert abs(out[off].sum() - (C.sum() - C[12, 12])) <= 1e-12 * C.sum()
