"""Seeded synthetic star fields shaped like the Pan-STARRS data the paper works with.

This module only makes inputs: star positions and fluxes, PSF profiles used to render them,
sky, Poisson noise, variance maps and detector masks.  It holds none of the PSF-matching
arithmetic (no kernel basis, no fit, no convolution by a solved kernel), so the CUDA path
and the FP64 oracle can both take their inputs from here without sharing method code.

Every array is produced from an explicit ``seed`` with ``numpy.random.default_rng``.
Images are float32 in electrons (gain 1, read noise 0), indexed ``[y, x]``; masks are uint16.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Detector mask bits of the synthetic inputs.  Bits 14 and 15 are left free for the
# convolution flags (CONV.BAD / CONV.POOR) that the PSF-matching path writes.
MASK_BAD = 1 << 0      # bad column or defect block
MASK_SAT = 1 << 1      # saturated core
MASK_BLEED = 1 << 2    # bleed trail from a saturated star
BADMASK = MASK_BAD | MASK_SAT | MASK_BLEED

FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


def fwhm_to_sigma(fwhm: float) -> float:
    return fwhm / FWHM_PER_SIGMA


def moffat_alpha(fwhm: float, beta: float) -> float:
    return fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))


# --------------------------------------------------------------------------------------
# PSF rendering (sampled at pixel centres, normalised so the continuous profile integrates
# to the star's flux)
# --------------------------------------------------------------------------------------

def _quad_form(dx, dy, e, theta):
    """Squared elliptical radius in units where the geometric-mean radius is preserved."""
    if e == 0.0:
        return dx * dx + dy * dy
    c, s = math.cos(theta), math.sin(theta)
    xr = c * dx + s * dy
    yr = -s * dx + c * dy
    q = 1.0 - e  # axis ratio b/a
    return xr * xr * q + yr * yr / q


def add_gaussian(img, x0, y0, flux, sigma, e=0.0, theta=0.0, radius=None):
    """Add ``flux`` times a (possibly elliptical) Gaussian density centred on (x0, y0)."""
    H, W = img.shape
    if radius is None:
        radius = int(math.ceil(7.0 * sigma / math.sqrt(max(1.0 - e, 1e-3)))) + 1
    xi, yi = int(round(x0)), int(round(y0))
    xa, xb = max(0, xi - radius), min(W, xi + radius + 1)
    ya, yb = max(0, yi - radius), min(H, yi + radius + 1)
    if xa >= xb or ya >= yb:
        return
    yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
    r2 = _quad_form(xx - x0, yy - y0, e, theta)
    img[ya:yb, xa:xb] += flux * np.exp(-0.5 * r2 / (sigma * sigma)) / (2.0 * math.pi * sigma * sigma)


def add_moffat(img, x0, y0, flux, fwhm, beta=3.0, e=0.0, theta=0.0, radius=None):
    """Add ``flux`` times a (possibly elliptical) Moffat profile centred on (x0, y0)."""
    H, W = img.shape
    alpha = moffat_alpha(fwhm, beta)
    if radius is None:
        radius = min(int(math.ceil(8.0 * alpha)) + 1, 60)
    xi, yi = int(round(x0)), int(round(y0))
    xa, xb = max(0, xi - radius), min(W, xi + radius + 1)
    ya, yb = max(0, yi - radius), min(H, yi + radius + 1)
    if xa >= xb or ya >= yb:
        return
    yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
    r2 = _quad_form(xx - x0, yy - y0, e, theta)
    norm = (beta - 1.0) / (math.pi * alpha * alpha)
    img[ya:yb, xa:xb] += flux * norm * (1.0 + r2 / (alpha * alpha)) ** (-beta)


# --------------------------------------------------------------------------------------
# Field recipes
# --------------------------------------------------------------------------------------

@dataclass
class Field:
    """One reference/science pair with variance maps and masks (all [y, x])."""
    ref: np.ndarray          # I1, float32
    sci: np.ndarray          # I2, float32
    var_ref: np.ndarray      # float32
    var_sci: np.ndarray      # float32
    mask_ref: np.ndarray     # uint16
    mask_sci: np.ndarray     # uint16
    manifest: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.ref.shape


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n))


def _bad_columns(rng, W, n_cols, cluster_max=1):
    cols = set()
    while len(cols) < n_cols:
        c0 = int(rng.integers(0, W))
        width = int(rng.integers(1, cluster_max + 1))
        for c in range(c0, min(W, c0 + width)):
            cols.add(c)
    return np.array(sorted(cols)[:n_cols], dtype=np.int64)


def small_gaussian_field(seed: int = 1, size: int = 512, n_stars: int = 200,
                         fwhm_ref: float = 4.0, fwhm_sci: float = 5.5, sky: float = 500.0,
                         flux_lo: float = 1e3, flux_hi: float = 1e5, bad_col_frac: float = 0.01,
                         noise: bool = True, width: int | None = None) -> Field:
    """512x512 pair of circular-Gaussian star fields (the small plain-method workload).

    200 stars at uniform positions, flux log-uniform in [1e3, 1e5] e-, FWHM 4.0 px in the
    reference and 5.5 px in the science image, sky 500 e- plus Poisson noise, variance =
    image / gain, and 1% bad columns (the same detector columns in both images).
    """
    rng = np.random.default_rng(seed)
    H = size
    W = size if width is None else width
    xs = rng.uniform(0, W - 1, n_stars)
    ys = rng.uniform(0, H - 1, n_stars)
    fl = _log_uniform(rng, flux_lo, flux_hi, n_stars)
    s1, s2 = fwhm_to_sigma(fwhm_ref), fwhm_to_sigma(fwhm_sci)
    ref = np.full((H, W), sky, np.float64)
    sci = np.full((H, W), sky, np.float64)
    for x, y, f in zip(xs, ys, fl):
        add_gaussian(ref, x, y, f, s1)
        add_gaussian(sci, x, y, f, s2)
    if noise:
        ref = rng.poisson(ref).astype(np.float64)
        sci = rng.poisson(sci).astype(np.float64)
    var_ref = ref.copy()
    var_sci = sci.copy()
    mask_ref = np.zeros((H, W), np.uint16)
    mask_sci = np.zeros((H, W), np.uint16)
    n_bad = int(round(bad_col_frac * W))
    cols = _bad_columns(rng, W, n_bad) if n_bad > 0 else np.zeros(0, np.int64)
    for m, im in ((mask_ref, ref), (mask_sci, sci)):
        m[:, cols] |= MASK_BAD
        im[:, cols] = 65535.0 if noise else 0.0
    return Field(ref.astype(np.float32), sci.astype(np.float32), var_ref.astype(np.float32),
                 var_sci.astype(np.float32), mask_ref, mask_sci,
                 dict(kind="small_gaussian", seed=seed, W=W, H=H, n_stars=n_stars,
                      fwhm_ref=fwhm_ref, fwhm_sci=fwhm_sci, sky=sky, bad_columns=cols.tolist(),
                      stars=np.stack([xs, ys, fl], 1)))


def elongated_pair(seed: int = 3, size: int = 256, n_stars: int = 120, sigma: float = 1.8,
                   e: float = 0.35, sky: float = 500.0, noise: bool = True) -> Field:
    """Pair whose PSFs are elongated in orthogonal directions (reference along x, science
    along y, axis ratio 1 - e, same area): neither can be matched to the other without
    deconvolution, the case the dual-kernel formulation addresses.  Stars uniform, flux
    log-uniform in [1e3, 1e5] e-, sky plus Poisson noise, variance = image, no mask."""
    rng = np.random.default_rng(seed)
    xs = rng.uniform(0, size - 1, n_stars)
    ys = rng.uniform(0, size - 1, n_stars)
    fl = _log_uniform(rng, 1e3, 1e5, n_stars)
    ref = np.full((size, size), sky, np.float64)
    sci = np.full((size, size), sky, np.float64)
    for x, y, f in zip(xs, ys, fl):
        add_gaussian(ref, x, y, f, sigma, e, 0.0)
        add_gaussian(sci, x, y, f, sigma, e, 0.5 * math.pi)
    if noise:
        ref = rng.poisson(ref).astype(np.float64)
        sci = rng.poisson(sci).astype(np.float64)
    m = np.zeros((size, size), np.uint16)
    return Field(ref.astype(np.float32), sci.astype(np.float32), ref.astype(np.float32),
                 sci.astype(np.float32), m, m.copy(),
                 dict(kind="elongated_pair", seed=seed, size=size, sigma=sigma, e=e))


def full_chip_field(seed: int = 2, W: int = 4846, H: int = 4868, n_stars: int = 2500,
                    fwhm_ref=(3.5, 4.5), fwhm_sci=(4.5, 6.5), e_max: float = 0.15,
                    beta: float = 3.0, sky: float = 500.0, flux_lo: float = 1e3,
                    flux_hi: float = 1e5, n_transients: int = 50, mask_frac: float = 0.03,
                    sat_level: float = 3500.0) -> Field:
    """Full GPC1-chip-shaped pair: Moffat beta=3 PSFs whose FWHM varies linearly in x.

    Reference FWHM 3.5->4.5 px and science 4.5->6.5 px across the chip; ellipticity up to
    0.15, as a smooth field over the chip (different in the two images); 2500 stars with
    log-uniform flux in [1e3, 1e5] e-; 50 point transients in the science image only.
    Masks (about ``mask_frac`` of each image): saturated cores above ``sat_level`` with
    vertical bleed trails, clustered bad columns and rectangular defect blocks.
    """
    rng = np.random.default_rng(seed)
    xs = rng.uniform(0, W - 1, n_stars)
    ys = rng.uniform(0, H - 1, n_stars)
    fl = _log_uniform(rng, flux_lo, flux_hi, n_stars)
    tx = rng.uniform(40, W - 41, n_transients)
    ty = rng.uniform(40, H - 41, n_transients)
    tf = _log_uniform(rng, 3e3, 3e4, n_transients)
    th_ref, th_sci = rng.uniform(0, math.pi, 2)

    def psf_params(x, y, fw):
        f = fw[0] + (fw[1] - fw[0]) * x / (W - 1)
        return f

    def ell(x, y, th0):
        e = e_max * (0.5 + 0.5 * math.sin(2 * math.pi * (x / W + 0.5 * y / H)))
        return e, th0 + math.pi * y / H

    ref = np.full((H, W), sky, np.float64)
    sci = np.full((H, W), sky, np.float64)
    for x, y, f in zip(xs, ys, fl):
        e1, t1 = ell(x, y, th_ref)
        e2, t2 = ell(y / H * W, x / W * H, th_sci)
        add_moffat(ref, x, y, f, psf_params(x, y, fwhm_ref), beta, e1, t1)
        add_moffat(sci, x, y, f, psf_params(x, y, fwhm_sci), beta, e2, t2)
    for x, y, f in zip(tx, ty, tf):
        e2, t2 = ell(y / H * W, x / W * H, th_sci)
        add_moffat(sci, x, y, f, psf_params(x, y, fwhm_sci), beta, e2, t2)
    ref = rng.poisson(ref).astype(np.float64)
    sci = rng.poisson(sci).astype(np.float64)
    var_ref, var_sci = ref.copy(), sci.copy()

    # detector defects shared by both images: clustered bad columns and defect blocks
    shared = np.zeros((H, W), np.uint16)
    cols = _bad_columns(rng, W, max(1, int(0.003 * W)), cluster_max=3)
    shared[:, cols] |= MASK_BAD
    masks = []
    for im, m_own in ((ref, None), (sci, None)):
        m = shared.copy()
        sat = im >= sat_level
        m[sat] |= MASK_SAT
        # bleed trails: saturated pixels spill charge along the column, length grows with the
        # number of saturated pixels in that column of the star
        cols_sat, counts = np.unique(np.nonzero(sat)[1], return_counts=True)
        ysat = np.nonzero(sat)
        for c in cols_sat:
            rows = ysat[0][ysat[1] == c]
            r0, r1 = rows.min(), rows.max()
            L = 3 * (r1 - r0 + 1)
            m[max(0, r0 - L):min(H, r1 + L + 1), c] |= MASK_BLEED
        im[sat] = sat_level
        masks.append(m)
    # defect blocks until the masked fraction of each image reaches mask_frac
    blocks = []
    while True:
        frac = max(float(np.mean((mm & BADMASK) != 0)) for mm in masks)
        if frac >= mask_frac:
            break
        bw, bh = int(rng.integers(20, 120)), int(rng.integers(20, 120))
        bx, by = int(rng.integers(0, W - bw)), int(rng.integers(0, H - bh))
        blocks.append((bx, by, bw, bh))
        for mm in masks:
            mm[by:by + bh, bx:bx + bw] |= MASK_BAD
    for im, mm in ((ref, masks[0]), (sci, masks[1])):
        bad = (mm & MASK_BAD) != 0
        im[bad] = 0.0
    return Field(ref.astype(np.float32), sci.astype(np.float32), var_ref.astype(np.float32),
                 var_sci.astype(np.float32), masks[0], masks[1],
                 dict(kind="full_chip", seed=seed, W=W, H=H, n_stars=n_stars, beta=beta,
                      fwhm_ref=fwhm_ref, fwhm_sci=fwhm_sci, e_max=e_max, sky=sky,
                      sat_level=sat_level, bad_columns=cols.tolist(), blocks=blocks,
                      masked_frac=[float(np.mean((mm & BADMASK) != 0)) for mm in masks],
                      stars=np.stack([xs, ys, fl], 1), transients=np.stack([tx, ty, tf], 1)))


def gaussian_pair(W: int, H: int, stars, sigma_ref: float, sigma_sci, flux_ratio: float = 1.0,
                  sky: float = 0.0) -> Field:
    """Noiseless pair of Gaussian star fields rendered over the whole image (no truncation).

    ``stars`` is a list of (x, y, flux).  ``sigma_sci`` is a number or a function of x giving
    the science Gaussian width; the science image carries ``flux_ratio`` times each flux.
    Variance maps are sky + image (Poisson expectation) floored at 1; masks are empty.
    """
    ref = np.full((H, W), sky, np.float64)
    sci = np.full((H, W), sky * flux_ratio, np.float64)
    big = max(W, H) + 1
    for x, y, f in stars:
        add_gaussian(ref, x, y, f, sigma_ref, radius=big)
        s2 = sigma_sci(x) if callable(sigma_sci) else sigma_sci
        add_gaussian(sci, x, y, f * flux_ratio, s2, radius=big)
    return Field(ref.astype(np.float32), sci.astype(np.float32),
                 np.maximum(ref, 1.0).astype(np.float32), np.maximum(sci, 1.0).astype(np.float32),
                 np.zeros((H, W), np.uint16), np.zeros((H, W), np.uint16),
                 dict(kind="gaussian_pair", W=W, H=H))


def white_noise(seed: int, W: int, H: int, sigma: float = 1.0):
    """Gaussian white noise image of standard deviation ``sigma`` (float64)."""
    return np.random.default_rng(seed).normal(0.0, sigma, (H, W))


def random_mask(seed: int, W: int, H: int, frac: float, bit: int = MASK_BAD):
    """uint16 mask with about ``frac`` of pixels carrying ``bit`` (independent pixels)."""
    rng = np.random.default_rng(seed)
    m = np.zeros((H, W), np.uint16)
    m[rng.random((H, W)) < frac] = bit
    return m


def exposure_chips(seed: int = 4, n_chips: int = 60, size_lo=(1200, 1200), size_hi=(4846, 4868),
                   scale: float = 1.0):
    """Per-chip recipe of the uneven-size exposure workload (sizes, PSF, masking, spatial order).

    Returns a list of dicts; ``scale`` shrinks the chip sizes for small test versions.
    Degrees are drawn from the 49/57/66/70-term sets; the basis widths follow the paper's
    ISIS prescription scaled by the chip's maximum FWHM, which callers compute.
    """
    rng = np.random.default_rng(seed)
    degree_sets = [(6, 4, 2), (7, 4, 2), (8, 4, 2), (7, 6, 2)]
    chips = []
    for i in range(n_chips):
        W = int(rng.integers(size_lo[0], size_hi[0] + 1) * scale)
        H = int(rng.integers(size_lo[1], size_hi[1] + 1) * scale)
        f_ref = float(rng.uniform(3.0, 8.0))
        f_sci = float(rng.uniform(3.0, 8.0))
        chips.append(dict(index=i, W=W, H=H, fwhm_ref=f_ref, fwhm_sci=f_sci,
                          mask_frac=float(rng.uniform(0.01, 0.20)),
                          spatial_order=int(rng.integers(1, 4)),
                          degrees=degree_sets[int(rng.integers(0, 4))],
                          seed=int(rng.integers(0, 2**31 - 1))))
    return chips


def chip_field(chip: dict, n_stars_per_mpix: float = 100.0, sky: float = 500.0) -> Field:
    """Render one chip of :func:`exposure_chips`: circular Gaussian PSFs, defect blocks."""
    rng = np.random.default_rng(chip["seed"])
    W, H = chip["W"], chip["H"]
    n = max(20, int(n_stars_per_mpix * W * H / 1e6))
    xs, ys = rng.uniform(0, W - 1, n), rng.uniform(0, H - 1, n)
    fl = _log_uniform(rng, 1e3, 1e5, n)
    s1, s2 = fwhm_to_sigma(chip["fwhm_ref"]), fwhm_to_sigma(chip["fwhm_sci"])
    ref = np.full((H, W), sky, np.float64)
    sci = np.full((H, W), sky, np.float64)
    for x, y, f in zip(xs, ys, fl):
        add_gaussian(ref, x, y, f, s1)
        add_gaussian(sci, x, y, f, s2)
    ref = rng.poisson(ref).astype(np.float64)
    sci = rng.poisson(sci).astype(np.float64)
    m = np.zeros((H, W), np.uint16)
    while float(np.mean(m != 0)) < chip["mask_frac"]:
        bw, bh = int(rng.integers(10, 80)), int(rng.integers(10, 80))
        bx, by = int(rng.integers(0, max(1, W - bw))), int(rng.integers(0, max(1, H - bh)))
        m[by:by + bh, bx:bx + bw] |= MASK_BAD
    ref[m != 0] = 0.0
    sci[m != 0] = 0.0
    return Field(ref.astype(np.float32), sci.astype(np.float32), ref.astype(np.float32),
                 sci.astype(np.float32), m.copy(), m.copy(), dict(kind="chip", **chip))


def skycell_warps(seed: int = 5, n_warps: int = 16, size: int = 6000, n_stars: int = 6000,
                  sky: float = 500.0, gap_range=(300, 700), block_range=(50, 600),
                  masked_range=(0.05, 0.40)):
    """Inputs of the stacking workload: warps of one skycell with uneven coverage.

    Returns (warps, sources): a list of dicts with image, variance, mask and the warp's PSF
    FWHM, and the (x, y, flux) source list shared by all warps.  Each warp's PSF is a
    Gaussian-core Moffat mixture with FWHM in [3.5, 7]; masked fraction 5-40% from chip-gap
    bands and defect blocks (``gap_range``, ``block_range`` and ``masked_range`` shrink them
    for small test versions).
    """
    rng = np.random.default_rng(seed)
    xs, ys = rng.uniform(0, size - 1, n_stars), rng.uniform(0, size - 1, n_stars)
    fl = _log_uniform(rng, 1e3, 1e5, n_stars)
    warps = []
    for i in range(n_warps):
        fw = float(rng.uniform(3.5, 7.0))
        frac_moffat = float(rng.uniform(0.0, 1.0))
        img = np.full((size, size), sky, np.float64)
        for x, y, f in zip(xs, ys, fl):
            add_gaussian(img, x, y, f * (1 - frac_moffat), fwhm_to_sigma(fw))
            if frac_moffat > 0:
                add_moffat(img, x, y, f * frac_moffat, fw, 3.0)
        img = rng.poisson(img).astype(np.float64)
        m = np.zeros((size, size), np.uint16)
        target = float(rng.uniform(*masked_range))
        # chip-gap bands
        gap = int(rng.integers(*gap_range))
        off = int(rng.integers(0, gap))
        for g0 in range(off, size, gap):
            m[:, g0:g0 + 12] |= MASK_BAD
        while float(np.mean(m != 0)) < target:
            bw, bh = int(rng.integers(*block_range)), int(rng.integers(*block_range))
            bx, by = int(rng.integers(0, size - bw)), int(rng.integers(0, size - bh))
            m[by:by + bh, bx:bx + bw] |= MASK_BAD
        img[m != 0] = 0.0
        warps.append(dict(image=img.astype(np.float32), var=np.maximum(img, 1.0).astype(np.float32),
                          mask=m, fwhm=fw, masked_frac=float(np.mean(m != 0)),
                          psf_model=(fw, fw, frac_moffat, 3.0)))
    return warps, np.stack([xs, ys, fl], 1)


# --------------------------------------------------------------------------------------
# Fast seeded generation on the GPU for large throughput workloads (torch; no method code)
# --------------------------------------------------------------------------------------

def torch_chip_pair(seed: int, W: int, H: int, fwhm_ref: float, fwhm_sci: float,
                    mask_frac: float, device, stars_per_mpix: float = 100.0,
                    sky: float = 500.0):
    """Reference / science pair of circular-Gaussian star fields rendered on the GPU.

    Stars at uniform sub-pixel positions (bilinear deposit, then a separable Gaussian blur),
    flux log-uniform in [1e3, 1e5] e-, sky plus Poisson noise, variance = image, and defect
    blocks (shared by both images) covering about ``mask_frac``.  Returns a dict of CUDA tensors
    (img, ref, var_img, var_ref, mask_img, mask_ref) with the masks as int16."""
    import torch
    import torch.nn.functional as F
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    n = max(20, int(stars_per_mpix * W * H / 1e6))
    xs = torch.rand(n, generator=g, device=device, dtype=torch.float64) * (W - 1)
    ys = torch.rand(n, generator=g, device=device, dtype=torch.float64) * (H - 1)
    fl = torch.exp(torch.rand(n, generator=g, device=device, dtype=torch.float64) *
                   (math.log(1e5) - math.log(1e3)) + math.log(1e3))

    def render(fwhm):
        img = torch.zeros(H * W, device=device, dtype=torch.float64)
        x0, y0 = xs.floor(), ys.floor()
        fx, fy = xs - x0, ys - y0
        for dx, dy, wgt in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)),
                            (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
            xi = (x0 + dx).clamp(0, W - 1).long()
            yi = (y0 + dy).clamp(0, H - 1).long()
            img.index_add_(0, yi * W + xi, fl * wgt)
        sig = fwhm_to_sigma(fwhm)
        r = int(math.ceil(5 * sig))
        t = torch.arange(-r, r + 1, device=device, dtype=torch.float64)
        k = torch.exp(-t * t / (2 * sig * sig))
        k = (k / k.sum()).float()
        im = img.float().view(1, 1, H, W)
        im = F.conv2d(F.pad(im, (r, r, 0, 0)), k.view(1, 1, 1, -1))
        im = F.conv2d(F.pad(im, (0, 0, r, r)), k.view(1, 1, -1, 1))
        return im.view(H, W) + sky

    ref = torch.poisson(render(fwhm_ref), generator=g)
    sci = torch.poisson(render(fwhm_sci), generator=g)
    m = torch.zeros((H, W), dtype=torch.int16, device=device)
    target = int(mask_frac * W * H)
    covered = 0
    rng = np.random.default_rng(int(seed))
    while covered < target:
        bw, bh = int(rng.integers(10, 80)), int(rng.integers(10, 80))
        bx, by = int(rng.integers(0, max(1, W - bw))), int(rng.integers(0, max(1, H - bh)))
        m[by:by + bh, bx:bx + bw] = MASK_BAD
        covered += bw * bh
    ref = ref.masked_fill(m != 0, 0.0)
    sci = sci.masked_fill(m != 0, 0.0)
    return dict(img=sci.contiguous(), ref=ref.contiguous(), var_img=sci.clone(),
                var_ref=ref.clone(), mask_img=m, mask_ref=m.clone())


def isis_prescription_sigmas(fwhm_max: float):
    """Gaussian widths of the paper's recommended ISIS basis (Sec. 3.1): FWHM 2.9, 4.8, 8.2 px
    scaled linearly by fwhm_max / 9, the scale clamped to [0.7, 1.2]; returned as sigmas."""
    scale = min(1.2, max(0.7, fwhm_max / 9.0))
    return tuple(fwhm_to_sigma(f * scale) for f in (2.9, 4.8, 8.2))


def torch_skycell_warps(seed: int, n_warps: int, size: int, n_src: int, device,
                        sky: float = 500.0, masked_range=(0.05, 0.40)):
    """Stacking inputs rendered on the GPU: ``n_warps`` warps of one ``size`` x ``size``
    skycell sharing a source list (uniform positions, flux log-uniform in [1e3, 1e5] e-).  Each
    warp's PSF is a core Gaussian plus a wing Gaussian of twice the width carrying a random
    fraction (0-30 %) of the flux, core FWHM U[3.5, 7] px; sky plus Poisson noise, variance =
    image; chip-gap bands (12 px every 300-700 px) and defect blocks bring the masked fraction
    to U[masked_range].  Returns (warps, sources): warps are dicts of CUDA tensors image, var,
    mask (int16) with the warp's fwhm; sources an (n, 3) float64 numpy array (x, y, flux)."""
    import torch
    import torch.nn.functional as F
    rng = np.random.default_rng(int(seed))
    xs = rng.uniform(0, size - 1, n_src)
    ys = rng.uniform(0, size - 1, n_src)
    fl = _log_uniform(rng, 1e3, 1e5, n_src)
    sources = np.stack([xs, ys, fl], 1)
    tx = torch.from_numpy(xs).to(device)
    ty = torch.from_numpy(ys).to(device)
    tf = torch.from_numpy(fl).to(device)
    x0, y0 = tx.floor(), ty.floor()
    fx, fy = tx - x0, ty - y0
    point = torch.zeros(size * size, device=device, dtype=torch.float64)
    for dx, dy, wgt in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)),
                        (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
        xi = (x0 + dx).clamp(0, size - 1).long()
        yi = (y0 + dy).clamp(0, size - 1).long()
        point.index_add_(0, yi * size + xi, tf * wgt)
    point = point.float().view(1, 1, size, size)

    def blur(sig):
        r = int(math.ceil(5 * sig))
        t = torch.arange(-r, r + 1, device=device, dtype=torch.float64)
        k = torch.exp(-t * t / (2 * sig * sig))
        k = (k / k.sum()).float()
        im = F.conv2d(F.pad(point, (r, r, 0, 0)), k.view(1, 1, 1, -1))
        return F.conv2d(F.pad(im, (0, 0, r, r)), k.view(1, 1, -1, 1)).view(size, size)

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    warps = []
    for _ in range(n_warps):
        fw = float(rng.uniform(3.5, 7.0))
        wing = float(rng.uniform(0.0, 0.3))
        sig = fwhm_to_sigma(fw)
        img = (1 - wing) * blur(sig) + wing * blur(2 * sig) + sky
        img = torch.poisson(img.double(), generator=g).float()
        m = torch.zeros((size, size), dtype=torch.int16, device=device)
        gap = int(rng.integers(300, 700))
        for g0 in range(int(rng.integers(0, gap)), size, gap):
            m[:, g0:g0 + 12] = MASK_BAD
        target = float(rng.uniform(*masked_range))
        covered = float((m != 0).float().mean())
        while covered < target:
            bw, bh = int(rng.integers(50, 600)), int(rng.integers(50, 600))
            bx, by = int(rng.integers(0, size - bw)), int(rng.integers(0, size - bh))
            m[by:by + bh, bx:bx + bw] = MASK_BAD
            covered = float((m != 0).float().mean())
        img = img.masked_fill(m != 0, 0.0)
        warps.append(dict(image=img.contiguous(), var=img.clamp_min(1.0).contiguous(), mask=m,
                          fwhm=fw))
    return warps, sources
