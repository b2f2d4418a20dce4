"""FP64 CPU oracle of the PSF-matching hot path.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  The library under ``paper_1901_09999_gb300`` never calls it, and it shares no code
with the CUDA path: its inputs come from ``paper_1901_09999_gb300.synth`` (which holds no method
arithmetic) or from the tests.

It computes, slowly and in float64, the plain definitions of the method of Price & Magnier,
"Pan-STARRS PSF-Matching for Subtraction and Stacking" (arXiv:1901.09999):

* kernel basis: ISIS Gaussian x polynomial terms (Sec. 2, Eq. 7) normalised to unit L2 norm and
  made zero-sum by subtracting a scaled central delta (Sec. 2, the zero-sum requirement);
* design vector and normal equations (Sec. 2, Eq. 3-6), with the spatial factors g_i taken at
  the stamp centres (Sec. 2) as ordinary monomials in normalised coordinates;
* normalisation b0 and background d0 solved first without variance weighting (Sec. 3.2);
* stamp selection per subregion (Sec. 3.3) and iterative rejection (Sec. 3.3, Sec. 3.6);
* application of the spatially varying kernel (Eq. 12), variance propagation (Eq. 13) with
  per-patch covariance factors (Sec. 4.3-4.4), the covariance pseudo-matrix (Eq. 10-11,
  Sec. 4.3-4.4), and CONV.BAD / CONV.POOR mask propagation (Sec. 3.4);
* PSF-homogenised stacking (Sec. 5.1).

Convolutions are direct 2-D sums with realised kernels, the design matrix is explicit, and the
normal equations are solved by Cholesky with an LU fallback.  Readings of points the paper
leaves open are stated next to the code that takes them.  Every function here is pinned by
tests in ``tests/test_oracle_*.py`` except where its docstring says "parity unpinned".
"""
from __future__ import annotations

import math
import warnings
from dataclasses import dataclass, field, replace

import numpy as np

CONV_BAD = 1 << 14
CONV_POOR = 1 << 15

STATUS_UNUSED = 0
STATUS_USED = 1
STATUS_REJECTED = 2


class OracleError(RuntimeError):
    pass


class TooFewStamps(OracleError):
    pass


@dataclass
class Basis:
    """ISIS basis (Eq. 7): Gaussian widths ``sigma`` with polynomial ``degree`` each, kernel
    half-width ``h`` (kernel (2h+1)^2) and spatial polynomial order ``S``."""
    sigma: tuple
    degree: tuple
    h: int
    S: int = 0

    @property
    def w(self):
        return 2 * self.h + 1


@dataclass
class Config:
    grid_nx: int = 6
    grid_ny: int = 5
    stamp_half: int | None = None      # s; None => s = h
    thresh_nsigma: float = 5.0
    reject_nsigma: float = 3.0
    soften_alpha: float = 0.1
    bad_frac: float = 0.2
    max_iter: int = 5
    var_tile: int = 64
    cov_grid: int = 5
    norm_mode: str = "separate"        # or "joint"
    badmask: int = 0x00FF
    conv_bad: int = CONV_BAD
    conv_poor: int = CONV_POOR
    max_cand: int = 8
    dual: bool = False                 # convolve both images (c_i != 0, Eq. 2)
    penalty: float = 1e-2              # lambda of the dual-kernel penalty scale (see below)

    def s(self, basis: Basis) -> int:
        return basis.h if self.stamp_half is None else self.stamp_half


# ----------------------------------------------------------------------------------------
# Basis (Sec. 2, Eq. 7 and the zero-sum requirement)
# ----------------------------------------------------------------------------------------

def basis_terms(basis: Basis):
    """Canonical order of kernel terms: Gaussian g ascending, then p = 0..d_g, then
    q = 0..d_g - p (the u^p v^q factor of Eq. 7)."""
    out = []
    for g, d in enumerate(basis.degree):
        for p in range(d + 1):
            for q in range(d - p + 1):
                out.append((g, p, q))
    return out


def spatial_terms(S: int):
    """Spatial monomials x^l y^m with l + m <= S, ordered l = 0..S, m = 0..S-l (Sec. 2)."""
    return [(l, m) for l in range(S + 1) for m in range(S - l + 1)]


def basis_kernels(basis: Basis):
    """Realised basis kernels B_k, shape (N_b, w, w) indexed [k, v+h, u+h].

    Eq. 7 prints the Gaussian factor as exp((u^2+v^2)/2s^2); the sign is garbled and the
    decaying form exp(-(u^2+v^2)/(2 s^2)) is used.  The normalisation constant psi_k is read as
    the one giving B'_k unit L2 norm.  The zero-sum requirement (Sec. 2) is met by
    subtracting s_k times the central delta, s_k = sum B'_k, for terms with p and q both even;
    for the others the sum is zero by symmetry and s_k = 0.
    Returns (B, s, psi).
    """
    h = basis.h
    u = np.arange(-h, h + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)          # U[v, u] = u, V[v, u] = v
    Bs, ss, psis = [], [], []
    for g, p, q in basis_terms(basis):
        sg = basis.sigma[g]
        raw = U ** p * V ** q * np.exp(-(U * U + V * V) / (2.0 * sg * sg))
        psi = 1.0 / math.sqrt(float(np.sum(raw * raw)))
        Bp = psi * raw
        sk = float(np.sum(Bp)) if (p % 2 == 0 and q % 2 == 0) else 0.0
        B = Bp.copy()
        B[h, h] -= sk
        Bs.append(B)
        ss.append(sk)
        psis.append(psi)
    return np.array(Bs), np.array(ss), np.array(psis)


def norm_coords(x, y, W, H):
    """Spatial coordinates scaled to [-1, 1] over the image."""
    xt = 2.0 * np.asarray(x, np.float64) / (W - 1) - 1.0 if W > 1 else np.zeros_like(x, np.float64)
    yt = 2.0 * np.asarray(y, np.float64) / (H - 1) - 1.0 if H > 1 else np.zeros_like(y, np.float64)
    return xt, yt


def spatial_values(x, y, W, H, S):
    """g_s(x, y) = xt^l yt^m for every spatial term, shape (N_s,) + shape(x)."""
    xt, yt = norm_coords(x, y, W, H)
    return np.array([xt ** l * yt ** m for l, m in spatial_terms(S)])


# ----------------------------------------------------------------------------------------
# Direct convolution (Eq. 12): O(x, y) = sum_{u,v} k(u, v) I(x-u, y-v), zero off the image
# ----------------------------------------------------------------------------------------

def shifted(img, du, dv):
    """Array J with J[y, x] = img[y - dv, x - du], zero where that falls off the image."""
    H, W = img.shape
    out = np.zeros_like(img)
    ys0, ys1 = max(0, dv), min(H, H + dv)
    xs0, xs1 = max(0, du), min(W, W + du)
    if ys0 < ys1 and xs0 < xs1:
        out[ys0:ys1, xs0:xs1] = img[ys0 - dv:ys1 - dv, xs0 - du:xs1 - du]
    return out


def direct_conv2d(img, K):
    """Direct 2-D convolution of a whole image with one kernel K[v+h, u+h] (Eq. 12)."""
    h = (K.shape[0] - 1) // 2
    img = np.asarray(img, np.float64)
    out = np.zeros_like(img)
    for v in range(-h, h + 1):
        for u in range(-h, h + 1):
            kv = K[v + h, u + h]
            if kv != 0.0:
                out += kv * shifted(img, u, v)
    return out


def conv_pixel(img, K, x, y):
    """Eq. 12 at one output pixel."""
    h = (K.shape[0] - 1) // 2
    H, W = img.shape
    acc = 0.0
    for v in range(-h, h + 1):
        yy = y - v
        if yy < 0 or yy >= H:
            continue
        for u in range(-h, h + 1):
            xx = x - u
            if 0 <= xx < W:
                acc += K[v + h, u + h] * float(img[yy, xx])
    return acc


# ----------------------------------------------------------------------------------------
# Stamp candidates (Sec. 3.3)
# ----------------------------------------------------------------------------------------

def lower_median_f32(values_f32):
    """Lower median ((n-1)//2-th order statistic) of a float32 array."""
    v = np.sort(np.asarray(values_f32, np.float32).ravel())
    if v.size == 0:
        raise OracleError("no unmasked pixels")
    return np.float32(v[(v.size - 1) // 2])


def extract_candidates(I1, I2, V1, V2, m1, m2, basis: Basis, cfg: Config):
    """Stamp candidates per subregion (Sec. 3.3).

    Readings: the detection image is S = I1 + I2 (float32 sum); the background is the lower
    median of S over pixels unmasked in both images; a source is a pixel that beats all of its
    8 neighbours under the order (value, -linear index); it is over threshold when
    (S - median) > thresh_nsigma * sqrt(V1 + V2) at the peak (float64 arithmetic on the float32
    inputs); its stamp footprint (radius s + h) must lie inside the image with no masked
    pixel (Sec. 3.3: no masked pixels that affect the kernel).  Subregion i spans
    floor(i W / nx) <= x < floor((i+1) W / nx) (likewise in y); candidates are ordered by
    (value descending, linear index ascending) and truncated to ``max_cand``.

    Returns an int32 array (n_regions, max_cand, 2) of (x, y), -1 for empty slots, regions in
    row-major order (region = j * nx + i), and the median.
    """
    H, W = I1.shape
    S = (np.asarray(I1, np.float32) + np.asarray(I2, np.float32)).astype(np.float32)
    bad = ((m1.astype(np.int64) | m2.astype(np.int64)) & cfg.badmask) != 0
    med = lower_median_f32(S[~bad])
    s, h = cfg.s(basis), basis.h
    R = s + h
    nx, ny = cfg.grid_nx, cfg.grid_ny
    cand = np.full((nx * ny, cfg.max_cand, 2), -1, np.int32)
    # footprint test: any masked pixel within Chebyshev radius R
    badi = bad.astype(np.int64)
    ii = np.zeros((H + 1, W + 1), np.int64)
    ii[1:, 1:] = np.cumsum(np.cumsum(badi, 0), 1)
    lists = [[] for _ in range(nx * ny)]
    thr_all = cfg.thresh_nsigma * np.sqrt(V1.astype(np.float64) + V2.astype(np.float64))
    for y in range(R, H - R):
        row_ok = (S[y, R:W - R].astype(np.float64) - np.float64(med)) > thr_all[y, R:W - R]
        for x in np.nonzero(row_ok)[0] + R:
            x = int(x)
            val = S[y, x]
            idx = y * W + x
            peak = True
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    nv = S[y + dy, x + dx]
                    nidx = (y + dy) * W + (x + dx)
                    if not (val > nv or (val == nv and idx < nidx)):
                        peak = False
            if not peak:
                continue
            nbad = ii[y + R + 1, x + R + 1] - ii[y - R, x + R + 1] - ii[y + R + 1, x - R] + ii[y - R, x - R]
            if nbad:
                continue
            rx = min(nx - 1, max(0, (x * nx) // W))
            while rx > 0 and x < (rx * W) // nx:
                rx -= 1
            while rx < nx - 1 and x >= ((rx + 1) * W) // nx:
                rx += 1
            ry = min(ny - 1, max(0, (y * ny) // H))
            while ry > 0 and y < (ry * H) // ny:
                ry -= 1
            while ry < ny - 1 and y >= ((ry + 1) * H) // ny:
                ry += 1
            lists[ry * nx + rx].append((-float(val), idx, x, y))
    for r, lst in enumerate(lists):
        lst.sort()
        for j, (_, _, x, y) in enumerate(lst[:cfg.max_cand]):
            cand[r, j] = (x, y)
    return cand, med


# ----------------------------------------------------------------------------------------
# Design matrix and normal equations (Eq. 3-6)
# ----------------------------------------------------------------------------------------

def _get(img, x0, y0, n, fill=0.0):
    """n x n window of img with top-left (x0, y0), ``fill`` off the image, float64."""
    H, W = img.shape
    out = np.full((n, n), fill, np.float64)
    xa, xb = max(0, x0), min(W, x0 + n)
    ya, yb = max(0, y0), min(H, y0 + n)
    if xa < xb and ya < yb:
        out[ya - y0:yb - y0, xa - x0:xb - x0] = img[ya:yb, xa:xb]
    return out


@dataclass
class StampData:
    x: int
    y: int
    C: np.ndarray        # (P, N_b) basis-convolved reference, C[p, k] = (B_k (x) R)(x_p, y_p)
    R: np.ndarray        # (P,) masked reference at the stamp pixels
    I2: np.ndarray       # (P,) science at the stamp pixels
    var: np.ndarray      # (P,) V1 + V2
    ok: np.ndarray       # (P,) pixel usable (unmasked, on image)
    F1: float            # footprint sum of R
    F2: float            # footprint sum of I2
    nfoot: int           # usable footprint pixels
    g: np.ndarray        # (N_s,) spatial factors at the stamp centre
    C2: np.ndarray = None  # (P, N_b) basis-convolved masked science (dual kernel), else None


def stamp_data(I1, I2, V1, V2, m1, m2, x, y, basis: Basis, cfg: Config, B=None) -> StampData:
    """Explicit design-matrix block of one stamp (Eq. 4): C[p, k] = sum_{u,v} B_k(u, v)
    R(x_p - u, y_p - v) over the (2s+1)^2 stamp pixels, R = I1 with masked pixels zeroed
    (Sec. 3.4: masked pixels do not contribute).  Also the footprint sums used by the
    normalisation (Sec. 3.2) and the spatial factors at the stamp centre (Sec. 2)."""
    if B is None:
        B, _, _ = basis_kernels(basis)
    H, W = I1.shape
    s, h = cfg.s(basis), basis.h
    n = 2 * (s + h) + 1
    bad = ((m1.astype(np.int64) | m2.astype(np.int64)) & cfg.badmask) != 0
    bad1 = (m1.astype(np.int64) & cfg.badmask) != 0
    Rimg = np.where(bad1, 0.0, I1.astype(np.float64))
    F = _get(Rimg, x - s - h, y - s - h, n)
    goodF = _get((~bad).astype(np.float64), x - s - h, y - s - h, n, fill=0.0) > 0.5
    I2F = _get(I2.astype(np.float64), x - s - h, y - s - h, n)
    P = (2 * s + 1) ** 2
    w = basis.w
    # patch matrix: Pm[p, t] = R(x_p - u_t, y_p - v_t), t = (v + h) * w + (u + h)
    Pm = np.empty((P, w * w))
    for v in range(-h, h + 1):
        for u in range(-h, h + 1):
            t = (v + h) * w + (u + h)
            y0 = h - v
            x0 = h - u
            Pm[:, t] = F[y0:y0 + 2 * s + 1, x0:x0 + 2 * s + 1].ravel()
    C = Pm @ B.reshape(B.shape[0], -1).T
    core = slice(h, h + 2 * s + 1)
    Rs = F[core, core].ravel()
    I2s = I2F[core, core].ravel()
    var = (_get(V1.astype(np.float64), x - s, y - s, 2 * s + 1)
           + _get(V2.astype(np.float64), x - s, y - s, 2 * s + 1)).ravel()
    ok = goodF[core, core].ravel()
    F1 = float(np.sum(np.where(goodF, F, 0.0)))
    F2 = float(np.sum(np.where(goodF, I2F, 0.0)))
    g = spatial_values(x, y, W, H, basis.S)
    C2 = None
    if cfg.dual:
        # the same basis applied to the science image, its masked pixels zeroed (Eq. 2 with
        # c_i != 0: the kernel terms g_i k_i (x) I2 join the design vector)
        bad2 = (m2.astype(np.int64) & cfg.badmask) != 0
        F2m = _get(np.where(bad2, 0.0, I2.astype(np.float64)), x - s - h, y - s - h, n)
        Pm2 = np.empty((P, w * w))
        for v in range(-h, h + 1):
            for u in range(-h, h + 1):
                t = (v + h) * w + (u + h)
                Pm2[:, t] = F2m[h - v:h - v + 2 * s + 1, h - u:h - u + 2 * s + 1].ravel()
        C2 = Pm2 @ B.reshape(B.shape[0], -1).T
    return StampData(x, y, C, Rs, I2s, var, ok, F1, F2, int(goodF.sum()), g, C2)


def solve_normalisation(stamps):
    """b0 and d0 by the unweighted fit of Sec. 3.2 (sigma = 1).

    Reading: the fit is made on per-stamp footprint sums, sum I2 = b0 sum I1 + d0 n_pix, so
    that b0 is the flux ratio (a pixel-wise two-term fit is biased when the PSFs differ)."""
    A = np.array([[st.F1, float(st.nfoot)] for st in stamps])
    y = np.array([st.F2 for st in stamps])
    M = A.T @ A
    v = A.T @ y
    b0, d0 = solve_spd(M, v)
    return float(b0), float(d0)


def solve_spd(M, v):
    """Solve M a = v by Cholesky, falling back to LU with partial pivoting."""
    try:
        L = np.linalg.cholesky(M)
        z = np.linalg.solve(L, v)
        return np.linalg.solve(L.T, z)
    except np.linalg.LinAlgError:
        try:
            return np.linalg.solve(M, v)
        except np.linalg.LinAlgError as e:
            raise OracleError("singular normal matrix") from e


# Numerical singularity of the normal equations (reading of the paper's "regular matrix
# methods", Eq. 5-6): a Cholesky pivot d_j within +-PIVOT_SINGULAR of its row's original
# diagonal M_jj leaves column j a combination of the earlier ones to within the working
# precision of a solve in ~48-bit arithmetic over a few hundred unknowns, so the system is
# singular; a pivot below -PIVOT_SINGULAR M_jj is indefiniteness by rounding and goes to LU.
PIVOT_SINGULAR = 1e-11


def _first_bad_pivot(M):
    """Relative size d_j / M_jj of the first pivot of a plain right-looking Cholesky of M that
    is not safely positive (within the singular band, negative or not finite); None if every
    pivot is above the band."""
    A = np.array(M, dtype=np.float64, copy=True)
    dg = np.diag(A).copy()
    n = A.shape[0]
    for j in range(n):
        d = A[j, j]
        if not np.isfinite(d) or d <= PIVOT_SINGULAR * dg[j]:
            return d / dg[j] if dg[j] != 0 else d
        l = A[j + 1:, j] / math.sqrt(d)
        A[j + 1:, j + 1:] -= np.outer(l, l)
    return None


def solve_normal(M, v):
    """Solve the normal equations M a = v (Eq. 5-6) by Cholesky, falling back to LU with
    partial pivoting when M is indefinite by rounding; OracleError("singular ...") when a pivot
    lies within the singular band (PIVOT_SINGULAR) or LU fails."""
    dg = np.diag(M)
    try:
        L = np.linalg.cholesky(M)
        if np.all(np.diag(L) ** 2 > PIVOT_SINGULAR * dg):
            z = np.linalg.solve(L, v)
            return np.linalg.solve(L.T, z)
    except np.linalg.LinAlgError:
        pass
    p = _first_bad_pivot(M)
    if p is not None and np.isfinite(p) and abs(p) <= PIVOT_SINGULAR:
        raise OracleError("singular normal matrix")
    try:
        a = np.linalg.solve(M, v)
    except np.linalg.LinAlgError as e:
        raise OracleError("singular normal matrix") from e
    if not np.all(np.isfinite(a)):
        raise OracleError("singular normal matrix")
    return a


def design_rows(st: StampData, n_s: int):
    """Rows of the concatenated design vector (Eq. 4) for the kernel terms of one stamp:
    A[p, k * N_s + s] = g_s(stamp centre) C[p, k]; with the dual kernel the terms applied to
    I2 follow, A[p, (N_b + k) * N_s + s] = g_s C2[p, k] (the c_i of Eq. 2)."""
    A = (st.C[:, :, None] * st.g[None, None, :]).reshape(st.C.shape[0], -1)
    if st.C2 is not None:
        A2 = (st.C2[:, :, None] * st.g[None, None, :]).reshape(st.C2.shape[0], -1)
        A = np.concatenate([A, A2], 1)
    return A


def penalty_terms(basis: Basis):
    """p_k = sum_{u,v} (u^2 + v^2)^2 k_k(u, v)^2 for each basis kernel (the penalty function of
    Yuan & Akerlof adopted in Sec. 2, before the scale Phi)."""
    B, _, _ = basis_kernels(basis)
    h = basis.h
    u = np.arange(-h, h + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    r4 = (U * U + V * V) ** 2
    return np.array([float(np.sum(r4 * Bk * Bk)) for Bk in B])


def add_penalty(M, basis: Basis, lam, offset=0):
    """Adds Phi p_i to the diagonal of the kernel unknowns (b_i and c_i; Eq. 5), each spatial
    term of a basis kernel taking that kernel's p_k.  Reading of Phi ("neither negligible nor
    dominant", Sec. 2): Phi = lam * sum_i M_ii / sum_i p_i over those unknowns, so that the
    penalty adds lam times the diagonal's total."""
    n_s = len(spatial_terms(basis.S))
    pk = penalty_terms(basis)
    n = 2 * len(pk) * n_s
    p = np.tile(np.repeat(pk, n_s), 2)
    idx = np.arange(offset, offset + n)
    phi = lam * float(np.trace(M[np.ix_(idx, idx)])) / float(p.sum())
    M = M.copy()
    M[idx, idx] += phi * p
    return M


def normal_equations(stamps, basis: Basis, mode: str, b0=None, d0=None, lam=0.0):
    """M and v of Eq. 5-6 with sigma^2 = V1 + V2, summed over the stamp pixels.

    mode "separate": unknowns are the kernel terms only, target I2 - b0 R - d0.
    mode "joint": unknowns are (b0, kernel terms, d0), target I2."""
    n_s = len(spatial_terms(basis.S))
    M = None
    v = None
    for st in stamps:
        A = design_rows(st, n_s)
        if mode == "joint":
            A = np.concatenate([st.R[:, None], A, np.ones((A.shape[0], 1))], 1)
            y = st.I2
        else:
            y = st.I2 - b0 * st.R - d0
        wgt = np.where(st.ok, 1.0 / st.var, 0.0)
        Mi = A.T @ (A * wgt[:, None])
        vi = A.T @ (wgt * y)
        M = Mi if M is None else M + Mi
        v = vi if v is None else v + vi
    if stamps and stamps[0].C2 is not None:
        M = add_penalty(M, basis, lam, 1 if mode == "joint" else 0)
    return M, v


@dataclass
class Solution:
    b0: float
    coeff: np.ndarray            # (N_b * N_s,) kernel coefficients, k-major, then d0 last
    d0: float
    basis: Basis
    W: int
    H: int
    cand: np.ndarray = None      # (n_regions, max_cand, 2)
    status: np.ndarray = None    # (n_regions, max_cand) STATUS_*
    chi2: np.ndarray = None      # (n_regions, max_cand) last chi^2 of each candidate (NaN if never used)
    chi2_mean: float = float("nan")
    chi2_rms: float = float("nan")
    n_iter: int = 0
    n_used: int = 0
    history: list = field(default_factory=list)
    dual: bool = False           # coeff holds (b terms, c terms, d0)

    @property
    def a(self):
        nb = len(basis_terms(self.basis))
        return self.coeff[:nb * len(spatial_terms(self.basis.S))].reshape(nb, -1)

    @property
    def c(self):
        """Coefficients of the terms applied to I2 (dual kernel), (N_b, N_s)."""
        nb, ns = len(basis_terms(self.basis)), len(spatial_terms(self.basis.S))
        return self.coeff[nb * ns:2 * nb * ns].reshape(nb, -1)


def stamp_model(st: StampData, sol_b0, a_flat, d0, n_s):
    return sol_b0 * st.R + design_rows(st, n_s) @ a_flat + d0


def stamp_chi2(st: StampData, b0, a_flat, d0, n_s, alpha):
    """Per-stamp quality (Sec. 3.6): mean over the stamp of residual^2 / (V1 + V2 + alpha |I2|),
    the variance softened by a scaled version of the flux (reading: alpha = 0.1 of |I2|)."""
    r = st.I2 - stamp_model(st, b0, a_flat, d0, n_s)
    den = st.var + alpha * np.abs(st.I2)
    q = np.where(st.ok, r * r / den, 0.0)
    return float(q.sum() / max(1, int(st.ok.sum())))


def solve_from_stamps(stamps, basis: Basis, cfg: Config):
    """One least-squares solve over a set of stamps; returns (b0, coeff, d0)."""
    n_s = len(spatial_terms(basis.S))
    lam = cfg.penalty if cfg.dual else 0.0
    if cfg.norm_mode == "joint":
        M, v = normal_equations(stamps, basis, "joint", lam=lam)
        a = solve_normal(M, v)
        return float(a[0]), a[1:-1], float(a[-1])
    b0, d0 = solve_normalisation(stamps)
    M, v = normal_equations(stamps, basis, "separate", b0, d0, lam)
    a = solve_normal(M, v)
    return b0, a, d0


def solve_kernel(I1, I2, V1, V2, m1, m2, basis: Basis, cfg: Config, cand=None) -> Solution:
    """Full solve with iterative stamp rejection (Sec. 3.3: discrepant stamps are removed and
    replaced over several solution iterations; Sec. 3.5: per-stamp matrices are built once).

    Reading of the rejection rule: after each solve, with chi^2 of every active stamp
    (``stamp_chi2``), reject stamps with chi^2 > mean + reject_nsigma * std (population std
    over active stamps) and replace each by the next candidate of its subregion; stop when
    nothing is rejected or after ``max_iter`` solves; fewer than 3 active stamps is an error
    (Sec. 3.7 cut "number of stamps used < 3").
    ``cand`` (n_regions, max_cand, 2) overrides the extractor."""
    H, W = I1.shape
    if cand is None:
        cand, _ = extract_candidates(I1, I2, V1, V2, m1, m2, basis, cfg)
    B, _, _ = basis_kernels(basis)
    n_reg, n_c = cand.shape[0], cand.shape[1]
    status = np.zeros((n_reg, n_c), np.int32)
    chi2 = np.full((n_reg, n_c), np.nan)
    ptr = np.zeros(n_reg, np.int64)
    cache = {}

    def get(r, j):
        if (r, j) not in cache:
            x, y = int(cand[r, j, 0]), int(cand[r, j, 1])
            cache[(r, j)] = stamp_data(I1, I2, V1, V2, m1, m2, x, y, basis, cfg, B)
        return cache[(r, j)]

    n_s = len(spatial_terms(basis.S))
    history = []
    n_iter = 0
    for it in range(cfg.max_iter):
        active = [(r, int(ptr[r])) for r in range(n_reg) if ptr[r] < n_c and cand[r, ptr[r], 0] >= 0]
        if len(active) < 3:
            raise TooFewStamps(f"{len(active)} stamps")
        b0, a, d0 = solve_from_stamps([get(r, j) for r, j in active], basis, cfg)
        n_iter = it + 1
        cs = np.array([stamp_chi2(get(r, j), b0, a, d0, n_s, cfg.soften_alpha) for r, j in active])
        for (r, j), c in zip(active, cs):
            chi2[r, j] = c
        mu, sd = float(cs.mean()), float(cs.std())
        history.append(dict(n_active=len(active), chi2_mean=mu, chi2_rms=sd))
        if it == cfg.max_iter - 1:
            break
        thr = mu + cfg.reject_nsigma * sd
        rej = [(r, j) for (r, j), c in zip(active, cs) if c > thr]
        history[-1]["rejected"] = rej
        history[-1]["threshold"] = thr
        if not rej:
            break
        for r, j in rej:
            status[r, j] = STATUS_REJECTED
            ptr[r] += 1
    for r, j in active:
        status[r, j] = STATUS_USED
    coeff = np.concatenate([a, [d0]])
    return Solution(b0, coeff, d0, basis, W, H, cand, status, chi2, mu, sd, n_iter, len(active),
                    history, cfg.dual)


# ----------------------------------------------------------------------------------------
# Applying the solution (Eq. 12-13, Sec. 3.4, Sec. 4.3-4.4)
# ----------------------------------------------------------------------------------------

def realise_kernel(sol: Solution, x, y):
    """K_{x,y}(u, v) = b0 delta + sum_k (sum_s a_{k,s} g_s(x, y)) B_k(u, v); [v+h, u+h]."""
    B, _, _ = basis_kernels(sol.basis)
    g = spatial_values(x, y, sol.W, sol.H, sol.basis.S)
    ak = sol.a @ g
    K = np.tensordot(ak, B, axes=(0, 0))
    h = sol.basis.h
    K[h, h] += sol.b0
    return K


def realise_kernel2(sol: Solution, x, y):
    """Dual kernel (Sec. 2): K2 = delta - sum_k (sum_s c_{k,s} g_s(x, y)) B_k, the kernel the
    difference applies to I2, so that D = K2 (x) I2 - K1 (x) I1 - d0."""
    B, _, _ = basis_kernels(sol.basis)
    g = spatial_values(x, y, sol.W, sol.H, sol.basis.S)
    K = -np.tensordot(sol.c @ g, B, axes=(0, 0))
    h = sol.basis.h
    K[h, h] += 1.0
    return K


def masked_ref(I1, m1, badmask):
    return np.where((m1.astype(np.int64) & badmask) != 0, 0.0, np.asarray(I1, np.float64))


def convolve_image(I1, m1, sol: Solution, badmask, I2=None, m2=None):
    """O(x, y) = sum_{u,v} K_{x,y}(u, v) R(x-u, y-v) + d0 over the whole image, R = I1 with
    masked pixels zeroed, K_{x,y} the kernel realised at the output pixel.  By linearity in
    the spatial factors this is sum_s g_s(x, y) (K_s (x) R)(x, y) with K_s = sum_k a_{k,s} B_k
    (plus b0 delta for the constant term).  With ``I2`` returns the difference I2 - O.  For a
    dual-kernel solution the terms sum_k c_k(x, y) B_k (x) R2 are added to O, R2 = I2 with the
    pixels masked in ``m2`` zeroed (Eq. 2), and the difference is returned."""
    B, _, _ = basis_kernels(sol.basis)
    H, W = I1.shape
    R = masked_ref(I1, m1, badmask)
    yy, xx = np.mgrid[0:H, 0:W]
    g = spatial_values(xx, yy, W, H, sol.basis.S)
    h = sol.basis.h
    out = np.full((H, W), sol.d0, np.float64)
    for si in range(g.shape[0]):
        Ks = np.tensordot(sol.a[:, si], B, axes=(0, 0))
        if si == 0:
            Ks = Ks.copy()
            Ks[h, h] += sol.b0
        out += g[si] * direct_conv2d(R, Ks)
    if sol.dual:
        R2 = masked_ref(I2, m2, badmask)
        for si in range(g.shape[0]):
            out += g[si] * direct_conv2d(R2, np.tensordot(sol.c[:, si], B, axes=(0, 0)))
    if I2 is not None:
        return np.asarray(I2, np.float64) - out
    return out


def _masked_window(img, m, badmask, x, y, h):
    """(2h+1)^2 window of img centred on (x, y) with masked and off-image pixels zero, and the
    window's own centre coordinates (h, h)."""
    H, W = img.shape
    out = np.zeros((2 * h + 1, 2 * h + 1))
    ya, yb, xa, xb = max(0, y - h), min(H, y + h + 1), max(0, x - h), min(W, x + h + 1)
    sub = np.asarray(img[ya:yb, xa:xb], np.float64)
    ok = (m[ya:yb, xa:xb].astype(np.int64) & badmask) == 0
    out[ya - (y - h):yb - (y - h), xa - (x - h):xb - (x - h)] = np.where(ok, sub, 0.0)
    return out


def convolve_pixel(I1, m1, sol: Solution, badmask, x, y, I2=None, m2=None):
    """Eq. 12 at one output pixel with the kernel realised there (plus d0); for a dual-kernel
    solution plus the terms applied to I2 (masked by m2)."""
    h = sol.basis.h
    R = _masked_window(I1, m1, badmask, x, y, h)
    o = conv_pixel(R, realise_kernel(sol, x, y), h, h) + sol.d0
    if sol.dual:
        R2 = _masked_window(I2, m2, badmask, x, y, h)
        Kc = np.zeros_like(R2) - realise_kernel2(sol, x, y)
        Kc[h, h] += 1.0
        o += conv_pixel(R2, Kc, h, h)
    return o


def tile_centres(n, tile):
    """Tiles [t*tile, min(n, (t+1)*tile)) and the centre of each tile's actual extent."""
    starts = np.arange(0, n, tile)
    ends = np.minimum(starts + tile, n)
    return starts, ends, (starts + ends - 1) / 2.0


def pseudo_conv(K, C_in):
    """Covariance pseudo-matrix of K (x) (noise with pseudo-matrix C_in), unnormalised
    (Eq. 10-11 written for a convolution): C(D) = sum_a sum_b K(a) K(b) C_in(D + a - b).
    Output size 2w + c - 2 for a w x w kernel and c x c input (Sec. 4.3).  Computed as
    T = K (x) C_in followed by the correlation of T with K."""
    w = K.shape[0]
    c = C_in.shape[0]
    n = 2 * w + c - 2
    # T = K (x) C_in, size w + c - 1
    T = np.zeros((w + c - 1, w + c - 1))
    for i in range(w):
        for j in range(w):
            if K[i, j] != 0.0:
                T[i:i + c, j:j + c] += K[i, j] * C_in
    # C(D) = sum_a K(a) T(D + a), D spans [-(w-1) - (w+c-2)/2 ...]; place by offsets
    out = np.zeros((n, n))
    # index of zero lag in T is (w-1)/2 + (c-1)/2; in out it is (n-1)/2
    for i in range(w):
        for j in range(w):
            if K[i, j] != 0.0:
                # a = (i - h, j - h); out[D] += K(a) T(D + a)  =>  out index = T index - a + shift
                out[w - 1 - i:w - 1 - i + w + c - 1, w - 1 - j:w - 1 - j + w + c - 1] += K[i, j] * T
    return out


def covariance_factor(K, C_in):
    """Central value of pseudo_conv(K, C_in) divided by sum K^2 (Sec. 4.3, the factor
    K = [sum k^2]^-1 absorbed in the pseudo-matrix; Sec. 4.4 per-patch factor)."""
    w = K.shape[0]
    c = C_in.shape[0]
    hc = (c - 1) // 2
    h = (w - 1) // 2
    # (K * C_in * K)(0) = sum_a sum_b K(a) K(b) C_in(a - b)
    tot = 0.0
    for dy in range(-hc, hc + 1):
        for dx in range(-hc, hc + 1):
            cv = C_in[dy + hc, dx + hc]
            if cv == 0.0:
                continue
            # sum_a K(a) K(a - d)
            tot += cv * float(np.sum(K * shifted(K, dx, dy)))
    return tot / float(np.sum(K * K))


def variance_image(V1, m1, sol: Solution, badmask, tile=64, C_in=None, V2=None, m2=None):
    """V'(x, y) = f_t sum_{u,v} K_t(u, v)^2 V1(x-u, y-v) (Eq. 13), K_t realised at the centre
    of the fixed tile t (Sec. 4.4: a constant kernel per patch), f_t the covariance factor of
    K_t (1 for white input).  With ``V2`` returns V2 + V' (Sec. 4.4: variances of a difference
    add)."""
    H, W = V1.shape
    Vm = masked_ref(V1, m1, badmask)
    if C_in is None:
        C_in = np.ones((1, 1))
    xs0, xs1, xc = tile_centres(W, tile)
    ys0, ys1, yc = tile_centres(H, tile)
    h = sol.basis.h
    out = np.zeros((H, W))
    for ty in range(len(ys0)):
        for tx in range(len(xs0)):
            K = realise_kernel(sol, xc[tx], yc[ty])
            f = covariance_factor(K, C_in)
            K2 = K * K
            ya, yb, xa, xb = ys0[ty], ys1[ty], xs0[tx], xs1[tx]
            sub = _get(Vm, int(xa) - h, int(ya) - h, max(yb - ya, xb - xa) + 2 * h)
            acc = np.zeros((yb - ya, xb - xa))
            for v in range(-h, h + 1):
                for u in range(-h, h + 1):
                    acc += K2[v + h, u + h] * sub[h - v:h - v + yb - ya, h - u:h - u + xb - xa]
            out[ya:yb, xa:xb] = f * acc
    if sol.dual:
        # Var(K2 (x) I2) with K2 = delta - sum c_k B_k per tile, the masked pixels of I2
        # contributing zero (white inputs)
        V2m = masked_ref(V2, m2, badmask)
        for ty in range(len(ys0)):
            for tx in range(len(xs0)):
                K2 = realise_kernel2(sol, xc[tx], yc[ty]) ** 2
                ya, yb, xa, xb = ys0[ty], ys1[ty], xs0[tx], xs1[tx]
                sub = _get(V2m, int(xa) - h, int(ya) - h, max(yb - ya, xb - xa) + 2 * h)
                acc = np.zeros((yb - ya, xb - xa))
                for v in range(-h, h + 1):
                    for u in range(-h, h + 1):
                        acc += K2[v + h, u + h] * sub[h - v:h - v + yb - ya, h - u:h - u + xb - xa]
                out[ya:yb, xa:xb] += acc
        return out
    if V2 is not None:
        out = out + np.asarray(V2, np.float64)
    return out


def variance_pixel(V1, m1, sol: Solution, badmask, x, y, tile=64, C_in=None, V2=None, m2=None):
    """Eq. 13 at one output pixel: f_t sum_{u,v} K_t(u, v)^2 V1(x-u, y-v) with K_t realised at
    the centre of the fixed tile that contains (x, y) (same tiles as ``variance_image``)."""
    H, W = V1.shape
    xa = (x // tile) * tile
    ya = (y // tile) * tile
    xc = (xa + min(W, xa + tile) - 1) / 2.0
    yc = (ya + min(H, ya + tile) - 1) / 2.0
    K = realise_kernel(sol, xc, yc)
    f = 1.0 if C_in is None else covariance_factor(K, C_in)
    h = sol.basis.h
    v = f * conv_pixel(_masked_window(V1, m1, badmask, x, y, h), K * K, h, h)
    if sol.dual:
        K2 = realise_kernel2(sol, xc, yc)
        return v + conv_pixel(_masked_window(V2, m2, badmask, x, y, h), K2 * K2, h, h)
    if V2 is not None:
        v += float(V2[y, x])
    return v


def r_bad(sol: Solution, bad_frac=0.2, second=False):
    """Box radius of CONV.BAD (Sec. 3.4): smallest r in [0, h] such that the sum of K^2 outside
    the box max(|u|, |v|) <= r is at most ``bad_frac`` of the total, K realised at the image
    centre (``second``: the dual kernel K2 applied to I2)."""
    realise = realise_kernel2 if second else realise_kernel
    K = realise(sol, (sol.W - 1) / 2.0, (sol.H - 1) / 2.0)
    h = sol.basis.h
    K2 = K * K
    tot = float(K2.sum())
    u = np.arange(-h, h + 1)
    cheb = np.maximum(np.abs(u)[:, None], np.abs(u)[None, :])
    for r in range(h + 1):
        if float(K2[cheb > r].sum()) <= bad_frac * tot:
            return r
    return h


QUALITY_FEW_STAMPS, QUALITY_MEAN_DEV, QUALITY_RMS_DEV = 1, 2, 4
QUALITY_MOMENT1, QUALITY_MOMENT2, QUALITY_DECONV = 8, 16, 32


def kernel_quality(K):
    """Diagnostics of one realised kernel K[v+h, u+h] (Sec. 3.7): its sum, first moments
    (sum u K / sum K, sum v K / sum K), central second moments, and the deconvolution measure:
    the kernel sum enclosed within radius r (u^2 + v^2 <= r^2) relative to the total, at its
    maximum over r = 0..h."""
    h = (K.shape[0] - 1) // 2
    U, V = np.meshgrid(np.arange(-h, h + 1, dtype=np.float64),
                       np.arange(-h, h + 1, dtype=np.float64))
    ks = float(K.sum())
    mx, my = float((U * K).sum()) / ks, float((V * K).sum()) / ks
    mxx = float(((U - mx) ** 2 * K).sum()) / ks
    myy = float(((V - my) ** 2 * K).sum()) / ks
    mxy = float(((U - mx) * (V - my) * K).sum()) / ks
    r2 = U * U + V * V
    deconv = max(float(K[r2 <= r * r].sum()) / ks for r in range(h + 1))
    return dict(kernel_sum=ks, mom_x=mx, mom_y=my, mom_xx=mxx, mom_yy=myy, mom_xy=mxy,
                deconv_max=deconv)


def quality(sol: Solution, n_used, chi2_mean, chi2_rms):
    """Quality record of a solution (Sec. 3.7): ``kernel_quality`` of the kernel realised at the
    image centre plus the paper's recommended cuts as flags (reading: the normalised mean and
    r.m.s. deviations are the mean and population std of the stamps' softened chi^2)."""
    q = kernel_quality(realise_kernel(sol, (sol.W - 1) / 2.0, (sol.H - 1) / 2.0))
    f = 0
    if n_used < 3:
        f |= QUALITY_FEW_STAMPS
    if chi2_mean > 0.5:
        f |= QUALITY_MEAN_DEV
    if chi2_rms > 0.3:
        f |= QUALITY_RMS_DEV
    if abs(q["mom_x"]) > 0.5 or abs(q["mom_y"]) > 0.5:
        f |= QUALITY_MOMENT1
    if q["mom_xx"] < 0 or q["mom_yy"] < 0:
        f |= QUALITY_MOMENT2
    if q["deconv_max"] > 1.03:
        f |= QUALITY_DECONV
    q["flags"] = f
    return q


def mask_image(m1, sol: Solution, cfg: Config, m2=None, rb=None):
    """Output mask (Sec. 3.4): m1 (| m2 for a difference) plus CONV.BAD where a masked pixel of
    the convolved image, or the image edge, lies within Chebyshev distance r_bad, else
    CONV.POOR where one lies within h."""
    H, W = m1.shape
    h = sol.basis.h
    if rb is None:
        rb = r_bad(sol, cfg.bad_frac)
    bad = (m1.astype(np.int64) & cfg.badmask) != 0
    padded = np.ones((H + 2 * h, W + 2 * h), bool)
    padded[h:h + H, h:h + W] = bad

    def near(r):
        out = np.zeros((H, W), bool)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                out |= padded[h + dy:h + dy + H, h + dx:h + dx + W]
        return out

    nb = near(rb)
    npoor = near(h)
    if sol.dual and m2 is not None:
        # both images are convolved: masked pixels of I2 spread through K2 the same way
        bad = (m2.astype(np.int64) & cfg.badmask) != 0
        padded = np.ones((H + 2 * h, W + 2 * h), bool)
        padded[h:h + H, h:h + W] = bad
        nb = nb | near(r_bad(sol, cfg.bad_frac, second=True))
        npoor = npoor | near(h)
    out = m1.astype(np.int64)
    if m2 is not None:
        out = out | m2.astype(np.int64)
    out = np.where(nb, out | cfg.conv_bad, out)
    out = np.where(~nb & npoor, out | cfg.conv_poor, out)
    return out.astype(np.uint16)


def mask_pixel(m1, sol: Solution, cfg: Config, x, y, m2=None, rb=None):
    """Output mask of one pixel (Sec. 3.4), by the same rule as ``mask_image``: CONV.BAD when a
    badmask pixel of m1 or the image edge lies within Chebyshev distance r_bad, else CONV.POOR
    when one lies within h."""
    H, W = m1.shape
    h = sol.basis.h
    if rb is None:
        rb = r_bad(sol, cfg.bad_frac)
    near_bad = near_poor = False
    rb2 = r_bad(sol, cfg.bad_frac, second=True) if (sol.dual and m2 is not None) else -1
    for dy in range(-h, h + 1):
        for dx in range(-h, h + 1):
            yy, xx = y + dy, x + dx
            off = not (0 <= yy < H and 0 <= xx < W)
            masked = off or (int(m1[yy, xx]) & cfg.badmask) != 0
            if masked:
                near_poor = True
                if max(abs(dx), abs(dy)) <= rb:
                    near_bad = True
            if rb2 >= 0 and (off or (int(m2[yy, xx]) & cfg.badmask) != 0):
                near_poor = True
                if max(abs(dx), abs(dy)) <= rb2:
                    near_bad = True
    out = int(m1[y, x])
    if m2 is not None:
        out |= int(m2[y, x])
    if near_bad:
        out |= cfg.conv_bad
    elif near_poor:
        out |= cfg.conv_poor
    return out


def pseudo_matrix(sol: Solution, cfg: Config, C_in=None, second=False):
    """Average covariance pseudo-matrix of the convolved image (Sec. 4.4): the mean over a
    cov_grid x cov_grid sample of kernels, at ((i + 1/2) W / n, (j + 1/2) H / n), of
    pseudo_conv(K, C_in) / sum K^2, divided by its central value (the covariance factor has
    already gone into the variance map)."""
    if C_in is None:
        C_in = np.ones((1, 1))
    n = cfg.cov_grid
    acc = None
    realise = realise_kernel2 if second else realise_kernel
    for j in range(n):
        for i in range(n):
            K = realise(sol, (i + 0.5) * sol.W / n, (j + 0.5) * sol.H / n)
            P = pseudo_conv(K, C_in) / float(np.sum(K * K))
            acc = P if acc is None else acc + P
    acc /= n * n
    c = (acc.shape[0] - 1) // 2
    return acc / acc[c, c]


def embed_centre(P, n):
    out = np.zeros((n, n))
    c = P.shape[0]
    o = (n - c) // 2
    out[o:o + c, o:o + c] = P
    return out


def combine_pseudo(Ps, weights):
    """Weighted average of pseudo-matrices (Sec. 4.4: adding or subtracting images), each
    embedded at the common centre."""
    n = max(P.shape[0] for P in Ps)
    acc = sum(wt * embed_centre(P, n) for P, wt in zip(Ps, weights))
    return acc / float(sum(weights))


def mean_unmasked(V, mask, cfg: Config):
    ok = (mask.astype(np.int64) & (cfg.badmask | cfg.conv_bad)) == 0
    return float(np.mean(np.asarray(V, np.float64)[ok])) if ok.any() else 0.0


def subtract(I1, I2, V1, V2, m1, m2, sol: Solution, cfg: Config, C1=None, C2=None):
    """Difference image D = I2 - (K (x) I1 + d0), its variance V2 + V', mask and pseudo-matrix
    (Sec. 4.4: variances sum; pseudo-matrices averaged with the mean variances as weights)."""
    if sol.dual:
        # D = K2 (x) I2 - K1 (x) I1 - d0 (Eq. 2): two convolved parts with independent noise;
        # their pseudo-matrices are averaged with the mean variances as weights (Sec. 4.4)
        D = convolve_image(I1, m1, sol, cfg.badmask, I2, m2)
        M = mask_image(m1, sol, cfg, m2)
        V1p = variance_image(V1, m1, replace(sol, dual=False), cfg.badmask, cfg.var_tile)
        Vd = variance_image(V1, m1, sol, cfg.badmask, cfg.var_tile, V2=V2, m2=m2)
        w1, w2 = mean_unmasked(V1p, M, cfg), mean_unmasked(Vd - V1p, M, cfg)
        P = combine_pseudo([pseudo_matrix(sol, cfg), pseudo_matrix(sol, cfg, second=True)],
                           [w1, w2])
        return D, Vd, M, P
    D = convolve_image(I1, m1, sol, cfg.badmask, I2)
    Vp = variance_image(V1, m1, sol, cfg.badmask, cfg.var_tile, C1)
    M = mask_image(m1, sol, cfg, m2)
    P1 = pseudo_matrix(sol, cfg, C1)
    if C2 is None:
        C2 = np.ones((1, 1))
    w1 = mean_unmasked(Vp, M, cfg)
    w2 = mean_unmasked(V2, M, cfg)
    P = combine_pseudo([P1, C2], [w1, w2])
    return D, Vp + np.asarray(V2, np.float64), M, P


# ----------------------------------------------------------------------------------------
# Stacking (Sec. 5.1)
# ----------------------------------------------------------------------------------------

def resample_pseudo(C_in, scale):
    """Pseudo-matrix of an image resampled by a non-integer scale (Sec. 4.4): bilinear
    interpolation of C_in at the input lags scale * D for output lags D (zero beyond C_in),
    then the entries off the centre scaled so that their sum is C_in's sum off the centre (the
    total covariance excluding the variance is kept).  Readings: the centre is C_in's; the
    output radius is floor(r_in / scale) (ratio rounded to 1e-9)."""
    C_in = np.asarray(C_in, np.float64)
    w_in = C_in.shape[0]
    r_in = (w_in - 1) // 2
    r = int(math.floor(r_in / scale + 1e-9))
    w = 2 * r + 1
    out = np.zeros((w, w))

    def at(x, y):
        return C_in[y, x] if 0 <= x < w_in and 0 <= y < w_in else 0.0

    for j in range(w):
        for i in range(w):
            px, py = scale * (i - r) + r_in, scale * (j - r) + r_in
            x0, y0 = int(math.floor(px)), int(math.floor(py))
            fx, fy = px - x0, py - y0
            out[j, i] = ((1 - fy) * ((1 - fx) * at(x0, y0) + fx * at(x0 + 1, y0)) +
                         fy * ((1 - fx) * at(x0, y0 + 1) + fx * at(x0 + 1, y0 + 1)))
    off = np.ones((w, w), bool)
    off[r, r] = False
    s_out = float(out[off].sum())
    s_in = float(C_in.sum() - C_in[r_in, r_in])
    if s_out != 0.0:
        out[off] *= s_in / s_out
    return out


def psf_profile_circular(r2, fwhm, moffat_frac, beta):
    """Circular PSF profile scaled to peak 1: the flux-normalised mixture (1 - a) Gaussian +
    a Moffat(beta) with a common FWHM, divided by its central value."""
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    g0 = 1.0 / (2.0 * math.pi * sig * sig)
    g = g0 * np.exp(-0.5 * r2 / (sig * sig))
    m = np.zeros_like(r2, dtype=np.float64)
    m0 = 0.0
    if moffat_frac > 0:
        al2 = fwhm * fwhm / (4.0 * (2.0 ** (1.0 / beta) - 1.0))
        m0 = (beta - 1.0) / (math.pi * al2)
        m = m0 * (1.0 + r2 / al2) ** (-beta)
    a = moffat_frac
    return ((1.0 - a) * g + a * m) / ((1.0 - a) * g0 + a * m0)


def envelope_fwhm(models, radius=0):
    """Envelope PSF of stack inputs (Sec. 5.1): each input's PSF realised as a circular profile
    with a common peak (readings: circular FWHM sqrt(major * minor), the same mixture), the
    maximum taken pixel by pixel over the offsets |u|, |v| <= R, and a circular Gaussian
    A exp(-r^2 / 2 s^2) fitted to it by least squares (A, s); returns 2 sqrt(2 ln 2) s.
    R = radius, or ceil(3 x the widest circular FWHM) when 0.  The fit: A eliminated
    (A = sum E g / sum g^2), s maximising (sum E g)^2 / sum g^2 over [0.2 s_min, 4 s_max]
    (the input Gaussian widths) by a dense scan then a bounded scalar minimisation."""
    from scipy.optimize import minimize_scalar
    fw = [math.sqrt(m[0] * m[1]) for m in models]
    R = radius if radius else int(math.ceil(3.0 * max(fw)))
    u = np.arange(-R, R + 1, dtype=np.float64)
    U, V = np.meshgrid(u, u)
    r2 = U * U + V * V
    E = np.zeros_like(r2)
    for f, (_, _, a, beta) in zip(fw, models):
        E = np.maximum(E, psf_profile_circular(r2, f, a, beta))
    k = 2.0 * math.sqrt(2.0 * math.log(2.0))

    def neg_h(s):
        g = np.exp(-0.5 * r2 / (s * s))
        return -float(np.sum(E * g)) ** 2 / float(np.sum(g * g))

    lo, hi = 0.2 * min(fw) / k, 4.0 * max(fw) / k
    grid = lo * (hi / lo) ** np.linspace(0.0, 1.0, 2001)
    vals = [neg_h(s) for s in grid]
    j = int(np.argmin(vals))
    a, b = grid[max(0, j - 1)], grid[min(len(grid) - 1, j + 1)]
    res = minimize_scalar(neg_h, bounds=(a, b), method="bounded",
                          options={"xatol": 1e-12 * b})
    return k * float(res.x)


def render_target(W, H, sources, fwhm, radius=None):
    """Fake target image (Sec. 5.1): circular Gaussian of the given FWHM at each source
    position, sampled at pixel centres, flux-normalised, on a zero background."""
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    if radius is None:
        radius = int(math.ceil(5.0 * sig))
    T = np.zeros((H, W))
    for x0, y0, f in sources:
        xi, yi = int(round(x0)), int(round(y0))
        xa, xb = max(0, xi - radius), min(W, xi + radius + 1)
        ya, yb = max(0, yi - radius), min(H, yi + radius + 1)
        if xa >= xb or ya >= yb:
            continue
        yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
        T[ya:yb, xa:xb] += f * np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * sig * sig)) / (2 * math.pi * sig * sig)
    return T


def stack(warps, sources, target_fwhm, bases, cfg: Config):
    """PSF-homogenised stack (Sec. 5.1, Sec. 5.2): each input is matched (c_i = 0) to a fake
    target rendered at the source positions, convolved with its kernel (image, variance,
    mask), and the convolved inputs are averaged per pixel with weights w_i = 1 / mean(V'_i)
    (reading: the paper's "weights set to the mean variance" as inverse-variance weights).
    Returns (image, variance, mask, count, pseudo-matrix, per-warp solutions)."""
    H, W = warps[0]["image"].shape
    T = render_target(W, H, sources, target_fwhm).astype(np.float32)
    zero = np.zeros((H, W), np.float32)
    zm = np.zeros((H, W), np.uint16)
    num = np.zeros((H, W))
    den = np.zeros((H, W))
    var = np.zeros((H, W))
    cnt = np.zeros((H, W), np.int32)
    Ps, pw, sols = [], [], []
    for wp, basis in zip(warps, bases):
        sol = solve_kernel(wp["image"], T, wp["var"], zero, wp["mask"], zm, basis, cfg)
        O = convolve_image(wp["image"], wp["mask"], sol, cfg.badmask)
        Vp = variance_image(wp["var"], wp["mask"], sol, cfg.badmask, cfg.var_tile)
        M = mask_image(wp["mask"], sol, cfg)
        ok = (M.astype(np.int64) & (cfg.badmask | cfg.conv_bad)) == 0
        mv = mean_unmasked(Vp, M, cfg)
        wgt = 1.0 / mv
        num += np.where(ok, wgt * O, 0.0)
        den += np.where(ok, wgt, 0.0)
        var += np.where(ok, wgt * wgt * Vp, 0.0)
        cnt += ok.astype(np.int32)
        Ps.append(pseudo_matrix(sol, cfg))
        pw.append(wgt * wgt * mv)
        sols.append(sol)
    img = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    vout = np.where(den > 0, var / np.where(den > 0, den * den, 1.0), 0.0)
    mout = np.where(cnt == 0, 1, 0).astype(np.uint16)
    P = combine_pseudo(Ps, pw)
    return img, vout, mout, cnt, P, sols


STACK_REJECT = 1 << 13


def stack_full(warps, sources, target_fwhm, bases, cfg: Config, clip_nsigma=5.0,
               reject_bit=STACK_REJECT):
    """PSF-homogenised stack with outlier rejection and the unconvolved companion stack
    (Sec. 5.1).  Readings where the paper is silent:

    * an outlier is a usable pixel of convolved input i, at a pixel where at least 3 inputs
      are usable, whose deviation from the median m of the usable convolved inputs there
      exceeds ``clip_nsigma`` times its error softened like the chi^2 of Sec. 3.6,
      |I'_i - m| > n sqrt(V'_i + alpha |m|) with alpha = cfg.soften_alpha (the median, unlike
      a mean, is not dragged by the outlier itself);
    * the matched filter that carries the outlier mask back to the unconvolved input is the
      CONV.BAD box of that input's kernel: an input pixel is rejected when an outlier lies
      within Chebyshev distance r_bad of it (the pixels that dominate the outlier's value);
    * rejected input pixels are masked (``reject_bit``) and the inputs convolved again with
      their unchanged kernels; weights stay w_i = 1 / mean(V'_i) from the first pass;
    * the unconvolved stack combines the original inputs with the same weights and the same
      rejected pixels excluded.

    Returns dict(conv=(I, V, mask, count), unconv=(I, V, mask, count), rejected=[outlier
    pixels per input], outliers=[outlier map per input], margins=[|I'_i - m| minus the
    threshold, NaN where input i is not tested], pass1=[(I'_i, V'_i, usable_i)], sols=[...],
    pm=pseudo-matrix of the convolved stack)."""
    H, W = warps[0]["image"].shape
    T = render_target(W, H, sources, target_fwhm).astype(np.float32)
    zero = np.zeros((H, W), np.float32)
    zm = np.zeros((H, W), np.uint16)
    sols, conv, wts = [], [], []
    for wp, basis in zip(warps, bases):
        sol = solve_kernel(wp["image"], T, wp["var"], zero, wp["mask"], zm, basis, cfg)
        O = convolve_image(wp["image"], wp["mask"], sol, cfg.badmask)
        Vp = variance_image(wp["var"], wp["mask"], sol, cfg.badmask, cfg.var_tile)
        M = mask_image(wp["mask"], sol, cfg)
        ok = (M.astype(np.int64) & (cfg.badmask | cfg.conv_bad)) == 0
        sols.append(sol)
        conv.append((O, Vp, ok))
        wts.append(1.0 / mean_unmasked(Vp, M, cfg))
    stackO = np.stack([np.where(ok, O, np.nan) for O, Vp, ok in conv])
    nuse = np.sum(np.isfinite(stackO), axis=0)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)  # pixels with no usable input
        med = np.nanmedian(np.where(nuse >= 3, stackO, np.nan), axis=0)
    rejected, bad_in, outliers, margins = [], [], [], []
    for (O, Vp, ok), w, sol in zip(conv, wts, sols):
        has = ok & (nuse >= 3)
        m = np.where(has, med, 0.0)
        margin = np.abs(O - m) - clip_nsigma * np.sqrt(Vp + cfg.soften_alpha * np.abs(m))
        out = has & (margin > 0.0)
        rejected.append(int(out.sum()))
        outliers.append(out)
        margins.append(np.where(has, margin, np.nan))
        rb = r_bad(sol, cfg.bad_frac)
        pad = np.zeros((H + 2 * rb, W + 2 * rb), bool)
        pad[rb:rb + H, rb:rb + W] = out
        grown = np.zeros((H, W), bool)
        for dy in range(-rb, rb + 1):
            for dx in range(-rb, rb + 1):
                grown |= pad[rb + dy:rb + dy + H, rb + dx:rb + dx + W]
        bad_in.append(grown)
    cfg2 = Config(**{**cfg.__dict__, "badmask": cfg.badmask | reject_bit})
    num = np.zeros((H, W)); den = np.zeros((H, W)); var = np.zeros((H, W))
    cnt = np.zeros((H, W), np.int32)
    unum = np.zeros((H, W)); uden = np.zeros((H, W)); uvar = np.zeros((H, W))
    ucnt = np.zeros((H, W), np.int32)
    for wp, sol, w, bad in zip(warps, sols, wts, bad_in):
        m2 = np.where(bad, wp["mask"] | reject_bit, wp["mask"]).astype(np.uint16)
        O = convolve_image(wp["image"], m2, sol, cfg2.badmask)
        Vp = variance_image(wp["var"], m2, sol, cfg2.badmask, cfg.var_tile)
        M = mask_image(m2, sol, cfg2)
        ok = (M.astype(np.int64) & (cfg2.badmask | cfg.conv_bad)) == 0
        num += np.where(ok, w * O, 0.0)
        den += np.where(ok, w, 0.0)
        var += np.where(ok, w * w * Vp, 0.0)
        cnt += ok.astype(np.int32)
        uok = (m2.astype(np.int64) & cfg2.badmask) == 0
        I = np.asarray(wp["image"], np.float64)
        Vin = np.asarray(wp["var"], np.float64)
        unum += np.where(uok, w * I, 0.0)
        uden += np.where(uok, w, 0.0)
        uvar += np.where(uok, w * w * Vin, 0.0)
        ucnt += uok.astype(np.int32)

    def finish(nm, dn, vr, ct):
        img = np.where(dn > 0, nm / np.where(dn > 0, dn, 1.0), 0.0)
        v = np.where(dn > 0, vr / np.where(dn > 0, dn * dn, 1.0), 0.0)
        return img, v, np.where(ct == 0, 1, 0).astype(np.uint16), ct

    Ps = [pseudo_matrix(sol, cfg) for sol in sols]
    return dict(conv=finish(num, den, var, cnt), unconv=finish(unum, uden, uvar, ucnt),
                rejected=rejected, outliers=outliers, margins=margins, pass1=conv, sols=sols,
                pm=combine_pseudo(Ps, wts), weights=wts)


# ----------------------------------------------------------------------------------------
# Binning (Sec. 4.3: binning as a box convolution followed by a change of scale)
# ----------------------------------------------------------------------------------------

def box_pseudo(C_in, b):
    """Pseudo-matrix of a b x b box sum of noise with pseudo-matrix C_in (unnormalised):
    pseudo_conv with the box kernel of ones (Eq. 10-11 written for the box)."""
    return pseudo_conv(np.ones((b, b)), C_in)


def bin_image(img, var, mask, b, badmask, C_in=None):
    """Integer binning by b (Sec. 4.3).  Output pixel (X, Y) covers input pixels
    [bX, bX + b) x [bY, bY + b) (partial blocks at the far edges are dropped).  Readings: the
    binned image is the sum of the block's unmasked pixels (flux kept); its mask the OR of the
    block's masks; its variance the covariance factor of the box times the sum of the block's
    unmasked variances, f = (box * C_in * box)(0) / b^2, like the per-patch factor of a
    convolution (Sec. 4.4); the binned pseudo-matrix is the box pseudo-matrix sampled at lags
    that are multiples of b and normalised to centre 1.  Returns (image, variance, mask,
    pseudo-matrix)."""
    if C_in is None:
        C_in = np.ones((1, 1))
    H, W = img.shape
    Hb, Wb = H // b, W // b
    ok = (mask.astype(np.int64) & badmask) == 0
    I = np.where(ok, np.asarray(img, np.float64), 0.0)[:Hb * b, :Wb * b]
    V = np.where(ok, np.asarray(var, np.float64), 0.0)[:Hb * b, :Wb * b]
    M = mask.astype(np.int64)[:Hb * b, :Wb * b]
    Ib = I.reshape(Hb, b, Wb, b).sum(axis=(1, 3))
    Vb = V.reshape(Hb, b, Wb, b).sum(axis=(1, 3))
    Mb = np.zeros((Hb, Wb), np.int64)
    for dy in range(b):
        for dx in range(b):
            Mb |= M[dy::b, dx::b]
    Pbox = box_pseudo(C_in, b)
    c = (Pbox.shape[0] - 1) // 2
    f = Pbox[c, c] / (b * b)
    r = c // b
    Pb = Pbox[c - r * b:c + r * b + 1:b, c - r * b:c + r * b + 1:b]
    return Ib, f * Vb, Mb.astype(np.uint16), Pb / Pb[r, r]
