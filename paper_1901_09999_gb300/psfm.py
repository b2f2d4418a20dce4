"""Python binding of libpsfm (the C ABI declared in include/psfm.h).

The functions named like the C entry points (``psfm_solve_kernel``, ``psfm_convolve``,
``psfm_subtract``, ``psfm_stack``, ``psfm_workspace_size`` ...) only marshal arguments:
torch CUDA tensors are passed as device pointers, the current torch stream as the CUDA
stream, and host results are converted to numpy.  Every pixel operation runs in the CUDA
kernels of libpsfm.  If the shared library is missing, importing the functions raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpsfm.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "psfm.h")

PSFM_OK = 0
STATUS = {0: "OK", 1: "BAD_ARG", 2: "TOO_FEW_STAMPS", 3: "SINGULAR", 4: "NONFINITE", 5: "CUDA",
          6: "TIMEOUT", 8: "WORKSPACE", 9: "UNSUPPORTED"}
OP_SOLVE, OP_CONVOLVE, OP_SUBTRACT, OP_STACK = 1, 2, 3, 4
NORM_SEPARATE, NORM_JOINT = 0, 1
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16X3, PREC_F32X2, PREC_BF16X6 = 0, 1, 2, 3, 4, 5
CAND_UNUSED, CAND_USED, CAND_REJECTED = 0, 1, 2
(QUALITY_FEW_STAMPS, QUALITY_MEAN_DEV, QUALITY_RMS_DEV, QUALITY_MOMENT1, QUALITY_MOMENT2,
 QUALITY_DECONV) = 1, 2, 4, 8, 16, 32
MAX_GAUSS = 4


class PsfmError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        super().__init__(f"{where}: psfm status {code} ({STATUS.get(int(code), '?')})")


class psfm_shape(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("pitch", C.c_int64)]


class psfm_stamp(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32)]


class psfm_basis_spec(C.Structure):
    _fields_ = [("n_gauss", C.c_int32), ("sigma", C.c_double * MAX_GAUSS),
                ("degree", C.c_int32 * MAX_GAUSS), ("half_width", C.c_int32),
                ("spatial_order", C.c_int32), ("bg_order", C.c_int32)]


class psfm_config(C.Structure):
    _fields_ = [("grid_nx", C.c_int32), ("grid_ny", C.c_int32), ("stamp_half", C.c_int32),
                ("max_cand", C.c_int32), ("thresh_nsigma", C.c_double),
                ("reject_nsigma", C.c_double), ("soften_alpha", C.c_double),
                ("bad_frac", C.c_double), ("max_iter", C.c_int32), ("var_tile", C.c_int32),
                ("cov_grid", C.c_int32), ("norm_mode", C.c_int32), ("precision", C.c_int32),
                ("badmask", C.c_uint16), ("conv_bad", C.c_uint16), ("conv_poor", C.c_uint16),
                ("nodata", C.c_uint16), ("dual", C.c_int32), ("penalty", C.c_double)]


class psfm_solution(C.Structure):
    _fields_ = [("b0", C.c_double), ("d0", C.c_double), ("coeff", C.POINTER(C.c_double)),
                ("n_coeff", C.c_int32), ("n_regions", C.c_int32), ("max_cand", C.c_int32),
                ("cand_capacity", C.c_int32), ("cand", C.POINTER(psfm_stamp)),
                ("cand_status", C.POINTER(C.c_int32)), ("chi2", C.POINTER(C.c_double)),
                ("n_used", C.c_int32), ("n_iter", C.c_int32), ("r_bad", C.c_int32),
                ("chi2_mean", C.c_double), ("chi2_rms", C.c_double), ("median", C.c_float),
                ("kernel_sum", C.c_double), ("mom_x", C.c_double), ("mom_y", C.c_double),
                ("mom_xx", C.c_double), ("mom_yy", C.c_double), ("mom_xy", C.c_double),
                ("deconv_max", C.c_double), ("quality_flags", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libpsfm.so (built by ``paper_1901_09999_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpsfm.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    P = C.POINTER
    lib.psfm_config_default.argtypes = [P(psfm_config)]
    lib.psfm_config_default.restype = None
    lib.psfm_status_string.argtypes = [i32]
    lib.psfm_status_string.restype = C.c_char_p
    lib.psfm_basis_size.argtypes = [P(psfm_basis_spec)]
    lib.psfm_basis_size.restype = i32
    lib.psfm_spatial_size.argtypes = [P(psfm_basis_spec)]
    lib.psfm_spatial_size.restype = i32
    lib.psfm_cov_width.argtypes = [P(psfm_basis_spec), i32, i32]
    lib.psfm_cov_width.restype = i32
    lib.psfm_workspace_size.argtypes = [i32, psfm_shape, P(psfm_basis_spec), P(psfm_config), i32]
    lib.psfm_workspace_size.restype = sz
    lib.psfm_solve_kernel.argtypes = [vp, vp, vp, vp, vp, vp, psfm_shape, P(psfm_stamp), i32,
                                      P(psfm_basis_spec), P(psfm_config), P(psfm_solution), vp,
                                      sz, vp]
    lib.psfm_solve_kernel.restype = i32
    lib.psfm_convolve.argtypes = [vp, vp, vp, vp, vp, vp, psfm_shape, P(psfm_basis_spec),
                                  P(psfm_config), P(psfm_solution), vp, i32, vp, i32, vp, vp, vp,
                                  vp, i32, vp, sz, vp]
    lib.psfm_convolve.restype = i32
    lib.psfm_subtract.argtypes = [vp, vp, vp, vp, vp, vp, psfm_shape, P(psfm_stamp), i32,
                                  P(psfm_basis_spec), P(psfm_config), vp, i32, vp, i32, vp, vp, vp,
                                  vp, i32, P(psfm_solution), vp, sz, vp]
    lib.psfm_subtract.restype = i32
    lib.psfm_stack.argtypes = [i32, P(vp), P(vp), P(vp), psfm_shape, P(P(C.c_double)), P(i32),
                               C.c_double, P(psfm_basis_spec), P(psfm_config), vp, vp, vp, vp, vp,
                               i32, P(psfm_solution), vp, sz, vp]
    lib.psfm_stack.restype = i32
    lib.psfm_convolve_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, psfm_shape, P(psfm_basis_spec),
                                          P(psfm_config), P(psfm_solution), vp, vp, vp, vp]
    lib.psfm_convolve_noalloc.restype = i32
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions include/psfm.h declares."""
    txt = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(psfm_\w+)\s*\(", txt, re.M)))


# ------------------------------------------------------------------------ host structures

def config(**kw) -> psfm_config:
    c = psfm_config()
    load().psfm_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


def basis_spec(sigma, degree, half_width, spatial_order=0) -> psfm_basis_spec:
    b = psfm_basis_spec()
    b.n_gauss = len(sigma)
    for i, (s, d) in enumerate(zip(sigma, degree)):
        b.sigma[i] = float(s)
        b.degree[i] = int(d)
    b.half_width = int(half_width)
    b.spatial_order = int(spatial_order)
    b.bg_order = 0
    return b


def basis_size(b):
    return load().psfm_basis_size(C.byref(b))


def spatial_size(b):
    return load().psfm_spatial_size(C.byref(b))


def cov_width(b, cov_in_w=1, cov_img_w=0):
    return load().psfm_cov_width(C.byref(b), cov_in_w, cov_img_w)


def status_string(s):
    return load().psfm_status_string(int(s)).decode()


def psfm_workspace_size(op, shape, basis, cfg, n_stamps=0) -> int:
    return int(load().psfm_workspace_size(op, shape, C.byref(basis), C.byref(cfg), n_stamps))


# ------------------------------------------------------------------------ torch marshalling

def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _shape_of(*tensors) -> psfm_shape:
    t0 = tensors[0]
    H, W = t0.shape
    pitch = t0.stride(0)
    for t in tensors:
        if t is None:
            continue
        if tuple(t.shape) != (H, W) or t.stride(1) != 1 or t.stride(0) != pitch:
            raise ValueError("all images must share shape and row pitch, unit column stride")
        if not t.is_cuda:
            raise ValueError("images must be CUDA tensors")
    return psfm_shape(W, H, pitch)


def _like(t, dtype=None):
    """Empty CUDA tensor with the shape and row pitch of ``t`` (the library writes rows at the
    input pitch, so outputs must share it)."""
    torch = _torch()
    H, W = t.shape
    pitch = t.stride(0)
    base = torch.empty((H, pitch), dtype=dtype or t.dtype, device=t.device)
    return base[:, :W]


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _workspace(op, shape, basis, cfg, n_stamps, workspace, device):
    torch = _torch()
    need = psfm_workspace_size(op, shape, basis, cfg, n_stamps)
    if need == 0:
        # an argument the library rejects: the call itself returns the precise status
        return None, 0
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    return workspace, need


class Solution:
    """Host copy of a psfm_solution with numpy arrays."""

    def __init__(self, ncoef, ncand):
        self.coeff = np.zeros(max(1, ncoef))
        self.cand = (psfm_stamp * max(1, ncand))()
        self.status = np.zeros(max(1, ncand), np.int32)
        self.chi2 = np.zeros(max(1, ncand))
        self.c = psfm_solution()
        self.c.coeff = self.coeff.ctypes.data_as(C.POINTER(C.c_double))
        self.c.n_coeff = ncoef
        self.c.cand_capacity = ncand
        self.c.cand = C.cast(self.cand, C.POINTER(psfm_stamp))
        self.c.cand_status = self.status.ctypes.data_as(C.POINTER(C.c_int32))
        self.c.chi2 = self.chi2.ctypes.data_as(C.POINTER(C.c_double))
        self.ncoef = ncoef
        self.ncand = ncand

    @classmethod
    def from_values(cls, b0, d0, coeff, r_bad=0):
        s = cls(len(coeff), 1)
        s.coeff[:] = coeff
        s.c.b0, s.c.d0, s.c.r_bad = float(b0), float(d0), int(r_bad)
        return s

    @property
    def b0(self):
        return self.c.b0

    @property
    def d0(self):
        return self.c.d0

    @property
    def r_bad(self):
        return self.c.r_bad

    @property
    def n_used(self):
        return self.c.n_used

    @property
    def n_iter(self):
        return self.c.n_iter

    @property
    def chi2_mean(self):
        return self.c.chi2_mean

    @property
    def chi2_rms(self):
        return self.c.chi2_rms

    @property
    def median(self):
        return self.c.median

    def quality(self) -> dict:
        """Quality diagnostics of the solution (Sec. 3.7) and the PSFM_QUALITY_* flags."""
        c = self.c
        return dict(n_used=c.n_used, chi2_mean=c.chi2_mean, chi2_rms=c.chi2_rms,
                    kernel_sum=c.kernel_sum, mom_x=c.mom_x, mom_y=c.mom_y, mom_xx=c.mom_xx,
                    mom_yy=c.mom_yy, mom_xy=c.mom_xy, deconv_max=c.deconv_max,
                    flags=c.quality_flags)

    def candidates(self):
        n = self.c.n_regions * self.c.max_cand
        xy = np.array([(self.cand[i].x, self.cand[i].y) for i in range(n)], np.int32)
        return (xy.reshape(self.c.n_regions, self.c.max_cand, 2),
                self.status[:n].reshape(self.c.n_regions, self.c.max_cand).copy(),
                self.chi2[:n].reshape(self.c.n_regions, self.c.max_cand).copy())


def _stamps_arg(stamps):
    if stamps is None or len(stamps) == 0:
        return None, 0, None
    arr = (psfm_stamp * len(stamps))(*[psfm_stamp(int(x), int(y)) for x, y in stamps])
    return C.cast(arr, C.POINTER(psfm_stamp)), len(stamps), arr


def _ncoef(basis, cfg):
    """Kernel coefficients of a solution: N_b N_s, twice that with the dual kernel."""
    return basis_size(basis) * spatial_size(basis) * (2 if getattr(cfg, "dual", 0) else 1)


def _ncand(basis, cfg, n_stamps):
    return n_stamps if n_stamps > 0 else cfg.grid_nx * cfg.grid_ny * cfg.max_cand


def psfm_solve_kernel(img, ref, var_img, var_ref, mask_img, mask_ref, basis, cfg, stamps=None,
                      workspace=None, stream=None) -> Solution:
    """Solve for the PSF-matching kernel on the GPU (C: psfm_solve_kernel)."""
    lib = load()
    shape = _shape_of(img, ref, var_img, var_ref, mask_img, mask_ref)
    sp, ns, _keep = _stamps_arg(stamps)
    ws, need = _workspace(OP_SOLVE, shape, basis, cfg, ns, workspace, img.device)
    sol = Solution(_ncoef(basis, cfg), _ncand(basis, cfg, ns))
    st = lib.psfm_solve_kernel(_ptr(img), _ptr(ref), _ptr(var_img), _ptr(var_ref), _ptr(mask_img),
                               _ptr(mask_ref), shape, sp, ns, C.byref(basis), C.byref(cfg),
                               C.byref(sol.c), _ptr(ws), need, _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_solve_kernel")
    return sol


def psfm_convolve(ref, var_ref, mask_ref, basis, cfg, sol: Solution, img=None, var_img=None,
                  mask_img=None, cov_ref=None, cov_img=None, out=None, out_var=None,
                  out_mask=None, want_var=True, want_mask=True, want_cov=True, workspace=None,
                  stream=None):
    """Apply a solved kernel (C: psfm_convolve).  Returns (out, out_var, out_mask, cov)."""
    torch = _torch()
    lib = load()
    shape = _shape_of(ref, var_ref, mask_ref, img, var_img, mask_img)
    dev = ref.device
    if out is None:
        out = _like(ref)
    if want_var and out_var is None:
        out_var = _like(ref)
    if want_mask and out_mask is None:
        out_mask = _like(mask_ref)
    _shape_of(ref, out, out_var, out_mask)
    c_ref = 1 if cov_ref is None else cov_ref.shape[0]
    c_img = 0 if img is None else (1 if cov_img is None else cov_img.shape[0])
    cov = None
    ncov = 0
    if want_cov:
        ncov = cov_width(basis, c_ref, c_img)
        cov = torch.empty((ncov, ncov), dtype=torch.float64, device=dev)
    ws, need = _workspace(OP_CONVOLVE, shape, basis, cfg, 0, workspace, dev)
    st = lib.psfm_convolve(_ptr(ref), _ptr(var_ref), _ptr(mask_ref), _ptr(img), _ptr(var_img),
                           _ptr(mask_img), shape, C.byref(basis), C.byref(cfg), C.byref(sol.c),
                           _ptr(cov_ref), c_ref, _ptr(cov_img), c_img if cov_img is not None else 0,
                           _ptr(out), _ptr(out_var), _ptr(out_mask), _ptr(cov), ncov, _ptr(ws), need,
                           _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_convolve")
    return out, out_var, out_mask, cov


def psfm_convolve_noalloc(ref, var_ref, mask_ref, basis, cfg, sol: Solution, img=None,
                          var_img=None, mask_img=None, out=None, out_var=None, out_mask=None,
                          stream=None):
    """psfm_convolve without a workspace, for callers that cannot allocate device memory
    (C: psfm_convolve_noalloc; images up to 4096 x 4096, no pseudo-matrix).  Output tensors
    may be passed in so that the call allocates nothing; the ones left as None are created
    here for convenience.  Returns (out, out_var, out_mask)."""
    lib = load()
    shape = _shape_of(ref, var_ref, mask_ref, img, var_img, mask_img)
    out = _like(ref) if out is None else out
    out_var = _like(ref) if out_var is None else out_var
    out_mask = _like(mask_ref) if out_mask is None else out_mask
    _shape_of(ref, out, out_var, out_mask)
    st = lib.psfm_convolve_noalloc(_ptr(ref), _ptr(var_ref), _ptr(mask_ref), _ptr(img),
                                   _ptr(var_img), _ptr(mask_img), shape, C.byref(basis),
                                   C.byref(cfg), C.byref(sol.c), _ptr(out), _ptr(out_var),
                                   _ptr(out_mask), _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_convolve_noalloc")
    return out, out_var, out_mask


def psfm_subtract(img, ref, var_img, var_ref, mask_img, mask_ref, basis, cfg, stamps=None,
                  cov_ref=None, cov_img=None, out=None, out_var=None, out_mask=None,
                  want_cov=True, workspace=None, stream=None, solution=True):
    """Solve and subtract in one call (C: psfm_subtract).

    Returns (diff, diff_var, diff_mask, cov, Solution or None)."""
    torch = _torch()
    lib = load()
    shape = _shape_of(img, ref, var_img, var_ref, mask_img, mask_ref)
    dev = img.device
    sp, ns, _keep = _stamps_arg(stamps)
    out = _like(img) if out is None else out
    out_var = _like(img) if out_var is None else out_var
    out_mask = _like(mask_img) if out_mask is None else out_mask
    _shape_of(img, out, out_var, out_mask)
    c_ref = 1 if cov_ref is None else cov_ref.shape[0]
    c_img = 1 if cov_img is None else cov_img.shape[0]
    cov, ncov = None, 0
    if want_cov:
        ncov = cov_width(basis, c_ref, c_img)
        cov = torch.empty((ncov, ncov), dtype=torch.float64, device=dev)
    ws, need = _workspace(OP_SUBTRACT, shape, basis, cfg, ns, workspace, dev)
    sol = Solution(_ncoef(basis, cfg), _ncand(basis, cfg, ns)) if solution else None
    st = lib.psfm_subtract(_ptr(img), _ptr(ref), _ptr(var_img), _ptr(var_ref), _ptr(mask_img),
                           _ptr(mask_ref), shape, sp, ns, C.byref(basis), C.byref(cfg),
                           _ptr(cov_ref), c_ref, _ptr(cov_img), c_img if cov_img is not None else 0,
                           _ptr(out), _ptr(out_var), _ptr(out_mask), _ptr(cov), ncov,
                           C.byref(sol.c) if sol else None, _ptr(ws), need, _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_subtract")
    return out, out_var, out_mask, cov, sol


def psfm_stack(imgs, vars_, masks, sources, target_fwhm, bases, cfg, want_cov=True,
               workspace=None, stream=None):
    """PSF-homogenised stack (C: psfm_stack).  ``sources`` is a list of (n, 3) float64 numpy
    arrays (x, y, flux) per input; ``bases`` a list of psfm_basis_spec.

    Returns (image, variance, mask, count, cov, [Solution])."""
    torch = _torch()
    lib = load()
    n = len(imgs)
    shape = _shape_of(*imgs, *vars_, *masks)
    dev = imgs[0].device
    out = _like(imgs[0])
    out_var = _like(imgs[0])
    out_mask = _like(masks[0])
    out_count = _like(imgs[0], torch.int32)
    srcs = [np.ascontiguousarray(s, np.float64) for s in sources]
    nsrc = (C.c_int32 * n)(*[len(s) for s in srcs])
    sp = (C.POINTER(C.c_double) * n)(*[s.ctypes.data_as(C.POINTER(C.c_double)) for s in srcs])
    bs = (psfm_basis_spec * n)(*bases)
    big = max(range(n), key=lambda i: psfm_workspace_size(OP_STACK, shape, bases[i], cfg, max(len(s) for s in srcs)))
    need = psfm_workspace_size(OP_STACK, shape, bases[big], cfg, max(len(s) for s in srcs))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    ncov = max(cov_width(b, 1, 0) for b in bases)
    cov = torch.empty((ncov, ncov), dtype=torch.float64, device=dev) if want_cov else None
    sols = [Solution(_ncoef(b, cfg), _ncand(b, cfg, 0)) for b in bases]
    csols = (psfm_solution * n)(*[s.c for s in sols])
    ptrs = lambda ts: (C.c_void_p * n)(*[t.data_ptr() for t in ts])
    st = lib.psfm_stack(n, ptrs(imgs), ptrs(vars_), ptrs(masks), shape, sp, nsrc, float(target_fwhm),
                        bs, C.byref(cfg), _ptr(out), _ptr(out_var), _ptr(out_mask), _ptr(out_count),
                        _ptr(cov), ncov if want_cov else 0, csols, _ptr(workspace), need,
                        _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_stack")
    for s, c in zip(sols, csols):
        s.c = c
    return out, out_var, out_mask, out_count, cov, sols


def psfm_bin(img, var, mask, b, badmask, cov_in=None, want_cov=True, stream=None):
    """Integer binning by b with variance, mask and pseudo-matrix (C: psfm_bin).  Returns
    (image, variance, mask, pseudo-matrix or None) at (H // b, W // b)."""
    torch = _torch()
    lib = load()
    vp, i32 = C.c_void_p, C.c_int32
    lib.psfm_bin_cov_width.argtypes = [i32, i32]
    lib.psfm_bin_cov_width.restype = i32
    lib.psfm_bin.argtypes = [vp, vp, vp, psfm_shape, i32, C.c_uint16, vp, i32, vp, vp, vp,
                             psfm_shape, vp, i32, vp, C.c_size_t, vp]
    lib.psfm_bin.restype = i32
    shape = _shape_of(img, var, mask)
    H, W = img.shape
    Hb, Wb = H // b, W // b
    out = torch.empty((Hb, Wb), dtype=torch.float32, device=img.device)
    out_var = torch.empty_like(out)
    out_mask = torch.empty((Hb, Wb), dtype=mask.dtype, device=img.device)
    cw = cov_in.shape[0] if cov_in is not None else 1
    nw = int(lib.psfm_bin_cov_width(cw, b))
    cov = torch.empty((nw, nw), dtype=torch.float64, device=img.device) if want_cov else None
    ws = torch.empty(4096, dtype=torch.uint8, device=img.device)
    st = lib.psfm_bin(_ptr(img), _ptr(var), _ptr(mask), shape, int(b), int(badmask),
                      _ptr(cov_in), cw, _ptr(out), _ptr(out_var), _ptr(out_mask),
                      psfm_shape(Wb, Hb, Wb), _ptr(cov), nw if want_cov else 0, _ptr(ws), 4096,
                      _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_bin")
    return out, out_var, out_mask, cov


STACK_REJECT = 1 << 13


def psfm_stack_full(imgs, vars_, masks, sources, target_fwhm, bases, cfg, clip_nsigma=5.0,
                    reject_bit=STACK_REJECT, want_cov=True, workspace=None, stream=None):
    """Stack with outlier rejection and the unconvolved companion stack (C: psfm_stack_full).

    Returns dict(conv=(image, variance, mask, count), unconv=(image, variance, mask, count),
    rejected=[outlier pixels per input], outliers=int32 plane with bit i set where input i is
    an outlier, cov=pseudo-matrix or None, sols=[Solution])."""
    torch = _torch()
    lib = load()
    vp, i32, P_ = C.c_void_p, C.c_int32, C.POINTER
    lib.psfm_stack_full_workspace_size.argtypes = [i32, psfm_shape, P_(psfm_basis_spec),
                                                   P_(psfm_config), i32]
    lib.psfm_stack_full_workspace_size.restype = C.c_size_t
    lib.psfm_stack_full.argtypes = [i32, P_(vp), P_(vp), P_(vp), psfm_shape, P_(P_(C.c_double)),
                                    P_(i32), C.c_double, P_(psfm_basis_spec), P_(psfm_config),
                                    C.c_double, C.c_uint16] + [vp] * 8 + [
                                    P_(i32), vp, vp, i32, P_(psfm_solution), vp, C.c_size_t, vp]
    lib.psfm_stack_full.restype = i32
    n = len(imgs)
    shape = _shape_of(*imgs, *vars_, *masks)
    dev = imgs[0].device
    srcs = [np.ascontiguousarray(s_, np.float64) for s_ in sources]
    nsrc = (C.c_int32 * n)(*[len(s_) for s_ in srcs])
    sp = (P_(C.c_double) * n)(*[s_.ctypes.data_as(P_(C.c_double)) for s_ in srcs])
    bs = (psfm_basis_spec * n)(*bases)
    need = int(lib.psfm_stack_full_workspace_size(n, shape, bs, C.byref(cfg),
                                                  max(len(s_) for s_ in srcs)))
    if need == 0:
        raise PsfmError(1, "psfm_stack_full_workspace_size")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    conv = (_like(imgs[0]), _like(imgs[0]), _like(masks[0]), _like(imgs[0], torch.int32))
    unconv = (_like(imgs[0]), _like(imgs[0]), _like(masks[0]), _like(imgs[0], torch.int32))
    ncov = max(cov_width(b, 1, 0) for b in bases)
    cov = torch.empty((ncov, ncov), dtype=torch.float64, device=dev) if want_cov else None
    sols = [Solution(_ncoef(b, cfg), _ncand(b, cfg, 0)) for b in bases]
    csols = (psfm_solution * n)(*[s_.c for s_ in sols])
    rej = (C.c_int32 * n)()
    outl = _like(imgs[0], torch.int32)
    ptrs = lambda ts: (vp * n)(*[t.data_ptr() for t in ts])
    st = lib.psfm_stack_full(n, ptrs(imgs), ptrs(vars_), ptrs(masks), shape, sp, nsrc,
                             float(target_fwhm), bs, C.byref(cfg), float(clip_nsigma),
                             int(reject_bit), *[_ptr(t) for t in conv], *[_ptr(t) for t in unconv],
                             rej, _ptr(outl), _ptr(cov), ncov if want_cov else 0, csols,
                             _ptr(workspace), need, _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_stack_full")
    for s_, c in zip(sols, csols):
        s_.c = c
    return dict(conv=conv, unconv=unconv, rejected=list(rej), outliers=outl, cov=cov, sols=sols)


def psfm_gram(cols, weights, precision, stream=None):
    """Weighted Gram of column blocks (C: psfm_gram).  ``cols`` (n_blocks, n_cols, n_pix) and
    ``weights`` (n_blocks, n_pix) are contiguous float32 CUDA tensors; returns the
    (n_blocks, n_cols, n_cols) float64 Gram."""
    torch = _torch()
    lib = load()
    lib.psfm_gram.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                              C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    lib.psfm_gram.restype = C.c_int32
    if cols.dtype != torch.float32 or weights.dtype != torch.float32:
        raise ValueError("cols and weights must be float32")
    cols, weights = cols.contiguous(), weights.contiguous()
    nb, nc, npix = cols.shape
    if tuple(weights.shape) != (nb, npix):
        raise ValueError("weights must be (n_blocks, n_pix)")
    G = torch.empty((nb, nc, nc), dtype=torch.float64, device=cols.device)
    ws = torch.empty(256, dtype=torch.uint8, device=cols.device)
    st = lib.psfm_gram(nb, nc, npix, _ptr(cols), _ptr(weights), int(precision), _ptr(G), _ptr(ws),
                       256, _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_gram")
    return G


class psfm_tune_entry(C.Structure):
    _fields_ = [("half_width", C.c_int32), ("spatial_order", C.c_int32), ("n_gauss", C.c_int32),
                ("degree", C.c_int32 * MAX_GAUSS), ("tile_rows", C.c_int32),
                ("plane_chunk", C.c_int32), ("ms", C.c_float)]


def _tune_types(lib):
    P_, i32 = C.POINTER, C.c_int32
    lib.psfm_tune_conv_workspace_size.argtypes = [i32, i32, P_(psfm_basis_spec)]
    lib.psfm_tune_conv_workspace_size.restype = C.c_size_t
    lib.psfm_tune_conv.argtypes = [i32, i32, P_(psfm_basis_spec), C.c_void_p, C.c_size_t,
                                   C.c_void_p, P_(psfm_tune_entry)]
    lib.psfm_tune_conv.restype = i32
    lib.psfm_tune_count.argtypes = []
    lib.psfm_tune_count.restype = i32
    lib.psfm_tune_get.argtypes = [i32, P_(psfm_tune_entry)]
    lib.psfm_tune_get.restype = i32
    lib.psfm_tune_set.argtypes = [P_(psfm_tune_entry)]
    lib.psfm_tune_set.restype = i32
    lib.psfm_tune_clear.argtypes = []
    lib.psfm_tune_clear.restype = None


def _entry_dict(e: psfm_tune_entry) -> dict:
    return {"half_width": e.half_width, "spatial_order": e.spatial_order, "n_gauss": e.n_gauss,
            "degree": list(e.degree)[:e.n_gauss], "tile_rows": e.tile_rows,
            "plane_chunk": e.plane_chunk, "ms": float(e.ms)}


def tune_conv(basis, width, height, stream=None) -> dict:
    """Autotune the image convolution's launch shape for the class of ``basis`` on a synthetic
    width x height image (C: psfm_tune_conv); the choice goes into the library's table and is
    returned as a dict."""
    torch = _torch()
    lib = load()
    _tune_types(lib)
    need = int(lib.psfm_tune_conv_workspace_size(int(width), int(height), C.byref(basis)))
    if need == 0:
        raise PsfmError(1, "psfm_tune_conv_workspace_size")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    e = psfm_tune_entry()
    st = lib.psfm_tune_conv(int(width), int(height), C.byref(basis), _ptr(ws), need,
                            _stream(stream), C.byref(e))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_tune_conv")
    return _entry_dict(e)


def tune_entries() -> list:
    """The library's tuning table as a list of dicts (C: psfm_tune_get)."""
    lib = load()
    _tune_types(lib)
    out = []
    for i in range(lib.psfm_tune_count()):
        e = psfm_tune_entry()
        if lib.psfm_tune_get(i, C.byref(e)) == PSFM_OK:
            out.append(_entry_dict(e))
    return out


def tune_set(entry: dict):
    """Adds or replaces one tuning-table entry (C: psfm_tune_set)."""
    lib = load()
    _tune_types(lib)
    e = psfm_tune_entry()
    e.half_width, e.spatial_order = int(entry["half_width"]), int(entry["spatial_order"])
    deg = list(entry["degree"])
    e.n_gauss = len(deg)
    for g, d in enumerate(deg):
        e.degree[g] = int(d)
    e.tile_rows, e.plane_chunk = int(entry["tile_rows"]), int(entry["plane_chunk"])
    e.ms = float(entry.get("ms", 0.0))
    st = lib.psfm_tune_set(C.byref(e))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_tune_set")


def tune_clear():
    lib = load()
    _tune_types(lib)
    lib.psfm_tune_clear()


def tune_save(path, device_name=""):
    """Writes the tuning table to a JSON file (with the device it was measured on)."""
    import json
    with open(path, "w") as f:
        json.dump({"version": 1, "device": device_name, "entries": tune_entries()}, f, indent=1)


def tune_load(path, device_name=None) -> int:
    """Loads tuning entries from a JSON file written by tune_save; entries measured on another
    device are skipped when ``device_name`` is given.  Returns the number loaded."""
    import json
    with open(path) as f:
        d = json.load(f)
    if device_name is not None and d.get("device") not in ("", device_name):
        return 0
    n = 0
    for e in d.get("entries", []):
        tune_set(e)
        n += 1
    return n


WAIT_LIMIT_DEFAULT = 1 << 24


def set_pipeline_wait_limit(polls):
    """Poll limit of the tensor-core Gram's pipeline waits on the current device (C:
    psfm_set_pipeline_wait_limit); a test hook for the PSFM_ERR_TIMEOUT path."""
    lib = load()
    lib.psfm_set_pipeline_wait_limit.argtypes = [C.c_uint32]
    lib.psfm_set_pipeline_wait_limit.restype = C.c_int32
    st = lib.psfm_set_pipeline_wait_limit(int(polls))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_set_pipeline_wait_limit")


def psfm_resample_cov(cov_in, scale, stream=None):
    """Pseudo-matrix of an image resampled by a non-integer scale (C: psfm_resample_cov).
    ``cov_in`` is a square float64 CUDA tensor of odd width; returns the resampled one."""
    torch = _torch()
    lib = load()
    lib.psfm_resample_cov_width.argtypes = [C.c_int32, C.c_double]
    lib.psfm_resample_cov_width.restype = C.c_int32
    lib.psfm_resample_cov.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_int32,
                                      C.c_void_p]
    lib.psfm_resample_cov.restype = C.c_int32
    cov_in = cov_in.contiguous()
    w_in = int(cov_in.shape[0])
    w = lib.psfm_resample_cov_width(w_in, float(scale))
    if w < 0:
        raise PsfmError(1, "psfm_resample_cov_width")
    out = torch.empty((w, w), dtype=torch.float64, device=cov_in.device)
    st = lib.psfm_resample_cov(_ptr(cov_in), w_in, float(scale), _ptr(out), w, _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_resample_cov")
    return out


class psfm_psf_model(C.Structure):
    _fields_ = [("fwhm_major", C.c_double), ("fwhm_minor", C.c_double),
                ("moffat_frac", C.c_double), ("beta", C.c_double)]


ENVELOPE_MAX_RADIUS = 64


def psfm_envelope_fwhm(models, radius=0, device=None, stream=None):
    """FWHM of the envelope PSF of stack inputs (C: psfm_envelope_fwhm).  ``models`` is a list of
    (fwhm_major, fwhm_minor, moffat_frac, beta) tuples; returns the target FWHM (float)."""
    torch = _torch()
    lib = load()
    lib.psfm_envelope_fwhm.argtypes = [C.c_int32, C.POINTER(psfm_psf_model), C.c_int32,
                                       C.POINTER(C.c_double), C.c_void_p, C.c_size_t, C.c_void_p]
    lib.psfm_envelope_fwhm.restype = C.c_int32
    arr = (psfm_psf_model * max(1, len(models)))(*[psfm_psf_model(*map(float, m)) for m in models])
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    out = C.c_double(0.0)
    st = lib.psfm_envelope_fwhm(len(models), arr, int(radius), C.byref(out), _ptr(ws), 256,
                                _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_envelope_fwhm")
    return out.value


# ------------------------------------------------------------------------ instrumentation

def _prof_types(lib):
    lib.psfm_profile_enable.argtypes = [C.c_int32]
    lib.psfm_profile_enable.restype = None
    lib.psfm_profile_count.argtypes = []
    lib.psfm_profile_count.restype = C.c_int32
    lib.psfm_profile_entry.argtypes = [C.c_int32, C.c_char_p, C.c_int32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.psfm_profile_entry.restype = C.c_int32
    lib.psfm_launch_count.argtypes = []
    lib.psfm_launch_count.restype = C.c_longlong


def psfm_profile_enable(on: bool):
    lib = load()
    _prof_types(lib)
    lib.psfm_profile_enable(1 if on else 0)


def psfm_launch_count() -> int:
    lib = load()
    _prof_types(lib)
    return int(lib.psfm_launch_count())


def fma_probe(n_blocks, iters, stream=None):
    """FP32 FMA throughput probe (C: psfm_fma_probe): enqueues the probe kernel on ``stream``
    and returns (flops of the launch, output tensor)."""
    torch = _torch()
    lib = load()
    lib.psfm_fma_probe.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double),
                                   C.c_void_p]
    lib.psfm_fma_probe.restype = C.c_int32
    out = torch.empty(n_blocks * 256, dtype=torch.float32, device="cuda")
    fl = C.c_double(0.0)
    st = lib.psfm_fma_probe(int(n_blocks), int(iters), _ptr(out), C.byref(fl), _stream(stream))
    if st != PSFM_OK:
        raise PsfmError(st, "psfm_fma_probe")
    return fl.value, out


def psfm_profile_read() -> dict:
    """{stage: (device ms total, kernel launches, calls)} since psfm_profile_enable(True)."""
    lib = load()
    _prof_types(lib)
    out = {}
    for i in range(lib.psfm_profile_count()):
        name = C.create_string_buffer(64)
        ms, nl, nc = C.c_double(), C.c_longlong(), C.c_longlong()
        if lib.psfm_profile_entry(i, name, 64, C.byref(ms), C.byref(nl), C.byref(nc)) == 0:
            out[name.value.decode()] = (ms.value, nl.value, nc.value)
    return out


# ------------------------------------------------------------------------ batches of chips

def _batch_types(lib):
    vp, i32, sz = C.c_void_p, C.c_int32, C.c_size_t
    P = C.POINTER
    lib.psfm_batch_workspace_size.argtypes = [i32, P(psfm_shape), P(psfm_basis_spec), P(psfm_config)]
    lib.psfm_batch_workspace_size.restype = sz
    lib.psfm_batch_create.argtypes = [i32, P(psfm_shape), P(psfm_basis_spec), P(psfm_config), i32,
                                      vp, sz, P(vp)]
    lib.psfm_batch_create.restype = i32
    lib.psfm_batch_subtract.argtypes = [vp] + [P(vp)] * 10 + [vp]
    lib.psfm_batch_subtract.restype = i32
    lib.psfm_batch_solutions.argtypes = [vp, P(psfm_solution), vp]
    lib.psfm_batch_solutions.restype = i32
    lib.psfm_batch_kernel_count.argtypes = [vp]
    lib.psfm_batch_kernel_count.restype = C.c_longlong
    lib.psfm_batch_destroy.argtypes = [vp]
    lib.psfm_batch_destroy.restype = None


class Batch:
    """Many chips subtracted by one call (C: psfm_batch_*).  ``chips`` is a list of dicts with
    the CUDA tensors img, ref, var_img, var_ref, mask_img, mask_ref; ``bases`` one
    psfm_basis_spec per chip.  Outputs are allocated here; run() enqueues (and on a
    non-default stream captures / replays a CUDA graph), solutions() synchronises."""

    def __init__(self, chips, bases, cfg, n_streams=4, want_cov=False):
        torch = _torch()
        self.lib = load()
        _batch_types(self.lib)
        self.n = len(chips)
        self.chips = chips
        self.bases = (psfm_basis_spec * self.n)(*bases)
        self.cfg = cfg
        shapes = [_shape_of(c["img"], c["ref"], c["var_img"], c["var_ref"], c["mask_img"],
                            c["mask_ref"]) for c in chips]
        self.shapes = (psfm_shape * self.n)(*shapes)
        need = int(self.lib.psfm_batch_workspace_size(self.n, self.shapes, self.bases, C.byref(cfg)))
        if need == 0:
            raise PsfmError(1, "psfm_batch_workspace_size")
        dev = chips[0]["img"].device
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)
        self.h = C.c_void_p()
        st = self.lib.psfm_batch_create(self.n, self.shapes, self.bases, C.byref(cfg), n_streams,
                                        _ptr(self.ws), need, C.byref(self.h))
        if st != PSFM_OK:
            raise PsfmError(st, "psfm_batch_create")
        self.diff = [_like(c["img"]) for c in chips]
        self.diff_var = [_like(c["img"]) for c in chips]
        self.diff_mask = [_like(c["mask_img"]) for c in chips]
        self.cov = [torch.empty((cov_width(b, 1, 1),) * 2, dtype=torch.float64, device=dev)
                    for b in bases] if want_cov else None

    def _arr(self, ts):
        return (C.c_void_p * self.n)(*[None if t is None else t.data_ptr() for t in ts])

    def run(self, stream=None):
        c = self.chips
        a = [self._arr([x[k] for x in c]) for k in ("img", "ref", "var_img", "var_ref",
                                                     "mask_img", "mask_ref")]
        st = self.lib.psfm_batch_subtract(self.h, *a, self._arr(self.diff), self._arr(self.diff_var),
                                          self._arr(self.diff_mask),
                                          self._arr(self.cov) if self.cov else None,
                                          _stream(stream))
        if st != PSFM_OK:
            raise PsfmError(st, "psfm_batch_subtract")

    def kernel_count(self):
        return int(self.lib.psfm_batch_kernel_count(self.h))

    def solutions(self, stream=None):
        sols = [Solution(_ncoef(b, self.cfg), _ncand(b, self.cfg, 0)) for b in self.bases]
        arr = (psfm_solution * self.n)(*[s.c for s in sols])
        st = self.lib.psfm_batch_solutions(self.h, arr, _stream(stream))
        for s, c in zip(sols, arr):
            s.c = c
        if st != PSFM_OK:
            raise PsfmError(st, "psfm_batch_solutions")
        return sols

    def close(self):
        if self.h:
            self.lib.psfm_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
