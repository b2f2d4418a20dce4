"""The C ABI library builds, loads without a GPU and exports every function include/psfm.h
declares; host-only entry points (defaults, sizes, argument checks) behave as documented."""
import ctypes as C

import pytest

from paper_1901_09999_gb300 import build as B
from paper_1901_09999_gb300 import psfm as P


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def test_exports_every_declared_function(lib):
    names = P.header_functions()
    assert {"psfm_solve_kernel", "psfm_convolve", "psfm_subtract", "psfm_stack",
            "psfm_workspace_size", "psfm_status_string"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_defaults_and_sizes(lib):
    cfg = P.config()
    assert (cfg.grid_nx, cfg.grid_ny, cfg.max_iter, cfg.var_tile, cfg.cov_grid) == (6, 5, 5, 64, 5)
    assert cfg.thresh_nsigma == 5.0 and cfg.reject_nsigma == 3.0 and cfg.bad_frac == 0.2
    assert cfg.conv_bad == 1 << 14 and cfg.conv_poor == 1 << 15
    b1 = P.basis_spec((0.7, 1.5, 3.0), (4, 2, 2), 10, 0)
    b2 = P.basis_spec((0.8, 1.6, 3.2), (6, 4, 2), 15, 2)
    assert P.basis_size(b1) == 27 and P.basis_size(b2) == 49
    assert P.spatial_size(b1) == 1 and P.spatial_size(b2) == 6
    assert P.cov_width(b2, 1, 0) == 61 and P.cov_width(b2, 5, 0) == 65 and P.cov_width(b2, 1, 101) == 101
    assert P.cov_width(b2, 2, 0) == -1
    assert P.status_string(2).startswith("fewer than 3")
    shape = P.psfm_shape(4846, 4868, 4848)
    for op in (P.OP_SOLVE, P.OP_CONVOLVE, P.OP_SUBTRACT):
        assert P.psfm_workspace_size(op, shape, b2, P.config(grid_nx=15, grid_ny=20)) > 0
    assert P.psfm_workspace_size(7, shape, b2, cfg) == 0
    bad = P.basis_spec((0.8,), (6,), 40, 0)          # half width above the maximum
    assert P.psfm_workspace_size(P.OP_CONVOLVE, shape, bad, cfg) == 0


def test_argument_errors_are_caught_on_the_host(lib):
    """Null or inconsistent arguments return BAD_ARG before any CUDA call."""
    cfg = P.config()
    b = P.basis_spec((1.0,), (2,), 5, 0)
    shape = P.psfm_shape(64, 64, 64)
    sol = P.Solution(6, 1)
    st = lib.psfm_convolve(None, None, None, None, None, None, shape, C.byref(b), C.byref(cfg),
                           C.byref(sol.c), None, 1, None, 0, None, None, None, None, 0, None, 0,
                           None)
    assert st == 1
    bad_shape = P.psfm_shape(64, 64, 32)             # pitch below width
    st = lib.psfm_solve_kernel(None, None, None, None, None, None, bad_shape, None, 0, C.byref(b),
                               C.byref(cfg), C.byref(sol.c), None, 0, None)
    assert st == 1
    cfg2 = P.config(var_tile=32)
    st = lib.psfm_convolve(None, None, None, None, None, None, shape, C.byref(b), C.byref(cfg2),
                           C.byref(sol.c), None, 1, None, 0, None, None, None, None, 0, None, 0,
                           None)
    assert st == 9


def test_envelope_argument_errors_are_caught_on_the_host(lib):
    """psfm_envelope_fwhm validates the models and sizes before any CUDA call."""
    lib.psfm_envelope_fwhm.argtypes = [C.c_int32, C.POINTER(P.psfm_psf_model), C.c_int32,
                                       C.POINTER(C.c_double), C.c_void_p, C.c_size_t, C.c_void_p]
    lib.psfm_envelope_fwhm.restype = C.c_int32
    out = C.c_double(0.0)
    ok = (P.psfm_psf_model * 1)(P.psfm_psf_model(4.0, 4.0, 0.0, 3.0))
    assert lib.psfm_envelope_fwhm(0, ok, 0, C.byref(out), None, 0, None) == 1
    assert lib.psfm_envelope_fwhm(1, ok, 0, C.byref(out), None, 0, None) == 8  # no workspace
    fake_ws = C.c_void_p(256)  # never dereferenced: the models are rejected first
    for m, r in (((4.0, 0.0, 0.0, 3.0), 0), ((4.0, 4.0, -0.1, 3.0), 0), ((4.0, 4.0, 0.2, 0.9), 0),
                 ((4.0, 4.0, 0.0, 3.0), 65), ((40.0, 40.0, 0.0, 3.0), 0)):
        arr = (P.psfm_psf_model * 1)(P.psfm_psf_model(*m))
        assert lib.psfm_envelope_fwhm(1, arr, r, C.byref(out), fake_ws, 256, None) == 1


def test_tuning_table_host_side(lib):
    """The convolution tuning table: entries are set, replaced per basis class, read back,
    persisted through JSON and cleared, all on the host; illegal shapes are rejected."""
    import os
    import tempfile
    P.tune_clear()
    e = {"half_width": 15, "spatial_order": 2, "degree": [6, 4, 2], "tile_rows": 64,
         "plane_chunk": 4, "ms": 1.5}
    P.tune_set(e)
    P.tune_set(dict(e, half_width=10, tile_rows=128))
    P.tune_set(dict(e, tile_rows=128, plane_chunk=0))   # replaces the first class
    got = sorted(P.tune_entries(), key=lambda x: x["half_width"])
    assert [(x["half_width"], x["tile_rows"], x["plane_chunk"]) for x in got] == \
        [(10, 128, 4), (15, 128, 0)]
    with pytest.raises(P.PsfmError):
        P.tune_set(dict(e, tile_rows=32))
    with pytest.raises(P.PsfmError):
        P.tune_set(dict(e, plane_chunk=3))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        P.tune_save(path, "dev")
        P.tune_clear()
        assert P.tune_entries() == []
        assert P.tune_load(path, "other") == 0
        assert P.tune_load(path, "dev") == 2
    assert sorted(x["half_width"] for x in P.tune_entries()) == [10, 15]
    P.tune_clear()
