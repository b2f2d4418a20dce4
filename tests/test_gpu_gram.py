"""The weighted Gram (Eq. 5-6) through psfm_gram: the FP64 mode against numpy, and the two
tensor-core modes (TF32; BF16 hi/lo split with three products, both with FP32 accumulation)
against their rounding bounds.  Wrong operand layouts or descriptors give errors of the order
of the entries themselves, far outside these bounds."""
import numpy as np
import pytest

from gpu_common import device
from paper_1901_09999_gb300 import psfm as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


def _data(seed, nb, nc, npix):
    """Random column blocks shaped like augmented stamp blocks: one constant column, weights
    like 1 / variance with some masked (zero-weight) pixels."""
    rng = np.random.default_rng(seed)
    cols = rng.normal(0.0, 1.0, (nb, nc, npix)).astype(np.float32)
    cols[:, nc - 2, :] = 1.0
    cols[:, 0, :] *= 300.0  # a column on another scale, as the reference pixels are
    w = rng.uniform(1e-3, 1e-2, (nb, npix)).astype(np.float32)
    w[:, ::17] = 0.0
    return cols, w


def _reference(cols, w):
    c, ww = cols.astype(np.float64), w.astype(np.float64)
    G = np.einsum("bip,bp,bjp->bij", c, ww, c)
    A = np.einsum("bip,bp,bjp->bij", np.abs(c), ww, np.abs(c))
    return G, A


@pytest.mark.parametrize("nc,npix", [(52, 961), (60, 441), (100, 70), (7, 33), (128, 64)])
def test_gram_modes_within_rounding_bounds(dev, nc, npix):
    import torch
    cols, w = _data(nc * 1000 + npix, 3, nc, npix)
    G, A = _reference(cols, w)
    tc, tw = torch.from_numpy(cols).to(dev), torch.from_numpy(w).to(dev)
    g64 = P.psfm_gram(tc, tw, P.PREC_FP64).cpu().numpy()
    assert np.all(np.abs(g64 - G) <= 1e-13 * A)
    u = 2.0 ** -24
    # TF32 keeps 10 fraction bits of each operand: product error < 2^-9 relative; FP32 sums
    bounds = {P.PREC_TF32: 2.0 ** -9 + 2.0 ** -18 + npix * u,
              # hi/lo BF16 split: |a - hi - lo| <= 2^-18 |a|; the lo*lo product is dropped
              P.PREC_BF16X3: 4 * 2.0 ** -18 + 3 * npix * u}
    med = {}
    for prec, eps in bounds.items():
        g = P.psfm_gram(tc, tw, prec).cpu().numpy()
        err = np.abs(g - G)
        assert np.all(err <= 2.0 * eps * A), (prec, float(np.max(err / A)))
        assert np.array_equal(g, np.swapaxes(g, 1, 2))
        med[prec] = float(np.median(err / A))
    print(f"nc={nc} npix={npix}: median |err| / sum|terms|: TF32 {med[P.PREC_TF32]:.2e}, "
          f"BF16x3 {med[P.PREC_BF16X3]:.2e}")
    # the split products really carry the low halves
    assert med[P.PREC_BF16X3] < 0.05 * med[P.PREC_TF32]


@pytest.mark.parametrize("nc,npix", [(52, 961), (60, 441), (64, 70), (7, 33), (40, 600),
                                     (64, 257)])
def test_split_product_gram_is_exact_to_double_float(dev, nc, npix):
    """BF16X6: the Gram as (sqrt(w) A)^T (sqrt(w) A), seven BF16 slices of the scaled columns,
    products exact on the tensor cores, levels 0..3 summed exactly as integers over 256-pixel
    groups.  sqrt(w) and the scaled columns carry 48 bits, so the Gram agrees with the FP64 one
    to a few units of 2^-48 of its terms (against 2^-9 for TF32)."""
    import torch
    cols, w = _data(nc * 7 + npix, 3, nc, npix)
    G, A = _reference(cols, w)
    tc, tw = torch.from_numpy(cols).to(dev), torch.from_numpy(w).to(dev)
    g = P.psfm_gram(tc, tw, P.PREC_BF16X6).cpu().numpy()
    err = np.abs(g - G)
    rel = float(np.max(err / np.where(A > 0, A, 1.0)))
    print(f"nc={nc} npix={npix}: BF16X6 max |err| / sum|terms| {rel:.2e}")
    assert rel <= 2.0 ** -40
    assert np.array_equal(g, np.swapaxes(g, 1, 2))


def test_gram_rejects_unsupported(dev):
    import torch
    cols, w = _data(5, 1, 130, 40)
    tc, tw = torch.from_numpy(cols).to(dev), torch.from_numpy(w).to(dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_gram(tc, tw, P.PREC_TF32)
    assert e.value.code == 9
    with pytest.raises(P.PsfmError) as e:
        P.psfm_gram(tc[:, :50].contiguous(), tw, P.PREC_F32X2)
    assert e.value.code == 9


def test_pipeline_wait_that_runs_out_returns_timeout(dev):
    """Failure detection without a fault: with the pipeline waits limited to zero polls, the
    first wait for a shared-memory buffer (at the third 32-pixel chunk) runs out; every CTA
    then waits for the MMAs it issued, frees its tensor memory and records PSFM_ERR_TIMEOUT,
    which the call returns.  With the default limit restored the same call succeeds and the
    context is intact."""
    import torch
    cols, w = _data(77, 4, 52, 200)
    G, A = _reference(cols, w)
    tc, tw = torch.from_numpy(cols).to(dev), torch.from_numpy(w).to(dev)
    try:
        P.set_pipeline_wait_limit(0)
        for prec in (P.PREC_TF32, P.PREC_BF16X3):
            with pytest.raises(P.PsfmError) as e:
                P.psfm_gram(tc, tw, prec)
            assert e.value.code == 6
    finally:
        P.set_pipeline_wait_limit(P.WAIT_LIMIT_DEFAULT)
    g = P.psfm_gram(tc, tw, P.PREC_BF16X3).cpu().numpy()
    assert np.all(np.abs(g - G) <= 2.0 * (4 * 2.0 ** -18 + 3 * 200 * 2.0 ** -24) * A)
    torch.cuda.synchronize()
