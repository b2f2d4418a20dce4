"""GPU parity of integer binning (psfm_bin, Sec. 4.3) against the FP64 oracle: sums, masks
and the binned variance and pseudo-matrix, on a ragged image with masks and a correlated
input pseudo-matrix."""
import numpy as np
import pytest

from gpu_common import device, host
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.mark.parametrize("b", [1, 2, 3, 4, 7])
def test_bin_matches_oracle(dev, b):
    import torch
    rng = np.random.default_rng(b)
    H, W = 203, 190
    img = rng.normal(500.0, 30.0, (H, W)).astype(np.float32)
    var = rng.uniform(400.0, 900.0, (H, W)).astype(np.float32)
    m = np.zeros((H, W), np.uint16)
    m[rng.random((H, W)) < 0.02] = 1
    m[rng.random((H, W)) < 0.01] |= 1 << 9  # a bit outside badmask: carried, not masking
    K = np.array([[0.0, 0.1, 0.05], [0.1, 0.6, 0.3], [0.02, 0.2, 0.0]])
    C = O.pseudo_conv(K, np.ones((1, 1)))
    C = C / C[2, 2]
    put = lambda a: torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).to(dev)
    out, ov, om, cov = P.psfm_bin(put(img), put(var), put(m), b, 0xFF,
                                  torch.from_numpy(C).to(dev))
    Ib, Vb, Mb, Pb = O.bin_image(img, var, m, b, 0xFF, C)
    assert np.array_equal(host(om), Mb)
    assert np.allclose(host(out), Ib, rtol=1e-6, atol=1e-3)
    assert np.allclose(host(ov), Vb, rtol=1e-6)
    assert np.allclose(cov.cpu().numpy(), Pb, rtol=1e-12, atol=1e-14)
