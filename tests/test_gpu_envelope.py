"""GPU envelope PSF of stack inputs (Sec. 5.1) through psfm_envelope_fwhm against the FP64
oracle: Gaussian inputs (the envelope is the widest), elliptical inputs (circularised), and
Gaussian-Moffat mixtures like the skycell warps', with the automatic and explicit radius."""
import numpy as np
import pytest

from gpu_common import device
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu

# FP32 profiles and double-float sums on the GPU: the fitted width agrees to about 1e-7.
FWHM_RTOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    return device()


def _random_models(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        f = rng.uniform(3.0, 8.0)
        e = rng.uniform(0.0, 0.2)
        out.append((f, f * (1 - e), rng.uniform(0.0, 1.0), rng.uniform(2.0, 5.0)))
    return out


@pytest.mark.parametrize("models,radius", [
    ([(4.0, 4.0, 0.0, 3.0), (6.2, 6.2, 0.0, 3.0), (5.0, 5.0, 0.0, 3.0)], 0),
    ([(6.0, 4.0, 0.0, 3.0)], 0),
    ([(5.0, 5.0, 1.0, 3.0)], 25),
    (_random_models(1, 5), 0),
    (_random_models(2, 16), 30),
    (_random_models(3, 32), 0),
])
def test_envelope_matches_oracle(dev, models, radius):
    g = P.psfm_envelope_fwhm(models, radius, device=dev)
    o = O.envelope_fwhm(models, radius)
    assert abs(g - o) <= FWHM_RTOL * o, (g, o)


def test_envelope_of_skycell_warps(dev):
    warps, _ = synth.skycell_warps(7, 6, 128, 5, gap_range=(40, 80), block_range=(5, 20),
                                   masked_range=(0.02, 0.05))
    models = [w["psf_model"] for w in warps]
    g = P.psfm_envelope_fwhm(models, device=dev)
    assert abs(g - O.envelope_fwhm(models)) <= FWHM_RTOL * g


def test_envelope_rejects_bad_models(dev):
    for models, radius in (([(0.0, 4.0, 0.0, 3.0)], 0), ([(4.0, 4.0, 1.5, 3.0)], 0),
                           ([(4.0, 4.0, 0.5, 1.0)], 0), ([(4.0, 4.0, 0.0, 3.0)], 65),
                           ([(30.0, 30.0, 0.0, 3.0)], 0), ([], 0)):
        with pytest.raises(P.PsfmError) as e:
            P.psfm_envelope_fwhm(models, radius, device=dev)
        assert e.value.code == 1
