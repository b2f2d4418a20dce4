"""Pseudo-matrix resampling by a non-integer scale (Sec. 4.4) through psfm_resample_cov against
the FP64 oracle (FP64 on both sides: sums in a different order only)."""
import numpy as np
import pytest

from gpu_common import device
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


def _pseudo(seed, w):
    ob = O.Basis((0.8, 1.6, 3.0), (4, 2, 2), (w - 1) // 4, 0)
    rng = np.random.default_rng(seed)
    nb = len(O.basis_terms(ob))
    coeff = np.concatenate([rng.normal(0, 0.05, nb), [0.0]])
    sol = O.Solution(1.0, coeff, 0.0, ob, 256, 256)
    return O.pseudo_matrix(sol, O.Config(cov_grid=1))


@pytest.mark.parametrize("scale", [0.55, 1.0, 1.37, 2.0, 2.5, 3.0, 7.9])
def test_resample_matches_oracle(dev, scale):
    import torch
    C = _pseudo(4, 33)
    g = P.psfm_resample_cov(torch.from_numpy(C).to(dev), scale).cpu().numpy()
    o = O.resample_pseudo(C, scale)
    assert g.shape == o.shape
    assert np.allclose(g, o, rtol=1e-12, atol=1e-14)


def test_resample_rejects_bad_sizes(dev):
    import torch
    C = torch.zeros((4, 4), dtype=torch.float64, device=dev)
    with pytest.raises(P.PsfmError):
        P.psfm_resample_cov(C, 1.5)
    with pytest.raises(P.PsfmError):
        P.psfm_resample_cov(torch.zeros((5, 5), dtype=torch.float64, device=dev), 0.0)
