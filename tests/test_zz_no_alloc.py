"""psfm_convolve_noalloc: the workspace-free convolution for callers that cannot allocate
device memory (for example a plugin whose host application owns the device memory pool, or a
real-time scheduler that bans allocation after start-up).

It must give the same image, variance and mask as psfm_convolve on the same inputs, on two
calls in a row with different inputs (its shared scratch must not carry state from one call
to the next).  Kept in a file collected last so that a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

from gpu_common import IMG_TOL_SIGMA, VAR_RTOL, device, host, specs, upload
from oracle import psfm_oracle as O
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu


def _solution(ob, W, H, seed):
    rng = np.random.default_rng(seed)
    nb, ns = len(O.basis_terms(ob)), len(O.spatial_terms(ob.S))
    a = rng.normal(0, 0.05, (nb, ns))
    a[0, 0] = 0.6
    return P.Solution.from_values(1.02, 1.5, a.ravel(), 2)


@pytest.mark.parametrize("diff", [True, False])
def test_noalloc_matches_workspace_entry_point(diff):
    dev = device()
    for call, (seed, W, H, S) in enumerate([(11, 301, 257, 2), (12, 200, 333, 1)]):
        f = synth.small_gaussian_field(seed, size=H, width=W, n_stars=W * H // 1500)
        b, c, ob, oc = specs((0.8, 1.7, 3.0), (4, 2, 2), 9, S, badmask=synth.BADMASK)
        sol = _solution(ob, W, H, seed)
        t = upload(f, dev, pad=call)
        kw = dict(img=t["sci"], var_img=t["var_sci"], mask_img=t["mask_sci"]) if diff else {}
        D0, V0, M0, _ = P.psfm_convolve(t["ref"], t["var_ref"], t["mask_ref"], b, c, sol,
                                        want_cov=False, **kw)
        D1, V1, M1 = P.psfm_convolve_noalloc(t["ref"], t["var_ref"], t["mask_ref"], b, c, sol, **kw)
        sig = np.sqrt(np.maximum(host(V0), 1e-30))
        assert float((np.abs(host(D1) - host(D0)) / sig).max()) <= IMG_TOL_SIGMA
        assert float((np.abs(host(V1) - host(V0)) / np.abs(host(V0))).max()) <= VAR_RTOL
        assert np.array_equal(host(M1), host(M0))


def test_noalloc_rejects_oversized_images():
    import torch
    dev = device()
    b, c, ob, oc = specs((1.0,), (2,), 4, 0)
    sol = P.Solution.from_values(1.0, 0.0, np.zeros(6), 0)
    img = torch.zeros((8, 4097), device=dev)
    m = torch.zeros((8, 4097), dtype=torch.int16, device=dev)
    with pytest.raises(P.PsfmError) as e:
        P.psfm_convolve_noalloc(img, img, m, b, c, sol)
    assert e.value.code == 8
