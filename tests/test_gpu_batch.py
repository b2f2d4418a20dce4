"""Batched subtraction (psfm_batch_* through the C ABI): chips of different sizes, bases and
spatial orders, run concurrently on several streams and replayed from a CUDA graph, give the
same results as one psfm_subtract per chip."""
import numpy as np
import pytest

from gpu_common import device, host, specs, upload
from paper_1901_09999_gb300 import psfm as P
from paper_1901_09999_gb300 import synth

pytestmark = pytest.mark.gpu


def _chips(dev):
    recipes = [(11, 300, 260, (0.7, 1.5, 3.0), (4, 2, 2), 8, 1),
               (12, 420, 380, (0.8, 1.6, 3.2), (6, 4, 2), 10, 2),
               (13, 257, 333, (0.9, 1.8), (3, 2), 7, 3)]
    chips, bases, fields = [], [], []
    for seed, W, H, sig, deg, h, S in recipes:
        f = synth.small_gaussian_field(seed, size=H, width=W, n_stars=W * H // 900)
        t = upload(f, dev)
        chips.append(dict(img=t["sci"], ref=t["ref"], var_img=t["var_sci"], var_ref=t["var_ref"],
                          mask_img=t["mask_sci"], mask_ref=t["mask_ref"]))
        bases.append(P.basis_spec(sig, deg, h, S))
        fields.append(f)
    return chips, bases


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_single_chip_calls(graph):
    import torch
    dev = device()
    chips, bases = _chips(dev)
    cfg = P.config(badmask=synth.BADMASK, grid_nx=4, grid_ny=4, precision=P.PREC_F32X2)
    ref = []
    for c, b in zip(chips, bases):
        D, V, M, cov, sol = P.psfm_subtract(c["img"], c["ref"], c["var_img"], c["var_ref"],
                                            c["mask_img"], c["mask_ref"], b, cfg)
        ref.append((host(D), host(V), host(M), cov.cpu().numpy(), sol))
    batch = P.Batch(chips, bases, cfg, n_streams=2, want_cov=True)
    stream = torch.cuda.Stream() if graph else None
    for rep in range(2):                      # second run replays the captured graph
        if stream is not None:
            with torch.cuda.stream(stream):
                batch.run(stream)
        else:
            batch.run(None)
        sols = batch.solutions(stream)
        assert batch.kernel_count() > 0
        for i, (D, V, M, cov, sol) in enumerate(ref):
            assert np.array_equal(host(batch.diff[i]), D)
            assert np.array_equal(host(batch.diff_var[i]), V)
            assert np.array_equal(host(batch.diff_mask[i]), M)
            assert np.allclose(batch.cov[i].cpu().numpy(), cov, rtol=1e-12, atol=1e-15)
            assert sols[i].b0 == sol.b0 and np.array_equal(sols[i].coeff, sol.coeff)
            assert sols[i].n_iter == sol.n_iter and sols[i].r_bad == sol.r_bad
    batch.close()
