"""Write the FP64 oracle's solution for the full-chip workload (seed 2) to
``full_chip_seed2_oracle.npz`` beside this script.

Calls only the oracle and the seeded input generator: the 4846 x 4868 Moffat chip of
``synth.full_chip_field(2)``, basis sigma (0.8, 1.6, 3.2), degrees (6, 4, 2), h = 15, spatial
order 2, 15 x 20 stamp grid, other options at their defaults (Sec. 3.3 stamps and rejection,
Sec. 3.2 normalisation).  The full-size GPU parity tests compare against this file and
evaluate the oracle at sampled pixels with the stored solution.

    python tests/golden/make_full_chip_solution.py      # about 3 minutes
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import psfm_oracle as O  # noqa: E402
from paper_1901_09999_gb300 import synth  # noqa: E402

SEED = 2
BASIS = ((0.8, 1.6, 3.2), (6, 4, 2), 15, 2)
GRID = (15, 20)


def main():
    f = synth.full_chip_field(SEED)
    ob = O.Basis(*BASIS)
    oc = O.Config(grid_nx=GRID[0], grid_ny=GRID[1], badmask=synth.BADMASK)
    cand, med = O.extract_candidates(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci,
                                     ob, oc)
    sol = O.solve_kernel(f.ref, f.sci, f.var_ref, f.var_sci, f.mask_ref, f.mask_sci, ob, oc,
                         cand)
    np.savez_compressed(
        os.path.join(HERE, "full_chip_seed2_oracle.npz"),
        seed=SEED, basis_sigma=np.array(BASIS[0]), degrees=np.array(BASIS[1]), h=BASIS[2],
        S=BASIS[3], grid=np.array(GRID), median=np.float32(med), cand=sol.cand,
        status=sol.status, chi2=sol.chi2, b0=sol.b0, d0=sol.d0, coeff=sol.coeff,
        n_iter=sol.n_iter, n_used=sol.n_used, r_bad=O.r_bad(sol))


if __name__ == "__main__":
    main()
