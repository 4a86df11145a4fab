"""Writes helmholtz2d_262k_ewald_rows.txt: the ground-truth potential (Eq. 1
with the image sum of Eq. 2, evaluated by Ewald splitting in oracle.ewald) at
16 seeded rows of the 2D-periodic Helmholtz workload with N = 262144 points.
Calls only oracle/ and the seeded input generator.  Runs on all host cores
(about 6 minutes on 8 cores).

    python tests/golden/make_helmholtz2d_262k_ewald_rows.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "helmholtz2d_262k_ewald_rows.txt")
E_SPLIT = 12.0


def _row(m):
    sys.path.insert(0, ROOT)
    from oracle import ewald
    from paper_2312_02376_gb300 import inputs
    W = inputs.helmholtz2d()
    u = ewald.potential(W.points, W.q.astype(np.complex128), [m], W.D, W.pdims, W.k, W.k0, E_SPLIT, chunk=2048)[0]
    return m, complex(u)


def main():
    sys.path.insert(0, ROOT)
    from paper_2312_02376_gb300 import inputs
    W = inputs.helmholtz2d()
    rows = np.random.default_rng(123).choice(W.N, 16, replace=False)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(_row, [int(m) for m in rows])
    with open(OUT, "w") as f:
        f.write("# Ewald-split ground truth of Eq. 1 (oracle.ewald, E = %g, tol 1e-15) at 16 rows of the\n" % E_SPLIT)
        f.write("# 2D-periodic Helmholtz + Bloch workload: cell 1 x 1 x 0.5, k = 2 pi 0.8, k0 = (0.3k, 0.1k, 0),\n")
        f.write("# N = 262144 (inputs.helmholtz2d()).  Written by make_helmholtz2d_262k_ewald_rows.py.\n")
        f.write("# row  re  im\n")
        for m, u in res:
            f.write("%d %.17e %.17e\n" % (m, u.real, u.imag))


if __name__ == "__main__":
    main()
