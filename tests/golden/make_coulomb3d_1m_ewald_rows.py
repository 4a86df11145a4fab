"""Writes coulomb3d_1m_ewald_rows.txt: the ground-truth potential (Eq. 1 with
the image sum of Eq. 2, 3D-periodic static kernel, evaluated by Ewald
splitting in oracle.ewald; tin-foil, i.e. equal to Eq. lgf_3 up to a constant
that cancels for neutral charges) at 16 seeded rows of the differentiated 3D
Coulomb workload, N = 10^6 uniform points in the unit cube, charges N(0,1)
minus their mean (inputs.coulomb3d_big(), whose FP32 charges are used with
their FP64 mean removed).  Calls only oracle/ and the seeded input generator.
Runs on all host cores (about 2 minutes on 8 cores).

    python tests/golden/make_coulomb3d_1m_ewald_rows.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "coulomb3d_1m_ewald_rows.txt")
E_SPLIT = 6.0


def _charges(W):
    q = W.q.astype(np.float64)
    return q - np.mean(q)


def _row(m):
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import ewald
    from paper_2312_02376_gb300 import inputs
    W = inputs.coulomb3d_big()
    u = ewald.potential(W.points, _charges(W).astype(np.complex128), [m], W.D, W.pdims, 0.0, W.k0, E_SPLIT)[0]
    return m, complex(u)


def main():
    sys.path.insert(0, ROOT)
    from paper_2312_02376_gb300 import inputs
    W = inputs.coulomb3d_big()
    rows = np.random.default_rng(123).choice(W.N, 16, replace=False)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(_row, [int(m) for m in rows])
    with open(OUT, "w") as f:
        f.write("# Ewald-split ground truth of Eq. 1 (oracle.ewald, k = 0, tin-foil, E = %g, tol 1e-15) at 16\n"
                % E_SPLIT)
        f.write("# rows of the 3D-periodic static Coulomb workload: unit cube, N = 1000000 uniform points,\n")
        f.write("# charges inputs.coulomb3d_big().q (FP32) minus their FP64 mean.\n")
        f.write("# Written by make_coulomb3d_1m_ewald_rows.py.\n")
        f.write("# row  re  im\n")
        for m, u in res:
            f.write("%d %.17e %.17e\n" % (m, u.real, u.imag))


if __name__ == "__main__":
    main()
