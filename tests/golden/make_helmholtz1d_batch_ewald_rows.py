"""Writes helmholtz1d_batch_ewald_rows.txt: the ground-truth potential (Eq. 1
with the image sum of Eq. 2 on a 1D lattice, evaluated by Ewald splitting in
oracle.ewald) at 8 seeded rows of the smallest and of the largest point set
of the batched 1D-periodic Helmholtz workload (inputs.helmholtz1d_batch()),
for its first and last right-hand sides.  Calls only oracle/ and the seeded
input generator (a few minutes on all host cores).

    python tests/golden/make_helmholtz1d_batch_ewald_rows.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "helmholtz1d_batch_ewald_rows.txt")
E_SPLIT = 2.0


def _job(args):
    si, r, m = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import ewald
    from paper_2312_02376_gb300 import inputs
    W = inputs.helmholtz1d_batch()[si]
    q = W.q[:, r].astype(np.complex128)
    u = ewald.potential(W.points, q, [m], W.D, W.pdims, W.k, W.k0, E_SPLIT)[0]
    return si, r, m, complex(u)


def picks():
    """(set index, right-hand side, row) of the stored values."""
    sys.path.insert(0, ROOT)
    from paper_2312_02376_gb300 import inputs
    sets = inputs.helmholtz1d_batch()
    Ns = [W.N for W in sets]
    out = []
    for si in (int(np.argmin(Ns)), int(np.argmax(Ns))):
        rows = np.random.default_rng(100 + si).choice(Ns[si], 8, replace=False)
        for r in (0, sets[si].nrhs - 1):
            out += [(si, r, int(m)) for m in rows]
    return out


def main():
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(_job, picks())
    with open(OUT, "w") as f:
        f.write("# Ewald-split ground truth of Eq. 1 on a 1D lattice (oracle.ewald, E = %g) at 8 rows of the\n"
                % E_SPLIT)
        f.write("# smallest and of the largest point set of the batched 1D-periodic Helmholtz workload\n")
        f.write("# (inputs.helmholtz1d_batch()), first and last right-hand side.  Written by\n")
        f.write("# make_helmholtz1d_batch_ewald_rows.py.\n")
        f.write("# set  rhs  row  re  im\n")
        for si, r, m, u in res:
            f.write("%d %d %d %.17e %.17e\n" % (si, r, m, u.real, u.imag))


if __name__ == "__main__":
    main()
