"""Writes helmholtz3d_16m_ewald_rows.txt: the ground-truth potential (Eq. 1
with the image sum of Eq. 2, evaluated by Ewald splitting in oracle.ewald) at
32 seeded rows -- 16 of the uniform points, 16 of the sphere-surface points --
of the 3D-periodic Helmholtz workload with a Bloch phase shift: unit cube,
k = 2 pi 2, k0 = (0.2k, 0.2k, 0), N = 1.6e7 (inputs.helmholtz3d()).
Calls only oracle/ and the seeded input generator.  The spectral half's
structure factor is formed once, the spatial halves row by row on all host
cores (about 10 minutes on 8 cores, 25 GB of host memory).

    python tests/golden/make_helmholtz3d_16m_ewald_rows.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "helmholtz3d_16m_ewald_rows.txt")
E_SPLIT = 6.0
TOL = 1e-15
_W = None


def _load():
    global _W
    if _W is None:
        sys.path.insert(0, ROOT)
        from paper_2312_02376_gb300 import inputs
        _W = inputs.helmholtz3d()
    return _W


def _row(args):
    m, setup = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import ewald
    W = _load()
    q = W.q.astype(np.complex128)
    L = np.asarray(W.D, np.float64)
    k0 = np.asarray(W.k0, np.complex128)
    _, rcut, _ = ewald.splitting_cutoffs(W.k, E_SPLIT, TOL)
    u = ewald.spatial_part(W.points, q, m, L, (0, 1, 2), W.k, k0, E_SPLIT, rcut)
    u += ewald.spectral_3d_at(setup, W.points[m])
    return m, complex(u)


def rows_of(W):
    """16 uniform and 16 sphere-surface points (the last quarter), seeded."""
    rng = np.random.default_rng(123)
    nu = (3 * W.N) // 4
    return np.concatenate([rng.choice(nu, 16, replace=False), nu + rng.choice(W.N - nu, 16, replace=False)])


def main():
    sys.path.insert(0, ROOT)
    from oracle import ewald
    W = _load()
    L = np.asarray(W.D, np.float64)
    k0 = np.asarray(W.k0, np.complex128)
    _, _, Gc = ewald.splitting_cutoffs(W.k, E_SPLIT, TOL)
    setup = ewald.spectral_3d_setup(W.points, W.q.astype(np.complex128), L, W.k, k0, E_SPLIT, Gc, chunk=4096)
    rows = rows_of(W)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(_row, [(int(m), setup) for m in rows])
    with open(OUT, "w") as f:
        f.write("# Ewald-split ground truth of Eq. 1 (oracle.ewald, E = %g, tol %g) at 32 rows (16 uniform, 16 on\n"
                % (E_SPLIT, TOL))
        f.write("# the sphere surfaces) of the 3D-periodic Helmholtz + Bloch workload: unit cube, k = 2 pi 2,\n")
        f.write("# k0 = (0.2k, 0.2k, 0), N = 16000000 (inputs.helmholtz3d()).  Written by\n")
        f.write("# make_helmholtz3d_16m_ewald_rows.py.\n")
        f.write("# row  re  im\n")
        for m, u in res:
            f.write("%d %.17e %.17e\n" % (m, u.real, u.imag))


if __name__ == "__main__":
    main()
