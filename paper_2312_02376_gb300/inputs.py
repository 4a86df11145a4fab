"""Seeded synthetic workloads (points, source strengths and problem sizes).

This module holds no arithmetic of the method: it only draws points and
source strengths with numpy's PCG64 generator and lists the problem
parameters of each workload.  The CUDA library and the FP64 oracles both take
their inputs from here.

The paper's own workloads are tetrahedral meshes of cubes and of a coaxial
cable (Sec. 4), which are not published; these synthetic point sets stand in
for them.  Each workload below is named by what it is.

  coulomb3d_4k      3D-periodic static Coulomb, unit cube, N = 4096 uniform,
                    charges +-1 in equal numbers (net zero), grid 32^3, p = 4,
                    one near-image layer, FP64.
  helmholtz2d_262k  2D-periodic (x, y) Helmholtz with a Bloch phase shift,
                    cell 1 x 1 x 0.5, k = 2 pi 0.8, k0 = (0.3k, 0.1k, 0),
                    N = 262144: half uniform, half on a sphere of radius 0.2
                    at the cell centre; sources CN(0, 1); grid 128 x 128 x 64,
                    p = 4; complex64 bulk, FP64 far series and correction.
  helmholtz1d_batch 16 sets, 1D-periodic along z Helmholtz, cell
                    1 x 0.25 x 0.25, k = 2 pi 0.5, N log-uniform in
                    [1e4, 5e5] (half uniform, half in 8 Gaussian clusters of
                    sigma 0.02), 64 complex64 right-hand sides; grid step
                    half the mean point spacing, correction radius 5 steps,
                    far grid 20 x 10 x 10.
  coulomb3d_1m      3D static Coulomb, N = 10^6 uniform, charges N(0,1) minus
                    their mean, grid 256^3, p = 4, FP32 bulk; energy gradient.
  helmholtz3d_16m   3D-periodic Helmholtz with Bloch phase, k = 2 pi 2,
                    k0 = (0.2k, 0.2k, 0), N = 1.6e7 (3/4 uniform, 1/4 on 8
                    spheres of radius 0.05), grid 512^3, p = 4, far grid
                    51^3 (ceil(4 k D), the library's default rule).

"Twins" are the same recipes at a smaller N and grid (for tests whose
oracle must finish in seconds).
"""
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2312_02376


@dataclass
class Workload:
    name: str
    D: tuple
    pdims: tuple
    k: float
    k0: tuple
    n: tuple                 # near grid nodes per axis (spanning [0, D])
    p: int
    layers: int
    b: int                   # correction radius (grid steps)
    nf: tuple                # far grid nodes per axis
    pf: int
    precision: str           # "fp64" or "fp32"
    N: int
    nrhs: int = 1
    points: np.ndarray = field(default=None, repr=False)
    q: np.ndarray = field(default=None, repr=False)


def _rng(index, salt=0):
    return np.random.Generator(np.random.PCG64(SEED_BASE + index + 1000 * salt))


def _sphere(rng, n, centre, radius):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return centre + radius * v


def _cn(rng, shape):
    """Circular complex normal CN(0,1): real and imaginary parts N(0, 1/2)."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def coulomb3d(N=4096, n=32, index=0, salt=0, b=5, nf=10):
    rng = _rng(index, salt)
    pts = rng.random((N, 3))
    q = np.concatenate([np.ones(N // 2), -np.ones(N - N // 2)])
    rng.shuffle(q)
    return Workload("coulomb3d_%d" % N, (1.0, 1.0, 1.0), (0, 1, 2), 0.0, (0.0, 0.0, 0.0),
                    (n, n, n), 4, 1, b, (nf, nf, nf), 4, "fp64", N, 1, pts, q.astype(np.float64))


def helmholtz2d(N=262144, n=(128, 128, 64), index=1, salt=0, b=4, nf=(21, 21, 11)):
    rng = _rng(index, salt)
    D = np.array([1.0, 1.0, 0.5])
    nu = N // 2
    uni = rng.random((nu, 3)) * D
    sph = _sphere(rng, N - nu, np.array([0.5, 0.5, 0.25]), 0.2)
    pts = np.concatenate([uni, sph])
    q = _cn(rng, N)
    k = 2 * np.pi * 0.8
    return Workload("helmholtz2d_%d" % N, tuple(D), (0, 1), k, (0.3 * k, 0.1 * k, 0.0),
                    tuple(n), 4, 1, b, tuple(nf), 4, "fp32", N, 1, pts, q.astype(np.complex64))


def helmholtz1d_set(N, index=2, salt=0, b=5, nrhs=64, rng=None, refine=2, nf=(20, 10, 10)):
    """One point set of the batched 1D-periodic Helmholtz workload: cell
    1 x 0.25 x 0.25, periodic along z (L_z = 0.25), k = 2 pi 0.5, no phase
    shift; half the points uniform, half in 8 Gaussian clusters (sigma 0.02,
    centres uniform, wrapped along z, redrawn if outside the cell in x or y);
    grid step (V/N)^(1/3) / refine (refine = 2: about eight nodes per point)
    and correction radius b = 5 steps, which meet the 1e-4 target against the
    1D-lattice Ewald sum (one node per point needs b = 5 on that grid, a
    correction list about eight times longer); far grid 20 x 10 x 10 (the
    length-1 open axis needs 20 nodes: with 13, ceil(4 k D), the far-zone
    interpolation alone leaves 1.9e-4 on the 2.9e5-point set); nrhs CN(0,1)
    sources."""
    rng = rng if rng is not None else _rng(index, salt)
    D = np.array([1.0, 0.25, 0.25])
    nu = N // 2
    uni = rng.random((nu, 3)) * D
    centres = rng.random((8, 3)) * D
    rest = N - nu
    per = np.full(8, rest // 8)
    per[: rest - per.sum()] += 1
    cl = []
    for c, cnt in zip(centres, per):
        pts = c + 0.02 * rng.standard_normal((cnt, 3))
        bad = np.any((pts[:, :2] < 0) | (pts[:, :2] >= D[:2]), axis=1)
        while bad.any():
            pts[bad] = c + 0.02 * rng.standard_normal((int(bad.sum()), 3))
            bad = np.any((pts[:, :2] < 0) | (pts[:, :2] >= D[:2]), axis=1)
        pts[:, 2] = np.mod(pts[:, 2], D[2])
        cl.append(pts)
    pts = np.concatenate([uni] + cl)
    h = (np.prod(D) / N) ** (1.0 / 3.0) / refine
    n = tuple(int(max(5, round(D[d] / h) + 1)) for d in range(3))
    q = _cn(rng, (N, nrhs)).astype(np.complex64)
    k = 2 * np.pi * 0.5
    return Workload("helmholtz1d_%d" % N, tuple(D), (2,), k, (0.0, 0.0, 0.0), n, 4, 1, b,
                    tuple(nf), 4, "fp32", N, nrhs, pts, q)


def helmholtz1d_batch(nsets=16, Nmin=10_000, Nmax=500_000, index=2, salt=0, b=5, nrhs=64):
    """The batched workload: nsets point sets with N log-uniform in
    [Nmin, Nmax] (helmholtz1d_set each)."""
    rng = _rng(index, salt)
    Ns = np.floor(np.exp(rng.uniform(np.log(Nmin), np.log(Nmax), nsets))).astype(np.int64)
    return [helmholtz1d_set(int(N), b=b, nrhs=nrhs, rng=rng) for N in Ns]


def coulomb3d_big(N=1_000_000, n=256, index=3, salt=0, b=5, nf=10):
    rng = _rng(index, salt)
    pts = rng.random((N, 3))
    q = rng.standard_normal(N)
    q = q - np.mean(q)
    return Workload("coulomb3d_%d" % N, (1.0, 1.0, 1.0), (0, 1, 2), 0.0, (0.0, 0.0, 0.0),
                    (n, n, n), 4, 1, b, (nf, nf, nf), 4, "fp32", N, 1, pts, q.astype(np.float32))


def helmholtz3d(N=16_000_000, n=512, index=4, salt=0, b=5, nf=51, uniform=0.75):
    """The 3D-periodic Helmholtz + Bloch recipe; `uniform` is the fraction
    of uniform points (the rest on the 8 spheres)."""
    rng = _rng(index, salt)
    nu = int(round(uniform * N))
    uni = rng.random((nu, 3))
    rest = N - nu
    centres = 0.05 + 0.9 * rng.random((8, 3))
    per = np.full(8, rest // 8)
    per[: rest - per.sum()] += 1
    sph = np.concatenate([_sphere(rng, c, centres[i], 0.05) for i, c in enumerate(per)])
    pts = np.concatenate([uni, sph])
    k = 2 * np.pi * 2.0
    q = _cn(rng, N)
    return Workload("helmholtz3d_%d" % N, (1.0, 1.0, 1.0), (0, 1, 2), k, (0.2 * k, 0.2 * k, 0.0),
                    (n, n, n), 4, 1, b, (nf, nf, nf), 4, "fp32", N, 1, pts, q.astype(np.complex64))


def coax(nt1=64, nt2=128, nz=16, L=1.0, W=5.0, r1=1.0, r2=2.0, nobs=8, r_out=2.3):
    """A coaxial line, periodic along z with period L (Sec. 4's 1D-periodic
    neutral coax): charges on regular lattices on two cylinders about the
    axis of a W x W x L cell, nt1 x nz points of total charge +1 at radius
    r1 and nt2 x nz points of total charge -1 at radius r2 (equal charge
    per point on each cylinder, so the set is exactly neutral).  Observers:
    nobs points on the axis and nobs points at radius r_out outside the outer
    cylinder (angles 2 pi j / nobs), at heights (j + 1/4) L / nobs.  Returns
    (sources (N, 3), strengths (N,), observers (2 nobs, 3))."""
    c = np.array([0.5 * W, 0.5 * W])

    def cylinder(r, nt, charge):
        th = (np.arange(nt) + 0.5) * 2.0 * np.pi / nt
        z = (np.arange(nz) + 0.5) * L / nz
        T, Z = np.meshgrid(th, z, indexing="ij")
        pts = np.stack([c[0] + r * np.cos(T).ravel(), c[1] + r * np.sin(T).ravel(), Z.ravel()], axis=1)
        return pts, np.full(len(pts), charge / len(pts))

    p1, q1 = cylinder(r1, nt1, 1.0)
    p2, q2 = cylinder(r2, nt2, -1.0)
    zo = (np.arange(nobs) + 0.25) * L / nobs
    ang = np.arange(nobs) * 2.0 * np.pi / nobs
    axis = np.stack([np.full(nobs, c[0]), np.full(nobs, c[1]), zo], axis=1)
    out = np.stack([c[0] + r_out * np.cos(ang), c[1] + r_out * np.sin(ang), zo], axis=1)
    return np.vstack([p1, p2]), np.concatenate([q1, q2]), np.vstack([axis, out])


def random_case(N, D, pdims, k, k0, n, p=4, layers=1, b=5, nf=(10, 10, 10), pf=4, seed=0,
                complex_q=True, neutral=False, precision="fp64", nrhs=1):
    """A small uniform case with arbitrary parameters (for parity tests)."""
    rng = _rng(100 + seed)
    D = np.asarray(D, np.float64)
    pts = rng.random((N, 3)) * D
    if complex_q:
        q = _cn(rng, (N, nrhs))
    else:
        q = rng.standard_normal((N, nrhs))
    if neutral:
        q = q - q.mean(axis=0, keepdims=True)
    if nrhs == 1:
        q = q[:, 0]
    return Workload("random_%d" % N, tuple(D), tuple(pdims), k, tuple(k0), tuple(n), p, layers, b,
                    tuple(nf), pf, precision, N, nrhs, pts, q)


def random_clustered_case(N, D, pdims, k, k0, n, p=4, layers=1, b=5, nf=(10, 10, 10), pf=4, seed=0,
                          complex_q=True, neutral=False, precision="fp64", nclusters=3, sigma_steps=0.4):
    """A small case whose points are half uniform and half in nclusters
    Gaussian clusters of standard deviation sigma_steps grid steps (boxes with
    tens of points, as on the sphere surfaces of the 3D workload), clipped
    into the closed cell."""
    rng = _rng(200 + seed)
    D = np.asarray(D, np.float64)
    h = D / (np.asarray(n) - 1)
    nu = N // 2
    centres = rng.random((nclusters, 3)) * D
    per = np.full(nclusters, (N - nu) // nclusters)
    per[: (N - nu) - per.sum()] += 1
    cl = [np.clip(c + sigma_steps * h * rng.standard_normal((cnt, 3)), 0.0, D) for c, cnt in zip(centres, per)]
    pts = np.concatenate([rng.random((nu, 3)) * D] + cl)
    if complex_q:
        q = _cn(rng, N)
    else:
        q = rng.standard_normal(N)
    if neutral:
        q = q - q.mean()
    return Workload("clustered_%d" % N, tuple(D), tuple(pdims), k, tuple(k0), tuple(n), p, layers, b,
                    tuple(nf), pf, precision, N, 1, pts, q)

