"""The seeded input recipes (host logic, no GPU): every workload generator
draws what its docstring states -- point counts per part, the cell, sphere
radii and cluster bounds, strength distributions and neutrality, grid rules
-- and the same seed gives the same arrays.  Run at reduced N where the full
workload would take gigabytes."""
import numpy as np
import pytest

from paper_2312_02376_gb300 import inputs


def test_coulomb3d_4k_recipe():
    W = inputs.coulomb3d()
    assert W.N == 4096 and W.points.shape == (4096, 3) and W.n == (32, 32, 32) and W.pdims == (0, 1, 2)
    assert np.all((W.points >= 0) & (W.points < 1))
    assert set(np.unique(W.q)) == {-1.0, 1.0} and W.q.sum() == 0.0
    assert W.k == 0.0 and W.precision == "fp64"


def test_helmholtz2d_recipe_half_uniform_half_on_the_sphere():
    W = inputs.helmholtz2d(N=8192, n=(32, 32, 16))
    D = np.array(W.D)
    assert W.D == (1.0, 1.0, 0.5) and W.pdims == (0, 1)
    uni, sph = W.points[:4096], W.points[4096:]
    assert np.all((uni >= 0) & (uni < D))
    r = np.linalg.norm(sph - np.array([0.5, 0.5, 0.25]), axis=1)
    assert np.allclose(r, 0.2, rtol=0, atol=1e-12)
    assert W.q.dtype == np.complex64
    # CN(0, 1): E|q|^2 = 1, real and imaginary parts of equal variance
    assert abs(np.mean(np.abs(W.q) ** 2) - 1.0) < 0.05
    assert abs(np.var(W.q.real) - np.var(W.q.imag)) < 0.05
    k = 2 * np.pi * 0.8
    assert W.k == pytest.approx(k) and W.k0 == pytest.approx((0.3 * k, 0.1 * k, 0.0))


def test_helmholtz1d_set_recipe():
    W = inputs.helmholtz1d_set(20000, nrhs=2)
    D = np.array(W.D)
    assert W.D == (1.0, 0.25, 0.25) and W.pdims == (2,) and W.k == pytest.approx(np.pi)
    assert W.q.shape == (20000, 2) and W.q.dtype == np.complex64
    # every point inside the cell: clusters redrawn in x and y, wrapped along z
    assert np.all((W.points >= 0) & (W.points < D))
    # grid step half the mean point spacing: about eight nodes per point
    h = (np.prod(D) / 20000) ** (1 / 3) / 2
    assert W.n == tuple(int(max(5, round(D[d] / h) + 1)) for d in range(3))
    nodes = np.prod(np.array(W.n) - 1)
    assert 6 < nodes / 20000 < 10
    assert W.b == 5 and W.nf == (20, 10, 10)
    # the clustered half: 8 clusters of standard deviation 0.02 about their centres
    # (x spread per cluster; a cluster near a face in x is truncated there)
    cl = W.points[10000:].reshape(8, 1250, 3)
    assert np.median(np.std(cl[:, :, 0], axis=1)) == pytest.approx(0.02, rel=0.1)


def test_helmholtz1d_batch_sizes_are_log_uniform_within_bounds():
    sets = inputs.helmholtz1d_batch(nsets=16, Nmin=200, Nmax=4000, nrhs=1)
    Ns = np.array([W.N for W in sets])
    assert len(sets) == 16 and np.all((Ns >= 200) & (Ns <= 4000))
    again = inputs.helmholtz1d_batch(nsets=16, Nmin=200, Nmax=4000, nrhs=1)
    assert [W.N for W in again] == list(Ns)
    assert all(np.array_equal(a.points, b.points) and np.array_equal(a.q, b.q) for a, b in zip(sets, again))


def test_coulomb3d_1m_recipe_is_neutral():
    W = inputs.coulomb3d_big(N=50000, n=32)
    assert W.q.dtype == np.float32 and abs(float(np.sum(W.q, dtype=np.float64))) < 1e-2
    assert np.all((W.points >= 0) & (W.points < 1)) and W.pdims == (0, 1, 2) and W.k == 0.0


def test_helmholtz3d_recipe_uniform_fraction_and_spheres():
    N = 16000
    W = inputs.helmholtz3d(N=N, n=32)
    nu = 12000
    assert np.all((W.points[:nu] >= 0) & (W.points[:nu] < 1))
    sph = W.points[nu:]
    # 8 spheres of radius 0.05, all inside the unit cell
    assert np.all((sph > 0) & (sph < 1))
    per = (N - nu) // 8
    for s in range(8):
        part = sph[s * per:(s + 1) * per]
        c = part.mean(axis=0)
        r = np.linalg.norm(part - c, axis=1)
        assert np.all(np.abs(r - 0.05) < 5e-3)
    k = 2 * np.pi * 2.0
    assert W.k == pytest.approx(k) and W.k0 == pytest.approx((0.2 * k, 0.2 * k, 0.0))
    assert W.nf == (51, 51, 51) and W.b == 5
    assert inputs.helmholtz3d(N=N, n=32, uniform=0.0).points.shape == (N, 3)


def test_coax_is_neutral_with_observers_on_the_axis_and_outside():
    src, q, obs = inputs.coax()
    assert abs(q.sum()) < 1e-15 and q[:64 * 16].sum() == pytest.approx(1.0)
    r = np.linalg.norm(src[:, :2] - 2.5, axis=1)
    assert np.allclose(r[:64 * 16], 1.0) and np.allclose(r[64 * 16:], 2.0)
    ro = np.linalg.norm(obs[:, :2] - 2.5, axis=1)
    assert np.allclose(ro[:8], 0.0) and np.allclose(ro[8:], 2.3)
    assert np.all((src[:, 2] > 0) & (src[:, 2] < 1)) and np.all((obs[:, 2] > 0) & (obs[:, 2] < 1))


def test_seeds_are_fixed_and_distinct():
    a, b = inputs.helmholtz2d(N=1024, n=(16, 16, 8)), inputs.helmholtz2d(N=1024, n=(16, 16, 8))
    assert np.array_equal(a.points, b.points) and np.array_equal(a.q, b.q)
    c = inputs.helmholtz2d(N=1024, n=(16, 16, 8), salt=1)
    assert not np.array_equal(a.points, c.points)
    r1 = inputs.random_case(100, (1, 1, 1), (0, 1, 2), 1.0, (0, 0, 0), (9, 9, 9), seed=3)
    r2 = inputs.random_clustered_case(100, (1, 1, 1), (0, 1, 2), 1.0, (0, 0, 0), (9, 9, 9), seed=3)
    assert not np.array_equal(r1.points, r2.points)
    assert np.all((r2.points >= 0) & (r2.points <= 1))
