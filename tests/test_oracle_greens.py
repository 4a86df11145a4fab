"""Pins for oracle.greens (Eq. 2, Eq. pgf, Eq. lgf) and oracle.ewald.

Each series is checked against something it is not built from:
brute-force image sums of Eq. 2 (which converge for a lossy wavenumber),
the independent Ewald splitting, a textbook lattice constant, and the
small-k limit that the paper states (Sec. 2, after Eq. lgf)."""
import os

import numpy as np
import pytest

from oracle import ewald, greens

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R = np.array([[0.3, 0.2, 0.15], [0.1, -0.4, 0.35], [0.45, 0.05, -0.2], [-0.33, 0.41, 0.02]])


def _brute(r, L, pd, k, k0, M):
    return greens.image_sum(r, L, pd, k, k0, greens.image_offsets(pd, M))


@pytest.mark.parametrize("pd", [(0,), (2,), (0, 1), (1, 2), (0, 1, 2)])
def test_pgf_matches_lossy_image_sum(pd):
    # Im k = -4: image terms decay like exp(-4 R); M = 10 cells -> < 1e-16
    L = np.array([1.0, 1.0, 1.0])
    k = 2.5 - 4.0j
    k0 = np.array([0.7 - 0.2j, 0.3 + 0.1j, -0.4 + 0.3j])
    k0 = np.where(np.isin(np.arange(3), pd), k0, 0)
    b = _brute(R, L, pd, k, k0, 10 if len(pd) < 3 else 9)
    s = greens.pgf(R, L, pd, k, k0)
    assert np.max(np.abs(b - s)) / np.max(np.abs(b)) < 1e-12


def test_pgf_converges_exponentially_fig2_parameters():
    # Fig. 2(a): L = 1, k = -1-j, k0 = (1-j, 1+j, -1+j), x = y = z = 0.5.
    # (Here |Im k0| = |Im k|, so the image sum of Eq. 2 itself does not
    # converge; the series is its continuation.)  The paper's claim is
    # exponential convergence in the number of terms: partial sums over
    # growing square windows of Floquet modes approach the limit
    # geometrically.
    Lx = Ly = 1.0
    k = -1.0 - 1.0j
    kx0, ky0 = 1 - 1j, 1 + 1j
    x = y = z = 0.5
    vals = []
    for M in range(2, 16):
        m = np.arange(-M, M + 1)
        kx = kx0 + 2 * np.pi * m / Lx
        ky = ky0 + 2 * np.pi * m / Ly
        kz = greens.csqrt_neg_imag(k * k - kx[:, None] ** 2 - ky[None, :] ** 2)
        t = np.exp(-1j * kx[:, None] * x - 1j * ky[None, :] * y - 1j * kz * abs(z)) / (2j * kz * Lx * Ly)
        vals.append(t.sum())
    err = np.abs(np.array(vals) - vals[-1])[:-1]
    assert err[-2] < 1e-14 * abs(vals[-1])
    # geometric decay: each extra shell of modes gains a factor > 5
    assert np.all(err[1:5] < 0.05 * err[:4])
    ref = greens.pgf(np.array([[x, y, z]]), np.ones(3), (0, 1), k, np.array([kx0, ky0, 0]))[0]
    assert abs(ref - vals[-1]) < 1e-13 * abs(ref)


def test_lgf3_equals_ewald_up_to_constant():
    L = np.array([1.0, 1.0, 1.0])
    a = ewald.greens_function(R, L, (0, 1, 2), 0.0, np.zeros(3), 3.0).real
    c = greens.lgf(R, L, (0, 1, 2))
    d = a - c
    assert np.ptp(d) < 1e-12


def test_lgf3_anisotropic_cell_vs_ewald():
    L = np.array([1.0, 0.7, 1.3])
    a = ewald.greens_function(R * 0.5, L, (0, 1, 2), 0.0, np.zeros(3), 3.0).real
    c = greens.lgf(R * 0.5, L, (0, 1, 2))
    assert np.ptp(a - c) < 1e-12


def _neutral_set():
    rng = np.random.default_rng(5)
    src = rng.random((6, 3)) * 0.6
    q = rng.standard_normal(6)
    q -= q.mean()
    return src, q


@pytest.mark.parametrize("pd", [(0,), (0, 1)])
def test_lgf_is_small_k_limit_of_pgf(pd):
    # Sec. 2: Eq. lgf_1 is the k0, k -> 0 limit of Eq. pgf_1 for neutral sources.
    L = np.array([1.0, 1.0, 1.0])
    src, q = _neutral_set()
    obs = np.array([0.31, 0.77, 0.93])
    kk = 1e-6 * (1 - 1j)
    pg = sum(qn * greens.pgf(obs - s, L, pd, kk, np.zeros(3)) for qn, s in zip(q, src))
    lg = sum(qn * greens.lgf(obs - s, L, pd) for qn, s in zip(q, src))
    assert abs(pg - lg) < 1e-6 * np.sum(np.abs(q))


def test_ewald3_helmholtz_vs_lossy_image_sum():
    L = np.array([1.0, 1.0, 0.5])
    k = 3.0 - 4.0j
    k0 = np.array([0.7 - 0.2j, 0.3 + 0.1j, 0.4])
    b = _brute(R, L, (0, 1, 2), k, k0, 14)
    for E in (2.0, 4.0):
        e = ewald.greens_function(R, L, (0, 1, 2), k, k0, E)
        assert np.max(np.abs(b - e)) / np.max(np.abs(b)) < 1e-11


def test_ewald2d_vs_lossy_image_sum_and_real_k_vs_pgf():
    L = np.array([1.0, 1.0, 0.5])
    k = 3.0 - 3.0j
    k0 = np.array([0.7 - 0.2j, 0.3 + 0.1j, 0.0])
    b = _brute(R, L, (0, 1), k, k0, 13)
    e = ewald.greens_function(R, L, (0, 1), k, k0, 3.0)
    assert np.max(np.abs(b - e)) / np.max(np.abs(b)) < 1e-13
    k = 2 * np.pi * 0.8
    k0 = np.array([0.3 * k, 0.1 * k, 0.0])
    e = ewald.greens_function(R, L, (0, 1), k, k0, 3.0)
    s = greens.pgf(R, L, (0, 1), k, k0)
    assert np.max(np.abs(e - s)) / np.max(np.abs(s)) < 1e-13


@pytest.mark.parametrize("pd", [(0,), (2,)])
def test_ewald1d_vs_lossy_image_sum_and_real_k_vs_pgf1(pd):
    # 1D lattice: the Ewald split with the exponential-integral spectral part
    # against the brute-force image sum for a lossy k (any E), and against
    # Eq. pgf_1 (the Hankel-function series) for real k
    pytest.importorskip("mpmath")
    L = np.array([0.5, 0.5, 0.5])
    L[pd[0]] = 0.25
    k = 3.0 - 2.0j
    k0 = np.zeros(3, complex)
    k0[pd[0]] = 0.7 - 0.1j
    b = _brute(R, L, pd, k, k0, 80)
    for E in (2.0, 3.5):
        e = ewald.greens_function(R, L, pd, k, k0, E)
        assert np.max(np.abs(b - e)) / np.max(np.abs(b)) < 1e-12
    for k, kz in ((2 * np.pi * 0.5, 0.0), (3.0, 0.9)):
        k0 = np.zeros(3)
        k0[pd[0]] = kz
        e = ewald.greens_function(R, L, pd, k, k0, 2.5)
        s = greens.pgf(R, L, pd, k, k0)
        assert np.max(np.abs(e - s)) / np.max(np.abs(s)) < 1e-12


def test_madelung_nacl():
    ref = float(open(os.path.join(GOLDEN, "madelung_nacl.txt")).read().split("\n")[-2])
    pts = np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5],
                    [.5, 0, 0], [0, .5, 0], [0, 0, .5], [.5, .5, .5]])
    q = np.array([1, 1, 1, 1, -1, -1, -1, -1], complex)
    for E in (3.0, 5.0):
        u = ewald.potential(pts, q, [0, 4], np.ones(3), (0, 1, 2), 0.0, np.zeros(3), E)
        assert abs(-u[0].real * 4 * np.pi * 0.5 - ref) < 1e-13
        assert abs(u[1].real * 4 * np.pi * 0.5 - ref) < 1e-13


def test_bloch_periodicity_of_series():
    # G^p(r + a) = exp(-j k0.a) G^p(r) for a lattice vector a (Eq. 2)
    L = np.array([1.0, 1.0, 0.5])
    k = 2 * np.pi * 0.8
    k0 = np.array([0.3 * k, 0.1 * k, 0.0])
    a = np.array([1.0, -1.0, 0.0])
    g1 = greens.pgf(R, L, (0, 1), k, k0)
    g2 = greens.pgf(R + a, L, (0, 1), k, k0)
    assert np.allclose(g2, np.exp(-1j * k0 @ a) * g1, rtol=1e-12, atol=0)
