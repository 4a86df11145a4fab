"""Ewald-split evaluation of the periodic sum (ground truth), FP64.
TEST INFRASTRUCTURE ONLY.

This is not one of the paper's algorithms: it evaluates the plain definition,
Eq. 1 with the image sum of Eq. 2 (self term n = m, i = 0 dropped, every other
image of every source kept), by the classical Ewald splitting so that both
halves converge exponentially.  For a splitting parameter E:

  spatial  f_E(R) = [e^{-jkR} erfc(RE - jk/2E) + e^{jkR} erfc(RE + jk/2E)] / (8 pi R)
           (k = 0: erfc(RE)/(4 pi R))
  3D lattice spectral part (Poisson summation, k_G = k0 + G, V = cell volume):
           (1/V) sum_G exp((k^2-|k_G|^2)/4E^2)/(|k_G|^2-k^2) exp(-j k_G.r)
  2D lattice (periodic x, y; z free; A = cell area, kz from Eq. pgf's branch):
           sum_{m,n} exp(-j kt.rho)/(4 j kz A)
                 * [e^{-j kz z} erfc(j kz/2E - zE) + e^{j kz z} erfc(j kz/2E + zE)]
  1D lattice (periodic x; L = period; rho = transverse distance; k_x = kx0 + 2 pi m / L): the 1D
           Fourier transform along x of the smooth complement G0 - f_E, written with the integral
           representation of G0 over s in [0, E] and expanded in powers of rho,
           (1/(4 pi L)) sum_m e^{-j k_x x} sum_q (-1)^q (rho E)^{2q} / q! E_{q+1}(-(k^2 - k_x^2)/4E^2)
           with E_p the generalized exponential integral, continued from losses (Im k < 0), i.e. its
           argument taken just above the negative real axis
  self     lim_{R->0} [f_E(R) - G0(R)] = jk erfc(jk/2E)/(4 pi) - E e^{k^2/4E^2}/(2 pi^{3/2})

As E -> infinity the 2D spectral part reduces term by term to Eq. pgf_2 and
the 3D one to the Fourier series of Eq. 2; the tests check independence of E
and agreement with brute-force image sums for a lossy wavenumber, and the 1D
lattice against Eq. pgf_1 (the Hankel-function series) for a real one.

For k = k0 = 0 on a 3D lattice the G = 0 term is dropped: this is the
"tin-foil" periodic Green's function, which solves -lap G = delta - 1/V with
zero cell mean.  Eq. lgf_3 solves the same equation, so the two differ by a
constant that cancels for neutral charges (Eq. neutral).
"""
import math

import numpy as np
from scipy import special

from .greens import csqrt_neg_imag

FOUR_PI = 4.0 * np.pi
SQRT_PI = np.sqrt(np.pi)


def exp_erfc(A, B):
    """exp(A) * erfc(B) for complex A, B without overflow of either factor."""
    A = np.asarray(A, np.complex128)
    B = np.asarray(B, np.complex128)
    out = np.empty(np.broadcast(A, B).shape, np.complex128)
    Ab, Bb = np.broadcast_arrays(A, B)
    pos = Bb.real > 0
    out[pos] = special.erfcx(Bb[pos]) * np.exp(Ab[pos] - Bb[pos] ** 2)
    out[~pos] = np.exp(Ab[~pos]) * special.erfc(Bb[~pos])
    return out


def spatial_kernel(R, k, E):
    """f_E(R) (see module docstring); R > 0."""
    R = np.asarray(R, np.float64)
    if k == 0:
        return special.erfc(R * E) / (FOUR_PI * R)
    a = 1j * k / (2.0 * E)
    return (exp_erfc(-1j * k * R, R * E - a) + exp_erfc(1j * k * R, R * E + a)) / (2.0 * FOUR_PI * R)


def self_term(k, E):
    """lim_{R->0} [f_E(R) - G0(R)]."""
    if k == 0:
        return -E / (2.0 * np.pi * SQRT_PI)
    return 1j * k * special.erfc(1j * k / (2.0 * E)) / FOUR_PI - E * np.exp(k * k / (4.0 * E * E)) / (2.0 * np.pi * SQRT_PI)


def spatial_part(points, q, m, L, pdims, k, k0, E, rcut):
    """The spatial half of Eq. 1 at point m: the sum over sources n and
    lattice images i of exp(-j k0.(i o L)) f_E(|r_m - r_n - i o L|) q_n over
    the pairs with |r_m - r_n - i o L| < rcut, the pair (n = m, i = 0)
    excluded, plus the self term q_m lim [f_E - G0].  Each source is first
    moved to its nearest image (i0 = round((r_m - r_n) / L) on the periodic
    axes); the images within rcut are then i = i0 + j with
    |j_d| <= ceil(rcut / L_d + 1/2).  pdims are the periodic axes (indices
    into points' columns)."""
    d0 = points[m] - points
    i0 = np.zeros_like(d0)
    for d in pdims:
        i0[:, d] = np.round(d0[:, d] / L[d])
    d0 = d0 - i0 * L
    ph0 = np.exp(-1j * ((i0 * L) @ k0))
    J = [int(np.ceil(rcut / L[d] + 0.5)) if d in pdims else 0 for d in range(3)]
    acc = 0.0 + 0.0j
    for jx in range(-J[0], J[0] + 1):
        for jy in range(-J[1], J[1] + 1):
            for jz in range(-J[2], J[2] + 1):
                sh = np.array([jx, jy, jz]) * L
                R = np.linalg.norm(d0 - sh, axis=1)
                sel = R < rcut
                if jx == 0 and jy == 0 and jz == 0:
                    sel[m] = False
                if not sel.any():
                    continue
                acc += np.exp(-1j * np.dot(k0, sh)) * np.sum(ph0[sel] * q[sel] * spatial_kernel(R[sel], k, E))
    return acc + q[m] * self_term(k, E)


def spectral_3d_setup(points, q, L, k, k0, E, Gc, chunk=2048):
    """The 3D lattice spectral half, the part shared by all targets: the
    wave vectors k_G = k0 + 2 pi (m_x / L_x, m_y / L_y, m_z / L_z) with
    |k_G| <= Gc and their weights W(k_G) = f(k_G) T(k_G) / V, f =
    exp((k^2 - |k_G|^2)/4E^2) / (|k_G|^2 - k^2), T(k_G) = sum_n q_n
    exp(+j k_G.r_n) the structure factor (G = 0 dropped for k = k0 = 0)."""
    V = np.prod(L)
    ms = [np.arange(-int(np.ceil(Gc * L[d] / (2 * np.pi))) - 1, int(np.ceil(Gc * L[d] / (2 * np.pi))) + 2)
          for d in range(3)]
    kx = k0[0] + 2 * np.pi * ms[0] / L[0]
    ky = k0[1] + 2 * np.pi * ms[1] / L[1]
    kz = k0[2] + 2 * np.pi * ms[2] / L[2]
    K2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.exp((k * k - K2) / (4 * E * E)) / (K2 - k * k)
    if k == 0 and not np.any(k0 != 0):
        f[np.abs(K2) == 0] = 0.0
    f[np.abs(K2) ** 0.5 > Gc + 2 * np.pi / L.min()] = 0.0
    # structure factor T(kG) = sum_n q_n exp(+j kG . r_n), separable in x, y, z
    T = np.zeros(K2.shape, np.complex128)
    for s0 in range(0, len(points), chunk):
        s1 = min(len(points), s0 + chunk)
        ex = np.exp(1j * np.outer(points[s0:s1, 0], kx))
        ey = np.exp(1j * np.outer(points[s0:s1, 1], ky))
        ez = np.exp(1j * np.outer(points[s0:s1, 2], kz))
        qa = q[s0:s1, None] * ex
        yz = (ey[:, :, None] * ez[:, None, :]).reshape(s1 - s0, -1)
        T += (qa.T @ yz).reshape(K2.shape)
    return kx, ky, kz, f * T / V


def spectral_3d_at(setup, r):
    """The 3D lattice spectral half at the point r: sum_G W(k_G) exp(-j k_G.r)."""
    kx, ky, kz, W = setup
    px = np.exp(-1j * kx * r[0])
    py = np.exp(-1j * ky * r[1])
    pz = np.exp(-1j * kz * r[2])
    return np.einsum("abc,a,b,c->", W, px, py, pz)


def splitting_cutoffs(k, E, tol=1e-15):
    """(X, rcut, Gc): erfc(X) ~ tol, the spatial cutoff X / E and the
    spectral one 2 E X + |k| + 1."""
    X = np.sqrt(-np.log(tol)) + 0.5
    return X, X / E, 2.0 * E * X + abs(k) + 1.0


def potential(points, q, tgt, L, pdims, k, k0, E, tol=1e-15, chunk=2048):
    """u at the points with indices tgt (Eq. 1, self term excluded), by Ewald
    splitting on a 3D or 2D lattice.  points (N,3), q (N,) complex.
    For the 2D lattice the periodic axes are relabelled to x, y."""
    points = np.asarray(points, np.float64)
    q = np.asarray(q, np.complex128)
    tgt = np.asarray(tgt, np.int64)
    L = np.asarray(L, np.float64)
    k0 = np.asarray(k0, np.complex128)
    pd = sorted(pdims)
    order = pd + [d for d in range(3) if d not in pd]
    points, L, k0 = points[:, order], L[order], k0[order]
    pdc = tuple(range(len(pd)))
    X, rcut, Gc = splitting_cutoffs(k, E, tol)
    u = np.zeros(len(tgt), np.complex128)
    # ---------------- spatial part -----------------------------------
    for t, m in enumerate(tgt):
        u[t] = spatial_part(points, q, m, L, pdc, k, k0, E, rcut)
    # ---------------- spectral part ----------------------------------
    if len(pd) == 3:
        V = np.prod(L)
        setup = spectral_3d_setup(points, q, L, k, k0, E, Gc, chunk)
        for t, m in enumerate(tgt):
            u[t] += spectral_3d_at(setup, points[m])
        if k == 0 and not np.any(k0 != 0):
            u += -np.sum(q) / (4 * E * E * V)
    elif len(pd) == 2:
        A = L[0] * L[1]
        Mx = int(np.ceil(Gc * L[0] / (2 * np.pi))) + 1
        My = int(np.ceil(Gc * L[1] / (2 * np.pi))) + 1
        kx = k0[0] + 2 * np.pi * np.arange(-Mx, Mx + 1) / L[0]
        ky = k0[1] + 2 * np.pi * np.arange(-My, My + 1) / L[1]
        KX, KY = np.meshgrid(kx, ky, indexing="ij")
        sel = np.hypot(np.abs(KX), np.abs(KY)) <= Gc + 2 * np.pi / min(L[0], L[1])
        KX, KY = KX[sel], KY[sel]
        kz = csqrt_neg_imag(k * k - KX ** 2 - KY ** 2)
        jkz = 1j * kz
        for t, m in enumerate(tgt):
            for s0 in range(0, len(points), chunk):
                d = points[m] - points[s0:s0 + chunk]
                z = d[:, 2][:, None]
                tph = np.exp(-1j * (np.outer(d[:, 0], KX) + np.outer(d[:, 1], KY)))
                br = exp_erfc(-1j * kz[None, :] * z, jkz[None, :] / (2 * E) - z * E) \
                    + exp_erfc(1j * kz[None, :] * z, jkz[None, :] / (2 * E) + z * E)
                u[t] += np.sum(q[s0:s0 + chunk, None] * tph * br / (4j * kz[None, :] * A))
    elif len(pd) == 1:
        Lx = L[0]
        Mx = int(np.ceil(Gc * Lx / (2 * np.pi))) + 1
        kx = k0[0] + 2 * np.pi * np.arange(-Mx, Mx + 1) / Lx
        # transverse extent fixes the number of powers of (rho E)^2 kept
        rho_max = np.hypot(np.ptp(points[:, 1]), np.ptp(points[:, 2]))
        Q = int(np.ceil(2.0 * (rho_max * E) ** 2 + 60))
        Etab = expint_table(Q, -(k * k - kx * kx) / (4 * E * E))          # (Q, modes)
        coef = np.array([(-1.0) ** qq / math.factorial(qq) for qq in range(Q)])
        for t, m in enumerate(tgt):
            for s0 in range(0, len(points), chunk):
                d = points[m] - points[s0:s0 + chunk]
                w = (d[:, 1] ** 2 + d[:, 2] ** 2) * E * E                 # (rho E)^2
                pw = w[:, None] ** np.arange(Q)[None, :] * coef[None, :]   # (n, Q)
                S = pw @ Etab                                             # (n, modes)
                ph = np.exp(-1j * np.outer(d[:, 0], kx))
                u[t] += np.sum(q[s0:s0 + chunk, None] * ph * S) / (FOUR_PI * Lx)
    else:
        raise ValueError("Ewald ground truth implemented for 1D, 2D and 3D lattices")
    return u


def expint_table(Q, z):
    """E_p(z) for p = 1..Q (rows) at the complex arguments z (columns), the
    argument moved just above the negative real axis (the outgoing branch).
    E_1 in arbitrary precision (mpmath), the higher orders by the recurrence
    E_{p+1}(z) = (e^{-z} - z E_p(z)) / p carried at 80 digits, which absorbs
    its growth of rounding errors (at most about e^{|z|}) for the |z| < 100
    of the modes kept."""
    import mpmath

    z = np.atleast_1d(np.asarray(z, np.complex128))
    out = np.empty((Q, len(z)), np.complex128)
    with mpmath.workdps(80):
        for j, zz in enumerate(z):
            zm = mpmath.mpc(zz.real, zz.imag if zz.imag != 0 else 1e-300)
            ez = mpmath.exp(-zm)
            e = mpmath.expint(1, zm)
            for p in range(1, Q + 1):
                out[p - 1, j] = complex(e)
                e = (ez - zm * e) / p
    return out


def greens_function(r, L, pdims, k, k0, E):
    """Single-source periodic Green's function G^p(r) by Ewald splitting
    (for r not on the lattice).  Implemented as the potential at r of a unit
    source at the origin."""
    r = np.atleast_2d(np.asarray(r, np.float64))
    out = np.empty(len(r), np.complex128)
    for i, rr in enumerate(r):
        pts = np.stack([rr, np.zeros(3)])
        qq = np.array([0.0, 1.0], np.complex128)
        out[i] = potential(pts, qq, [0], L, pdims, k, k0, E)[0]
    return out
