"""Periodic Green's functions, FP64.  TEST INFRASTRUCTURE ONLY.

Everything here follows Sec. 2 of arXiv 2312.02376 with the paper's
engineering convention (time factor e^{jwt}, j = sqrt(-1)):

  G0(r)  = exp(-j k |r|) / (4 pi |r|)                                (Eq. 2)
  G^p(r) = sum_i exp(-j k0.(i o L)) G0(r - i o L)                    (Eq. 2)
           i runs over the periodic axes only ("i o L" = componentwise).

Spectral (Floquet) forms, Eq. pgf:
  1D (periodic axis x, rho = sqrt(y^2+z^2)):
      sum_m  exp(-j kx_m x) H0^(2)(krho_m rho) / (4 j Lx)
  2D (periodic x, y; z free):
      sum_{m,n} exp(-j kx_m x - j ky_n y - j kz_mn |z|) / (2 j kz_mn Lx Ly)
  3D: the 2D series times the z-image geometric factor of Eq. pgf_3.
  kx_m = kx0 + 2 pi m/Lx, ky_n = ky0 + 2 pi n/Ly (the paper prints L_z in the
  ky_n definition; Ly is the only reading under which the 2D series is the
  Floquet expansion of Eq. 2), krho_m = (k^2 - kx_m^2)^(1/2),
  kz_mn = (k^2 - kx_m^2 - ky_n^2)^(1/2), square roots with Im <= 0 and, for a
  positive real radicand, the positive root (outgoing waves).

Neutral static ("NPSP", k = k0 = 0) forms, Eq. lgf_1 / lgf_2 / lgf_3.  They
are defined up to an additive constant, which cancels for neutral charges
(Eq. neutral).

The far-zone table of Sec. 3.2 is G_far = G^p - G_near where G_near keeps the
images |i_d| <= i_d of Eq. 2 (Eq. 4).

Axes: the paper writes 1D periodicity along x and 2D along x,y.  Another
choice of periodic axes is handled by relabelling the axes before evaluating
the series (the periodic axes first, in increasing order).
"""
import numpy as np
from scipy import special

FOUR_PI = 4.0 * np.pi


def G0(R, k):
    """Free-space Green's function exp(-jkR)/(4 pi R) (Eq. 2); R > 0."""
    R = np.asarray(R, dtype=np.float64)
    return np.exp(-1j * k * R) / (FOUR_PI * R)


def csqrt_neg_imag(z):
    """Square root with Im <= 0; for a positive real radicand the positive
    root (the branch of Sec. 2 after Eq. pgf)."""
    s = np.sqrt(np.asarray(z, dtype=np.complex128))
    # numpy's principal root has Re >= 0 and Im sign of z.imag; flip roots
    # with Im > 0 to the lower half plane.
    flip = s.imag > 0
    s = np.where(flip, -s, s)
    return s


def image_offsets(pdims, layers):
    """All integer image vectors i with i_d in [-layers, layers] on periodic
    axes and 0 elsewhere (the near-zone image set of Eq. 4)."""
    rng = [np.arange(-layers, layers + 1) if d in pdims else np.zeros(1, np.int64) for d in range(3)]
    I = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    return I.astype(np.int64)


def image_sum(r, L, pdims, k, k0, images):
    """Truncated Eq. 2: sum over the given image vectors of
    exp(-j k0.(i o L)) G0(r - i o L).  r: (..., 3)."""
    r = np.asarray(r, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    k0 = np.asarray(k0, dtype=np.complex128)
    out = np.zeros(r.shape[:-1], dtype=np.complex128)
    for i in images:
        shift = i * L
        R = np.linalg.norm(r - shift, axis=-1)
        out += np.exp(-1j * np.dot(k0, shift)) * np.exp(-1j * k * R) / (FOUR_PI * R)
    return out


# --------------------------------------------------------------------------
# axis relabelling
# --------------------------------------------------------------------------
def _canonical(r, L, k0, pdims):
    """Reorder axes so the periodic ones come first.  Returns r', L', k0'."""
    pd = sorted(pdims)
    order = pd + [d for d in range(3) if d not in pd]
    r = np.asarray(r, dtype=np.float64)[..., order]
    return r, np.asarray(L, dtype=np.float64)[order], np.asarray(k0, dtype=np.complex128)[order]


# --------------------------------------------------------------------------
# Eq. pgf (Floquet / spectral series)
# --------------------------------------------------------------------------
def _mode_range(kc, Lc, decay_len, k, extra=4):
    """Symmetric index window for Floquet modes k_m = kc + 2 pi m / Lc such
    that exp(-|k_m| * decay_len) is below ~1e-18 outside it."""
    kmax = 42.0 / max(decay_len, 1e-300) + abs(k) + abs(kc)
    M = int(np.ceil(kmax * Lc / (2.0 * np.pi))) + extra
    return np.arange(-M, M + 1)


def pgf1_canon(x, rho, Lx, k, kx0):
    """Eq. pgf_1 at arrays x, rho (periodic axis x).  Each point gets its own
    truncation (rho sets the decay rate)."""
    x = np.atleast_1d(np.asarray(x, np.float64))
    rho = np.atleast_1d(np.asarray(rho, np.float64))
    out = np.zeros(np.broadcast(x, rho).shape, np.complex128)
    xb, rb = np.broadcast_arrays(x, rho)
    for idx in np.ndindex(out.shape):
        m = _mode_range(kx0, Lx, rb[idx], k)
        kxm = kx0 + 2.0 * np.pi * m / Lx
        krho = csqrt_neg_imag(k * k - kxm * kxm)
        terms = np.exp(-1j * kxm * xb[idx]) * special.hankel2(0, krho * rb[idx]) / (4j * Lx)
        out[idx] = np.sum(terms[np.argsort(np.abs(terms))])
    return out


def _pgf2_modes(z_abs, Lx, Ly, k, kx0, ky0):
    m = _mode_range(kx0, Lx, z_abs, k)
    n = _mode_range(ky0, Ly, z_abs, k)
    kx = kx0 + 2.0 * np.pi * m / Lx
    ky = ky0 + 2.0 * np.pi * n / Ly
    kz = csqrt_neg_imag(k * k - kx[:, None] ** 2 - ky[None, :] ** 2)
    return kx, ky, kz


def pgf2_canon_grid(xs, ys, z, Lx, Ly, k, kx0, ky0):
    """Eq. pgf_2 on the tensor grid xs (x) ys at one height z != 0.
    The double sum over (m, n) is written as Ex @ F @ Ey^T with
    Ex[x, m] = exp(-j kx_m x), F[m, n] = exp(-j kz |z|)/(2 j kz Lx Ly),
    Ey[y, n] = exp(-j ky_n y): the same sum, grouped by a matrix product."""
    kx, ky, kz = _pgf2_modes(abs(z), Lx, Ly, k, kx0, ky0)
    F = np.exp(-1j * kz * abs(z)) / (2j * kz * Lx * Ly)
    Ex = np.exp(-1j * np.outer(np.asarray(xs, np.float64), kx))
    Ey = np.exp(-1j * np.outer(np.asarray(ys, np.float64), ky))
    return Ex @ F @ Ey.T


def pgf3_canon_grid(xs, ys, z, Lx, Ly, Lz, k, kx0, ky0, kz0):
    """Eq. pgf_3 on the tensor grid xs (x) ys at one height z, 0<|z|<Lz.
    Same grouping as pgf2_canon_grid; the z factor is the paper's bracket."""
    dlen = min(abs(z), Lz - abs(z))
    kx, ky, kz = _pgf2_modes(dlen, Lx, Ly, k, kx0, ky0)
    em = np.exp(-1j * (kz - kz0) * Lz)
    ep = np.exp(-1j * (kz + kz0) * Lz)
    # the bracket of Eq. pgf_3 with each numerator's exponentials combined,
    # e^{-j(kz-kz0)Lz} e^{-j kz z} = e^{-j kz (Lz+z)} e^{j kz0 Lz} and
    # e^{-j(kz+kz0)Lz} e^{+j kz z} = e^{-j kz (Lz-z)} e^{-j kz0 Lz},
    # so that no factor overflows for strongly evanescent modes
    zfac = (np.exp(-1j * kz * abs(z))
            + np.exp(-1j * kz * (Lz + z) + 1j * kz0 * Lz) / (1.0 - em)
            + np.exp(-1j * kz * (Lz - z) - 1j * kz0 * Lz) / (1.0 - ep))
    F = zfac / (2j * kz * Lx * Ly)
    Ex = np.exp(-1j * np.outer(np.asarray(xs, np.float64), kx))
    Ey = np.exp(-1j * np.outer(np.asarray(ys, np.float64), ky))
    return Ex @ F @ Ey.T


def pgf(r, L, pdims, k, k0):
    """Eq. pgf at points r (..., 3), evaluated point by point."""
    rc, Lc, kc = _canonical(r, L, k0, pdims)
    shape = rc.shape[:-1]
    rc = rc.reshape(-1, 3)
    out = np.zeros(rc.shape[0], np.complex128)
    P = len(pdims)
    for i, (x, y, z) in enumerate(rc):
        if P == 1:
            out[i] = pgf1_canon(x, np.hypot(y, z), Lc[0], k, kc[0])[0]
        elif P == 2:
            out[i] = pgf2_canon_grid([x], [y], z, Lc[0], Lc[1], k, kc[0], kc[1])[0, 0]
        elif P == 3:
            out[i] = pgf3_canon_grid([x], [y], z, Lc[0], Lc[1], Lc[2], k, kc[0], kc[1], kc[2])[0, 0]
        else:
            raise ValueError("pgf needs 1-3 periodic axes")
    return out.reshape(shape)


# --------------------------------------------------------------------------
# Eq. lgf (neutral static)
# --------------------------------------------------------------------------
def _k0_sum_x(x, Lx, rho_list):
    """(1/(pi Lx)) sum_{m>=1} K0(2 pi m rho / Lx) cos(2 pi m x / Lx), summed
    over every rho in rho_list (the inner lattice sums of Eq. lgf).
    x may be an array; the result has its shape."""
    x = np.asarray(x, np.float64)
    total = np.zeros(x.shape)
    for rho in rho_list:
        mmax = int(np.ceil(42.0 * Lx / (2.0 * np.pi * rho))) + 2
        m = np.arange(mmax, 0, -1)                       # small terms first
        kk = special.k0(2.0 * np.pi * m * rho / Lx)
        total = total + np.cos(2.0 * np.pi * np.multiply.outer(x, m) / Lx) @ kk
    return total / (np.pi * Lx)


def lgf1_canon(x, y, z, Lx):
    rho = np.hypot(y, z)
    return -np.log(rho) / (2.0 * np.pi * Lx) + _k0_sum_x(x, Lx, [rho])


def _lattice_rhos(y, z, Ly, Lz, Lx, with_k):
    """All sqrt((n Ly + y)^2 + (k Lz + z)^2) whose K0 terms can exceed 1e-18
    of the m = 1 scale (K0(2 pi rho/Lx) ~ exp(-2 pi rho / Lx))."""
    rmax = 42.0 * Lx / (2.0 * np.pi) + Ly + (Lz if with_k else 0.0)
    N = int(np.ceil(rmax / Ly)) + 1
    K = int(np.ceil(rmax / Lz)) + 1 if with_k else 0
    out = []
    for n in range(-N, N + 1):
        for kk in range(-K, K + 1):
            r = np.hypot(n * Ly + y, kk * Lz + z if with_k else z)
            if r <= rmax:
                out.append(r)
    out.sort(reverse=True)
    return out


def _log_line_array(y, zz, Ly, Lx):
    """-(1/(4 pi Lx)) ln(1 - 2 exp(-2 pi|z|/Ly) cos(2 pi y/Ly) + exp(-4 pi|z|/Ly))."""
    a = np.exp(-2.0 * np.pi * abs(zz) / Ly)
    return -np.log1p(-2.0 * a * np.cos(2.0 * np.pi * y / Ly) + a * a) / (4.0 * np.pi * Lx)


def lgf2_canon(x, y, z, Lx, Ly):
    val = -abs(z) / (2.0 * Lx * Ly) + _log_line_array(y, z, Ly, Lx)
    return val + _k0_sum_x(x, Lx, _lattice_rhos(y, z, Ly, 1.0, Lx, False))


def lgf3_canon(x, y, z, Lx, Ly, Lz):
    val = (z * z - abs(z) * Lz) / (2.0 * Lx * Ly * Lz)
    K = int(np.ceil(42.0 * Ly / (2.0 * np.pi * Lz))) + 2
    logs = [_log_line_array(y, kk * Lz + z, Ly, Lx) for kk in range(-K, K + 1)]
    logs.sort(key=abs)
    val += np.sum(logs)
    return val + _k0_sum_x(x, Lx, _lattice_rhos(y, z, Ly, Lz, Lx, True))


def lgf(r, L, pdims):
    """Eq. lgf at points r (..., 3), evaluated point by point."""
    rc, Lc, _ = _canonical(r, L, np.zeros(3), pdims)
    shape = rc.shape[:-1]
    rc = rc.reshape(-1, 3)
    out = np.zeros(rc.shape[0], np.float64)
    P = len(pdims)
    for i, (x, y, z) in enumerate(rc):
        if P == 1:
            out[i] = lgf1_canon(x, y, z, Lc[0])
        elif P == 2:
            out[i] = lgf2_canon(x, y, z, Lc[0], Lc[1])
        elif P == 3:
            out[i] = lgf3_canon(x, y, z, Lc[0], Lc[1], Lc[2])
        else:
            raise ValueError("lgf needs 1-3 periodic axes")
    return out.reshape(shape)


def is_npsp(k, k0):
    """No-phase static periodic case of Sec. 2: k = k0 = 0."""
    return k == 0 and not np.any(np.asarray(k0) != 0)


def periodic_gf(r, L, pdims, k, k0):
    """G^p by the rapidly converging series: Eq. lgf for NPSP, Eq. pgf else."""
    if is_npsp(k, k0):
        return lgf(r, L, pdims).astype(np.complex128)
    return pgf(r, L, pdims, k, k0)
