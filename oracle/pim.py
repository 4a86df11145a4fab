"""The FFT-PIM operator (arXiv 2312.02376, Sec. 3) in FP64 with a DIRECT
grid convolution.  TEST INFRASTRUCTURE ONLY.

u = u_near + u_far (Eq. 5) at N points that are both sources and observers.

Readings of the paper taken here (where it is silent or ambiguous):
  * self term: Eq. 5's "n != m" drops only the singular (n = m, image 0) term;
    self-images are kept (the only choice under which the neutral static
    result does not depend on the PGF's additive constant, Sec. 2).
  * near grid: Eq. grid with Delta removed from both Eq. grida and Eq. gridb
    (Sec. 3.3): n nodes l*h, l = 0..n-1, h = D/(n-1) per axis, spanning the
    closed cell [0, D]; a period L = D is n-1 grid steps.  Boxes are the
    n-1 grid cells per axis.
  * interpolation: p = polynomial degree, p+1 nodes per axis (Sec. 3.2); the
    stencil rule is in oracle.lagrange.
  * padding: G_near has no periodicity, so every axis is treated as aperiodic
    (Sec. 3.3 step 2); here the convolution is summed directly.
  * grid kernel at zero offset: g(0) = 0 (the paper does not define it).
  * boxes (Sec. 3.3 step 4: "boxes defined by Delta"): boxes of one grid
    step, placed so that all points of a box share one interpolation stencil
    (node-centred for even p, the grid cells for odd p), as in the
    box-adaptive integral method the near zone is built on.
  * correction region: for every near image i the pair (m, n) is corrected
    for that image only when the boxes B(m) and B(n) + i o (n-1) are at most
    b grid steps apart (minimum distance between the boxes, i.e. |r - r_m|
    <= D^ER with D^ER = b steps; Sec. 3.3 step 4 with the single-extra-image
    rule).  The grid part of the correction uses the image-i component of the
    tabulated kernel; the weights are those of steps 1 and 3.
  * far grids: source nodes l*Delta, observer nodes l*Delta + Delta/2,
    Delta = D/N_f (Eq. grid); Lagrange order p_f, same stencil rule.
  * neutral static case (k = k0 = 0): q must satisfy Eq. neutral to a
    relative tolerance tau; the residual mean is removed in FP64 before the
    apply.  The adjoint removes the mean of its result (the projector is
    self-adjoint).
Axes with a periodic lattice have L_d = D_d (rectangular lattice, Sec. 2).
"""
from dataclasses import dataclass, field

import numpy as np

from . import greens, lagrange


@dataclass
class Params:
    D: tuple                     # cell extents (D_x, D_y, D_z); L_d = D_d on periodic axes
    pdims: tuple                 # periodic axes, subset of (0, 1, 2)
    k: complex                   # wavenumber (Eq. 2 uses k_0)
    k0: tuple                    # phase-shift vector (k_x0, k_y0, k_z0), 0 on free axes
    n: tuple                     # near grid nodes per axis
    p: int = 4                   # near Lagrange degree
    layers: int = 1              # i_d, near-zone image layers (Eq. 4)
    b: int = 2                   # correction radius in boxes
    nf: tuple = (10, 10, 10)     # far grid nodes per axis
    pf: int = 4                  # far Lagrange degree
    neutral_tol: float = 1e-6
    region: str = "ball"         # "ball": box min-distance <= b steps; "cube": Chebyshev <= b

    def __post_init__(self):
        self.D = np.asarray(self.D, np.float64)
        self.n = np.asarray(self.n, np.int64)
        self.nf = np.asarray(self.nf, np.int64)
        self.k0 = np.asarray(self.k0, np.complex128)
        self.pdims = tuple(sorted(self.pdims))
        for d in range(3):
            if d not in self.pdims and self.k0[d] != 0:
                raise ValueError("phase shift on a non-periodic axis")

    @property
    def h(self):
        return self.D / (self.n - 1)

    @property
    def nL(self):
        """Grid steps per period (L = D = (n-1) h)."""
        return self.n - 1

    @property
    def delta_f(self):
        return self.D / self.nf

    @property
    def npsp(self):
        return len(self.pdims) > 0 and greens.is_npsp(self.k, self.k0)

    def images(self):
        return greens.image_offsets(self.pdims, self.layers)


# --------------------------------------------------------------------------
# stencils
# --------------------------------------------------------------------------
def near_stencils(P, pts, frozen=None):
    """Near stencil starts s (N,3), weights w (N,3,p+1), their x-derivatives
    dw (N,3,p+1) and boxes B (N,3).  frozen = (s, B) keeps the stencil
    starts and boxes of another position set (frozen topology)."""
    s = np.empty((len(pts), 3), np.int64)
    w = np.empty((len(pts), 3, P.p + 1))
    dw = np.empty((len(pts), 3, P.p + 1))
    B = np.empty((len(pts), 3), np.int64)
    for d in range(3):
        s[:, d], t = lagrange.stencil_start(pts[:, d], P.h[d], P.n[d], P.p)
        B[:, d] = lagrange.stencil_box(pts[:, d], P.h[d], P.n[d], P.p)
        if frozen is not None:
            s[:, d], B[:, d] = frozen[0][:, d], frozen[1][:, d]
            t = pts[:, d] / P.h[d] - s[:, d]
        w[:, d, :] = lagrange.weights(t, P.p)
        dw[:, d, :] = lagrange.dweights(t, P.p) / P.h[d]
    return s, w, B, dw


def far_stencils(P, pts, observer, frozen=None):
    """Far stencils on the source grid (observer=False) or on the observer
    grid shifted by Delta/2 (observer=True), Eq. grid: starts, weights and
    x-derivatives of the weights.  frozen = fixed stencil starts."""
    s = np.empty((len(pts), 3), np.int64)
    w = np.empty((len(pts), 3, P.pf + 1))
    dw = np.empty((len(pts), 3, P.pf + 1))
    for d in range(3):
        shift = 0.5 * P.delta_f[d] if observer else 0.0
        s[:, d], t = lagrange.stencil_start(pts[:, d], P.delta_f[d], P.nf[d], P.pf, shift)
        if frozen is not None:
            s[:, d] = frozen[:, d]
            t = (pts[:, d] - shift) / P.delta_f[d] - s[:, d]
        w[:, d, :] = lagrange.weights(t, P.pf)
        dw[:, d, :] = lagrange.dweights(t, P.pf) / P.delta_f[d]
    return s, w, dw


def _stencil_nodes(s, w, p):
    """Flattened 3D stencil: node indices (N,(p+1)^3,3) and weights (N,(p+1)^3),
    weight = w_x[jx] w_y[jy] w_z[jz] (tensor-product Lagrange, Sec. 3.2)."""
    j = np.arange(p + 1)
    J = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1).reshape(-1, 3)
    idx = s[:, None, :] + J[None, :, :]
    wt = w[:, 0, J[:, 0]] * w[:, 1, J[:, 1]] * w[:, 2, J[:, 2]]
    return idx, wt


def _stencil_grad_nodes(s, w, dw, p, d):
    """Node indices and the x_d-derivative of the tensor-product weights."""
    j = np.arange(p + 1)
    J = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1).reshape(-1, 3)
    idx = s[:, None, :] + J[None, :, :]
    f = [dw if k == d else w for k in range(3)]
    wt = f[0][:, 0, J[:, 0]] * f[1][:, 1, J[:, 1]] * f[2][:, 2, J[:, 2]]
    return idx, wt


def gather_grad(U, s, w, dw, p):
    """(N, 3): sum_a grad_x omega_m(a) U(a)."""
    out = np.zeros((len(s), 3), np.complex128)
    for d in range(3):
        idx, wt = _stencil_grad_nodes(s, w, dw, p, d)
        out[:, d] = np.sum(wt * U[idx[..., 0], idx[..., 1], idx[..., 2]], axis=1)
    return out


def spread(shape, s, w, p, q):
    """Q(a) = sum_n omega_n(a) q_n (step 1 of Sec. 3.2 / 3.3)."""
    idx, wt = _stencil_nodes(s, w, p)
    flat = np.ravel_multi_index((idx[..., 0], idx[..., 1], idx[..., 2]), shape).ravel()
    vals = (wt * q[:, None]).ravel()
    size = int(np.prod(shape))
    Q = np.bincount(flat, weights=vals.real, minlength=size) + 1j * np.bincount(flat, weights=vals.imag, minlength=size)
    return Q.reshape(shape)


def gather(U, s, w, p):
    """u_m = sum_a omega_m(a) U(a) (step 3 of Sec. 3.2 / 3.3)."""
    idx, wt = _stencil_nodes(s, w, p)
    return np.sum(wt * U[idx[..., 0], idx[..., 1], idx[..., 2]], axis=1)


# --------------------------------------------------------------------------
# near zone
# --------------------------------------------------------------------------
def grid_kernel(P, delta):
    """g(delta) = G0(delta o h) with g(0) = 0.  delta: (..., 3) integers."""
    r = np.asarray(delta, np.float64) * P.h
    R = np.linalg.norm(r, axis=-1)
    out = np.zeros(R.shape, np.complex128)
    nz = R > 0
    out[nz] = greens.G0(R[nz], P.k)
    return out


def near_table(P):
    """K(delta) = sum_{i in near images} exp(-j k0.(i o L)) g(delta - i o (n-1))
    for delta in [-(n-1), n-1]^3, stored at index delta + (n-1)  (G_near of
    Eq. 4 on the grid, Sec. 3.3 step 2)."""
    ax = [np.arange(-(P.n[d] - 1), P.n[d]) for d in range(3)]
    dl = np.stack(np.meshgrid(*ax, indexing="ij"), -1)
    K = np.zeros(dl.shape[:-1], np.complex128)
    for i in P.images():
        ph = np.exp(-1j * np.dot(P.k0, i * P.D))
        K += ph * grid_kernel(P, dl - i * P.nL)
    return K


def conv_direct_full(P, K, Q):
    """U(a) = sum_c K(a - c) Q(c) for every node a, summed directly: for each
    shift (dz, dy) the x-sum is a Toeplitz matrix product."""
    n = P.n
    U = np.zeros(tuple(n), np.complex128)
    ix = np.arange(n[0])
    for dy in range(-(n[1] - 1), n[1]):
        for dz in range(-(n[2] - 1), n[2]):
            # a_y = c_y + dy, a_z = c_z + dz
            ay0, ay1 = max(0, dy), min(n[1], n[1] + dy)
            az0, az1 = max(0, dz), min(n[2], n[2] + dz)
            if ay0 >= ay1 or az0 >= az1:
                continue
            # T[ax, cx] = K(ax - cx, dy, dz)
            T = K[(ix[:, None] - ix[None, :]) + n[0] - 1, dy + n[1] - 1, dz + n[2] - 1]
            Qs = Q[:, ay0 - dy:ay1 - dy, az0 - dz:az1 - dz]
            U[:, ay0:ay1, az0:az1] += np.einsum("ac,cyz->ayz", T, Qs)
    return U


def conv_direct_at(P, K, Q, nodes):
    """U(a) = sum_c K(a - c) Q(c) at the listed nodes only (row sampling)."""
    n = P.n
    out = np.empty(len(nodes), np.complex128)
    for t, (ax, ay, az) in enumerate(nodes):
        # K index for c: a - c + n - 1, c = 0..n-1 -> the block [a, a+n-1] reversed
        blk = K[ax:ax + n[0], ay:ay + n[1], az:az + n[2]][::-1, ::-1, ::-1]
        out[t] = np.sum(blk * Q)
    return out


def in_region(P, dB):
    """Error-correction region of Sec. 3.3 step 4 for box offsets dB (..., 3).
    "ball": the two boxes are at most b grid steps apart (minimum distance
    between the boxes, |r - r_m| <= D^ER with D^ER = b steps);
    "cube": Chebyshev box distance at most b."""
    dB = np.abs(dB)
    if P.region == "cube":
        return np.max(dB, axis=-1) <= P.b
    gap = np.maximum(dB - 1, 0)
    return np.sum(gap * gap, axis=-1) <= P.b * P.b


def correction_pairs(P, B, rows=None):
    """All (m, n, image) whose boxes B(m) and B(n) + i o (n-1) lie in each
    other's error-correction region (in_region: minimum box distance at most
    b steps, or Chebyshev distance for region "cube"; Sec. 3.3 step 4 with the
    single-extra-image rule).  Returns arrays m, n, image index."""
    rows = np.arange(len(B)) if rows is None else np.asarray(rows)
    I = P.images()
    M, Nn, Ii = [], [], []
    for m in rows:
        for ii, i in enumerate(I):
            nn = np.nonzero(in_region(P, B[m][None, :] - B - i * P.nL))[0]
            M.append(np.full(len(nn), m))
            Nn.append(nn)
            Ii.append(np.full(len(nn), ii))
    cat = lambda a: np.concatenate(a).astype(np.int64) if a else np.zeros(0, np.int64)
    return cat(M), cat(Nn), cat(Ii)


def correction_values_explicit(P, pts, s, w, m, n, ii, batch=256):
    """c = exp(-j k0.(i o L)) [G0(r_m - r_n - i o L) - G_grid,i(m, n)] with
    G_grid,i(m,n) = sum_a sum_c omega_m(a) omega_n(c) g(a - c - i o (n-1))
    (Eq. er; exact part omitted for m = n, i = 0).  The values of g at the
    integer offsets that occur are looked up in a table of g."""
    I = P.images()
    out = np.empty(len(m), np.complex128)
    if len(m) == 0:
        return out
    base = s[m] - s[n] - I[ii] * P.nL
    R = int(np.max(np.abs(base))) + P.p
    ax = np.arange(-R, R + 1)
    gt = grid_kernel(P, np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1))
    for b0 in range(0, len(m), batch):
        sl = slice(b0, b0 + batch)
        mm, nn, iv = m[sl], n[sl], I[ii[sl]]
        ia, wa = _stencil_nodes(s[mm], w[mm], P.p)
        ic, wc = _stencil_nodes(s[nn], w[nn], P.p)
        dl = ia[:, :, None, :] - ic[:, None, :, :] - (iv * P.nL)[:, None, None, :] + R
        g = gt[dl[..., 0], dl[..., 1], dl[..., 2]]
        grid = np.einsum("ta,tc,tac->t", wa, wc, g)
        r = pts[mm] - pts[nn] - iv * P.D
        R2 = np.linalg.norm(r, axis=1)
        exact = np.zeros(len(mm), np.complex128)
        selfpair = (mm == nn) & ~np.any(iv != 0, axis=1)
        ok = ~selfpair
        exact[ok] = greens.G0(R2[ok], P.k)
        ph = np.exp(-1j * (iv * P.D) @ P.k0)
        out[sl] = ph * (exact - grid)
    return out


def correction_values(P, pts, s, w, m, n, ii, batch=8192):
    """Same values as correction_values_explicit, with the grid part summed
    through the tensor-product identity of the weights:

      sum_a sum_c omega_m(a) omega_n(c) g(a - c - i o (n-1))
        = sum_{e in [-p,p]^3} g(s_m - s_n - i o (n-1) + e) Cx(e_x) Cy(e_y) Cz(e_z),
      Cd(e) = sum_{j - l = e} w_{m,d}[j] w_{n,d}[l]   (1D weight correlation),

    which is the explicit double sum with a = s_m + j, c = s_n + l grouped by
    e = j - l (the tests check the two agree)."""
    I = P.images()
    out = np.empty(len(m), np.complex128)
    if len(m) == 0:
        return out
    p = P.p
    base_all = s[m] - s[n] - I[ii] * P.nL
    R = int(np.max(np.abs(base_all))) + p
    ax = np.arange(-R, R + 1)
    gt = grid_kernel(P, np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1))
    e = np.arange(-p, p + 1)
    E = np.stack(np.meshgrid(e, e, e, indexing="ij"), -1).reshape(-1, 3)
    for b0 in range(0, len(m), batch):
        sl = slice(b0, b0 + batch)
        mm, nn, iv = m[sl], n[sl], I[ii[sl]]
        base = base_all[sl]
        C = np.zeros((len(mm), 3, 2 * p + 1))
        for d in range(3):
            for j in range(p + 1):
                for l in range(p + 1):
                    C[:, d, j - l + p] += w[mm, d, j] * w[nn, d, l]
        idx = base[:, None, :] + E[None, :, :] + R
        g = gt[idx[..., 0], idx[..., 1], idx[..., 2]]
        wgt = C[:, 0, E[:, 0] + p] * C[:, 1, E[:, 1] + p] * C[:, 2, E[:, 2] + p]
        grid = np.sum(wgt * g, axis=1)
        r = pts[mm] - pts[nn] - iv * P.D
        R2 = np.linalg.norm(r, axis=1)
        exact = np.zeros(len(mm), np.complex128)
        selfpair = (mm == nn) & ~np.any(iv != 0, axis=1)
        ok = ~selfpair
        exact[ok] = greens.G0(R2[ok], P.k)
        ph = np.exp(-1j * (iv * P.D) @ P.k0)
        out[sl] = ph * (exact - grid)
    return out


def correction_grads(P, pts, s, w, dw, m, n, ii, batch=8192):
    """D = d/dr_m of exp(-j k0.(i o L)) [G0(r_m - r_n - i o L) - G_grid,i(m, n)]
    for each listed pair, (len, 3) complex: the gradient of the exact term
    and of the grid term, whose x_d derivative replaces w_m,d by its
    derivative in the tensor-product identity of correction_values."""
    I = P.images()
    out = np.zeros((len(m), 3), np.complex128)
    if len(m) == 0:
        return out
    p = P.p
    base_all = s[m] - s[n] - I[ii] * P.nL
    R = int(np.max(np.abs(base_all))) + p
    ax = np.arange(-R, R + 1)
    gt = grid_kernel(P, np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1))
    e = np.arange(-p, p + 1)
    E = np.stack(np.meshgrid(e, e, e, indexing="ij"), -1).reshape(-1, 3)
    for b0 in range(0, len(m), batch):
        sl = slice(b0, b0 + batch)
        mm, nn, iv = m[sl], n[sl], I[ii[sl]]
        base = base_all[sl]
        C = np.zeros((len(mm), 3, 2 * p + 1))
        dC = np.zeros((len(mm), 3, 2 * p + 1))
        for d in range(3):
            for j in range(p + 1):
                for l in range(p + 1):
                    C[:, d, j - l + p] += w[mm, d, j] * w[nn, d, l]
                    dC[:, d, j - l + p] += dw[mm, d, j] * w[nn, d, l]
        idx = base[:, None, :] + E[None, :, :] + R
        g = gt[idx[..., 0], idx[..., 1], idx[..., 2]]
        r = pts[mm] - pts[nn] - iv * P.D
        Rr = np.linalg.norm(r, axis=1)
        selfpair = (mm == nn) & ~np.any(iv != 0, axis=1)
        ph = np.exp(-1j * (iv * P.D) @ P.k0)
        for d in range(3):
            fac = [dC[:, 0] if d == 0 else C[:, 0], dC[:, 1] if d == 1 else C[:, 1], dC[:, 2] if d == 2 else C[:, 2]]
            wgt = fac[0][:, E[:, 0] + p] * fac[1][:, E[:, 1] + p] * fac[2][:, E[:, 2] + p]
            grid = np.sum(wgt * g, axis=1)
            ex = np.zeros(len(mm), np.complex128)
            ok = ~selfpair
            # d/dx G0(R) = G0(R) (-jk - 1/R) x/R
            G = greens.G0(Rr[ok], P.k)
            ex[ok] = G * (-1j * P.k - 1.0 / Rr[ok]) * r[ok, d] / Rr[ok]
            out[sl, d] = ph * (ex - grid)
    return out


# --------------------------------------------------------------------------
# far zone
# --------------------------------------------------------------------------
def far_table(P):
    """F(delta) = G_far(delta o Delta + Delta/2), delta in [-(N_f-1), N_f-1]^3,
    stored at index delta + N_f - 1 (Sec. 3.2: G_far = G^p - G_near, G^p by
    the series of Eq. pgf, or Eq. lgf in the neutral static case)."""
    if len(P.pdims) == 0:
        return None
    dF = P.delta_f
    ax = [np.arange(-(P.nf[d] - 1), P.nf[d]) * dF[d] + 0.5 * dF[d] for d in range(3)]
    T = series_on_grid(P, ax)
    # subtract the near images (Eq. 4)
    r = np.stack(np.meshgrid(*ax, indexing="ij"), -1)
    T = T - greens.image_sum(r, P.D, P.pdims, P.k, P.k0, P.images())
    return T


def series_on_grid(P, ax):
    """G^p on the tensor grid ax[0] x ax[1] x ax[2] by Eq. pgf / Eq. lgf."""
    pd = list(P.pdims)
    order = pd + [d for d in range(3) if d not in pd]
    cax = [ax[d] for d in order]
    L = P.D[order]
    kc = P.k0[order]
    shape = tuple(len(a) for a in cax)
    out = np.zeros(shape, np.complex128)
    X = np.asarray(cax[0])
    if P.npsp:
        for iy, y in enumerate(cax[1]):
            for iz, z in enumerate(cax[2]):
                if len(pd) == 1:
                    v = _lgf1_x(X, y, z, L[0])
                elif len(pd) == 2:
                    v = _lgf2_x(X, y, z, L[0], L[1])
                else:
                    v = _lgf3_x(X, y, z, L[0], L[1], L[2])
                out[:, iy, iz] = v
    elif len(pd) == 1:
        for iy, y in enumerate(cax[1]):
            for iz, z in enumerate(cax[2]):
                for ix, x in enumerate(X):
                    out[ix, iy, iz] = greens.pgf1_canon(x, np.hypot(y, z), L[0], P.k, kc[0])[0]
    elif len(pd) == 2:
        for iz, z in enumerate(cax[2]):
            out[:, :, iz] = greens.pgf2_canon_grid(X, cax[1], z, L[0], L[1], P.k, kc[0], kc[1])
    else:
        for iz, z in enumerate(cax[2]):
            out[:, :, iz] = greens.pgf3_canon_grid(X, cax[1], z, L[0], L[1], L[2], P.k, kc[0], kc[1], kc[2])
    inv = np.argsort(order)
    return np.transpose(out, inv)


def _lgf1_x(X, y, z, Lx):
    return greens.lgf1_canon(np.asarray(X), y, z, Lx)


def _lgf2_x(X, y, z, Lx, Ly):
    return greens.lgf2_canon(np.asarray(X), y, z, Lx, Ly)


def _lgf3_x(X, y, z, Lx, Ly, Lz):
    return greens.lgf3_canon(np.asarray(X), y, z, Lx, Ly, Lz)


def far_sum(P, F, qg, adjoint=False, direct=None):
    """Eq. 8: u(a) = sum_b F(a - b) q(b) over the far grid (observer nodes a,
    source nodes b); adjoint: u(b) = sum_a conj(F(a - b)) q(a).  Summed
    directly, one source node at a time (the shifted slice of the table F
    over all a), for far grids up to 30000 nodes (direct = None) or when
    direct is True; else as the linear convolution of F with q by a library
    FFT convolution (scipy.signal.fftconvolve), sliced to the observer nodes."""
    nf = tuple(int(v) for v in P.nf)
    if direct is False or (direct is None and qg.size > 30000):
        from scipy.signal import fftconvolve
        Fk = np.conj(F[::-1, ::-1, ::-1]) if adjoint else F
        full = fftconvolve(Fk, qg, mode="full")
        return full[nf[0] - 1:2 * nf[0] - 1, nf[1] - 1:2 * nf[1] - 1, nf[2] - 1:2 * nf[2] - 1]
    u = np.zeros(nf, np.complex128)
    for b in zip(*np.nonzero(qg)):
        sl = tuple(slice(nf[d] - 1 - b[d], 2 * nf[d] - 1 - b[d]) for d in range(3))
        if adjoint:
            # u(c) += conj(F(b - c)) q(b): the table reversed about b
            rs = tuple(slice(nf[d] - 1 + b[d], b[d] - 1 if b[d] > 0 else None, -1) for d in range(3))
            u += np.conj(F[rs]) * qg[b]
        else:
            u += F[sl] * qg[b]
    return u


def far_apply(P, F, ss, ws, so, wo, q):
    """Steps 1-3 of Sec. 3.2: project (Eq. projection), direct grid sum
    (Eq. 8), interpolate (Eq. interpolation)."""
    nf = tuple(P.nf)
    qg = spread(nf, ss, ws, P.pf, q)
    return gather(far_sum(P, F, qg), so, wo, P.pf)


def far_apply_adjoint(P, F, ss, ws, so, wo, v):
    nf = tuple(P.nf)
    vg = spread(nf, so, wo, P.pf, v)
    return gather(far_sum(P, F, vg, adjoint=True), ss, ws, P.pf)


def far_matrix(P, F):
    """Dense A[a, b] = F(a - b) over the far grid (observer a, source b)."""
    nf = P.nf
    J = np.stack(np.meshgrid(*[np.arange(v) for v in nf], indexing="ij"), -1).reshape(-1, 3)
    d = J[:, None, :] - J[None, :, :] + (nf - 1)
    return F[d[..., 0], d[..., 1], d[..., 2]]


# --------------------------------------------------------------------------
# the operator
# --------------------------------------------------------------------------
@dataclass
class Plan:
    P: Params
    pts: np.ndarray
    K: np.ndarray = field(default=None, repr=False)
    F: np.ndarray = field(default=None, repr=False)
    frozen: object = field(default=None, repr=False)   # a Plan whose stencils, boxes and pairs are kept

    def __post_init__(self):
        P = self.P
        self.pts = np.asarray(self.pts, np.float64)
        if np.any(self.pts < 0) or np.any(self.pts > P.D[None, :]):
            raise ValueError("points outside the closed cell [0, D]")
        if np.any(P.n < P.p + 1) or (len(P.pdims) and np.any(P.nf < P.pf + 1)):
            raise ValueError("grid smaller than the stencil")
        if self.K is None:
            self.K = near_table(P)
        if self.F is None:
            self.F = far_table(P)
        fz = self.frozen
        self.s, self.w, self.B, self.dw = near_stencils(P, self.pts, None if fz is None else (fz.s, fz.B))
        if len(P.pdims):
            self.ss, self.ws, self.dws = far_stencils(P, self.pts, False, None if fz is None else fz.ss)
            self.so, self.wo, self.dwo = far_stencils(P, self.pts, True, None if fz is None else fz.so)
        self._corr = None

    # --- neutrality (Eq. neutral) ----------------------------------------
    def regularise(self, q):
        q = np.asarray(q, np.complex128)
        if not self.P.npsp:
            return q
        tot = np.sum(q)
        if abs(tot) > self.P.neutral_tol * np.sum(np.abs(q)):
            raise ValueError("charges are not neutral (Eq. neutral)")
        return q - tot / len(q)

    def corrections(self):
        if self._corr is None:
            if self.frozen is not None:
                m, n, ii = self.frozen.corrections()[:3]
            else:
                m, n, ii = correction_pairs(self.P, self.B)
            c = correction_values(self.P, self.pts, self.s, self.w, m, n, ii)
            self._corr = (m, n, ii, c)
        return self._corr

    def apply(self, q, full_conv=True):
        """u = A q at every point."""
        P = self.P
        q = self.regularise(q)
        Q = spread(tuple(P.n), self.s, self.w, P.p, q)
        U = conv_direct_full(P, self.K, Q) if full_conv else None
        u = gather(U, self.s, self.w, P.p)
        m, n, ii, c = self.corrections()
        u += np.bincount(m, weights=(c * q[n]).real, minlength=len(q)) \
            + 1j * np.bincount(m, weights=(c * q[n]).imag, minlength=len(q))
        if len(P.pdims):
            u += far_apply(P, self.F, self.ss, self.ws, self.so, self.wo, q)
        return u

    def apply_rows(self, q, rows):
        """u_m for m in rows only; the grid potential is summed only at the
        stencil nodes of those rows (for large inputs)."""
        return self.rows_from(self.rows_prepare(q), rows)

    def rows_prepare(self, q):
        """The part of apply_rows shared by all rows: the regularised sources,
        the near grid charges (step 1) and the far grid potentials (Eq. 8)."""
        P = self.P
        q = self.regularise(q)
        Q = spread(tuple(P.n), self.s, self.w, P.p, q)
        ug = None
        if len(P.pdims):
            nf = tuple(P.nf)
            qg = spread(nf, self.ss, self.ws, P.pf, q)
            ug = far_sum(P, self.F, qg)
        return q, Q, ug

    def rows_from(self, state, rows):
        """The per-row part of apply_rows: the grid potential at the rows'
        stencil nodes (step 2), the gather (step 3), the correction (step 4)
        and the far gather."""
        P = self.P
        q, Q, ug = state
        rows = np.asarray(rows, np.int64)
        idx, wt = _stencil_nodes(self.s[rows], self.w[rows], P.p)
        flat = idx.reshape(-1, 3)
        uniq, inv = np.unique(flat, axis=0, return_inverse=True)
        Uv = conv_direct_at(P, self.K, Q, uniq)
        u = np.sum(wt * Uv[inv.reshape(wt.shape)], axis=1)
        m, n, ii = correction_pairs(P, self.B, rows)
        c = correction_values(P, self.pts, self.s, self.w, m, n, ii)
        pos = {int(r): t for t, r in enumerate(rows)}
        for mm, v in zip(m, c * q[n]):
            u[pos[int(mm)]] += v
        if ug is not None:
            u += gather(ug, self.so[rows], self.wo[rows], P.pf)
        return u

    def apply_adjoint(self, v):
        """w = A^H v, the conjugate transpose of every step of apply()."""
        P = self.P
        v = np.asarray(v, np.complex128)
        V = spread(tuple(P.n), self.s, self.w, P.p, v)
        # (C_K)^H: U'(c) = sum_a conj(K(a - c)) V(a) = conv with K'(d) = conj(K(-d))
        Kh = np.conj(self.K[::-1, ::-1, ::-1])
        U = conv_direct_full(P, Kh, V)
        w = gather(U, self.s, self.w, P.p)
        m, n, ii, c = self.corrections()
        t = np.conj(c) * v[m]
        w += np.bincount(n, weights=t.real, minlength=len(v)) + 1j * np.bincount(n, weights=t.imag, minlength=len(v))
        if len(P.pdims):
            w += far_apply_adjoint(P, self.F, self.ss, self.ws, self.so, self.wo, v)
        if P.npsp:
            w = w - np.mean(w)
        return w

    def position_grad(self, q, g):
        """(N, 3) real: d/dr_k Re sum_m conj(g_m) u_m with u = A(r) q, the
        stencil starts, boxes and pair list held fixed (frozen topology).
        Terms: observer side conj(g_k) grad_omega_k . U and source side
        q_k conj(grad_omega_k . V) with V the adjoint grid potential of g,
        for the near grid and the far grids, and for every pair of row k of
        the correction list with D = d d_i(k, n)/d r_k:
        conj(g_k) phase_i D q_n + q_k conj(g_n) phase_{-i} D
        (the source-side term uses d_i(m, k) = d_{-i}(k, m))."""
        P = self.P
        q = self.regularise(q)
        g = np.asarray(g, np.complex128)
        Q = spread(tuple(P.n), self.s, self.w, P.p, q)
        U = conv_direct_full(P, self.K, Q)
        Gs = spread(tuple(P.n), self.s, self.w, P.p, g)
        V = conv_direct_full(P, np.conj(self.K[::-1, ::-1, ::-1]), Gs)
        obs = gather_grad(U, self.s, self.w, self.dw, P.p)
        src = gather_grad(V, self.s, self.w, self.dw, P.p)
        out = np.real(np.conj(g)[:, None] * obs) + np.real(q[:, None] * np.conj(src))
        if len(P.pdims):
            nf = tuple(P.nf)
            uf = far_sum(P, self.F, spread(nf, self.ss, self.ws, P.pf, q))
            vf = far_sum(P, self.F, spread(nf, self.so, self.wo, P.pf, g), adjoint=True)
            obs_f = gather_grad(uf, self.so, self.wo, self.dwo, P.pf)
            src_f = gather_grad(vf, self.ss, self.ws, self.dws, P.pf)
            out += np.real(np.conj(g)[:, None] * obs_f) + np.real(q[:, None] * np.conj(src_f))
        m, n, ii = self.corrections()[:3]
        D = correction_grads(P, self.pts, self.s, self.w, self.dw, m, n, ii)
        I = P.images()
        ph_minus = np.exp(1j * (I[ii] * P.D) @ P.k0)        # phase of image -i
        ph = np.exp(-1j * (I[ii] * P.D) @ P.k0)
        # D already carries phase_i; the source-side term needs phase_{-i}
        t1 = np.real(np.conj(g[m])[:, None] * D * q[n][:, None])
        t2 = np.real(q[m][:, None] * np.conj(g[n])[:, None] * D * (ph_minus / ph)[:, None])
        for d in range(3):
            out[:, d] += np.bincount(m, weights=t1[:, d] + t2[:, d], minlength=len(q))
        return out



# ---------------------------------------------------------------------------
# observer points apart from the sources (Sec. 4.1's accuracy test: the
# potential evaluated at points that carry no source)
# ---------------------------------------------------------------------------
def apply_observers(P, src, obs, q):
    """u at the observers obs (M, 3) due to strengths q at the sources src
    (N, 3): Eq. 1 with r_m an observer.  The operator of the point set
    [src; obs] in which the observers carry zero strength, read at the
    observers' rows.  Neutral static case: Eq. neutral holds for q over the
    sources, whose residual mean is removed there only."""
    src = np.asarray(src, np.float64)
    obs = np.asarray(obs, np.float64)
    q = np.asarray(q, np.complex128)
    if P.npsp:
        if abs(np.sum(q)) > P.neutral_tol * np.sum(np.abs(q)):
            raise ValueError("charges are not neutral (Eq. neutral)")
        q = q - np.mean(q)
    full = np.concatenate([q, np.zeros(len(obs), np.complex128)])
    return Plan(P, np.vstack([src, obs])).apply(full)[len(src):]


def apply_observers_adjoint(P, src, obs, v):
    """The adjoint of apply_observers: strengths at the sources from values v
    at the observers (the source rows of A^H applied to [0; v]), projected on
    the sources' neutral subspace in the neutral static case."""
    src = np.asarray(src, np.float64)
    full = np.concatenate([np.zeros(len(src), np.complex128), np.asarray(v, np.complex128)])
    w = Plan(P, np.vstack([src, np.asarray(obs, np.float64)])).apply_adjoint(full)[:len(src)]
    return w - np.mean(w) if P.npsp else w
