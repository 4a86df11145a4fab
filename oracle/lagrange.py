"""Lagrange interpolation on a uniform grid, FP64.  TEST INFRASTRUCTURE ONLY.

Sec. 3.2 (Eq. PGF_interp and the text after it): a q-th order Lagrange
interpolation uses (q+1) nodes per dimension, (q+1)^3 in 3D, and the source
and observer coefficients are the same functions of position.  The paper does
not say how the q+1 nodes are placed around a point nor what happens at the
edge of the grid; the reading used here (stencil centred on the point, then
clamped into the grid) is:

    even p : s = floor(x/h + 1/2) - p/2
    odd  p : s = floor(x/h)       - (p-1)/2
    s      = min(max(s, 0), n-1-p)
    t      = x/h - s                     (local coordinate, in [0, p] inside)
    w_j(t) = prod_{l != j} (t - l)/(j - l),   j = 0..p

For the observer grid of the far zone (nodes shifted by +Delta/2, Eq. grid)
the same rule is applied to x - Delta/2.
"""
import numpy as np


def stencil_start(x, h, n, p, shift=0.0):
    """First stencil node index per coordinate (int64 array) and the local
    coordinate t = (x - shift)/h - s.  Decided in FP64."""
    x = np.asarray(x, dtype=np.float64)
    u = (x - shift) / h if shift != 0.0 else x / h
    if p % 2 == 0:
        s = np.floor(u + 0.5).astype(np.int64) - p // 2
    else:
        s = np.floor(u).astype(np.int64) - (p - 1) // 2
    s = np.clip(s, 0, n - 1 - p)
    return s, u - s


def weights(t, p):
    """Lagrange basis values w_j(t), j = 0..p, for the nodes 0..p.
    t: array (...,) -> (..., p+1)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.ones(t.shape + (p + 1,), dtype=np.float64)
    for j in range(p + 1):
        for l in range(p + 1):
            if l != j:
                out[..., j] *= (t - l) / (j - l)
    return out


def dweights(t, p):
    """d/dt of the Lagrange basis, by the product rule:
    w_j'(t) = sum_{k != j} [1/(j-k)] prod_{l != j,k} (t-l)/(j-l)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros(t.shape + (p + 1,), dtype=np.float64)
    for j in range(p + 1):
        for k in range(p + 1):
            if k == j:
                continue
            term = np.full(t.shape, 1.0 / (j - k))
            for l in range(p + 1):
                if l != j and l != k:
                    term = term * (t - l) / (j - l)
            out[..., j] += term
    return out


def box_index(x, h, n):
    """Box (cell of the grid) containing x: floor(x/h) clamped to [0, n-1]."""
    b = np.floor(np.asarray(x, dtype=np.float64) / h).astype(np.int64)
    return np.clip(b, 0, n - 1)


def stencil_box(x, h, n, p):
    """Box of x in the sense of the box-adaptive integral method: the set of
    points that share one interpolation stencil.  Even p: the box centred on
    node b = floor(x/h + 1/2), b in [0, n-1]; odd p: the grid cell
    b = floor(x/h), b in [0, n-2].  All points of a box have the stencil
    start min(max(b - lo, 0), n-1-p), lo = p/2 or (p-1)/2."""
    u = np.asarray(x, dtype=np.float64) / h
    if p % 2 == 0:
        return np.clip(np.floor(u + 0.5).astype(np.int64), 0, n - 1)
    return np.clip(np.floor(u).astype(np.int64), 0, n - 2)
