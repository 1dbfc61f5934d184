"""Cubic B-spline interpolation of an image, FP64.

The paper samples both images at the mesh nodes by "spline interpolation"
(abstract; Sec. 2.1, the definition of ``Re(X)``).  It names no degree and no
boundary rule.  Reading adopted: cubic B-spline, whole-sample mirror boundary,
coefficients by the recursive prefilter of M. Unser, "Splines: a perfect fit
for signal and image processing", IEEE SPM 16(6), 1999 (pole ``z1 = sqrt(3)-2``,
gain ``(1-z1)(1-1/z1) = 6``), applied along rows and then along columns.

Test infrastructure: see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np

Z1 = math.sqrt(3.0) - 2.0


def prefilter_axis(s: np.ndarray, axis: int) -> np.ndarray:
    """B-spline coefficients along one axis (Unser 1999, causal + anticausal).

    With ``c = 6 s`` and the mirror-periodic extension of period ``2N-2``:
      causal:     c+(0) = sum over one period of z^k c~(k), / (1 - z^(2N-2))
                  c+(n) = c(n) + z c+(n-1)
      anticausal: c-(N-1) = z / (z^2 - 1) * (c+(N-1) + z c+(N-2))
                  c-(n) = z (c-(n+1) - c+(n))
    The result ``c-`` satisfies (c(k-1) + 4 c(k) + c(k+1)) / 6 = s(k) with
    mirrored neighbours at both ends.
    """
    c = 6.0 * np.moveaxis(np.asarray(s, dtype=np.float64), axis, 0).copy()
    n = c.shape[0]
    if n == 1:
        return np.moveaxis(c / 6.0, 0, axis)
    z = Z1
    period = 2 * n - 2
    k = np.arange(n, dtype=np.float64)
    init = np.tensordot(z ** k, c, axes=(0, 0))
    if n > 2:
        j = np.arange(1, n - 1, dtype=np.float64)
        init = init + np.tensordot(z ** (period - j), c[1:n - 1], axes=(0, 0))
    cp = np.empty_like(c)
    cp[0] = init / (1.0 - z ** period)
    for i in range(1, n):
        cp[i] = c[i] + z * cp[i - 1]
    cm = np.empty_like(c)
    cm[n - 1] = (z / (z * z - 1.0)) * (cp[n - 1] + z * cp[n - 2])
    for i in range(n - 2, -1, -1):
        cm[i] = z * (cm[i + 1] - cp[i])
    return np.moveaxis(cm, 0, axis)


def prefilter_2d(img: np.ndarray) -> np.ndarray:
    """Coefficients of a (H, W) image: rows (x) first, then columns (y)."""
    return prefilter_axis(prefilter_axis(img, 1), 0)


def mirror_index(k: np.ndarray, n: int) -> np.ndarray:
    """Whole-sample mirror extension of integer index ``k`` into ``[0, n)``."""
    k = np.asarray(k, dtype=np.int64)
    if n == 1:
        return np.zeros_like(k)
    period = 2 * n - 2
    k = np.abs(k) % period
    return np.where(k >= n, period - k, k)


def cubic_weights(t: np.ndarray):
    """Cubic B-spline weights of the taps at i-1, i, i+1, i+2 for t in [0,1)."""
    t2 = t * t
    t3 = t2 * t
    w0 = (1.0 - t) ** 3 / 6.0
    w1 = (3.0 * t3 - 6.0 * t2 + 4.0) / 6.0
    w2 = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) / 6.0
    w3 = t3 / 6.0
    return (w0, w1, w2, w3)


def cubic_dweights(t: np.ndarray):
    """Derivatives of :func:`cubic_weights` with respect to t."""
    t2 = t * t
    d0 = -0.5 * (1.0 - t) ** 2
    d1 = 1.5 * t2 - 2.0 * t
    d2 = -1.5 * t2 + t + 0.5
    d3 = 0.5 * t2
    return (d0, d1, d2, d3)


def cubic_d2weights(t: np.ndarray):
    """Second derivatives of :func:`cubic_weights` with respect to t."""
    return (1.0 - t, 3.0 * t - 2.0, 1.0 - 3.0 * t, t + 0.0 * t)


def hessian(coef: np.ndarray, x, y):
    """Second derivatives (d2/dx2, d2/dxdy, d2/dy2) of the spline at (x, y),
    FP64, with the same mirror extension as :func:`evaluate`."""
    coef = np.asarray(coef, dtype=np.float64)
    H, W = coef.shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ix = np.floor(x)
    iy = np.floor(y)
    tx, ty = x - ix, y - iy
    ix = ix.astype(np.int64)
    iy = iy.astype(np.int64)
    wx, wy = cubic_weights(tx), cubic_weights(ty)
    dx, dy = cubic_dweights(tx), cubic_dweights(ty)
    ex, ey = cubic_d2weights(tx), cubic_d2weights(ty)
    hxx = np.zeros(np.broadcast(x, y).shape)
    hxy = np.zeros_like(hxx)
    hyy = np.zeros_like(hxx)
    for m in range(4):
        rows = mirror_index(iy - 1 + m, H)
        for n in range(4):
            c = coef[rows, mirror_index(ix - 1 + n, W)]
            hxx += wy[m] * ex[n] * c
            hxy += dy[m] * dx[n] * c
            hyy += ey[m] * wx[n] * c
    return hxx, hxy, hyy


def evaluate(coef: np.ndarray, x, y, grad: bool = False):
    """Spline value (and optionally d/dx, d/dy) at points (x, y), FP64.

    Coordinates are never clamped: outside the image the mirror extension of
    the coefficients applies.
    """
    coef = np.asarray(coef, dtype=np.float64)
    H, W = coef.shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ix = np.floor(x)
    iy = np.floor(y)
    tx = x - ix
    ty = y - iy
    ix = ix.astype(np.int64)
    iy = iy.astype(np.int64)
    wx = cubic_weights(tx)
    wy = cubic_weights(ty)
    if grad:
        dx = cubic_dweights(tx)
        dy = cubic_dweights(ty)
    val = np.zeros(np.broadcast(x, y).shape)
    gx = np.zeros_like(val)
    gy = np.zeros_like(val)
    for m in range(4):
        rows = mirror_index(iy - 1 + m, H)
        for n in range(4):
            cols = mirror_index(ix - 1 + n, W)
            c = coef[rows, cols]
            val += wy[m] * wx[n] * c
            if grad:
                gx += wy[m] * dx[n] * c
                gy += dy[m] * wx[n] * c
    if grad:
        return val, gx, gy
    return val
