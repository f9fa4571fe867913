"""SO(2) filter models for the FP64 oracle (test infrastructure only).

A filter with angular bandwidth K is written, as in Sec. 4.1 ("Filter
Decomposition"), as

    F(x) = sum_{k=-K..K} f_k(|x|) exp(i k theta(x)),  theta(x) = atan2(x_y, x_x),

with x_x the column offset and x_y the row offset.  At x = 0 the angle is
undefined; only the k = 0 term is kept there (F(0) = f_0(0)).

Rotating a filter by an angle alpha is (T_alpha F)(x) = F(R(-alpha) x) with
R(a) = [[cos a, -sin a], [sin a, cos a]]; on a single harmonic exp(i k theta)
this multiplies by exp(-i k alpha) (Sec. 3, "Example n = 1"; Sec. 4.1).

Three ways to give f_k(r):
  * :class:`AnalyticGaussPow` -- f_k(r) = a_k r^|k| exp(-r^2 / (2 sigma^2)).
  * :class:`RadialTable` -- samples f_k(i*dr) with a cubic Hermite interpolant
    (the paper does not say how f_k is evaluated between radii; this
    interpolant *defines* the filter for every consumer).
  * :func:`decompose_sampled` -- a sampled filter image, expressed in polar
    coordinates and transformed by a DFT along each circle (Sec. 4.1,
    "Filter Decomposition"), giving a :class:`RadialTable`.
"""
from __future__ import annotations

import math

import numpy as np


class AnalyticGaussPow:
    """f_k(r) = a_k * r^|k| * exp(-r^2 / (2 sigma^2)), k = -K..K (a[k + K])."""

    def __init__(self, a, sigma: float):
        self.a = np.asarray(a, np.complex128)
        self.K = (len(self.a) - 1) // 2
        self.sigma = float(sigma)

    def radial(self, k: int, r):
        r = np.asarray(r, np.float64)
        return self.a[k + self.K] * r ** abs(k) * np.exp(-r * r / (2 * self.sigma ** 2))

    @property
    def r_max(self):
        return math.inf


class RadialTable:
    """f_k at r_i = i * dr, i = 0..n-1, interpolated by a cubic Hermite spline.

    On [r_i, r_{i+1}] with t = r/dr - i:
        f = h00(t) v_i + h10(t) m_i + h01(t) v_{i+1} + h11(t) m_{i+1},
        h00 = 2t^3 - 3t^2 + 1, h10 = t^3 - 2t^2 + t, h01 = -2t^3 + 3t^2,
        h11 = t^3 - t^2,
    tangents m_i = (v_{i+1} - v_{i-1}) / 2 (in units of one table step),
    with v_{-1} = (-1)^k v_1 (f_k extended to negative radius, since
    f_k(-r) exp(i k (theta + pi)) = f_k(r) exp(i k theta)) and v_n = 0.
    f_k(r) = 0 for r / dr > (n-1) + 1e-9: the support is closed, and a
    lattice point on its boundary circle stays inside however the rotated
    coordinate rounds (the spline need not vanish at the last sample).
    """

    def __init__(self, fk, dr: float):
        self.fk = np.asarray(fk, np.complex128)  # shape (2K+1, n)
        self.K = (self.fk.shape[0] - 1) // 2
        self.n = self.fk.shape[1]
        self.dr = float(dr)

    @property
    def r_max(self):
        return (self.n - 1) * self.dr

    def radial(self, k: int, r):
        return hermite_eval(self.fk[k + self.K], self.dr, k, r)


def hermite_eval(v, dr: float, parity: int, r):
    """Cubic Hermite interpolant of samples v_i = f(i dr) (see RadialTable),
    with f extended to negative radius as f(-r) = (-1)^parity f(r), v_n = 0,
    and f = 0 for r / dr > n - 1 + 1e-9."""
    r = np.asarray(r, np.float64)
    v = np.asarray(v, np.complex128)
    n = len(v)
    ext = np.zeros(n + 3, np.complex128)      # ext[j + 1] = v_j, j = -1..n+1
    ext[1:n + 1] = v
    ext[0] = ((-1) ** abs(parity)) * v[1] if n > 1 else 0.0
    u = r / dr
    i = np.floor(u).astype(np.int64)
    inside = (u <= n - 1 + 1e-9) & (i >= 0)
    i = np.clip(i, 0, n - 1)
    t = u - i
    vi = ext[i + 1]
    vi1 = ext[i + 2]
    mi = 0.5 * (ext[i + 2] - ext[i])
    mi1 = 0.5 * (ext[i + 3] - ext[i + 1])
    t2 = t * t
    t3 = t2 * t
    val = ((2 * t3 - 3 * t2 + 1) * vi + (t3 - 2 * t2 + t) * mi
           + (-2 * t3 + 3 * t2) * vi1 + (t3 - t2) * mi1)
    return np.where(inside, val, 0.0)


def filter_eval(filt, x, y):
    """F(x, y) = sum_k f_k(r) exp(i k theta); F(0) = f_0(0)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    r = np.hypot(x, y)
    th = np.arctan2(y, x)
    at0 = r == 0
    out = np.zeros(np.broadcast(x, y).shape, np.complex128)
    for k in range(-filt.K, filt.K + 1):
        term = filt.radial(k, r) * np.exp(1j * k * th)
        if k != 0:
            term = np.where(at0, 0.0, term)
        out += term
    return out


def rotated_filter_eval(filt, dx, dy, alpha):
    """(T_alpha F)(d) = F(R(-alpha) d), with the rotated coordinate formed
    explicitly: x' = cos(a) dx + sin(a) dy, y' = -sin(a) dx + cos(a) dy."""
    c = np.cos(alpha)
    s = np.sin(alpha)
    return filter_eval(filt, c * dx + s * dy, -s * dx + c * dy)


# ------------------------------------------------------ filter decomposition ---

def keys_weight(x):
    """Keys cubic convolution kernel with a = -1/2."""
    a = -0.5
    x = np.abs(np.asarray(x, np.float64))
    return np.where(x <= 1, (a + 2) * x ** 3 - (a + 3) * x ** 2 + 1,
                    np.where(x < 2, a * x ** 3 - 5 * a * x ** 2 + 8 * a * x - 4 * a, 0.0))


def sample_bicubic(img, cx, cy):
    """Keys bicubic sample of ``img`` (rows = y, cols = x) at continuous pixel
    coordinates (cx, cy); pixels outside the image count as zero."""
    img = np.asarray(img, np.float64)
    hh, ww = img.shape
    cx = np.asarray(cx, np.float64)
    cy = np.asarray(cy, np.float64)
    x0 = np.floor(cx).astype(np.int64)
    y0 = np.floor(cy).astype(np.int64)
    tx = cx - x0
    ty = cy - y0
    out = np.zeros(np.broadcast(cx, cy).shape)
    for jy in range(-1, 3):
        wy = keys_weight(ty - jy)
        yy = y0 + jy
        for jx in range(-1, 3):
            wx = keys_weight(tx - jx)
            xx = x0 + jx
            ok = (yy >= 0) & (yy < hh) & (xx >= 0) & (xx < ww)
            v = img[np.clip(yy, 0, hh - 1), np.clip(xx, 0, ww - 1)]
            out += np.where(ok, wx * wy * v, 0.0)
    return out


def decompose_sampled(img, K: int, dr: float, n_theta: int, r_max: float | None = None):
    """Angular-harmonic decomposition of a sampled, centred filter image.

    Sec. 4.1 "Filter Decomposition": express F in polar coordinates, then take
    a 1D DFT along every circle.  Here the image (side 2R+1, centre pixel R)
    is resampled at radii r_i = i*dr (r_i <= r_max, default R) and angles
    theta_t = 2 pi t / n_theta with the Keys bicubic kernel, and

        f_k(r_i) = (1/n_theta) sum_t P(r_i, theta_t) exp(-i k theta_t),  |k| <= K.

    Returns a :class:`RadialTable`; at r = 0 the k != 0 entries are set to 0.
    """
    img = np.asarray(img, np.float64)
    side = img.shape[0]
    R = (side - 1) // 2
    if r_max is None:
        r_max = float(R)
    n_r = int(math.floor(r_max / dr + 1e-9)) + 1
    r = np.arange(n_r) * dr
    th = 2 * math.pi * np.arange(n_theta) / n_theta
    rr, tt = np.meshgrid(r, th, indexing="ij")
    polar = sample_bicubic(img, R + rr * np.cos(tt), R + rr * np.sin(tt))  # (n_r, n_theta)
    fk = np.zeros((2 * K + 1, n_r), np.complex128)
    for k in range(-K, K + 1):
        fk[k + K] = (polar * np.exp(-1j * k * th)[None, :]).sum(axis=1) / n_theta
    fk[:, 0] = 0.0
    fk[K, 0] = polar[0, 0]
    return RadialTable(fk, dr)
