"""FP64 oracle for scale-adaptive extended convolution and smoothing (Sec. 8;
test infrastructure only).

Filter (Sec. 8: F_k(r) = e^{ik log r} f_k; radially symmetric, so f_k are
constants c_k):

    F(d) = P(ln|d|)  for r_min <= |d| <= r_max,   F(0) = c_delta,   else 0,
    P(u) = sum_{k=-(n-1)..n-1} c_k exp(i w_k u),  w_k = 2 pi k / L,
    c_{-k} = conj(c_k)  (P is real).

Scaling by s multiplies the k-th harmonic by exp(-i w_k ln s), i.e. the
transformed filter is F_s(d) = P(ln|d| - ln s) on the same support, with the
centre tap unchanged (it is the trivial representation).  The support window
is fixed: the paper leaves it open, and only this reading keeps the filter a
finite sum of scale harmonics.

Extended convolution (Eq. Def-EConv) with this family, gathered at p:

    ({A, s} * F)(p) = sum_{d} A(p - d) F_{s(p - d)}(d).

Smoothing (Eq. normalization and the unit-integral signal H~ = H / s^2):
    mode 0:  {H, s} * F
    mode 1:  {H, s} * F / {1, s} * F
    mode 2:  {H/s^2, s} * F / {1/s^2, s} * F
"""
from __future__ import annotations

import numpy as np


class MellinFilter:
    def __init__(self, c, log_period, r_min, r_max, centre_tap):
        self.c = np.asarray(c, np.complex128)   # c_0 .. c_{n-1}
        self.n = len(self.c)
        self.L = float(log_period)
        self.r_min = float(r_min)
        self.r_max = float(r_max)
        self.centre_tap = float(centre_tap)

    def profile(self, u):
        """P(u), summed over k = -(n-1)..n-1 (real part; imaginary part is rounding)."""
        u = np.asarray(u, np.float64)
        out = np.zeros(u.shape, np.complex128)
        for k in range(-(self.n - 1), self.n):
            ck = self.c[k] if k >= 0 else np.conj(self.c[-k])
            out += ck * np.exp(1j * 2 * np.pi * k / self.L * u)
        return out.real

    def scaled(self, dx, dy, s):
        """F_s(d) = P(ln|d| - ln s) on the support window, c_delta at d = 0."""
        r = np.hypot(np.asarray(dx, np.float64), np.asarray(dy, np.float64))
        s = np.asarray(s, np.float64)
        inside = (r >= self.r_min) & (r <= self.r_max)
        rr = np.where(r > 0, r, 1.0)
        val = np.where(inside, self.profile(np.log(rr) - np.log(s)), 0.0)
        return np.where(r == 0, self.centre_tap, val)

    def box_radius(self):
        return int(np.floor(self.r_max))


def ext_conv_scale(A, s, filt: MellinFilter):
    """Full-image {A, s} * F as a scatter: out(q + d) += A(q) F_{s(q)}(d)."""
    A = np.asarray(A, np.float64)
    s = np.asarray(s, np.float64)
    R = filt.box_radius()
    out = np.zeros(A.shape)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            if dx * dx + dy * dy > filt.r_max ** 2:
                continue
            contrib = A * filt.scaled(dx, dy, s)
            out += np.roll(contrib, (dy, dx), axis=(0, 1))
    return out


def ext_conv_scale_at(A, s, filt: MellinFilter, pixels):
    """{A, s} * F gathered at ``pixels`` (rows of (row, col))."""
    A = np.asarray(A, np.float64)
    s = np.asarray(s, np.float64)
    h, w = A.shape
    R = filt.box_radius()
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    keep = dx * dx + dy * dy <= filt.r_max ** 2
    dx = dx[keep]
    dy = dy[keep]
    pix = np.asarray(pixels, np.int64).reshape(-1, 2)
    out = np.zeros(len(pix))
    for n, (py, px) in enumerate(pix):
        qy = (py - dy) % h
        qx = (px - dx) % w
        out[n] = np.sum(A[qy, qx] * filt.scaled(dx, dy, s[qy, qx]))
    return out


def smooth(img, s, filt: MellinFilter, mode: int = 2, pixels=None):
    """Scale-adaptive smoothing of a (C, h, w) image in one of the three
    modes above; full image, or only at ``pixels``."""
    img = np.asarray(img, np.float64)
    s = np.asarray(s, np.float64)
    w = 1.0 / (s * s) if mode == 2 else np.ones_like(s)
    conv = ext_conv_scale if pixels is None else (
        lambda A, ss, f: ext_conv_scale_at(A, ss, f, pixels))
    num = [conv(ch * w, s, filt) for ch in img]
    if mode == 0:
        return np.stack(num)
    den = conv(w, s, filt)
    return np.stack([n / den for n in num])
