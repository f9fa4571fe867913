"""FP64 oracle for extended convolution with a joint rotation x scale field
(transformation fields of rotations and isotropic scales, the extension the
paper's conclusion names; Eq. Def-EConv with the angular harmonics of Sec. 4.1
and the log-radial harmonics of Sec. 8), test infrastructure only.

Filter in log-polar harmonics:

    F(d) = Q(theta(d), ln|d|)  for r_min <= |d| <= r_max,  F(0) = c_delta,  else 0,
    Q(phi, u) = sum_{|k| <= K} sum_{|j| <= n-1} c_{k,j} exp(i k phi) exp(i w_j u),
    w_j = 2 pi j / L,   c_{-k,-j} = conj(c_{k,j})  (F is real).

The coefficients are given as c[k, j + n - 1] for k = 0..K; in row k = 0 only
j >= 0 is read (the rest follows from the symmetry).

A similarity g = (alpha, s) acts by (T_g F)(d) = F(R(-alpha) d / s), read in
log-polar coordinates on the fixed support window (as the scale family of
Sec. 8 is):

    (T_g F)(d) = Q(theta(d) - alpha, ln|d| - ln s)  for r_min <= |d| <= r_max,
    (T_g F)(0) = c_delta,

so harmonic (k, j) is multiplied by exp(-i k alpha) exp(-i w_j ln s).

Extended convolution (Eq. Def-EConv), gathered at p:
    ({A, g} * F)(p) = sum_d A(p - d) (T_{g(p - d)} F)(d).
Smoothing, as for the scale oracle:
    mode 0:  {H, g} * F
    mode 1:  {H, g} * F / {1, g} * F                 (Eq. normalization)
    mode 2:  {H/s^2, g} * F / {1/s^2, g} * F
"""
from __future__ import annotations

import numpy as np


class SimilarityFilter:
    def __init__(self, c, log_period, r_min, r_max, centre_tap):
        self.c = np.asarray(c, np.complex128)          # (K + 1, 2n - 1)
        self.K = self.c.shape[0] - 1
        self.n = (self.c.shape[1] + 1) // 2
        self.L = float(log_period)
        self.r_min = float(r_min)
        self.r_max = float(r_max)
        self.centre_tap = float(centre_tap)

    def coef(self, k: int, j: int) -> complex:
        """c_{k,j} for any k in [-K, K], j in [-(n-1), n-1], by the real symmetry."""
        if k < 0 or (k == 0 and j < 0):
            return complex(np.conj(self.c[-k, -j + self.n - 1]))
        return complex(self.c[k, j + self.n - 1])

    def q(self, phi, u):
        """Q(phi, u), every harmonic summed (real part; the imaginary part is rounding)."""
        phi = np.asarray(phi, np.float64)
        u = np.asarray(u, np.float64)
        out = np.zeros(np.broadcast(phi, u).shape, np.complex128)
        for k in range(-self.K, self.K + 1):
            for j in range(-(self.n - 1), self.n):
                out += self.coef(k, j) * np.exp(1j * (k * phi + 2 * np.pi * j / self.L * u))
        return out.real

    def transformed(self, dx, dy, alpha, s):
        """(T_g F)(d) for g = (alpha, s), broadcast over all arguments."""
        dx = np.asarray(dx, np.float64)
        dy = np.asarray(dy, np.float64)
        r = np.hypot(dx, dy)
        inside = (r >= self.r_min) & (r <= self.r_max)
        rr = np.where(r > 0, r, 1.0)
        val = np.where(inside, self.q(np.arctan2(dy, dx) - alpha, np.log(rr) - np.log(s)), 0.0)
        return np.where(r == 0, self.centre_tap, val)

    def box_radius(self):
        return int(np.floor(self.r_max))


def _offsets(filt: SimilarityFilter):
    R = filt.box_radius()
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    keep = dx * dx + dy * dy <= filt.r_max ** 2
    return dx[keep], dy[keep]


def conv_at(A, alpha, s, filt: SimilarityFilter, pixels):
    """{A, g} * F gathered at ``pixels`` (rows of (row, col)), periodic."""
    A = np.asarray(A, np.float64)
    alpha = np.asarray(alpha, np.float64)
    s = np.asarray(s, np.float64)
    h, w = A.shape
    dx, dy = _offsets(filt)
    pix = np.asarray(pixels, np.int64).reshape(-1, 2)
    out = np.zeros(len(pix))
    for n, (py, px) in enumerate(pix):
        qy, qx = (py - dy) % h, (px - dx) % w
        out[n] = np.sum(A[qy, qx] * filt.transformed(dx, dy, alpha[qy, qx], s[qy, qx]))
    return out


def conv(A, alpha, s, filt: SimilarityFilter):
    """Full-image {A, g} * F as a scatter: out(q + d) += A(q) (T_{g(q)} F)(d)."""
    A = np.asarray(A, np.float64)
    alpha = np.asarray(alpha, np.float64)
    s = np.asarray(s, np.float64)
    out = np.zeros(A.shape)
    for dx, dy in zip(*_offsets(filt)):
        out += np.roll(A * filt.transformed(dx, dy, alpha, s), (dy, dx), axis=(0, 1))
    return out


def smooth(img, alpha, s, filt: SimilarityFilter, mode: int = 1, pixels=None):
    """(C, h, w) image through one of the three modes; full image, or at ``pixels``."""
    img = np.asarray(img, np.float64)
    s = np.asarray(s, np.float64)
    wgt = 1.0 / (s * s) if mode == 2 else np.ones_like(s)
    op = (lambda A: conv(A, alpha, s, filt)) if pixels is None else (lambda A: conv_at(A, alpha, s, filt, pixels))
    num = [op(ch * wgt) for ch in img]
    if mode == 0:
        return np.stack(num)
    den = op(wgt)
    return np.stack([x / den for x in num])


def conv_from_components(A, alpha, s, filt: SimilarityFilter):
    """The same operator by its harmonic form: for every (k, j), the signal
    modulated by e^{-ik alpha} e^{-i w_j ln s}, convolved (periodic, direct
    sum over the window) with c_{k,j} e^{ik theta} e^{i w_j ln r}; plus the
    centre tap times A.  Real part of the complex sum."""
    A = np.asarray(A, np.float64)
    alpha = np.asarray(alpha, np.float64)
    ls = np.log(np.asarray(s, np.float64))
    dx, dy = _offsets(filt)
    r = np.hypot(dx, dy).astype(np.float64)
    inside = (r >= filt.r_min) & (r <= filt.r_max) & (r > 0)
    th = np.arctan2(dy, dx)
    lr = np.log(np.where(r > 0, r, 1.0))
    out = np.zeros(A.shape, np.complex128)
    for k in range(-filt.K, filt.K + 1):
        for j in range(-(filt.n - 1), filt.n):
            wj = 2 * np.pi * j / filt.L
            U = A * np.exp(-1j * (k * alpha + wj * ls))
            g = np.where(inside, filt.coef(k, j) * np.exp(1j * (k * th + wj * lr)), 0.0)
            for n in np.nonzero(g)[0]:
                out += np.roll(U, (dy[n], dx[n]), axis=(0, 1)) * g[n]
    return out.real + filt.centre_tap * A
