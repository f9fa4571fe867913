"""FP64 oracle for the normalised extended convolution of Sec. 8 (Eq.
normalization) with a rotation field, as used for Line Integral Convolution
(Sec. 8, last application), and for the anisotropic Gaussian filter that
application uses (test infrastructure only).

* Normalised convolution: out_c = ({H_c, T} * F) / ({1, T} * F) for every
  channel c, both extended convolutions as in oracle.so2 (Eq. Def-EConv); for
  a rotation field no division of the signal by |T|^2 is needed (Sec. 8).
* Anisotropic Gaussian F(x, y) = exp(-x^2 / (2 su^2) - y^2 / (2 sv^2)) (long
  along x when su > sv).  Written in polar form,
      F(r, theta) = exp(-A r^2) exp(B r^2 cos 2 theta),
      A = (1/su^2 + 1/sv^2) / 4,  B = (1/sv^2 - 1/su^2) / 4,
  and the Jacobi-Anger expansion exp(z cos p) = sum_n I_n(z) e^{i n p} gives
  its angular components in closed form:
      f_{2n}(r) = exp(-A r^2) I_n(B r^2) = exp(-r^2 / (2 su^2)) ive(n, B r^2),
      f_k = 0 for odd k
  (ive the exponentially scaled modified Bessel function, which keeps the
  product finite for large r).
"""
from __future__ import annotations

import numpy as np
from scipy import special

from .so2 import ext_conv_so2, ext_conv_so2_at


def aniso_gauss(x, y, su: float, sv: float):
    return np.exp(-np.asarray(x, np.float64) ** 2 / (2 * su * su) - np.asarray(y, np.float64) ** 2 / (2 * sv * sv))


def aniso_gauss_table(su: float, sv: float, K: int, dr: float, r_max: float):
    """Radial table f_k(i dr), k = -K..K, i = 0..floor(r_max / dr), of the
    anisotropic Gaussian's angular components (closed form above),
    complex128 of shape (2K + 1, n)."""
    n = int(np.floor(r_max / dr + 1e-9)) + 1
    r = np.arange(n) * dr
    B = (1.0 / (sv * sv) - 1.0 / (su * su)) / 4.0
    fk = np.zeros((2 * K + 1, n), np.complex128)
    for k in range(-K, K + 1):
        if k % 2 == 0:
            fk[k + K] = np.exp(-r * r / (2 * su * su)) * special.ive(abs(k) // 2, B * r * r)
    return fk


def normalized_conv_so2(H, filt, alpha, radius: int):
    """Full-image normalised extended convolution; H has shape (channels, h, w)
    or (h, w).  Real part, float64."""
    H = np.asarray(H, np.float64)
    D = ext_conv_so2(np.ones(H.shape[-2:]), filt, alpha, radius).real
    if H.ndim == 2:
        return ext_conv_so2(H, filt, alpha, radius).real / D
    return np.stack([ext_conv_so2(Hc, filt, alpha, radius).real / D for Hc in H])


def normalized_conv_so2_at(H, filt, alpha, radius: int, pixels):
    """The same at ``pixels`` (array of (row, col)); H of shape (h, w)."""
    H = np.asarray(H, np.float64)
    num = ext_conv_so2_at(H, filt, alpha, radius, pixels).real
    den = ext_conv_so2_at(np.ones(H.shape), filt, alpha, radius, pixels).real
    return num / den
