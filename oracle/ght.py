"""FP64 oracle for the pattern-detection front end of Sec. 5 (test
infrastructure only).

* Signal and field, Eq. signal and Eq. theta: H = |grad I| and
  theta = atan2(dI/dy, dI/dx).  Reading: central differences with periodic
  indices, dI/dx(y, x) = (I(y, x+1) - I(y, x-1)) / 2 (x = column, y = row).
* Consensus filter, Eq. opt_filt (and its derivation in the appendix): every
  pattern point q near the centre c votes with weight |grad P(q)| into the bin
  at the centre's position in the frame of q, whose x-axis is the gradient
  direction: d = R(-theta_P(q)) (c - q).  Reading: the points q are the
  pattern pixels with |q - c| <= eps (the support disk of the appendix), and
  the unit impulse is discretised as a bilinear splat onto the integer
  offsets, which keeps each vote's mass.  The box is [-R, R]^2 with
  R = ceil(eps) + 1, so every splat lands inside it.
* Detection: the extended convolution {H, theta} * F of Eq. Def-EConv, with F
  band-limited to |k| <= K (oracle.so2, oracle.filters_so2).

R(a) = [[cos a, -sin a], [sin a, cos a]] acting on (x, y), as everywhere in
the SO(2) oracle.
"""
from __future__ import annotations

import math

import numpy as np


def gradient_field(I):
    """(H, theta) of an image: |grad I| and atan2(dI/dy, dI/dx), central
    differences, periodic indices, float64."""
    I = np.asarray(I, np.float64)
    gx = 0.5 * (np.roll(I, -1, axis=1) - np.roll(I, 1, axis=1))
    gy = 0.5 * (np.roll(I, -1, axis=0) - np.roll(I, 1, axis=0))
    return np.hypot(gx, gy), np.arctan2(gy, gx)


def consensus_radius(eps: float) -> int:
    """Half side R of the filter box for a support radius eps."""
    return int(math.ceil(eps)) + 1


def consensus_from_gradient(mag, theta, centre, eps: float):
    """Consensus filter of Eq. opt_filt from a pattern's gradient magnitude and
    direction: (2R+1)^2 float64 array, offset d = (dx, dy) at [dy + R, dx + R].
    centre = (cy, cx), integer pixel of the pattern centre."""
    mag = np.asarray(mag, np.float64)
    theta = np.asarray(theta, np.float64)
    cy, cx = centre
    R = consensus_radius(eps)
    F = np.zeros((2 * R + 1, 2 * R + 1))
    hp, wp = mag.shape
    for qy in range(hp):
        for qx in range(wp):
            oy, ox = cy - qy, cx - qx           # c - q
            if ox * ox + oy * oy > eps * eps or mag[qy, qx] == 0.0:
                continue
            c, s = math.cos(theta[qy, qx]), math.sin(theta[qy, qx])
            dx = c * ox + s * oy                # R(-theta) (c - q)
            dy = -s * ox + c * oy
            x0, y0 = math.floor(dx), math.floor(dy)
            fx, fy = dx - x0, dy - y0
            wgt = mag[qy, qx]
            for yy, wy in ((y0, 1.0 - fy), (y0 + 1, fy)):
                for xx, wx in ((x0, 1.0 - fx), (x0 + 1, fx)):
                    F[yy + R, xx + R] += wgt * wy * wx
    return F


def consensus_filter(P, centre, eps: float):
    """Consensus filter of the pattern image P (its gradient by gradient_field)."""
    mag, theta = gradient_field(P)
    return consensus_from_gradient(mag, theta, centre, eps)
