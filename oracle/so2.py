"""FP64 oracle for SO(2) extended convolution and correlation (test
infrastructure only).

Discretisation (the paper states the operators as integrals over the plane):
integrals become unit-weight sums over the integer lattice, indices are taken
mod (h, w), and the filter is summed over the square box B = [-R, R]^2 of
offsets d = (dx, dy) (dx = column, dy = row).  A box wider than the image
wraps and its taps accumulate.

* Extended correlation, Eq. Def-ECorr (Sec. 2.1): the filter is transformed by
  T(p) at the *output* point and gathered,
      out(p) = sum_{d in B} H(p + d) * conj(F(R(-alpha(p)) d)).
* Extended convolution, Eq. Def-EConv (Sec. 2.2): the filter is transformed by
  T(q) at the *input* point and scattered,
      out(q + d) += H(q) * F(R(-alpha(q)) d)   for all q and d in B.
* Quantised-rotation sweep (Sec. 5.2, the "O(N) rotations of the filter"
  comparison): S(p, j) = sum_d H(p + d) conj(F(R(-alpha_j) d)) with
  alpha_j = 2 pi j / J, then max over j and the smallest maximising j.

Every value is computed per point from the closed-form expansion of F at the
explicitly rotated coordinate; the steering identity is never used here.
"""
from __future__ import annotations

import numpy as np

from .filters_so2 import rotated_filter_eval


def box_offsets(radius: int):
    dy, dx = np.mgrid[-radius:radius + 1, -radius:radius + 1]
    return dx.ravel().astype(np.int64), dy.ravel().astype(np.int64)


def ext_corr_so2(H, filt, alpha, radius: int):
    """Full-image extended correlation (Eq. Def-ECorr), complex128 result."""
    H = np.asarray(H, np.float64)
    alpha = np.asarray(alpha, np.float64)
    out = np.zeros(H.shape, np.complex128)
    for dx, dy in zip(*box_offsets(radius)):
        shifted = np.roll(H, (-dy, -dx), axis=(0, 1))          # H[p + d]
        out += shifted * np.conj(rotated_filter_eval(filt, float(dx), float(dy), alpha))
    return out


def ext_conv_so2(H, filt, alpha, radius: int):
    """Full-image extended convolution (Eq. Def-EConv) as a scatter."""
    H = np.asarray(H, np.float64)
    alpha = np.asarray(alpha, np.float64)
    out = np.zeros(H.shape, np.complex128)
    for dx, dy in zip(*box_offsets(radius)):
        contrib = H * rotated_filter_eval(filt, float(dx), float(dy), alpha)  # indexed by q
        out += np.roll(contrib, (dy, dx), axis=(0, 1))                     # lands on q + d
    return out


def ext_corr_so2_at(H, filt, alpha, radius: int, pixels):
    """Eq. Def-ECorr evaluated only at ``pixels`` (array of (row, col))."""
    H = np.asarray(H, np.float64)
    alpha = np.asarray(alpha, np.float64)
    h, w = H.shape
    pix = np.asarray(pixels, np.int64).reshape(-1, 2)
    dx, dy = box_offsets(radius)
    out = np.zeros(len(pix), np.complex128)
    for n, (py, px) in enumerate(pix):
        vals = H[(py + dy) % h, (px + dx) % w]
        f = rotated_filter_eval(filt, dx.astype(np.float64), dy.astype(np.float64),
                                float(alpha[py, px]))
        out[n] = np.sum(vals * np.conj(f))
    return out


def ext_conv_so2_at(H, filt, alpha, radius: int, pixels):
    """Eq. Def-EConv gathered at ``pixels``: out(p) = sum_d H(p - d) F(R(-alpha(p - d)) d)."""
    H = np.asarray(H, np.float64)
    alpha = np.asarray(alpha, np.float64)
    h, w = H.shape
    pix = np.asarray(pixels, np.int64).reshape(-1, 2)
    dx, dy = box_offsets(radius)
    out = np.zeros(len(pix), np.complex128)
    for n, (py, px) in enumerate(pix):
        qy = (py - dy) % h
        qx = (px - dx) % w
        f = rotated_filter_eval(filt, dx.astype(np.float64), dy.astype(np.float64),
                                alpha[qy, qx])
        out[n] = np.sum(H[qy, qx] * f)
    return out


def rotated_filter_bank(filt, radius: int, J: int):
    """(J, |B|) table of F(R(-alpha_j) d), alpha_j = 2 pi j / J."""
    dx, dy = box_offsets(radius)
    bank = np.zeros((J, dx.size), np.complex128)
    for j in range(J):
        bank[j] = rotated_filter_eval(filt, dx.astype(np.float64), dy.astype(np.float64),
                                      2 * np.pi * j / J)
    return bank


def sweep_so2_at(H, filt, radius: int, J: int, pixels, bank=None):
    """Scores S(p, j) (complex; real for a real filter) at ``pixels``."""
    H = np.asarray(H, np.float64)
    h, w = H.shape
    pix = np.asarray(pixels, np.int64).reshape(-1, 2)
    dx, dy = box_offsets(radius)
    if bank is None:
        bank = rotated_filter_bank(filt, radius, J)
    patches = H[(pix[:, 0:1] + dy[None, :]) % h, (pix[:, 1:2] + dx[None, :]) % w]
    return patches @ np.conj(bank).T


def sweep_so2_fft(H, filt, radius: int, J: int, workers: int = -1):
    """Full-image scores S(p, j) via one FFT correlation per rotated filter
    (Sec. 5.2's "convolve with O(N) rotations" form; the FFT is a library step).

    Returns (max over j, first argmax, the full (J, h, w) score stack is not
    kept).  Real filters only."""
    import scipy.fft as sfft
    H = np.asarray(H, np.float64)
    h, w = H.shape
    dx, dy = box_offsets(radius)
    Hf = sfft.rfft2(H, workers=workers)
    best = np.full((h, w), -np.inf)
    arg = np.zeros((h, w), np.int64)
    second = np.full((h, w), -np.inf)
    for j in range(J):
        f = rotated_filter_eval(filt, dx.astype(np.float64), dy.astype(np.float64),
                                2 * np.pi * j / J).real
        grid = np.zeros((h, w))
        np.add.at(grid, (dy % h, dx % w), f)
        s = sfft.irfft2(Hf * np.conj(sfft.rfft2(grid, workers=workers)), s=(h, w),
                        workers=workers)
        upd = s > best
        second = np.where(upd, best, np.maximum(second, s))
        arg = np.where(upd, j, arg)
        best = np.where(upd, s, best)
    return best, arg, second


def component_correlation_fft(H, filt, k: int, radius: int, workers: int = -1):
    """G_k of component_correlation through the FFT (Sec. 4.1 "Standard
    Correlation" done as the paper does it; the FFT is a library step):
    F_k sampled on the box and wrapped onto the image grid (taps of a box
    wider than the image accumulate), G_k = IFFT(FFT(H) conj(FFT(F_k)))."""
    import scipy.fft as sfft
    H = np.asarray(H, np.float64)
    h, w = H.shape
    dx, dy = box_offsets(radius)
    r = np.hypot(dx, dy).astype(np.float64)
    th = np.arctan2(dy, dx).astype(np.float64)
    fk = filt.radial(k, r) * np.exp(1j * k * th)
    if k != 0:
        fk = np.where(r == 0, 0.0, fk)
    grid = np.zeros((h, w), np.complex128)
    np.add.at(grid, (dy % h, dx % w), fk)
    return sfft.ifft2(sfft.fft2(H, workers=workers) * np.conj(sfft.fft2(grid, workers=workers)), workers=workers)


def sweep_so2_steered(H, filt, K: int, radius: int, J: int, workers: int = -1, chunk: int = 1 << 18):
    """Whole-image sweep by the paper's own route (Sec. 4.1 for a real filter,
    then max over the quantised angles of Sec. 5): the K + 1 component
    correlations through the FFT, then at every alpha_j = 2 pi j / J the
    linear combination S(p, j) = G_0(p) + 2 sum_{k=1..K} Re(e^{i k alpha_j}
    G_k(p)) (a matrix product over the components, a library step), then per
    pixel the maximum and the smallest maximising j.  Returns (best, arg)."""
    G = [component_correlation_fft(H, filt, k, radius, workers) for k in range(K + 1)]
    h, w = np.shape(H)
    P = h * w
    cols = [G[0].real.ravel()]
    for k in range(1, K + 1):
        cols += [G[k].real.ravel(), G[k].imag.ravel()]
    A = np.stack(cols, axis=1)                                    # (P, 2K + 1)
    B = np.zeros((2 * K + 1, J))
    a = 2 * np.pi * np.arange(J) / J
    B[0] = 1.0
    for k in range(1, K + 1):
        B[2 * k - 1] = 2 * np.cos(k * a)                           # 2 Re(e^{ika} G) = 2 cos Re G - 2 sin Im G
        B[2 * k] = -2 * np.sin(k * a)
    best = np.empty(P)
    arg = np.empty(P, np.int64)
    for c in range(0, P, chunk):
        S = A[c:c + chunk] @ B
        arg[c:c + chunk] = np.argmax(S, axis=1)
        best[c:c + chunk] = S[np.arange(S.shape[0]), arg[c:c + chunk]]
    return best.reshape(h, w), arg.reshape(h, w)


def component_correlation(H, filt, k: int, radius: int):
    """Sec. 4.1 "Standard Correlation": G_k(p) = sum_{d in B} H(p + d) conj(F_k(d)),
    F_k(d) = f_k(|d|) e^{i k theta(d)} (F_k(0) = 0 for k != 0)."""
    H = np.asarray(H, np.float64)
    dx, dy = box_offsets(radius)
    r = np.hypot(dx, dy).astype(np.float64)
    th = np.arctan2(dy, dx).astype(np.float64)
    fk = filt.radial(k, r) * np.exp(1j * k * th)
    if k != 0:
        fk = np.where(r == 0, 0.0, fk)
    out = np.zeros(H.shape, np.complex128)
    for n in range(dx.size):
        out += np.roll(H, (-dy[n], -dx[n]), axis=(0, 1)) * np.conj(fk[n])
    return out


def sweep_from_components(G, K: int, J: int):
    """Sec. 4.1 "Linear Combination" at every alpha_j = 2 pi j / J for a real
    filter: S(p, j) = sum_{k=-K..K} e^{i k alpha_j} G_k(p) with
    G_{-k} = conj(G_k).  ``G`` is a list [G_0, ..., G_K]; returns (J, ...)."""
    S = []
    for j in range(J):
        a = 2 * np.pi * j / J
        s = np.zeros(np.shape(G[0]), np.complex128)
        for k in range(-K, K + 1):
            g = G[k] if k >= 0 else np.conj(G[-k])
            s = s + np.exp(1j * k * a) * g
        S.append(s)
    return np.stack(S)
