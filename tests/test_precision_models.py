"""Precision model of storing the scale path's steered spectra in BF16
(CPU only).  The scale-adaptive convolution (Sec. 8) is computed as one
convolution per log-radial harmonic of the steered signal,
    {A, s} * F = sum_k (A e^{-i w_k ln s}) * F_k + c_delta A,
F_k(d) = c_k e^{i w_k ln|d|} on the annulus, so the only intermediates that
could be stored in a narrower type are the steered spectra FFT(A e^{-i w_k ln s}).
The model rounds them (real and imaginary parts) to BF16, or splits them into
BF16 hi + lo, and measures the output error against FP64: a single BF16 is
far outside the 1e-4 bar of the mixed-precision forms, and hi + lo meets it
but carries the same four bytes per value as FP32.  There is no contraction
to move to the tensor cores either: the harmonics are summed per frequency
with a different filter value each, a batched dot product of length n_h with
no reuse."""
import numpy as np

import synth
from oracle.scale import MellinFilter, ext_conv_scale


def bf16(x):
    a = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def harmonic_conv(A, s, filt, rounding=None):
    h, w = A.shape
    R = filt.box_radius()
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    r = np.hypot(dx, dy)
    inside = (r >= filt.r_min) & (r <= filt.r_max)
    lr = np.log(np.where(r > 0, r, 1.0))
    out = np.zeros((h, w), np.complex128)
    for k in range(-(filt.n - 1), filt.n):
        ck = filt.c[k] if k >= 0 else np.conj(filt.c[-k])
        wk = 2 * np.pi * k / filt.L
        grid = np.zeros((h, w), np.complex128)
        np.add.at(grid, (dy % h, dx % w), np.where(inside, ck * np.exp(1j * wk * lr), 0.0))
        S = np.fft.fft2(A * np.exp(-1j * wk * np.log(s)))
        if rounding == "bf16":
            S = bf16(S.real) + 1j * bf16(S.imag)
        elif rounding == "bf16x2":
            hr, hi = bf16(S.real), bf16(S.imag)
            S = (hr + bf16(S.real - hr)) + 1j * (hi + bf16(S.imag - hi))
        out += np.fft.ifft2(S * np.fft.fft2(grid))
    return out.real + filt.centre_tap * A


def test_bf16_steered_spectra_error_model():
    rng = np.random.default_rng(0)
    n = 64
    A = rng.uniform(0, 1, (n, n))
    s = np.exp(rng.uniform(0, np.log(8.0), (n, n)))
    c = synth.mellin_gaussian_coeffs(n_h=24, log_period=8.0)
    filt = MellinFilter(c, 8.0, 1.0, 10.0, 1.0)
    ref = ext_conv_scale(A, s, filt)
    exact = harmonic_conv(A, s, filt)
    assert np.linalg.norm(exact - ref) / np.linalg.norm(ref) < 1e-11   # the model is the operator
    e1 = np.linalg.norm(harmonic_conv(A, s, filt, "bf16") - ref) / np.linalg.norm(ref)
    e2 = np.linalg.norm(harmonic_conv(A, s, filt, "bf16x2") - ref) / np.linalg.norm(ref)
    print(f"steered spectra in BF16: rel-L2 {e1:.2e}; BF16 hi+lo: {e2:.2e}")
    assert e1 > 1e-4
    assert e2 < 1e-4
