"""Pins of the FP64 oracle of the normalised extended convolution (Sec. 8,
Eq. normalization) and of the anisotropic Gaussian's angular components used
for Line Integral Convolution.  CPU only."""
import math

import numpy as np

from oracle.filters_so2 import RadialTable, filter_eval
from oracle.normalized import (aniso_gauss, aniso_gauss_table, normalized_conv_so2, normalized_conv_so2_at)
from oracle.so2 import box_offsets


def _quadrature_components(su, sv, K, r, n_theta=4096):
    """f_k(r) = (1 / 2 pi) int F(r cos t, r sin t) e^{-ikt} dt by the trapezoidal
    rule (spectrally accurate for a smooth periodic integrand)."""
    t = 2 * math.pi * np.arange(n_theta) / n_theta
    vals = aniso_gauss(np.outer(r, np.cos(t)), np.outer(r, np.sin(t)), su, sv)
    out = np.zeros((2 * K + 1, len(r)), np.complex128)
    for k in range(-K, K + 1):
        out[k + K] = (vals * np.exp(-1j * k * t)).mean(axis=1)
    return out


def test_closed_form_components_match_angular_quadrature():
    """The Jacobi-Anger / Bessel closed form against direct quadrature of the
    angular Fourier integral, including the vanishing odd components."""
    su, sv, K, dr = 6.0, 1.5, 10, 0.25
    fk = aniso_gauss_table(su, sv, K, dr, 20.0)
    r = np.arange(fk.shape[1]) * dr
    ref = _quadrature_components(su, sv, K, r)
    assert np.abs(fk - ref).max() <= 1e-13


def test_isotropic_gaussian_has_only_the_zero_component():
    fk = aniso_gauss_table(3.0, 3.0, 6, 0.5, 12.0)
    r = np.arange(fk.shape[1]) * 0.5
    np.testing.assert_allclose(fk[6].real, np.exp(-r * r / 18.0), atol=1e-15)
    assert np.abs(np.delete(fk, 6, axis=0)).max() == 0.0


def test_band_limited_sum_reconstructs_a_mildly_anisotropic_gaussian():
    """With enough components the table filter evaluates to F itself (up to the
    cubic-Hermite interpolation between radial samples)."""
    su, sv = 4.0, 3.0
    filt = RadialTable(aniso_gauss_table(su, sv, 12, 0.05, 14.0), 0.05)
    rng = np.random.default_rng(1)
    x, y = rng.uniform(-9, 9, 400), rng.uniform(-9, 9, 400)
    np.testing.assert_allclose(filter_eval(filt, x, y).real, aniso_gauss(x, y, su, sv), atol=2e-6)


def _small(seed, h=20, w=24):
    rng = np.random.default_rng(seed)
    H = rng.uniform(0, 1, (h, w))
    alpha = rng.uniform(0, 2 * math.pi, (h, w))
    filt = RadialTable(aniso_gauss_table(3.0, 1.0, 6, 0.25, 5.0), 0.25)
    return H, alpha, filt


def test_constant_signal_is_reproduced_exactly():
    """Normalisation makes every output a weighted average: a constant image
    comes back unchanged whatever the field."""
    _, alpha, filt = _small(2)
    out = normalized_conv_so2(np.full(alpha.shape, 0.37), filt, alpha, 5)
    np.testing.assert_allclose(out, 0.37, rtol=1e-12)


def test_zero_field_is_fft_convolution_divided_by_the_filter_sum():
    """alpha = 0: numerator = periodic convolution with F sampled on the box,
    denominator = the sum of the samples (a constant)."""
    H, alpha, filt = _small(3)
    R = 5
    dx, dy = box_offsets(R)
    g = np.zeros(H.shape, np.complex128)
    np.add.at(g, (dy % H.shape[0], dx % H.shape[1]), filter_eval(filt, dx.astype(float), dy.astype(float)))
    conv = np.fft.ifft2(np.fft.fft2(H) * np.fft.fft2(g)).real
    got = normalized_conv_so2(H, filt, np.zeros_like(H), R)
    np.testing.assert_allclose(got, conv / g.real.sum(), atol=1e-12)


def test_sampled_form_and_channels_match_the_full_image():
    H, alpha, filt = _small(4)
    full = normalized_conv_so2(np.stack([H, 1 - H]), filt, alpha, 5)
    pix = np.array([(0, 0), (3, 7), (19, 23), (10, 12)])
    np.testing.assert_allclose(normalized_conv_so2_at(H, filt, alpha, 5, pix), full[0][tuple(pix.T)], rtol=1e-12)
    np.testing.assert_allclose(full[1], 1 - full[0], atol=1e-12)   # linear in H, weights sum to one
