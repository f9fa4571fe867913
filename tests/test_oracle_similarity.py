"""Pins of the FP64 oracle of extended convolution with a joint rotation x
scale field (log-polar harmonics: the angular components of Sec. 4.1 times
the log-radial ones of Sec. 8): a separable filter against its closed form,
identity and constant fields against library FFT convolution, the scale-only
and rotation-only special cases against the (separately pinned) scale and
SO(2) oracles, the impulse response (Sec. 2.3), and the normalised modes.
CPU only."""
import math

import numpy as np

from oracle.scale import MellinFilter, ext_conv_scale
from oracle.similarity import SimilarityFilter, conv, conv_at, smooth
from oracle.so2 import ext_conv_so2

LP = 6.0                     # log-period
W1 = 2 * math.pi / LP        # w_1


def separable_filter(r_min=1.0, r_max=5.0, cd=0.4):
    """c_{k,j} = a_k b_j with A(phi) = 1 + cos(2 phi + 0.3), B(u) = 0.3 + cos(w_1 u - 0.7)."""
    a = {0: 1.0, 2: 0.5 * np.exp(0.3j)}
    b = {-1: 0.5 * np.exp(0.7j), 0: 0.3, 1: 0.5 * np.exp(-0.7j)}
    c = np.zeros((3, 3), np.complex128)
    for k, ak in a.items():
        for j, bj in b.items():
            c[k, j + 1] = ak * bj
    return SimilarityFilter(c, LP, r_min, r_max, cd)


def closed_form(dx, dy, alpha, s, r_min=1.0, r_max=5.0, cd=0.4):
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    rr = np.where(r > 0, r, 1.0)
    v = (1 + np.cos(2 * (th - alpha) + 0.3)) * (0.3 + np.cos(W1 * (np.log(rr) - np.log(s)) - 0.7))
    v = np.where((r >= r_min) & (r <= r_max), v, 0.0)
    return np.where(r == 0, cd, v)


def fft_conv(A, vals, dx, dy):
    g = np.zeros(A.shape)
    np.add.at(g, (dy % A.shape[0], dx % A.shape[1]), vals)
    return np.fft.ifft2(np.fft.fft2(A) * np.fft.fft2(g)).real


def box(R):
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    return dx.ravel(), dy.ravel()


def test_separable_filter_matches_its_closed_form():
    f = separable_filter()
    rng = np.random.default_rng(0)
    dx, dy = rng.uniform(-6, 6, 300), rng.uniform(-6, 6, 300)
    dx[:3], dy[:3] = 0.0, 0.0
    for alpha, s in ((0.0, 1.0), (0.9, 1.7), (-2.1, 0.6)):
        np.testing.assert_allclose(f.transformed(dx, dy, alpha, s), closed_form(dx, dy, alpha, s), atol=1e-13)


def test_identity_and_constant_fields_are_fft_convolutions():
    f = separable_filter()
    rng = np.random.default_rng(1)
    A = rng.standard_normal((18, 20))
    dx, dy = box(5)
    one = np.ones_like(A)
    np.testing.assert_allclose(conv(A, 0 * one, one, f), fft_conv(A, closed_form(dx, dy, 0.0, 1.0), dx, dy),
                               atol=1e-11)
    np.testing.assert_allclose(conv(A, 1.1 * one, 1.6 * one, f),
                               fft_conv(A, closed_form(dx, dy, 1.1, 1.6), dx, dy), atol=1e-11)


def test_scale_only_filter_equals_the_scale_oracle():
    """K = 0: the rotation field drops out and the operator is Sec. 8's."""
    rng = np.random.default_rng(2)
    n = 4
    c = np.zeros((1, 2 * n - 1), np.complex128)
    c[0, n - 1:] = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    c[0, n - 1] = c[0, n - 1].real
    f = SimilarityFilter(c, 5.0, 1.0, 6.0, 0.7)
    A = rng.standard_normal((16, 16))
    s = rng.uniform(1.0, 2.5, A.shape)
    alpha = rng.uniform(0, 2 * math.pi, A.shape)
    ref = ext_conv_scale(A, s, MellinFilter(c[0, n - 1:], 5.0, 1.0, 6.0, 0.7))
    np.testing.assert_allclose(conv(A, alpha, s, f), ref, atol=1e-11)


class _AngularOnly:
    """Adapter giving the SO(2) oracle the radial functions f_k(r) = c_{k,0} on the annulus."""

    def __init__(self, f: SimilarityFilter):
        self.f, self.K = f, f.K

    def radial(self, k, r):
        r = np.asarray(r, np.float64)
        v = np.where((r >= self.f.r_min) & (r <= self.f.r_max), self.f.coef(k, 0), 0.0)
        return np.where(r == 0, self.f.centre_tap if k == 0 else 0.0, v)


def test_rotation_only_filter_equals_the_so2_oracle():
    """One log-radial harmonic (j = 0): the scale field drops out and the
    operator is the SO(2) extended convolution of Sec. 4.1."""
    rng = np.random.default_rng(3)
    K = 3
    c = np.zeros((K + 1, 1), np.complex128)
    c[:, 0] = rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)
    c[0, 0] = c[0, 0].real
    f = SimilarityFilter(c, 4.0, 0.95, 4.05, -0.3)   # no lattice point on the window's edges
    A = rng.standard_normal((14, 15))
    alpha = rng.uniform(0, 2 * math.pi, A.shape)
    s = rng.uniform(0.5, 3.0, A.shape)
    ref = ext_conv_so2(A, _AngularOnly(f), alpha, 4).real
    np.testing.assert_allclose(conv(A, alpha, s, f), ref, atol=1e-11)


def test_impulse_response_is_the_filter_transformed_at_the_impulse():
    f = separable_filter()
    rng = np.random.default_rng(4)
    A = np.zeros((20, 20))
    A[7, 11] = 1.0
    alpha = rng.uniform(0, 2 * math.pi, A.shape)
    s = rng.uniform(0.7, 2.0, A.shape)
    out = conv(A, alpha, s, f)
    dx, dy = box(5)
    ref = np.zeros(A.shape)
    ref[(7 + dy) % 20, (11 + dx) % 20] = closed_form(dx, dy, alpha[7, 11], s[7, 11])
    np.testing.assert_allclose(out, ref, atol=1e-13)


def test_normalised_modes_reproduce_constants_and_sampled_form_agrees():
    f = separable_filter(cd=1.5)
    rng = np.random.default_rng(5)
    h, w = 16, 18
    alpha = rng.uniform(0, 2 * math.pi, (h, w))
    s = rng.uniform(0.8, 1.6, (h, w))
    img = np.full((2, h, w), 0.3)
    img[1] = -2.0
    for mode in (1, 2):
        np.testing.assert_allclose(smooth(img, alpha, s, f, mode), img, rtol=1e-12)
    A = rng.standard_normal((h, w))
    full = conv(A, alpha, s, f)
    pix = np.array([(0, 0), (5, 17), (15, 3)])
    np.testing.assert_allclose(conv_at(A, alpha, s, f, pix), full[tuple(pix.T)], atol=1e-12)


def test_harmonic_form_equals_the_brute_force():
    """The steering identity the GPU path uses: one convolution per log-polar
    harmonic of the signal modulated by e^{-ik alpha} e^{-i w_j ln s}."""
    from oracle.similarity import conv_from_components
    rng = np.random.default_rng(6)
    K, n = 2, 3
    c = rng.standard_normal((K + 1, 2 * n - 1)) + 1j * rng.standard_normal((K + 1, 2 * n - 1))
    f = SimilarityFilter(c, 5.0, 0.95, 4.5, 0.6)
    A = rng.standard_normal((12, 13))
    alpha = rng.uniform(0, 2 * math.pi, A.shape)
    s = rng.uniform(0.6, 2.2, A.shape)
    np.testing.assert_allclose(conv_from_components(A, alpha, s, f), conv(A, alpha, s, f), atol=1e-10)
