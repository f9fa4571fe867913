"""Pins of the scale-adaptive (Mellin) FP64 oracle: closed-form Gaussian
profiles, library FFT convolution, the unit-integral property stated in
Sec. 8, and exact reproduction of constant images.  CPU only."""
import math

import numpy as np
import pytest

import synth
from oracle.scale import MellinFilter, ext_conv_scale, ext_conv_scale_at, smooth


def small_filter(r_max=7.0):
    c = synth.mellin_gaussian_coeffs()
    return MellinFilter(c, 8.0, 1.0, r_max, 1.0)


def gaussian_grid(h, w, sigma, r_min, r_max, centre):
    g = np.zeros((h, w))
    R = int(r_max)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            r = math.hypot(dx, dy)
            if r == 0:
                g[0, 0] += centre
            elif r_min <= r <= r_max:
                g[dy % h, dx % w] += math.exp(-r * r / (2 * sigma * sigma))
    return g


def test_profile_matches_gaussian_family():
    f = small_filter()
    u = np.linspace(-math.log(8), math.log(64), 5001)
    assert np.max(np.abs(f.profile(u) - np.exp(-np.exp(2 * u) / 2))) < 5e-7
    # scaled filter = Gaussian of width s (direction of the scale action)
    d = np.arange(1, 8, dtype=np.float64)
    for s in (1.0, 1.6, 2.5):
        np.testing.assert_allclose(f.scaled(d, 0 * d, s), np.exp(-d * d / (2 * s * s)), atol=5e-7)


@pytest.mark.parametrize("s0", [1.0, 1.7])
def test_constant_scale_is_fft_convolution_with_gaussian(s0):
    rng = np.random.default_rng(3)
    h, w = 20, 23
    A = rng.standard_normal((h, w))
    f = small_filter()
    s = np.full((h, w), s0)
    got = ext_conv_scale(A, s, f)
    g = gaussian_grid(h, w, s0, 1.0, 7.0, 1.0)
    expect = np.fft.ifft2(np.fft.fft2(A) * np.fft.fft2(g)).real
    # fit error (<= 1e-7 per tap) times ~150 taps
    np.testing.assert_allclose(got, expect, atol=5e-5)


def test_unit_integral_scaling():
    """Sec. 8: scaling the filter by s scales its integral by s^2."""
    f = MellinFilter(synth.mellin_gaussian_coeffs(), 8.0, 1.0, 64.0, 1.0)
    dy, dx = np.mgrid[-64:65, -64:65]
    sums = [np.sum(f.scaled(dx, dy, s)) / (s * s) for s in (1.0, 2.0, 3.5, 6.0)]
    np.testing.assert_allclose(sums, 2 * np.pi, rtol=1e-5)


def test_constant_image_is_reproduced_exactly():
    rng = np.random.default_rng(5)
    h, w = 16, 18
    s = rng.uniform(1.0, 2.0, (h, w))
    img = np.full((2, h, w), 0.37)
    for mode in (1, 2):
        out = smooth(img, s, small_filter(), mode=mode)
        np.testing.assert_allclose(out, 0.37, rtol=1e-13)


def test_gather_form_matches_scatter_form():
    rng = np.random.default_rng(8)
    h, w = 17, 19
    A = rng.standard_normal((h, w))
    s = rng.uniform(1.0, 2.0, (h, w))
    f = small_filter()
    full = ext_conv_scale(A, s, f)
    pix = np.array([[0, 0], [16, 18], [5, 9], [11, 2]])
    np.testing.assert_allclose(ext_conv_scale_at(A, s, f, pix), full[pix[:, 0], pix[:, 1]],
                               atol=1e-12)


def test_unnormalised_smoothing_darkens_small_scales():
    """Sec. 8 discussion of the failure modes: without the division, regions
    with narrow filters accumulate less and come out darker."""
    h, w = 24, 24
    s = np.where(np.arange(w)[None, :] < w // 2, 1.0, 2.0) * np.ones((h, 1))
    img = np.ones((1, h, w))
    raw = smooth(img, s, small_filter(), mode=0)[0]
    assert raw[:, 3:9].mean() < raw[:, 15:21].mean()


def test_unit_integral_normalisation_stops_bleeding_across_the_mask():
    """Sec. 8 discussion of the failure modes: dividing by {1, T} * F restores
    the luminance but, with H not divided by |T|^2, the wide filters of the
    large-scale side carry s^2 times the mass of the narrow ones and bleed
    across the mask boundary; with H / |T|^2 every source spreads unit mass.
    Step image 0 | 1 on a step mask s = 1 | 3 (periodic, so two boundaries):
    the sharp side next to the boundary picks up more of the other side in
    mode 1 than in mode 2, both stay in [0, 1], and far from the boundaries
    (beyond the filter reach) both reproduce the image."""
    h, w = 8, 48
    left = np.arange(w)[None, :] < w // 2
    s = np.where(left, 1.0, 3.0) * np.ones((h, 1))
    img = np.where(left, 0.0, 1.0)[None] * np.ones((1, h, 1))
    f = small_filter(r_max=10.0)
    m1 = smooth(img, s, f, mode=1)[0]
    m2 = smooth(img, s, f, mode=2)[0]
    near = [w // 2 - 2, w // 2 - 1]               # sharp side, next to the boundary at w / 2
    assert m1[:, near].mean() > m2[:, near].mean() + 1e-3
    for m in (m1, m2):   # a normalised average; the fitted profile's lobes (< 5e-7) may overshoot slightly
        assert m.min() > -1e-6 and m.max() < 1 + 1e-6
    # columns farther than the widest filter's reach (10 px) from both boundaries (w/2 and 0 = w)
    far_left = [11, 12]
    np.testing.assert_allclose(m1[:, far_left], 0.0, atol=1e-9)
    np.testing.assert_allclose(m2[:, far_left], 0.0, atol=1e-9)


def test_disk_profile_matches_the_smoothed_disk():
    """Depth-defocus filter (Sec. 8): 64 Mellin frequencies reproduce the
    radially smoothed disk indicator 1 / (1 + e^{(ln r - ln s) / tau}) to 1e-6."""
    f = MellinFilter(synth.mellin_disk_coeffs(), 8.0, 1.0, 64.0, 1.0)
    u = np.linspace(-math.log(8), math.log(64), 5001)
    assert np.max(np.abs(f.profile(u) - 1.0 / (1.0 + np.exp(u / 0.1)))) < 1e-6
    d = np.arange(1, 30, dtype=np.float64)
    for s in (2.0, 5.5):
        np.testing.assert_allclose(f.scaled(d, 0 * d, s), 1.0 / (1.0 + (d / s) ** 10), atol=1e-6)


def test_disk_integral_scales_with_the_square_of_the_scale():
    """Sum of the lattice taps / s^2 against 2 pi int P(ln r) r dr (a 1D
    quadrature of the smoothed disk, about pi): the lattice sum converges to
    the integral as the disk grows, within the design range s <= 8 (the fit
    covers u = ln r - ln s >= -ln 8 on radii r >= 1; beyond it the
    log-periodic basis repeats and the centre of a larger disk is lost)."""
    f = MellinFilter(synth.mellin_disk_coeffs(), 8.0, 1.0, 64.0, 1.0)
    r = np.linspace(1e-6, 64.0, 400001)
    area = 2 * math.pi * np.trapezoid(r / (1.0 + r ** 10), r)
    dy, dx = np.mgrid[-64:65, -64:65]
    for s, tol in ((2.0, 3e-2), (4.0, 1e-3), (8.0, 1e-5)):
        assert abs(np.sum(f.scaled(dx, dy, s)) / (s * s) - area) <= tol * area
