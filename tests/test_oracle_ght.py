"""Pins of the FP64 oracle of the pattern-detection front end (Sec. 5): the
gradient signal and field, the voted consensus filter (Eq. opt_filt) and
detection by extended convolution.  CPU only."""
import math

import numpy as np

import synth
from oracle.filters_so2 import decompose_sampled
from oracle.ght import consensus_filter, consensus_from_gradient, consensus_radius, gradient_field
from oracle.so2 import ext_conv_so2, ext_conv_so2_at


def test_gradient_of_a_ramp_is_its_slope():
    """Central differences are exact on a linear ramp (away from the periodic seam)."""
    h, w, a, b = 24, 32, 0.7, -1.3
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    H, th = gradient_field(a * x + b * y)
    inner = (slice(1, h - 1), slice(1, w - 1))
    np.testing.assert_allclose(H[inner], math.hypot(a, b), rtol=1e-13)
    np.testing.assert_allclose(th[inner], math.atan2(b, a), atol=1e-13)


def test_gradient_of_a_periodic_wave_closed_form():
    """(sin(om (x+1)) - sin(om (x-1))) / 2 = sin(om) cos(om x) holds on the whole
    periodic grid, seam included; the y-derivative of a row-constant image is 0."""
    h, w, m = 16, 40, 3
    om = 2 * math.pi * m / w
    x = np.arange(w, dtype=np.float64)
    I = np.tile(np.sin(om * x), (h, 1))
    H, th = gradient_field(I)
    g = math.sin(om) * np.cos(om * x)
    np.testing.assert_allclose(H, np.tile(np.abs(g), (h, 1)), atol=1e-14)
    nz = np.abs(g) > 1e-9
    np.testing.assert_allclose(th[:, nz], np.tile(np.where(g[nz] > 0, 0.0, math.pi), (h, 1)), atol=1e-12)


def test_single_votes_land_in_the_gradient_frame():
    """One point q with gradient angle theta votes at d = R(-theta)(c - q):
    theta = 0 keeps the offset, theta = pi/2 turns (-3, 0) into (0, 3); a
    fractional target splits the vote bilinearly."""
    eps = 6.0
    R = consensus_radius(eps)
    c = (8, 8)
    for theta, want in ((0.0, {(0, -3): 1.0}), (math.pi / 2, {(3, 0): 1.0})):
        mag = np.zeros((17, 17))
        th = np.zeros((17, 17))
        mag[8, 11] = 2.5          # q = c + (3, 0): c - q = (-3, 0)
        th[8, 11] = theta
        F = consensus_from_gradient(mag, th, c, eps)
        exp = np.zeros_like(F)
        for (dy, dx), v in want.items():
            exp[dy + R, dx + R] = 2.5 * v
        np.testing.assert_allclose(F, exp, atol=1e-15)
    # theta = atan2(1, 2): R(-theta) (-3, -4)... target (dx, dy) = (c ox + s oy, -s ox + c oy)
    mag = np.zeros((17, 17))
    th = np.zeros((17, 17))
    mag[12, 11] = 1.0             # q = c + (3, 4): c - q = (-3, -4)
    th[12, 11] = math.atan2(1.0, 2.0)
    F = consensus_from_gradient(mag, th, c, eps)
    cs, sn = 2 / math.sqrt(5), 1 / math.sqrt(5)
    dx, dy = cs * -3 + sn * -4, -sn * -3 + cs * -4
    x0, y0 = math.floor(dx), math.floor(dy)
    fx, fy = dx - x0, dy - y0
    exp = np.zeros_like(F)
    exp[y0 + R, x0 + R] = (1 - fx) * (1 - fy)
    exp[y0 + R, x0 + 1 + R] = fx * (1 - fy)
    exp[y0 + 1 + R, x0 + R] = (1 - fx) * fy
    exp[y0 + 1 + R, x0 + 1 + R] = fx * fy
    np.testing.assert_allclose(F, exp, atol=1e-14)


def test_consensus_filter_keeps_the_vote_mass():
    rng = np.random.default_rng(5)
    P = synth.smooth_random_template(rng, 12, 2.0)
    eps = 10.5
    F = consensus_filter(P, (12, 12), eps)
    mag, _ = gradient_field(P)
    yy, xx = np.mgrid[-12:13, -12:13]
    assert abs(F.sum() - mag[xx ** 2 + yy ** 2 <= eps ** 2].sum()) <= 1e-12 * F.sum()


def test_consensus_filter_is_invariant_under_rotating_the_pattern():
    """Votes are cast in each point's gradient frame, so rotating the pattern
    about its centre leaves the filter unchanged (exact for quarter turns,
    which map the lattice and the central differences onto themselves).  A
    rotation of the wrong sense would turn the filter by a half turn."""
    rng = np.random.default_rng(11)
    P = synth.smooth_random_template(rng, 15, 2.5)
    F0 = consensus_filter(P, (15, 15), 13.0)
    for k in (1, 2, 3):
        Fk = consensus_filter(np.rot90(P, k), (15, 15), 13.0)
        np.testing.assert_allclose(Fk, F0, atol=1e-12 * np.abs(F0).max())


def _plant(img, P, centre, k):
    r = P.shape[0] // 2
    cy, cx = centre
    img[cy - r:cy + r + 1, cx - r:cx + r + 1] += np.rot90(P, k)


def test_detection_response_is_rotation_invariant_and_peaks_at_the_centres():
    """Four copies of a pattern, turned by quarter turns, in a 96 x 96 image:
    the extended convolution of the gradient signal with the band-limited
    consensus filter, steered by the gradient field, responds equally at the
    four centres (the detection is rotation invariant), and those responses
    are the four largest in the image."""
    rng = np.random.default_rng(21)
    P = synth.smooth_random_template(rng, 8, 1.5)
    img = np.zeros((96, 96))
    centres = [(24, 24), (24, 72), (72, 24), (72, 72)]
    for k, c in enumerate(centres):
        _plant(img, P, c, k)
    H, th = gradient_field(img)
    F = consensus_filter(P, (8, 8), 7.0)
    R = consensus_radius(7.0)
    filt = decompose_sampled(F, 8, 0.25, 128)
    at = ext_conv_so2_at(H, filt, th, R, np.array(centres)).real
    np.testing.assert_allclose(at, at[0], rtol=1e-9)
    full = ext_conv_so2(H, filt, th, R).real
    top = np.argsort(full.ravel())[::-1][:4]
    got = sorted((int(i // 96), int(i % 96)) for i in top)
    assert got == sorted(centres), got
