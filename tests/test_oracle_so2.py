"""Pins of the SO(2) FP64 oracle against facts fixed by the paper and by
mathematics (closed forms, library special cases, lattice symmetries, the
paper's worked examples).  CPU only."""
import math
import pathlib

import numpy as np
import pytest

from oracle.filters_so2 import (AnalyticGaussPow, RadialTable, decompose_sampled,
                                filter_eval, rotated_filter_eval)
from oracle.so2 import (box_offsets, ext_conv_so2, ext_conv_so2_at, ext_corr_so2,
                        ext_corr_so2_at, sweep_so2_at, sweep_so2_fft)
import synth

GOLDEN = pathlib.Path(__file__).with_name("golden")


# ---------------------------------------------------------------- helpers ---

def cartesian_gauss_pow(a, sigma, x, y):
    """Same analytic filter written without angles: r^|k| e^{ik theta} equals
    (x + i y)^k for k >= 0 and (x - i y)^|k| for k < 0."""
    K = (len(a) - 1) // 2
    z = np.asarray(x, np.float64) + 1j * np.asarray(y, np.float64)
    g = np.exp(-(np.abs(z) ** 2) / (2 * sigma ** 2))
    out = np.zeros(z.shape, np.complex128)
    for k in range(-K, K + 1):
        zz = z ** k if k >= 0 else np.conj(z) ** (-k)
        out += a[k + K] * zz * g
    return out


def filter_grid(values, dx, dy, h, w):
    g = np.zeros((h, w), np.complex128)
    np.add.at(g, (dy % h, dx % w), values)
    return g


def fft_corr(H, g):
    return np.fft.ifft2(np.fft.fft2(H) * np.conj(np.fft.fft2(g)))


def fft_conv(H, g):
    return np.fft.ifft2(np.fft.fft2(H) * np.fft.fft2(g))


def small_problem(seed=7, h=18, w=22, K=3, sigma=2.0):
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((h, w))
    a = synth.random_gauss_pow_coeffs(seed + 1, K)
    alpha = rng.uniform(0, 2 * math.pi, (h, w))
    return H, AnalyticGaussPow(a, sigma), a, alpha


# ------------------------------------------------------------- filter model ---

def test_polar_eval_matches_cartesian_closed_form():
    a = synth.random_gauss_pow_coeffs(3, 5)
    f = AnalyticGaussPow(a, 3.0)
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-9, 9, (2, 500))
    x[:3] = [0.0, 2.0, 0.0]
    y[:3] = [0.0, 0.0, -3.0]
    np.testing.assert_allclose(filter_eval(f, x, y), cartesian_gauss_pow(a, 3.0, x, y),
                               rtol=1e-12, atol=1e-12)
    # Hermitian coefficients -> real filter
    assert np.max(np.abs(filter_eval(f, x, y).imag)) < 1e-12


def _paper_matrices():
    rows = {}
    for line in (GOLDEN / "paper_tmatrix.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        vals = np.array([float(v) for v in parts[2:]])
        m = (vals[0::2] + 1j * vals[1::2]).reshape(3, 3)
        rows.setdefault(parts[0], []).append((float(parts[1]), m))
    return rows


class _AngularBasisFilter:
    """Filter sum_k c_k exp(-r^2/2) e^{ik theta} for the paper's worked-example bases."""

    def __init__(self, ck):
        self.c = np.asarray(ck, np.complex128)
        self.K = (len(self.c) - 1) // 2

    def radial(self, k, r):
        return self.c[k + self.K] * np.exp(-np.asarray(r) ** 2 / 2)


def _basis_harmonics(name):
    # each basis function as harmonic coefficients for k = -2..2 (index k + 2)
    if name == "diag":   # e^{2i th}, e^{-2i th}, 1  (Sec. 3, Example n = 3)
        return [np.array([0, 0, 0, 0, 1]), np.array([1, 0, 0, 0, 0]), np.array([0, 0, 1, 0, 0])]
    # cos^2, sin^2, cos sin  (Sec. 3, Example n = 3 revisited)
    return [np.array([0.25, 0, 0.5, 0, 0.25]), np.array([-0.25, 0, 0.5, 0, -0.25]),
            np.array([0.25j, 0, 0, 0, -0.25j])]


def test_basis_harmonic_expansions():
    th = np.linspace(0, 2 * np.pi, 17)
    expect = [np.cos(th) ** 2, np.sin(th) ** 2, np.cos(th) * np.sin(th)]
    for vec, e in zip(_basis_harmonics("cossin"), expect):
        got = sum(vec[k + 2] * np.exp(1j * k * th) for k in range(-2, 3))
        np.testing.assert_allclose(got, e, atol=1e-14)


@pytest.mark.parametrize("name", ["diag", "cossin"])
def test_rotation_action_matches_paper_worked_example(name):
    """Rotating F = sum_i a_i F_i by Theta equals sum_i (T(Theta) a)_i F_i with
    the matrices printed in Sec. 3 (fixture tests/golden/paper_tmatrix.txt)."""
    basis = _basis_harmonics(name)
    rng = np.random.default_rng(11)
    a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    x, y = rng.uniform(-3, 3, (2, 200))
    for theta, T in _paper_matrices()[name]:
        filt = _AngularBasisFilter(sum(ai * b for ai, b in zip(a, basis)))
        rotated = rotated_filter_eval(filt, x, y, theta)
        b = T @ a
        expect = filter_eval(_AngularBasisFilter(sum(bi * v for bi, v in zip(b, basis))), x, y)
        np.testing.assert_allclose(rotated, expect, atol=1e-12)


def test_radial_table_hermite_properties():
    dr = 0.5
    r_nodes = np.arange(12) * dr
    # even quadratic for k = 0, odd linear for k = 1, zero elsewhere
    fk = np.zeros((3, 12), np.complex128)
    fk[1] = 2.0 - 0.3 * r_nodes ** 2
    fk[2] = 1.5 * r_nodes
    fk[0] = np.conj(fk[2]) * -1
    t = RadialTable(fk, dr)
    np.testing.assert_allclose(t.radial(0, r_nodes), fk[1], atol=1e-14)
    r = np.linspace(0, r_nodes[-2], 301)   # last interval sees v_n = 0
    np.testing.assert_allclose(t.radial(0, r), 2.0 - 0.3 * r ** 2, atol=1e-12)
    np.testing.assert_allclose(t.radial(1, r), 1.5 * r, atol=1e-12)
    assert np.all(t.radial(0, np.array([r_nodes[-1] + 1e-9, 100.0])) == 0)


# ------------------------------------------------------- filter decomposition ---

def test_decomposition_recovers_band_limited_filter():
    """A sampled image of an exactly band-limited filter decomposes back into
    its own harmonics, up to bicubic resampling error (about 0.1% here) and
    lattice aliasing into k +- 4; a flipped sign (k <-> -k), a dropped 1/n
    or a shifted angle origin would be off by O(1)."""
    a = synth.random_gauss_pow_coeffs(5, 3)
    R, sigma = 16, 4.0
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    img = cartesian_gauss_pow(a, sigma, dx, dy).real
    tab = decompose_sampled(img, K=5, dr=0.25, n_theta=64)
    r = np.arange(tab.n) * 0.25
    ref = AnalyticGaussPow(a, sigma)
    scale = max(np.max(np.abs(ref.radial(k, r))) for k in range(-3, 4))
    m = r <= 11
    for k in range(-5, 6):
        expect = np.asarray(ref.radial(k, r) if abs(k) <= 3 else 0 * r)
        err = np.max(np.abs(tab.fk[k + 5][m] - expect[m]))
        assert err <= 2.5e-3 * scale, (k, err, scale)


def test_decomposition_lattice_symmetry():
    rng = np.random.default_rng(1)
    img = synth.smooth_random_template(rng, 10, 2.0)
    tab = decompose_sampled(img, K=8, dr=0.5, n_theta=64)
    # rot by +90 deg: T'(x) = T(R(-pi/2) x) -> f'_k = f_k e^{-ik pi/2}
    rot = np.empty_like(img)
    R = 10
    for iy in range(2 * R + 1):
        for ix in range(2 * R + 1):
            x, y = ix - R, iy - R
            rot[iy, ix] = img[-x + R, y + R]   # T(R(-pi/2)(x, y)) = T(y, -x)
    tab2 = decompose_sampled(rot, K=8, dr=0.5, n_theta=64)
    k = np.arange(-8, 9)[:, None]
    np.testing.assert_allclose(tab2.fk, tab.fk * np.exp(-1j * k * np.pi / 2), atol=1e-12)
    # an image with the 4-fold lattice symmetry has only k = 0 mod 4
    iso = img + np.rot90(img) + np.rot90(img, 2) + np.rot90(img, 3)
    t3 = decompose_sampled(iso, K=8, dr=0.5, n_theta=64)
    for kk in range(-8, 9):
        if kk % 4:
            assert np.max(np.abs(t3.fk[kk + 8])) < 1e-12


# ---------------------------------------------------------------- operators ---

def test_corr_alpha_zero_is_fft_correlation():
    H, filt, a, _ = small_problem()
    R = 4
    dx, dy = box_offsets(R)
    g = filter_grid(cartesian_gauss_pow(a, 2.0, dx, dy), dx, dy, *H.shape)
    got = ext_corr_so2(H, filt, np.zeros_like(H), R)
    np.testing.assert_allclose(got, fft_corr(H, g), atol=1e-11)


def test_conv_alpha_zero_is_fft_convolution():
    H, filt, a, _ = small_problem(seed=9)
    R = 4
    dx, dy = box_offsets(R)
    g = filter_grid(cartesian_gauss_pow(a, 2.0, dx, dy), dx, dy, *H.shape)
    got = ext_conv_so2(H, filt, np.zeros_like(H), R)
    np.testing.assert_allclose(got, fft_conv(H, g), atol=1e-11)


def test_box_larger_than_image_wraps_and_accumulates():
    H, filt, a, _ = small_problem(seed=3, h=5, w=6)
    R = 4                      # 9x9 box on a 5x6 torus
    dx, dy = box_offsets(R)
    g = filter_grid(cartesian_gauss_pow(a, 2.0, dx, dy), dx, dy, *H.shape)
    np.testing.assert_allclose(ext_corr_so2(H, filt, np.zeros_like(H), R), fft_corr(H, g),
                               atol=1e-11)
    np.testing.assert_allclose(ext_conv_so2(H, filt, np.zeros_like(H), R), fft_conv(H, g),
                               atol=1e-11)


@pytest.mark.parametrize("c", [0.3, 2.0, -1.2])
def test_constant_field_is_analytically_rotated_filter(c):
    """alpha == c: T(c) multiplies a_k by e^{-ikc} (Sec. 3 Example n = 1)."""
    H, filt, a, _ = small_problem(seed=5)
    R = 4
    K = (len(a) - 1) // 2
    a_rot = a * np.exp(-1j * np.arange(-K, K + 1) * c)
    dx, dy = box_offsets(R)
    g = filter_grid(cartesian_gauss_pow(a_rot, 2.0, dx, dy), dx, dy, *H.shape)
    alpha = np.full(H.shape, c)
    np.testing.assert_allclose(ext_corr_so2(H, filt, alpha, R), fft_corr(H, g), atol=1e-10)
    np.testing.assert_allclose(ext_conv_so2(H, filt, alpha, R), fft_conv(H, g), atol=1e-10)


def _rot90_problem(H, alpha):
    """H'(p) = H(Q^-1 p), alpha'(p) = alpha(Q^-1 p) + pi/2, Q = +90 deg:
    Q^-1 (x, y) = (y, -x) on the n x n torus."""
    n = H.shape[0]
    y, x = np.mgrid[0:n, 0:n]
    sy, sx = (-x) % n, y          # Q^-1 p = (x', y') = (y, -x)
    return H[sy, sx], alpha[sy, sx] + np.pi / 2, (sy, sx)


def test_corr_and_conv_exact_90_degree_equivariance():
    H, filt, a, alpha = small_problem(seed=21, h=16, w=16)
    R = 3
    H2, alpha2, idx = _rot90_problem(H, alpha)
    out = ext_corr_so2(H, filt, alpha, R)
    out2 = ext_corr_so2(H2, filt, alpha2, R)
    np.testing.assert_allclose(out2, out[idx], atol=1e-10)
    outc = ext_conv_so2(H, filt, alpha, R)
    outc2 = ext_conv_so2(H2, filt, alpha2, R)
    np.testing.assert_allclose(outc2, outc[idx], atol=1e-10)


def test_conv_impulse_response_is_transformed_filter():
    """Sec. 2.3: the response of extended convolution to a delta at q0 is the
    filter transformed by T(q0), translated to q0."""
    h = w = 20
    a = synth.random_gauss_pow_coeffs(2, 4)
    filt = AnalyticGaussPow(a, 2.0)
    rng = np.random.default_rng(4)
    alpha = rng.uniform(0, 2 * np.pi, (h, w))
    q0 = (7, 12)
    H = np.zeros((h, w))
    H[q0] = 1.0
    R = 5
    out = ext_conv_so2(H, filt, alpha, R)
    c = alpha[q0]
    K = 4
    a_rot = a * np.exp(-1j * np.arange(-K, K + 1) * c)
    expect = np.zeros((h, w), np.complex128)
    dx, dy = box_offsets(R)
    expect[(q0[0] + dy) % h, (q0[1] + dx) % w] = cartesian_gauss_pow(a_rot, 2.0, dx, dy)
    np.testing.assert_allclose(out, expect, atol=1e-12)


def test_sampled_pixel_forms_match_full_image():
    H, filt, a, alpha = small_problem(seed=13, h=15, w=17)
    R = 3
    pix = np.array([[0, 0], [14, 16], [7, 3], [2, 11]])
    full = ext_corr_so2(H, filt, alpha, R)
    np.testing.assert_allclose(ext_corr_so2_at(H, filt, alpha, R, pix), full[pix[:, 0], pix[:, 1]],
                               atol=1e-11)
    fullc = ext_conv_so2(H, filt, alpha, R)
    np.testing.assert_allclose(ext_conv_so2_at(H, filt, alpha, R, pix),
                               fullc[pix[:, 0], pix[:, 1]], atol=1e-11)


# -------------------------------------------------------------------- sweep ---

def test_sweep_fixed_angle_is_field_correlation():
    H, filt, a, _ = small_problem(seed=17, h=14, w=14)
    R, J = 3, 8
    pix = np.array([[y, x] for y in range(14) for x in range(14)])
    S = sweep_so2_at(H, filt, R, J, pix)
    for j in (0, 3, 5):
        corr = ext_corr_so2(H, filt, np.full(H.shape, 2 * np.pi * j / J), R)
        np.testing.assert_allclose(S[:, j], corr.ravel(), atol=1e-10)
    best, arg, _ = sweep_so2_fft(H, filt, R, J)
    np.testing.assert_allclose(best.ravel(), S.real.max(axis=1), atol=1e-10)


def test_sweep_rot90_shifts_argmax_by_quarter_turn():
    H, filt, a, _ = small_problem(seed=23, h=16, w=16)
    R, J = 3, 12
    H2, _, idx = _rot90_problem(H, np.zeros_like(H))
    b1, a1, s1 = sweep_so2_fft(H, filt, R, J)
    b2, a2, s2 = sweep_so2_fft(H2, filt, R, J)
    np.testing.assert_allclose(b2, b1[idx], atol=1e-10)
    clear = (b1 - s1)[idx] > 1e-9
    assert np.all((a2[clear] - a1[idx][clear]) % J == J // 4)


def test_sweep_detects_planted_templates():
    prob = synth.so2_match_problem(seed=99, size=160, n_plant=3, radius=12, K=8, J=32)
    tab = decompose_sampled(prob["template"], prob["K"], prob["dr"], prob["n_theta"])
    best, arg, _ = sweep_so2_fft(prob["H"], tab, prob["radius"], prob["J"])
    J = prob["J"]
    for (cy, cx), beta in zip(prob["centres"], prob["betas"]):
        win = best[cy - 2:cy + 3, cx - 2:cx + 3]
        iy, ix = np.unravel_index(np.argmax(win), win.shape)
        assert abs(iy - 2) <= 1 and abs(ix - 2) <= 1
        j_true = round(beta * J / (2 * np.pi)) % J
        dj = (arg[cy, cx] - j_true) % J
        assert min(dj, J - dj) <= 1


def test_component_steering_matches_bruteforce_sweep():
    """The Sec. 4.1 algorithm (components, then linear combination) reproduces
    the definition evaluated with explicitly rotated filters -- pins
    component_correlation and sweep_from_components against the brute force."""
    from oracle.so2 import component_correlation, sweep_from_components
    H, filt, a, _ = small_problem(seed=31, h=12, w=14, K=3)
    R, J = 3, 10
    G = [component_correlation(H, filt, k, R) for k in range(0, 4)]
    S = sweep_from_components(G, 3, J)
    pix = np.array([[y, x] for y in range(12) for x in range(14)])
    ref = sweep_so2_at(H, filt, R, J, pix)
    np.testing.assert_allclose(S.reshape(J, -1).T, ref, atol=1e-10)
    # and the components alone are standard correlations with F_k (FFT)
    dx, dy = box_offsets(R)
    for k in range(4):
        comp = AnalyticGaussPow(np.where(np.arange(-3, 4) == k, a, 0), 2.0)
        g = filter_grid(cartesian_gauss_pow(comp.a, 2.0, dx, dy), dx, dy, 12, 14)
        np.testing.assert_allclose(G[k], fft_corr(H, g), atol=1e-10)


def test_fft_sweep_route_matches_bruteforce_on_sampled_template():
    """The two oracle routes to the sweep (per-pixel brute force and FFT
    correlation per rotated filter) agree on a planted-template image."""
    prob = synth.so2_match_problem(seed=832, size=128, n_plant=3, radius=12, K=8, J=32)
    tab = decompose_sampled(prob["template"], 8, prob["dr"], prob["n_theta"])
    best, arg, _ = sweep_so2_fft(prob["H"], tab, prob["radius"], 32)
    pix = np.array([[y, x] for y in range(0, 128, 3) for x in range(0, 128, 5)] + [[127, 127]])
    S = sweep_so2_at(prob["H"], tab, prob["radius"], 32, pix).real
    np.testing.assert_allclose(best[pix[:, 0], pix[:, 1]], S.max(axis=1), atol=1e-12)


def test_fft_components_match_bruteforce_components():
    """component_correlation_fft (FFT route) equals the brute-force sum over
    the box, also with a box wider than the image (wrapped taps)."""
    from oracle.so2 import component_correlation, component_correlation_fft
    H, filt, a, _ = small_problem(seed=33, h=12, w=14, K=3)
    for R in (3, 9):
        for k in range(4):
            np.testing.assert_allclose(component_correlation_fft(H, filt, k, R), component_correlation(H, filt, k, R),
                                       atol=1e-11)


def test_steered_sweep_route_matches_bruteforce_and_fft_routes():
    """sweep_so2_steered (components by FFT, linear combination at every
    angle, max) agrees with the per-pixel brute force with rotated filters and
    with the per-rotated-filter FFT route, maxima and first argmax."""
    from oracle.so2 import sweep_so2_steered
    prob = synth.so2_match_problem(seed=834, size=96, n_plant=2, radius=12, K=6, J=24)
    tab = decompose_sampled(prob["template"], 6, prob["dr"], prob["n_theta"])
    best, arg = sweep_so2_steered(prob["H"], tab, 6, prob["radius"], 24, chunk=1000)
    b2, a2, second = sweep_so2_fft(prob["H"], tab, prob["radius"], 24)
    np.testing.assert_allclose(best, b2, atol=1e-12 * np.abs(b2).max())
    clear = (b2 - second) > 1e-9 * np.abs(b2).max()
    assert np.array_equal(arg[clear], a2[clear])
    pix = np.array([[y, x] for y in range(0, 96, 7) for x in range(0, 96, 5)])
    S = sweep_so2_at(prob["H"], tab, prob["radius"], 24, pix).real
    np.testing.assert_allclose(best[pix[:, 0], pix[:, 1]], S.max(axis=1), atol=1e-12 * np.abs(S).max())


def test_boundary_taps_are_rotation_invariant():
    """A lattice offset on the support circle |d| = (n-1) dr keeps its value
    under rotation, whatever the rounding of the rotated coordinate."""
    rng = np.random.default_rng(4)
    fk = rng.standard_normal((5, 49)) + 1j * rng.standard_normal((5, 49))
    fk[0] = np.conj(fk[4]); fk[1] = np.conj(fk[3]); fk[2] = fk[2].real
    tab = RadialTable(fk, 0.25)               # support r <= 12
    for (dx, dy) in [(0, -12), (12, 0), (0, 12), (-12, 0)]:
        base = tab.radial(1, 12.0)
        for a in np.linspace(0, 2 * np.pi, 97):
            c, s = np.cos(a), np.sin(a)
            r = np.hypot(c * dx + s * dy, -s * dx + c * dy)
            np.testing.assert_allclose(tab.radial(1, r), base, rtol=1e-9, atol=1e-12)
