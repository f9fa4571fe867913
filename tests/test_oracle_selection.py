"""Pins of the fixed-budget component selection oracle (Sec. 5 "Band-Limiting
Revisited"): the rotation-averaged error of steering with a subset equals
the dropped lattice energy (orthogonality over the rotation angle), and
keeping the largest energies beats every other subset of the same size.
CPU only."""
import numpy as np

import synth
from oracle.filters_so2 import AnalyticGaussPow, decompose_sampled
from oracle.selection import (component_energy, select_components, steered_error_sq,
                              sweep_subset_from_components)
from oracle.so2 import component_correlation, sweep_from_components


def _filters():
    rng = np.random.default_rng(12)
    a = synth.random_gauss_pow_coeffs(12, 6)
    yield AnalyticGaussPow(a, 2.5), 6, 7
    tpl = synth.smooth_random_template(rng, 9, 1.5)
    yield decompose_sampled(tpl, 8, 0.25, 128), 8, 9


def test_rotation_averaged_error_equals_the_dropped_energy():
    for filt, K, R in _filters():
        E = component_energy(filt, K, R)
        for ks in ([0], [0, 1], [0, 2, 5], list(range(K + 1)), select_components(E, 3)):
            dropped = sum(2 * E[k] for k in range(1, K + 1) if k not in ks)
            got = steered_error_sq(filt, K, R, ks, 2 * K + 3)
            assert abs(got - dropped) <= 1e-10 * max(1.0, E.sum()), (ks, got, dropped)


def test_energy_selection_is_optimal_for_its_budget():
    rng = np.random.default_rng(3)
    for filt, K, R in _filters():
        E = component_energy(filt, K, R)
        for budget in (2, 3, 5):
            best = select_components(E, budget)
            assert best[0] == 0 and len(best) == budget
            err = steered_error_sq(filt, K, R, best, 2 * K + 3)
            lowest = list(range(budget))
            assert err <= steered_error_sq(filt, K, R, lowest, 2 * K + 3) + 1e-12
            for _ in range(10):
                other = [0] + sorted(rng.choice(np.arange(1, K + 1), budget - 1, replace=False).tolist())
                assert err <= steered_error_sq(filt, K, R, other, 2 * K + 3) + 1e-12


def test_subset_sweep_limits():
    """The full list gives the full sweep; the list [0] gives the constant G_0."""
    rng = np.random.default_rng(4)
    H = rng.standard_normal((12, 14))
    filt, K, R = next(_filters())
    G = [component_correlation(H, filt, k, R) for k in range(K + 1)]
    J = 12
    np.testing.assert_allclose(sweep_subset_from_components(G, list(range(K + 1)), J),
                               sweep_from_components(G, K, J).real, atol=1e-12)
    S0 = sweep_subset_from_components(G, [0], J)
    np.testing.assert_allclose(S0, np.broadcast_to(G[0].real, S0.shape), atol=1e-12)


def test_rotate_pattern_quarter_turn_and_identity():
    """Rotating the sampled pattern by 0 returns it and by a quarter turn is
    the exact lattice rotation d -> R(-pi/2) d (spline interpolation is exact
    at lattice points); the rotated copy of a pattern sampled from an
    analytic band-limited filter matches that filter's rotation."""
    from oracle.selection import rotate_pattern
    rng = np.random.default_rng(3)
    P = synth.smooth_random_template(rng, 10, 2.0)
    np.testing.assert_allclose(rotate_pattern(P, 0.0), P, atol=1e-12)
    q = rotate_pattern(P, np.pi / 2)
    R = 10
    for dy in range(-R, R + 1, 3):
        for dx in range(-R, R + 1, 4):
            # R(-pi/2) (dx, dy) = (dy, -dx)
            assert abs(q[dy + R, dx + R] - P[-dx + R, dy + R]) < 1e-9


def test_rotated_copies_sweep_matches_direct_correlation():
    """B = 1 is the plain correlation with the pattern (brute force), and
    with B = 4 the maximum is over the four exact quarter turns."""
    from oracle.selection import rotate_pattern, rotated_copies_sweep
    rng = np.random.default_rng(4)
    P = synth.smooth_random_template(rng, 4, 1.0)
    H = rng.standard_normal((14, 12))
    R = 4
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]

    def corr(f):
        out = np.zeros_like(H)
        for a, b, v in zip(dy.ravel(), dx.ravel(), f.ravel()):
            out += np.roll(H, (-a, -b), axis=(0, 1)) * v
        return out
    best1, arg1 = rotated_copies_sweep(H, P, 1)
    np.testing.assert_allclose(best1, corr(P), atol=1e-10)
    assert np.all(arg1 == 0)
    best4, arg4 = rotated_copies_sweep(H, P, 4)
    ref = np.stack([corr(rotate_pattern(P, np.pi * j / 2)) for j in range(4)])
    np.testing.assert_allclose(best4, ref.max(axis=0), atol=1e-10)
    np.testing.assert_array_equal(arg4, ref.argmax(axis=0))
    quarter = np.stack([corr(np.rot90(P, j)) for j in range(4)])
    np.testing.assert_allclose(np.sort(ref, axis=0), np.sort(quarter, axis=0), atol=1e-9)
