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
