"""Pins of the proposal oracles: MLP gradients by finite differences, loss
antipodal invariance, the score upper bound, and refinement behaviour."""
import math

import numpy as np

import synth
from oracle import mlp
from oracle.so3 import (SHFilter, channel_layout, component_correlation_at, quat_mul, quat_exp, quat_to_matrix,
                        refine, score_from_channels, upper_bound)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(rng, 12, hidden=9)
    X = rng.standard_normal((7, 12))
    qt = rng.standard_normal((7, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    g = mlp.backward(p, mlp.forward(p, X), qt)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + 1e-6
            lp = mlp.loss(mlp.forward(p, X)["o"], qt)
            flat[idx] = old - 1e-6
            lm = mlp.loss(mlp.forward(p, X)["o"], qt)
            flat[idx] = old
            fd = (lp - lm) / 2e-6
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 + 1e-5 * abs(fd), (name, idx)


def test_loss_is_antipodally_invariant():
    rng = np.random.default_rng(1)
    o = rng.standard_normal((5, 4))
    qt = rng.standard_normal((5, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    assert abs(mlp.loss(o, qt) - mlp.loss(o, -qt)) < 1e-15
    assert mlp.loss(qt * 3.0, qt) < 1e-15


def _template_channels(L=3, seed=2, rot=None):
    prob = synth.so3_match_problem(seed=seed, size=24, n_plant=1, L=L, radius=4, dr=0.25, noise_sigma=0.0)
    F = SHFilter(prob["tables"], prob["dr"])
    c = prob["centres"][0]
    lay, n = channel_layout(L)
    chan = np.zeros(n)
    for (l, a, b, ch) in lay:
        g = component_correlation_at(prob["V"], F, l, a, b, prob["radius"], c[None])[0]
        chan[ch] = g.real
        if not (a == 0 and b == 0):
            chan[ch + 1] = g.imag
    return chan, prob["quats"][0]


def test_upper_bound_dominates_every_rotation():
    chan, _ = _template_channels()
    ub = upper_bound(chan, 3)
    rng = np.random.default_rng(3)
    for _ in range(40):
        R = quat_to_matrix(synth.haar_quaternion(rng))
        assert abs(score_from_channels(chan, 3, R)) <= ub * (1 + 1e-12)


def test_refinement_is_monotone_and_approaches_the_planted_rotation():
    chan, qtrue = _template_channels()
    rng = np.random.default_rng(4)
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    q0 = quat_mul(qtrue, quat_exp(0.3 * axis))          # 0.3 rad away
    s0 = score_from_channels(chan, 3, quat_to_matrix(q0))
    q1, s1 = refine(chan, 3, q0)
    assert s1 >= s0

    def ang(a, b):
        return 2 * math.acos(min(1.0, abs(float(np.dot(a, b)))))
    assert ang(q1, qtrue) < ang(q0, qtrue)
