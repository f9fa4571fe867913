"""Pins of the proposal oracles: MLP gradients by finite differences, loss
antipodal invariance, the score upper bound, and refinement behaviour."""
import math

import numpy as np
import pytest

import synth
from oracle import mlp
from oracle.so3 import (SHFilter, channel_layout, component_correlation_at, quat_mul, quat_exp, quat_to_matrix,
                        refine, score_from_channels, upper_bound)


def test_mlp_forward_literal_values():
    """A 3 -> 2 -> 2 -> 4 network with small exact weights, worked by hand:
    sample 1 keeps unit 1 of layer 1 and both units of layer 2 on; sample 2
    switches off both layer-1 units and unit 1 of layer 2, so the output is
    biases alone through W3.
      x1 = (2, 1, -2):  z1 = (0.5, -1),  h1 = (0.5, 0),  z2 = (0.5, 0.5),
                        o = (0.5, 1, 1, -0.5),  |o|^2 = 2.5
      x2 = (-2, 0, 1):  z1 = (-1, -6),   h1 = (0, 0),    z2 = (-0.5, 1),
                        o = (0, 2, 2, -3),      |o|^2 = 17
    Loss against q*1 = (1, 0, 0, 0), q*2 = (0, 0, 0, 1): 1 - 0.25/2.5 = 0.9
    and 1 - 9/17 = 8/17, mean (0.9 + 8/17) / 2."""
    p = dict(W1=np.array([[1.0, -1.0, 0.5], [0.0, 2.0, -1.0]]), b1=np.array([0.5, -5.0]),
             W2=np.array([[2.0, 1.0], [-1.0, 3.0]]), b2=np.array([-0.5, 1.0]),
             W3=np.array([[1.0, 0.0], [0.0, 2.0], [-1.0, 1.0], [3.0, -2.0]]), b3=np.array([0.0, 0.0, 1.0, -1.0]))
    X = np.array([[2.0, 1.0, -2.0], [-2.0, 0.0, 1.0]])
    c = mlp.forward(p, X)
    np.testing.assert_array_equal(c["z1"], [[0.5, -1.0], [-1.0, -6.0]])
    np.testing.assert_array_equal(c["h1"], [[0.5, 0.0], [0.0, 0.0]])
    np.testing.assert_array_equal(c["z2"], [[0.5, 0.5], [-0.5, 1.0]])
    np.testing.assert_array_equal(c["h2"], [[0.5, 0.5], [0.0, 1.0]])
    np.testing.assert_array_equal(c["o"], [[0.5, 1.0, 1.0, -0.5], [0.0, 2.0, 2.0, -3.0]])
    q = mlp.quaternion(c["o"])
    np.testing.assert_allclose(q[0], np.array([0.5, 1.0, 1.0, -0.5]) / np.sqrt(2.5), rtol=0, atol=1e-15)
    np.testing.assert_allclose(q[1], np.array([0.0, 2.0, 2.0, -3.0]) / np.sqrt(17.0), rtol=0, atol=1e-15)
    qt = np.array([[1.0, 0, 0, 0], [0, 0, 0, 1.0]])
    assert abs(mlp.loss(c["o"], qt) - (0.9 + 8.0 / 17.0) / 2) < 1e-15


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


def test_adam_first_step_is_signed_learning_rate():
    """Algorithm 1 of Kingma & Ba: after bias correction the first step is
    -lr * g / (|g| + eps), i.e. -lr * sign(g) for |g| >> eps; without the
    corrections it would be lr * 0.1 / sqrt(0.001) = 3.16 lr."""
    rng = np.random.default_rng(5)
    p = {"W": rng.standard_normal((3, 4)), "b": rng.standard_normal(4)}
    g = {"W": rng.standard_normal((3, 4)), "b": np.array([0.5, -2.0, 1e-3, 0.0])}
    st = {}
    out = mlp.adam_step(p, g, st, lr=0.01)
    np.testing.assert_allclose(out["W"] - p["W"], -0.01 * np.sign(g["W"]), rtol=1e-6)
    np.testing.assert_allclose(out["b"][:3] - p["b"][:3], -0.01 * np.sign(g["b"][:3]), rtol=1e-4)
    assert out["b"][3] == p["b"][3]                      # zero gradient: no move
    assert st["t"] == 1


def test_adam_minimises_a_quadratic():
    p = {"w": np.array([0.0, 10.0])}
    st = {}
    for _ in range(3000):
        g = {"w": 2.0 * (p["w"] - np.array([3.0, -1.0]))}
        p = mlp.adam_step(p, g, st, lr=0.02)
    np.testing.assert_allclose(p["w"], [3.0, -1.0], atol=1e-2)


def test_nuclear_bound_dominates_and_is_tight_for_a_pure_rotation():
    """|S(R)| <= sum_l |G_l|_* <= upper_bound; if G_l = C^l(R0) for every l
    the bound is reached at R0 (S(R0) = sum_l tr(C^H C) = sum_l (2l+1))."""
    from oracle.so3 import nuclear_bound, wigner_by_projection
    chan, _ = _template_channels()
    nb, ub = nuclear_bound(chan, 3), upper_bound(chan, 3)
    assert nb <= ub * (1 + 1e-12)
    rng = np.random.default_rng(6)
    for _ in range(20):
        R = quat_to_matrix(synth.haar_quaternion(rng))
        assert abs(score_from_channels(chan, 3, R)) <= nb * (1 + 1e-12)
    R0 = quat_to_matrix(synth.haar_quaternion(rng))
    lay, n = channel_layout(3)
    pure = np.zeros(n)
    for (l, a, b, ch) in lay:
        c = wigner_by_projection(l, R0)[a + l, b + l]
        pure[ch] = c.real
        if not (a == 0 and b == 0):
            pure[ch + 1] = c.imag
    assert abs(nuclear_bound(pure, 3) - 16.0) < 1e-9
    assert abs(score_from_channels(pure, 3, R0) - 16.0) < 1e-9
    assert upper_bound(pure, 3) == pytest.approx(16.0)
