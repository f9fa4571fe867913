"""Pins of the FP64 oracle of the SO(3) extended convolution (Eq. Def-EConv
with a rotation at every input voxel; the component form of Sec. 9): the
identity and constant fields reduce to library FFT convolution with the
(analytically rotated) filter, the impulse response is the filter rotated by
the field at the impulse (Sec. 2.3), the operator is the adjoint of the
extended correlation with the same field, exact 90-degree lattice
equivariance, and the component form equals the brute force.  CPU only."""
import math

import numpy as np

import synth
from oracle.so3 import (SHFilter, box_offsets3, conv_so3, conv_so3_at, conv_so3_from_components, corr_so3_at,
                        filter_eval, quat_field_matrices, quat_mul, quat_to_matrix, rotated_filter_eval)


def small_filter(seed=1, L=2, radius=3.0, dr=0.25):
    return SHFilter(synth.so3_filter_tables(seed, L, radius, dr), dr)


def fft_conv(V, kernel_vals, radius):
    """Periodic convolution of V with box samples kernel_vals[d] by numpy's FFT."""
    dx, dy, dz = box_offsets3(radius)
    g = np.zeros(V.shape, np.complex128)
    np.add.at(g, (dz % V.shape[0], dy % V.shape[1], dx % V.shape[2]), kernel_vals)
    return np.fft.ifftn(np.fft.fftn(V) * np.fft.fftn(g))


def test_identity_field_is_ordinary_convolution():
    rng = np.random.default_rng(1)
    F = small_filter()
    V = rng.standard_normal((6, 7, 8))
    Q = np.zeros(V.shape + (4,))
    Q[..., 0] = 1.0
    dx, dy, dz = box_offsets3(2)
    ref = fft_conv(V, filter_eval(F, dx, dy, dz), 2)
    np.testing.assert_allclose(conv_so3(V, F, 2, Q), ref, atol=1e-12)


def test_constant_field_is_convolution_with_the_rotated_filter():
    rng = np.random.default_rng(2)
    F = small_filter(seed=2)
    V = rng.standard_normal((7, 6, 6))
    q = synth.haar_quaternion(rng)
    Q = np.broadcast_to(q, V.shape + (4,))
    dx, dy, dz = box_offsets3(3)
    ref = fft_conv(V, rotated_filter_eval(F, quat_to_matrix(q), dx.astype(float), dy.astype(float),
                                          dz.astype(float)), 3)
    np.testing.assert_allclose(conv_so3(V, F, 3, Q), ref, atol=1e-12)


def test_impulse_response_is_the_filter_rotated_at_the_impulse():
    """Convolving delta_q0 gives T_{R(q0)} F centred at q0, whatever the field
    elsewhere (the scatter form's delta response, Sec. 2.3)."""
    rng = np.random.default_rng(3)
    F = small_filter(seed=3)
    shape = (9, 9, 9)
    V = np.zeros(shape)
    q0 = (4, 3, 5)
    V[q0] = 1.0
    Q = rng.standard_normal(shape + (4,))
    out = conv_so3(V, F, 3, Q)
    dx, dy, dz = box_offsets3(3)
    Rm = quat_to_matrix(Q[q0])
    expect = np.zeros(shape, np.complex128)
    expect[(q0[0] + dz) % 9, (q0[1] + dy) % 9, (q0[2] + dx) % 9] = rotated_filter_eval(
        F, Rm, dx.astype(float), dy.astype(float), dz.astype(float))
    np.testing.assert_allclose(out, expect, atol=1e-12)


def test_convolution_is_the_adjoint_of_the_extended_correlation():
    """sum_p O_H(p) W(p) = sum_q H(q) S_W(q, R(q)), S the extended correlation
    of W with the same rotation field (gather form)."""
    rng = np.random.default_rng(4)
    F = small_filter(seed=4)
    shape = (6, 5, 6)
    H, W = rng.standard_normal(shape), rng.standard_normal(shape)
    Q = rng.standard_normal(shape + (4,))
    lhs = np.sum(conv_so3(H, F, 2, Q) * W)
    Rms = quat_field_matrices(Q)
    rhs = 0.0
    for idx in np.ndindex(shape):
        rhs += H[idx] * np.conj(corr_so3_at(W, F, 2, [Rms[idx]], [idx])[0, 0])
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))
    assert abs(lhs.imag) <= 1e-12


def test_lattice_quarter_turn_equivariance():
    """V'(x) = V(Q^-1 x), R'(x) = Q R(Q^-1 x) for the quarter turn Q about z
    give O'(x) = O(Q^-1 x) exactly (cubic periodic volume)."""
    rng = np.random.default_rng(5)
    F = small_filter(seed=5)
    n = 6
    V = rng.standard_normal((n, n, n))
    Qf = rng.standard_normal((n, n, n, 4))
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    src = (zz, (-xx) % n, yy)                 # Q^-1 (x, y, z) = (y, -x, z)
    qz = np.array([math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)])
    assert np.allclose(quat_to_matrix(qz) @ [1, 0, 0], [0, 1, 0])
    V2 = V[src]
    Q2 = np.stack([quat_mul(qz, q) for q in Qf[src].reshape(-1, 4)]).reshape(Qf.shape)
    out = conv_so3(V, F, 2, Qf)
    np.testing.assert_allclose(conv_so3(V2, F, 2, Q2), out[src], atol=1e-12)


def test_component_form_equals_the_brute_force():
    rng = np.random.default_rng(6)
    for L, radius, shape in ((3, 2, (5, 6, 7)), (1, 4, (4, 4, 6))):   # the second box wraps the volume
        F = small_filter(seed=6 + L, L=L, radius=radius + 0.5)
        V = rng.standard_normal(shape)
        Q = rng.standard_normal(shape + (4,))
        brute = conv_so3(V, F, radius, Q)
        np.testing.assert_allclose(conv_so3_from_components(V, F, radius, Q), brute, atol=1e-11)
        assert np.abs(brute.imag).max() <= 1e-12      # a real filter gives a real output
        vox = [(0, 0, 0), (shape[0] - 1, 2, 3)]
        np.testing.assert_allclose(conv_so3_at(V, F, radius, Q, vox), brute[tuple(np.array(vox).T)], atol=1e-13)
