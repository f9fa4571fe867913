"""Pins of the SO(3) FP64 oracle (Sec. 9): textbook spherical harmonics, the
defining property and group laws of the rotation matrices C^l(R), library
FFT correlation at R = I, exact octahedral lattice equivariance, and the
component/Wigner form against the brute-force definition.  CPU only."""
import math

import numpy as np
import pytest

import synth
from oracle.so3 import (SHFilter, box_offsets3, component_correlation, corr_so3_at, filter_eval, quat_to_matrix,
                        sph_harm, sweep_from_components, wigner_by_projection)


def rand_rot(rng):
    return quat_to_matrix(synth.haar_quaternion(rng))


def small_filter(seed=1, L=2, radius=3.0, dr=0.25):
    return SHFilter(synth.so3_filter_tables(seed, L, radius, dr), dr)


def test_spherical_harmonics_textbook_forms():
    rng = np.random.default_rng(0)
    th = rng.uniform(0, np.pi, 50)
    ph = rng.uniform(-np.pi, np.pi, 50)
    s, c = np.sin(th), np.cos(th)
    e = np.exp(1j * ph)
    pi = math.pi
    expect = {
        (0, 0): np.full_like(th, 0.5 / math.sqrt(pi)),
        (1, 0): math.sqrt(3 / (4 * pi)) * c,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s * e,
        (1, -1): math.sqrt(3 / (8 * pi)) * s / e,
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * c * c - 1),
        (2, 1): -math.sqrt(15 / (8 * pi)) * s * c * e,
        (2, 2): math.sqrt(15 / (32 * pi)) * s * s * e * e,
        (2, -2): math.sqrt(15 / (32 * pi)) * s * s / (e * e),
    }
    for (l, m), v in expect.items():
        np.testing.assert_allclose(sph_harm(l, m, th, ph), v, atol=1e-13)


def test_spherical_harmonics_orthonormal():
    from scipy.special import roots_legendre
    xs, ws = roots_legendre(16)
    th = np.arccos(xs)
    ph = 2 * np.pi * np.arange(33) / 33
    T, P = np.meshgrid(th, ph, indexing="ij")
    W = (ws[:, None] * (2 * np.pi / 33)) * np.ones_like(P)
    idx = [(l, m) for l in range(7) for m in range(-l, l + 1)]
    Ys = np.stack([sph_harm(l, m, T, P).ravel() for l, m in idx])
    gram = (Ys * W.ravel()) @ np.conj(Ys).T
    np.testing.assert_allclose(gram, np.eye(len(idx)), atol=1e-12)


def test_rotation_matrix_about_z_is_diagonal_phase():
    g = 0.7
    Rz = np.array([[math.cos(g), -math.sin(g), 0], [math.sin(g), math.cos(g), 0], [0, 0, 1]])
    for l in range(4):
        C = wigner_by_projection(l, Rz)
        np.testing.assert_allclose(C, np.diag(np.exp(-1j * np.arange(-l, l + 1) * g)), atol=1e-12)


@pytest.mark.parametrize("l", [1, 2, 4, 6])
def test_rotation_matrices_group_laws_and_definition(l):
    rng = np.random.default_rng(l)
    R1, R2 = rand_rot(rng), rand_rot(rng)
    C1, C2 = wigner_by_projection(l, R1), wigner_by_projection(l, R2)
    np.testing.assert_allclose(C1 @ np.conj(C1).T, np.eye(2 * l + 1), atol=1e-12)
    # T_{R1} T_{R2} = T_{R1 R2}  =>  C(R1 R2) = C(R2) C(R1)
    np.testing.assert_allclose(wigner_by_projection(l, R1 @ R2), C2 @ C1, atol=1e-12)
    # defining expansion at arbitrary (non-quadrature) points
    x = rng.standard_normal((3, 40))
    x /= np.linalg.norm(x, axis=0)
    xr = R1.T @ x
    r, th, ph = np.ones(40), np.arccos(x[2]), np.arctan2(x[1], x[0])
    thr, phr = np.arccos(np.clip(xr[2], -1, 1)), np.arctan2(xr[1], xr[0])
    for a in range(-l, l + 1):
        lhs = sph_harm(l, a, thr, phr)
        rhs = sum(C1[a + l, b + l] * sph_harm(l, b, th, ph) for b in range(-l, l + 1))
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_identity_rotation_is_fft_correlation():
    rng = np.random.default_rng(2)
    V = rng.standard_normal((8, 9, 10))
    F = small_filter()
    rad = 3
    dx, dy, dz = box_offsets3(rad)
    g = np.zeros(V.shape, np.complex128)
    np.add.at(g, (dz % 8, dy % 9, dx % 10), filter_eval(F, dx.astype(float), dy.astype(float), dz.astype(float)))
    ref = np.fft.ifftn(np.fft.fftn(V) * np.conj(np.fft.fftn(g)))
    vox = np.array([[z, y, x] for z in range(8) for y in range(9) for x in range(10)])
    S = corr_so3_at(V, F, rad, [np.eye(3)], vox)[:, 0]
    np.testing.assert_allclose(S, ref.ravel(), atol=1e-10)


def test_octahedral_lattice_equivariance():
    """V'(p) = V(Q^-1 p) for a lattice rotation Q  =>  S'(p, R) = S(Q^-1 p, Q^-1 R)."""
    rng = np.random.default_rng(3)
    n = 9
    V = rng.standard_normal((n, n, n))
    F = small_filter(seed=4)
    Q = np.array([[0, -1, 0], [0, 0, -1], [1, 0, 0]], np.float64)   # (x,y,z) -> (-y,-z,x)
    Qi = Q.T
    Qint = Qi.astype(np.int64)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    src = np.einsum("ij,j...->i...", Qint, np.stack([x, y, z])) % n   # Q^-1 p in (x, y, z)
    V2 = V[src[2], src[1], src[0]]
    vox = np.array([[1, 2, 3], [4, 0, 8], [7, 7, 1]])
    Rs = [rand_rot(rng) for _ in range(3)]
    S2 = corr_so3_at(V2, F, 3, Rs, vox)
    q = np.einsum("ij,nj->ni", Qint, vox[:, ::-1]) % n   # Q^-1 p as (x, y, z)
    S1 = corr_so3_at(V, F, 3, [Qi @ R for R in Rs], q[:, ::-1])
    np.testing.assert_allclose(S2, S1, atol=1e-10)


def test_component_form_matches_bruteforce():
    """Sec. 9: S(p, R) = sum_{l,a,b} conj(C^l_ab(R)) G_l^{ab}(p)."""
    rng = np.random.default_rng(5)
    V = rng.standard_normal((7, 8, 6))
    L, rad = 2, 2
    F = small_filter(seed=6, L=L, radius=2.0)
    G = [np.stack([np.stack([component_correlation(V, F, l, a, b, rad) for b in range(-l, l + 1)])
                   for a in range(-l, l + 1)]) for l in range(L + 1)]
    vox = np.array([[z, y, x] for z in range(7) for y in range(8) for x in range(6)])
    for _ in range(3):
        R = rand_rot(rng)
        Cs = [wigner_by_projection(l, R) for l in range(L + 1)]
        S = sweep_from_components(G, Cs).ravel()
        ref = corr_so3_at(V, F, rad, [R], vox)[:, 0]
        np.testing.assert_allclose(S, ref, atol=1e-10)
    # real filter and signal: the score is real
    assert np.max(np.abs(ref.imag)) < 1e-10


def test_planted_template_peaks_at_its_rotation():
    prob = synth.so3_match_problem(seed=11, size=24, n_plant=1, L=3, radius=4, dr=0.25)
    F = SHFilter(prob["tables"], prob["dr"])
    c = prob["centres"][0]
    Rtrue = quat_to_matrix(prob["quats"][0])
    rng = np.random.default_rng(0)
    Rs = [Rtrue] + [rand_rot(rng) for _ in range(20)]
    vox = np.array([c] + [(c + np.array(o)) % 24 for o in [(1, 0, 0), (0, -1, 0), (0, 0, 2), (-2, 1, 0)]])
    S = corr_so3_at(prob["V"], F, prob["radius"], Rs, vox).real
    assert np.argmax(S[0]) == 0
    assert S[0, 0] > S[1:, 0].max()


def test_component_correlation_at_voxels_matches_full():
    from oracle.so3 import component_correlation_at
    rng = np.random.default_rng(9)
    V = rng.standard_normal((6, 7, 8))
    F = small_filter(seed=2, L=2, radius=2.0)
    vox = np.array([[0, 0, 0], [5, 6, 7], [2, 3, 4]])
    for (l, a, b) in [(0, 0, 0), (1, 1, -1), (2, -2, 1)]:
        full = component_correlation(V, F, l, a, b, 2)
        np.testing.assert_allclose(component_correlation_at(V, F, l, a, b, 2, vox),
                                   full[vox[:, 0], vox[:, 1], vox[:, 2]], atol=1e-12)


def test_channel_layout_counts_and_pairing():
    """(2l+1)^2 real channels per degree; G_l^{-a,-b} = (-1)^{a+b} conj G_l^{ab}
    for a real filter and signal (the pairing the layout relies on)."""
    from oracle.so3 import channel_layout
    lay, n = channel_layout(6)
    assert n == 455 and len(lay) == 231
    rng = np.random.default_rng(10)
    V = rng.standard_normal((6, 6, 6))
    F = small_filter(seed=3, L=2, radius=2.0)
    for (l, a, b) in [(1, 1, 0), (2, 1, -2), (2, 0, 1)]:
        g = component_correlation(V, F, l, a, b, 2)
        gm = component_correlation(V, F, l, -a, -b, 2)
        np.testing.assert_allclose(gm, (-1) ** (a + b) * np.conj(g), atol=1e-12)


@pytest.mark.parametrize("l", [1, 3, 6])
def test_rotation_generators_are_the_derivative_of_the_definition(l):
    """A_i from the ladder relations equals the central difference of C^l
    computed from its definition (projection) about e_i."""
    from oracle.so3 import quat_exp, rotation_generators
    h = 1e-5
    for i, A in enumerate(rotation_generators(l)):
        e = np.zeros(3)
        e[i] = h
        Cp = wigner_by_projection(l, quat_to_matrix(quat_exp(e)))
        Cm = wigner_by_projection(l, quat_to_matrix(quat_exp(-e)))
        np.testing.assert_allclose(A, (Cp - Cm) / (2 * h), atol=1e-8)


def test_score_gradient_matches_finite_differences():
    from oracle.so3 import channel_layout, quat_exp, quat_mul, score_from_channels, score_gradient
    rng = np.random.default_rng(12)
    _, n = channel_layout(4)
    chan = rng.standard_normal(n)
    q = synth.haar_quaternion(rng)
    g = score_gradient(chan, 4, quat_to_matrix(q))
    h = 1e-5
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (score_from_channels(chan, 4, quat_to_matrix(quat_mul(q, quat_exp(e))))
              - score_from_channels(chan, 4, quat_to_matrix(quat_mul(q, quat_exp(-e))))) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd))
