"""The seeded input generators shared by the oracle and the CUDA path:
reproducible from their seeds, and with the ranges and structure the
workloads state.  CPU only."""
import math

import numpy as np

import synth


def test_so3_conv_problem_is_seeded_and_its_field_is_unit_quaternions():
    a = synth.so3_conv_problem(seed=3, shape=(16, 16, 16), L=2, radius=3)
    b = synth.so3_conv_problem(seed=3, shape=(16, 16, 16), L=2, radius=3)
    np.testing.assert_array_equal(a["V"], b["V"])
    np.testing.assert_array_equal(a["Q"], b["Q"])
    assert a["Q"].shape == (16, 16, 16, 4) and a["Q"].dtype == np.float32
    np.testing.assert_allclose(np.linalg.norm(a["Q"].astype(np.float64), axis=-1), 1.0, atol=1e-6)
    assert abs(float(a["V"].std()) - 1.0) < 1e-5
    assert len(a["tables"]) == 3 and a["tables"][2].shape[0] == 5


def test_similarity_problem_ranges_and_brush():
    p = synth.similarity_problem(seed=4, size=(64, 96))
    assert p["img"].shape == (3, 64, 96)
    assert p["s"].min() >= 1.0 - 1e-6 and p["s"].max() <= 3.0 + 1e-6
    assert p["alpha"].min() >= 0.0 and p["alpha"].max() < 2 * math.pi
    c = p["c"]
    assert c.shape == (5, 15)
    # separable: c_{k,j} = a_k b_j (rank one), and b_{-j} = conj(b_j)
    assert np.linalg.matrix_rank(c, tol=1e-10 * np.abs(c).max()) == 1
    np.testing.assert_allclose(c[0, ::-1], np.conj(c[0]), atol=1e-14)


def test_brush_matches_its_design_within_the_fit():
    """A(phi) B(ln r) with A = exp(1.5 (cos phi - 1)) and a Gaussian B (sigma 2)
    on radii 1-16 at scales 1-3, to the band limit and the Mellin fit (1e-2)."""
    c = synth.similarity_brush_coeffs()
    K, nj = c.shape[0] - 1, c.shape[1]
    n = (nj + 1) // 2
    r = np.linspace(1, 16, 40)
    phi = np.linspace(-math.pi, math.pi, 41)
    R, PH = np.meshgrid(r, phi)
    for s in (1.0, 2.0, 3.0):
        u = np.log(R) - math.log(s)
        q = np.zeros(R.shape, np.complex128)
        for k in range(-K, K + 1):
            for j in range(-(n - 1), n):
                ckj = c[k, j + n - 1] if (k > 0 or (k == 0 and j >= 0)) else np.conj(c[-k, -j + n - 1])
                q += ckj * np.exp(1j * (k * PH + 2 * math.pi * j / 6.0 * u))
        ref = np.exp(1.5 * (np.cos(PH) - 1)) * np.exp(-(R / s) ** 2 / 8.0)
        assert np.abs(q.real - ref).max() < 1e-2
