"""GPU parity of extended convolution with a joint rotation x scale field
(log-polar harmonics: the angular components of Sec. 4.1 times the
log-radial ones of Sec. 8) through the C ABI against the FP64 oracle.

Tolerance: 1e-5 of the output scale (FP32 FFT path over all harmonics; modes
1 and 2 divide two such results); K = 0 agrees with the scale path to 1e-6."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.similarity import SimilarityFilter, smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_13188_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def plan(ec):
    p = ec.Plan(0)
    yield p
    p.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def random_problem(seed, h, w, channels, K, n_h, r_min=0.95, r_max=7.5, lp=5.0, cd=0.8):
    rng = np.random.default_rng(seed)
    c = (rng.standard_normal((K + 1, 2 * n_h - 1)) + 1j * rng.standard_normal((K + 1, 2 * n_h - 1))) / (K + n_h)
    c[0, n_h - 1] = abs(c[0, n_h - 1]) + 1.0          # a positive mean keeps the denominators away from 0
    img = rng.uniform(0, 1, (channels, h, w)).astype(np.float32)
    alpha = rng.uniform(0, 2 * math.pi, (h, w)).astype(np.float32)
    s = rng.uniform(1.0, 1.8, (h, w)).astype(np.float32)
    return dict(img=img, alpha=alpha, s=s, c=c, log_period=lp, r_min=r_min, r_max=r_max, centre_tap=cd)


def run(ec, plan, p, mode, host=False):
    C, h, w = p["img"].shape
    if host:
        out = np.zeros((C, h, w), np.float32)
        ec.ext_conv_similarity(plan, p["img"], C, h, w, p["c"], p["log_period"], p["r_min"], p["r_max"],
                               p["centre_tap"], p["alpha"], p["s"], mode, out)
        return out
    out = torch.empty((C, h, w), dtype=torch.float32, device="cuda")
    ec.ext_conv_similarity(plan, dev(p["img"]), C, h, w, p["c"], p["log_period"], p["r_min"], p["r_max"],
                           p["centre_tap"], dev(p["alpha"]), dev(p["s"]), mode, out)
    plan.sync()
    return out.cpu().numpy()


def oracle_at(p, mode, pix):
    f = SimilarityFilter(p["c"], p["log_period"], p["r_min"], p["r_max"], p["centre_tap"])
    return smooth(p["img"], p["alpha"], p["s"], f, mode, pixels=pix)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("h,w,K,n_h", [(96, 128, 3, 4), (64, 64, 0, 5), (160, 96, 5, 1)])
def test_similarity_conv_matches_oracle(ec, plan, mode, h, w, K, n_h):
    p = random_problem(h + w + K + n_h, h, w, 2, K, n_h)
    got = run(ec, plan, p, mode)
    rng = np.random.default_rng(mode)
    pix = np.stack([rng.integers(0, h, 80), rng.integers(0, w, 80)], 1)
    pix = np.concatenate([pix, [[0, 0], [h - 1, w - 1]]])
    ref = oracle_at(p, mode, pix)
    scale = np.abs(ref).max()
    err = max(float(np.abs(got[c][tuple(pix.T)] - ref[c]).max()) for c in range(2)) / scale
    print(f"similarity conv {h}x{w} K={K} n_h={n_h} mode {mode}: error {err:.2e} of scale")
    assert err <= 1e-5


def test_rotation_free_filter_equals_the_scale_path(ec, plan):
    p = random_problem(7, 128, 128, 1, 0, 6)
    got = run(ec, plan, p, 2)
    out = torch.empty((1, 128, 128), dtype=torch.float32, device="cuda")
    ec.ext_conv_scale(plan, dev(p["img"]), 1, 128, 128, p["c"][0, 5:], p["log_period"], p["r_min"], p["r_max"],
                      p["centre_tap"], dev(p["s"]), 2, out)
    plan.sync()
    ref = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def test_normalised_modes_reproduce_constant_images(ec, plan):
    p = random_problem(8, 64, 96, 2, 2, 3)
    p["img"][0] = 0.4
    p["img"][1] = -1.5
    for mode in (1, 2):
        got = run(ec, plan, p, mode)
        np.testing.assert_allclose(got[0], 0.4, rtol=2e-5)
        np.testing.assert_allclose(got[1], -1.5, rtol=2e-5)


def test_workload_size_sampled(ec, plan):
    """The 2048^2 x 3 brush workload (K = 4, 8 log-radial harmonics, radii 1-16)."""
    p = synth.similarity_problem(seed=synth.seed_for(10))
    got = run(ec, plan, p, 2)
    rng = np.random.default_rng(3)
    pix = np.stack([rng.integers(0, 2048, 40), rng.integers(0, 2048, 40)], 1)
    ref = oracle_at(p, 2, pix)
    err = max(float(np.abs(got[c][tuple(pix.T)] - ref[c]).max()) for c in range(3)) / np.abs(ref).max()
    print(f"similarity workload 2048^2x3: error {err:.2e} of scale")
    assert err <= 1e-5


def test_host_buffers_match_device(ec, plan):
    p = random_problem(9, 64, 64, 1, 2, 2)
    np.testing.assert_array_equal(run(ec, plan, p, 1, host=True), run(ec, plan, p, 1))


def test_rejects_bad_arguments(ec, plan):
    p = random_problem(10, 32, 32, 1, 1, 2)
    out = np.zeros((1, 32, 32), np.float32)
    args = (p["log_period"], p["r_min"], p["r_max"], p["centre_tap"], p["alpha"], p["s"])
    for c, mode in ((p["c"], 3), (np.zeros((66, 3), np.complex128), 1), (np.zeros((2, 129), np.complex128), 1)):
        with pytest.raises(ec.ExtError):
            ec.ext_conv_similarity(plan, p["img"], 1, 32, 32, c, *args, mode, out)


def test_window_wider_than_the_image_wraps(ec, plan):
    """r_max = 20 on a 32 x 48 image: the harmonic grids wrap (accumulated taps)."""
    p = random_problem(11, 32, 48, 1, 2, 3, r_min=0.95, r_max=20.0)
    got = run(ec, plan, p, 1)
    rng = np.random.default_rng(11)
    pix = np.stack([rng.integers(0, 32, 30), rng.integers(0, 48, 30)], 1)
    ref = oracle_at(p, 1, pix)
    assert np.abs(got[0][tuple(pix.T)] - ref[0]).max() <= 1e-5 * np.abs(ref).max()


def test_high_angular_order(ec, plan):
    """K = 12 with 2 log-radial harmonics: the phasor powers up to u^12."""
    p = random_problem(12, 64, 96, 1, 12, 2)
    got = run(ec, plan, p, 0)
    rng = np.random.default_rng(12)
    pix = np.stack([rng.integers(0, 64, 40), rng.integers(0, 96, 40)], 1)
    ref = oracle_at(p, 0, pix)
    assert np.abs(got[0][tuple(pix.T)] - ref[0]).max() <= 1e-5 * np.abs(ref).max()
