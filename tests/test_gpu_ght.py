"""GPU parity of the pattern-detection front end of Sec. 5 (gradient signal
and field, voted consensus filter, detection by extended convolution)
through the C ABI against the FP64 oracle.

Tolerances: signal within 1e-6 of its maximum, field within 2e-6 rad where
the gradient is not negligible (FP32 differences, hypotf, atan2f); the
consensus filter is FP64 on both sides (1e-12 of its maximum); the detection
response within 2e-5 of its scale (FP32 FFT path, FP32 field)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.filters_so2 import decompose_sampled
from oracle.ght import consensus_filter as consensus_ref, consensus_radius, gradient_field as gradient_ref
from oracle.so2 import ext_conv_so2_at

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


def _plant(img, P, centre, k):
    r = P.shape[0] // 2
    cy, cx = centre
    img[cy - r:cy + r + 1, cx - r:cx + r + 1] += np.rot90(P, k)


@pytest.mark.parametrize("h,w", [(96, 128), (1, 64), (37, 5), (2048, 2048)])
def test_gradient_field_matches_oracle(ec, plan, h, w):
    rng = np.random.default_rng(h * 7 + w)
    I = synth.periodic_gaussian_blur(rng.standard_normal((h, w)), 1.5).astype(np.float32)
    Hg = torch.empty((h, w), dtype=torch.float32, device="cuda")
    Tg = torch.empty((h, w), dtype=torch.float32, device="cuda")
    ec.ext_gradient_field(plan, dev(I), h, w, Hg, Tg)
    plan.sync()
    Hr, Tr = gradient_ref(I)
    Hn, Tn = Hg.cpu().numpy(), Tg.cpu().numpy()
    scale = max(float(Hr.max()), 1e-30)
    assert np.abs(Hn - Hr).max() <= 1e-6 * scale
    ok = Hr > 1e-3 * scale
    d = np.angle(np.exp(1j * (Tn[ok].astype(np.float64) - Tr[ok])))
    assert np.abs(d).max() <= 2e-6


def test_gradient_field_host_buffers_match_device(ec, plan):
    rng = np.random.default_rng(3)
    I = rng.standard_normal((40, 48)).astype(np.float32)
    Hg = torch.empty((40, 48), dtype=torch.float32, device="cuda")
    Tg = torch.empty((40, 48), dtype=torch.float32, device="cuda")
    ec.ext_gradient_field(plan, dev(I), 40, 48, Hg, Tg)
    Hh = np.zeros((40, 48), np.float32)
    Th = np.zeros((40, 48), np.float32)
    ec.ext_gradient_field(plan, I, 40, 48, Hh, Th)
    np.testing.assert_array_equal(Hh, Hg.cpu().numpy())
    np.testing.assert_array_equal(Th, Tg.cpu().numpy())


@pytest.mark.parametrize("radius,eps,centre", [(12, 10.5, (12, 12)), (20, 18.0, (20, 20)), (9, 4.0, (6, 11)),
                                               (5, 0.0, (5, 5))])
def test_consensus_filter_matches_oracle(ec, plan, radius, eps, centre):
    rng = np.random.default_rng(radius)
    P = synth.smooth_random_template(rng, radius, 2.0)
    R = ec.ext_consensus_radius(eps)
    assert R == consensus_radius(eps)
    F = np.zeros((2 * R + 1, 2 * R + 1))
    ec.ext_consensus_filter(plan, P, P.shape[0], P.shape[1], centre[0], centre[1], eps, F)
    ref = consensus_ref(P, centre, eps)
    assert np.abs(F - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)


def test_consensus_filter_rejects_bad_arguments(ec, plan):
    P = np.ones((9, 9))
    F = np.zeros((9, 9))
    for cy, cx, eps in ((9, 0, 2.0), (0, -1, 2.0), (4, 4, -1.0), (4, 4, 1e9)):
        with pytest.raises(ec.ExtError):
            ec.ext_consensus_filter(plan, P, 9, 9, cy, cx, eps, F)


def test_detection_matches_oracle_and_finds_the_turned_copies(ec, plan):
    """Four quarter-turned copies of a pattern in a 256 x 256 image: the GPU
    response (gradient signal and field, consensus filter band-limited to
    K = 8, extended convolution) against the oracle at the centres and at
    random pixels; equal responses at the four centres (detection is rotation
    invariant), which are the four largest in the image."""
    from paper_2006_13188_gb300 import ght
    rng = np.random.default_rng(17)
    P = synth.smooth_random_template(rng, 10, 1.5)
    img = np.zeros((256, 256))
    centres = [(48, 48), (48, 200), (200, 48), (200, 200)]
    for k, c in enumerate(centres):
        _plant(img, P, c, k)
    img = img.astype(np.float32)
    eps, K = 9.0, 8
    filt, F = ght.consensus_filter(plan, P, (10, 10), eps, K)
    out = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    ght.detect(plan, dev(img), 256, 256, filt, out)
    plan.sync()
    got = out.cpu().numpy()
    Hr, Tr = gradient_ref(img)
    filt_ref = decompose_sampled(consensus_ref(P, (10, 10), eps), K, 0.25, 128)
    pix = np.array(centres + [tuple(p) for p in rng.integers(0, 256, (200, 2))])
    ref = ext_conv_so2_at(Hr, filt_ref, Tr, consensus_radius(eps), pix).real
    scale = np.abs(ref).max()
    err = np.abs(got[pix[:, 0], pix[:, 1]] - ref).max() / scale
    print(f"detection 256^2 K={K}: max error {err:.2e} of the response scale")
    assert err <= 2e-5
    at = got[tuple(np.array(centres).T)]
    np.testing.assert_allclose(at, at[0], rtol=1e-4)
    top = np.argsort(got.ravel())[::-1][:4]
    assert sorted((int(i // 256), int(i % 256)) for i in top) == sorted(centres)
