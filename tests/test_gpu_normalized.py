"""GPU parity of the normalised extended convolution (Sec. 8, Eq.
normalization; Line Integral Convolution with an anisotropic Gaussian)
through the C ABI against the FP64 oracle.

Tolerance: outputs within 1e-5 of the output scale (both extended
convolutions run the FP32 FFT path; the quotient of two FP32 results)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.filters_so2 import RadialTable
from oracle.normalized import aniso_gauss_table, normalized_conv_so2_at

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


def _lic_problem(seed, h, w, channels, su=6.0, sv=1.2, K=12, R=14):
    rng = np.random.default_rng(seed)
    H = rng.uniform(0, 1, (channels, h, w)).astype(np.float32)
    alpha = synth.random_angle_field(seed, h, w).astype(np.float32)
    fk = aniso_gauss_table(su, sv, K, 0.25, float(R))
    return H, alpha, fk, R


@pytest.mark.parametrize("h,w,channels", [(128, 160, 2), (64, 64, 1), (256, 96, 3)])
def test_normalized_conv_matches_oracle(ec, plan, h, w, channels):
    H, alpha, fk, R = _lic_problem(h + w, h, w, channels)
    F = ec.FilterSO2.table(fk, 0.25, R)
    out = torch.empty((channels, h, w), dtype=torch.float32, device="cuda")
    ec.ext_conv_so2_normalized(plan, dev(H), channels, h, w, F, dev(alpha), out)
    plan.sync()
    got = out.cpu().numpy()
    filt = RadialTable(fk, 0.25)
    rng = np.random.default_rng(1)
    pix = np.stack([rng.integers(0, h, 120), rng.integers(0, w, 120)], axis=1)
    pix = np.concatenate([pix, [[0, 0], [h - 1, w - 1]]])
    err = 0.0
    for c in range(channels):
        ref = normalized_conv_so2_at(H[c], filt, alpha, R, pix)
        err = max(err, float(np.abs(got[c][tuple(pix.T)] - ref).max()))
    print(f"normalised conv {channels}x{h}x{w}: max error {err:.2e}")
    assert err <= 1e-5


def test_normalized_conv_reproduces_constant_images(ec, plan):
    _, alpha, fk, R = _lic_problem(5, 96, 128, 1)
    F = ec.FilterSO2.table(fk, 0.25, R)
    H = np.full((2, 96, 128), 0.625, np.float32)
    H[1] = -3.0
    out = torch.empty((2, 96, 128), dtype=torch.float32, device="cuda")
    ec.ext_conv_so2_normalized(plan, dev(H), 2, 96, 128, F, dev(alpha), out)
    plan.sync()
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[0], 0.625, rtol=1e-5)
    np.testing.assert_allclose(got[1], -3.0, rtol=1e-5)


def test_normalized_conv_host_buffers_match_device(ec, plan):
    H, alpha, fk, R = _lic_problem(7, 64, 96, 2)
    F = ec.FilterSO2.table(fk, 0.25, R)
    out_d = torch.empty((2, 64, 96), dtype=torch.float32, device="cuda")
    ec.ext_conv_so2_normalized(plan, dev(H), 2, 64, 96, F, dev(alpha), out_d)
    out_h = np.zeros((2, 64, 96), np.float32)
    ec.ext_conv_so2_normalized(plan, H, 2, 64, 96, F, alpha, out_h)
    np.testing.assert_array_equal(out_h, out_d.cpu().numpy())


def test_normalized_conv_rejects_bad_channel_counts(ec, plan):
    H, alpha, fk, R = _lic_problem(8, 32, 32, 1)
    F = ec.FilterSO2.table(fk, 0.25, R)
    out = np.zeros((1, 32, 32), np.float32)
    for ch in (0, 65):
        with pytest.raises(ec.ExtError):
            ec.ext_conv_so2_normalized(plan, H, ch, 32, 32, F, alpha, out)
