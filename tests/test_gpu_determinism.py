"""Run-to-run determinism on the GPU (the build's stand-in for a race
detector, which is not available here): the same call twice gives
bit-identical outputs -- the FP32 and split-BF16 SO(2) sweeps, the scale
smoothing, the batched path, and the SO(3) sweeps whose blocks fold results
with atomics (the fold is order-independent by construction)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_13188_gb300 as m
    m.lib()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def twice(fn):
    a = fn()
    b = fn()
    return a, b


def test_so2_sweeps_are_deterministic(ec):
    plan = ec.Plan(0)
    prob = synth.so2_match_problem(seed=41, size=(256, 384), n_plant=3, radius=16, K=16, J=64)
    F = ec.FilterSO2.sampled(prob["template"], 16, prob["dr"], prob["n_theta"])
    H = dev(prob["H"])
    for prec in (ec.EXT_PREC_FP32, ec.EXT_PREC_BF16X3):
        def run():
            mx = torch.empty((256, 384), dtype=torch.float32, device="cuda")
            am = torch.empty((256, 384), dtype=torch.int32, device="cuda")
            ec.ext_corr_so2(plan, H, 256, 384, F, None, 64, mx, am, prec)
            plan.sync()
            return mx.cpu().numpy(), am.cpu().numpy()
        (m1, a1), (m2, a2) = twice(run)
        np.testing.assert_array_equal(m1, m2)
        np.testing.assert_array_equal(a1, a2)
    plan.close()


def test_scale_smoothing_is_deterministic(ec):
    plan = ec.Plan(0)
    prob = synth.scale_smoothing_problem(seed=5, size=(256, 512), n_cells=40)
    img, s, c = dev(prob["img"]), dev(prob["s"]), prob["c"]

    def run():
        out = torch.empty((3, 256, 512), dtype=torch.float32, device="cuda")
        ec.ext_conv_scale(plan, img, 3, 256, 512, c, prob["log_period"], prob["r_min"], prob["r_max"],
                          prob["centre_tap"], s, 2, out)
        plan.sync()
        return out.cpu().numpy()
    a, b = twice(run)
    np.testing.assert_array_equal(a, b)
    plan.close()


def test_so3_sweeps_are_deterministic(ec):
    plan = ec.Plan(0)
    rng = np.random.default_rng(9)
    L, n = 6, 20001
    nch = ec.ext_so3_channels(L)
    G = dev(rng.standard_normal((nch, n)).astype(np.float32))
    quats = np.array([synth.haar_quaternion(rng) for _ in range(300)])
    dirs = np.array([synth.haar_quaternion(rng) for _ in range(20)])
    for grid in (False, True):
        def run():
            mx = torch.empty(n, dtype=torch.float32, device="cuda")
            am = torch.empty(n, dtype=torch.int32, device="cuda")
            if grid:
                ec.ext_sweep_so3_grid(plan, G, n, L, dirs, 24, mx, am, ec.EXT_PREC_BF16X3)
            else:
                ec.ext_sweep_so3(plan, G, n, L, quats, mx, am, ec.EXT_PREC_BF16X3)
            plan.sync()
            return mx.cpu().numpy(), am.cpu().numpy()
        (m1, a1), (m2, a2) = twice(run)
        np.testing.assert_array_equal(m1, m2)
        np.testing.assert_array_equal(a1, a2)
    plan.close()
