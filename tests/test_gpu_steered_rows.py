"""GPU parity of the steered forward row passes at the line lengths that take
the component-loop kernel (1024, 2048: one row per block, the per-pixel
inputs held in registers across the block's components), against the
oracles at sampled pixels (every row, corners included), plus agreement of
the row-pass forms (staged lines, steering in the first stage's loads,
component loop with hardware or sincospif phasors) with one another.

Tolerances: the oracles' 1e-5 of the output scale.  The row-pass forms
compute the same FFT in FP32 with differently rounded phases (the hardware
sine and cosine within about 4e-7 absolute); each lies within about 1.5e-6
of the oracle, so two of them agree within 5e-6 rel-L2."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.filters_so2 import AnalyticGaussPow
from oracle.scale import MellinFilter, smooth as scale_smooth
from oracle.similarity import SimilarityFilter, smooth as simil_smooth
from oracle.so2 import ext_conv_so2_at as conv_ref_at

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
FORMS_REL_L2 = 5e-6


@pytest.fixture(scope="module")
def ec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_13188_gb300 as m
    m.lib()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def plan_with_form(ec, monkeypatch, form):
    """A plan whose steered row passes use form 0 (staged lines), 1 (steering
    in the first stage's loads), 2 (component loop with the hardware sine and
    cosine, the default) or 3 (component loop with sincospif)."""
    monkeypatch.setenv("EXT_STEER_MODE", str(form))
    p = ec.Plan(0)
    monkeypatch.delenv("EXT_STEER_MODE")
    return p


def sample_pixels(seed, h, w, n):
    """n random pixels plus one in every row and the four corners."""
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, h, n), rng.integers(0, w, n)], 1)
    rows = np.stack([np.arange(h), rng.integers(0, w, h)], 1)
    corners = np.array([[0, 0], [0, w - 1], [h - 1, 0], [h - 1, w - 1]])
    return np.concatenate([pix, rows, corners])


def scale_problem(seed, h, w, channels=3, s_max=3.0):
    rng = np.random.default_rng(seed)
    img = rng.uniform(0, 1, (channels, h, w)).astype(np.float32)
    s = synth.periodic_gaussian_blur(rng.uniform(1.0, s_max, (h, w)), 3.0)
    return img, np.clip(s, 1.0, s_max).astype(np.float32)


def run_scale(ec, plan, img, s, c, r_max, mode):
    C, h, w = img.shape
    out = torch.empty((C, h, w), dtype=torch.float32, device="cuda")
    ec.ext_conv_scale(plan, dev(img), C, h, w, c, 8.0, 1.0, r_max, 1.0, dev(s), mode, out)
    plan.sync()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_scale_component_loop_sampled(ec, mode):
    h, w, r_max = 32, 1024, 12.0
    img, s = scale_problem(10 + mode, h, w)
    c = synth.mellin_gaussian_coeffs()
    plan = ec.Plan(0)
    got = run_scale(ec, plan, img, s, c, r_max, mode)
    plan.close()
    pix = sample_pixels(mode, h, w, 96)
    ref = scale_smooth(img, s, MellinFilter(c, 8.0, 1.0, r_max, 1.0), mode=mode, pixels=pix)
    err = max(float(np.abs(got[ch][tuple(pix.T)] - ref[ch]).max()) for ch in range(3)) / np.abs(ref).max()
    print(f"scale {h}x{w} mode {mode}: error {err:.2e} of scale")
    assert err <= REL_L2


@pytest.mark.parametrize("mode", [0, 2])
def test_similarity_component_loop_sampled(ec, mode):
    h, w, K, n_h = 48, 1024, 3, 4
    rng = np.random.default_rng(77 + mode)
    c = (rng.standard_normal((K + 1, 2 * n_h - 1)) + 1j * rng.standard_normal((K + 1, 2 * n_h - 1))) / (K + n_h)
    c[0, n_h - 1] = abs(c[0, n_h - 1]) + 1.0
    img = rng.uniform(0, 1, (2, h, w)).astype(np.float32)
    alpha = rng.uniform(0, 2 * math.pi, (h, w)).astype(np.float32)
    s = rng.uniform(1.0, 1.8, (h, w)).astype(np.float32)
    plan = ec.Plan(0)
    out = torch.empty((2, h, w), dtype=torch.float32, device="cuda")
    ec.ext_conv_similarity(plan, dev(img), 2, h, w, c, 5.0, 0.95, 7.5, 0.8, dev(alpha), dev(s), mode, out)
    plan.sync()
    got = out.cpu().numpy()
    plan.close()
    pix = sample_pixels(mode, h, w, 64)
    ref = simil_smooth(img, alpha, s, SimilarityFilter(c, 5.0, 0.95, 7.5, 0.8), mode, pixels=pix)
    scale = np.abs(ref).max()
    err = max(float(np.abs(got[ch][tuple(pix.T)] - ref[ch]).max()) for ch in range(2)) / scale
    print(f"similarity {h}x{w} mode {mode}: error {err:.2e} of scale")
    assert err <= 1e-5


def test_so2_conv_component_loop_sampled(ec):
    prob = synth.so2_conv_problem(seed=5, size=1024)
    h, w = 64, 1024
    H = prob["H"][:h].copy()
    alpha = prob["alpha"][:h].copy()
    F = ec.FilterSO2.analytic(prob["a"], prob["sigma"], prob["radius"])
    plan = ec.Plan(0)
    out = torch.empty((h, w), dtype=torch.float32, device="cuda")
    ec.ext_conv_so2(plan, dev(H), h, w, F, dev(alpha), out)
    plan.sync()
    got = out.cpu().numpy()
    plan.close()
    pix = sample_pixels(5, h, w, 96)
    ref = conv_ref_at(H, AnalyticGaussPow(prob["a"], prob["sigma"]), alpha, prob["radius"], pix).real
    err = float(np.abs(got[tuple(pix.T)] - ref).max()) / np.abs(ref).max()
    print(f"so2 conv {h}x{w}: error {err:.2e} of scale")
    assert err <= REL_L2


def test_row_pass_forms_agree(ec, monkeypatch):
    """Scale (24 harmonics), similarity (68 log-polar harmonics) and SO(2)
    extended convolution at 2048-point rows through each row-pass form."""
    h, w = 32, 2048
    img, s = scale_problem(3, h, w)
    c_scale = synth.mellin_gaussian_coeffs()
    c_sim = synth.similarity_brush_coeffs()
    rng = np.random.default_rng(4)
    alpha = rng.uniform(0, 2 * math.pi, (h, w)).astype(np.float32)
    prob = synth.so2_conv_problem(seed=6, size=2048)
    results = []
    for form in (0, 1, 2, 3):
        plan = plan_with_form(ec, monkeypatch, form)
        r = {"scale": run_scale(ec, plan, img, s, c_scale, 24.0, 2)}
        out = torch.empty((3, h, w), dtype=torch.float32, device="cuda")
        ec.ext_conv_similarity(plan, dev(img), 3, h, w, c_sim, 6.0, 1.0, 16.0, 1.0, dev(alpha), dev(s), 2, out)
        plan.sync()
        r["similarity"] = out.cpu().numpy()
        F = ec.FilterSO2.analytic(prob["a"], prob["sigma"], prob["radius"])
        o2 = torch.empty((h, w), dtype=torch.float32, device="cuda")
        ec.ext_conv_so2(plan, dev(prob["H"][:h].copy()), h, w, F, dev(prob["alpha"][:h].copy()), o2)
        plan.sync()
        r["so2"] = o2.cpu().numpy()
        plan.close()
        results.append(r)
    for key in results[0]:
        for form in (0, 1, 3):
            err = rel_l2(results[form][key], results[2][key])
            print(f"{key}: form {form} vs component loop rel-L2 {err:.2e}")
            assert err < FORMS_REL_L2
