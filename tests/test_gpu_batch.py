"""Batched correlation sweep over images of uneven sizes, bandwidths and angle
counts (one captured CUDA graph per batch): every image matches the
single-image call exactly, and the FP64 oracle at sampled pixels."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.filters_so2 import decompose_sampled
from oracle.so2 import sweep_so2_at

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_13188_gb300 as m
    m.lib()
    return m


# (h, w, template side, K, J): sizes with factors 2, 3, 5, 7, 11, 13; non-square
CASES = [(128, 192, 33, 4, 32), (320, 256, 45, 8, 36), (448, 128, 41, 16, 100),
         (256, 256, 65, 16, 64), (704, 192, 37, 8, 128), (832, 128, 35, 4, 44)]


def make_batch(ec, seed=0):
    items, probs = [], []
    for i, (h, w, side, K, J) in enumerate(CASES):
        desc = dict(h=h, w=w, side=side, radius=(side - 1) // 2, K=K, J=J, seed=seed * 1000 + i)
        prob = synth.batched_image(desc)
        F = ec.FilterSO2.sampled(prob["template"], K, prob["dr"], prob["n_theta"])
        H = torch.from_numpy(prob["H"]).cuda()
        mx = torch.empty((h, w), dtype=torch.float32, device="cuda")
        am = torch.empty((h, w), dtype=torch.int32, device="cuda")
        items.append((H, h, w, F, J, mx, am))
        probs.append(prob)
    return items, probs


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batch_matches_single_image_calls_and_oracle(ec, prec):
    precision = ec.EXT_PREC_FP32 if prec == "fp32" else ec.EXT_PREC_BF16X3
    plan = ec.Plan(0)
    items, probs = make_batch(ec)
    ec.ext_batch_corr_so2(plan, items, precision)
    plan.sync()
    single = ec.Plan(0)
    rng = np.random.default_rng(5)
    for (H, h, w, F, J, mx, am), prob in zip(items, probs):
        mx1 = torch.empty_like(mx)
        am1 = torch.empty_like(am)
        ec.ext_corr_so2(single, H, h, w, F, None, J, mx1, am1, precision)
        single.sync()
        assert torch.equal(mx, mx1) and torch.equal(am, am1), (h, w)
        K = prob["K"]
        tab = decompose_sampled(prob["template"], K, prob["dr"], prob["n_theta"])
        (cy, cx), = prob["centres"]
        pix = np.array([((cy + dy) % h, (cx + dx) % w) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
                       + [(int(rng.integers(0, h)), int(rng.integers(0, w))) for _ in range(64)])
        S = sweep_so2_at(prob["H"], tab, prob["radius"], J, pix).real
        got = mx.cpu().numpy()[pix[:, 0], pix[:, 1]]
        arg = am.cpu().numpy()[pix[:, 0], pix[:, 1]]
        scale = np.abs(S).max()
        tol = 1e-5 if prec == "fp32" else 1e-4
        window = 1e-6 if prec == "fp32" else 2e-4
        assert np.max(np.abs(got - S.max(axis=1))) <= tol * scale, (h, w)
        srt = np.sort(S, axis=1)
        clear = (srt[:, -1] - srt[:, -2]) > window * scale
        assert np.all(arg[clear] == S.argmax(axis=1)[clear]), (h, w)
        # the planted template is found at its angle
        j_true = round(prob["betas"][0] * J / (2 * math.pi)) % J
        dj = (int(am.cpu().numpy()[cy, cx]) - j_true) % J
        assert min(dj, J - dj) <= 1, (h, w)
    plan.close()
    single.close()


def test_batch_graph_replay_reads_new_data(ec):
    plan = ec.Plan(0)
    items, probs = make_batch(ec, seed=3)
    ec.ext_batch_corr_so2(plan, items)
    plan.sync()
    first = [it[5].clone() for it in items]
    # same descriptors (replayed graph), new pixel data in place
    for it in items:
        it[0].mul_(-1.0)
    ec.ext_batch_corr_so2(plan, items)
    plan.sync()
    single = ec.Plan(0)
    for (H, h, w, F, J, mx, am), old in zip(items, first):
        mx1 = torch.empty_like(mx)
        am1 = torch.empty_like(am)
        ec.ext_corr_so2(single, H, h, w, F, None, J, mx1, am1, ec.EXT_PREC_BF16X3)
        single.sync()
        assert torch.equal(mx, mx1) and torch.equal(am, am1)
        assert not torch.equal(mx, old)
    plan.close()
    single.close()


def test_batch_rebuilds_template_spectra_when_a_filter_changes(ec):
    """The template spectra are kept between calls; a changed filter (another
    template, or the same arrays rewritten in place) rebuilds them."""
    plan = ec.Plan(0)
    items, probs = make_batch(ec, seed=4)
    ec.ext_batch_corr_so2(plan, items)
    plan.sync()
    rng = np.random.default_rng(8)
    h, w, side, K, J = CASES[2]
    tpl = synth.smooth_random_template(rng, (side - 1) // 2, 3.0)
    H, h, w, F, J, mx, am = items[2]
    items[2] = (H, h, w, ec.FilterSO2.sampled(tpl, K, probs[2]["dr"], probs[2]["n_theta"]), J, mx, am)
    ec.ext_batch_corr_so2(plan, items)
    plan.sync()
    single = ec.Plan(0)
    for (H, h, w, F, J, mx, am) in items:
        mx1 = torch.empty_like(mx)
        am1 = torch.empty_like(am)
        ec.ext_corr_so2(single, H, h, w, F, None, J, mx1, am1, ec.EXT_PREC_BF16X3)
        single.sync()
        assert torch.equal(mx, mx1) and torch.equal(am, am1)
    # the same filter arrays rewritten in place
    F3 = items[3][3]
    F3._img[...] = np.flipud(F3._img).copy()
    ec.ext_batch_corr_so2(plan, items)
    plan.sync()
    H, h, w, F, J, mx, am = items[3]
    mx1 = torch.empty_like(mx)
    am1 = torch.empty_like(am)
    ec.ext_corr_so2(single, H, h, w, F, None, J, mx1, am1, ec.EXT_PREC_BF16X3)
    single.sync()
    assert torch.equal(mx, mx1) and torch.equal(am, am1)
    plan.close()
    single.close()
