"""GPU parity of fixed-budget component selection (Sec. 5 "Band-Limiting
Revisited"): lattice energies, the selection rule, and the sweep over a
component subset, through the C ABI against the FP64 oracle.

Tolerances: energies FP64 on both sides (1e-8 relative); subset sweep maxima
within 1e-5 (FP32 sweep) or 1e-4 (split-BF16 sweep) of the score scale,
argmax identical outside the tie window."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.filters_so2 import AnalyticGaussPow, decompose_sampled
from oracle.selection import component_energy, select_components, sweep_subset_from_components
from oracle.so2 import component_correlation

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


def test_energies_match_oracle(ec, plan):
    a = synth.random_gauss_pow_coeffs(5, 6)
    Fa = ec.FilterSO2.analytic(a, 2.5, 9)
    Ea = ec.ext_filter_so2_energy(plan, Fa)
    np.testing.assert_allclose(Ea, component_energy(AnalyticGaussPow(a, 2.5), 6, 9), rtol=1e-8)
    tpl = synth.smooth_random_template(np.random.default_rng(6), 12, 2.0)
    Fs = ec.FilterSO2.sampled(tpl, 10, 0.25, 128)
    Es = ec.ext_filter_so2_energy(plan, Fs)
    np.testing.assert_allclose(Es, component_energy(decompose_sampled(tpl, 10, 0.25, 128), 10, 12), rtol=1e-8)
    from paper_2006_13188_gb300 import selection
    for budget in (1, 3, 6, 11, 20):
        assert selection.select(plan, Fs, budget) == select_components(Es, budget)


@pytest.mark.parametrize("precision,tol", [("EXT_PREC_FP32", 1e-5), ("EXT_PREC_BF16X3", 1e-4)])
@pytest.mark.parametrize("ks", [[0, 1, 2, 3], [0, 2, 5, 7], [0], [0, 8]])
def test_subset_sweep_matches_oracle(ec, plan, precision, tol, ks):
    p2 = synth.so2_match_problem(seed=31, size=96, n_plant=2, radius=10, K=8, J=40)
    K, J, R = p2["K"], p2["J"], p2["radius"]
    F = ec.FilterSO2.sampled(p2["template"], K, p2["dr"], p2["n_theta"])
    mx = torch.empty((96, 96), dtype=torch.float32, device="cuda")
    am = torch.empty((96, 96), dtype=torch.int32, device="cuda")
    ec.ext_corr_so2_subset(plan, dev(p2["H"]), 96, 96, F, ks, J, mx, am, getattr(ec, precision))
    plan.sync()
    tab = decompose_sampled(p2["template"], K, p2["dr"], p2["n_theta"])
    G = [component_correlation(p2["H"], tab, k, R) if k in ks else np.zeros((96, 96)) for k in range(K + 1)]
    S = sweep_subset_from_components(G, ks, J).reshape(J, -1).T
    scale = np.abs(S).max()
    got_m, got_a = mx.cpu().numpy().ravel(), am.cpu().numpy().ravel()
    assert np.abs(got_m - S.max(axis=1)).max() <= tol * scale
    srt = np.sort(S, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 2 * tol * scale
    assert np.all(got_a[clear] == S.argmax(axis=1)[clear])


def test_full_list_equals_the_band_limited_sweep(ec, plan):
    p2 = synth.so2_match_problem(seed=32, size=128, n_plant=2, radius=12, K=8, J=36)
    F = ec.FilterSO2.sampled(p2["template"], 8, p2["dr"], p2["n_theta"])
    out = {}
    for name in ("subset", "full"):
        mx = torch.empty((128, 128), dtype=torch.float32, device="cuda")
        am = torch.empty((128, 128), dtype=torch.int32, device="cuda")
        if name == "subset":
            ec.ext_corr_so2_subset(plan, dev(p2["H"]), 128, 128, F, list(range(9)), 36, mx, am, ec.EXT_PREC_BF16X3)
        else:
            ec.ext_corr_so2(plan, dev(p2["H"]), 128, 128, F, None, 36, mx, am, ec.EXT_PREC_BF16X3)
        plan.sync()
        out[name] = (mx.cpu().numpy(), am.cpu().numpy())
    np.testing.assert_array_equal(out["subset"][0], out["full"][0])
    np.testing.assert_array_equal(out["subset"][1], out["full"][1])


def test_subset_rejects_bad_lists(ec, plan):
    F = ec.FilterSO2.analytic(synth.random_gauss_pow_coeffs(2, 4), 2.0, 6)
    H = np.zeros((32, 32), np.float32)
    mx = np.zeros((32, 32), np.float32)
    am = np.zeros((32, 32), np.int32)
    for ks in ([], [1, 2], [0, 2, 2], [0, 3, 1], [0, 5]):
        with pytest.raises(ec.ExtError):
            ec.ext_corr_so2_subset(plan, H, 32, 32, F, ks, 8, mx, am, ec.EXT_PREC_FP32)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _detected(resp, centres, radius):
    """Planted centres among the len(centres) strongest local maxima (peaks
    at least one box apart, periodic), within 2 px."""
    from scipy import ndimage
    h, w = resp.shape
    mx = ndimage.maximum_filter(resp, size=2 * radius + 1, mode="wrap")
    pk = np.argwhere(resp == mx)
    top = pk[np.argsort(-resp[pk[:, 0], pk[:, 1]])[:len(centres)]]
    found = 0
    for c in centres:
        d = np.abs(top - np.asarray(c))
        d = np.minimum(d, np.array([h, w]) - d)
        found += bool(np.any(d.max(axis=1) <= 2))
    return found


def test_band_limited_budget_beats_rotated_copies(ec, plan):
    """Fig. f:frequency (Sec. 5 "Band-Limiting Revisited"): with the same
    number B of standard correlations, steering the B largest-energy angular
    components (the GPU's subset sweep over 64 angles) approximates exact
    rotation-independent matching -- the maximum over 128 rotated copies of a
    pattern that is not band-limited -- better than correlating with B
    rotated copies, and finds every planted pattern from a smaller budget."""
    from oracle.selection import rotated_copies_sweep
    prob = synth.so2_match_problem(seed=77, size=512, n_plant=8, radius=24, K=32, J=64, blur=1.5)
    H, T, R = prob["H"], prob["template"], prob["radius"]
    truth, _ = rotated_copies_sweep(H, T, 128)
    F = ec.FilterSO2.sampled(T, 32, prob["dr"], prob["n_theta"])
    E = ec.ext_filter_so2_energy(plan, F)
    mx = torch.empty((512, 512), dtype=torch.float32, device="cuda")
    am = torch.empty((512, 512), dtype=torch.int32, device="cuda")
    Hd = dev(H)
    last = None
    for B in (2, 3, 5, 9, 13):
        ks = ec.ext_select_components(E, B)
        ec.ext_corr_so2_subset(plan, Hd, 512, 512, F, ks, 64, mx, am, ec.EXT_PREC_FP32)
        plan.sync()
        bl = mx.cpu().numpy().astype(np.float64)
        rot, _ = rotated_copies_sweep(H, T, B)
        e_bl, e_rot = _rel(bl, truth), _rel(rot, truth)
        d_bl, d_rot = _detected(bl, prob["centres"], R), _detected(rot, prob["centres"], R)
        print(f"budget {B}: components {ks}: error {e_bl:.3f}, {d_bl}/8 found; "
              f"{B} rotated copies: error {e_rot:.3f}, {d_rot}/8 found")
        assert e_bl < e_rot
        assert d_bl == 8
        if last is not None:
            assert e_bl < last
        last = e_bl
