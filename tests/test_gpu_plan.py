"""The plan options and failure paths on the GPU, through the C ABI:
a bounded device-side wait that runs out (EXT_ERR_TIMEOUT, plan usable
afterwards), an injected allocation failure (EXT_ERR_OOM, then normal
service), the plan's default precision, the autotuner (same results as the
built-in choice, cache written and reused), and resuming the proposal
network's training from a checkpoint."""
import os

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


def _problem():
    return synth.so2_match_problem(seed=31, size=128, n_plant=2, radius=12, K=8, J=32)


def _sweep(ec, plan, prob, precision):
    F = ec.FilterSO2.sampled(prob["template"], prob["K"], prob["dr"], prob["n_theta"])
    mx = torch.empty((128, 128), dtype=torch.float32, device="cuda")
    am = torch.empty((128, 128), dtype=torch.int32, device="cuda")
    ec.ext_corr_so2(plan, dev(prob["H"]), 128, 128, F, None, prob["J"], mx, am, precision)
    plan.sync()
    return mx.cpu().numpy(), am.cpu().numpy()


def test_bounded_wait_runs_out_and_the_plan_recovers(ec):
    """A kernel waits on an mbarrier that nothing completes, with a 1 ms
    budget: the wait gives up, ext_plan_sync reports EXT_ERR_TIMEOUT once,
    and the plan then computes as before."""
    plan = ec.Plan(0, wait_budget_ns=1_000_000)
    prob = _problem()
    ref = _sweep(ec, plan, prob, ec.EXT_PREC_BF16X3)
    plan.selftest_timeout()
    with pytest.raises(ec.ExtError) as e:
        plan.sync()
    assert e.value.status == 5
    plan.sync()                                   # the status word was cleared
    got = _sweep(ec, plan, prob, ec.EXT_PREC_BF16X3)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    plan.close()


@pytest.mark.parametrize("after", [0, 3])
def test_injected_allocation_failure(ec, after):
    """The (after+1)-th device allocation of the plan fails as out of memory:
    the call returns EXT_ERR_OOM before computing anything wrong, and the
    next call completes and agrees with a plan without injection."""
    prob = _problem()
    ref_plan = ec.Plan(0)
    ref = _sweep(ec, ref_plan, prob, ec.EXT_PREC_FP32)
    ref_plan.close()
    plan = ec.Plan(0, fault_inject=ec.EXT_FAULT_ALLOC, fault_after=after)
    with pytest.raises(ec.ExtError) as e:
        _sweep(ec, plan, prob, ec.EXT_PREC_FP32)
    assert e.value.status == 4
    got = _sweep(ec, plan, prob, ec.EXT_PREC_FP32)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    plan.close()


def test_default_precision_comes_from_the_plan(ec):
    prob = _problem()
    plan = ec.Plan(0, precision=ec.EXT_PREC_BF16X3)
    a = _sweep(ec, plan, prob, ec.EXT_PREC_DEFAULT)
    b = _sweep(ec, plan, prob, ec.EXT_PREC_BF16X3)
    c = _sweep(ec, plan, prob, ec.EXT_PREC_FP32)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    plan.close()


def test_autotuner_keeps_results_and_reuses_its_cache(ec, tmp_path):
    """The tuned pass variant gives the built-in choice's results (within
    FP32 rounding); the cache file names the shape class, and a new plan that
    reads it launches only one variant on its first call."""
    prob = _problem()
    ref_plan = ec.Plan(0)
    ref = _sweep(ec, ref_plan, prob, ec.EXT_PREC_FP32)
    ref_plan.close()
    cache = tmp_path / "tune.txt"
    plan = ec.Plan(0, autotune=True, tune_cache=str(cache))
    got = _sweep(ec, plan, prob, ec.EXT_PREC_FP32)
    scale = np.abs(ref[0]).max()
    assert np.max(np.abs(got[0] - ref[0])) <= 1e-6 * scale
    assert np.mean(got[1] == ref[1]) >= 0.999
    plan.close()
    text = cache.read_text()
    assert "components 128x128 K=8" in text, text
    plan2 = ec.Plan(0, autotune=True, tune_cache=str(cache))
    plan2.profile_read()
    _sweep(ec, plan2, prob, ec.EXT_PREC_FP32)
    counts = plan2.profile_read()
    assert counts["rows_r2c"][1] == 1, counts
    plan2.close()


def test_training_resumes_from_a_checkpoint(ec, tmp_path):
    """Ten Adam steps, a checkpoint, ten more steps; a new network loaded from
    the checkpoint and given the same ten steps ends with the same weights.
    A checkpoint of other shapes is refused (EXT_ERR_CHECKPOINT) and leaves
    the network unchanged."""
    rng = np.random.default_rng(4)
    C, H, n, batch = 35, 64, 256, 64
    X = rng.standard_normal((n, C)).astype(np.float32)
    qt = rng.standard_normal((n, 4))
    qt = (qt / np.linalg.norm(qt, axis=1, keepdims=True)).astype(np.float32)
    rows = rng.integers(0, n, 20 * batch).astype(np.int32)
    plan = ec.Plan(0)
    a = ec.MLP(plan, C, H)
    a.set_params(synth.mlp_init(3, C, H))
    ec.ext_mlp_train(a, X, qt, n, 2, rows[:10 * batch], None, 10, batch, 1e-3, None)
    path = tmp_path / "net.ckpt"
    a.save(path)
    assert ec.ext_mlp_checkpoint_info(path) == (C, H, 10)
    ec.ext_mlp_train(a, X, qt, n, 2, rows[10 * batch:], None, 10, batch, 1e-3, None)
    b = ec.MLP(plan, C, H)
    b.load(path)
    ec.ext_mlp_train(b, X, qt, n, 2, rows[10 * batch:], None, 10, batch, 1e-3, None)
    pa, pb = a.get_params(), b.get_params()
    for k in pa:
        np.testing.assert_array_equal(pa[k], pb[k], err_msg=k)
    other = ec.MLP(plan, C, 32)
    other.save(tmp_path / "other.ckpt")
    before = b.get_params()
    with pytest.raises(ec.ExtError) as e:
        b.load(tmp_path / "other.ckpt")
    assert e.value.status == 6
    after = b.get_params()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    plan.close()
