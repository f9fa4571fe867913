"""The allocation-free sweep entry point, for callers that cannot let the
library allocate device memory (their device memory is owned by their own
allocator, or they cannot afford the synchronisation cudaMalloc implies).

It must give the same maxima and argmax as the planned ext_sweep_so2 (FP32)
on two calls in a row -- the second with a different bandwidth and angle
count, so that the shared scratch table really is rewritten per call -- and
agree with the FP64 oracle's steering sum (maxima within 1e-5 of the score
scale, argmax identical outside the 1e-6 tie window), so that an error
shared by the two entry points' table or kernel would not pass.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

from oracle.so2 import sweep_from_components

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _components(rng, K, n):
    return rng.standard_normal((2 * K + 1, n)).astype(np.float32)


def test_noalloc_sweep_matches_planned_sweep_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_13188_gb300 as ec
    ec.lib()
    plan = ec.Plan(0)
    rng = np.random.default_rng(2024)
    for K, J, n in [(16, 64, 4099), (5, 36, 1003)]:
        G = torch.from_numpy(_components(rng, K, n)).cuda()
        ref_max = torch.empty(n, device="cuda")
        ref_arg = torch.empty(n, dtype=torch.int32, device="cuda")
        ec.ext_sweep_so2(plan, G, n, K, J, ref_max, ref_arg, ec.EXT_PREC_FP32)
        got_max = torch.full((n,), float("nan"), device="cuda")
        got_arg = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        ec.ext_sweep_so2_noalloc(G, n, K, J, got_max, got_arg)
        torch.cuda.synchronize()
        r, g = ref_max.cpu().numpy(), got_max.cpu().numpy()
        scale = np.abs(r).max()
        assert np.max(np.abs(g - r)) <= 1e-5 * scale, (K, J)
        assert np.array_equal(got_arg.cpu().numpy(), ref_arg.cpu().numpy()), (K, J)
        G64 = G.cpu().numpy().astype(np.float64)
        Gc = [G64[0]] + [G64[2 * k - 1] + 1j * G64[2 * k] for k in range(1, K + 1)]
        S = sweep_from_components(Gc, K, J).real.T
        oscale = np.abs(S).max()
        assert np.max(np.abs(g - S.max(axis=1))) <= 1e-5 * oscale, (K, J)
        srt = np.sort(S, axis=1)
        clear = (srt[:, -1] - srt[:, -2]) > 1e-6 * oscale
        assert np.all(got_arg.cpu().numpy()[clear] == S.argmax(axis=1)[clear]), (K, J)
    plan.close()


def test_noalloc_sweep_rejects_sizes_beyond_its_table():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_13188_gb300 as ec
    x = torch.zeros(64, device="cuda")
    a = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(ec.ExtError) as e:
        ec.ext_sweep_so2_noalloc(x, 1, 16, 129, x, a)
    assert e.value.status == 2
    with pytest.raises(ec.ExtError) as e:
        ec.ext_sweep_so2_noalloc(x, 1, 17, 8, x, a)
    assert e.value.status == 2
