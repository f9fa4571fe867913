"""GPU parity of the SO(3) extended convolution (Eq. Def-EConv with a rotation
at every input voxel; component form of Sec. 9) through the C ABI against the
FP64 oracle.

Tolerance: relative L2 error <= 1e-5 over the compared voxels (the FP32 FFT
path: one complex transform per unique (l, a, b), products summed in FP32);
L = 0 steering is exact, so its output cannot depend on the field."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle.so3 import SHFilter, box_offsets3, conv_so3_at, filter_eval, quat_to_matrix, rotated_filter_eval

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


def run(ec, plan, V, prob, Q):
    nz, ny, nx = V.shape
    out = torch.empty(V.shape, dtype=torch.float32, device="cuda")
    ec.ext_conv_so3(plan, dev(V), nz, ny, nx, prob["tables"], prob["dr"], prob["radius"], dev(Q), out)
    plan.sync()
    return out.cpu().numpy()


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))


def sample_voxels(rng, shape, n):
    vox = np.stack([rng.integers(0, s, n) for s in shape], axis=1)
    return np.concatenate([vox, [[0, 0, 0], [s - 1 for s in shape]]])


def fft_conv(V, vals, radius):
    dx, dy, dz = box_offsets3(radius)
    g = np.zeros(V.shape, np.complex128)
    np.add.at(g, (dz % V.shape[0], dy % V.shape[1], dx % V.shape[2]), vals)
    return np.fft.ifftn(np.fft.fftn(V.astype(np.float64)) * np.fft.fftn(g)).real


@pytest.mark.parametrize("shape,L,radius", [((32, 32, 32), 3, 4), ((32, 48, 64), 2, 5), ((64, 64, 64), 6, 6)])
def test_conv_so3_matches_oracle(ec, plan, shape, L, radius):
    prob = synth.so3_conv_problem(seed=sum(shape) + L, shape=shape, L=L, radius=radius, field_sigma=2.0)
    got = run(ec, plan, prob["V"], prob, prob["Q"])
    F = SHFilter(prob["tables"], prob["dr"])
    vox = sample_voxels(np.random.default_rng(L), shape, 60 if L == 6 else 120)
    ref = conv_so3_at(prob["V"], F, radius, prob["Q"], vox).real
    err = rel_l2(got[tuple(vox.T)], ref)
    print(f"SO(3) conv {shape} L={L} R={radius}: relative L2 {err:.2e}")
    assert err <= 1e-5


def test_identity_and_constant_fields_over_the_whole_volume(ec, plan):
    """Identity field: ordinary convolution with F; a constant field: convolution
    with the rotated filter (both by numpy's FFT of the box samples)."""
    shape = (32, 32, 48)
    prob = synth.so3_conv_problem(seed=3, shape=shape, L=4, radius=5)
    F = SHFilter(prob["tables"], prob["dr"])
    dx, dy, dz = (c.astype(float) for c in box_offsets3(5))
    Q = np.zeros(shape + (4,), np.float32)
    Q[..., 0] = 1.0
    got = run(ec, plan, prob["V"], prob, Q)
    assert rel_l2(got, fft_conv(prob["V"], filter_eval(F, dx, dy, dz), 5)) <= 1e-5
    q = synth.haar_quaternion(np.random.default_rng(4))
    Q[:] = q.astype(np.float32)
    got = run(ec, plan, prob["V"], prob, Q)
    ref = fft_conv(prob["V"], rotated_filter_eval(F, quat_to_matrix(Q[0, 0, 0].astype(np.float64)), dx, dy, dz), 5)
    assert rel_l2(got, ref) <= 1e-5


def test_impulse_response_is_the_rotated_filter(ec, plan):
    shape = (32, 32, 32)
    prob = synth.so3_conv_problem(seed=5, shape=shape, L=6, radius=6)
    V = np.zeros(shape, np.float32)
    q0 = (7, 20, 30)
    V[q0] = 1.0
    got = run(ec, plan, V, prob, prob["Q"])
    F = SHFilter(prob["tables"], prob["dr"])
    dx, dy, dz = box_offsets3(6)
    Rm = quat_to_matrix(prob["Q"][q0].astype(np.float64))
    ref = np.zeros(shape)
    ref[(q0[0] + dz) % 32, (q0[1] + dy) % 32, (q0[2] + dx) % 32] = rotated_filter_eval(
        F, Rm, dx.astype(float), dy.astype(float), dz.astype(float)).real
    assert rel_l2(got, ref) <= 1e-5


def test_box_wider_than_the_volume_wraps(ec, plan):
    shape = (32, 32, 32)
    prob = synth.so3_conv_problem(seed=6, shape=shape, L=1, radius=20, dr=0.25)
    got = run(ec, plan, prob["V"], prob, prob["Q"])
    vox = sample_voxels(np.random.default_rng(6), shape, 12)
    ref = conv_so3_at(prob["V"], SHFilter(prob["tables"], prob["dr"]), 20, prob["Q"], vox).real
    assert rel_l2(got[tuple(vox.T)], ref) <= 1e-5


def test_degree_zero_ignores_the_field(ec, plan):
    shape = (32, 64, 32)
    prob = synth.so3_conv_problem(seed=7, shape=shape, L=0, radius=5)
    a = run(ec, plan, prob["V"], prob, prob["Q"])
    Q = np.zeros(shape + (4,), np.float32)
    Q[..., 0] = 1.0
    np.testing.assert_array_equal(a, run(ec, plan, prob["V"], prob, Q))


def test_chunked_components_match_oracle(ec, plan):
    """256^3 with L = 3 (44 unique entries) exceeds the workspace budget of
    modulated planes and runs in two chunks whose partial results are summed."""
    shape = (256, 256, 256)
    prob = synth.so3_conv_problem(seed=8, shape=shape, L=3, radius=4)
    got = run(ec, plan, prob["V"], prob, prob["Q"])
    vox = sample_voxels(np.random.default_rng(8), shape, 40)
    ref = conv_so3_at(prob["V"], SHFilter(prob["tables"], prob["dr"]), 4, prob["Q"], vox).real
    assert rel_l2(got[tuple(vox.T)], ref) <= 1e-5


def test_host_buffers_match_device(ec, plan):
    shape = (32, 32, 64)
    prob = synth.so3_conv_problem(seed=9, shape=shape, L=2, radius=4)
    a = run(ec, plan, prob["V"], prob, prob["Q"])
    b = np.zeros(shape, np.float32)
    ec.ext_conv_so3(plan, prob["V"], *shape, prob["tables"], prob["dr"], 4, prob["Q"], b)
    np.testing.assert_array_equal(a, b)


def test_rejects_bad_arguments(ec, plan):
    shape = (32, 32, 32)
    prob = synth.so3_conv_problem(seed=10, shape=shape, L=1, radius=3)
    out = np.zeros(shape, np.float32)
    Qd = dev(np.concatenate([prob["Q"].ravel(), np.zeros(1, np.float32)]))
    with pytest.raises(ec.ExtError):       # device field not 16-byte aligned
        ec.ext_conv_so3(plan, prob["V"], *shape, prob["tables"], prob["dr"], 3, Qd[1:], out)
    with pytest.raises(ec.ExtError):       # unsupported transform length
        ec.ext_conv_so3(plan, np.zeros((40, 32, 32), np.float32), 40, 32, 32, prob["tables"], prob["dr"], 3,
                        np.zeros((40, 32, 32, 4), np.float32), np.zeros((40, 32, 32), np.float32))
    tables7 = synth.so3_filter_tables(1, 7, 3.0, 0.25)
    with pytest.raises(ec.ExtError):       # degree above 6
        ec.ext_conv_so3(plan, prob["V"], *shape, tables7, 0.25, 3, prob["Q"], out)
