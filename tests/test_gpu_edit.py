"""Spectral editing on the GPU (lfa_spectral_edit) against the FP64 oracle's projection of the
edited operator onto the kernel taps. Tolerance: the backward's, relative 1e-4 in norm; the
exact full-support case by its spectrum, 1e-5 * sigma_max."""
import numpy as np
import pytest
import torch

import lfa_workloads as W
import oracle as O
from paper_2506_05617_gb300.torch_api import LfaPlan

from test_gpu_parity import rand_w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


def safe_threshold(s):
    """A threshold in the widest gap of the spectrum's middle, so fp32 and fp64 agree on each side."""
    v = np.sort(s.ravel())
    lo, hi = len(v) // 4, 3 * len(v) // 4
    k = lo + int(np.argmax(np.diff(v[lo:hi])))
    return 0.5 * (v[k] + v[k + 1])


@pytest.mark.parametrize("half", [False, True])
@pytest.mark.parametrize("shape", [(4, 4, 3, 3, 8, 8), (6, 3, 3, 3, 5, 7), (3, 5, 5, 3, 6, 6), (64, 64, 3, 3, 6, 6)])
@pytest.mark.parametrize("mode", ["clip", "clamp", "threshold", "rank"])
def test_spectral_edit_matches_oracle(shape, mode, half):
    c_out, c_in, kh, kw, n, m = shape
    w = rand_w(c_out, c_in, kh, kw, seed=51)
    s_ref = O.lfa_svd(w, n, m, compute_uv=False)
    smax = float(s_ref.max())
    a, b = {"clip": (0.7 * smax, 0.0), "clamp": (0.3 * smax, 0.8 * smax),
            "threshold": (safe_threshold(s_ref), 0.0), "rank": (max(1, min(c_out, c_in) // 2), 0.0)}[mode]
    plan = LfaPlan([shape], vectors=True, half_output=half)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    got = plan.spectral_edit(sig, U, V, mode, a, b)[0].cpu().numpy()
    ref = O.spectral_edit(w, n, m, mode, a, b)
    assert np.linalg.norm(got - ref) <= 1e-4 * max(np.linalg.norm(ref), 1e-30) + 1e-7
    plan.close()


def test_full_support_clip_is_exact():
    c, k = 8, 6
    w = rand_w(c, c, k, k, seed=52)
    s = O.lfa_svd(w, k, k, compute_uv=False)
    cap = 0.6 * float(s.max())
    plan = LfaPlan([(c, c, k, k, k, k)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    we = plan.spectral_edit(sig, U, V, "clip", cap)[0].cpu().numpy()
    s2 = O.lfa_svd(we, k, k, compute_uv=False)
    assert np.max(np.abs(np.sort(s2.ravel()) - np.sort(np.minimum(s, cap).ravel()))) <= 1e-5 * s.max()
    plan.close()


def test_conv64_n32_clip_full_size():
    lay = W.layers("conv64_k3_n32")[0]
    w = W.weights(lay)
    plan = LfaPlan([(lay.c_out, lay.c_in, lay.kh, lay.kw, lay.n, lay.m)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    got = plan.spectral_edit(sig, U, V, "clip", 1.0)[0].cpu().numpy()
    ref = O.spectral_edit(w, lay.n, lay.m, "clip", 1.0)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    plan.close()


@pytest.mark.parametrize("half", [False, True])
@pytest.mark.parametrize("shape", [(4, 4, 3, 3, 8, 8), (6, 3, 3, 3, 5, 7), (3, 5, 5, 3, 6, 6), (16, 16, 3, 3, 8, 8)])
def test_pseudo_inverse_projection_matches_oracle(shape, half):
    """Kernel of the c_out -> c_in convolution nearest to the pseudo-inverse (values <= a dropped).
    1/sigma amplifies the fp32 error of small values: the tolerance is 1e-4 * sigma_max / a."""
    c_out, c_in, kh, kw, n, m = shape
    w = rand_w(c_out, c_in, kh, kw, seed=53)
    s_ref = O.lfa_svd(w, n, m, compute_uv=False)
    v = np.sort(s_ref.ravel())
    lo, hi = len(v) // 5, 3 * len(v) // 5
    k = lo + int(np.argmax(np.diff(v[lo:hi])))
    a = 0.5 * (v[k] + v[k + 1])
    plan = LfaPlan([shape], vectors=True, half_output=half)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    got = plan.spectral_edit(sig, U, V, "pinv", a)[0].cpu().numpy()
    ref = O.pinv_projection(w, n, m, a)
    assert got.shape == (c_in, c_out, kh, kw)
    assert np.linalg.norm(got - ref) <= 1e-4 * (float(v[-1]) / a) * np.linalg.norm(ref)
    plan.close()


def test_pseudo_inverse_of_a_scaled_identity_is_exact_and_strided_layers_are_refused():
    from paper_2506_05617_gb300 import lfa as C
    w = np.zeros((5, 5, 3, 3), np.float32)
    w[:, :, 1, 1] = 2.0 * np.eye(5)
    plan = LfaPlan([(5, 5, 3, 3, 6, 4)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    got = plan.spectral_edit(sig, U, V, "pinv", 0.0)[0].cpu().numpy()
    ref = np.zeros_like(w)
    ref[:, :, 1, 1] = 0.5 * np.eye(5)
    assert np.max(np.abs(got - ref)) <= 1e-6
    plan.close()
    plan = LfaPlan([(4, 2, 3, 3, 4, 4, -1, -1, 2, 2)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(rand_w(4, 2, 3, 3, seed=54)).cuda()])
    with pytest.raises(C.LfaError) as ei:
        plan.spectral_edit(sig, U, V, "pinv", 0.0)
    assert ei.value.status == C.LFA_ERR_UNSUPPORTED
    plan.close()


@pytest.mark.parametrize("mode", ["clip", "pinv"])
def test_spectral_edit_on_the_tensor_core_route(mode):
    """A 128 -> 160 layer (both sides >= 128 channels): the edit's projection runs through the
    tensor-core G product (for the pseudo-inverse on the transposed layer, U and V exchanged)."""
    from paper_2506_05617_gb300 import lfa as C
    c_out, c_in, kh, kw, n, m = 160, 128, 3, 3, 2, 3
    assert C.lfa_debug_backward_route(c_out, c_in, kh, kw) == 2
    assert C.lfa_debug_backward_route(c_in, c_out, kh, kw) == 2
    w = rand_w(c_out, c_in, kh, kw, seed=53)
    s_ref = O.lfa_svd(w, n, m, compute_uv=False)
    plan = LfaPlan([(c_out, c_in, kh, kw, n, m)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    if mode == "clip":
        a = 0.7 * float(s_ref.max())
        got = plan.spectral_edit(sig, U, V, "clip", a)[0].cpu().numpy()
        ref = O.spectral_edit(w, n, m, "clip", a)
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    else:
        # threshold in the widest gap of the spectrum's lower part (fp32 and fp64 agree on each side);
        # 1/sigma amplifies the fp32 error of small values: tolerance 1e-4 * sigma_max / a
        v = np.sort(s_ref.ravel())
        lo, hi = len(v) // 5, 3 * len(v) // 5
        k = lo + int(np.argmax(np.diff(v[lo:hi])))
        a = 0.5 * (v[k] + v[k + 1])
        got = plan.spectral_edit(sig, U, V, "pinv", a)[0].cpu().numpy()
        ref = O.pinv_projection(w, n, m, a)
        assert np.linalg.norm(got - ref) <= 1e-4 * (float(v[-1]) / a) * np.linalg.norm(ref)
    plan.close()
