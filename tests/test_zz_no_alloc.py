"""lfa_svd_backward_noalloc: the backward pass for callers that cannot call cudaMalloc
(their device memory belongs to another allocator, or they cannot afford the device
synchronisation an allocation may cause). It must give what lfa_svd_backward gives, on
consecutive calls that reuse its fixed scratch array.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest
import torch

import lfa_workloads as W
from paper_2506_05617_gb300 import lfa as C

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4   # the tolerance of the backward parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


SPECS = [(64, 64, 3, 3, 32, 32), (5, 3, 3, 3, 6, 5), (3, 7, 5, 3, 7, 4),
         (12, 4, 3, 3, 5, 6, -1, -1, 2, 2),     # strided: the G route
         (64, 3, 7, 7, 16, 16),                 # stride 1 with 49 taps: the G route
         (512, 512, 3, 3, 7, 7)]                # the ResNet-18 body's 512@7 layer: fused, 28 MB of partials


def _rand_w(spec, seed):
    c_out, c_in, kh, kw = spec[:4]
    w = np.random.default_rng(seed).standard_normal((c_out, c_in, kh, kw)) / np.sqrt(c_in * kh * kw)
    return torch.from_numpy(w.astype(np.float32)).cuda()


def _check(plan, spec, U, V, sig_shape, flags, seed):
    g = torch.from_numpy(W.upstream_gradient(tuple(sig_shape), seed=seed)).cuda()
    ref = plan.backward([g], U, V)[0]
    dw = torch.full_like(ref, float("nan"))
    C.lfa_svd_backward_noalloc(spec, flags, g.data_ptr(), U[0].data_ptr(), V[0].data_ptr(), dw.data_ptr(),
                               torch.cuda.current_stream())
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(dw - ref) / torch.linalg.norm(ref))
    assert err <= REL_TOL, (spec, seed, err)


@pytest.mark.parametrize("half_output", [False, True])
@pytest.mark.parametrize("spec", SPECS, ids=lambda s: "x".join(str(v) for v in s))
def test_noalloc_backward_matches_planned_backward_twice(spec, half_output):
    from paper_2506_05617_gb300.torch_api import LfaPlan
    plan = LfaPlan([spec], vectors=True, half_output=half_output)
    sig, U, V = plan.svd([_rand_w(spec, 1)])
    flags = C.LFA_HALF_OUTPUT if half_output else 0
    for call in range(2):
        _check(plan, spec, U, V, sig[0].shape, flags, 10 + call)
    plan.close()


def test_noalloc_alternating_layers_ignore_stale_scratch():
    """Large, small, large, ...: each call must rebuild every table and partial sum it reads, whatever
    the previous call (another frequency count, chunking, route or layout) left in the array."""
    from paper_2506_05617_gb300.torch_api import LfaPlan
    order = [SPECS[0], SPECS[1], SPECS[4], SPECS[3], SPECS[0], SPECS[4], SPECS[1], SPECS[3], SPECS[0]]
    plans = {}
    for i, spec in enumerate(order):
        if spec not in plans:
            plan = LfaPlan([spec], vectors=True)
            plans[spec] = (plan,) + tuple(plan.svd([_rand_w(spec, 3)]))
        plan, sig, U, V = plans[spec]
        _check(plan, spec, U, V, sig[0].shape, 0, 100 + i)
    for p in plans.values():
        p[0].close()


def test_noalloc_rejects_layers_beyond_the_scratch_size():
    # 512 x 512 with 7 x 7 taps: one chunk of partial sums is 51 MB, more than the array holds
    with pytest.raises(C.LfaError) as ei:
        C.lfa_svd_backward_noalloc((512, 512, 7, 7, 64, 64), 0, 1, 1, 1, 1, None)
    assert ei.value.status == C.LFA_ERR_UNSUPPORTED
