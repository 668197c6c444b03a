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


@pytest.mark.parametrize("half_output", [False, True])
@pytest.mark.parametrize("spec", [(64, 64, 3, 3, 32, 32), (5, 3, 3, 3, 6, 5), (3, 7, 5, 3, 7, 4),
                                  (12, 4, 3, 3, 5, 6, -1, -1, 2, 2)])
def test_noalloc_backward_matches_planned_backward_twice(spec, half_output):
    from paper_2506_05617_gb300.torch_api import LfaPlan
    c_out, c_in, kh, kw, n, m = spec[:6]
    w = np.random.default_rng(1).standard_normal((c_out, c_in, kh, kw)) / np.sqrt(c_in * kh * kw)
    w = torch.from_numpy(w.astype(np.float32)).cuda()
    plan = LfaPlan([spec], vectors=True, half_output=half_output)
    sig, U, V = plan.svd([w])
    flags = C.LFA_HALF_OUTPUT if half_output else 0
    stream = torch.cuda.current_stream()
    for call in range(2):
        g = torch.from_numpy(W.upstream_gradient(tuple(sig[0].shape), seed=10 + call)).cuda()
        ref = plan.backward([g], U, V)[0]
        dw = torch.full_like(ref, float("nan"))
        C.lfa_svd_backward_noalloc(spec, flags, g.data_ptr(), U[0].data_ptr(), V[0].data_ptr(), dw.data_ptr(),
                                   stream)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(dw - ref) / torch.linalg.norm(ref))
        assert err <= REL_TOL, (call, err)
    plan.close()


def test_noalloc_rejects_layers_beyond_the_scratch_size():
    with pytest.raises(C.LfaError) as ei:
        C.lfa_svd_backward_noalloc((512, 512, 3, 3, 64, 64), 0, 1, 1, 1, 1, None)
    assert ei.value.status == C.LFA_ERR_UNSUPPORTED
