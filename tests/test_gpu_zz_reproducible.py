"""LFA_REPRODUCIBLE: with vectors the blocked route normally warm-starts a symbol from its
neighbouring frequency's V when that symbol is already done, so which symbols start warm depends
on timing. With the flag every symbol starts from W = I: no warm starts, bitwise identical
results from call to call, the same tolerance to the FP64 oracle (test_gpu_parity's)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan

from test_gpu_parity import check_factors, check_sigma, rand_w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


def test_reproducible_flag_turns_warm_starts_off_and_repeats_bitwise():
    c_out, c_in, k, n, m = 256, 256, 3, 8, 8
    w = torch.from_numpy(rand_w(c_out, c_in, k, k, seed=71)).cuda()
    try:
        # four CTAs and eight runs: without the flag most symbols of this layer start warm
        C.lfa_debug_set_bj_grid(4, 8)
        plan = LfaPlan([(c_out, c_in, k, k, n, m)], vectors=True, variant=C.LFA_VARIANT_BLOCKED,
                       reproducible=True)
        outs = []
        for _ in range(2):
            sig, U, V = plan.svd([w])
            torch.cuda.synchronize()
            st, info = plan.info()
            assert st == C.LFA_OK, info
            prof, _ = C.lfa_debug_bj_profile(plan.handle)
            assert prof["warm_starts"] == 0
            outs.append([t[0].cpu().numpy().copy() for t in (sig, U, V)])
        plan.close()
    finally:
        C.lfa_debug_set_bj_grid(0, 0)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    s, U, V = outs[0]
    wn = w.cpu().numpy()
    check_sigma(wn, n, m, s)
    half = O.half_grid(n, m)
    check_factors(O.symbols(wn, n, m)[half], s[half], U, V)
