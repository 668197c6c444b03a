"""Every register-resident Jacobi variant, forced on a ragged problem that fills most of its
capacity, against the FP64 oracle (values, and vectors where the variant holds them).

Covers the variants the built-in choice never picks (those with two teams per thread, which
only the autotuner selects) as well as the cluster variants."""
import re

import numpy as np
import pytest
import torch

from paper_2506_05617_gb300 import lfa as C

from test_gpu_parity import check_sigma, check_vectors, gpu_svd, rand_w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


def shape_for(v, vectors):
    npairs, lanes, mr, wr, cs, ppt = (int(x) for x in re.findall(r"\d+", C.lfa_variant_name(v)))
    rows = mr * lanes
    cols = min(2 * npairs, wr * lanes) if vectors else 2 * npairs
    c_out = rows if rows <= 8 else rows - 3
    c_in = min(cols, c_out)
    c_in = c_in - 1 if c_in > 4 else c_in
    return c_out, c_in


@pytest.mark.parametrize("vectors", [False, True], ids=["values", "vectors"])
@pytest.mark.parametrize("v", range(C.lfa_debug_variant_count()), ids=lambda v: C.lfa_variant_name(v))
def test_forced_variant_matches_oracle(v, vectors):
    c_out, c_in = shape_for(v, vectors)
    n, m = 3, 2
    w = rand_w(c_out, c_in, 3, 3, seed=100 + v)
    plan, (s, U, V), st, info = gpu_svd(w, n, m, vectors=vectors, variant=v)
    if plan.meta[0]["variant"] != v:
        plan.close()
        pytest.skip("variant not instantiated for this mode")
    assert st == C.LFA_OK, info
    check_sigma(w, n, m, s)
    assert np.all(np.diff(s, axis=1) <= 0)
    if vectors:
        check_vectors(w, n, m, s, U, V)
    plan.close()


def logged_variants():
    out = []
    for v in range(C.lfa_debug_variant_count()):
        npairs, lanes, mr, wr, cs, ppt = (int(x) for x in re.findall(r"\d+", C.lfa_variant_name(v)))
        if ppt == 1 and npairs in (16, 32, 64, 128, 256) and npairs * lanes // cs >= 32:
            out.append(v)
    return out


@pytest.mark.parametrize("v", logged_variants(), ids=lambda v: C.lfa_variant_name(v) + "_log")
def test_forced_rotation_log_route_matches_oracle(v):
    """Vectors through the values-mode forward with the rotation log, the W replay, the finalize
    and the zero-column completion, forced on every variant that has a replay configuration."""
    c_out, c_in = shape_for(v, vectors=False)
    c_in = min(c_in, 512)
    n, m = 3, 2
    w = rand_w(c_out, c_in, 3, 3, seed=200 + v)
    plan, (s, U, V), st, info = gpu_svd(w, n, m, vectors=True, variant=v | C.LFA_VARIANT_LOGGED)
    assert plan.meta[0]["variant"] == v | C.LFA_VARIANT_LOGGED, plan.meta[0]
    assert st == C.LFA_OK, info
    check_sigma(w, n, m, s)
    assert np.all(np.diff(s, axis=1) <= 0)
    check_vectors(w, n, m, s, U, V)
    plan.close()
