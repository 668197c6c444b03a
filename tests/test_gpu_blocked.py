"""The blocked Jacobi route on the tcgen05 tensor cores (options.variant = LFA_VARIANT_BLOCKED)
against the FP64 oracle, with the tolerances of test_gpu_parity: sigma within 1e-5 sigma_max,
||A v - sigma u|| <= 1e-5 sigma_max, U and V orthonormal to 1e-5, reconstruction."""
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


BLOCKED = [
    # c_out, c_in, k, n, m, vectors
    (128, 128, 3, 3, 2, True),     # one cluster of 2 CTAs
    (256, 256, 3, 2, 2, True),     # cluster of 4
    (512, 512, 3, 2, 2, True),     # cluster of 8, 512 x 512
    (512, 512, 3, 2, 2, False),
    (300, 200, 3, 2, 2, True),     # ragged: 300 rows, 200 columns padded to 384
    (200, 200, 1, 2, 3, True),
    (400, 130, 3, 2, 1, True),
    (384, 384, 3, 2, 2, True),     # cluster of 6
    (512, 512, 3, 4, 4, True),     # 10 symbols over the CTAs
    (200, 300, 3, 2, 2, True),     # wide: X = A^*, threshold capped at 2^-20
]


@pytest.mark.parametrize("spec", BLOCKED, ids=lambda s: "x".join(str(v) for v in s[:5]) + ("v" if s[5] else ""))
def test_blocked_route_matches_oracle(spec):
    c_out, c_in, k, n, m, vec = spec
    w = rand_w(c_out, c_in, k, k, seed=3 * c_out + c_in)
    plan = LfaPlan([(c_out, c_in, k, k, n, m)], vectors=vec, variant=C.LFA_VARIANT_BLOCKED)
    assert plan.meta[0]["variant"] == C.LFA_VARIANT_BLOCKED
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    s = sig[0].cpu().numpy()
    check_sigma(w, n, m, s)
    assert np.all(np.diff(s, axis=1) <= 0)
    if vec:
        half = O.half_grid(n, m)
        check_factors(O.symbols(w, n, m)[half], s[half], U[0].cpu().numpy(), V[0].cpu().numpy())
    print(f"{spec}: sweeps/symbol {info['sweeps'] / info['symbols']:.1f}, rotations {info['rotations']}")
    plan.close()


def test_blocked_route_is_the_default_for_wide_channel_layers():
    """Tall or square symbols of 256 to 512 columns take the blocked route by default (and with the
    committed autotuner cache) when the layer has enough symbols to fill the GPU (74 half-grid
    symbols at 12 x 12, 100 at 14 x 14, 34 at 8 x 8 for 384 columns); a 512-channel layer on 4 x 4 (10 symbols), 128 columns and
    wide symbols keep the element-wise kernels."""
    import os
    cache = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2506_05617_gb300", "tune_gb300.txt")
    for spec, vec, blocked in [((512, 512, 3, 3, 12, 12), True, True), ((512, 512, 3, 3, 12, 12), False, True),
                               ((256, 256, 3, 3, 14, 14), True, True), ((300, 256, 3, 3, 14, 14), True, True),
                               ((384, 384, 3, 3, 8, 8), False, True), ((192, 192, 3, 3, 14, 14), True, True),
                               ((512, 512, 3, 3, 4, 4), False, False), ((512, 512, 3, 3, 7, 7), False, False),
                               ((128, 128, 3, 3, 4, 4), True, False), ((256, 512, 3, 3, 14, 14), True, False)]:
        for tc in (None, cache):
            plan = LfaPlan([spec], vectors=vec, tune_cache=tc)
            assert (plan.meta[0]["variant"] == C.LFA_VARIANT_BLOCKED) == blocked, (spec, vec, tc)
            plan.close()


def test_blocked_layers_share_a_launch():
    """Layers whose symbols pad to the same size go through one blocked launch (items of several
    layers in one queue): two 256 x 256 layers, and a 300 x 256 and a 384 x 256 one (both padded to
    384 rows: a second launch shared by layers of different row counts) on 14 x 14, values and
    vectors, checked against the oracle on sampled half-grid frequencies of each layer."""
    specs = [(256, 256, 3, 3, 14, 14), (256, 256, 3, 3, 14, 14), (300, 256, 3, 3, 14, 14), (384, 256, 3, 3, 14, 14)]
    ws = [rand_w(co, ci, kh, kw, seed=90 + i) for i, (co, ci, kh, kw, n, m) in enumerate(specs)]
    plan = LfaPlan(specs, vectors=True)
    assert all(mt["variant"] == C.LFA_VARIANT_BLOCKED for mt in plan.meta)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    for i, ((co, ci, kh, kw, n, m), w) in enumerate(zip(specs, ws)):
        half = O.half_grid(n, m)
        pick = np.sort(np.random.default_rng(i).choice(len(half), 12, replace=False))
        f = half[pick]
        s = sig[i].cpu().numpy()
        s_ref = O.lfa_svd(w, n, m, compute_uv=False, freqs=f)
        smax = float(s_ref.max())
        assert np.max(np.abs(s[f].astype(np.float64) - s_ref)) <= 1e-5 * smax
        check_factors(O.symbols(w, n, m)[f], s[f], U[i].cpu().numpy()[pick], V[i].cpu().numpy()[pick])
    plan.close()


WARM = [
    # c_out, c_in, k, n, m
    (256, 256, 3, 8, 8),     # square
    (300, 200, 3, 8, 7),     # ragged: 200 columns padded to 256, K of the warm product 224
    (200, 300, 3, 7, 8),     # wide: X = A^*, the warm start takes U of the previous symbol
]


@pytest.mark.parametrize("spec", WARM, ids=lambda s: "x".join(str(v) for v in s))
def test_blocked_warm_starts_match_oracle(spec):
    """Warm starts: each symbol after the first of a run of neighbouring frequencies starts its
    sweeps from X = A W with W the previous symbol's V (the invariant X = A W holds for any
    starting W). Four CTAs and eight runs, so that most symbols find their predecessor done; the
    factors against the oracle as for cold starts, and fewer sweeps than the same layer with every
    symbol started from W = I."""
    c_out, c_in, k, n, m = spec
    w = rand_w(c_out, c_in, k, k, seed=7 * c_out + c_in)
    half = O.half_grid(n, m)
    sweeps = {}
    try:
        for runs in (8, -1):
            C.lfa_debug_set_bj_grid(4, runs)
            plan = LfaPlan([(c_out, c_in, k, k, n, m)], vectors=True, variant=C.LFA_VARIANT_BLOCKED)
            sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
            torch.cuda.synchronize()
            st, info = plan.info()
            assert st == C.LFA_OK, info
            prof, ctas = C.lfa_debug_bj_profile(plan.handle)
            assert ctas == 4
            if runs > 0:
                # runs of ceil(F_h / 8) symbols; the first symbol of each of the 8 runs starts cold
                assert prof["warm_starts"] >= len(half) // 2, (prof["warm_starts"], len(half))
            else:
                assert prof["warm_starts"] == 0
            s = sig[0].cpu().numpy()
            check_sigma(w, n, m, s)
            check_factors(O.symbols(w, n, m)[half], s[half], U[0].cpu().numpy(), V[0].cpu().numpy())
            sweeps[runs] = info["sweeps"]
            plan.close()
    finally:
        C.lfa_debug_set_bj_grid(0, 0)
    assert sweeps[8] < sweeps[-1], sweeps


def test_blocked_warm_start_runs_cross_layers_of_one_launch():
    """Runs of warm starts span the symbols of all layers of one blocked launch: a 256 -> 200 and a
    256 -> 256 layer (both padded to 256 x 256, one launch); a run that passes into the next layer
    starts that layer's first symbol cold (its predecessor has other columns). Four CTAs, eight
    runs; both layers against the oracle, and fewer sweeps than with cold starts only."""
    specs = [(256, 200, 3, 3, 8, 7), (256, 256, 3, 3, 7, 8)]
    ws = [rand_w(co, ci, kh, kw, seed=61 + i) for i, (co, ci, kh, kw, n, m) in enumerate(specs)]
    total = sum(len(O.half_grid(n, m)) for (_, _, _, _, n, m) in specs)
    sweeps = {}
    try:
        for runs in (8, -1):
            C.lfa_debug_set_bj_grid(4, runs)
            plan = LfaPlan(specs, vectors=True, variant=C.LFA_VARIANT_BLOCKED)
            assert all(mt["variant"] == C.LFA_VARIANT_BLOCKED for mt in plan.meta)
            sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
            torch.cuda.synchronize()
            st, info = plan.info()
            assert st == C.LFA_OK, info
            prof, _ = C.lfa_debug_bj_profile(plan.handle)
            if runs > 0:
                assert prof["warm_starts"] >= total // 2, (prof["warm_starts"], total)
            else:
                assert prof["warm_starts"] == 0
            for i, ((co, ci, kh, kw, n, m), w) in enumerate(zip(specs, ws)):
                s = sig[i].cpu().numpy()
                check_sigma(w, n, m, s)
                half = O.half_grid(n, m)
                check_factors(O.symbols(w, n, m)[half], s[half], U[i].cpu().numpy(), V[i].cpu().numpy())
            sweeps[runs] = info["sweeps"]
            plan.close()
    finally:
        C.lfa_debug_set_bj_grid(0, 0)
    assert sweeps[8] < sweeps[-1], sweeps
