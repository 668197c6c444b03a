"""Frequency-sharded plans (lfa_options_t.shard_rank / shard_count) on one GPU: each shard
decomposes its contiguous range of the half grid, and the shards' backward contributions sum to
the unsharded dL/dw (what one all-reduce over the ranks of a multi-GPU job computes).

Tolerances as in test_gpu_parity: sigma within 1e-5 sigma_max of the FP64 oracle; dL/dw within
1e-4 relative (fp32 sums over frequencies in another grouping)."""
import numpy as np
import pytest
import torch

import lfa_workloads as W
import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


@pytest.mark.parametrize("spec,R", [((16, 16, 3, 3, 9, 8), 3), ((64, 48, 3, 3, 16, 16), 2), ((128, 128, 5, 5, 6, 6), 4)])
def test_shards_match_oracle_and_sum_to_the_full_backward(spec, R):
    c_out, c_in, kh, kw, n, m = spec
    w = W.weights(W.Layer(c_out, c_in, kh, kw, n, m, "normal", 2.0, 90 + R))
    wt = torch.from_numpy(w).cuda()
    half = O.half_grid(n, m)
    s_ref = O.lfa_svd(w, n, m, compute_uv=False)[half]
    smax = float(s_ref.max())
    full = LfaPlan([spec], vectors=True, half_output=True)
    sig_f, U_f, V_f = full.svd([wt])
    g = torch.from_numpy(W.upstream_gradient(tuple(sig_f[0].shape), seed=3)).cuda()
    dw_full = full.backward([g], U_f, V_f)[0]
    total = torch.zeros_like(dw_full)
    covered = 0
    for r in range(R):
        F_h, first, count = C.lfa_debug_shard_range(n, m, r, R)
        plan = LfaPlan([spec], vectors=True, half_output=True, shard=(r, R))
        assert plan.meta[0]["F_h"] == count
        q = C.lfa_layer_query(plan.handle, 0, with_half_grid=True)
        assert np.array_equal(np.asarray(q["half_grid"]), half[first:first + count])
        sig, U, V = plan.svd([wt])
        torch.cuda.synchronize()
        st, info = plan.info()
        assert st == C.LFA_OK, info
        s = sig[0].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(s - s_ref[first:first + count])) <= 1e-5 * smax
        S = O.symbols(w, n, m)[half[first:first + count]]
        Uu, Vv = U[0].cpu().numpy().astype(np.complex128), V[0].cpu().numpy().astype(np.complex128)
        res = np.einsum("hoi,his->hos", S, Vv) - Uu * s[:, None, :]
        assert np.max(np.linalg.norm(res, axis=1)) <= 1e-5 * smax
        total += plan.backward([g[first:first + count]], U, V)[0]
        with pytest.raises(C.LfaError) as ei:                 # the max term spans every shard
            plan.regulariser_grad(sig, 1e-2)
        assert ei.value.status == C.LFA_ERR_UNSUPPORTED
        covered += count
        plan.close()
    torch.cuda.synchronize()
    assert covered == len(half)
    err = float(torch.linalg.norm(total - dw_full) / torch.linalg.norm(dw_full))
    assert err <= 1e-4, err
    full.close()
