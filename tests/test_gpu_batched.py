"""The largest plan (64 layers) of mixed small shapes, kernel sizes, strides and tori in one
batched, graph-replayed forward with vectors and one backward, layer by layer against the FP64
oracle (sigma within 1e-5 sigma_max, dL/dw relative 1e-4)."""
import numpy as np
import pytest
import torch

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


def layer_specs():
    rng = np.random.default_rng(9)
    specs = []
    for i in range(64):
        c_out, c_in = (int(x) for x in rng.integers(1, 17, size=2))
        k = int(rng.choice([1, 3, 5]))
        n, m = (int(x) for x in rng.integers(2, 7, size=2))
        s = 2 if (i % 8 == 7 and c_in * 4 <= 512) else 1
        specs.append((c_out, c_in, k, k, n, m, -1, -1, s, s))
    return specs


def test_sixty_four_mixed_layers_in_one_plan():
    specs = layer_specs()
    ws = [(np.random.default_rng(100 + i).standard_normal(sp[:4]) / np.sqrt(sp[1] * sp[2] * sp[3]))
          .astype(np.float32) for i, sp in enumerate(specs)]
    plan = LfaPlan(specs, vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    dsig = [torch.ones_like(s) for s in sig]
    dw = plan.backward(dsig, U, V)
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    for sp, w, s, g in zip(specs, ws, sig, dw):
        c_out, c_in, kh, kw, n, m, _, _, sh, sw = sp
        if sh == 1:
            s_ref, U_ref, V_ref = O.lfa_svd(w, n, m)
            dw_ref = O.lfa_backward(w, n, m, np.ones_like(s_ref), U_ref, V_ref)
        else:
            s_ref, U_ref, V_ref = O.lfa_svd_strided(w, n, m, sh, sw)
            dw_ref = O.lfa_backward_strided(w, n, m, sh, sw, np.ones_like(s_ref), U_ref, V_ref)
        s = s.cpu().numpy()
        assert s.shape == s_ref.shape, sp
        assert np.max(np.abs(s - s_ref)) <= 1e-5 * max(float(s_ref.max()), 1e-30), sp
        # d(sum sigma)/dw = sum_k Re(U_k V_k^* e^{-i theta y}) involves the polar factor U V^*, which
        # is unique when no singular value vanishes: compare where the symbols have full rank
        if s_ref.min() > 1e-3 * s_ref.max():
            got = g.cpu().numpy()
            assert np.linalg.norm(got - dw_ref) <= 1e-4 * np.linalg.norm(dw_ref) + 1e-6, sp
    plan.close()
