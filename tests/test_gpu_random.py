"""Seeded random layers against the FP64 oracle: channel counts 1..40, kernels 1..7 (also larger
than the torus, so taps alias), tori 1..9 with n != m, any tap origin, strides 1..3, both sigma
layouts, values and vectors. Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan

from test_gpu_parity import check_factors, SIG_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


def random_layer(i):
    rng = np.random.default_rng(1000 + i)
    c_out, c_in = (int(x) for x in rng.integers(1, 41, size=2))
    kh, kw = (int(x) for x in rng.integers(1, 8, size=2))
    n, m = (int(x) for x in rng.integers(1, 10, size=2))
    ph, pw = int(rng.integers(-1, kh)), int(rng.integers(-1, kw))
    sh, sw = (int(x) for x in rng.choice([1, 1, 1, 2, 3], size=2))
    while c_in * sh * sw > 512:
        sh, sw = 1, 1
    w = (rng.standard_normal((c_out, c_in, kh, kw)) / np.sqrt(c_in * kh * kw)).astype(np.float32)
    return (c_out, c_in, kh, kw, n, m, ph, pw, sh, sw), w, bool(rng.integers(0, 2))


@pytest.mark.parametrize("i", range(40))
def test_random_layer_matches_oracle(i):
    spec, w, half = random_layer(i)
    c_out, c_in, kh, kw, n, m, ph, pw, sh, sw = spec
    plan = LfaPlan([spec], vectors=True, half_output=half)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, (spec, info)
    s_ref = O.lfa_svd_strided(w, n, m, sh, sw, ph, pw, compute_uv=False)
    hg = O.half_grid(n, m)
    s = sig[0].cpu().numpy()
    ref = s_ref[hg] if half else s_ref
    assert s.shape == ref.shape, spec
    smax = max(float(s_ref.max()), 1e-30)
    assert np.max(np.abs(s - ref)) <= SIG_TOL * smax, spec
    S = O.symbols_strided(w, n, m, sh, sw, ph, pw)[hg]
    check_factors(S, s if half else s[hg], U[0].cpu().numpy(), V[0].cpu().numpy())
    plan.close()
