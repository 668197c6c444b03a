"""Seeded random layers against the FP64 oracle: channel counts 1..40 (and 33..400), kernels 1..7
(also larger than the torus, so taps alias), tori 1..9 with n != m, any tap origin, strides 1..3,
both sigma layouts; values, vectors, the backward and the lifting. Tolerances as in
test_gpu_parity.py; the backward and the lifting are checked on the GPU's own factors (1e-5)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan

from test_gpu_parity import check_factors, SIG_TOL
from test_gpu_strided import full_grid, half_dsigma
import lfa_workloads as W

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
    Uh, Vh = U[0].cpu().numpy(), V[0].cpu().numpy()
    check_factors(S, s if half else s[hg], Uh, Vh)
    check_backward_and_lift(plan, spec, w, half, U, V, Uh, Vh)
    plan.close()


def check_backward_and_lift(plan, spec, w, half, U, V, Uh, Vh):
    """dL/dw against the oracle's formula on the same (GPU) factors, and lifted vectors against
    the oracle's lift of those factors (both well posed whatever basis the SVD chose)."""
    c_out, c_in, kh, kw, n, m, ph, pw, sh, sw = spec
    r = Uh.shape[2]
    g = W.upstream_gradient((n * m, r), seed=c_out + 3 * c_in)
    ds = torch.from_numpy(half_dsigma(g, n, m) if half else g).cuda()
    dw = plan.backward([ds], U, V)[0].cpu().numpy()
    Uf = full_grid(Uh.astype(np.complex128), n, m)
    Vf = full_grid(Vh.astype(np.complex128), n, m)
    ref = O.lfa_backward_strided(w, n, m, sh, sw, g, Uf, Vf, ph, pw)
    assert np.linalg.norm(dw - ref) <= 1e-5 * np.linalg.norm(ref) + 1e-6 * np.linalg.norm(w), spec
    f = (n * m) // 2
    j, l = divmod(f, m)
    uh, vh = plan.expand(0, U[0], V[0], f * r, r)
    ru, rv = O.lift_strided(Uf[f], Vf[f], j, l, n, m, sh, sw)
    assert np.max(np.abs(uh.cpu().numpy() - ru)) <= 2e-6, spec
    assert np.max(np.abs(vh.cpu().numpy() - rv)) <= 2e-6, spec


def random_large_layer(i):
    rng = np.random.default_rng(5000 + i)
    c_out, c_in = (int(x) for x in rng.integers(33, 401, size=2))
    k = int(rng.choice([1, 3]))
    n, m = (int(x) for x in rng.integers(1, 4, size=2))
    s = int(rng.choice([1, 1, 2]))
    if c_in * s * s > 512:
        s = 1
    w = (rng.standard_normal((c_out, c_in, k, k)) / np.sqrt(c_in * k * k)).astype(np.float32)
    return (c_out, c_in, k, k, n, m, -1, -1, s, s), w, bool(rng.integers(0, 2))


@pytest.mark.parametrize("i", range(12))
def test_random_large_layer_matches_oracle(i):
    """Channel counts 33..400 (cluster, rotation-log and completion kernels), values and vectors,
    backward and lifting on the GPU's own factors."""
    spec, w, half = random_large_layer(i)
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
    assert np.max(np.abs(s - ref)) <= SIG_TOL * float(s_ref.max()), spec
    S = O.symbols_strided(w, n, m, sh, sw, ph, pw)[hg]
    Uh, Vh = U[0].cpu().numpy(), V[0].cpu().numpy()
    check_factors(S, s if half else s[hg], Uh, Vh)
    check_backward_and_lift(plan, spec, w, half, U, V, Uh, Vh)
    plan.close()
