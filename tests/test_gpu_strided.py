"""Parity of strided convolutions (crystals: the fine input's s_h s_w polyphase components per
coarse cell, symbol c_out x c_in s_h s_w) between the CUDA path and the FP64 oracle.

Tolerances as in test_gpu_parity.py: sigma within 1e-5 * sigma_max; vectors by residuals,
reconstruction and orthonormality; symbols elementwise 1e-6 * max|A_k|; dL/dw relative 1e-4."""
import numpy as np
import pytest
import torch

import lfa_workloads as W
import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan, LfaSvd

from test_gpu_parity import check_factors, rand_w, SIG_TOL, VEC_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


STRIDED = [
    # c_out, c_in, kh, kw, n, m, sh, sw, vectors
    (8, 4, 3, 3, 5, 4, 2, 2, True),       # 8 x 16 (wide)
    (32, 8, 3, 3, 6, 6, 2, 2, True),      # 32 x 32
    (64, 3, 7, 7, 12, 10, 2, 2, True),    # stem-like, tall 64 x 12
    (16, 16, 3, 3, 4, 5, 2, 1, True),     # stride along one axis: 16 x 32
    (24, 6, 5, 5, 3, 3, 3, 3, True),      # stride 3: 24 x 54
    (16, 8, 1, 1, 4, 4, 2, 2, True),      # 1x1 stride 2: three of four components untouched (zero columns)
    (12, 4, 4, 4, 5, 5, 2, 2, True),      # even kernel
    (5, 2, 3, 3, 1, 1, 2, 2, True),       # a single coarse frequency
    (6, 3, 5, 5, 2, 3, 2, 2, True),       # taps alias on the fine torus (5 > 2 * 2)
    (128, 64, 3, 3, 3, 4, 2, 2, True),    # 128 x 256: cluster kernel
    (256, 128, 3, 3, 2, 3, 2, 2, False),  # 256 x 512 values
    (256, 128, 3, 3, 2, 2, 2, 2, True),   # 256 x 512 vectors: rotation log + replay
    (128, 64, 1, 1, 3, 3, 2, 2, True),    # 128 x 256 of rank 64: cluster kernel + completion
    (256, 128, 1, 1, 2, 2, 2, 2, True),   # 256 x 512 of rank 128: rotation log + completion
]


def ids(s):
    return "x".join(str(v) for v in s[:6]) + f"s{s[6]}{s[7]}" + ("v" if s[8] else "")


def strided_plan(w, n, m, sh, sw, **kw):
    c_out, c_in, kh, kw_ = w.shape
    return LfaPlan([(c_out, c_in, kh, kw_, n, m, -1, -1, sh, sw)], **kw)


def run(w, n, m, sh, sw, **kw):
    plan = strided_plan(w, n, m, sh, sw, **kw)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    return plan, sig[0], (U[0] if U else None), (V[0] if V else None)


@pytest.mark.parametrize("spec", STRIDED, ids=ids)
def test_strided_svd_matches_oracle(spec):
    c_out, c_in, kh, kw, n, m, sh, sw, vec = spec
    w = rand_w(c_out, c_in, kh, kw, seed=c_out * 13 + c_in + kh)
    plan, s, U, V = run(w, n, m, sh, sw, vectors=vec)
    s = s.cpu().numpy()
    s_ref = O.lfa_svd_strided(w, n, m, sh, sw, compute_uv=False)
    assert s.shape == s_ref.shape == (n * m, min(c_out, c_in * sh * sw))
    smax = float(s_ref.max())
    assert np.max(np.abs(s - s_ref)) <= SIG_TOL * smax
    assert np.all(np.diff(s, axis=1) <= 0)
    if vec:
        half = O.half_grid(n, m)
        S = O.symbols_strided(w, n, m, sh, sw)[half]
        check_factors(S, s[half], U.cpu().numpy(), V.cpu().numpy())
    plan.close()


@pytest.mark.parametrize("spec", [STRIDED[0], STRIDED[2], STRIDED[4], STRIDED[9]], ids=ids)
def test_strided_plain_path_and_symbols(spec):
    c_out, c_in, kh, kw, n, m, sh, sw, _ = spec
    w = rand_w(c_out, c_in, kh, kw, seed=3)
    plan, s, _, _ = run(w, n, m, sh, sw, vectors=False, plain=True)
    s_ref = O.lfa_svd_strided(w, n, m, sh, sw, compute_uv=False)
    assert np.max(np.abs(s.cpu().numpy() - s_ref)) <= SIG_TOL * s_ref.max()
    A = plan.symbols(0, torch.from_numpy(w).cuda()).cpu().numpy()
    A_ref = O.symbols_strided(w, n, m, sh, sw)[O.half_grid(n, m)]
    assert A.shape == A_ref.shape
    assert np.max(np.abs(A - A_ref)) <= 1e-6 * np.max(np.abs(A_ref))
    plan.close()


def test_strided_padding_origin():
    w = rand_w(6, 3, 3, 4, seed=9)
    n, m, sh, sw = 4, 3, 2, 2
    plan = LfaPlan([(6, 3, 3, 4, n, m, 0, 3, sh, sw)], vectors=False)
    s = plan.svd([torch.from_numpy(w).cuda()])[0][0].cpu().numpy()
    s_ref = O.lfa_svd_strided(w, n, m, sh, sw, 0, 3, compute_uv=False)
    assert np.max(np.abs(s - s_ref)) <= SIG_TOL * s_ref.max()
    plan.close()


def test_strided_lifted_vectors_are_singular_pairs_of_the_dense_operator():
    c_out, c_in, k, n, m, sh, sw = 6, 2, 3, 3, 4, 2, 2
    w = rand_w(c_out, c_in, k, k, seed=11)
    plan, s, U, V = run(w, n, m, sh, sw, vectors=True)
    r = s.shape[1]
    uh, vh = plan.expand(0, U, V, 0, n * m * r)
    assert tuple(vh.shape) == (n * m * r, c_in, sh * n, sw * m)
    A = O.dense_operator_strided(w.astype(np.float64), n, m, sh, sw)
    uh = uh.cpu().numpy().reshape(n * m * r, -1).astype(np.complex128)
    vh = vh.cpu().numpy().reshape(n * m * r, -1).astype(np.complex128)
    sv = s.cpu().numpy().reshape(-1).astype(np.float64)
    smax = sv.max()
    assert np.max(np.linalg.norm(vh @ A.T - sv[:, None] * uh, axis=1)) <= 2 * VEC_TOL * smax
    assert np.max(np.abs(np.linalg.norm(vh, axis=1) - 1)) <= VEC_TOL
    # against the oracle's lift of the GPU's own factors (same phases): elementwise
    Uc, Vc = U.cpu().numpy(), V.cpu().numpy()
    half = list(O.half_grid(n, m))
    for f in (0, 5, 7):
        j, l = divmod(f, m)
        ref_u, ref_v = O.lift_strided(Uc[half.index(f)], Vc[half.index(f)], j, l, n, m, sh, sw)
        np.testing.assert_allclose(vh[f * r:(f + 1) * r], ref_v.reshape(r, -1), atol=2e-6)
        np.testing.assert_allclose(uh[f * r:(f + 1) * r], ref_u.reshape(r, -1), atol=2e-6)
    plan.close()


def full_grid(X, n, m):
    """Factors of every frequency from the half-grid ones: X_{-k} = conj(X_k)."""
    half = list(O.half_grid(n, m))
    pos = {f: i for i, f in enumerate(half)}
    out = []
    for f in range(n * m):
        fc = ((-(f // m)) % n) * m + (-(f % m)) % m
        out.append(X[pos[f]] if f in pos else np.conj(X[pos[fc]]))
    return np.stack(out)


def half_dsigma(g, n, m):
    """Half-grid dL/dsigma: a half-grid row stands for its conjugate pair, g~ = g_f + g_fc."""
    half = O.half_grid(n, m)
    fc = [((-(f // m)) % n) * m + (-(f % m)) % m for f in half]
    return np.stack([g[f] + (g[c] if c != f else 0) for f, c in zip(half, fc)]).astype(np.float32)


@pytest.mark.parametrize("half_output", [False, True])
@pytest.mark.parametrize("shape", [(8, 4, 3, 3, 5, 4, 2, 2), (24, 6, 5, 5, 3, 3, 3, 3), (64, 3, 7, 7, 6, 5, 2, 2),
                                   (16, 8, 1, 1, 4, 4, 2, 2), (128, 64, 3, 3, 3, 3, 2, 2)],
                         ids=lambda s: "x".join(map(str, s)))
def test_strided_backward_matches_oracle(shape, half_output):
    """The kernel's dL/dw against the oracle's formula on the same (GPU) factors, tightly; and the
    whole forward + backward against the oracle's own SVD where r is small. (With many singular
    values a random per-index dL/dsigma makes dL/dw depend on the basis chosen inside nearly
    degenerate singular subspaces, so only the first comparison is well posed there.)"""
    c_out, c_in, kh, kw, n, m, sh, sw = shape
    w = rand_w(c_out, c_in, kh, kw, seed=17)
    plan, s, U, V = run(w, n, m, sh, sw, vectors=True, half_output=half_output)
    r = min(c_out, c_in * sh * sw)
    g = W.upstream_gradient((n * m, r), seed=19)
    ds = torch.from_numpy(half_dsigma(g, n, m) if half_output else g).cuda()
    dw = plan.backward([ds], [U], [V])[0].cpu().numpy()
    Uf = full_grid(U.cpu().numpy().astype(np.complex128), n, m)
    Vf = full_grid(V.cpu().numpy().astype(np.complex128), n, m)
    dw_same = O.lfa_backward_strided(w, n, m, sh, sw, g, Uf, Vf)
    assert np.linalg.norm(dw - dw_same) / np.linalg.norm(dw_same) <= 1e-5
    if r <= 32:
        s_ref, U_ref, V_ref = O.lfa_svd_strided(w, n, m, sh, sw)
        dw_ref = O.lfa_backward_strided(w, n, m, sh, sw, g, U_ref, V_ref)
        assert np.linalg.norm(dw - dw_ref) / np.linalg.norm(dw_ref) <= 1e-4
    plan.close()


def test_strided_autograd_and_sum_of_squares_gradient():
    """d/dw sum sigma^2 = 2 n m w when taps do not alias (Parseval), through autograd."""
    c_out, c_in, k, n, m, sh, sw = 32, 8, 3, 6, 6, 2, 2
    w = torch.from_numpy(rand_w(c_out, c_in, k, k, seed=23)).cuda().requires_grad_(True)
    plan = strided_plan(w.detach().cpu().numpy(), n, m, sh, sw, vectors=True)
    (sig,) = LfaSvd.apply(plan, w)
    (sig ** 2).sum().backward()
    ref = 2 * n * m * w.detach()
    assert torch.linalg.norm(w.grad - ref) / torch.linalg.norm(ref) <= 1e-4
    plan.close()


def test_strided_spectral_edit_full_support_is_exact():
    """No two taps alias on the fine torus, so each tap's operator has n m unit entries that no
    other tap shares and the projection is exact: clip(inf) leaves the operator, and w, as it is."""
    c_out, c_in, k, n, m, sh, sw = 16, 4, 3, 5, 4, 2, 2
    w = rand_w(c_out, c_in, k, k, seed=29)
    plan, s, U, V = run(w, n, m, sh, sw, vectors=True)
    out = plan.spectral_edit([s], [U], [V], "clip", 1e30)[0].cpu().numpy()
    assert np.max(np.abs(out - w)) <= 1e-5 * np.max(np.abs(w))
    plan.close()


def test_resnet18_strided_layers_full_size():
    """The stride-2 layers of a ResNet-18 (stem 7x7 on 224, stage 2/3 3x3 and 1x1 shortcuts) in one
    plan with vectors and backward: sampled sigma against the oracle, Parseval, and the closed-form
    gradient of sum sigma^2."""
    lays = W.layers("resnet18_strided")
    ws = [W.weights(l) for l in lays]
    plan = LfaPlan([l.desc() for l in lays], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    dw = plan.backward([2 * s for s in sig], U, V)
    for i, (l, w) in enumerate(zip(lays, ws)):
        s = sig[i].cpu().numpy()
        assert s.shape == (l.F, l.r)
        fr = np.sort(np.random.default_rng(i).choice(l.F, 8, replace=False))
        s_ref = O.lfa_svd_strided(w, l.n, l.m, l.sh, l.sw, compute_uv=False, freqs=fr)
        assert np.max(np.abs(s[fr] - s_ref)) <= SIG_TOL * float(s.max())
        np.testing.assert_allclose(np.sum(s.astype(np.float64) ** 2),
                                   l.n * l.m * np.sum(w.astype(np.float64) ** 2), rtol=2e-5)
        ref = 2 * l.n * l.m * w.astype(np.float64)
        assert np.linalg.norm(dw[i].cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-4
    plan.close()
