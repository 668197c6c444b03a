"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic, stated by the method's accuracy target):
  * singular values: |sigma_gpu - sigma_oracle| <= 1e-5 * sigma_max, per frequency, sorted;
  * singular vectors (not unique: phases, degenerate subspaces): orthonormality
    ||U^* U - I||_max <= 1e-5 (same for V) and ||A_k v - sigma u|| <= 1e-5 * sigma_max for every
    shape (the relation the method's accuracy target names). One-sided Jacobi on X = A_k
    (c_out >= c_in) keeps A_k w = x exactly up to rounding; for wide symbols it works on
    X = A_k^* and keeps A_k^* u = sigma v exactly, while A_k v - sigma u is bounded by the final
    column orthogonality, tau ||A_k||_F, which the library's threshold for wide symbols
    (at most 2^-20) keeps below 1e-5 sigma_max. The other relation, A_k^* u - sigma v for tall
    symbols, has that bound with tau = max(2^-22, 4 sqrt(M) 2^-24) and is checked against
    max(1e-5 sigma_max, 1.5 tau ||A_k||_F);
    reconstruction ||A_k - U S V^*||_max <= 1e-5 * sigma_max * max(1, r/64): every entry of the
    reconstruction sums r column contributions whose fp32 rounding grows with the ~r * sweeps
    rotations each column takes, so the bound scales with r beyond the 64-column symbols;
  * symbols (unique): elementwise <= 1e-6 * max|A_k| (one fp32 rounding per tap);
  * dL/dw: ||dw_gpu - dw_oracle|| / ||dw_oracle|| <= 1e-4, and <= 1e-3 against FP64 central
    finite differences.
"""
import os

import numpy as np
import pytest
import torch

import lfa_workloads as W
import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan

pytestmark = pytest.mark.gpu

SIG_TOL = 1e-5
VEC_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


def rand_w(c_out, c_in, kh, kw, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((c_out, c_in, kh, kw)) * scale / np.sqrt(c_in * kh * kw)).astype(np.float32)


def gpu_svd(w, n, m, pad=(-1, -1), vectors=True, half_output=False, **kw):
    c_out, c_in, kh, kw_ = w.shape
    plan = LfaPlan([(c_out, c_in, kh, kw_, n, m) + tuple(pad)], vectors=vectors, half_output=half_output, **kw)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    torch.cuda.synchronize()
    st, info = plan.info()
    out = (sig[0].cpu().numpy(), U[0].cpu().numpy() if U else None, V[0].cpu().numpy() if V else None)
    return plan, out, st, info


def check_sigma(w, n, m, s_gpu, pad=(-1, -1), half=None):
    s_ref = O.lfa_svd(w, n, m, *pad, compute_uv=False)
    smax = max(float(s_ref.max()), 1e-30)
    if half is not None:
        s_ref = s_ref[half]
    err = np.max(np.abs(s_gpu.astype(np.float64) - s_ref)) if s_ref.size else 0.0
    assert err <= SIG_TOL * smax, f"sigma err {err / smax:.3e} * sigma_max"
    return err / smax


def check_vectors(w, n, m, s_full, U, V, pad=(-1, -1)):
    half = O.half_grid(n, m)
    check_factors(O.symbols(w, n, m, *pad)[half], s_full[half], U, V)


def check_factors(S, s, U, V):
    """Singular triplets (s, U, V) of the half-grid symbols S [F_h, c_out, c_in] (see the header)."""
    s = s.astype(np.float64)
    smax = max(float(np.max(s)), 1e-30)
    U = U.astype(np.complex128)
    V = V.astype(np.complex128)
    r = s.shape[1]
    c_out, c_in = S.shape[1], S.shape[2]
    rec = np.einsum("hos,hs,his->hoi", U, s, np.conj(V))
    res_f = np.einsum("hoi,his->hos", S, V) - U * s[:, None, :]               # A v - sigma u
    res_a = np.einsum("hoi,hos->his", np.conj(S), U) - V * s[:, None, :]      # A^* u - sigma v
    eye = np.eye(r)
    M = max(c_out, c_in)
    tau = max(2.0 ** -22, 4.0 * np.sqrt(M) * 2.0 ** -24)
    fro = float(np.max(np.linalg.norm(S.reshape(S.shape[0], -1), axis=1)))
    # A^* u - sigma v: exact for wide symbols, bounded by tau ||A_k||_F for tall ones
    adj_bound = smax if c_out < c_in else max(smax, 1.5 * tau * fro / VEC_TOL)
    errs = {
        "reconstruction": np.max(np.abs(rec - S)) / smax / max(1.0, r / 64),
        "residual A v - sigma u": np.max(np.linalg.norm(res_f, axis=1)) / smax,
        "residual A^* u - sigma v": np.max(np.linalg.norm(res_a, axis=1)) / adj_bound,
        "U orthonormality": np.max(np.abs(np.einsum("hos,hot->hst", np.conj(U), U) - eye)),
        "V orthonormality": np.max(np.abs(np.einsum("hos,hot->hst", np.conj(V), V) - eye)),
    }
    assert all(v <= VEC_TOL for v in errs.values()), "; ".join(f"{k} {v:.2e}" for k, v in errs.items())


SHAPES = [
    # c_out, c_in, kh, kw, n, m, pad
    (4, 4, 3, 3, 8, 8, (-1, -1)),
    (3, 5, 3, 3, 5, 7, (-1, -1)),
    (5, 3, 3, 3, 6, 5, (-1, -1)),
    (1, 1, 3, 3, 7, 4, (-1, -1)),
    (1, 1, 1, 1, 1, 1, (-1, -1)),
    (7, 7, 5, 5, 4, 3, (-1, -1)),     # taps alias (k > n)
    (16, 16, 3, 3, 9, 9, (-1, -1)),
    (32, 32, 3, 3, 8, 8, (-1, -1)),
    (64, 64, 3, 3, 8, 8, (-1, -1)),
    (64, 3, 7, 7, 12, 12, (-1, -1)),  # tall 64 x 3 symbols (stem)
    (3, 64, 7, 7, 6, 6, (-1, -1)),    # wide
    (48, 40, 3, 3, 5, 6, (-1, -1)),
    (64, 17, 3, 3, 4, 5, (-1, -1)),
    (2, 2, 2, 3, 5, 5, (0, 1)),       # even kernel, explicit origin
    (33, 33, 3, 3, 4, 4, (0, 0)),     # corner origin
    (8, 12, 3, 5, 3, 9, (-1, -1)),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(v) for v in s[:6]))
def test_values_and_vectors_match_oracle(shape):
    c_out, c_in, kh, kw, n, m, pad = shape
    w = rand_w(c_out, c_in, kh, kw, seed=c_out * 1000 + c_in * 10 + n)
    plan, (s, U, V), st, info = gpu_svd(w, n, m, pad)
    assert st == C.LFA_OK, info
    assert s.shape == (n * m, min(c_out, c_in))
    check_sigma(w, n, m, s, pad)
    assert np.all(np.diff(s, axis=1) <= 0)
    check_vectors(w, n, m, s, U, V, pad)
    plan.close()


@pytest.mark.parametrize("shape", SHAPES[:9], ids=lambda s: "x".join(str(v) for v in s[:6]))
def test_values_only_and_half_output(shape):
    c_out, c_in, kh, kw, n, m, pad = shape
    w = rand_w(c_out, c_in, kh, kw, seed=7 + n)
    plan, (s, _, _), st, _ = gpu_svd(w, n, m, pad, vectors=False, half_output=True)
    assert st == C.LFA_OK
    half = O.half_grid(n, m)
    assert s.shape == (len(half), min(c_out, c_in))
    check_sigma(w, n, m, s, pad, half=half)
    plan.close()


@pytest.mark.parametrize("shape", SHAPES[:9], ids=lambda s: "x".join(str(v) for v in s[:6]))
def test_plain_path_matches_oracle(shape):
    c_out, c_in, kh, kw, n, m, pad = shape
    w = rand_w(c_out, c_in, kh, kw, seed=11 + n)
    plan, (s, _, _), st, _ = gpu_svd(w, n, m, pad, vectors=False, plain=True)
    assert st == C.LFA_OK
    check_sigma(w, n, m, s, pad)
    plan.close()


def test_symbols_match_oracle_elementwise():
    for (c_out, c_in, kh, kw, n, m, pad) in SHAPES:
        w = rand_w(c_out, c_in, kh, kw, seed=3)
        plan = LfaPlan([(c_out, c_in, kh, kw, n, m) + pad])
        S = plan.symbols(0, torch.from_numpy(w).cuda()).cpu().numpy()
        ref = O.symbols(w, n, m, *pad)[O.half_grid(n, m)]
        scale = max(np.max(np.abs(ref)), 1e-30)
        assert np.max(np.abs(S - ref)) <= 1e-6 * scale * max(1, kh * kw / 9), (c_out, c_in, n, m)
        plan.close()


def test_conv4_matches_dense_definition_and_golden():
    lay = W.layers("conv4_k3_n8")[0]
    w = W.weights(lay)
    plan, (s, U, V), st, _ = gpu_svd(w, lay.n, lay.m)
    assert st == C.LFA_OK
    dense = np.sort(O.dense_svd(w, lay.n, lay.m))[::-1]
    assert np.max(np.abs(np.sort(s.ravel())[::-1] - dense)) <= SIG_TOL * dense[0]
    gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "conv4_k3_n8_sigma.txt"))
    assert np.max(np.abs(s - gold)) <= SIG_TOL * dense[0]
    # all 256 global singular vectors: expanded on the GPU, checked on the dense operator
    A = O.dense_operator(w, lay.n, lay.m)
    Ut, Vt = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    uh, vh = plan.expand(0, Ut, Vt, 0, lay.n * lay.m * lay.r)
    uh = uh.cpu().numpy().reshape(256, -1).T.astype(np.complex128)
    vh = vh.cpu().numpy().reshape(256, -1).T.astype(np.complex128)
    sv = s.ravel().astype(np.float64)
    assert np.max(np.linalg.norm(A @ vh - uh * sv, axis=0)) <= VEC_TOL * dense[0]
    assert np.max(np.abs(vh.conj().T @ vh - np.eye(256))) <= VEC_TOL
    assert np.max(np.abs(uh.conj().T @ uh - np.eye(256))) <= VEC_TOL
    plan.close()


def test_expansion_is_the_lift_of_the_symbol_vectors():
    c_out, c_in, k, n, m = 5, 3, 3, 6, 7
    w = rand_w(c_out, c_in, k, k, seed=5)
    plan, (s, U, V), st, _ = gpu_svd(w, n, m)
    r = 3
    first, count = 17, 60
    uh, vh = plan.expand(0, torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), first, count)
    uh, vh = uh.cpu().numpy(), vh.cpu().numpy()
    half = list(O.half_grid(n, m))
    for q in range(first, first + count):
        f, sidx = divmod(q, r)
        j, l = divmod(f, m)
        fc = ((-j) % n) * m + ((-l) % m)
        if f in half:
            Uf, Vf = U[half.index(f)], V[half.index(f)]
        else:
            Uf, Vf = np.conj(U[half.index(fc)]), np.conj(V[half.index(fc)])
        ru, rv = O.lift(Uf[:, sidx:sidx + 1], Vf[:, sidx:sidx + 1], j, l, n, m)
        np.testing.assert_allclose(uh[q - first], ru[0], atol=2e-6)
        np.testing.assert_allclose(vh[q - first], rv[0], atol=2e-6)
        res = O.apply_operator(w, vh[q - first].astype(np.complex128)) - s[f, sidx] * uh[q - first]
        assert np.linalg.norm(res) <= VEC_TOL * s.max()
    plan.close()


def test_batched_layers_uneven_shapes_one_plan():
    specs = [(4, 4, 3, 3, 8, 8), (64, 64, 3, 3, 6, 6), (64, 3, 7, 7, 10, 10), (16, 32, 3, 3, 5, 7),
             (1, 1, 3, 3, 3, 3), (64, 64, 3, 3, 7, 5), (40, 64, 1, 1, 4, 4)]
    ws = [rand_w(*sp[:4], seed=100 + i) for i, sp in enumerate(specs)]
    for vectors in (False, True):
        plan = LfaPlan(specs, vectors=vectors)
        sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
        torch.cuda.synchronize()
        st, info = plan.info()
        assert st == C.LFA_OK, info
        for i, sp in enumerate(specs):
            s = sig[i].cpu().numpy()
            check_sigma(ws[i], sp[4], sp[5], s)
            if vectors:
                check_vectors(ws[i], sp[4], sp[5], s, U[i].cpu().numpy(), V[i].cpu().numpy())
        plan.close()


def test_graph_replay_with_new_buffers():
    w = rand_w(16, 16, 3, 3, seed=9)
    plan = LfaPlan([(16, 16, 3, 3, 6, 6)], vectors=True)
    wt = torch.from_numpy(w).cuda()
    out1 = plan.svd([wt])
    out2 = plan.svd([wt])                       # replay with fresh buffers: new capture
    out3 = plan.svd([wt], out=out2)             # replay into the same buffers
    torch.cuda.synchronize()
    for out in (out1, out2, out3):
        check_sigma(w, 6, 6, out[0][0].cpu().numpy())
    plan.close()


# ----------------------------------------------------------------------------- edge cases
def test_zero_kernel_gives_zero_values_and_unitary_factors():
    w = np.zeros((6, 4, 3, 3), np.float32)
    plan, (s, U, V), st, info = gpu_svd(w, 4, 5)
    assert st == C.LFA_OK, info
    assert np.all(s == 0)
    r = 4
    assert np.max(np.abs(np.einsum("hos,hot->hst", np.conj(U), U) - np.eye(r))) <= VEC_TOL
    assert np.max(np.abs(np.einsum("hos,hot->hst", np.conj(V), V) - np.eye(r))) <= VEC_TOL
    plan.close()


def test_rank_deficient_kernel():
    w = rand_w(5, 5, 3, 3, seed=12)
    w[4] = w[1]
    plan, (s, U, V), st, _ = gpu_svd(w, 6, 6)
    check_sigma(w, 6, 6, s)
    assert np.all(s[:, -1] <= SIG_TOL * s.max())
    check_vectors(w, 6, 6, s, U, V)
    plan.close()


def test_delta_kernel_unit_values():
    c = 8
    w = np.zeros((c, c, 3, 3), np.float32)
    w[:, :, 1, 1] = np.eye(c)
    plan, (s, U, V), st, _ = gpu_svd(w, 5, 5)
    assert np.max(np.abs(s - 1)) <= 1e-6
    plan.close()


def test_nonfinite_input_is_reported_not_hung():
    w = rand_w(8, 8, 3, 3, seed=1)
    w[2, 3, 1, 1] = np.nan
    plan, (s, U, V), st, info = gpu_svd(w, 4, 4)
    assert st == C.LFA_ERR_NONFINITE
    assert info["nonfinite"] > 0
    plan.close()


def test_fault_injection_nonconverge_and_launch(monkeypatch):
    w = rand_w(16, 16, 3, 3, seed=2)
    monkeypatch.setenv("LFA_FAULT_INJECT", "nonconverge")
    plan, _, st, info = gpu_svd(w, 5, 5)
    assert st == C.LFA_ERR_NOT_CONVERGED and info["unconverged"] > 0
    plan.close()
    monkeypatch.setenv("LFA_FAULT_INJECT", "launch")
    plan = LfaPlan([(16, 16, 3, 3, 5, 5)], use_graph=0)
    with pytest.raises(C.LfaError) as ei:
        plan.svd([torch.from_numpy(w).cuda()])
    assert ei.value.status == C.LFA_ERR_CUDA
    plan.close()


# ----------------------------------------------------------------------------- backward
@pytest.mark.parametrize("shape", [(4, 4, 3, 3, 8, 8), (5, 3, 3, 3, 6, 5), (3, 5, 5, 3, 4, 7),
                                   (64, 64, 3, 3, 6, 6), (64, 3, 7, 7, 9, 9), (16, 16, 5, 5, 3, 3)])
def test_backward_matches_oracle(shape):
    c_out, c_in, kh, kw, n, m = shape
    w = rand_w(c_out, c_in, kh, kw, seed=21)
    r = min(c_out, c_in)
    g = W.upstream_gradient((n * m, r), seed=22)
    plan, (s, U, V), st, _ = gpu_svd(w, n, m)
    dw = plan.backward([torch.from_numpy(g).cuda()], [torch.from_numpy(U).cuda()], [torch.from_numpy(V).cuda()])
    dw = dw[0].cpu().numpy()
    s_ref, U_ref, V_ref = O.lfa_svd(w, n, m)
    dw_ref = O.lfa_backward(w, n, m, g, U_ref, V_ref)
    err = np.linalg.norm(dw - dw_ref) / np.linalg.norm(dw_ref)
    assert err <= 1e-4, err
    plan.close()


def test_backward_half_output_matches_oracle():
    c, k, n, m = 6, 3, 5, 6
    w = rand_w(c, c, k, k, seed=31)
    half = O.half_grid(n, m)
    gh = W.upstream_gradient((len(half), c), seed=32)
    plan, (s, U, V), st, _ = gpu_svd(w, n, m, half_output=True)
    dw = plan.backward([torch.from_numpy(gh).cuda()], [torch.from_numpy(U).cuda()],
                       [torch.from_numpy(V).cuda()])[0].cpu().numpy()
    g_full = np.zeros((n * m, c))
    g_full[half] = gh                      # the half-grid value carries the gradient alone
    s_ref, U_ref, V_ref = O.lfa_svd(w, n, m)
    dw_ref = O.lfa_backward(w, n, m, g_full, U_ref, V_ref)
    assert np.linalg.norm(dw - dw_ref) / np.linalg.norm(dw_ref) <= 1e-4
    plan.close()


def test_regulariser_gradient_vs_finite_differences():
    """Spectral regulariser (sigma_max + lam * sum (sigma-1)^2) at c=4, n=8: GPU dL/dw vs FP64 FD."""
    lay = W.layers("conv4_k3_n8")[0]
    w = W.weights(lay).astype(np.float32)
    lam = 1e-2
    plan = LfaPlan([(4, 4, 3, 3, 8, 8)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    ds, loss = plan.regulariser_grad(sig, lam)
    dw = plan.backward(ds, U, V)[0].cpu().numpy()
    s_gpu = sig[0].cpu().numpy()
    np.testing.assert_allclose(ds[0].cpu().numpy(), O.regulariser_grad_sigma(s_gpu, lam), atol=1e-6)
    assert abs(float(loss[0]) - O.regulariser_loss([s_gpu], lam)) <= 1e-5 * abs(O.regulariser_loss([s_gpu], lam))
    w64 = w.astype(np.float64)

    def L(wv):
        return O.regulariser_loss([O.lfa_svd(wv, 8, 8, compute_uv=False)], lam)

    h = 1e-6
    fd = np.zeros_like(w64)
    for idx in np.ndindex(w64.shape):
        wp = w64.copy(); wp[idx] += h
        wm = w64.copy(); wm[idx] -= h
        fd[idx] = (L(wp) - L(wm)) / (2 * h)
    assert np.linalg.norm(dw - fd) / np.linalg.norm(fd) <= 1e-3
    plan.close()


def test_autograd_function():
    from paper_2506_05617_gb300.torch_api import LfaSvd
    w = rand_w(4, 4, 3, 3, seed=41)
    plan = LfaPlan([(4, 4, 3, 3, 8, 8)], vectors=True)
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    (s,) = LfaSvd.apply(plan, wt)
    loss = (s ** 2).sum()
    loss.backward()
    # d(sum sigma^2)/dw = 2 n m w (Parseval)
    np.testing.assert_allclose(wt.grad.cpu().numpy(), 2 * 64 * w, rtol=1e-4, atol=1e-5)
    plan.close()


# ----------------------------------------------------------------------------- workload sizes
def test_conv64_n32_full_size_values_vectors_and_backward():
    """The 64->64 3x3 layer on 32x32 in the benchmark's launch configuration."""
    lay = W.layers("conv64_k3_n32")[0]
    w = W.weights(lay)
    plan, (s, U, V), st, info = gpu_svd(w, lay.n, lay.m)
    assert st == C.LFA_OK, info
    check_sigma(w, lay.n, lay.m, s)
    check_vectors(w, lay.n, lay.m, s, U, V)
    g = W.upstream_gradient((lay.F, lay.r), seed=2)
    dw = plan.backward([torch.from_numpy(g).cuda()], [torch.from_numpy(U).cuda()],
                       [torch.from_numpy(V).cuda()])[0].cpu().numpy()
    s_ref, U_ref, V_ref = O.lfa_svd(w, lay.n, lay.m)
    dw_ref = O.lfa_backward(w, lay.n, lay.m, g, U_ref, V_ref)
    assert np.linalg.norm(dw - dw_ref) / np.linalg.norm(dw_ref) <= 1e-4
    plan.close()


def test_stem_3to64_n224_values_and_sampled_vectors():
    lay = W.layers("stem3to64_k7_n224")[0]
    w = W.weights(lay)
    plan, (s, U, V), st, info = gpu_svd(w, lay.n, lay.m)
    assert st == C.LFA_OK, info
    check_sigma(w, lay.n, lay.m, s)
    half = O.half_grid(lay.n, lay.m)
    pick = np.random.default_rng(0).choice(len(half), 300, replace=False)
    S = O.symbols(w, lay.n, lay.m)[half[pick]]
    ss = s[half[pick]].astype(np.float64)
    Uu, Vv = U[pick].astype(np.complex128), V[pick].astype(np.complex128)
    res = np.einsum("hoi,his->hos", S, Vv) - Uu * ss[:, None, :]
    assert np.max(np.linalg.norm(res, axis=1)) <= VEC_TOL * s.max()
    plan.close()


def test_resnet18_c64_layers_values():
    lays = [l for l in W.layers("resnet18_body") if max(l.c_out, l.c_in) <= 64]
    ws = [W.weights(l) for l in lays]
    plan = LfaPlan([(l.c_out, l.c_in, l.kh, l.kw, l.n, l.m) for l in lays], vectors=False)
    sig, _, _ = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    torch.cuda.synchronize()
    assert plan.info()[0] == C.LFA_OK
    for l, w, s in zip(lays, ws, sig):
        check_sigma(w, l.n, l.m, s.cpu().numpy())
    plan.close()
