"""Parity of the large-channel kernels (one symbol per CTA with up to 1024 threads, or per
thread-block cluster of 2 to 16 CTAs) with the FP64 oracle, and the full-size multi-layer
workloads checked on sampled frequencies and by identities that hold at any size.

Tolerances as in test_gpu_parity.py: sigma within 1e-5 * sigma_max; vectors by residual,
reconstruction and orthonormality within 1e-5 (* sigma_max where scaled)."""
import numpy as np
import pytest
import torch

import lfa_workloads as W
import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan

from test_gpu_parity import check_sigma, check_vectors, gpu_svd, rand_w, SIG_TOL, VEC_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


LARGE = [
    # c_out, c_in, k, n, m, vectors
    (128, 64, 3, 4, 3, True),     # tall 128 x 64
    (64, 128, 3, 3, 4, True),     # wide
    (128, 128, 3, 4, 3, True),    # cluster of 2
    (128, 128, 3, 4, 3, False),   # one CTA of 1024 threads
    (100, 77, 3, 3, 3, True),     # ragged
    (256, 128, 3, 3, 3, True),    # cluster of 4
    (256, 256, 3, 3, 2, True),    # cluster of 8
    (200, 200, 1, 2, 3, True),
    (256, 256, 3, 3, 3, False),
    (512, 256, 3, 2, 3, False),   # cluster of 8, 16 rows per lane
    (512, 512, 3, 2, 3, False),   # cluster of 16
    (300, 450, 3, 2, 2, False),
    (512, 512, 3, 2, 3, True),    # vectors through the rotation log + replay
    (512, 256, 3, 2, 2, True),
    (256, 512, 3, 2, 2, True),    # wide: V from the normalised columns, U from the replay
    (400, 400, 1, 1, 2, True),
]


@pytest.mark.parametrize("spec", LARGE, ids=lambda s: "x".join(str(v) for v in s[:5]) + ("v" if s[5] else ""))
def test_large_channels_match_oracle(spec):
    c_out, c_in, k, n, m, vec = spec
    w = rand_w(c_out, c_in, k, k, seed=c_out + 7 * c_in)
    plan, (s, U, V), st, info = gpu_svd(w, n, m, vectors=vec)
    assert st == C.LFA_OK, info
    check_sigma(w, n, m, s)
    assert np.all(np.diff(s, axis=1) <= 0)
    if vec:
        check_vectors(w, n, m, s, U, V)
    plan.close()


@pytest.mark.parametrize("shape", [(128, 128, 4), (200, 160, 7), (512, 256, 16), (256, 512, 3)],
                         ids=lambda s: "x".join(map(str, s)))
def test_rank_deficient_symbols_get_complete_orthonormal_factors(shape):
    """1x1 kernels of rank q: every symbol has rank q, so the factor built from X has N - q exactly
    zero columns that must be completed to an orthonormal basis (cluster and rotation-log paths)."""
    c_out, c_in, q = shape
    rng = np.random.default_rng(q)
    w = (rng.standard_normal((c_out, q)) @ rng.standard_normal((q, c_in)) / np.sqrt(q * c_in))
    w = w.astype(np.float32).reshape(c_out, c_in, 1, 1)
    plan, (s, U, V), st, info = gpu_svd(w, 2, 2, vectors=True)
    assert st == C.LFA_OK, info
    check_sigma(w, 2, 2, s)
    assert np.all(s[:, q:] <= SIG_TOL * s.max())
    check_vectors(w, 2, 2, s, U, V)
    plan.close()


def test_large_backward_matches_oracle():
    c_out, c_in, k, n, m = 128, 96, 3, 3, 4
    w = rand_w(c_out, c_in, k, k, seed=5)
    g = W.upstream_gradient((n * m, min(c_out, c_in)), seed=6)
    plan, (s, U, V), st, _ = gpu_svd(w, n, m)
    dw = plan.backward([torch.from_numpy(g).cuda()], [torch.from_numpy(U).cuda()],
                       [torch.from_numpy(V).cuda()])[0].cpu().numpy()
    s_ref, U_ref, V_ref = O.lfa_svd(w, n, m)
    dw_ref = O.lfa_backward(w, n, m, g, U_ref, V_ref)
    assert np.linalg.norm(dw - dw_ref) / np.linalg.norm(dw_ref) <= 1e-4
    plan.close()


def sampled_sigma_check(w, lay, s, nsample, seed):
    rng = np.random.default_rng(seed)
    fr = np.sort(rng.choice(lay.F, min(nsample, lay.F), replace=False))
    s_ref = O.lfa_svd(w, lay.n, lay.m, compute_uv=False, freqs=fr)
    # sigma_max of the whole layer from the GPU values (checked against the oracle's sample)
    smax = float(s.max())
    assert np.max(np.abs(s[fr].astype(np.float64) - s_ref)) <= SIG_TOL * smax
    # Parseval over every frequency: sum sigma^2 = n m ||w||_F^2 (k <= n)
    np.testing.assert_allclose(np.sum(s.astype(np.float64) ** 2), lay.n * lay.m * np.sum(w.astype(np.float64) ** 2),
                               rtol=2e-5)


def test_resnet18_body_all_layers_one_plan():
    """The 16-layer ResNet-18-shaped stack (uneven c_out, c_in and n) in one plan, values only."""
    lays = W.layers("resnet18_body")
    ws = [W.weights(l) for l in lays]
    plan = LfaPlan([(l.c_out, l.c_in, l.kh, l.kw, l.n, l.m) for l in lays], vectors=False)
    sig, _, _ = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    assert info["symbols"] == sum((l.F + (1 + (l.n % 2 == 0)) * (1 + (l.m % 2 == 0))) // 2 for l in lays)
    for i, (l, w, s) in enumerate(zip(lays, ws, sig)):
        sampled_sigma_check(w, l, s.cpu().numpy(), 24, seed=i)
    plan.close()


def test_regulariser_workload_c128_full_size():
    """4 layers 128->128 on 32x32, k = 3, 5, 3, 5: values + vectors + backward.

    Checks at full size: sampled sigma against the oracle, residuals of sampled symbols, and the
    closed-form gradient of sum sigma^2 (= 2 n m w) through the hand-written backward."""
    lays = W.layers("reg4_c128_n32")
    ws = [W.weights(l) for l in lays]
    plan = LfaPlan([(l.c_out, l.c_in, l.kh, l.kw, l.n, l.m) for l in lays], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    dw = plan.backward([2 * s for s in sig], U, V)
    for i, (l, w) in enumerate(zip(lays, ws)):
        s = sig[i].cpu().numpy()
        sampled_sigma_check(w, l, s, 16, seed=10 + i)
        half = O.half_grid(l.n, l.m)
        pick = np.random.default_rng(i).choice(len(half), 8, replace=False)
        S = O.symbols(w, l.n, l.m, freqs=half[pick])
        Uu = U[i][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
        Vv = V[i][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
        ss = s[half[pick]].astype(np.float64)
        res = np.einsum("hoi,his->hos", S, Vv) - Uu * ss[:, None, :]
        assert np.max(np.linalg.norm(res, axis=1)) <= VEC_TOL * s.max()
        assert np.max(np.abs(np.einsum("hos,hot->hst", np.conj(Vv), Vv) - np.eye(l.r))) <= VEC_TOL
        ref = 2 * l.n * l.m * w.astype(np.float64)
        got = dw[i].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
    plan.close()


def test_conv512_values_sampled():
    lay = W.layers("conv512_k3_n64")[0]
    w = W.weights(lay)
    plan, (s, _, _), st, info = gpu_svd(w, lay.n, lay.m, vectors=False)
    assert st == C.LFA_OK, info
    sampled_sigma_check(w, lay, s, 6, seed=3)
    plan.close()


def test_conv512_n64_values_and_vectors_sampled():
    """512->512 3x3 on 64x64 (2050 half-grid symbols, the benchmark layer): values on 24 random
    frequencies plus the four self-conjugate ones and the GPU's argmax frequency (whose oracle
    value pins the layer's sigma_max), Parseval over all 2.1M values; vectors (residual
    A v - sigma u, orthonormality) on 8 half-grid frequencies including f = 0 and the argmax's
    representative."""
    lay = W.layers("conv512_k3_n64")[0]
    w = W.weights(lay)
    n, m = lay.n, lay.m
    plan = LfaPlan([(lay.c_out, lay.c_in, lay.kh, lay.kw, n, m)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    s = sig[0].cpu().numpy()
    fmax = int(np.argmax(s) // lay.r)
    selfc = [0, (n // 2) * m, m // 2, (n // 2) * m + m // 2]
    rnd = np.random.default_rng(8).choice(lay.F, 24, replace=False)
    fr = np.unique(np.concatenate([rnd, selfc, [fmax]]))
    s_ref = O.lfa_svd(w, n, m, compute_uv=False, freqs=fr)
    smax = float(s.max())
    k = int(np.searchsorted(fr, fmax))
    assert abs(float(s_ref[k].max()) - smax) <= SIG_TOL * smax          # the layer's sigma_max
    assert float(s_ref.max()) <= smax * (1 + SIG_TOL)
    assert np.max(np.abs(s[fr].astype(np.float64) - s_ref)) <= SIG_TOL * smax
    np.testing.assert_allclose(np.sum(s.astype(np.float64) ** 2), n * m * np.sum(w.astype(np.float64) ** 2),
                               rtol=2e-5)
    half = O.half_grid(n, m)
    fcm = ((-(fmax // m)) % n) * m + (-(fmax % m)) % m
    hmax = int(np.searchsorted(half, min(fmax, fcm)))
    pick = np.unique(np.concatenate([[0, hmax], np.random.default_rng(1).choice(len(half), 6, replace=False)]))
    S = O.symbols(w, n, m, freqs=half[pick])
    Uu = U[0][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
    Vv = V[0][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
    ss = s[half[pick]].astype(np.float64)
    res = np.einsum("hoi,his->hos", S, Vv) - Uu * ss[:, None, :]
    assert np.max(np.linalg.norm(res, axis=1)) <= VEC_TOL * smax
    for X in (Uu, Vv):
        assert np.max(np.abs(np.einsum("hos,hot->hst", np.conj(X), X) - np.eye(lay.r))) <= VEC_TOL
    plan.close()


def test_conv512_n64_backward_on_sampled_frequencies():
    """The benchmark layer's backward (tensor-core G over 17 blocks of the 2050 symbols) with the
    upstream gradient kept on 6 sampled frequencies and their conjugates: equal to the oracle's
    backward over those frequencies with the GPU's own U, V (1e-5 relative)."""
    lay = W.layers("conv512_k3_n64")[0]
    w = W.weights(lay)
    n, m, r = lay.n, lay.m, lay.r
    plan = LfaPlan([(lay.c_out, lay.c_in, lay.kh, lay.kw, n, m)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    half = O.half_grid(n, m)
    pick = np.array([0, 1, 700, 1500, 2048, 2049])           # first, middle and last G blocks
    f = half[pick]
    fc = ((-(f // m)) % n) * m + (-(f % m)) % m
    keep = np.zeros(n * m, bool)
    keep[f] = True
    keep[fc] = True
    g = W.upstream_gradient((n * m, r), seed=17) * keep[:, None]
    dw = plan.backward([torch.from_numpy(g.astype(np.float32)).cuda()], U, V)[0].cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    full_f = np.flatnonzero(keep)
    hpos = {int(h): q for q, h in enumerate(half)}
    Ug = U[0][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
    Vg = V[0][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
    loc = {int(h): q for q, h in enumerate(f)}
    Uf = np.empty((len(full_f), lay.c_out, r), np.complex128)
    Vf = np.empty((len(full_f), lay.c_in, r), np.complex128)
    for q, ff in enumerate(full_f):
        fcc = ((-(ff // m)) % n) * m + (-(ff % m)) % m
        if ff in loc:
            Uf[q], Vf[q] = Ug[loc[ff]], Vg[loc[ff]]
        else:
            Uf[q], Vf[q] = np.conj(Ug[loc[fcc]]), np.conj(Vg[loc[fcc]])
    ref = O.lfa_backward(w, n, m, g[full_f], Uf, Vf, freqs=full_f)
    assert np.linalg.norm(dw - ref) / np.linalg.norm(ref) <= 1e-5
    plan.close()


def test_conv64_n256_values_and_vectors_sampled():
    """64->64 3x3 on 256x256 (32,770 half-grid symbols, the largest point of the n sweep): sampled
    values and vectors against the oracle, Parseval over all 4.2M singular values."""
    lay = W.Layer(64, 64, 3, 3, 256, 256, "normal", 2.0, 2)
    w = W.weights(lay)
    plan = LfaPlan([(lay.c_out, lay.c_in, lay.kh, lay.kw, lay.n, lay.m)], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    s = sig[0].cpu().numpy()
    assert s.shape == (lay.F, 64)
    sampled_sigma_check(w, lay, s, 8, seed=9)
    half = O.half_grid(lay.n, lay.m)
    pick = np.random.default_rng(10).choice(len(half), 6, replace=False)
    S = O.symbols(w, lay.n, lay.m, freqs=half[pick])
    Uu = U[0][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
    Vv = V[0][torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.complex128)
    ss = s[half[pick]].astype(np.float64)
    res = np.einsum("hoi,his->hos", S, Vv) - Uu * ss[:, None, :]
    assert np.max(np.linalg.norm(res, axis=1)) <= VEC_TOL * s.max()
    for X in (Uu, Vv):
        assert np.max(np.abs(np.einsum("hos,hot->hst", np.conj(X), X) - np.eye(lay.r))) <= VEC_TOL
    plan.close()


def test_paper_shape_at_n2048_values_sampled():
    """The paper's 16->16 3x3 shape at n = 2048 (2,097,154 half-grid symbols, 67M singular values):
    sampled frequencies against the oracle, Parseval over all of them, conjugate mirror."""
    lay = W.Layer(16, 16, 3, 3, 2048, 2048, "normal", 2.0, 6)
    w = W.weights(lay)
    plan, (s, _, _), st, info = gpu_svd(w, lay.n, lay.m, vectors=False)
    assert st == C.LFA_OK, info
    assert s.shape == (lay.F, 16)
    sampled_sigma_check(w, lay, s, 8, seed=4)
    fr = np.random.default_rng(5).choice(lay.F, 64, replace=False)
    j, l = fr // lay.m, fr % lay.m
    fc = ((-j) % lay.n) * lay.m + (-l) % lay.m
    assert np.array_equal(s[fr], s[fc])
    plan.close()


def test_regulariser_workload_c128_backward_matches_oracle_on_sampled_frequencies():
    """The regulariser workload at full size (4 x 128->128 on 32x32, k = 3, 5, 3, 5) with its real
    loss: dsigma = lfa_regulariser_grad (1 at the layer's sigma_max plus 2 lam (sigma - 1)). The GPU
    backward is restricted to sampled frequencies by zeroing dsigma elsewhere (each sampled
    half-grid frequency keeps itself and its conjugate; sigma_max's frequency is always sampled),
    and compared with the oracle's backward over the same frequencies, once with the oracle's own
    FP64 U, V (sigma simple there) and once with the GPU's U, V. Tolerance 1e-4 relative."""
    lays = W.layers("reg4_c128_n32")
    ws = [W.weights(l) for l in lays]
    plan = LfaPlan([(l.c_out, l.c_in, l.kh, l.kw, l.n, l.m) for l in lays], vectors=True)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda() for w in ws])
    dsig, _ = plan.regulariser_grad(sig, 1e-2)
    torch.cuda.synchronize()
    st, info = plan.info()
    assert st == C.LFA_OK, info
    masks, samples = [], []
    for i, l in enumerate(lays):
        half = O.half_grid(l.n, l.m)
        s = sig[i].cpu().numpy()
        fmax = int(np.argmax(s) // l.r)
        hmax = int(np.searchsorted(half, min(fmax, ((-(fmax // l.m)) % l.n) * l.m + (-(fmax % l.m)) % l.m)))
        pick = np.unique(np.concatenate([[hmax], np.random.default_rng(20 + i).choice(len(half), 8, replace=False)]))
        f = half[pick]
        fc = ((-(f // l.m)) % l.n) * l.m + (-(f % l.m)) % l.m
        keep = np.zeros(l.F, bool)
        keep[f] = True
        keep[fc] = True
        masks.append(torch.from_numpy(keep).cuda())
        samples.append((pick, f, np.flatnonzero(keep)))
    g_masked = [d * m[:, None] for d, m in zip(dsig, masks)]
    dw = plan.backward(g_masked, U, V)
    for i, (l, w) in enumerate(zip(lays, ws)):
        pick, f, full_f = samples[i]
        g = g_masked[i].cpu().numpy().astype(np.float64)
        assert g[np.argmax(sig[i].cpu().numpy()) // l.r].max() >= 1.0     # the sigma_max term is in the sample
        s_or, U_or, V_or = O.lfa_svd(w, l.n, l.m, compute_uv=True, freqs=full_f)
        gaps = np.min(-np.diff(s_or, axis=1)) / s_or.max()
        assert gaps > 1e-6                                                # simple singular values
        ref = O.lfa_backward(w, l.n, l.m, g[full_f], U_or, V_or, freqs=full_f)
        got = dw[i].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (i, err)
        # the same sum with the GPU's factors (conjugate frequencies take conj(U), conj(V))
        half = O.half_grid(l.n, l.m)
        hpos = {int(h): k for k, h in enumerate(half)}
        Ug, Vg = U[i].cpu().numpy().astype(np.complex128), V[i].cpu().numpy().astype(np.complex128)
        Uf = np.empty((len(full_f), l.c_out, l.r), np.complex128)
        Vf = np.empty((len(full_f), l.c_in, l.r), np.complex128)
        for k, ff in enumerate(full_f):
            fcc = ((-(ff // l.m)) % l.n) * l.m + (-(ff % l.m)) % l.m
            if ff in hpos:
                Uf[k], Vf[k] = Ug[hpos[ff]], Vg[hpos[ff]]
            else:
                Uf[k], Vf[k] = np.conj(Ug[hpos[fcc]]), np.conj(Vg[hpos[fcc]])
        ref_g = O.lfa_backward(w, l.n, l.m, g[full_f], Uf, Vf, freqs=full_f)
        assert np.linalg.norm(got - ref_g) / np.linalg.norm(ref_g) <= 1e-4
    plan.close()
