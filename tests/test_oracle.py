"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: a library
routine (torch's circular conv2d, LAPACK on the dense matrix, numpy's FFT), a
closed form, an identity (Parseval), brute force on a tiny input, or finite
differences. Chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import oracle as O
import lfa_workloads as W

RNG = np.random.default_rng(12345)


def rand_w(c_out, c_in, kh, kw, seed):
    return np.random.default_rng(seed).standard_normal((c_out, c_in, kh, kw)) / np.sqrt(c_in * kh * kw)


def torch_circular_conv(w, f, ph, pw):
    """PyTorch cross-correlation on a circularly padded input: out(x) = sum w[a,b] f(x + (a-ph, b-pw))."""
    kh, kw = w.shape[2], w.shape[3]
    ft = torch.as_tensor(f)[None]
    ft = Fnn.pad(ft, (pw, kw - 1 - pw, ph, kh - 1 - ph), mode="circular")
    return Fnn.conv2d(ft, torch.as_tensor(w))[0].numpy()


# ----------------------------------------------------------------- the operator definition
@pytest.mark.parametrize("c_out,c_in,kh,kw,n,m,pad", [
    (3, 2, 3, 3, 5, 4, (-1, -1)),
    (2, 3, 3, 5, 6, 7, (-1, -1)),
    (2, 2, 3, 3, 5, 5, (0, 0)),      # corner origin
    (1, 2, 2, 4, 4, 6, (1, 3)),      # even kernel, explicit origin
])
def test_dense_operator_is_torch_circular_conv(c_out, c_in, kh, kw, n, m, pad):
    w = rand_w(c_out, c_in, kh, kw, 1)
    ph, pw = O.origin(kh, kw, *pad)
    A = O.dense_operator(w, n, m, *pad)
    f = RNG.standard_normal((c_in, n, m))
    ref = torch_circular_conv(w, f, ph, pw)
    np.testing.assert_allclose(A @ f.ravel(), ref.ravel(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.apply_operator(w, f, *pad), ref, rtol=1e-12, atol=1e-12)
    g = RNG.standard_normal((c_out, n, m))
    np.testing.assert_allclose(O.apply_adjoint(w, g, *pad).ravel(), A.T @ g.ravel(), rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------- the convolution theorem
@pytest.mark.parametrize("c_out,c_in,k,n,m", [
    (4, 4, 3, 8, 8), (3, 5, 3, 4, 6), (5, 2, 3, 5, 3), (2, 2, 5, 4, 3), (3, 3, 1, 4, 4), (1, 1, 3, 7, 5),
])
def test_dense_svd_is_union_of_symbol_svds(c_out, c_in, k, n, m):
    w = rand_w(c_out, c_in, k, k, 2)
    dense = np.sort(O.dense_svd(w, n, m))[::-1]
    s = O.lfa_svd(w, n, m, compute_uv=False)
    r = min(c_out, c_in)
    assert s.shape == (n * m, r)
    union = np.sort(s.ravel())[::-1]
    tol = 1e-12 * dense[0]
    np.testing.assert_allclose(dense[:n * m * r], union, atol=tol, rtol=0)
    # the dense (c_out nm) x (c_in nm) operator has min(c_out, c_in) nm singular values
    assert dense.size == n * m * r


def test_lifted_vectors_form_the_dense_svd():
    """U^_k = F_k U_k, V^_k = F_k V_k: A V^ = U^ S, and the stacked V^ (all k, s) is unitary."""
    c, k, n, m = 3, 3, 4, 5
    w = rand_w(c, c, k, k, 3)
    A = O.dense_operator(w, n, m)
    s, U, V = O.lfa_svd(w, n, m)
    cols_u, cols_v, sig = [], [], []
    for f in range(n * m):
        j, l = divmod(f, m)
        uh, vh = O.lift(U[f], V[f], j, l, n, m)
        cols_u.append(uh.reshape(c, -1))
        cols_v.append(vh.reshape(c, -1))
        sig.append(s[f])
    Uh = np.concatenate(cols_u).T
    Vh = np.concatenate(cols_v).T
    S = np.concatenate(sig)
    np.testing.assert_allclose(A @ Vh, Uh * S[None, :], atol=1e-12)
    np.testing.assert_allclose(A.T @ Uh, Vh * S[None, :], atol=1e-12)
    np.testing.assert_allclose(Vh.conj().T @ Vh, np.eye(c * n * m), atol=1e-12)
    np.testing.assert_allclose(Uh.conj().T @ Uh, np.eye(c * n * m), atol=1e-12)


def test_symbol_factorisation():
    w = rand_w(3, 4, 3, 3, 4)
    s, U, V = O.lfa_svd(w, 4, 4)
    S = O.symbols(w, 4, 4)
    rec = np.einsum("fos,fs,fis->foi", U, s, np.conj(V))
    np.testing.assert_allclose(rec, S, atol=1e-13)
    assert np.all(np.diff(s, axis=1) <= 0)


# ----------------------------------------------------------------- FFT route (library FFT)
@pytest.mark.parametrize("pad", [(-1, -1), (0, 0), (2, 1)])
def test_fft_route_gives_conjugate_symbols(pad):
    w = rand_w(3, 2, 3, 4, 5)
    n, m = 6, 5
    np.testing.assert_allclose(O.fft_symbols(w, n, m, *pad), np.conj(O.symbols(w, n, m, *pad)), atol=1e-13)
    s1 = O.lfa_svd(w, n, m, *pad, compute_uv=False)
    s2 = np.linalg.svd(O.fft_symbols(w, n, m, *pad), compute_uv=False)
    np.testing.assert_allclose(s1, s2, atol=1e-13)


def test_single_channel_is_fft_magnitude():
    """c = 1: sigma(k) = |sum_y w_y e^{2 pi i <k,y>}|, i.e. |FFT| of the folded kernel."""
    w = rand_w(1, 1, 5, 3, 6)
    n, m = 7, 6
    s = O.lfa_svd(w, n, m, compute_uv=False)[:, 0]
    K = O.folded_kernel(w, n, m)[0, 0]
    mag = np.abs(np.fft.ifft2(K)).ravel() * n * m
    np.testing.assert_allclose(s, mag, atol=1e-13)


# ----------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,m", [(4, 4), (8, 6), (5, 7)])
def test_periodic_laplacian_closed_form(n, m):
    """5-point Laplacian: eigenvalues 4 sin^2(pi j/n) + 4 sin^2(pi l/m) on the periodic grid (textbook)."""
    w = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], dtype=np.float64)[None, None]
    s = O.lfa_svd(w, n, m, compute_uv=False)[:, 0].reshape(n, m)
    j = np.arange(n)[:, None]
    l = np.arange(m)[None, :]
    ref = 4 * np.sin(np.pi * j / n) ** 2 + 4 * np.sin(np.pi * l / m) ** 2
    np.testing.assert_allclose(s, ref, atol=1e-13)


def test_averaging_stencil_closed_form():
    """1-D forward average (f(x) + f(x+1))/2 along rows: |cos(pi j / n)| for every l."""
    n, m = 6, 3
    w = np.zeros((1, 1, 2, 1))
    w[0, 0, :, 0] = 0.5
    s = O.lfa_svd(w, n, m, pad_h=0, pad_w=0, compute_uv=False)[:, 0].reshape(n, m)
    ref = np.abs(np.cos(np.pi * np.arange(n) / n))[:, None] * np.ones((1, m))
    np.testing.assert_allclose(s, ref, atol=1e-14)


@pytest.mark.parametrize("shift", [(1, 1), (0, 2), (2, 0)])
def test_delta_kernels_give_unit_singular_values(shift):
    c, k, n = 4, 3, 5
    w = np.zeros((c, c, k, k))
    w[:, :, shift[0], shift[1]] = np.eye(c)   # centred delta is the identity, the others are shifts
    s = O.lfa_svd(w, n, n, compute_uv=False)
    np.testing.assert_allclose(s, 1.0, atol=1e-14)
    w2 = -2.5 * w
    np.testing.assert_allclose(O.lfa_svd(w2, n, n, compute_uv=False), 2.5, atol=1e-13)


def test_one_by_one_conv_repeats_channel_matrix_spectrum():
    w = rand_w(5, 3, 1, 1, 7)
    n, m = 4, 3
    s = O.lfa_svd(w, n, m, compute_uv=False)
    ref = np.linalg.svd(w[:, :, 0, 0], compute_uv=False)
    np.testing.assert_allclose(s, np.broadcast_to(ref, s.shape), atol=1e-14)


def test_channel_diagonal_kernel_is_union_of_single_channel_spectra():
    c, n, m = 3, 6, 4
    w = np.zeros((c, c, 3, 3))
    per = []
    for i in range(c):
        wi = rand_w(1, 1, 3, 3, 20 + i)
        w[i, i] = wi[0, 0]
        per.append(np.abs(np.fft.ifft2(O.folded_kernel(wi, n, m)[0, 0])).ravel() * n * m)
    s = O.lfa_svd(w, n, m, compute_uv=False)
    np.testing.assert_allclose(np.sort(s, axis=1), np.sort(np.stack(per, 1), axis=1), atol=1e-13)


# ----------------------------------------------------------------- identities and invariants
@pytest.mark.parametrize("c_out,c_in,k,n,m", [(4, 4, 3, 8, 8), (6, 3, 5, 4, 3), (2, 5, 7, 3, 4)])
def test_parseval(c_out, c_in, k, n, m):
    """sum sigma^2 = ||A||_F^2 = n m ||w folded onto the torus||_F^2 (taps alias when k > n)."""
    w = rand_w(c_out, c_in, k, k, 8)
    s = O.lfa_svd(w, n, m, compute_uv=False)
    K = O.folded_kernel(w, n, m)
    np.testing.assert_allclose(np.sum(s ** 2), n * m * np.sum(K ** 2), rtol=1e-12)
    if k <= min(n, m):
        np.testing.assert_allclose(np.sum(s ** 2), n * m * np.sum(w ** 2), rtol=1e-12)


def test_aliasing_kernel_larger_than_torus():
    w = rand_w(2, 3, 5, 5, 9)
    n, m = 4, 3
    dense = np.sort(O.dense_svd(w, n, m))[::-1][: n * m * 2]
    s = np.sort(O.lfa_svd(w, n, m, compute_uv=False).ravel())[::-1]
    np.testing.assert_allclose(dense, s, atol=1e-12 * dense[0])


def test_conjugate_symmetry_and_half_grid():
    w = rand_w(3, 3, 3, 3, 10)
    for n, m in [(4, 4), (5, 4), (4, 5), (5, 7), (1, 3), (2, 2), (1, 1)]:
        S = O.symbols(w, n, m)
        s = O.lfa_svd(w, n, m, compute_uv=False)
        hg = O.half_grid(n, m)
        n_self = (1 + (n % 2 == 0)) * (1 + (m % 2 == 0))
        assert len(hg) == (n * m + n_self) // 2
        seen = set()
        for f in hg:
            j, l = divmod(int(f), m)
            fc = ((-j) % n) * m + ((-l) % m)
            np.testing.assert_allclose(S[fc], np.conj(S[f]), atol=1e-13)
            np.testing.assert_allclose(s[fc], s[f], atol=1e-13)
            seen.update({int(f), int(fc)})
        assert seen == set(range(n * m))


def test_transposed_convolution_has_same_spectrum():
    """A^T is the conv with channels swapped and taps flipped (origin mirrored)."""
    c_out, c_in, k, n, m = 4, 2, 3, 5, 6
    w = rand_w(c_out, c_in, k, k, 11)
    wt = np.ascontiguousarray(w.transpose(1, 0, 2, 3)[:, :, ::-1, ::-1])
    At = O.dense_operator(wt, n, m, pad_h=k - 1 - k // 2, pad_w=k - 1 - k // 2)
    np.testing.assert_allclose(At, O.dense_operator(w, n, m).T, atol=1e-15)
    s1 = O.lfa_svd(w, n, m, compute_uv=False)
    s2 = O.lfa_svd(wt, n, m, pad_h=k - 1 - k // 2, pad_w=k - 1 - k // 2, compute_uv=False)
    np.testing.assert_allclose(np.sort(s1.ravel()), np.sort(s2.ravel()), atol=1e-13)


def test_rank_deficient_kernel():
    """A duplicated output channel makes every symbol rank-deficient: one zero per frequency."""
    w = rand_w(3, 3, 3, 3, 12)
    w[2] = w[1]
    n, m = 4, 4
    s = O.lfa_svd(w, n, m, compute_uv=False)
    assert np.all(s[:, 2] <= 1e-13 * s.max())
    dense = O.dense_svd(w, n, m)
    assert np.sum(dense <= 1e-12 * dense.max()) == n * m


def test_sigma_max_by_power_iteration_through_torch_conv():
    """Largest singular value of a 16-channel layer on 12x12 by power iteration on the operator.

    A is applied with torch's circular conv2d and A^T by autograd through it, so nothing of the
    oracle is used on this side.
    """
    c, n = 16, 12
    w = rand_w(c, c, 3, 3, 13)
    wt = torch.as_tensor(w)

    def A(x):
        return Fnn.conv2d(Fnn.pad(x, (1, 1, 1, 1), mode="circular"), wt)

    x = torch.as_tensor(np.random.default_rng(0).standard_normal((1, c, n, n)))
    for _ in range(3000):
        x = x.detach().requires_grad_(True)
        y = A(x)
        (g,) = torch.autograd.grad(y, x, y)          # A^T A x
        x = g / g.norm()
    lam = float(A(x).norm() / x.norm())
    s = O.lfa_svd(w, n, n, compute_uv=False)
    assert abs(lam - s.max()) <= 1e-9 * s.max()


# ----------------------------------------------------------------- backward
def test_backward_matches_central_finite_differences():
    c_out, c_in, k, n, m = 3, 2, 3, 4, 5
    w = rand_w(c_out, c_in, k, k, 14)
    lam = 1e-2

    def loss(wv):
        return O.regulariser_loss([O.lfa_svd(wv, n, m, compute_uv=False)], lam)

    s, U, V = O.lfa_svd(w, n, m)
    g = O.regulariser_grad_sigma(s, lam)
    dW = O.lfa_backward(w, n, m, g, U, V)
    h = 1e-6
    fd = np.zeros_like(w)
    for idx in np.ndindex(w.shape):
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        fd[idx] = (loss(wp) - loss(wm)) / (2 * h)
    np.testing.assert_allclose(dW, fd, rtol=1e-6, atol=1e-8)


def test_backward_matches_dense_svd_autograd():
    """Regulariser gradient through torch.linalg.svdvals of the dense 256x256 operator (c=4, n=8)."""
    lay = W.layers("conv4_k3_n8")[0]
    w = W.weights(lay).astype(np.float64)
    n, m, lam = lay.n, lay.m, 1e-2
    A = torch.as_tensor(O.dense_operator(w, n, m))
    # differentiate through the dense matrix, then chain rule dL/dw = sum over the entries each tap fills
    A.requires_grad_(True)
    sv = torch.linalg.svdvals(A)
    L = sv.max() + lam * ((sv - 1.0) ** 2).sum()
    (gA,) = torch.autograd.grad(L, A)
    gA = gA.numpy()
    dW_ref = np.zeros_like(w)
    basis = np.zeros_like(w)
    for idx in np.ndindex(w.shape):
        basis[idx] = 1.0
        dW_ref[idx] = np.sum(gA * O.dense_operator(basis, n, m))
        basis[idx] = 0.0
    s, U, V = O.lfa_svd(w, n, m)
    dW = O.lfa_backward(w, n, m, O.regulariser_grad_sigma(s, lam), U, V)
    np.testing.assert_allclose(dW, dW_ref, rtol=1e-8, atol=1e-10)


def test_backward_of_frobenius_norm_closed_form():
    """d(sum sigma^2)/dw = 2 n m w for k <= n (Parseval), checked with g = 2 sigma."""
    w = rand_w(3, 4, 3, 3, 15)
    n, m = 5, 4
    s, U, V = O.lfa_svd(w, n, m)
    dW = O.lfa_backward(w, n, m, 2 * s, U, V)
    np.testing.assert_allclose(dW, 2 * n * m * w, rtol=1e-11, atol=1e-12)


# ----------------------------------------------------------------- spectral editing
@pytest.mark.parametrize("mode,a,b", [("clip", 0.8, 0), ("clamp", 0.3, 0.9), ("threshold", 0.5, 0), ("rank", 2, 0)])
def test_spectral_edit_matches_dense_projection(mode, a, b):
    """The symbol-side projection equals the projection of the dense edited operator onto taps."""
    w = rand_w(3, 3, 3, 3, 31)
    n, m = 4, 5
    np.testing.assert_allclose(O.spectral_edit(w, n, m, mode, a, b), O.dense_spectral_edit(w, n, m, mode, a, b),
                               atol=1e-12)


def _edit_input():
    """Descending rows of singular values with ties, zeros and entries equal to the parameters."""
    rng = np.random.default_rng(41)
    s = np.sort(rng.uniform(0.0, 2.0, (7, 6)), axis=1)[:, ::-1].copy()
    s[0, :] = [1.5, 0.9, 0.5, 0.5, 0.3, 0.0]      # exact parameter values 0.5 and 0.3, a zero
    s[1, :] = 0.7                                 # a fully degenerate frequency
    return s


def test_edit_values_clip_properties():
    s = _edit_input()
    out = O.edit_values(s, "clip", 0.6)
    assert np.all(out <= 0.6)
    keep = s <= 0.6
    assert np.array_equal(out[keep], s[keep])           # unchanged below the cap
    assert np.all(out[~keep] == 0.6)                     # capped above it


def test_edit_values_clamp_properties():
    s = _edit_input()
    lo, hi = 0.3, 0.9
    out = O.edit_values(s, "clamp", lo, hi)
    assert np.all((out >= lo) & (out <= hi))             # swapped bounds would break this
    inside = (s >= lo) & (s <= hi)
    assert np.array_equal(out[inside], s[inside])
    assert np.all(out[s < lo] == lo) and np.all(out[s > hi] == hi)
    assert np.array_equal(out, np.clip(s, lo, hi))       # the library's clip routine agrees


def test_edit_values_threshold_properties():
    s = _edit_input()
    a = 0.5
    out = O.edit_values(s, "threshold", a)
    assert np.all(out[s < a] == 0.0)
    kept = s >= a
    assert np.array_equal(out[kept], s[kept])            # values equal to a are kept (>=, not >)
    assert out[0, 2] == 0.5 and out[0, 3] == 0.5 and out[0, 4] == 0.0


@pytest.mark.parametrize("a,k", [(0, 0), (2, 2), (2.4, 2), (2.6, 3), (6, 6), (9, 6)])
def test_edit_values_rank_properties(a, k):
    s = _edit_input() + 1.0                              # all positive: non-zeros are countable
    out = O.edit_values(s, "rank", a)
    assert np.all(np.count_nonzero(out, axis=1) == k)    # round(a) values per frequency
    assert np.array_equal(out[:, :k], s[:, :k])          # the leading (largest) ones
    assert np.all(out[:, k:] == 0.0)


@pytest.mark.parametrize("mode,a,b", [("clamp", 0.3, 0.9), ("threshold", 0.5, 0), ("rank", 2, 0)])
def test_spectral_edit_is_exact_for_a_kernel_covering_the_torus(mode, a, b):
    """With kh = n and kw = m every operator is a convolution, so the edited kernel's spectrum
    is the edited spectrum itself; checked by properties of the multiset, not by phi."""
    wf = rand_w(3, 3, 4, 4, 34)
    n = m = 4
    smax = O.lfa_svd(wf, n, m, compute_uv=False).max()
    s = O.lfa_svd(wf, n, m, compute_uv=False)
    aa, bb = (a * smax, b * smax) if mode != "rank" else (a, b)
    got = O.lfa_svd(O.spectral_edit(wf, n, m, mode, aa, bb), n, m, compute_uv=False)
    if mode == "clamp":
        np.testing.assert_allclose(np.sort(got.ravel()), np.sort(np.clip(s, aa, bb).ravel()), atol=1e-12)
    elif mode == "threshold":
        nz = np.sort(got.ravel())[::-1][: int(np.sum(s >= aa))]
        np.testing.assert_allclose(nz, np.sort(s[s >= aa])[::-1], atol=1e-12)
        assert np.sum(got > 1e-9) == np.sum(s >= aa)
    else:
        np.testing.assert_allclose(got[:, :2], s[:, :2], atol=1e-12)   # per frequency, leading two
        assert np.all(got[:, 2:] < 1e-9)


def test_spectral_edit_identity_and_full_support():
    w = rand_w(3, 2, 3, 3, 32)
    n, m = 5, 4
    # phi = identity (clip far above sigma_max) returns the kernel itself
    np.testing.assert_allclose(O.spectral_edit(w, n, m, "clip", 1e9), w, atol=1e-12)
    # a kernel covering the whole torus represents every operator: the edit is exact
    wf = rand_w(3, 3, 4, 4, 33)
    n = m = 4
    s = O.lfa_svd(wf, n, m, compute_uv=False)
    c = 0.6 * s.max()
    we = O.spectral_edit(wf, n, m, "clip", c)
    np.testing.assert_allclose(np.sort(O.lfa_svd(we, n, m, compute_uv=False).ravel()),
                               np.sort(np.minimum(s, c).ravel()), atol=1e-12)


# ----------------------------------------------------------------- strided convolutions (crystals)
@pytest.mark.parametrize("c_out,c_in,kh,kw,n,m,sh,sw", [
    (3, 2, 3, 3, 4, 3, 2, 2), (2, 3, 3, 5, 3, 4, 2, 1), (4, 2, 1, 1, 3, 3, 2, 2), (2, 2, 4, 4, 3, 2, 2, 3)])
def test_strided_dense_operator_is_torch_strided_circular_conv(c_out, c_in, kh, kw, n, m, sh, sw):
    w = rand_w(c_out, c_in, kh, kw, 41)
    ph, pw = kh // 2, kw // 2
    A = O.dense_operator_strided(w, n, m, sh, sw)
    f = RNG.standard_normal((c_in, sh * n, sw * m))
    ft = Fnn.pad(torch.as_tensor(f)[None], (pw, kw - 1 - pw, ph, kh - 1 - ph), mode="circular")
    ref = Fnn.conv2d(ft, torch.as_tensor(w), stride=(sh, sw))[0].numpy()
    assert ref.shape == (c_out, n, m)
    np.testing.assert_allclose(A @ f.ravel(), ref.ravel(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("c_out,c_in,kh,kw,n,m,sh,sw", [
    (3, 2, 3, 3, 4, 3, 2, 2), (8, 2, 3, 3, 3, 3, 2, 2), (2, 3, 3, 5, 3, 4, 2, 1), (5, 1, 5, 5, 3, 3, 3, 3)])
def test_strided_dense_svd_is_union_of_crystal_symbol_svds(c_out, c_in, kh, kw, n, m, sh, sw):
    w = rand_w(c_out, c_in, kh, kw, 42)
    dense = np.sort(np.linalg.svd(O.dense_operator_strided(w, n, m, sh, sw), compute_uv=False))[::-1]
    s = O.lfa_svd_strided(w, n, m, sh, sw, compute_uv=False)
    r = min(c_out, c_in * sh * sw)
    assert s.shape == (n * m, r)
    np.testing.assert_allclose(dense[: n * m * r], np.sort(s.ravel())[::-1], atol=1e-12 * dense[0])
    # Parseval: when no two taps alias on the fine torus, every tap appears once per coarse site
    if kh <= sh * n and kw <= sw * m:
        np.testing.assert_allclose(np.sum(s ** 2), n * m * np.sum(w ** 2), rtol=1e-12)


def test_stride_one_reduces_to_the_plain_symbols():
    w = rand_w(3, 4, 3, 5, 43)
    np.testing.assert_allclose(O.symbols_strided(w, 5, 4, 1, 1), O.symbols(w, 5, 4), atol=1e-14)


def test_strided_single_tap_is_a_subsampling():
    """One tap: each output samples one input entry, so every singular value is |w| (closed form)."""
    w = np.zeros((2, 2, 3, 3))
    w[:, :, 1, 2] = 1.5 * np.eye(2)
    s = O.lfa_svd_strided(w, 3, 4, 2, 2, compute_uv=False)
    np.testing.assert_allclose(s, 1.5, atol=1e-14)


def test_strided_lifted_vectors_and_backward():
    c_out, c_in, k, n, m, sh, sw = 3, 2, 3, 3, 4, 2, 2
    w = rand_w(c_out, c_in, k, k, 44)
    A = O.dense_operator_strided(w, n, m, sh, sw)
    s, U, V = O.lfa_svd_strided(w, n, m, sh, sw)
    for f in (0, 5, 7):
        j, l = divmod(f, m)
        uh, vh = O.lift_strided(U[f], V[f], j, l, n, m, sh, sw)
        for q in range(s.shape[1]):
            np.testing.assert_allclose(A @ vh[q].ravel(), s[f, q] * uh[q].ravel(), atol=1e-12)
            assert abs(np.linalg.norm(vh[q]) - 1) < 1e-12
    g = W.upstream_gradient(s.shape, seed=45).astype(np.float64)

    def L(wv):
        return float(np.sum(g * O.lfa_svd_strided(wv, n, m, sh, sw, compute_uv=False)))

    dW = O.lfa_backward_strided(w, n, m, sh, sw, g, U, V)
    h = 1e-6
    fd = np.zeros_like(w)
    for idx in np.ndindex(w.shape):
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        fd[idx] = (L(wp) - L(wm)) / (2 * h)
    np.testing.assert_allclose(dW, fd, rtol=1e-6, atol=1e-8)


# ----------------------------------------------------------------- zero (Dirichlet) boundary conditions
@pytest.mark.parametrize("c_out,c_in,kh,kw,n,m", [(3, 2, 3, 3, 5, 4), (2, 3, 5, 3, 4, 6), (2, 2, 1, 1, 3, 3)])
def test_dirichlet_operator_is_torch_zero_padded_conv(c_out, c_in, kh, kw, n, m):
    w = rand_w(c_out, c_in, kh, kw, 61)
    A = O.dense_operator_dirichlet(w, n, m)
    f = RNG.standard_normal((c_in, n, m))
    ref = Fnn.conv2d(torch.as_tensor(f)[None], torch.as_tensor(w), padding=(kh // 2, kw // 2))[0].numpy()
    np.testing.assert_allclose(A @ f.ravel(), ref.ravel(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,m,k", [(4, 4, 3), (5, 3, 3), (3, 4, 5)])
def test_dirichlet_spectrum_interlaces_the_periodic_one_on_the_padded_torus(n, m, k):
    """The zero-padded operator on n x m is a compression S^T A S of the periodic operator on the
    (n + k - 1) x (m + k - 1) torus (no wrap-around reaches the grid), so its singular values are
    bounded one by one by the periodic ones (interlacing for submatrices)."""
    w = rand_w(3, 3, k, k, 62)
    sd = np.sort(np.linalg.svd(O.dense_operator_dirichlet(w, n, m), compute_uv=False))[::-1]
    sp = np.sort(O.dense_svd(w, n + k - 1, m + k - 1))[::-1]
    assert np.all(sd <= sp[: sd.size] + 1e-12)


def test_dirichlet_equals_periodic_for_1x1_kernels():
    w = rand_w(4, 3, 1, 1, 63)
    np.testing.assert_allclose(O.dense_operator_dirichlet(w, 4, 5), O.dense_operator(w, 4, 5), atol=0)


# ----------------------------------------------------------------- pseudo-inverse projected on taps
@pytest.mark.parametrize("c_out,c_in,k,n,m,a", [(3, 2, 3, 4, 5, 0.0), (2, 3, 3, 5, 4, 0.0), (3, 3, 3, 4, 4, 0.3)])
def test_pinv_projection_matches_the_dense_pseudo_inverse(c_out, c_in, k, n, m, a):
    w = rand_w(c_out, c_in, k, k, 71)
    got = O.pinv_projection(w, n, m, a)
    ref = O.dense_pinv_projection(w, n, m, a)
    assert got.shape == (c_in, c_out, k, k)
    np.testing.assert_allclose(got, ref, atol=1e-10 * np.max(np.abs(ref)))


def test_pinv_of_a_scaled_identity_kernel_is_exact():
    """w = 2 delta I: the operator is 2 Id, its inverse 0.5 Id, itself a 3x3 kernel."""
    w = np.zeros((3, 3, 3, 3))
    w[:, :, 1, 1] = 2.0 * np.eye(3)
    ref = np.zeros_like(w)
    ref[:, :, 1, 1] = 0.5 * np.eye(3)
    np.testing.assert_allclose(O.pinv_projection(w, 4, 5, 0.0), ref, atol=1e-14)
