"""FP64 CPU oracle for the SVD of stride-1 periodic multi-channel 2-D convolutions.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module. The product path (the CUDA
library and its Python binding) never calls it, and it imports nothing from the
product package.

What it computes, and where the paper defines it (arXiv 2506.05617, Sec. III):

* ``dense_operator`` -- the convolution as a multiplication operator on the
  periodic crystal torus, (A f)(x) = sum_{y in N} M_y f(x + y) ("Convolutional
  Mappings"), unrolled into the dense (c_out*n*m) x (c_in*n*m) matrix that the
  paper's brute-force baseline decomposes (Sec. I, Sec. IV "Runtime Analysis").
  ``dense_svd`` is its full LAPACK SVD. This is the plain definition.
* ``symbols`` -- the symbol A_k = sum_{y in N} M_y exp(2 pi i <k, y>) at every
  frequency k of the frequency torus T*_{n,m} ("Convolution Theorem"; line 4 of
  Algorithm 1).
* ``lfa_svd`` -- Algorithm 1: a LAPACK SVD A_k = U_k S_k V_k^* of every symbol.
* ``lift`` -- the global singular vectors U^_k = F_k^out U_k and V^_k = F_k^in V_k,
  whose columns are (channel vector) (x) (Fourier mode / sqrt(nm)).
* ``fft_symbols`` -- the FFT route of the paper's comparison system (Sec. II,
  Sec. IV): a 2-D FFT of the zero-padded, origin-shifted kernel. It yields the
  complex conjugate of the symbol, so the same singular values.
* ``lfa_backward`` -- dL/dw for a loss L(sigma): with d(sigma_s) = Re(u_s^* dA_k v_s)
  and dA_k/dw[o,i,a,b] = exp(2 pi i <k, y_ab>) e_o e_i^T (symbol definition above),
  dL/dw[o,i,a,b] = sum_k sum_s g_{k,s} Re(conj(U_k[o,s]) V_k[i,s] exp(2 pi i <k,y_ab>)).

Conventions (readings of the paper where it is ambiguous):
* Rows of the torus are n (index j of the frequency, a of the tap, x1 of the
  pixel); columns are m (l, b, x2). Frequencies are enumerated row-major,
  f = j*m + l. The paper's Algorithm 1 loops X over n and Y over m.
* Tap (a, b) sits at offset y = (a - p_h, b - p_w); p defaults to floor(k/2),
  the stencil centred at x. The exponent sign is +, as in the symbol definition
  (cross-correlation, f(x + y)).
* The symbol is c_out x c_in. For c_in != c_out only r = min(c_in, c_out)
  singular values per frequency are returned; the dense operator has
  |c_out - c_in|*n*m further singular values that are exactly zero.
* Singular values are sorted in descending order within each frequency.
* Phases are reduced exactly on integers: (j*(a - p_h)) mod n, then exp in fp64.

Every function works in float64 / complex128. Inputs may be float32 arrays; they
are upcast exactly.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "origin", "dense_operator", "dense_svd", "symbols", "fft_symbols", "lfa_svd",
    "lift", "apply_operator", "apply_adjoint", "half_grid", "lfa_backward",
    "regulariser_loss", "regulariser_grad_sigma", "folded_kernel", "edit_values",
    "spectral_edit", "dense_spectral_edit", "pinv_projection", "dense_pinv_projection", "dense_operator_strided", "symbols_strided",
    "lfa_svd_strided", "lfa_backward_strided", "lift_strided", "dense_operator_dirichlet",
]


def origin(kh: int, kw: int, pad_h: int = -1, pad_w: int = -1):
    """Tap origin p = (p_h, p_w); -1 selects floor(k/2), the centred stencil (Sec. III, 3x3 stencil figure)."""
    return (kh // 2 if pad_h < 0 else pad_h, kw // 2 if pad_w < 0 else pad_w)


# --------------------------------------------------------------------------- O1: the definition
def dense_operator(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """Dense periodic operator, Sec. III "Convolutional Mappings": (A f)(x) = sum_y M_y f(x + y).

    Row index (o, x1, x2) -> o*n*m + x1*m + x2; column index (i, z1, z2) likewise.
    Entry [(o, x), (i, x + y_ab mod (n, m))] accumulates w[o, i, a, b]; taps that
    alias (k > n) add up, as the periodic torus requires.
    """
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    F = n * m
    A = np.zeros((c_out * F, c_in * F), dtype=np.float64)
    x1, x2 = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    pix = (x1 * m + x2).ravel()
    for a in range(kh):
        for b in range(kw):
            src = (((x1 + a - ph) % n) * m + ((x2 + b - pw) % m)).ravel()
            for o in range(c_out):
                for i in range(c_in):
                    np.add.at(A, (o * F + pix, i * F + src), w[o, i, a, b])
    return A


def dense_svd(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1, compute_uv: bool = False):
    """Full LAPACK SVD of the dense operator (the paper's explicit baseline)."""
    A = dense_operator(w, n, m, pad_h, pad_w)
    return np.linalg.svd(A, compute_uv=compute_uv)


def apply_operator(w, f, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """(A f)(o, x) = sum_{i,a,b} w[o,i,a,b] f(i, x + y_ab) on the torus, without forming A.

    ``f`` is [c_in, n, m] (real or complex); returns [c_out, n, m]. Used for residuals
    at sizes where the dense matrix does not fit.
    """
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    f = np.asarray(f)
    out = np.zeros((c_out,) + f.shape[1:], dtype=np.result_type(f.dtype, np.float64))
    for a in range(kh):
        for b in range(kw):
            # g(i, x) = f(i, x + y): shifting by -y brings x + y to x
            g = np.roll(f, shift=(-(a - ph), -(b - pw)), axis=(1, 2))
            out += np.tensordot(w[:, :, a, b], g, axes=([1], [0]))
    return out


def apply_adjoint(w, g, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """(A^T g)(i, z) = sum_{o,a,b} w[o,i,a,b] g(o, z - y_ab); ``g`` is [c_out, n, m]."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    g = np.asarray(g)
    out = np.zeros((c_in,) + g.shape[1:], dtype=np.result_type(g.dtype, np.float64))
    for a in range(kh):
        for b in range(kw):
            h = np.roll(g, shift=(a - ph, b - pw), axis=(1, 2))
            out += np.tensordot(w[:, :, a, b].T, h, axes=([1], [0]))
    return out


# --------------------------------------------------------------------------- O2: Algorithm 1
def _phase(n: int, m: int, dy1: int, dy2: int) -> np.ndarray:
    """exp(2 pi i <k, y>) for all k = (j/n, l/m) of T*_{n,m}, y = (dy1, dy2); shape [n, m].

    The integer products j*dy1 and l*dy2 are reduced mod n and mod m before the
    exponential, so the phase is exact up to one fp64 rounding of exp.
    """
    j = np.arange(n)[:, None]
    l = np.arange(m)[None, :]
    t = ((j * dy1) % n) / n + ((l * dy2) % m) / m
    return np.exp(2j * np.pi * t)


def symbols(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1, freqs=None) -> np.ndarray:
    """Symbols A_k = sum_{y in N} M_y exp(2 pi i <k, y>) for all n*m frequencies (Sec. III, Alg. 1 line 4).

    Returns complex128 [n*m, c_out, c_in]; frequency f = j*m + l is k = (j/n, l/m).
    ``freqs`` (optional index array) restricts the output to those frequencies, in that order.
    """
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    sel = np.arange(n * m) if freqs is None else np.asarray(freqs)
    S = np.zeros((len(sel), c_out, c_in), dtype=np.complex128)
    for a in range(kh):
        for b in range(kw):
            S += _phase(n, m, a - ph, b - pw).reshape(n * m)[sel][:, None, None] * w[None, :, :, a, b]
    return S


def fft_symbols(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """FFT route (the paper's comparison system, Sec. II and IV): fft2 of the zero-padded kernel.

    The kernel is placed on the n x m grid at its offsets y_ab mod (n, m) (rolled by -p,
    aliasing taps added), then transformed with numpy's FFT over the spatial axes.
    numpy's forward FFT uses exp(-2 pi i ...), so the result is conj(A_k). Returns
    complex128 [n*m, c_out, c_in].
    """
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    K = np.zeros((c_out, c_in, n, m), dtype=np.float64)
    for a in range(kh):
        for b in range(kw):
            K[:, :, (a - ph) % n, (b - pw) % m] += w[:, :, a, b]
    Fk = np.fft.fft2(K, axes=(2, 3))                      # [c_out, c_in, n, m]
    return np.ascontiguousarray(Fk.transpose(2, 3, 0, 1)).reshape(n * m, c_out, c_in)


def lfa_svd(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1, compute_uv: bool = True, freqs=None):
    """Algorithm 1 in FP64: a LAPACK SVD of the symbol at every frequency of T*_{n,m}.

    Returns ``sigma`` [n*m, r] (descending per frequency) and, when ``compute_uv``,
    ``U`` [n*m, c_out, r] and ``V`` [n*m, c_in, r] with A_k = U_k diag(sigma_k) V_k^*.
    ``freqs`` restricts the loop to those frequencies (rows follow ``freqs``).
    """
    S = symbols(w, n, m, pad_h, pad_w, freqs)
    if not compute_uv:
        return np.linalg.svd(S, compute_uv=False)
    U, s, Vh = np.linalg.svd(S, full_matrices=False)
    V = np.conj(np.swapaxes(Vh, 1, 2))
    return s, U, V


def lift(U_k, V_k, j: int, l: int, n: int, m: int):
    """Global singular vectors of one frequency, U^_k = F_k^out U_k and V^_k = F_k^in V_k (Sec. III).

    ``U_k`` [c_out, q] and ``V_k`` [c_in, q] hold q symbol singular vectors. The
    Fourier mode is f_k(x) = exp(2 pi i (j x1 / n + l x2 / m)) / sqrt(n m) on the
    row-major grid. Returns u_hat [q, c_out, n, m] and v_hat [q, c_in, n, m].
    """
    t = ((j * np.arange(n))[:, None] % n) / n + ((l * np.arange(m))[None, :] % m) / m
    mode = np.exp(2j * np.pi * t) / np.sqrt(n * m)
    u_hat = np.einsum("cq,xy->qcxy", np.asarray(U_k), mode)
    v_hat = np.einsum("cq,xy->qcxy", np.asarray(V_k), mode)
    return u_hat, v_hat


def half_grid(n: int, m: int) -> np.ndarray:
    """Frequencies f = j*m + l that represent their conjugate pair {k, -k}.

    For a real kernel A_{-k} = conj(A_k) (symbol definition), so one member of each
    pair carries all the information. The representative is the member with the
    smaller row-major index; self-conjugate frequencies represent themselves.
    Returned in increasing order; its length is (n*m + s)/2 with s the number of
    self-conjugate frequencies.
    """
    j, l = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    f = (j * m + l).ravel()
    fc = (((-j) % n) * m + ((-l) % m)).ravel()
    return f[f <= fc]


def folded_kernel(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """Kernel folded onto the torus: taps with equal offsets mod (n, m) added; [c_out, c_in, n, m]."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    K = np.zeros((c_out, c_in, n, m))
    for a in range(kh):
        for b in range(kw):
            K[:, :, (a - ph) % n, (b - pw) % m] += w[:, :, a, b]
    return K


# --------------------------------------------------------------------------- backward
def lfa_backward(w, n: int, m: int, g, U, V, pad_h: int = -1, pad_w: int = -1, freqs=None) -> np.ndarray:
    """dL/dw from the upstream gradient ``g`` = dL/dsigma [n*m, r] and the per-frequency U, V.

    Uses d(sigma_s) = Re(u_s^* dA_k v_s) for a simple singular value and the symbol
    definition dA_k/dw[o,i,a,b] = exp(2 pi i <k, y_ab>) e_o e_i^T, summed over the
    full frequency grid:
        dW[o,i,a,b] = sum_k Re( sum_s g[k,s] conj(U_k[o,s]) V_k[i,s] exp(2 pi i <k, y_ab>) ).
    ``freqs`` restricts the sum to those frequencies (rows of g, U, V follow ``freqs``).
    """
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    g = np.asarray(g, dtype=np.float64)
    H = np.einsum("fs,fos,fis->foi", g, np.conj(U), V)   # [F, c_out, c_in]
    dW = np.zeros_like(w)
    for a in range(kh):
        for b in range(kw):
            ph_k = _phase(n, m, a - ph, b - pw).reshape(n * m)
            if freqs is not None:
                ph_k = ph_k[np.asarray(freqs)]
            dW[:, :, a, b] = np.real(np.einsum("f,foi->oi", ph_k, H))
    return dW


def regulariser_loss(sigmas, lam: float) -> float:
    """Spectral regulariser over layers: sum_layers max(sigma) + lam * sum (sigma - 1)^2."""
    return float(sum(np.max(s) + lam * np.sum((np.asarray(s, np.float64) - 1.0) ** 2) for s in sigmas))


def regulariser_grad_sigma(sigma, lam: float) -> np.ndarray:
    """d/dsigma of max(sigma) + lam * sum (sigma - 1)^2 for one layer's [F, r] array.

    The max term contributes 1 at the first maximiser in row-major order. The largest
    singular value is attained at both k and -k, but sigma_k and sigma_{-k} are the same
    function of w, so either member gives the same gradient through ``lfa_backward``.
    """
    s = np.asarray(sigma, np.float64)
    g = 2.0 * lam * (s - 1.0)
    idx = np.unravel_index(int(np.argmax(s)), s.shape)
    g[idx] += 1.0
    return g


# --------------------------------------------------------------------------- spectral editing
def edit_values(sigma, mode: str, a: float, b: float = 0.0) -> np.ndarray:
    """The map phi applied to every singular value (applications of Sec. I-II: clipping the
    spectral norm, hard thresholding / low rank). ``sigma`` is [F, r], descending per row.

    clip: min(s, a); clamp: min(max(s, a), b); threshold: s if s >= a else 0;
    rank: the first round(a) values of every frequency kept, the rest 0.
    """
    s = np.asarray(sigma, np.float64)
    if mode == "clip":
        return np.minimum(s, a)
    if mode == "clamp":
        return np.minimum(np.maximum(s, a), b)
    if mode == "threshold":
        return np.where(s >= a, s, 0.0)
    if mode == "rank":
        out = s.copy()
        out[:, int(round(a)):] = 0.0
        return out
    raise ValueError(mode)


def spectral_edit(w, n: int, m: int, mode: str, a: float, b: float = 0.0, pad_h: int = -1, pad_w: int = -1):
    """The kh x kw kernel nearest (Frobenius norm of the operator) to U phi(S) V^*.

    The edited operator B has symbols B_k = U_k phi(S_k) V_k^*. The operators of single taps,
    T[(o, x), (i, x + y_ab)] = 1, are mutually orthogonal with <T, T> = n m when no taps alias
    (k <= n, m), so the projection of B onto their span has weights
        w'[o,i,a,b] = <B, T_oiab> / (n m) = (1/(n m)) sum_k Re(B_k[o,i] exp(-2 pi i <k, y_ab>)).
    """
    s, U, V = lfa_svd(w, n, m, pad_h, pad_w)
    g = edit_values(s, mode, a, b) / (n * m)
    return lfa_backward(w, n, m, g, U, V, pad_h, pad_w)


def dense_spectral_edit(w, n: int, m: int, mode: str, a: float, b: float = 0.0, pad_h: int = -1, pad_w: int = -1):
    """The same projection from the dense operator: full LAPACK SVD, phi on the values grouped
    by frequency through the lifted vectors, then <B, T_oiab> / <T, T> with the tap operators
    built entry by entry (small sizes only). Independent of the symbol formula."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    s, U, V = lfa_svd(w, n, m, pad_h, pad_w)
    sp = edit_values(s, mode, a, b)
    B = np.zeros((c_out * n * m, c_in * n * m), dtype=np.complex128)
    for f in range(n * m):
        j, l = divmod(f, m)
        uh, vh = lift(U[f], V[f], j, l, n, m)
        Uf = uh.reshape(uh.shape[0], -1).T          # [c_out n m, r]
        Vf = vh.reshape(vh.shape[0], -1).T
        B += (Uf * sp[f][None, :]) @ Vf.conj().T
    out = np.zeros_like(w)
    basis = np.zeros_like(w)
    for idx in np.ndindex(w.shape):
        basis[idx] = 1.0
        T = dense_operator(basis, n, m, pad_h, pad_w)
        out[idx] = np.real(np.sum(B * T)) / np.sum(T * T)
        basis[idx] = 0.0
    return out


def pinv_projection(w, n: int, m: int, a: float, pad_h: int = -1, pad_w: int = -1):
    """The kh x kw kernel [c_in, c_out, kh, kw] of a c_out -> c_in convolution nearest to the
    pseudo-inverse A^+ of the layer (singular values <= a treated as zero), the pseudo-inverse
    application of Sec. II. A^+ has the symbols B_k = V_k S_k^+ U_k^* (same Fourier modes), so the
    projection is the formula of ``spectral_edit`` with the roles of U and V exchanged:
        w'[i,o,a,b] = (1/(n m)) sum_k Re(B_k[i,o] exp(-2 pi i <k, y_ab>)).
    """
    w = np.asarray(w, dtype=np.float64)
    s, U, V = lfa_svd(w, n, m, pad_h, pad_w)
    inv = np.where(s > a, 1.0 / np.where(s > a, s, 1.0), 0.0)
    shape_t = np.zeros((w.shape[1], w.shape[0], w.shape[2], w.shape[3]))
    return lfa_backward(shape_t, n, m, inv / (n * m), V, U, pad_h, pad_w)


def dense_pinv_projection(w, n: int, m: int, a: float, pad_h: int = -1, pad_w: int = -1):
    """The same kernel from the dense operator: LAPACK pseudo-inverse of the unrolled matrix
    (values <= a dropped), then <A^+, T> / <T, T> for the tap operators T of a c_out -> c_in
    convolution built entry by entry (small sizes only). Independent of the symbols."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    A = dense_operator(w, n, m, pad_h, pad_w)
    Uu, sv, Vh = np.linalg.svd(A, full_matrices=False)
    keep = sv > a
    B = (Vh[keep].T / sv[keep]) @ Uu[:, keep].T                    # [c_in n m, c_out n m]
    out = np.zeros((c_in, c_out, kh, kw))
    basis = np.zeros_like(out)
    for idx in np.ndindex(out.shape):
        basis[idx] = 1.0
        T = dense_operator(basis, n, m, pad_h, pad_w)
        out[idx] = np.sum(B * T) / np.sum(T * T)
        basis[idx] = 0.0
    return out


# --------------------------------------------------------------------------- strided convolutions
# A stride-(s_h, s_w) convolution maps an input on the fine (s_h n) x (s_w m) torus to an output on
# the coarse n x m torus, (A f)(o, x) = sum_{i,a,b} w[o,i,a,b] f(i, s x + y_ab). Seen as a crystal
# (Sec. III "Introduction to Lattices and Crystals"), the input has s_h s_w points per coarse unit
# cell: the polyphase components f(i, s x + u), u in [0, s_h) x [0, s_w). A tap at offset
# y = s q + u (q = floor(y / s) componentwise) couples component u at coarse offset q, so the
# Fourier modes of the coarse torus are again invariant and the symbol is the c_out x (c_in s_h s_w)
# matrix  A_k[o, (i, u)] = sum_{taps with y mod s = u} w[o,i,a,b] exp(2 pi i <k, q>).
# Columns are ordered (i, u_h, u_w) -> i s_h s_w + u_h s_w + u_w.

def dense_operator_strided(w, n: int, m: int, s_h: int, s_w: int, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """Dense strided periodic operator: row (o, x1, x2) of the coarse grid, column (i, z1, z2) of the
    fine grid, entry [(o, x), (i, s x + y_ab mod (s_h n, s_w m))] += w[o, i, a, b]."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    N1, N2 = s_h * n, s_w * m
    A = np.zeros((c_out * n * m, c_in * N1 * N2), dtype=np.float64)
    x1, x2 = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    pix = (x1 * m + x2).ravel()
    for a in range(kh):
        for b in range(kw):
            src = (((s_h * x1 + a - ph) % N1) * N2 + ((s_w * x2 + b - pw) % N2)).ravel()
            for o in range(c_out):
                for i in range(c_in):
                    np.add.at(A, (o * n * m + pix, i * N1 * N2 + src), w[o, i, a, b])
    return A


def symbols_strided(w, n: int, m: int, s_h: int, s_w: int, pad_h: int = -1, pad_w: int = -1, freqs=None):
    """Strided symbols [n m (or len(freqs)), c_out, c_in s_h s_w] (see the block comment above)."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    S = s_h * s_w
    sel = np.arange(n * m) if freqs is None else np.asarray(freqs)
    out = np.zeros((len(sel), c_out, c_in * S), dtype=np.complex128)
    for a in range(kh):
        for b in range(kw):
            qh, uh = divmod(a - ph, s_h)      # python floor division: y = s q + u, 0 <= u < s
            qw, uw = divmod(b - pw, s_w)
            phase = _phase(n, m, qh, qw).reshape(n * m)[sel]
            cols = np.arange(c_in) * S + uh * s_w + uw
            out[:, :, cols] += phase[:, None, None] * w[None, :, :, a, b]
    return out


def lfa_svd_strided(w, n: int, m: int, s_h: int, s_w: int, pad_h: int = -1, pad_w: int = -1,
                    compute_uv: bool = True, freqs=None):
    """Per-frequency LAPACK SVD of the strided symbols (Algorithm 1 on the crystal)."""
    S = symbols_strided(w, n, m, s_h, s_w, pad_h, pad_w, freqs)
    if not compute_uv:
        return np.linalg.svd(S, compute_uv=False)
    U, sv, Vh = np.linalg.svd(S, full_matrices=False)
    return sv, U, np.conj(np.swapaxes(Vh, 1, 2))


def lfa_backward_strided(w, n: int, m: int, s_h: int, s_w: int, g, U, V, pad_h: int = -1, pad_w: int = -1,
                         freqs=None):
    """dL/dw for the strided operator: dW[o,i,a,b] = sum_k Re(sum_s g conj(U[o,s]) V[(i,u_ab),s] exp(2 pi i <k,q_ab>)),
    the sum over all n m frequencies, or over ``freqs`` (then g, U, V hold those rows only)."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    S = s_h * s_w
    H = np.einsum("fs,fos,fcs->foc", np.asarray(g, np.float64), np.conj(U), V)   # [F, c_out, c_in S]
    dW = np.zeros_like(w)
    for a in range(kh):
        for b in range(kw):
            qh, uh = divmod(a - ph, s_h)
            qw, uw = divmod(b - pw, s_w)
            phase = _phase(n, m, qh, qw).reshape(n * m)
            if freqs is not None:
                phase = phase[np.asarray(freqs)]
            cols = np.arange(c_in) * S + uh * s_w + uw
            dW[:, :, a, b] = np.real(np.einsum("f,foi->oi", phase, H[:, :, cols]))
    return dW


def lift_strided(U_k, V_k, j: int, l: int, n: int, m: int, s_h: int, s_w: int):
    """Global singular vectors of a strided operator: u_hat on the coarse grid [q, c_out, n, m] as in
    ``lift``; v_hat on the fine grid [q, c_in, s_h n, s_w m] with v_hat[i, s x + u] = V[(i,u)] f_k(x)."""
    c_in_s = np.asarray(V_k).shape[0]
    S = s_h * s_w
    c_in = c_in_s // S
    t = ((j * np.arange(n))[:, None] % n) / n + ((l * np.arange(m))[None, :] % m) / m
    mode = np.exp(2j * np.pi * t) / np.sqrt(n * m)
    u_hat = np.einsum("cq,xy->qcxy", np.asarray(U_k), mode)
    Vr = np.asarray(V_k).reshape(c_in, s_h, s_w, -1)                 # [i, u_h, u_w, q]
    v = np.einsum("iabq,xy->qixayb", Vr, mode)                        # [q, i, x1, u_h, x2, u_w]
    v_hat = v.reshape(v.shape[0], c_in, n * s_h, m * s_w)
    return u_hat, v_hat


# --------------------------------------------------------------------------- boundary conditions
# LFA is exact for periodic boundary conditions (Sec. III); the paper compares its spectra with
# those of the same convolution under zero (Dirichlet) padding (Sec. III "Boundary Conditions"),
# where the operator is no longer block-diagonalised by Fourier modes and only a dense SVD applies.

def dense_operator_dirichlet(w, n: int, m: int, pad_h: int = -1, pad_w: int = -1) -> np.ndarray:
    """Dense zero-padded convolution on an n x m grid: row (o, x1, x2), column (i, z1, z2) with
    z = x + y_ab inside the grid (taps that leave it read zero): entry += w[o, i, a, b]."""
    w = np.asarray(w, dtype=np.float64)
    c_out, c_in, kh, kw = w.shape
    ph, pw = origin(kh, kw, pad_h, pad_w)
    A = np.zeros((c_out * n * m, c_in * n * m), dtype=np.float64)
    for a in range(kh):
        for b in range(kw):
            for x1 in range(n):
                z1 = x1 + a - ph
                if not 0 <= z1 < n:
                    continue
                for x2 in range(m):
                    z2 = x2 + b - pw
                    if not 0 <= z2 < m:
                        continue
                    rows = np.arange(c_out) * n * m + x1 * m + x2
                    cols = np.arange(c_in) * n * m + z1 * m + z2
                    A[np.ix_(rows, cols)] += w[:, :, a, b]
    return A
