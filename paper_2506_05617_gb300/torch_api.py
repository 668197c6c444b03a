"""PyTorch-facing wrapper over the C ABI: torch supplies device memory and streams only.

``LfaPlan`` owns a C plan and allocates the output tensors; ``LfaSvd`` is the
``torch.autograd.Function`` whose forward is ``lfa_svd`` and whose backward is
``lfa_svd_backward`` (dL/dw from dL/dsigma, Sec. III symbol derivative). All
arithmetic runs in the CUDA library.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from . import lfa as C


def _layer_tuple(d):
    L = C.layer_desc(d)
    t = tuple(getattr(L, k) for k, _ in L._fields_)
    return t[:8] + tuple(max(1, v) for v in t[8:])


class LfaPlan:
    """A plan over ``layers``: each (c_out, c_in, kh, kw, n, m[, pad_h, pad_w[, stride_h, stride_w]]).

    A strided layer's symbol has c_in * stride_h * stride_w columns (the input's polyphase
    components); its V has that many rows and its v_hat lives on the (stride_h n) x (stride_w m)
    input torus."""

    def __init__(self, layers: Sequence, vectors: bool = False, half_output: bool = False,
                 plain: bool = False, tol: float = 0.0, max_sweeps: int = 0, variant: int = -1,
                 use_graph: int = -1, tune_cache: Optional[str] = None, shard: tuple = (0, 1),
                 fft_route: bool = False, reproducible: bool = False):
        self.layers = [_layer_tuple(d) for d in layers]
        self.vectors = bool(vectors)
        self.half_output = bool(half_output)
        flags = C.LFA_VALUES | (C.LFA_VECTORS if vectors else 0) | (C.LFA_HALF_OUTPUT if half_output else 0) \
            | (C.LFA_PLAIN if plain else 0) | (C.LFA_FFT_ROUTE if fft_route else 0) \
            | (C.LFA_REPRODUCIBLE if reproducible else 0)
        self.shard = (int(shard[0]), int(shard[1]))
        self.handle = C.lfa_plan(self.layers, flags, tol, max_sweeps, variant, use_graph, tune_cache,
                                 self.shard[0], self.shard[1])
        self.meta = [C.lfa_layer_query(self.handle, i) for i in range(len(self.layers))]

    # ------------------------------------------------------------------ shapes
    def symbol_cols(self, i):
        c_in, sh, sw = self.layers[i][1], self.layers[i][8], self.layers[i][9]
        return c_in * sh * sw

    def sigma_shape(self, i):
        c_out, n, m = self.layers[i][0], self.layers[i][4], self.layers[i][5]
        r = min(c_out, self.symbol_cols(i))
        return (self.meta[i]["F_h"], r) if self.half_output else (n * m, r)

    def u_shape(self, i):
        c_out = self.layers[i][0]
        return (self.meta[i]["F_h"], c_out, min(c_out, self.symbol_cols(i)))

    def v_shape(self, i):
        c_out, ci = self.layers[i][0], self.symbol_cols(i)
        return (self.meta[i]["F_h"], ci, min(c_out, ci))

    def alloc(self, device="cuda"):
        sig = [torch.empty(self.sigma_shape(i), dtype=torch.float32, device=device) for i in range(len(self.layers))]
        if not self.vectors:
            return sig, None, None
        U = [torch.empty(self.u_shape(i), dtype=torch.complex64, device=device) for i in range(len(self.layers))]
        V = [torch.empty(self.v_shape(i), dtype=torch.complex64, device=device) for i in range(len(self.layers))]
        return sig, U, V

    # ------------------------------------------------------------------ calls
    def svd(self, weights: Sequence[torch.Tensor], out=None, stream=None):
        ws = [w.contiguous() for w in weights]
        for i, w in enumerate(ws):
            if w.dtype != torch.float32 or not w.is_cuda or tuple(w.shape) != tuple(self.layers[i][:4]):
                raise ValueError(f"layer {i}: weights must be float32 CUDA [{self.layers[i][:4]}]")
        sig, U, V = out if out is not None else self.alloc(ws[0].device)
        stream = stream if stream is not None else torch.cuda.current_stream(ws[0].device)
        C.lfa_svd(self.handle, [w.data_ptr() for w in ws], [s.data_ptr() for s in sig],
                  [u.data_ptr() for u in U] if U else None, [v.data_ptr() for v in V] if V else None, stream)
        return sig, U, V

    def backward(self, dsigma: Sequence[torch.Tensor], U, V, dw=None, stream=None):
        if dw is None:
            dw = [torch.empty(self.layers[i][:4], dtype=torch.float32, device=U[0].device)
                  for i in range(len(self.layers))]
        ds = [d.contiguous().float() for d in dsigma]
        stream = stream if stream is not None else torch.cuda.current_stream(U[0].device)
        C.lfa_svd_backward(self.handle, [d.data_ptr() for d in ds], [u.data_ptr() for u in U],
                           [v.data_ptr() for v in V], [d.data_ptr() for d in dw], stream)
        return dw

    def regulariser_grad(self, sigma, lam: float, dsigma=None, loss=None, stream=None):
        if dsigma is None:
            dsigma = [torch.empty_like(s) for s in sigma]
        if loss is None:
            loss = [torch.empty((), dtype=torch.float32, device=sigma[0].device) for _ in sigma]
        stream = stream if stream is not None else torch.cuda.current_stream(sigma[0].device)
        C.lfa_regulariser_grad(self.handle, [s.data_ptr() for s in sigma], lam, [d.data_ptr() for d in dsigma],
                               [l.data_ptr() for l in loss], stream)
        return dsigma, loss

    def spectral_edit(self, sigma, U, V, mode: str, a: float, b: float = 0.0, stream=None):
        """Kernels nearest to the operators with edited singular values (see lfa_spectral_edit);
        mode "pinv" returns [c_in, c_out, kh, kw] kernels nearest to the pseudo-inverses."""
        modes = {"clip": C.LFA_EDIT_CLIP, "clamp": C.LFA_EDIT_CLAMP, "threshold": C.LFA_EDIT_THRESHOLD,
                 "rank": C.LFA_EDIT_RANK, "pinv": C.LFA_EDIT_PINV}
        def shape(i):
            c_out, c_in, kh, kw = self.layers[i][:4]
            return (c_in, c_out, kh, kw) if mode == "pinv" else (c_out, c_in, kh, kw)
        out = [torch.empty(shape(i), dtype=torch.float32, device=U[0].device) for i in range(len(self.layers))]
        stream = stream if stream is not None else torch.cuda.current_stream(U[0].device)
        C.lfa_spectral_edit(self.handle, [s.data_ptr() for s in sigma], [u.data_ptr() for u in U],
                            [v.data_ptr() for v in V], modes[mode], a, b, [o.data_ptr() for o in out], stream)
        return out

    def symbols(self, layer: int, w: torch.Tensor, stream=None):
        c_out = self.layers[layer][0]
        out = torch.empty((self.meta[layer]["F_h"], c_out, self.symbol_cols(layer)), dtype=torch.complex64,
                          device=w.device)
        stream = stream if stream is not None else torch.cuda.current_stream(w.device)
        C.lfa_symbols(self.handle, layer, w.contiguous().data_ptr(), out.data_ptr(), stream)
        return out

    def fft_symbols(self, layer: int, w: torch.Tensor, stream=None):
        """The half-grid symbols through the FFT route (plan made with fft_route=True)."""
        c_out = self.layers[layer][0]
        out = torch.empty((self.meta[layer]["F_h"], c_out, self.symbol_cols(layer)), dtype=torch.complex64,
                          device=w.device)
        stream = stream if stream is not None else torch.cuda.current_stream(w.device)
        C.lfa_fft_symbols(self.handle, layer, w.contiguous().data_ptr(), out.data_ptr(), stream)
        return out

    def expand(self, layer: int, U, V, first: int, count: int, stream=None):
        c_out, c_in, kh, kw, n, m, _, _, sh, sw = self.layers[layer]
        dev = (U if U is not None else V).device
        u_hat = torch.empty((count, c_out, n, m), dtype=torch.complex64, device=dev) if U is not None else None
        v_hat = torch.empty((count, c_in, sh * n, sw * m), dtype=torch.complex64, device=dev) \
            if V is not None else None
        stream = stream if stream is not None else torch.cuda.current_stream(dev)
        C.lfa_expand(self.handle, layer, U.data_ptr() if U is not None else 0, V.data_ptr() if V is not None else 0,
                     first, count, u_hat.data_ptr() if u_hat is not None else 0,
                     v_hat.data_ptr() if v_hat is not None else 0, stream)
        return u_hat, v_hat

    def info(self):
        return C.lfa_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            C.lfa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LfaSvd(torch.autograd.Function):
    """sigma = LFA-SVD(w) per layer; backward gives dL/dw through the hand-written kernel."""

    @staticmethod
    def forward(ctx, plan: LfaPlan, *weights):
        if not plan.vectors:
            raise ValueError("LfaSvd needs a plan created with vectors=True")
        sig, U, V = plan.svd(weights)
        ctx.plan = plan
        ctx.save_for_backward(*U, *V)
        ctx.nl = len(weights)
        return tuple(sig)

    @staticmethod
    def backward(ctx, *dsig):
        saved = ctx.saved_tensors
        U, V = list(saved[:ctx.nl]), list(saved[ctx.nl:])
        dsig = [d if d is not None else torch.zeros(ctx.plan.sigma_shape(i), device=U[0].device)
                for i, d in enumerate(dsig)]
        dw = ctx.plan.backward(dsig, U, V)
        return (None, *dw)


def svd(weights: Sequence[torch.Tensor], n: int, m: Optional[int] = None, vectors: bool = True,
        stride=1, **kw):
    """Convenience: singular values (and U, V) of each conv layer with an n x m output torus
    (stride (s_h, s_w), or one int for both: the input torus is s_h n x s_w m)."""
    m = n if m is None else m
    sh, sw = (stride, stride) if isinstance(stride, int) else tuple(stride)
    plan = LfaPlan([tuple(w.shape) + (n, m, -1, -1, sh, sw) for w in weights], vectors=vectors, **kw)
    sig, U, V = plan.svd(weights)
    return plan, sig, U, V
