"""Thin Python binding of the C ABI in ``include/lfa.h`` (argument marshalling only).

Each function has the name of the C entry point it calls and takes plain Python
values: device pointers as ints, per-layer pointer lists as Python lists of ints,
streams as ints (``torch.cuda.Stream.cuda_stream``) or None. Every step of the
computation runs in the CUDA library; if ``liblfa.so`` is missing this module
raises instead of computing anything another way.

A non-OK status raises :class:`LfaError` except where a function documents that it
returns the status (``lfa_get_info``).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int32, c_int64, c_uint16, c_uint32, c_void_p
from typing import Iterable, List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
# LFA_DEBUG=1 loads the index-checked build (build.py --debug)
LIB_PATH = os.path.join(HERE, "lib", "liblfa_debug.so" if os.environ.get("LFA_DEBUG") == "1" else "liblfa.so")

# flags (include/lfa.h)
LFA_VALUES = 0x1
LFA_VECTORS = 0x2
LFA_HALF_OUTPUT = 0x4
LFA_PLAIN = 0x8
LFA_FFT_ROUTE = 0x10
LFA_REPRODUCIBLE = 0x20
LFA_VARIANT_LOGGED = 0x10000   # options.variant flag: values variant + rotation log + W replay
LFA_VARIANT_BLOCKED = 0x20000  # options.variant value: blocked Jacobi on the tensor cores

# spectral editing modes
LFA_EDIT_CLIP = 0
LFA_EDIT_CLAMP = 1
LFA_EDIT_THRESHOLD = 2
LFA_EDIT_RANK = 3
LFA_EDIT_PINV = 4

# status codes
LFA_OK = 0
LFA_ERR_INVALID_ARG = 1
LFA_ERR_UNSUPPORTED = 2
LFA_ERR_OOM = 3
LFA_ERR_CUDA = 4
LFA_ERR_NOT_CONVERGED = 5
LFA_ERR_NONFINITE = 6
LFA_ERR_TIMEOUT = 7

# every symbol include/lfa.h and include/lfa_debug.h declare
EXPORTS = [
    "lfa_plan", "lfa_svd", "lfa_symbols", "lfa_fft_symbols", "lfa_expand", "lfa_svd_backward", "lfa_svd_backward_noalloc",
    "lfa_regulariser_grad", "lfa_spectral_edit",
    "lfa_destroy", "lfa_get_info", "lfa_layer_query", "lfa_status_string", "lfa_variant_name",
    "lfa_last_cuda_error", "lfa_kernel_launches", "lfa_version",
    "lfa_debug_schedule", "lfa_debug_half_grid", "lfa_debug_choose_variant", "lfa_debug_variant_count",
    "lfa_debug_tuned_variant", "lfa_debug_variant_fits", "lfa_debug_logged_ok", "lfa_debug_half_position",
    "lfa_debug_shard_range", "lfa_debug_tc_gram", "lfa_debug_tc_update", "lfa_debug_bj_profile",
    "lfa_debug_set_bj_ctas_per_sm", "lfa_debug_set_bj_grid", "lfa_debug_bj_occupancy", "lfa_debug_backward_route",
]


class LayerDesc(ctypes.Structure):
    _fields_ = [("c_out", c_int32), ("c_in", c_int32), ("kh", c_int32), ("kw", c_int32),
                ("n", c_int32), ("m", c_int32), ("pad_h", c_int32), ("pad_w", c_int32),
                ("stride_h", c_int32), ("stride_w", c_int32)]


def layer_desc(d) -> "LayerDesc":
    """LayerDesc from a LayerDesc or (c_out, c_in, kh, kw, n, m[, pad_h, pad_w[, stride_h, stride_w]])."""
    if isinstance(d, LayerDesc):
        return d
    d = tuple(int(x) for x in d)
    if len(d) not in (6, 8, 10):
        raise ValueError(f"layer description needs 6, 8 or 10 integers, got {len(d)}")
    d = d + (-1, -1, 1, 1)[len(d) - 6:]
    return LayerDesc(*d)


class Options(ctypes.Structure):
    _fields_ = [("tol", c_float), ("max_sweeps", c_int32), ("variant", c_int32),
                ("use_graph", c_int32), ("tune_cache", c_char_p), ("shard_rank", c_int32),
                ("shard_count", c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("symbols", c_int64), ("singular_values", c_int64), ("unconverged", c_int64),
                ("nonfinite", c_int64), ("sweeps", c_int64), ("rotations", c_int64),
                ("plan_device_bytes", c_int64), ("nlayers", c_int32), ("max_sweeps", c_int32),
                ("tol", c_float), ("tc_grams", c_int64), ("tc_updates", c_int64), ("debug_error", c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LfaError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().lfa_status_string(status).decode()
        if status == LFA_ERR_CUDA:
            msg += f" (cudaError {lib().lfa_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [status {status}]")


_LIB = None


def lib():
    """The loaded ``liblfa.so`` (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"the LFA CUDA library is not built ({LIB_PATH} missing); "
                           "run `python -m paper_2506_05617_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    PP = POINTER(c_void_p)
    sig = {
        "lfa_plan": (c_int32, [POINTER(c_void_p), POINTER(LayerDesc), c_int32, c_uint32, POINTER(Options)]),
        "lfa_svd": (c_int32, [P, PP, PP, PP, PP, P]),
        "lfa_symbols": (c_int32, [P, c_int32, P, P, P]),
        "lfa_fft_symbols": (c_int32, [P, c_int32, P, P, P]),
        "lfa_expand": (c_int32, [P, c_int32, P, P, c_int64, c_int64, P, P, P]),
        "lfa_svd_backward": (c_int32, [P, PP, PP, PP, PP, P]),
        "lfa_svd_backward_noalloc": (c_int32, [POINTER(LayerDesc), c_uint32, P, P, P, P, P]),
        "lfa_regulariser_grad": (c_int32, [P, PP, c_float, PP, PP, P]),
        "lfa_spectral_edit": (c_int32, [P, PP, PP, PP, c_int32, c_float, c_float, PP, P]),
        "lfa_destroy": (c_int32, [P]),
        "lfa_get_info": (c_int32, [P, POINTER(Info)]),
        "lfa_layer_query": (c_int32, [P, c_int32, POINTER(c_int64), POINTER(c_int32), POINTER(c_int32),
                                      POINTER(c_int32)]),
        "lfa_status_string": (c_char_p, [c_int32]),
        "lfa_variant_name": (c_char_p, [c_int32]),
        "lfa_last_cuda_error": (c_int32, []),
        "lfa_version": (c_int32, []),
        "lfa_kernel_launches": (c_int64, []),
        "lfa_debug_schedule": (c_int32, [c_int32, POINTER(c_uint16), c_int64]),
        "lfa_debug_half_grid": (c_int64, [c_int32, c_int32, POINTER(c_int32), c_int64]),
        "lfa_debug_choose_variant": (c_int32, [c_int32, c_int32, c_int32]),
        "lfa_debug_variant_count": (c_int32, []),
        "lfa_debug_tuned_variant": (c_int32, [c_char_p, c_int32, c_int32, c_int32]),
        "lfa_debug_variant_fits": (c_int32, [c_int32, c_int32, c_int32, c_int32]),
        "lfa_debug_logged_ok": (c_int32, [c_int32, c_int32, c_int32]),
        "lfa_debug_half_position": (c_int64, [c_int32, c_int32, c_int32]),
        "lfa_debug_shard_range": (c_int64, [c_int32, c_int32, c_int32, c_int32, POINTER(c_int64), POINTER(c_int64)]),
        "lfa_debug_tc_gram": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
        "lfa_debug_tc_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                          c_void_p, c_void_p]),
        "lfa_debug_bj_profile": (c_int32, [P, POINTER(ctypes.c_uint64), POINTER(c_int32)]),
        "lfa_debug_set_bj_ctas_per_sm": (None, [c_int32]),
        "lfa_debug_set_bj_grid": (None, [c_int32, c_int32]),
        "lfa_debug_bj_occupancy": (c_int32, [c_int32, POINTER(c_int32)]),
        "lfa_debug_backward_route": (c_int32, [c_int32] * 6),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _check(status: int, where: str):
    if status != LFA_OK:
        raise LfaError(status, where)


def _ptrs(values: Optional[Sequence[int]], n: int):
    if values is None:
        return None
    arr = (c_void_p * n)()
    for i, v in enumerate(values):
        arr[i] = c_void_p(int(v)) if v else None
    return ctypes.cast(arr, POINTER(c_void_p))


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    return int(getattr(s, "cuda_stream", s)) or None


# ----------------------------------------------------------------------------- entry points
def lfa_plan(layers: Iterable, flags: int = LFA_VALUES, tol: float = 0.0, max_sweeps: int = 0,
             variant: int = -1, use_graph: int = -1, tune_cache: Optional[str] = None,
             shard_rank: int = 0, shard_count: int = 1) -> int:
    """Creates a plan; ``layers`` holds LayerDesc or
    (c_out, c_in, kh, kw, n, m[, pad_h, pad_w[, stride_h, stride_w]])."""
    descs = [layer_desc(d) for d in layers]
    arr = (LayerDesc * max(1, len(descs)))(*descs)
    opt = Options(float(tol), int(max_sweeps), int(variant), int(use_graph),
                  tune_cache.encode() if tune_cache else None, int(shard_rank), int(shard_count))
    h = c_void_p()
    _check(lib().lfa_plan(ctypes.byref(h), arr, len(descs), int(flags), ctypes.byref(opt)), "lfa_plan")
    return int(h.value)


def lfa_svd(plan: int, w: Sequence[int], sigma: Sequence[int], U: Optional[Sequence[int]] = None,
            V: Optional[Sequence[int]] = None, stream=None) -> None:
    n = len(w)
    _check(lib().lfa_svd(c_void_p(plan), _ptrs(w, n), _ptrs(sigma, n), _ptrs(U, n), _ptrs(V, n),
                         _stream(stream)), "lfa_svd")


def lfa_symbols(plan: int, layer: int, w: int, out: int, stream=None) -> None:
    _check(lib().lfa_symbols(c_void_p(plan), layer, c_void_p(w), c_void_p(out), _stream(stream)), "lfa_symbols")


def lfa_fft_symbols(plan: int, layer: int, w: int, out: int, stream=None) -> None:
    _check(lib().lfa_fft_symbols(c_void_p(plan), layer, c_void_p(w), c_void_p(out), _stream(stream)),
           "lfa_fft_symbols")


def lfa_expand(plan: int, layer: int, U: int, V: int, first: int, count: int, u_hat: int, v_hat: int,
               stream=None) -> None:
    _check(lib().lfa_expand(c_void_p(plan), layer, c_void_p(U or None), c_void_p(V or None), first, count,
                            c_void_p(u_hat or None), c_void_p(v_hat or None), _stream(stream)), "lfa_expand")


def lfa_svd_backward(plan: int, dsigma: Sequence[int], U: Sequence[int], V: Sequence[int], dw: Sequence[int],
                     stream=None) -> None:
    n = len(dw)
    _check(lib().lfa_svd_backward(c_void_p(plan), _ptrs(dsigma, n), _ptrs(U, n), _ptrs(V, n), _ptrs(dw, n),
                                  _stream(stream)), "lfa_svd_backward")


def lfa_svd_backward_noalloc(layer, flags: int, dsigma: int, U: int, V: int, dw: int, stream=None) -> None:
    """Backward of one layer without any device allocation (no plan); see include/lfa.h."""
    desc = layer_desc(layer)
    _check(lib().lfa_svd_backward_noalloc(ctypes.byref(desc), int(flags), c_void_p(dsigma), c_void_p(U),
                                          c_void_p(V), c_void_p(dw), _stream(stream)), "lfa_svd_backward_noalloc")


def lfa_regulariser_grad(plan: int, sigma: Sequence[int], lam: float, dsigma: Sequence[int],
                         loss: Optional[Sequence[int]] = None, stream=None) -> None:
    n = len(sigma)
    _check(lib().lfa_regulariser_grad(c_void_p(plan), _ptrs(sigma, n), float(lam), _ptrs(dsigma, n),
                                      _ptrs(loss, n), _stream(stream)), "lfa_regulariser_grad")


def lfa_spectral_edit(plan: int, sigma: Sequence[int], U: Sequence[int], V: Sequence[int], mode: int, a: float,
                      b: float, w_out: Sequence[int], stream=None) -> None:
    n = len(sigma)
    _check(lib().lfa_spectral_edit(c_void_p(plan), _ptrs(sigma, n), _ptrs(U, n), _ptrs(V, n), int(mode), float(a),
                                   float(b), _ptrs(w_out, n), _stream(stream)), "lfa_spectral_edit")


def lfa_destroy(plan: int) -> None:
    _check(lib().lfa_destroy(c_void_p(plan)), "lfa_destroy")


def lfa_get_info(plan: int):
    """Returns (status, info dict); status is LFA_OK, LFA_ERR_NOT_CONVERGED, LFA_ERR_NONFINITE or
    LFA_ERR_TIMEOUT."""
    info = Info()
    st = lib().lfa_get_info(c_void_p(plan), ctypes.byref(info))
    if st not in (LFA_OK, LFA_ERR_NOT_CONVERGED, LFA_ERR_NONFINITE, LFA_ERR_TIMEOUT):
        raise LfaError(st, "lfa_get_info")
    return st, info.as_dict()


def lfa_layer_query(plan: int, layer: int, with_half_grid: bool = False):
    F_h = c_int64()
    r = c_int32()
    v = c_int32()
    _check(lib().lfa_layer_query(c_void_p(plan), layer, ctypes.byref(F_h), ctypes.byref(r), ctypes.byref(v),
                                 None), "lfa_layer_query")
    half = None
    if with_half_grid:
        buf = (c_int32 * F_h.value)()
        _check(lib().lfa_layer_query(c_void_p(plan), layer, None, None, None, buf), "lfa_layer_query")
        half = list(buf)
    return {"F_h": F_h.value, "r": r.value, "variant": v.value,
            "variant_name": lfa_variant_name(v.value), "half_grid": half}


def lfa_status_string(status: int) -> str:
    return lib().lfa_status_string(status).decode()


def lfa_variant_name(variant: int) -> str:
    return lib().lfa_variant_name(variant).decode()


def lfa_last_cuda_error() -> int:
    return lib().lfa_last_cuda_error()


def lfa_kernel_launches() -> int:
    return lib().lfa_kernel_launches()


def lfa_version() -> int:
    return lib().lfa_version()


def lfa_debug_schedule(ncols: int) -> List[List[tuple]]:
    rounds = ncols - 1
    buf = (c_uint16 * (rounds * ncols))()
    got = lib().lfa_debug_schedule(ncols, buf, len(buf))
    if got < 0:
        raise ValueError(f"lfa_debug_schedule({ncols}) failed: {got}")
    np_ = ncols // 2
    return [[(buf[(t * np_ + k) * 2], buf[(t * np_ + k) * 2 + 1]) for k in range(np_)] for t in range(got)]


def lfa_debug_half_grid(n: int, m: int) -> List[int]:
    cnt = lib().lfa_debug_half_grid(n, m, None, 0)
    if cnt < 0:
        raise ValueError("invalid torus")
    buf = (c_int32 * cnt)()
    lib().lfa_debug_half_grid(n, m, buf, cnt)
    return list(buf)


def lfa_debug_choose_variant(M: int, N: int, vectors: bool) -> int:
    return lib().lfa_debug_choose_variant(M, N, int(bool(vectors)))


def lfa_debug_variant_count() -> int:
    return lib().lfa_debug_variant_count()


def lfa_debug_tuned_variant(path: str, M: int, N: int, vectors: bool) -> int:
    return lib().lfa_debug_tuned_variant(path.encode(), M, N, int(vectors))


def lfa_debug_variant_fits(v: int, M: int, N: int, vectors: bool) -> bool:
    return bool(lib().lfa_debug_variant_fits(v, M, N, int(bool(vectors))))


def lfa_debug_logged_ok(v: int, M: int, N: int) -> bool:
    return bool(lib().lfa_debug_logged_ok(v, M, N))


def lfa_debug_half_position(n: int, m: int, f: int) -> int:
    return lib().lfa_debug_half_position(n, m, f)


def lfa_debug_shard_range(n: int, m: int, rank: int, count: int):
    """(F_h, first, count) of shard ``rank`` of ``count`` on an n x m torus; F_h = -1 on invalid input."""
    a, c = c_int64(0), c_int64(0)
    F_h = lib().lfa_debug_shard_range(n, m, rank, count, ctypes.byref(a), ctypes.byref(c))
    return int(F_h), int(a.value), int(c.value)


def lfa_debug_tc_gram(Xr: int, Xi: int, ld: int, Mp: int, cols: int, D: int, stream=None) -> int:
    """Tensor-core Gram of one block pair (see include/lfa_debug.h); returns the status code."""
    return int(lib().lfa_debug_tc_gram(c_void_p(Xr), c_void_p(Xi), ld, Mp, c_void_p(cols), c_void_p(D),
                                       _stream(stream)))


def lfa_debug_tc_update(Pr: int, Pi: int, Or: int, Oi: int, ld: int, rows: int, cols: int, Q: int,
                        stream=None) -> int:
    """Tensor-core update Y Q of one block pair (see include/lfa_debug.h); returns the status code."""
    return int(lib().lfa_debug_tc_update(c_void_p(Pr), c_void_p(Pi), c_void_p(Or), c_void_p(Oi), ld, rows,
                                         c_void_p(cols), c_void_p(Q), _stream(stream)))


BJ_PHASES = ("gram", "inner", "update", "assembly", "output", "symbol")


def lfa_debug_bj_profile(plan: int):
    """Phase clock cycles of the blocked route in the plan's last forward (summed over its CTAs),
    plus "warm_starts" (symbols started from their predecessor's V), and the CTA count of its
    launch: (dict, ctas)."""
    out = (ctypes.c_uint64 * 7)()
    ctas = c_int32(0)
    st = lib().lfa_debug_bj_profile(c_void_p(plan), out, ctypes.byref(ctas))
    if st != LFA_OK:
        raise LfaError(st, "lfa_debug_bj_profile")
    return {k: int(v) for k, v in zip(BJ_PHASES + ("warm_starts",), out)}, int(ctas.value)


def lfa_debug_set_bj_ctas_per_sm(n: int) -> None:
    """CTAs per SM of the blocked route in plans created afterwards (0: the kernel's choice)."""
    lib().lfa_debug_set_bj_ctas_per_sm(int(n))


def lfa_debug_set_bj_grid(max_ctas: int, runs: int) -> None:
    """Blocked route in plans created afterwards: at most max_ctas CTAs (<= 0: the kernel's count)
    and `runs` warm-start runs per layer (0: two per CTA, < 0: no warm starts)."""
    lib().lfa_debug_set_bj_grid(int(max_ctas), int(runs))


def lfa_debug_bj_occupancy(vectors: bool):
    """(CTAs per SM, registers per thread, static shared bytes, dynamic shared bytes, CTAs per SM with
    32 KB of dynamic shared memory) of the blocked route's kernel."""
    out = (c_int32 * 5)()
    st = lib().lfa_debug_bj_occupancy(1 if vectors else 0, out)
    if st != LFA_OK:
        raise LfaError(st, "lfa_debug_bj_occupancy")
    return tuple(int(v) for v in out)


BACKWARD_ROUTES = {2: "tensor-core", 1: "fused", 0: "cuda-core"}


def lfa_debug_backward_route(c_out: int, c_in: int, kh: int, kw: int, stride_h: int = 1, stride_w: int = 1) -> int:
    """The backward route of a layer: 2 tensor-core G product, 1 fused CUDA-core, 0 CUDA-core G + taps."""
    return int(lib().lfa_debug_backward_route(c_out, c_in, kh, kw, stride_h, stride_w))
