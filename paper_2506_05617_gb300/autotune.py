"""Autotuner for the Jacobi kernel variants.

For every distinct Jacobi problem (M = max(c_out, c_in), N = min(c_out, c_in), with or
without vectors) of the given layers, each register-resident variant that can hold it is
timed through the C ABI (`lfa_svd` on a one-layer plan forced to that variant, CUDA
events around graph replays), and the fastest is written to a text cache, one line per
problem: ``M N vectors variant  # name ms``. `lfa_plan` reads that file when it is passed
as `lfa_options.tune_cache`; problems without a line use the built-in choice.

    python -m paper_2506_05617_gb300.autotune --workload conv64_k3_n32 --out tune.txt
"""
from __future__ import annotations

import argparse
import os
import sys
from typing import Dict, Iterable, List, Tuple

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def candidates(M: int, N: int, vectors: bool) -> List[int]:
    """Variant ids that can hold an M x N problem, by the library's own rules: register-resident
    variants (with W when vectors), with vectors also the values-mode variants that can run the
    rotation log and the W replay (flagged LFA_VARIANT_LOGGED), and for 128 to 512 columns the
    blocked tensor-core route (LFA_VARIANT_BLOCKED)."""
    from . import lfa as C
    out = []
    for v in range(C.lfa_debug_variant_count()):
        if C.lfa_debug_variant_fits(v, M, N, vectors):
            out.append(v)
        if vectors and C.lfa_debug_logged_ok(v, M, N):
            out.append(v | C.LFA_VARIANT_LOGGED)
    if M <= 512 and 128 <= N <= 512:
        out.append(C.LFA_VARIANT_BLOCKED)   # the blocked tensor-core route
    return out


def time_variant(layer: Tuple[int, ...], vectors: bool, variant: int, reps: int = 5) -> float:
    """Median milliseconds of lfa_svd for one layer forced to `variant` (inf if it cannot run)."""
    import numpy as np
    import torch
    from . import lfa as C
    from .torch_api import LfaPlan
    try:
        plan = LfaPlan([layer], vectors=vectors, variant=variant)
    except C.LfaError:
        return float("inf")
    if plan.meta[0]["variant"] != variant:
        plan.close()
        return float("inf")
    c_out, c_in, kh, kw = layer[:4]
    w = torch.randn(c_out, c_in, kh, kw, device="cuda") / (c_in * kh * kw) ** 0.5
    out = plan.alloc()
    for _ in range(2):
        plan.svd([w], out=out)
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        plan.svd([w], out=out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    st, info = plan.info()
    plan.close()
    if st != C.LFA_OK:
        return float("inf")
    return float(np.median(ts))


def tune(layers: Iterable[Tuple[int, ...]], vectors: bool, verbose: bool = True) -> Dict[Tuple[int, int, int], Tuple[int, float]]:
    from . import lfa as C
    best: Dict[Tuple[int, int, int], Tuple[int, float]] = {}
    for layer in layers:
        c_out = layer[0]
        cols = layer[1] * (layer[8] if len(layer) > 8 else 1) * (layer[9] if len(layer) > 9 else 1)
        key = (max(c_out, cols), min(c_out, cols), int(vectors))   # the symbol's shape
        if key in best:
            continue
        res = []
        for v in candidates(key[0], key[1], vectors):
            ms = time_variant(tuple(layer), vectors, v)
            res.append((ms, v))
            if verbose:
                print(f"  M={key[0]} N={key[1]} vec={int(vectors)} {C.lfa_variant_name(v):32s} {ms:9.3f} ms",
                      file=sys.stderr)
        res.sort()
        if res and res[0][0] < float("inf"):
            best[key] = (res[0][1], res[0][0])
    return best


def write_cache(path: str, best: Dict[Tuple[int, int, int], Tuple[int, float]]):
    from . import lfa as C
    old = {}
    if os.path.exists(path):
        for line in open(path):
            parts = line.split("#")[0].split()
            if len(parts) in (4, 5):
                old[tuple(int(x) for x in parts[:3])] = line.rstrip("\n")
    for (M, N, vec), (v, ms) in best.items():
        if v == C.LFA_VARIANT_BLOCKED:
            route = "0 blocked"
        elif v & C.LFA_VARIANT_LOGGED:
            route = f"{v & (C.LFA_VARIANT_LOGGED - 1)} log"
        else:
            route = f"{v}"
        old[(M, N, vec)] = f"{M} {N} {vec} {route}  # {C.lfa_variant_name(v)} {ms:.3f} ms"
    with open(path, "w") as fh:
        fh.write("# LFA Jacobi variant cache: M N vectors variant  (written by paper_2506_05617_gb300.autotune)\n")
        for k in sorted(old):
            fh.write(old[k] + "\n")


def main():
    sys.path.insert(0, ROOT)
    import lfa_workloads as W
    from . import build as B
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", action="append", default=None, choices=sorted(W.WORKLOADS))
    ap.add_argument("--out", required=True)
    ap.add_argument("--values", action="store_true", help="tune the values-only kernels too")
    a = ap.parse_args()
    B.build()
    names = a.workload or ["conv64_k3_n32"]
    layers = []
    for nm in names:
        layers += [l.desc() for l in W.layers(nm)]
    best = tune(layers, vectors=True)
    if a.values:
        best.update(tune(layers, vectors=False))
    write_cache(a.out, best)
    print(open(a.out).read())


if __name__ == "__main__":
    main()
