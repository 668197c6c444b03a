"""Host-side checks of the CUDA library that need no GPU: it builds, loads, exports every
symbol the headers declare, and its plan-time logic (Jacobi schedule, half grid, variant
choice, argument validation) is right."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2506_05617_gb300 import build as B
from paper_2506_05617_gb300 import lfa as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(lfa_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = C.lib()
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(C.EXPORTS)


@pytest.mark.parametrize("ncols", [4, 8, 16, 32, 64, 128, 256, 512])
def test_schedule_covers_every_pair_once_and_keeps_one_column(ncols):
    rounds = C.lfa_debug_schedule(ncols)
    assert len(rounds) == ncols - 1
    seen = set()
    for t, rnd in enumerate(rounds):
        cols = [c for p in rnd for c in p]
        assert sorted(cols) == list(range(ncols))          # a perfect matching
        for a, b in rnd:
            seen.add((min(a, b), max(a, b)))
        if t + 1 < len(rounds):
            for (a, b), (a2, b2) in zip(rnd, rounds[t + 1]):
                assert len({a, b} & {a2, b2}) == 1          # each team keeps exactly one column
    assert len(seen) == ncols * (ncols - 1) // 2


@pytest.mark.parametrize("n,m", [(1, 1), (1, 2), (2, 2), (3, 5), (8, 8), (7, 6), (224, 224), (32, 32)])
def test_half_grid_matches_oracle(n, m):
    assert C.lfa_debug_half_grid(n, m) == [int(f) for f in O.half_grid(n, m)]


def test_variant_choice():
    assert C.lfa_debug_variant_count() >= 9
    for M, N in [(4, 4), (64, 3), (64, 64), (32, 32), (16, 8), (64, 16), (1, 1), (128, 64), (128, 128),
                 (256, 128), (256, 256)]:
        for vec in (False, True):
            v = C.lfa_debug_choose_variant(M, N, vec)
            assert v >= 0, (M, N, vec)
            name = C.lfa_variant_name(v)
            npairs, lanes, mr, wr, cs, ppt = (int(x) for x in re.findall(r"\d+", name))
            assert M <= mr * lanes and N <= 2 * npairs
            assert ppt == 1          # the built-in choice keeps one team per thread
            if vec:
                assert N <= wr * lanes
    assert C.lfa_debug_choose_variant(513, 8, True) == -1
    assert C.lfa_debug_choose_variant(512, 512, True) == -1      # vectors at c = 512 need more registers
    assert C.lfa_debug_choose_variant(512, 512, False) >= 0
    assert C.lfa_variant_name(-1) == "none"


def test_status_strings_and_version():
    for s in range(8):
        assert C.lfa_status_string(s)
    assert C.lfa_status_string(99) == "unknown status"
    assert C.lfa_version() >= 100


@pytest.mark.parametrize("bad", [
    (0, 4, 3, 3, 8, 8), (4, 4, 0, 3, 8, 8), (4, 4, 3, 3, 0, 8), (4, 600, 3, 3, 8, 8),
    (4, 4, 3, 3, 8, 8, 3, 1), (4, 4, 16, 3, 8, 8), (4, 4, 3, 3, 8, 8, -2, 0),
    # strides: at most 8, not negative, and c_in * s_h * s_w symbol columns at most 512
    (4, 4, 3, 3, 8, 8, -1, -1, 9, 1), (4, 4, 3, 3, 8, 8, -1, -1, 2, -1), (4, 129, 3, 3, 8, 8, -1, -1, 2, 2),
])
def test_plan_rejects_invalid_layers_without_touching_the_gpu(bad):
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([bad], C.LFA_VALUES)
    assert ei.value.status == C.LFA_ERR_INVALID_ARG


def test_layer_descriptions_accept_6_8_or_10_integers():
    assert tuple(getattr(C.layer_desc((4, 5, 3, 3, 8, 9)), k) for k, _ in C.LayerDesc._fields_) == \
        (4, 5, 3, 3, 8, 9, -1, -1, 1, 1)
    assert C.layer_desc((4, 5, 3, 3, 8, 9, 0, 2)).pad_w == 2
    assert C.layer_desc((4, 5, 3, 3, 8, 9, -1, -1, 2, 3)).stride_w == 3
    with pytest.raises(ValueError):
        C.layer_desc((4, 5, 3, 3, 8, 9, 0))


def test_plan_rejects_bad_flags_and_counts():
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], 0x100)
    assert ei.value.status == C.LFA_ERR_INVALID_ARG
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], C.LFA_PLAIN | C.LFA_VECTORS)
    assert ei.value.status == C.LFA_ERR_INVALID_ARG
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([], C.LFA_VALUES)
    assert ei.value.status == C.LFA_ERR_INVALID_ARG


def test_header_constants_match_the_binding():
    """Every numeric LFA_* constant of lfa.h (flags, variants, edit modes, status codes, sizes) has
    the same value in the ctypes binding."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lfa.h")).read(), flags=re.S)
    defs = {}
    for name, val in re.findall(r"#define\s+(LFA_[A-Z0-9_]+)\s+\(?((?:0x[0-9a-fA-F]+|\d+)u?(?:\s*<<\s*\d+)?)\)?", txt):
        defs[name] = eval(val.replace("u", ""), {})
    for name, val in re.findall(r"\b(LFA_[A-Z0-9_]+)\s*=\s*(\d+)", txt):   # enumerators
        defs[name] = int(val)
    assert {"LFA_VECTORS", "LFA_REPRODUCIBLE", "LFA_VARIANT_BLOCKED", "LFA_ERR_TIMEOUT"} <= set(defs)
    for name, v in defs.items():
        if hasattr(C, name):
            assert getattr(C, name) == v, name
    missing = [n for n in defs if not hasattr(C, n) and not n.endswith("_H_")]
    assert all(n.startswith("LFA_NOALLOC") or n.startswith("LFA_VERSION") or n == "LFA_API" for n in missing), missing


def test_plan_flags_validation_accepts_reproducible():
    """LFA_REPRODUCIBLE is a valid plan flag: without a GPU the plan then fails only at the device."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], C.LFA_VALUES | C.LFA_VECTORS | C.LFA_REPRODUCIBLE)
    assert ei.value.status in (C.LFA_ERR_CUDA, C.LFA_ERR_UNSUPPORTED)
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], C.LFA_VALUES | 0x40)
    assert ei.value.status == C.LFA_ERR_INVALID_ARG


def test_null_plan_calls_are_rejected():
    L = C.lib()
    assert L.lfa_svd(None, None, None, None, None, None) == C.LFA_ERR_INVALID_ARG
    assert L.lfa_svd_backward(None, None, None, None, None, None) == C.LFA_ERR_INVALID_ARG
    assert L.lfa_destroy(None) == C.LFA_OK
    assert L.lfa_get_info(None, None) == C.LFA_ERR_INVALID_ARG


def test_fault_injection_alloc_is_reported(monkeypatch):
    monkeypatch.setenv("LFA_FAULT_INJECT", "alloc")
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], C.LFA_VALUES)
    assert ei.value.status == C.LFA_ERR_OOM


def test_plan_without_gpu_fails_with_a_status():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(C.LfaError) as ei:
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], C.LFA_VALUES)
    assert ei.value.status in (C.LFA_ERR_CUDA, C.LFA_ERR_UNSUPPORTED)


def test_tune_cache_parsing_and_rotation_log_routes(tmp_path):
    """The autotuner cache selects a variant (or the rotation-log route) per problem; lines that
    name a variant unable to hold the problem are ignored."""
    cache = tmp_path / "tune.txt"
    cache.write_text("# comment\n64 64 1 9  # in registers\n128 128 1 12 log  # rotation log\n"
                     "128 128 0 12\n32 32 1 16\n512 512 1 16 log\n")
    LOG = C.LFA_VARIANT_LOGGED
    assert C.lfa_debug_tuned_variant(str(cache), 64, 64, True) == 9
    assert C.lfa_debug_tuned_variant(str(cache), 128, 128, True) == 12 | LOG
    assert C.lfa_debug_tuned_variant(str(cache), 128, 128, False) == 12
    assert C.lfa_debug_tuned_variant(str(cache), 32, 32, True) == -1       # 16 holds no vectors
    assert C.lfa_debug_tuned_variant(str(cache), 512, 512, True) == 16 | LOG
    assert C.lfa_debug_tuned_variant(str(cache), 100, 100, True) == -1
    assert C.lfa_debug_tuned_variant(str(tmp_path / "missing.txt"), 64, 64, True) == -1
    # the blocked tensor-core route by keyword, for the sizes it serves
    blk = tmp_path / "blk.txt"
    blk.write_text("512 512 1 0 blocked\n600 64 1 0 blocked\n256 256 0 0 blocked\n")
    assert C.lfa_debug_tuned_variant(str(blk), 512, 512, True) == C.LFA_VARIANT_BLOCKED
    assert C.lfa_debug_tuned_variant(str(blk), 256, 256, False) == C.LFA_VARIANT_BLOCKED
    assert C.lfa_debug_tuned_variant(str(blk), 600, 64, True) == -1          # more than 512 rows
    assert C.lfa_variant_name(C.LFA_VARIANT_BLOCKED) == "blocked_tc_b32"
    assert C.lfa_variant_name(12 | LOG).endswith("_log")
    # the route exists exactly where a replay configuration serves the variant's pairs
    for v in range(C.lfa_debug_variant_count()):
        npairs, lanes, mr, wr, cs, ppt = (int(x) for x in re.findall(r"\d+", C.lfa_variant_name(v)))
        expect = ppt == 1 and npairs in (16, 32, 64, 128, 256) and npairs * lanes // cs >= 32
        M, N = min(mr * lanes, 512), min(2 * npairs, 512)
        assert C.lfa_debug_logged_ok(v, M, N) == expect, C.lfa_variant_name(v)


def test_committed_tune_cache_parses_for_every_entry():
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2506_05617_gb300", "tune_gb300.txt")
    for line in open(path):
        parts = line.split("#")[0].split()
        if not parts:
            continue
        M, N, vec = (int(x) for x in parts[:3])
        got = C.lfa_debug_tuned_variant(path, M, N, bool(vec))
        assert got >= 0, line
        word = parts[4] if len(parts) == 5 else ""
        if word == "blocked":
            assert got == C.LFA_VARIANT_BLOCKED, line
        else:
            assert (got & C.LFA_VARIANT_LOGGED) == (C.LFA_VARIANT_LOGGED if word == "log" else 0), line


@pytest.mark.parametrize("n,m", [(1, 1), (1, 7), (6, 1), (2, 2), (3, 3), (4, 5), (5, 4), (8, 8), (7, 9), (32, 32), (9, 16)])
def test_half_position_closed_form_matches_the_list(n, m):
    """The lifting kernel's closed-form position of a frequency's representative in the half grid,
    against the oracle's half-grid list and conjugation rule, for every frequency."""
    half = list(O.half_grid(n, m))
    pos = {f: i for i, f in enumerate(half)}
    for f in range(n * m):
        j, l = divmod(f, m)
        fc = ((-j) % n) * m + (-l) % m
        rep = f if f in pos else fc
        assert C.lfa_debug_half_position(n, m, f) == pos[rep], (n, m, f)
    assert C.lfa_debug_half_position(n, m, n * m) == -1


def test_every_variant_shared_memory_layout_fits(tmp_path):
    """tests/layout_check.cu, compiled for the host, walks every Jacobi variant (values, and
    values+vectors where built): the unit tail holds the four control words and one float per warp,
    a CTA stays within 227 KB, and neighbouring teams' mailbox slots are 2 L mod 16 float2 apart."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "layout_check")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    os.path.join(ROOT, "tests", "layout_check.cu")], check=True, capture_output=True, timeout=300)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    lines = res.stdout.strip().splitlines()
    assert res.returncode == 0, res.stdout
    assert all(ln.endswith(" ok") for ln in lines)
    ids = {int(ln.split()[0]) for ln in lines}
    assert ids == set(range(C.lfa_debug_variant_count()))
    smem = [int(re.search(r"smem=(\d+)", ln).group(1)) for ln in lines]
    assert max(smem) <= 227 * 1024


AUTOTUNE_SHAPES = [(4, 4), (9, 3), (33, 17), (64, 12), (64, 64), (100, 77), (128, 128), (200, 200),
                   (256, 128), (256, 256), (400, 400), (512, 256), (512, 512)]


def test_autotuner_candidates_are_exactly_what_a_cache_line_can_select(tmp_path):
    """Every route the autotuner times is one that a cache line can select for that problem, and
    every route a cache line can select is timed (register variants, rotation-log routes and the
    blocked tensor-core route)."""
    from paper_2506_05617_gb300 import autotune as A
    cache = str(tmp_path / "tune.txt")
    nv = C.lfa_debug_variant_count()
    for M, N in AUTOTUNE_SHAPES:
        for vec in (False, True):
            accepted = set()
            routes = [("0 blocked", C.LFA_VARIANT_BLOCKED)]
            for v in range(nv):
                routes += [(f"{v}", v), (f"{v} log", v | C.LFA_VARIANT_LOGGED)]
            for route, want in routes:
                if route.endswith("log") and not vec:
                    continue
                with open(cache, "w") as fh:
                    fh.write(f"{M} {N} {int(vec)} {route}\n")
                if C.lfa_debug_tuned_variant(cache, M, N, vec) == want:
                    accepted.add(want)
            cands = A.candidates(M, N, vec)
            assert len(cands) == len(set(cands))
            assert set(cands) == accepted, (M, N, vec, sorted(set(cands) ^ accepted))
            assert cands, (M, N, vec)
            # the built-in choice is among them; with vectors and no register variant that holds
            # W, the plan runs the values-mode choice through the rotation log
            bi = C.lfa_debug_choose_variant(M, N, vec)
            if bi < 0:
                assert vec
                bi = C.lfa_debug_choose_variant(M, N, False) | C.LFA_VARIANT_LOGGED
            assert bi in cands


def test_autotuner_cache_round_trips_through_the_library(tmp_path):
    from paper_2506_05617_gb300 import autotune as A
    cache = str(tmp_path / "tune.txt")
    with open(cache, "w") as fh:
        fh.write("# an older cache\n64 64 1 9  # kept\n100 77 0 7\n")
    logged = [v for v in A.candidates(128, 128, True) if v & C.LFA_VARIANT_LOGGED][0]
    A.write_cache(cache, {(128, 128, 1): (logged, 1.5), (100, 77, 0): (A.candidates(100, 77, False)[-1], 0.2)})
    assert C.lfa_debug_tuned_variant(cache, 128, 128, True) == logged
    assert C.lfa_debug_tuned_variant(cache, 100, 77, False) == A.candidates(100, 77, False)[-1]
    assert C.lfa_debug_tuned_variant(cache, 64, 64, True) == 9          # untouched line kept
    lines = [ln for ln in open(cache) if not ln.startswith("#")]
    assert len(lines) == 3 and lines == sorted(lines, key=lambda ln: tuple(int(x) for x in ln.split()[:3]))


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built CUDA library every call raises: there is no CPU or other fallback."""
    monkeypatch.setattr(C, "_LIB", None)
    monkeypatch.setattr(C, "LIB_PATH", str(tmp_path / "liblfa.so"))
    with pytest.raises(RuntimeError, match="not built"):
        C.lib()
    with pytest.raises(RuntimeError, match="not built"):
        C.lfa_plan([(4, 4, 3, 3, 8, 8)], C.LFA_VALUES)
    from paper_2506_05617_gb300.torch_api import LfaPlan
    with pytest.raises(RuntimeError, match="not built"):
        LfaPlan([(4, 4, 3, 3, 8, 8)])


def test_backward_route_choice():
    """Stride-1 layers with 128 channels and more on both sides and at most 25 taps take the
    tensor-core backward; other stride-1 layers with at most 25 taps the fused CUDA-core kernel; the
    rest the CUDA-core G product and tap projection."""
    assert C.lfa_debug_backward_route(512, 512, 3, 3) == 2
    assert C.lfa_debug_backward_route(128, 128, 5, 5) == 2
    assert C.lfa_debug_backward_route(130, 140, 1, 1) == 2
    assert C.lfa_debug_backward_route(128, 96, 3, 3) == 1
    assert C.lfa_debug_backward_route(64, 64, 3, 3) == 1
    assert C.lfa_debug_backward_route(256, 256, 7, 7) == 0
    assert C.lfa_debug_backward_route(256, 128, 3, 3, 2, 2) == 0
    assert C.lfa_debug_backward_route(0, 128, 3, 3) == -1
