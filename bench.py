#!/usr/bin/env python
"""Benchmark of the LFA SVD hot path on GB300 (one JSON line on stdout, rank 0).

A step is one pass of the whole path over one synthetic layer batch:
  forward (symbol assembly fused with the batched one-sided Jacobi SVD, values and
  vectors, one persistent graph-replayed launch) -> spectral-regulariser dL/dsigma
  -> backward dL/dw -> lifting of the r global singular vector pairs of one frequency.
Metric: singular values per second (full-grid count n*m*r per layer per step).

Default workload: the largest configuration, one 512->512 3x3 stride-1 periodic conv on a
64x64 torus (4096 frequencies, 2050 decomposed on the half grid), values + vectors. Other
workloads (--workload): conv64_k3_n32, resnet18_body, reg4_c128_n32, stem3to64_k7_n224, ...

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]

With torchrun (N > 1) every rank runs the same per-GPU workload on its own seeded
weights (independent layers: weak scaling, no collective on the data path); the
step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lfa_workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
DEFAULT_TUNE = os.path.join(ROOT, "paper_2506_05617_gb300", "tune_gb300.txt")
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
LAM = 1e-2
METRIC = "singular values/sec and layers/sec (batched+backward vs plain) at σ err ≤1e-5·σ_max"
# workloads whose configuration asks for singular values only
VALUES_ONLY = {"resnet18_body", "paper_c16_k3_n256"}


def nominal_svd_flops(M: int, N: int, vectors: bool) -> float:
    """Golub-Van Loan dense SVD operation counts (M >= N), x4 for complex arithmetic."""
    if vectors:
        return 4.0 * (14.0 * M * N * N + 8.0 * N ** 3)
    return 4.0 * (4.0 * M * N * N - 4.0 * N ** 3 / 3.0)


def layer_flops(l: W.Layer, vectors: bool) -> float:
    """Nominal flops of one forward over a layer: assembly + SVD per half-grid symbol."""
    M, N = max(l.c_out, l.cols), min(l.c_out, l.cols)
    F_h = (l.n * l.m + (1 + (l.n % 2 == 0)) * (1 + (l.m % 2 == 0))) // 2
    return F_h * (4.0 * l.c_out * l.c_in * l.kh * l.kw + nominal_svd_flops(M, N, vectors))


def executed_flops(layers, info, vectors: bool) -> float:
    """Flops the Jacobi kernel executed, from its device counters: every pair of every round forms
    three dot products over M complex rows (16 real flops per row), and every applied rotation
    updates two columns of X (M rows) and, with vectors, of W (N rows) at 24 flops per row.
    Per-layer sizes are averaged over symbols (exact for a single layer)."""
    syms = sum((l.F + (1 + (l.n % 2 == 0)) * (1 + (l.m % 2 == 0))) // 2 for l in layers)
    M = sum(max(l.c_out, l.cols) * l.F for l in layers) / max(1, sum(l.F for l in layers))
    N = sum(min(l.c_out, l.cols) * l.F for l in layers) / max(1, sum(l.F for l in layers))
    pairs_per_sweep = N * (N - 1) / 2 + (N / 2 if int(N) % 2 else 0)
    dots = info["sweeps"] * pairs_per_sweep * 16.0 * M
    rots = info["rotations"] * 24.0 * (M + (N if vectors else 0))
    return dots + rots


def kernel_sha16() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("jacobi.cuh", "jacobi_variants.cuh", "lfa_internal.cuh", "blocked.cu", "tc_ptx.cuh"):
        with open(os.path.join(ROOT, "paper_2506_05617_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, info=None):
    """DRAM bytes per launch of the Jacobi kernel from the committed ncu capture, or None when
    there is none for this workload or the kernel source changed since it was taken. A capture of
    the blocked route on a smaller case gives bytes per block-pair Gram (each Gram reads the pair's
    columns of X, each update rewrites them and W's): scaled by the launch's own Gram count."""
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(prof)).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sha16") != kernel_sha16():
        return None
    if "bytes_per_gram" in rec:
        return rec["bytes_per_gram"] * info["tc_grams"] if info else None
    return rec.get("bytes_per_launch")


def rank_seed(layer: W.Layer, rank: int) -> int:
    """Seed of a rank's weights: every rank decomposes its own independent layers (weak scaling)."""
    return layer.seed + 1000 * rank


def reduce_max(values, dist=None, device="cpu"):
    """Element-wise max over ranks (the identity without a process group)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def aggregate_rate(units_per_rank_step: float, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank_step * steps / (slowest_ms / 1e3)


def lift_bytes_per_pair(l: W.Layer) -> int:
    """Bytes the lifting kernel writes per vector pair: u_hat on the n x m torus (c_out channels)
    and v_hat on the input torus s_h n x s_w m (c_in channels), complex64."""
    return 8 * (l.c_out * l.n * l.m + l.c_in * l.sh * l.n * l.sw * l.m)


def lift_pairs(l: W.Layer, target_bytes: int = 512 << 20) -> int:
    """Vector pairs per timed lifting launch: enough to write about target_bytes (more than the
    L2 holds), at most every pair of the layer."""
    return int(min(l.F * l.r, max(1, -(-target_bytes // lift_bytes_per_pair(l)))))


def fp32_peak_tflops() -> float:
    return SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


# nominal dense tensor-core rates of GB300: TF32 1.1 and BF16 2.25 PFLOP/s
TF32_PER_BF16 = 1.1 / 2.25


def tf32_peak_tflops(peaks: dict):
    """TF32 tensor peak: the measured sustained cuBLAS BF16 rate (the kernel runs for seconds inside
    a step) times the nominal TF32 / BF16 ratio; the fallback figure when nothing was measured."""
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    if bf16:
        return float(bf16) * TF32_PER_BF16, "measured sustained bf16 x nominal TF32/BF16 ratio (1.1/2.25)"
    return 1700.0 * TF32_PER_BF16, "fallback sustained bf16 (1.7 PFLOP/s) x nominal TF32/BF16 ratio (1.1/2.25)"


def blocked_tensor_flops(l: W.Layer, grams: int, updates: int, vectors: bool) -> float:
    """Tensor-core flops the blocked route issued, from its device counters: a block-pair Gram is the
    real 128 x 128 product over Mp rows and an update the real product of every 128-row tile of X
    (and W) with the 128 x 128 real form of Q - I, each as three TF32 products."""
    M, N = max(l.c_out, l.cols), min(l.c_out, l.cols)
    Mp, Np = -(-M // 128) * 128, -(-N // 128) * 128
    per_row = 3 * 2 * 128 * 128
    return grams * per_row * Mp + updates * per_row * (Mp + (Np if vectors else 0))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle leg
def oracle_sample_step(w, lay: W.Layer, freqs, g_seed: int, vectors: bool = True):
    """One bounded sample of the step on the FP64 oracle (CPU): symbols + SVD (U, V) of the
    sampled frequencies, regulariser gradient, their dL/dw contribution, lifted vectors
    (values only: symbols + SVD values)."""
    import oracle as O
    st = (lay.sh, lay.sw) != (1, 1)
    if not vectors:
        return oracle_values(w, lay, freqs), None, None, None
    if st:
        s, U, V = O.lfa_svd_strided(w, lay.n, lay.m, lay.sh, lay.sw, lay.pad_h, lay.pad_w, freqs=freqs)
    else:
        s, U, V = O.lfa_svd(w, lay.n, lay.m, compute_uv=True, freqs=freqs)
    g = O.regulariser_grad_sigma(s, LAM)
    f0 = int(freqs[0])
    j, l = divmod(f0, lay.m)
    if st:
        dw = O.lfa_backward_strided(w, lay.n, lay.m, lay.sh, lay.sw, g, U, V, lay.pad_h, lay.pad_w, freqs=freqs)
        uh, vh = O.lift_strided(U[0], V[0], j, l, lay.n, lay.m, lay.sh, lay.sw)
    else:
        dw = O.lfa_backward(w, lay.n, lay.m, g, U, V, freqs=freqs)
        uh, vh = O.lift(U[0], V[0], j, l, lay.n, lay.m)
    return s, dw, uh, vh


def oracle_values(w, lay: W.Layer, freqs):
    """FP64 oracle singular values of the sampled frequencies (any stride)."""
    import oracle as O
    if (lay.sh, lay.sw) != (1, 1):
        return O.lfa_svd_strided(w, lay.n, lay.m, lay.sh, lay.sw, lay.pad_h, lay.pad_w, compute_uv=False,
                                 freqs=freqs)
    return O.lfa_svd(w, lay.n, lay.m, compute_uv=False, freqs=freqs)


def layer_name(l: W.Layer) -> str:
    return f"{l.c_out}x{l.c_in}x{l.kh}x{l.kw}@{l.n}x{l.m}" + (f"/s{l.sh}x{l.sw}" if (l.sh, l.sw) != (1, 1) else "")


def run_oracle(lay: W.Layer, seconds: float, nfreq: int, steps: int | None = None, vectors: bool = True):
    """Times the oracle on sampled frequencies of the workload; returns the cpu_baseline dict."""
    w = W.weights(lay)
    rng = np.random.default_rng(123)
    nf = min(nfreq, lay.F)
    done, sig = 0, 0
    t0 = time.perf_counter()
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    times = []
    while True:
        freqs = np.sort(rng.choice(lay.F, nf, replace=False))
        ts = time.perf_counter()
        oracle_sample_step(w, lay, freqs, 0, vectors)
        times.append(time.perf_counter() - ts)
        done += 1
        sig += nf * lay.r
        if steps is not None and done >= steps:
            break
        if steps is None and time.perf_counter() - t0 >= seconds:
            break
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return {"value": sig / wall, "unit": "singular values/s", "cores": round(cpu / wall, 2),
            "s_per_frequency": wall / (done * nf),
            "cores_available": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} x {nf} of {lay.F} frequencies of {lay.c_out}->{lay.c_in} k={lay.kh} n={lay.n}: "
                      + ("FP64 symbols + LAPACK SVD with U,V + regulariser grad + dL/dw + one lifted pair"
                         if vectors else "FP64 symbols + LAPACK SVD values"),
            "seconds": round(wall, 3), "step_s": times}


def run_oracle_one_core(workload: str, seconds: float, nfreq: int, vectors: bool):
    """The same oracle sample on one host core: a fresh interpreter whose BLAS/LAPACK and OpenMP
    pools are limited to one thread before numpy loads (a thread count cannot change afterwards).
    Returns the cpu_baseline-style dict, or a dict with "error"."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload", workload,
           "--cpu-seconds", str(seconds), "--cpu-freqs", str(nfreq)] + ([] if vectors else ["--values-only"])
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=max(120.0, 6 * seconds))
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": f"one-core oracle leg failed: {e}"}


def run_fft_route(lay: W.Layer, svd_s_per_freq: float, vectors: bool, budget_s: float = 5.0):
    """The paper's comparison route (Sec. II, Table II) on the host in FP64: numpy's fft2 of the
    zero-padded kernel gives every symbol at once, then one LAPACK SVD per frequency (full grid, no
    conjugate symmetry, as in the paper). The transform is timed on a block of output channels and
    scaled to the layer (its cost is proportional to the channel pairs); the per-frequency SVD time
    is the oracle leg's. Table III splits the paper's time the same way (s_F, s_SVD)."""
    import oracle as O
    rows = max(1, min(lay.c_out, int(2 ** 27 // (16 * lay.c_in * lay.n * lay.m))))   # <= 2 GiB complex
    sub = W.weights(lay)[:rows]
    t0 = time.perf_counter()
    reps = 0
    while True:
        O.fft_symbols(sub, lay.n, lay.m, lay.pad_h, lay.pad_w)
        reps += 1
        if time.perf_counter() - t0 >= budget_s or reps >= 20:
            break
    t_rows = (time.perf_counter() - t0) / reps
    t_fft = t_rows * lay.c_out / rows
    t_svd = svd_s_per_freq * lay.F
    return {"transform_s": t_fft, "svd_s": t_svd, "total_s": t_fft + t_svd,
            "value": lay.n_sigma / (t_fft + t_svd), "unit": "singular values/s",
            "sample": f"fft2 of {rows} of {lay.c_out} output channels timed ({reps} reps) and scaled; "
                      f"SVD time = {lay.F} full-grid frequencies x the oracle leg's time per frequency"
                      + (" (values and vectors)" if vectors else " (values)")}


# ----------------------------------------------------------------------------- GPU arm
def run_lfa(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_2506_05617_gb300 import build as B
    from paper_2506_05617_gb300 import lfa as C
    from paper_2506_05617_gb300.torch_api import LfaPlan

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # one process per node compiles (the others would race on the same build folder), then all load
    if local_rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    B.build()

    layers = W.layers(args.workload)
    vectors = not (args.values_only or args.workload in VALUES_ONLY)
    # each rank gets its own seeded weights (independent units)
    ws = [torch.from_numpy(W.weights(l, seed=rank_seed(l, rank))).to(dev) for l in layers]
    specs = [l.desc() for l in layers]
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    w_ptrs = [w.data_ptr() for w in ws]

    def make_step(plan):
        """Output buffers of one step and the calls that fill them: forward (lfa_svd) and the rest
        of the step (regulariser gradient, backward, lifting of r vector pairs of layer 0)."""
        sig, U, V = plan.alloc(dev)
        s_ptrs = [s.data_ptr() for s in sig]
        outs = list(sig)
        if not vectors:
            return outs, (lambda: C.lfa_svd(plan.handle, w_ptrs, s_ptrs, None, None, sptr)), (lambda: None)
        dsig = [torch.empty_like(s) for s in sig]
        loss = [torch.empty((), device=dev) for _ in sig]
        dw = [torch.empty_like(w) for w in ws]
        l0 = layers[0]
        f_exp = 1 if l0.F > 1 else 0
        cnt = min(l0.r, 64)                   # vector pairs of one frequency lifted per step
        uh = torch.empty((cnt, l0.c_out, l0.n, l0.m), dtype=torch.complex64, device=dev)
        vh = torch.empty((cnt, l0.c_in, l0.sh * l0.n, l0.sw * l0.m), dtype=torch.complex64, device=dev)
        u_ptrs = [u.data_ptr() for u in U]
        v_ptrs = [v.data_ptr() for v in V]
        ds_ptrs = [d.data_ptr() for d in dsig]
        lo_ptrs = [x.data_ptr() for x in loss]
        dw_ptrs = [d.data_ptr() for d in dw]
        outs += list(U) + list(V) + dsig + dw + loss + [uh, vh]

        def forward():
            C.lfa_svd(plan.handle, w_ptrs, s_ptrs, u_ptrs, v_ptrs, sptr)

        def rest():
            C.lfa_regulariser_grad(plan.handle, s_ptrs, LAM, ds_ptrs, lo_ptrs, sptr)
            C.lfa_svd_backward(plan.handle, ds_ptrs, u_ptrs, v_ptrs, dw_ptrs, sptr)
            C.lfa_expand(plan.handle, 0, u_ptrs[0], v_ptrs[0], f_exp * l0.r, cnt, uh.data_ptr(), vh.data_ptr(), sptr)

        return outs, forward, rest

    plan = LfaPlan(specs, vectors=vectors, tune_cache=args.tune_cache)
    outs, forward, rest = make_step(plan)
    sig = outs[:len(layers)]

    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        forward()
        rest()
    barrier()
    st, info = plan.info()
    if st != C.LFA_OK:
        raise RuntimeError(f"forward reported status {st}: {info}")

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    launches0 = C.lfa_kernel_launches()
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.25)
    barrier()
    for i in range(K):
        flush.fill_(i & 0xff)                       # L2 flush (untimed, outside the events)
        ev[i][0].record(stream)
        forward()
        ev[i][1].record(stream)
        rest()
        ev[i][2].record(stream)
    barrier()
    launches = C.lfa_kernel_launches() - launches0
    time.sleep(0.15)
    clocks = clk.stop()
    step_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(K)]
    fwd_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]
    total_ms = float(sum(step_ms))
    fwd_mean = float(sum(fwd_ms) / K)
    total_ms, fwd_mean = reduce_max([total_ms, fwd_mean], dist, dev)
    st, info = plan.info()

    # ---- plain per-layer forward-only path (materialised symbols, per-layer launches, no graph)
    plain = LfaPlan(specs, vectors=False, plain=True, tune_cache=args.tune_cache)
    psig, _, _ = plain.alloc(dev)
    pw = [w.data_ptr() for w in ws]
    pp = [s.data_ptr() for s in psig]
    for _ in range(3):
        C.lfa_svd(plain.handle, pw, pp, None, None, sptr)
    barrier()
    # the plain and end-to-end legs repeat the step about 20 s worth (at least 2, at most K, 50)
    reps_aux = max(2, min(K, 50, int(20000.0 / max(total_ms / K, 1e-3)) + 1))
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps_aux)]
    for e in pev:
        flush.fill_(1)
        e[0].record(stream)
        C.lfa_svd(plain.handle, pw, pp, None, None, sptr)
        e[1].record(stream)
    barrier()
    plain_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in pev]))

    # ---- the FFT route, the paper's comparison system (Table II), on the same GPU: the symbols of
    # every channel pair from one batched cuFFT transform, then the plain path's Jacobi; timed as a
    # forward, and its symbol stage alone against the direct tap sums of the plain path
    fft_leg = None
    if not args.no_fft_route and all((l.sh, l.sw) == (1, 1) for l in layers):
        fplan = LfaPlan(specs, vectors=False, fft_route=True, tune_cache=args.tune_cache)
        fsig, _, _ = fplan.alloc(dev)
        fp = [x.data_ptr() for x in fsig]
        for _ in range(2):
            C.lfa_svd(fplan.handle, pw, fp, None, None, sptr)
        barrier()
        fev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps_aux)]
        for e in fev:
            flush.fill_(4)
            e[0].record(stream)
            C.lfa_svd(fplan.handle, pw, fp, None, None, sptr)
            e[1].record(stream)
        barrier()
        fft_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in fev]))
        l0 = layers[0]
        symb = torch.empty((plain.meta[0]["F_h"], l0.c_out, l0.cols), dtype=torch.complex64, device=dev)
        stage = {}
        for name, call in (("fft_symbols_ms", lambda: C.lfa_fft_symbols(fplan.handle, 0, pw[0], symb.data_ptr(), sptr)),
                           ("assembly_symbols_ms", lambda: C.lfa_symbols(plain.handle, 0, pw[0], symb.data_ptr(), sptr))):
            call()
            barrier()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(5)
            a_.record(stream)
            for _ in range(5):
                call()
            b_.record(stream)
            barrier()
            stage[name] = a_.elapsed_time(b_) / 5
        fft_leg = {"forward_values_ms": fft_ms, "layers_per_s": len(layers) / (fft_ms / 1e3), **stage,
                   "layer0_symbols": f"{plain.meta[0]['F_h']} half-grid symbols of {l0.c_out}x{l0.cols}",
                   "route": "cuFFT batched R2C of the zero-padded kernel per channel pair + gather, then the "
                            "plain path's Jacobi (values)"}
        del symb
        fplan.close()

    peaks = {}
    if os.path.exists(PEAKS_FILE):
        try:
            peaks = json.load(open(PEAKS_FILE))
        except (OSError, ValueError):
            peaks = {}

    # ---- the lifting kernel alone (HBM-write bound): vector pairs of layer 0 writing about
    # 512 MiB per launch, more than L2 holds, so back-to-back launches each go to DRAM
    lift = None
    if vectors and not args.no_lift_roofline:
        l0 = layers[0]
        per_pair = lift_bytes_per_pair(l0)
        cnt = lift_pairs(l0)
        luh = torch.empty((cnt, l0.c_out, l0.n, l0.m), dtype=torch.complex64, device=dev)
        lvh = torch.empty((cnt, l0.c_in, l0.sh * l0.n, l0.sw * l0.m), dtype=torch.complex64, device=dev)
        u0, v0 = outs[len(layers)], outs[2 * len(layers)]     # U and V of layer 0

        def lift_call():
            C.lfa_expand(plan.handle, 0, u0.data_ptr(), v0.data_ptr(), 0, cnt, luh.data_ptr(), lvh.data_ptr(), sptr)

        for _ in range(3):
            lift_call()
        barrier()
        la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        la.record(stream)
        for _ in range(reps):
            lift_call()
        lb.record(stream)
        barrier()
        lift_ms = la.elapsed_time(lb) / reps
        gbs = per_pair * cnt / (lift_ms * 1e-3) / 1e9
        hbm = peaks.get("hbm_gbs")
        hbm_peak, hbm_src = (float(hbm), "measured copy bandwidth") if hbm else (6800.0, "fallback")
        lift = {"kernel": "expand_kernel (lifting, layer 0)", "bound": "hbm", "pairs": cnt,
                "bytes_per_launch": int(per_pair * cnt), "us_per_launch": lift_ms * 1e3,
                "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "peak_source": hbm_src,
                "timing": f"mean of {reps} back-to-back launches, each writing more than L2 holds"}
        del luh, lvh

    # ---- end to end through the public API from pinned host buffers, pipelined as a serving loop
    # would run it: step i's outputs go back to the host on a copy stream while step i + 1
    # computes into the other of two output sets (two plans, one captured graph each). Every
    # step's host-to-device input copy and device-to-host output copy is inside the timed region,
    # and so is the L2 flush between steps.
    e2e = None
    if not args.no_e2e:
        plan2 = LfaPlan(specs, vectors=vectors, tune_cache=args.tune_cache)
        sets = [(outs, forward, rest), make_step(plan2)]
        hw = [w.cpu().pin_memory() for w in ws]
        hout = [[torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in st_[0]] for st_ in sets]
        h2d = sum(x.numel() * x.element_size() for x in hw)
        d2h = sum(x.numel() * x.element_size() for x in hout[0])
        copy = torch.cuda.Stream(dev)
        for st_ in sets:                      # warm both graphs
            st_[1]()
            st_[2]()
        KE = reps_aux
        done = [torch.cuda.Event() for _ in range(2)]      # output set free again (its copy finished)
        ready = [torch.cuda.Event() for _ in range(KE)]    # step i computed
        for e in done:
            e.record(copy)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        t0.record(stream)
        for i in range(KE):
            b = i & 1
            souts, sfwd, srest = sets[b]
            flush.fill_(2)
            for d, h in zip(ws, hw):
                d.copy_(h, non_blocking=True)
            stream.wait_event(done[b])
            sfwd()
            srest()
            ready[i].record(stream)
            copy.wait_event(ready[i])
            with torch.cuda.stream(copy):
                for d, h in zip(souts, hout[b]):
                    h.copy_(d, non_blocking=True)
            done[b].record(copy)
        stream.wait_stream(copy)
        t1.record(stream)
        barrier()
        e2e_ms = t0.elapsed_time(t1) / KE
        (e2e_ms,) = reduce_max([e2e_ms], dist, dev)
        sig_per_step = sum(l.n_sigma for l in layers)
        e2e = {"value": aggregate_rate(sig_per_step, 1, world, e2e_ms), "unit": "singular values/s",
               "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "pipelined": "outputs of step i copied to the host while step i+1 computes (2 output sets)",
               "steps": KE}
        plan2.close()

    sig_per_step = sum(l.n_sigma for l in layers)
    ms_per_step = total_ms / K
    value = aggregate_rate(sig_per_step, K, world, total_ms)
    flops = sum(layer_flops(l, vectors) for l in layers)
    peak = fp32_peak_tflops()
    achieved = flops / (fwd_mean / 1e3) / 1e12
    traffic = measured_traffic(args.workload, info)
    routes = [m["variant"] for m in plan.meta]
    if routes[0] == C.LFA_VARIANT_BLOCKED:
        # the dominant kernel is the blocked Jacobi on the tensor cores (all layers of the workload
        # on that route): roofline against the TF32 tensor peak
        tpeak, tsrc = tf32_peak_tflops(peaks)
        executed = blocked_tensor_flops(layers[0], info["tc_grams"], info["tc_updates"], vectors)
        roofline = {
            "kernel": "bj_kernel (blocked one-sided Jacobi, tcgen05 3xTF32 Gram and block updates, %s)" % (
                "values+vectors" if vectors else "values"),
            "bound": "tensor",
            "achieved": achieved,
            "peak": tpeak,
            "unit": "TFLOP/s",
            "frac": achieved / tpeak,
            "traffic": traffic,
            "peak_source": tsrc,
            "flops_model": "nominal Golub-Van Loan complex SVD counts (x4) + symbol assembly, per half-grid symbol",
            "executed_sweeps_per_symbol": info["sweeps"] / max(1, info["symbols"]),
            "tensor_grams": info["tc_grams"],
            "tensor_updates": info["tc_updates"],
            "executed_tflops": executed / (fwd_mean / 1e3) / 1e12,
            "executed_frac": executed / (fwd_mean / 1e3) / 1e12 / tpeak,
            "executed_model": "tensor flops issued: 3 TF32 products per real block product (Gram and update)",
        }
    else:
        roofline = {
            "kernel": "jacobi_kernel (fused symbol assembly + one-sided Jacobi, %s)" % (
                "values+vectors" if vectors else "values"),
            "bound": "alu",
            "achieved": achieved,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "peak_source": f"derived: {SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz",
            "flops_model": "nominal Golub-Van Loan complex SVD counts (x4) + symbol assembly, per half-grid symbol",
            "executed_sweeps_per_symbol": info["sweeps"] / max(1, info["symbols"]),
            "rotations": info["rotations"],
            "executed_tflops": executed_flops(layers, info, vectors) / (fwd_mean / 1e3) / 1e12,
            "executed_frac": executed_flops(layers, info, vectors) / (fwd_mean / 1e3) / 1e12 / peak,
        }

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "singular values/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded He-normal weights; the paper's weights are unstated)",
        "config": {
            "workload": args.workload,
            "layers": [layer_name(l) for l in layers],
            "outputs": "values+vectors (U, V per half-grid frequency)" if vectors else "values only",
            "step": ("fwd(assembly+Jacobi, graph) + regulariser dL/dsigma + bwd dL/dw + lift min(r, 64) vector "
                     "pairs of one frequency"
                     if vectors else "fwd(assembly+Jacobi, all layers in one graph-replayed launch per variant)"),
            "l2": f"flushed between timed steps ({args.flush_mb} MB write, outside the timed events)",
            "parallelism": f"dp{world} (independent layers per rank)",
        },
        "layers_per_s": world * len(layers) * K / (total_ms / 1e3),
        "symbols_per_s": world * sum(l.F for l in layers) * K / (total_ms / 1e3),
        "fwd_ms": fwd_mean,
        "plain_fwd_values_ms": plain_ms,
        "plain_layers_per_s": len(layers) / (plain_ms / 1e3),
        "fft_route": fft_leg,
        "roofline": roofline,
        "routes": [C.lfa_variant_name(v) for v in routes],
        "clocks": clocks,
        "gpu_launches": int(launches),
        "accuracy": {"unconverged": info["unconverged"], "nonfinite": info["nonfinite"]},
        "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")} if peaks else None,
    }
    if lift is not None:
        out["lift_roofline"] = lift
    if e2e is not None:
        out["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = run_oracle(layers[0], args.cpu_seconds, args.cpu_freqs, vectors=vectors)
        # the sampled oracle frequencies also give an accuracy check of this run's sigma
        rng = np.random.default_rng(5)
        fr = np.sort(rng.choice(layers[0].F, min(64, layers[0].F), replace=False))
        s_ref = oracle_values(W.weights(layers[0], seed=layers[0].seed), layers[0], fr)
        s_gpu = sig[0].cpu().numpy()[fr]
        cb["sigma_err_vs_oracle_rel_sigma_max"] = float(np.max(np.abs(s_gpu - s_ref)) / s_ref.max())
        cb.pop("step_s", None)
        one = run_oracle_one_core(args.workload, args.cpu_seconds, max(1, args.cpu_freqs // 4), vectors)
        one.pop("step_s", None)
        cb["one_core"] = one
        cb["fft_route"] = run_fft_route(layers[0], cb["s_per_frequency"], vectors)
        out["cpu_baseline"] = cb
    if dist is not None:
        dist.destroy_process_group()
    plan.close()
    plain.close()
    return out


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on bounded samples of the same workload."""
    layers = W.layers(args.workload)
    vectors = not (args.values_only or args.workload in VALUES_ONLY)
    lay = layers[0]
    w = W.weights(lay)
    rng = np.random.default_rng(7)
    nf = min(args.cpu_freqs, lay.F)
    for _ in range(args.warmup):
        oracle_sample_step(w, lay, np.sort(rng.choice(lay.F, nf, replace=False)), 0, vectors)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(w, lay, np.sort(rng.choice(lay.F, nf, replace=False)), 0, vectors)
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    value = args.steps * nf * lay.r / wall
    sample = f"{nf} of {lay.F} frequencies per step of layer 0 " + (
        "(FP64 oracle: symbols, LAPACK SVD with U,V, regulariser, dL/dw, lift)" if vectors
        else "(FP64 oracle: symbols, LAPACK SVD values)")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "singular values/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded He-normal weights)",
        "config": {"workload": args.workload,
                   "layers": [layer_name(l) for l in layers],
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "singular values/s", "cores": round(cpu / wall, 2),
                         "cores_available": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "singular values/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def run_forward_once(args):
    """One forward of the workload on cuda:0 through the public API (no graph), for profiling; with
    --with-backward (and vectors) also the regulariser gradient and the backward of that step."""
    import torch
    from paper_2506_05617_gb300 import build as B
    from paper_2506_05617_gb300.torch_api import LfaPlan
    B.build()
    layers = W.layers(args.workload)
    vectors = not (args.values_only or args.workload in VALUES_ONLY)
    plan = LfaPlan([l.desc() for l in layers], vectors=vectors, use_graph=0, tune_cache=args.tune_cache)
    ws = [torch.from_numpy(W.weights(l)).cuda() for l in layers]
    sig, U, V = plan.svd(ws)
    if args.with_backward and vectors:
        dsig, _ = plan.regulariser_grad(sig, LAM)
        plan.backward(dsig, U, V)
    torch.cuda.synchronize()
    st, info = plan.info()
    print(json.dumps({"workload": args.workload, "routes": [m["variant_name"] for m in plan.meta], "status": st,
                      "sweeps_per_symbol": info["sweeps"] / max(1, info["symbols"]),
                      "tc_grams": info["tc_grams"], "tc_updates": info["tc_updates"]}))
    plan.close()
    return 0 if st == 0 else 1


def run_sweep(args):
    """O(N) study: the 64->64 3x3 layer at each torus size n (values + vectors forward), one JSON
    line per n. The time per symbol stays flat once the GPU is full, so the time grows with the
    number of frequencies n^2, i.e. linearly in the operator size N = c n^2."""
    import torch
    from paper_2506_05617_gb300 import build as B
    from paper_2506_05617_gb300.torch_api import LfaPlan
    B.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device=dev)
    for n in (int(x) for x in args.sweep_n.split(",")):
        lay = W.conv64_sweep(n)[0]
        w = torch.from_numpy(W.weights(lay)).to(dev)
        for vectors in (True, False):
            plan = LfaPlan([lay.desc()], vectors=vectors, tune_cache=args.tune_cache)
            out = plan.alloc(dev)
            for _ in range(max(3, args.warmup)):
                plan.svd([w], out=out)
            ts = []
            for _ in range(args.steps):
                flush.fill_(3)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                plan.svd([w], out=out)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            st, info = plan.info()
            F_h = plan.meta[0]["F_h"]
            plan.close()
            ms = float(np.median(ts))
            print(json.dumps({"sweep": "n", "workload": "conv64_k3", "n": n, "outputs": "values+vectors" if vectors
                              else "values", "ms": ms, "symbols_half_grid": F_h,
                              "singular_values_per_s": n * n * lay.r / (ms / 1e3),
                              "us_per_half_grid_symbol": ms * 1e3 / F_h, "status": st,
                              "sweeps_per_symbol": info["sweeps"] / max(1, info["symbols"])}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lfa", "reference"], default="lfa")
    ap.add_argument("--workload", default="conv512_k3_n64", choices=sorted(W.WORKLOADS))
    ap.add_argument("--flush-mb", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-freqs", type=int, default=None,
                    help="oracle frequencies per sample step (default: 64, or 2 for 512-channel layers)")
    ap.add_argument("--cpu-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fft-route", action="store_true", help="skip the GPU FFT-route (comparison) leg")
    ap.add_argument("--forward-once", action="store_true",
                    help="build the workload's plan, run one forward (values + vectors unless values-only) and "
                         "exit: the small launch a profiler captures")
    ap.add_argument("--with-backward", action="store_true",
                    help="with --forward-once: also the regulariser gradient and the backward")
    ap.add_argument("--values-only", action="store_true", help="values only (no vectors, backward, lifting)")
    ap.add_argument("--tune-cache", default=DEFAULT_TUNE if os.path.exists(DEFAULT_TUNE) else None,
                    help="autotuner cache file read by lfa_plan")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-lift-roofline", action="store_true",
                    help="skip the separate timing of the lifting kernel on a larger-than-L2 output")
    ap.add_argument("--sweep-n", default=None,
                    help="comma-separated torus sizes: run the O(N) study of the 64->64 layer instead "
                         "(one JSON line per n and output mode)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_freqs is None:
        lay0 = W.layers(args.workload)[0]
        args.cpu_freqs = 2 if max(lay0.c_out, lay0.cols) >= 512 else 64
    if args.cpu_leg:
        # the one-core oracle leg, run by run_oracle_one_core in a fresh interpreter
        vectors = not (args.values_only or args.workload in VALUES_ONLY)
        print(json.dumps(run_oracle(W.layers(args.workload)[0], args.cpu_seconds, args.cpu_freqs, vectors=vectors)))
        return 0
    if args.sweep_n:
        return run_sweep(args)
    if args.forward_once:
        return run_forward_once(args)
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0
    out = run_lfa(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
