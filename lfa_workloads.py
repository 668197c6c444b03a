"""Seeded synthetic workloads for the LFA SVD of periodic convolutions.

This module holds only shapes, seeds and random-number recipes. It contains no
arithmetic of the method (no symbols, no phases, no SVD), so both the FP64
oracle and the CUDA path may draw their inputs from it without sharing any of
the method's code.

Weights follow PyTorch's conv layout ``[c_out][c_in][k_h][k_w]`` (the paper's
implementation works on PyTorch channel-first tensors, Sec. IV "Runtime
Analysis"). Every tensor is drawn in float64 with ``numpy.random.default_rng``
and rounded to float32 once; the oracle upcasts those float32 values, so a
parity error measures only the SVD, not the rounding of the inputs.

The paper trains no network for its measurements and does not state its weight
values (Sec. IV, c_in = c_out = 16 random tensors), so these seeded tensors
stand in for them. Layer shapes follow common CNN layers: a ResNet-18 body
(3x3 convolutions at 56/28/14/7 pixels) and a 7x7 stem.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict
from typing import List

import numpy as np


@dataclass(frozen=True)
class Layer:
    """One periodic convolution: weight [c_out, c_in, kh, kw], output on an n x m torus.

    ``pad_h``/``pad_w`` is the tap origin p: tap (a, b) acts at offset
    (a - pad_h, b - pad_w). -1 means floor(k/2) (the centred stencil).
    ``sh``/``sw`` is the stride: the input lives on the (sh n) x (sw m) torus.
    """
    c_out: int
    c_in: int
    kh: int
    kw: int
    n: int
    m: int
    init: str = "normal"      # "normal": N(0, gain/(c_in*kh*kw)); "uniform": U(-1,1)*sqrt(6/fan_in)
    gain: float = 2.0
    seed: int = 0
    pad_h: int = -1
    pad_w: int = -1
    sh: int = 1
    sw: int = 1

    @property
    def cols(self) -> int:
        """Columns of a symbol: the input channels times the polyphase components per cell."""
        return self.c_in * self.sh * self.sw

    @property
    def r(self) -> int:
        return min(self.c_out, self.cols)

    def desc(self):
        """(c_out, c_in, kh, kw, n, m, pad_h, pad_w, stride_h, stride_w)."""
        return (self.c_out, self.c_in, self.kh, self.kw, self.n, self.m, self.pad_h, self.pad_w, self.sh, self.sw)

    @property
    def F(self) -> int:
        return self.n * self.m

    @property
    def n_sigma(self) -> int:
        return self.n * self.m * self.r

    def origin(self):
        ph = self.kh // 2 if self.pad_h < 0 else self.pad_h
        pw = self.kw // 2 if self.pad_w < 0 else self.pad_w
        return ph, pw

    def asdict(self):
        return asdict(self)


def weights(layer: Layer, seed: int | None = None) -> np.ndarray:
    """Seeded float32 weight tensor [c_out, c_in, kh, kw] (drawn in float64, rounded once)."""
    rng = np.random.default_rng(layer.seed if seed is None else seed)
    shape = (layer.c_out, layer.c_in, layer.kh, layer.kw)
    fan_in = layer.c_in * layer.kh * layer.kw
    if layer.init == "normal":
        w = rng.standard_normal(shape) * np.sqrt(layer.gain / fan_in)
    elif layer.init == "uniform":
        w = rng.uniform(-1.0, 1.0, shape) * np.sqrt(6.0 / fan_in)
    else:
        raise ValueError(f"unknown init {layer.init!r}")
    return w.astype(np.float32)


def upstream_gradient(shape, seed: int) -> np.ndarray:
    """Seeded float32 upstream gradient dL/dsigma of the given shape, N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape).astype(np.float32)


def _resnet18_body() -> List[Layer]:
    spec = ([(64, 64, 56)] * 4 + [(64, 128, 28)] + [(128, 128, 28)] * 3
            + [(128, 256, 14)] + [(256, 256, 14)] * 3
            + [(256, 512, 7)] + [(512, 512, 7)] * 3)
    return [Layer(c_out=co, c_in=ci, kh=3, kw=3, n=n, m=n, init="normal", gain=2.0, seed=300 + i)
            for i, (ci, co, n) in enumerate(spec)]


def _resnet18_strided() -> List[Layer]:
    # the stride-2 layers of a ResNet-18 whose symbols have at most 512 columns: the 7x7 stem on a
    # 224 input (112 output) and the first 3x3 conv and 1x1 shortcut of stages 2 and 3
    spec = [(3, 64, 7, 112), (64, 128, 3, 28), (64, 128, 1, 28), (128, 256, 3, 14), (128, 256, 1, 14)]
    return [Layer(c_out=co, c_in=ci, kh=k, kw=k, n=n, m=n, init="normal", gain=2.0, seed=500 + i, sh=2, sw=2)
            for i, (ci, co, k, n) in enumerate(spec)]


# Named workloads. Sizes are the paper-shaped synthetic stand-ins.
WORKLOADS = {
    # single 4->4 3x3 conv on 8x8: 256 singular values; the dense 256x256 operator is the cross-check
    "conv4_k3_n8": [Layer(4, 4, 3, 3, 8, 8, "normal", 1.0, 1)],
    # single ResNet-style 64->64 3x3 conv on 32x32 (1024 symbols, 514 on the half grid)
    "conv64_k3_n32": [Layer(64, 64, 3, 3, 32, 32, "normal", 2.0, 2)],
    # 16 stride-1 3x3 layers shaped like a ResNet-18 body, uneven c_in, c_out and n
    "resnet18_body": _resnet18_body(),
    # spectral regulariser workload: 4 layers 128->128 on 32x32 with k = 3, 5, 3, 5
    "reg4_c128_n32": [Layer(128, 128, k, k, 32, 32, "normal", 2.0, 400 + i)
                      for i, k in enumerate([3, 5, 3, 5])],
    # large square: 512->512 3x3 on 64x64
    "conv512_k3_n64": [Layer(512, 512, 3, 3, 64, 64, "uniform", 0.0, 51)],
    # the same layer on the 7x7 torus of a ResNet-18's last stage (25 half-grid symbols): the small
    # case of the 512-channel kernels for profiling
    "conv512_k3_n7": [Layer(512, 512, 3, 3, 7, 7, "uniform", 0.0, 51)],
    # the same layer on 16x16 (130 half-grid symbols: one wave of one symbol per SM)
    "conv512_k3_n16": [Layer(512, 512, 3, 3, 16, 16, "uniform", 0.0, 51)],
    # stem: 3->64 7x7 on 224x224 (tall 64x3 symbols)
    "stem3to64_k7_n224": [Layer(64, 3, 7, 7, 224, 224, "uniform", 0.0, 52)],
    # stride-2 layers (crystals with 4 polyphase components per coarse cell)
    "resnet18_strided": _resnet18_strided(),
    # the paper's runtime shape: 16->16 3x3 (Table II uses n = 256 ... 16384)
    "paper_c16_k3_n256": [Layer(16, 16, 3, 3, 256, 256, "normal", 2.0, 6)],
}


def conv64_sweep(n: int) -> List[Layer]:
    """The 64->64 3x3 layer at a swept input size n (O(N) scaling study)."""
    return [Layer(64, 64, 3, 3, n, n, "normal", 2.0, 2)]


def layers(name: str) -> List[Layer]:
    return list(WORKLOADS[name])
