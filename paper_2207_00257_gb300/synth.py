"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no convolution arithmetic: it only draws tensors. Both the
CUDA path and the CPU oracle receive exactly the tensors made here.

Recipe (the paper's workload is ResNet-50 trained on synthetic ImageNet-shaped
inputs, Sec. 6.C; the layer shapes below are its bottleneck convolutions):

* every tensor is drawn on the CPU from ``torch.Generator().manual_seed(seed)``
  in the order x, w, b, then g (upstream gradient);
* "uniform" tensors are ``rand * 2 - 1`` (U[-1, 1]); biases are U[-0.1, 0.1];
* activations are N(0, 1); ``relu_normal`` activations are max(N(0, 1), 0);
* He-normal filters have std sqrt(2 / (C*R*S));
* integer tensors are drawn uniformly from a closed integer range.

Tensors come back as float32 CPU tensors in the requested layout
(NCHW with KCRS filters, or NHWC with KRSC filters).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import torch

_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "tests", "golden")


@dataclass
class ConvShape:
    N: int
    C: int
    H: int
    W: int
    K: int
    R: int
    S: int
    stride: tuple = (1, 1)
    pad: tuple = (0, 0)
    dil: tuple = (1, 1)
    layout: str = "NHWC"
    tag: str = ""

    def __post_init__(self):
        for name in ("stride", "pad", "dil"):
            v = getattr(self, name)
            if isinstance(v, int):
                setattr(self, name, (v, v))
            else:
                setattr(self, name, tuple(v))

    @property
    def P(self):
        return (self.H + 2 * self.pad[0] - self.dil[0] * (self.R - 1) - 1) // self.stride[0] + 1

    @property
    def Q(self):
        return (self.W + 2 * self.pad[1] - self.dil[1] * (self.S - 1) - 1) // self.stride[1] + 1

    @property
    def flops(self):
        return 2 * self.N * self.K * self.P * self.Q * self.C * self.R * self.S

    def x_shape(self):
        return ((self.N, self.C, self.H, self.W) if self.layout == "NCHW"
                else (self.N, self.H, self.W, self.C))

    def w_shape(self):
        return ((self.K, self.C, self.R, self.S) if self.layout == "NCHW"
                else (self.K, self.R, self.S, self.C))

    def y_shape(self):
        return ((self.N, self.K, self.P, self.Q) if self.layout == "NCHW"
                else (self.N, self.P, self.Q, self.K))


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator()
    g.manual_seed(int(seed))
    return g


def _uniform(shape, g, scale=1.0):
    return (torch.rand(shape, generator=g, dtype=torch.float32) * 2 - 1) * scale


def make_inputs(shape: ConvShape, seed: int, x_dist="normal", w_dist="he", bias=True,
                grad=False):
    """Draw (x, w, b, g) float32 tensors for one convolution.

    x_dist: "normal" | "relu_normal" | "uniform" | ("int", lo, hi)
    w_dist: "he" | "uniform" | ("int", lo, hi)
    b: U[-0.1, 0.1] (or ("int", lo, hi) when x_dist is integer), None if not bias.
    g: N(0, 1) upstream gradient of y's shape if grad, else None.
    """
    gen = _gen(seed)
    xs, ws, ys = shape.x_shape(), shape.w_shape(), shape.y_shape()
    if isinstance(x_dist, tuple):
        x = torch.randint(x_dist[1], x_dist[2] + 1, xs, generator=gen).float()
    elif x_dist == "normal":
        x = torch.randn(xs, generator=gen, dtype=torch.float32)
    elif x_dist == "relu_normal":
        x = torch.randn(xs, generator=gen, dtype=torch.float32).clamp_min(0.0)
    elif x_dist == "uniform":
        x = _uniform(xs, gen)
    else:
        raise ValueError(x_dist)
    if isinstance(w_dist, tuple):
        w = torch.randint(w_dist[1], w_dist[2] + 1, ws, generator=gen).float()
    elif w_dist == "he":
        w = torch.randn(ws, generator=gen, dtype=torch.float32) * math.sqrt(
            2.0 / (shape.C * shape.R * shape.S))
    elif w_dist == "uniform":
        w = _uniform(ws, gen)
    else:
        raise ValueError(w_dist)
    b = None
    if bias:
        if isinstance(x_dist, tuple):
            b = torch.randint(-8, 9, (shape.K,), generator=gen).float()
        else:
            b = _uniform((shape.K,), gen, 0.1)
    g = torch.randn(ys, generator=gen, dtype=torch.float32) if grad else None
    return x, w, b, g


# ---- the workloads ----

def config_tiny_fp32():
    """Single FP32 NCHW conv: N=1, C=3, 32x32, K=16, 3x3, stride 1, pad 1; seed 0, U[-1,1]."""
    return ConvShape(1, 3, 32, 32, 16, 3, 3, 1, 1, 1, layout="NCHW", tag="tiny_fp32_nchw")


def resnet_layers(batch: int = 32):
    """ResNet-50 bottleneck layer set, NHWC, batch 32 (each with bias + ReLU)."""
    return [
        ConvShape(batch, 256, 56, 56, 64, 1, 1, 1, 0, 1, tag="L1_1x1_256to64_56"),
        ConvShape(batch, 64, 56, 56, 64, 3, 3, 1, 1, 1, tag="L2_3x3_64to64_56"),
        ConvShape(batch, 64, 56, 56, 256, 1, 1, 1, 0, 1, tag="L3_1x1_64to256_56"),
        ConvShape(batch, 128, 56, 56, 128, 3, 3, 2, 1, 1, tag="L4_3x3s2_128to128_56to28"),
    ]


def config_fp8():
    """FP8-E4M3 forward: N=64, C=K=256, 28x28, 3x3, pad 1, x = ReLU(N(0,1)), He w."""
    return ConvShape(64, 256, 28, 28, 256, 3, 3, 1, 1, 1, tag="fp8_64x256x28_3x3")


def config_backward():
    """Backward: N=32, C=K=128, 56x56, 3x3, pad 1, g = N(0,1)."""
    return ConvShape(32, 128, 56, 56, 128, 3, 3, 1, 1, 1, tag="bwd_32x128x56_3x3")


def config_backward_fd():
    """Finite-difference check size: N=1, C=K=4, 6x6, 3x3, pad 1."""
    return ConvShape(1, 4, 6, 6, 4, 3, 3, 1, 1, 1, tag="bwd_fd_tiny")


def grouped_problems(path: str | None = None):
    """The 64 independent problems of the grouped launch.

    Drawn once with numpy.random.default_rng(1) by tests/golden/make_grouped_shapes.py
    and committed as JSON so that a numpy upgrade cannot change them."""
    path = path or os.path.join(_GOLDEN, "grouped_shapes_seed1.json")
    with open(path) as f:
        rows = json.load(f)["problems"]
    return [ConvShape(r["N"], r["C"], r["H"], r["W"], r["K"], r["R"], r["S"],
                      r["stride"], r["pad"], 1, tag=f"g{i}") for i, r in enumerate(rows)]


def sample_indices(total: int, count: int, seed: int):
    """Seeded sample of linear output indices (sorted, unique), always including
    the first and last element so the ragged tail is checked."""
    import numpy as np
    if total <= count:
        return np.arange(total, dtype=np.int64)
    rng = np.random.default_rng(seed)
    idx = rng.choice(total, size=count - 2, replace=False)
    return np.unique(np.concatenate([idx, [0, total - 1]]).astype(np.int64))
