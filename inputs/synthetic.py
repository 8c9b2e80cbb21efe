"""Seeded synthetic workloads for the encrypted matmul / convolution / CNN path.

This module is shared by the tests, the oracle runs and the benchmark. It
draws the plaintext inputs -- images, matrices, kernel and dense weights,
biases, request traces -- and holds none of the scheme's arithmetic.

The paper evaluates on MNIST with trained weights (Sec. V, Table "tab1"),
neither of which is available here; these seeded draws stand in for them with
the shapes and value ranges of the workloads:

* images: pixels uniform on [0, 1] (the paper normalises pixels to [0, 1],
  Sec. V-B),
* matmul operands: entries uniform on [-1, 1],
* kernel / dense weights and biases: normal with mean 0 and the stated
  standard deviation.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Scheme parameter presets: ring degree, prime bit sizes, scale.
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class ParamPreset:
    name: str
    log_n: int
    q_bits: Tuple[int, ...]      # q_0 (base prime) first, then q_1 .. q_L
    n_special: int               # K special primes of the key-switching modulus P
    special_bits: int
    alpha: int                   # primes per key-switching digit
    log_scale: float
    sigma: float = 3.2


# 4x8 . 8x4 matmul, N = 2^13, Q = 60 + 40 + 40 bits, P = 60 bits, scale 2^40.
MATMUL_SMALL = ParamPreset("matmul_n13", 13, (60, 40, 40), 1, 60, 1, 40.0)
# One conv + x^2 layer on a 64x64 image, N = 2^15, Q = 60 + 8 x 40, P = 60.
CONV_LAYER = ParamPreset("conv_n15", 15, (60,) + (40,) * 8, 1, 60, 1, 40.0)
# Three-layer CNN on 128x128 images, N = 2^16, Q = 60 + 12 x 45, P = 2 x 60,
# digits of alpha = 2 primes (beta = 7 digits at the top level).
CNN_N16 = ParamPreset("cnn_n16", 16, (60,) + (45,) * 12, 2, 60, 2, 45.0)
# The same chain with three key-switching digits (dnum = 3: alpha = 5 primes a digit) and
# K = 5 special primes of 60 bits, so that P (300 bits) exceeds the largest digit (240 bits).
CNN_N16_DNUM3 = ParamPreset("cnn_n16_dnum3", 16, (60,) + (45,) * 12, 5, 60, 5, 45.0)


def small_preset(log_n: int, q_bits=(60, 40, 40, 40), n_special=1, special_bits=60,
                 alpha=1, log_scale=40.0) -> ParamPreset:
    """A reduced-ring preset for fast tests (same prime rule, smaller N)."""
    return ParamPreset(f"small_n{log_n}", log_n, tuple(q_bits), n_special,
                       special_bits, alpha, float(log_scale))


# ---------------------------------------------------------------------------
# Workload draws.
# ---------------------------------------------------------------------------

def matmul_operands(m: int, n: int, p: int, seed: int = 101):
    """A (m x n) and B (n x p) with entries uniform on [-1, 1]."""
    g = _rng(seed)
    a = g.uniform(-1.0, 1.0, size=(m, n))
    b = g.uniform(-1.0, 1.0, size=(n, p))
    return a, b


def images(batch: int, h: int, w: int, seed: int) -> np.ndarray:
    """Grayscale images [batch][h][w], pixels uniform on [0, 1]."""
    return _rng(seed).uniform(0.0, 1.0, size=(batch, h, w))


def conv_weights(c_out: int, c_in: int, k: int, std: float, seed: int):
    """Kernels [c_out][c_in][k][k] and biases [c_out], both N(0, std^2)."""
    g = _rng(seed)
    w = g.normal(0.0, std, size=(c_out, c_in, k, k))
    b = g.normal(0.0, std, size=(c_out,))
    return w, b


@dataclasses.dataclass
class CnnWeights:
    conv1_w: np.ndarray
    conv1_b: np.ndarray
    conv2_w: np.ndarray
    conv2_b: np.ndarray
    fc_w: np.ndarray      # [10][16 * h2 * w2], flattened in (channel, row, col) order
    fc_b: np.ndarray


def cnn_shapes(side: int):
    """Spatial sizes through conv 5x5 s2 -> conv 3x3 s2 for a side x side image."""
    h1 = (side - 5) // 2 + 1
    h2 = (h1 - 3) // 2 + 1
    return h1, h2


def cnn_weights(side: int = 128, std: float = 0.05, seed: int = 302) -> CnnWeights:
    """Random-init weights of conv 8x5x5 s2 -> x^2 -> conv 16x3x3 s2 -> x^2 -> FC 10.

    The conv weights are drawn from `seed`; the FC layer depends on the image
    side, so it is drawn from a stream of its own, seeded by (seed, side).
    """
    g = _rng(seed)
    c1w = g.normal(0.0, std, size=(8, 1, 5, 5))
    c1b = g.normal(0.0, std, size=(8,))
    c2w = g.normal(0.0, std, size=(16, 8, 3, 3))
    c2b = g.normal(0.0, std, size=(16,))
    _, h2 = cnn_shapes(side)
    gf = _rng(seed * 1000003 + side)
    fcw = gf.normal(0.0, std, size=(10, 16 * h2 * h2))
    fcb = gf.normal(0.0, std, size=(10,))
    return CnnWeights(c1w, c1b, c2w, c2b, fcw, fcb)


@dataclasses.dataclass
class Table1Weights:
    """Table I's CNN: CONV (c kernels k x k, stride 1) -> ACT-1 -> FC-1 -> ACT-2 -> FC-2."""
    conv_w: np.ndarray  # [c][k][k]
    conv_b: np.ndarray  # [c]
    fc1_w: np.ndarray   # [c][ho][wo][fc1_out], inputs in (channel, row, column) order
    fc1_b: np.ndarray   # [fc1_out]
    fc2_w: np.ndarray   # [fc1_out][fc2_out]
    fc2_b: np.ndarray   # [fc2_out]


def table1_weights(h: int = 28, w: int = 28, c: int = 4, k: int = 3, fc1_out: int = 64, fc2_out: int = 10,
                   seed: int = 202) -> Table1Weights:
    """Synthetic weights of Table I's shapes (the trained MNIST weights are not available):
    kernels and biases N(0, 0.1^2); dense weights N(0, 1 / fan_in) scaled by 0.5 so that the
    activations stay in the range the degree-3 fits of Table I were made for; dense biases
    N(0, 0.05^2)."""
    g = _rng(seed)
    ho, wo = h - k + 1, w - k + 1
    n1 = c * ho * wo
    return Table1Weights(
        conv_w=g.normal(0.0, 0.1, size=(c, k, k)),
        conv_b=g.normal(0.0, 0.1, size=(c,)),
        fc1_w=g.normal(0.0, 0.5 / np.sqrt(n1), size=(c, ho, wo, fc1_out)),
        fc1_b=g.normal(0.0, 0.05, size=(fc1_out,)),
        fc2_w=g.normal(0.0, 0.5 / np.sqrt(fc1_out), size=(fc1_out, fc2_out)),
        fc2_b=g.normal(0.0, 0.05, size=(fc2_out,)),
    )


def batched_matmul_shapes(count: int = 64, seed: int = 401,
                          choices=(16, 32, 64, 128, 256)) -> List[Tuple[int, int, int]]:
    """(m, n, p) triples drawn i.i.d. uniformly from `choices`."""
    g = _rng(seed)
    return [tuple(int(x) for x in g.choice(choices, size=3)) for _ in range(count)]


def poisson_trace(n_requests: int, rate: float = 20.0, seed_arrival: int = 501,
                  seed_side: int = 502, sides=(64, 128, 256)):
    """Arrival times (s) of a Poisson stream and an image side per request."""
    ga = _rng(seed_arrival)
    gs = _rng(seed_side)
    gaps = ga.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps)
    side = gs.choice(sides, size=n_requests)
    return t, side
