"""Slot layouts of the paper's multi-ciphertext method (oracle side).

TEST INFRASTRUCTURE. Plain numpy restatement of how data are placed in and
read back from ciphertext slots:

* image column layout (abstract; Sec. I-C): an h x w image is w ciphertexts,
  ciphertext j holding column j; row r of image b sits at slot b*H + g*r
  (H the block stride, one image per block as in the virtual ciphertexts of
  Sec. III-D; g the row gap, 1 for an input image),
* matmul operands (abstract; Sec. I-C): A (m x n) is n ciphertexts, A_k
  holding column k at slots i < m; B (n x p) is n ciphertexts, B~_k holding row
  k tiled with period p over every slot (tau_b's tiling, Sec. III-A),
* matmul result: p ciphertexts D_idx, slot i of D_idx = C[i][(i + idx) mod p].
"""
from __future__ import annotations

import numpy as np


def image_columns(images: np.ndarray, slots: int, H: int, gap: int = 1) -> np.ndarray:
    """images [B][h][w] -> slot vectors [w][slots]."""
    B, h, w = images.shape
    if B * H > slots or gap * (h - 1) >= H:
        raise ValueError("images do not fit the blocks")
    z = np.zeros((w, slots))
    for b in range(B):
        for i in range(h):
            z[:, b * H + gap * i] = images[b, i, :]
    return z


def image_from_columns(z: np.ndarray, B: int, H: int, gap: int, h_valid: int) -> np.ndarray:
    """slot vectors [..., w][slots] -> [..., B, h_valid, w] (valid rows only)."""
    lead = z.shape[:-2]
    w = z.shape[-2]
    out = np.zeros(lead + (B, h_valid, w))
    for b in range(B):
        for i in range(h_valid):
            out[..., b, i, :] = z[..., :, b * H + gap * i]
    return out


def matrix_a_columns(A: np.ndarray, slots: int) -> np.ndarray:
    """A [m][n] -> [n][slots], slot i of A_k = A[i][k]."""
    m, n = A.shape
    z = np.zeros((n, slots))
    z[:, :m] = A.T
    return z


def matrix_b_rows(Bm: np.ndarray, slots: int) -> np.ndarray:
    """B [n][p] -> [n][slots], slot s of B~_k = B[k][s mod p]."""
    n, p = Bm.shape
    if slots % p:
        raise ValueError("p must divide the slot count")
    return np.tile(Bm, (1, slots // p))


def matmul_from_diagonals(d: np.ndarray, m: int, p: int) -> np.ndarray:
    """slot vectors [p][slots] of D_idx -> C [m][p]."""
    C = np.zeros((m, p))
    for idx in range(p):
        for i in range(m):
            C[i, (i + idx) % p] = d[idx, i]
    return C


def logits_from_fc(z: np.ndarray, B: int, H: int) -> np.ndarray:
    """slot vectors [out][slots] -> logits [B][out] (slot b*H of output o)."""
    return np.stack([z[:, b * H] for b in range(B)])
