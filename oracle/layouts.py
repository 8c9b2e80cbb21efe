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


# ---------------------------------------------------------------------------
# zero-rotation ("volley") matmul layout
# ---------------------------------------------------------------------------
# The revolver of Alg. 3 turns B's rows past A's columns by rotations; with B~_k
# tiled with period p over the whole ring, slot s of B~_k holds B[k][s mod p].
# Placing copies of A's column k at block starts t*M + o (M = 1 mod p) lines slot
# t*M + o + i up with B[k][(t + o + i) mod p], i.e. with the t-th revolver
# position shifted by o, so one product per k yields p' diagonals at once and no
# rotation is needed. Blocks must fit the S slots; when all p do not, the
# positions are split into G groups, group g starting at idx = g*per with block
# offset o_g = (g*per) mod p.

def volley_geometry(slots: int, m: int, p: int):
    """-> (M, per, G, offsets): block stride, positions per ciphertext, groups."""
    if m < 1 or p < 1 or slots % p:
        raise ValueError("p must divide the slot count")
    M = m + (1 - m) % p if p > 1 else m
    if (p - 1) * M + m <= slots:
        return M, p, 1, [0]
    per = (slots - m - (p - 1)) // M + 1
    if per < 1:
        raise ValueError("matrix does not fit the slots")
    G = -(-p // per)
    return M, per, G, [(g * per) % p for g in range(G)]


def matrix_a_volley(A: np.ndarray, slots: int, p: int) -> np.ndarray:
    """A [m][n] -> [G][n][slots]: slot t*M + o_g + i of group g, column k = A[i][k]."""
    m, n = A.shape
    M, per, G, off = volley_geometry(slots, m, p)
    z = np.zeros((G, n, slots))
    for g in range(G):
        for t in range(min(per, p - g * per)):
            z[g, :, t * M + off[g]: t * M + off[g] + m] = A.T
    return z


def matmul_from_volley(d: np.ndarray, m: int, p: int) -> np.ndarray:
    """slot vectors [G][slots] of the volley products -> C [m][p]."""
    slots = d.shape[-1]
    M, per, G, off = volley_geometry(slots, m, p)
    C = np.zeros((m, p))
    for g in range(G):
        for t in range(min(per, p - g * per)):
            idx = g * per + t
            for i in range(m):
                C[i, (i + idx) % p] = d[g, t * M + off[g] + i]
    return C
