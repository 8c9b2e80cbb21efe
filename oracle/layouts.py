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


# ---------------------------------------------------------------------------
# single-ciphertext layout of the paper's original method (virtual ciphertexts)
# ---------------------------------------------------------------------------
# Sec. III-D packs several images into one ciphertext as virtual ciphertexts; in
# this reading image b is row-major inside a block of Hb x Wb slots starting at
# slot b Hb Wb (row r at b Hb Wb + r Wb), zeros elsewhere, so Rot by pos and by
# pos Wb move one column / one row inside every block at once (Alg. 1, Alg. 4).

def vr_images(images: np.ndarray, slots: int, Hb: int, Wb: int) -> np.ndarray:
    """images [B][h][w] -> slot vectors [n_ct][slots] (slots // (Hb Wb) images per ciphertext)."""
    B, h, w = images.shape
    per = slots // (Hb * Wb)
    if per < 1 or h > Hb or w > Wb:
        raise ValueError("images do not fit the blocks")
    n_ct = -(-B // per)
    z = np.zeros((n_ct, slots))
    for b in range(B):
        base = (b % per) * Hb * Wb
        for r in range(h):
            z[b // per, base + r * Wb: base + r * Wb + w] = images[b, r]
    return z


def vr_images_from(z: np.ndarray, B: int, h: int, w: int, Hb: int, Wb: int) -> np.ndarray:
    """slot vectors [n_ct][slots] -> [B][h][w] (the top-left h x w of every block)."""
    per = z.shape[-1] // (Hb * Wb)
    out = np.zeros((B, h, w))
    for b in range(B):
        base = (b % per) * Hb * Wb
        for r in range(h):
            out[b, r] = z[b // per, base + r * Wb: base + r * Wb + w]
    return out


def _blocks(mat: np.ndarray, slots: int, Hb: int, Wb: int) -> np.ndarray:
    """an h x w matrix replicated into every block -> slot vector"""
    h, w = mat.shape
    v = np.zeros(slots)
    for b in range(slots // (Hb * Wb)):
        for r in range(h):
            v[b * Hb * Wb + r * Wb: b * Hb * Wb + r * Wb + w] = mat[r]
    return v


def vr_kernelspanner(K: np.ndarray, h: int, w: int, slots: int, Hb: int, Wb: int) -> np.ndarray:
    """Kernelspanner (Sec. III-C) in every block: [k*k][slots], offset (r, c) at index r k + c."""
    from .slot_sim import kernelspanner
    P = kernelspanner(K, h, w)
    k = K.shape[0]
    return np.stack([_blocks(P[(r, c)], slots, Hb, Wb) for r in range(k) for c in range(k)])


def vr_masks(k: int, h: int, w: int, slots: int, Hb: int, Wb: int) -> np.ndarray:
    """Alg. 4's offset masks in every block: [k*k][slots], offset (r, c) at index r k + c."""
    from .slot_sim import offset_mask
    return np.stack([_blocks(offset_mask(h, w, k, r, c).reshape(h, w), slots, Hb, Wb)
                     for r in range(k) for c in range(k)])


def vr_bias(k0: float, k: int, h: int, w: int, slots: int, Hb: int, Wb: int) -> np.ndarray:
    """Alg. 4's initial accumulator: k0 at every valid output position of every block."""
    from .slot_sim import bias_block
    return _blocks(bias_block(k0, h, w, k), slots, Hb, Wb)


def vr_matrix_a(A: np.ndarray, slots: int) -> np.ndarray:
    """tau_a (Sec. III-A): A [m][n] row-major, slot i n + j = A[i][j]."""
    m, n = A.shape
    z = np.zeros(slots)
    z[: m * n] = A.reshape(-1)
    return z


def vr_matrix_b(Bm: np.ndarray, slots: int) -> np.ndarray:
    """tau_b (Sec. III-A) over the whole ring: B transposed and tiled by rows with period p,
    slot i n + j = B[j][i mod p] for every row i < slots / n (whole-ring tiling, so that Rot by
    idx n is RowShifter applied idx times)."""
    n, p = Bm.shape
    rows = slots // n
    if slots % n or rows % p:
        raise ValueError("n must divide the slots and p the row count")
    return np.stack([Bm[:, i % p] for i in range(rows)]).reshape(-1)


def vr_matmul_masks(m: int, n: int, p: int, slots: int) -> np.ndarray:
    """Alg. 3's plaintexts: [0] the column-0 mask of SumColVec (1 at slots i n, i < m), then for
    idx < p the mask F_idx keeping slot i n + ((i + idx) mod p), i < m -> [1 + p][slots]."""
    out = np.zeros((1 + p, slots))
    out[0, np.arange(m) * n] = 1.0
    for idx in range(p):
        out[1 + idx, np.arange(m) * n + (np.arange(m) + idx) % p] = 1.0
    return out


def vr_matmul_from(z: np.ndarray, m: int, n: int, p: int) -> np.ndarray:
    """Alg. 3's result slot vector -> C [m][p] (C[i][c] at slot i n + c)."""
    return np.stack([z[i * n: i * n + p] for i in range(m)])


def vrot_masks(n: int, hw: int, r: int, slots: int) -> np.ndarray:
    """Alg. 5's masks for virtual ciphertexts held as rows of n slots (image of hw <= n values at
    the start of each row): F1 keeps row positions j < hw - r, F2 keeps hw - r <= j < hw -> [2][slots]."""
    F = np.zeros((2, slots))
    for row in range(slots // n):
        F[0, row * n: row * n + hw - r] = 1.0
        F[1, row * n + hw - r: row * n + hw] = 1.0
    return F


def vrot_slots(v: np.ndarray, n: int, hw: int, r: int) -> np.ndarray:
    """What vRot computes: every row's first hw entries rotated left by r, the rest 0."""
    out = np.zeros_like(v)
    for row in range(v.shape[-1] // n):
        seg = v[..., row * n: row * n + hw]
        out[..., row * n: row * n + hw] = np.roll(seg, -r, axis=-1)
    return out
