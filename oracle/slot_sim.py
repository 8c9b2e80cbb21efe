"""Plaintext slot simulator of the paper's slot-level algorithms.

TEST INFRASTRUCTURE. Each ciphertext is modelled by its slot vector; Rot(v, l)
is the cyclic left shift of Sec. II-A; Add / Mul / cMul are slotwise. This lets
the paper's worked examples and the readings taken where its text is garbled
be checked without encryption:

* SumForConv (Alg. 1) with the row pass applied to the column-summed vector
  (a separable k x k box sum), then the valid-position mask of its example,
* Kernelspanner (Sec. III-C, the 4x4, k = 2 example): the kernel tiled from
  offset (r, c) at every position where a whole copy fits, and the bias block,
* homomorphic convolution (Alg. 4) built from the two, with the offset mask
  (hth - r) mod k = 0, (wth - c) mod k = 0, hth + k <= h, wth + k <= w,
* the multi-ciphertext matmul of Alg. 3 over n ciphertexts per operand
  (D_idx = sum_k A_k * Rot(B~_k, idx)), and the column-layout convolution.
"""
from __future__ import annotations

import numpy as np


def rot(v: np.ndarray, l: int) -> np.ndarray:
    """Rot(ct, l): cyclic left rotation by l slots (Sec. II-A)."""
    return np.roll(v, -l)


def sum_for_conv(v: np.ndarray, h: int, w: int, k: int, separable: bool = True) -> np.ndarray:
    """Alg. 1 without the bias/mask: k x k window sums of a row-major h x w vector.

    separable=True is the reading used throughout (row pass on the
    column-summed vector); separable=False is the literal text, which rotates
    the input in the row pass and gives a cross, not a box.
    """
    acc = np.zeros_like(v)
    for pos in range(k):
        acc = acc + rot(v, pos)
    src = acc if separable else v
    out = acc.copy()
    for pos in range(1, k):
        out = out + rot(src, pos * w)
    return out


def valid_mask(h: int, w: int, k: int) -> np.ndarray:
    """1 where a whole k x k window fits (the positions kept in Alg. 1's example)."""
    m = np.zeros((h, w))
    m[: h - k + 1, : w - k + 1] = 1
    return m.reshape(-1)


def kernelspanner(K: np.ndarray, h: int, w: int) -> dict:
    """Offset (r, c) -> h x w matrix with K tiled from (r, c) where a copy fits."""
    k = K.shape[0]
    out = {}
    for r in range(k):
        for c in range(k):
            P = np.zeros((h, w))
            for top in range(r, h - k + 1, k):
                for left in range(c, w - k + 1, k):
                    P[top:top + k, left:left + k] = K
            out[(r, c)] = P
    return out


def bias_block(k0: float, h: int, w: int, k: int) -> np.ndarray:
    B = np.zeros((h, w))
    B[: h - k + 1, : w - k + 1] = k0
    return B


def offset_mask(h: int, w: int, k: int, r: int, c: int) -> np.ndarray:
    F = np.zeros((h, w))
    for hth in range(h):
        for wth in range(w):
            if (hth - r) % k == 0 and (wth - c) % k == 0 and hth + k <= h and wth + k <= w:
                F[hth, wth] = 1
    return F.reshape(-1)


def conv_alg4(I: np.ndarray, K: np.ndarray, k0: float) -> np.ndarray:
    """Alg. 4 on one image in one slot vector; returns the h x w result matrix."""
    h, w = I.shape
    k = K.shape[0]
    v = I.reshape(-1)
    acc = bias_block(k0, h, w, k).reshape(-1)
    for (r, c), P in kernelspanner(K, h, w).items():
        t = v * P.reshape(-1)
        t = sum_for_conv(t, h, w, k)
        acc = acc + t * offset_mask(h, w, k, r, c)
    return acc.reshape(h, w)


def matmul_multi_ct(A: np.ndarray, Bm: np.ndarray, slots: int) -> np.ndarray:
    """The n-ciphertext matmul on slot vectors; returns the p diagonal vectors."""
    m, n = A.shape
    _, p = Bm.shape
    Acols = np.zeros((n, slots))
    Acols[:, :m] = A.T
    Brows = np.tile(Bm, (1, slots // p))
    D = np.zeros((p, slots))
    for idx in range(p):
        for k in range(n):
            D[idx] += Acols[k] * rot(Brows[k], idx)
    return D


def conv_columns(images: np.ndarray, K: np.ndarray, bias, stride: int, slots: int, H: int, gap: int = 1):
    """Column-layout convolution on slot vectors.

    images [B][C][h][w] -> output slot vectors [O][w'][slots] with row gap
    gap * stride.
    """
    Bn, C, h, w = images.shape
    O, _, k, _ = K.shape
    X = np.zeros((C, w, slots))
    for b in range(Bn):
        for i in range(h):
            X[:, :, b * H + gap * i] = images[b, :, i, :]
    wo = (w - k) // stride + 1
    Y = np.zeros((O, wo, slots))
    for o in range(O):
        for jp in range(wo):
            for c in range(C):
                for b in range(k):
                    for a in range(k):
                        Y[o, jp] += K[o, c, a, b] * rot(X[c, stride * jp + b], gap * a)
            if bias is not None:
                Y[o, jp] += bias[o]
    return Y
