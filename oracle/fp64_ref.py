"""FP64 plaintext references: what the encrypted layers must decrypt to.

TEST INFRASTRUCTURE. The definitions the paper gives for the layers:

* matrix product C = A B, C[i][j] = sum_k A[i][k] B[k][j] (Sec. III-A),
* convolution, valid (no padding), no kernel flip (Sec. II-C):
  out[i'][j'] = k_0 + sum_{a,b < k} K[a][b] I[s i' + a][s j' + b], extended to
  channels by summing over input channels (Sec. IV-B) and to stride s,
* square activation x -> x^2, and the dense layer out = W flatten(x) + b with
  flatten in (channel, row, column) order.
"""
from __future__ import annotations

import numpy as np


def matmul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    return A @ B


def conv2d(x: np.ndarray, K: np.ndarray, bias, stride: int) -> np.ndarray:
    """x [B][C][h][w], K [O][C][k][k], bias [O] or None -> [B][O][h'][w']."""
    Bn, C, h, w = x.shape
    O, C2, k, _ = K.shape
    assert C == C2
    ho = (h - k) // stride + 1
    wo = (w - k) // stride + 1
    out = np.zeros((Bn, O, ho, wo))
    for a in range(k):
        for b in range(k):
            patch = x[:, :, a:a + stride * (ho - 1) + 1:stride, b:b + stride * (wo - 1) + 1:stride]
            out += np.einsum("bchw,oc->bohw", patch, K[:, :, a, b])
    if bias is not None:
        out += np.asarray(bias)[None, :, None, None]
    return out


def dense(x: np.ndarray, W: np.ndarray, bias) -> np.ndarray:
    """x [B][...] flattened per image, W [out][features] -> [B][out]."""
    y = x.reshape(x.shape[0], -1) @ W.T
    if bias is not None:
        y = y + np.asarray(bias)[None, :]
    return y


def cnn(images: np.ndarray, wts) -> np.ndarray:
    """conv 5x5 s2 -> x^2 -> conv 3x3 s2 -> x^2 -> dense, images [B][h][w] -> [B][10]."""
    x = images[:, None, :, :]
    x = conv2d(x, wts.conv1_w, wts.conv1_b, 2) ** 2
    x = conv2d(x, wts.conv2_w, wts.conv2_b, 2) ** 2
    return dense(x, wts.fc_w, wts.fc_b)
