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


def table1_cnn(images: np.ndarray, wts, act1, act2) -> np.ndarray:
    """Table I's CNN in FP64 on images [B][h][w]: CONV (wts.conv_w [c][k][k] + bias, stride 1,
    valid), ACT-1, FC-1 over the (channel, row, column)-ordered features, ACT-2, FC-2 -> logits
    [B][fc2_out]; act1, act2 the coefficients of x^0 .. x^3."""
    c, k = wts.conv_w.shape[0], wts.conv_w.shape[1]
    y = conv2d(images[:, None], wts.conv_w[:, None], wts.conv_b, 1)  # [B][c][ho][wo]
    act = lambda v, a: a[0] + a[1] * v + a[2] * v ** 2 + a[3] * v ** 3  # noqa: E731
    y = act(y, act1)
    z = act(y.reshape(y.shape[0], -1) @ wts.fc1_w.reshape(-1, wts.fc1_w.shape[-1]) + wts.fc1_b, act2)
    return z @ wts.fc2_w + wts.fc2_b
