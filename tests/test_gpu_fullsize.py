"""Parity at the workloads' full sizes, in the launch configuration bench.py uses.

The CUDA path runs the whole layer / network; the oracle computes a sample of
the output ciphertexts one by one (the first and the last output column of
every channel, so the ragged last column is covered) from the same integer
plaintexts and seed, and they are compared bit for bit. The full decrypted
outputs are checked against the FP64 closed forms.
"""
from __future__ import annotations

import numpy as np
import pytest

from inputs import synthetic
from oracle import Oracle, fp64_ref, layouts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_18646_gb300 as pkg
    pkg.load()
    return pkg


def _columns(o, imgs, H):
    """Oracle-encoded integer plaintexts of the image columns (block stride H)."""
    z = layouts.image_columns(imgs, o.slots, H)
    return np.stack([o.encode(v) for v in z])


def test_conv_layer_n15_64x64(lib):
    """One conv layer: 64x64 image, 4 kernels 3x3 stride 1, x^2; N = 2^15, 1 special + 8 x 40 + 60-bit primes."""
    from paper_2512_18646_gb300 import api
    pre = synthetic.CONV_LAYER
    o = Oracle.from_preset(pre, seed=201)
    g = api.Context.from_preset(pre, seed=201)
    o.keygen([1, 2])
    g.keygen([1, 2])
    img = synthetic.images(1, 64, 64, seed=201)
    K, bias = synthetic.conv_weights(4, 1, 3, 0.1, seed=202)
    H = 64
    m = _columns(o, img, H)
    gx = g.encrypt_coeffs(m, o.L1, o.scale, 0)
    gy = g.conv2d(gx, 1, 1, K, bias, 1)
    g.square(gy)  # three components (relinearisation deferred)
    got = gy.export().reshape(4, 62, 3, o.L1 - 2, o.N)
    # oracle: output columns 0 and 61 of every channel
    cols = [0, 1, 2, 59, 60, 61, 62, 63]
    X = np.zeros((1, 64, 2, o.L1, o.N), np.uint64)
    for j in cols:
        X[0, j] = o.encrypt(m[j], o.L1, j)
    sel = [(c, jp) for c in range(4) for jp in (0, 61)]
    oy = o.square(o.conv2d(X, 1, K, bias, 1, o.scale, sel=sel))
    for t, (c, jp) in enumerate(sel):
        assert np.array_equal(got[c, jp], oy[t]), (c, jp)
    # FP64 over the whole layer
    ref = fp64_ref.conv2d(img[:, None], K, bias, 1) ** 2          # [1][4][62][62]
    dec = g.decrypt_image(gy, 1, H, 1, 62)[0].reshape(4, 62, 62)  # [ch][col][row]
    assert np.abs(dec.transpose(0, 2, 1) - ref[0]).max() < 1e-4


def test_cnn_n16_128x128(lib):
    """The CNN of bench.py at N = 2^16 on 256 images: conv-1 outputs sampled bit for bit, logits vs FP64."""
    from paper_2512_18646_gb300 import api
    pre = synthetic.CNN_N16
    B, side, H = 256, 128, 128
    o = Oracle.from_preset(pre, seed=301)
    g = api.Context.from_preset(pre, seed=301)
    o.keygen([1, 2, 3, 4])
    g.keygen([1, 2, 3, 4, 8, 16, 32, 64])
    imgs = synthetic.images(B, side, side, seed=301)
    w = synthetic.cnn_weights(side, seed=302)
    m = _columns(o, imgs, H)
    gx = g.encrypt_coeffs(m, o.L1, o.scale, 0)
    gy = g.conv2d(gx, 1, 1, w.conv1_w, w.conv1_b, 2)
    got = gy.export().reshape(8, 62, 2, o.L1 - 1, o.N)
    # oracle: conv-1 output columns 0 and 61 (inputs 0..4 and 122..126)
    X = np.zeros((1, 128, 2, o.L1, o.N), np.uint64)
    for j in list(range(5)) + list(range(122, 127)):
        X[0, j] = o.encrypt(m[j], o.L1, j)
    sel = [(c, jp) for c in range(8) for jp in (0, 61)]
    oy = o.conv2d(X, 1, w.conv1_w, w.conv1_b, 2, o.scale, sel=sel)
    for t, (c, jp) in enumerate(sel):
        assert np.array_equal(got[c, jp], oy[t]), (c, jp)
    # the rest of the network on the GPU, logits against the FP64 CNN
    g.square(gy)
    y = g.conv2d(gy, 8, 2, w.conv2_w, w.conv2_b, 2)
    g.square(y)
    _, h2 = synthetic.cnn_shapes(side)
    pts = g.fc_prepare(w.fc_w, 16, h2, h2, 4, H, B, y.limbs)
    z = g.fc_apply(y, pts, w.fc_b)
    logits = layouts.logits_from_fc(g.decrypt_slots(z), B, H)
    ref = fp64_ref.cnn(imgs, w)
    assert np.abs(logits - ref).max() < 1e-4
