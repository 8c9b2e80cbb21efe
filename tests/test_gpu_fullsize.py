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
    """The CNN of bench.py at N = 2^16 on 256 images: conv-1 and conv-2 outputs sampled bit for bit
    (the oracle computes the conv-1 columns that conv-2 needs itself), logits vs FP64.

    Conv-2 (8 input channels, 3x3: 72 terms per output) takes the 96-bit multiply-accumulate's
    mid-sum reduction and its second pass of 8 output channels at the full size."""
    from paper_2512_18646_gb300 import api
    pre = synthetic.CNN_N16
    B, side, H = 256, 128, 128
    h1, h2 = synthetic.cnn_shapes(side)
    o = Oracle.from_preset(pre, seed=301)
    g = api.Context.from_preset(pre, seed=301)
    o.keygen([1, 2, 3, 4])
    g.keygen([1, 2, 3, 4, 8, 16, 32, 64])
    imgs = synthetic.images(B, side, side, seed=301)
    w = synthetic.cnn_weights(side, seed=302)
    m = _columns(o, imgs, H)
    gx = g.encrypt_coeffs(m, o.L1, o.scale, 0)
    gy = g.conv2d(gx, 1, 1, w.conv1_w, w.conv1_b, 2)
    # conv-2's first and last output column (jp2 = 0 and h2 - 1) read conv-1 output columns
    # 2 jp2 + b (b < 3) of every channel, which read input columns 4 jp2 .. 4 jp2 + 8
    wins = (0, h2 - 1)
    got1 = {(jp2, c, b): gy.slice(c * h1 + 2 * jp2 + b, 1).export()[0]
            for jp2 in wins for c in range(8) for b in range(3)}
    g.square(gy)
    sc = o.scale * o.scale / o.q[o.L1 - 2]
    assert gy.scale == sc
    y = g.conv2d(gy, 8, 2, w.conv2_w, w.conv2_b, 2)
    # the oracle from its own encryptions of each 9-column input window (the convolution is the same
    # at every column offset, so a window's outputs are output columns 0..2 / 0 of the window)
    for jp2 in wins:
        X = np.stack([o.encrypt(m[j], o.L1, j) for j in range(4 * jp2, 4 * jp2 + 9)])[None]
        sel = [(c, b) for c in range(8) for b in range(3)]
        oy = o.conv2d(X, 1, w.conv1_w, w.conv1_b, 2, o.scale, sel=sel)
        for t, (c, b) in enumerate(sel):
            assert np.array_equal(got1[(jp2, c, b)], oy[t]), ("conv-1", jp2, c, b)
        X2 = o.square(oy).reshape(8, 3, 3, o.L1 - 2, o.N)
        oy2 = o.conv2d(X2, 2, w.conv2_w, w.conv2_b, 2, sc, sel=[(c, 0) for c in range(16)])
        for c in range(16):
            got = y.slice(c * h2 + jp2, 1).export()[0]
            assert np.array_equal(got, oy2[c]), ("conv-2", c, jp2)
        del X, oy, X2, oy2
    del got1
    # the rest of the network on the GPU, logits against the FP64 CNN
    g.square(y)
    pts = g.fc_prepare(w.fc_w, 16, h2, h2, 4, H, B, y.limbs)
    z = g.fc_apply(y, pts, w.fc_b)
    logits = layouts.logits_from_fc(g.decrypt_slots(z), B, H)
    ref = fp64_ref.cnn(imgs, w)
    assert np.abs(logits - ref).max() < 1e-4


def test_fc_n16_480_columns(lib):
    """The CNN's dense layer at its full size and level (N = 2^16, 9 limbs, 16 x 30 = 480 input
    ciphertexts, rows at gap 4 in blocks of 128, 10 outputs) on seeded random residues and random
    plaintexts: outputs 0 and 9 (the first and the second pass over outputs) bit for bit against the
    oracle. 480 columns reduce the 96-bit sums of the 45-bit limbs several times per output."""
    from paper_2512_18646_gb300 import api
    pre = synthetic.CNN_N16
    c_in, w_in, gap, H, out_dim, lp = 16, 30, 4, 128, 10, 9
    o = Oracle.from_preset(pre, seed=303)
    g = api.Context.from_preset(pre, seed=303)
    steps = [4, 8, 16, 32, 64]
    o.keygen(steps)
    g.keygen(steps)
    rng = np.random.default_rng(303)
    X = np.empty((c_in * w_in, 2, lp, o.N), np.uint64)
    for i in range(lp):
        X[:, :, i, :] = rng.integers(0, o.primes[i], (c_in * w_in, 2, o.N), dtype=np.uint64)
    pts = rng.integers(-(1 << 62), 1 << 62, (out_dim, c_in, w_in, o.N), dtype=np.int64)
    bias = rng.normal(0, 0.05, out_dim)
    gz = g.fc_apply(g.import_coeffs(X, o.scale), g.fc_prepare_coeffs(pts, gap, H, lp), bias)
    sel = [0, out_dim - 1]
    oz = o.fc(X.reshape(c_in, w_in, 2, lp, o.N), gap, H, pts[sel], bias, o.scale, sel)
    got = gz.export()
    for t, oi in enumerate(sel):
        assert np.array_equal(got[oi], oz[t]), oi


def test_conv_layer_encrypted_kernels_n15_64x64(lib):
    """The conv layer with the model provider's encrypted kernels at N = 2^15: sampled output columns bit
    for bit against the oracle (same kernel plaintexts and seeds), the whole layer against FP64."""
    from paper_2512_18646_gb300 import api
    pre = synthetic.CONV_LAYER
    o = Oracle.from_preset(pre, seed=203)
    g = api.Context.from_preset(pre, seed=203)
    o.keygen([1, 2])
    g.keygen([1, 2])
    img = synthetic.images(1, 64, 64, seed=201)
    K, bias = synthetic.conv_weights(4, 1, 3, 0.1, seed=202)
    H = 64
    m = _columns(o, img, H)
    gx = g.encrypt_coeffs(m, o.L1, o.scale, 0)
    gw = g.encrypt_conv_weights(K, o.L1, 9000)
    gy = g.conv2d_enc(gx, 1, 1, gw, bias, 4, 3, 1)
    got = gy.export().reshape(4, 62, 2, o.L1 - 1, o.N)
    cols = [0, 1, 2, 61, 62, 63]
    X = np.zeros((1, 64, 2, o.L1, o.N), np.uint64)
    for j in cols:
        X[0, j] = o.encrypt(m[j], o.L1, j)
    mw = o.conv_weight_plaintexts(K, o.L1)
    ow = np.stack([o.encrypt(mw[i], o.L1, 9000 + i) for i in range(len(mw))])
    sel = [(c, jp) for c in range(4) for jp in (0, 61)]
    oy = o.conv2d_enc(X, 1, ow, bias, 4, 3, 1, o.scale, sel=sel)
    for t, (c, jp) in enumerate(sel):
        assert np.array_equal(got[c, jp], oy[t]), (c, jp)
    ref = fp64_ref.conv2d(img[:, None], K, bias, 1)
    dec = g.decrypt_image(gy, 1, H, 1, 62)[0].reshape(4, 62, 62)
    assert np.abs(dec.transpose(0, 2, 1) - ref[0]).max() < 1e-4


def test_matmul_volley_and_act3_n16(lib):
    """At the CNN parameters (N = 2^16, 13 limbs): a zero-rotation matmul of the batched workload's
    largest shape class (m = p = 256, three groups) bit for bit against the oracle and within 1e-4 of
    FP64, then Table I's ACT-1 on its outputs bit for bit."""
    from paper_2512_18646_gb300 import api
    from tests.test_oracle_pins import act_polynomials
    pre = synthetic.CNN_N16
    o = Oracle.from_preset(pre, seed=411)
    g = api.Context.from_preset(pre, seed=411)
    o.keygen([])
    g.keygen([])
    m_, n_, p_ = 256, 8, 256
    A, Bm = synthetic.matmul_operands(m_, n_, p_, seed=412)
    M, per, G, _ = layouts.volley_geometry(o.slots, m_, p_)
    assert G == 3
    ma = np.stack([o.encode(v) for v in layouts.matrix_a_volley(A, o.slots, p_).reshape(G * n_, o.slots)])
    mb = np.stack([o.encode(v) for v in layouts.matrix_b_rows(Bm, o.slots)])
    ga = g.encrypt_coeffs(ma, o.L1, o.scale, 0)
    gb = g.encrypt_coeffs(mb, o.L1, o.scale, 100)
    oa = np.stack([o.encrypt(ma[i], o.L1, i) for i in range(len(ma))]).reshape(G, n_, 2, o.L1, o.N)
    ob = np.stack([o.encrypt(mb[i], o.L1, 100 + i) for i in range(n_)])
    gd = g.matmul_volley(ga, gb)
    od = o.matmul_volley(oa, ob)
    assert np.array_equal(gd.export(), od)
    assert np.abs(g.decrypt_matrix_volley(gd, m_, p_) - A @ Bm).max() < 1e-4
    sd = o.scale * o.scale / o.q[o.L1 - 1]
    assert gd.scale == sd
    c = act_polynomials()["ACT-1"]
    gy = g.poly_act(gd, c)
    oy, sy = o.poly_act3(od, c, sd)
    assert np.array_equal(gy.export(), oy) and gy.scale == sy
