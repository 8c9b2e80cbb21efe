"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Ciphertexts are compared limb by limb, bit for bit, in the coefficient domain:
both sides start from the same integer plaintexts and the same seeded
randomness (inputs/he_random.h) and follow the same canonical schedules.
Decrypted results are also checked against FP64 closed forms. Sizes span
several NTT tiles and ragged counts (sets not a multiple of any chunk).
"""
from __future__ import annotations

import numpy as np
import pytest

from inputs import synthetic
from oracle import Oracle, fp64_ref, layouts
from tests.gpu_pairs import encode_columns, encrypt_both, image_columns_both, make_pair, pair_from_preset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_18646_gb300 as pkg
    pkg.load()
    return pkg


# ---------------------------------------------------------------------------
# transform and encryption
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log_n", [4, 5, 10, 13, 16])
def test_ntt_matches_oracle(lib, log_n):
    o, g = make_pair(log_n, (60, 40, 45), 2, 60, 1, 40.0, steps=None)
    rng = np.random.default_rng(log_n)
    a = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.primes])[None]  # [1][np][N]
    fwd = g.ntt(a, 0)
    for pi in range(len(o.primes)):
        assert np.array_equal(fwd[0, pi], o.ntt(a[0, pi], pi)), pi
    assert np.array_equal(g.ntt(fwd, 0, inverse=True), a)
    # several polynomials per launch, a prime offset
    b = np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.primes[1:3]]) for _ in range(3)])
    fb = g.ntt(b, 1)
    for t in range(3):
        for i in range(2):
            assert np.array_equal(fb[t, i], o.ntt(b[t, i], 1 + i))


@pytest.mark.parametrize("log_n", [10, 13, 15, 16])
def test_ntt_every_geometry_matches_oracle(lib, log_n):
    """Every transform geometry the autotuner may pick (column stages n1, columns per block) computes
    the oracle's transform bit for bit, forward and inverse; the autotuner returns one of them."""
    from paper_2512_18646_gb300._lib import HeError
    o, g = make_pair(log_n, (60, 40, 45), 2, 60, 1, 40.0, steps=None)
    rng = np.random.default_rng(100 + log_n)
    a = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.primes])[None]
    want = np.stack([o.ntt(a[0, pi], pi) for pi in range(len(o.primes))])
    tried = 0
    for n1 in range(2, 9):
        for cols in (4, 8, 16, 32):
            try:
                g.ntt_set_geometry(n1, cols)
            except HeError:
                continue
            tried += 1
            fwd = g.ntt(a, 0)
            assert np.array_equal(fwd[0], want), (n1, cols)
            assert np.array_equal(g.ntt(fwd, 0, inverse=True), a), (n1, cols)
    assert tried >= 2
    n1, cols, us = g.ntt_autotune(64)
    assert us > 0
    g.ntt_set_geometry(n1, cols)  # the tuned choice is a supported geometry
    assert np.array_equal(g.ntt(a, 0)[0], want)
    g.ntt_set_geometry(0, 0)


def test_encrypt_matches_oracle(lib):
    o, g = make_pair(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=3, steps=[])
    z = np.random.default_rng(1).uniform(-1, 1, (5, o.slots))
    m = encode_columns(o, z)
    for limbs in (4, 2, 1):
        oc, gc = encrypt_both(o, g, m, limbs, ct_id_base=100 + limbs)
        assert np.array_equal(gc.export(), oc)
    # decryption on the device reads the same message
    d = g.decrypt_slots(gc)
    assert np.abs(d - z).max() < 1e-6


def test_encoder_matches_oracle_encoder(lib):
    o, g = make_pair(12, (60, 40), 1, 60, 1, 40.0, steps=[])
    A = np.random.default_rng(2).uniform(-1, 1, (6, 9))
    gc = g.encrypt_matrix_a(A, 7)
    z = layouts.matrix_a_columns(A, o.slots)
    m = encode_columns(o, z)
    oc = np.stack([o.encrypt(m[i], o.L1, 7 + i) for i in range(9)])
    ge = gc.export()
    # independent encoders may round a coefficient differently by one unit;
    # the difference of the two ciphertexts is then that small plaintext
    diff = o.decrypt_coeffs(ge[0]) - o.decrypt_coeffs(oc[0])
    assert np.abs(diff).max() <= 1
    assert np.abs(g.decrypt_slots(gc)[:, :6] - A.T).max() < 1e-6


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("params", [
    (10, (60, 40, 40, 40), 1, 60, 1, 40.0),          # one special prime, digits of one prime
    (11, (60, 45, 45, 45, 45, 45), 2, 60, 2, 45.0),   # CNN shape: two specials, digits of two
])
def test_rotation_matches_oracle(lib, params):
    steps = [0, 1, 3, 5, -2, 17]
    o, g = make_pair(*params, seed=5, steps=[s for s in steps if s])
    z = np.random.default_rng(3).uniform(-1, 1, (3, o.slots))
    m = encode_columns(o, z)
    for limbs in (o.L1, 2):
        oc, gc = encrypt_both(o, g, m, limbs, ct_id_base=30)
        r = g.rotate(gc, steps).export().reshape(3, len(steps), 2, limbs, o.N)
        for c in range(3):
            ref = o.rotate(oc[c], steps)
            for t in range(len(steps)):
                assert np.array_equal(r[c, t], ref[t]), (limbs, c, steps[t])
    dz = g.decrypt_slots(g.rotate(gc, [1]))
    assert np.abs(dz - np.roll(z, -1, axis=1)).max() < 1e-5


def test_mul_rescale_relin_matches_oracle(lib):
    o, g = make_pair(11, (60, 45, 45, 45, 45), 2, 60, 2, 45.0, seed=6, steps=[])
    rng = np.random.default_rng(4)
    x, y = rng.uniform(-1, 1, (4, o.slots)), rng.uniform(-1, 1, (4, o.slots))
    ox, gx = encrypt_both(o, g, encode_columns(o, x), ct_id_base=0)
    oy, gy = encrypt_both(o, g, encode_columns(o, y), ct_id_base=10)
    gm = g.mul(gx, gy)
    assert gm.polys == 3  # Mul = tensor + rescale; relinearisation is deferred
    m3 = gm.export()
    for c in range(4):
        assert np.array_equal(m3[c], o.rescale(o.tensor(ox[c], oy[c])))
    g.relinearize(gm)
    m2 = gm.export()
    for c in range(4):
        assert np.array_equal(m2[c], o.relin(o.rescale(o.tensor(ox[c], oy[c]))))
    assert np.abs(g.decrypt_slots(gm) - x * y).max() < 1e-5
    sq = g.square(gx).export()
    for c in range(4):
        assert np.array_equal(sq[c], o.square(ox[c:c + 1])[0])


def test_rescale_matches_oracle_on_random_residues(lib):
    o, g = make_pair(10, (60, 40, 40, 40), 1, 60, 1, 40.0, steps=None)
    rng = np.random.default_rng(5)
    ct = np.stack([np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.q])
                             for _ in range(2)]) for _ in range(7)])
    gs = g.import_coeffs(ct, 2.0 ** 40)
    assert np.array_equal(gs.export(), ct)
    g.rescale(gs)
    out = gs.export()
    for c in range(7):
        assert np.array_equal(out[c], o.rescale(ct[c]))


# ---------------------------------------------------------------------------
# layers at small sizes: bit-exact and FP64
# ---------------------------------------------------------------------------
def test_matmul_small_config_matches_oracle_and_fp64(lib):
    """The 4x8 . 8x4 matmul at N = 2^13, Q = 60 + 40 + 40 bits, P = 60 bits."""
    pre = synthetic.MATMUL_SMALL
    o, g = pair_from_preset(pre, seed=101, steps=list(range(1, 4)))
    A, Bm = synthetic.matmul_operands(4, 8, 4, seed=101)
    oa, ga = encrypt_both(o, g, encode_columns(o, layouts.matrix_a_columns(A, o.slots)), ct_id_base=0)
    ob, gb = encrypt_both(o, g, encode_columns(o, layouts.matrix_b_rows(Bm, o.slots)), ct_id_base=100)
    gd = g.matmul(ga, gb, 4, 4)
    od = o.matmul(oa, ob, 4)
    assert np.array_equal(gd.export(), od)
    C = g.decrypt_matrix(gd, 4, 4)
    assert np.abs(C - A @ Bm).max() < 1e-4
    # the library's own encoders (he_encrypt_matrix_a/b) give the same product within tolerance
    C2 = g.decrypt_matrix(g.matmul(g.encrypt_matrix_a(A, 0), g.encrypt_matrix_b(Bm, 100), 4, 4), 4, 4)
    assert np.abs(C2 - A @ Bm).max() < 1e-4


@pytest.mark.parametrize("m,n,p", [(5, 3, 8), (16, 7, 1), (3, 1, 2)])
def test_matmul_ragged_shapes(lib, m, n, p):
    o, g = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=9, steps=list(range(1, max(p, 2))))
    rng = np.random.default_rng(m * 100 + n * 10 + p)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    oa, ga = encrypt_both(o, g, encode_columns(o, layouts.matrix_a_columns(A, o.slots)), ct_id_base=0)
    ob, gb = encrypt_both(o, g, encode_columns(o, layouts.matrix_b_rows(Bm, o.slots)), ct_id_base=50)
    gd = g.matmul(ga, gb, m, p)
    assert np.array_equal(gd.export(), o.matmul(oa, ob, p))
    assert np.abs(g.decrypt_matrix(gd, m, p) - A @ Bm).max() < 1e-5


@pytest.mark.parametrize("m,n,p,g", [(5, 3, 8, 4), (6, 2, 8, 3), (16, 5, 32, 0), (3, 2, 4, 4), (4, 3, 1, 0)])
def test_matmul_bsgs_matches_oracle_and_revolver(lib, m, n, p, g):
    """Baby-step giant-step revolver: bit-exact with the oracle's schedule, decrypting to A @ B and
    to the plain revolver's diagonals (g = 0 picks the power of two nearest sqrt(p))."""
    gg = g
    if g == 0:
        gg = 1
        while 4 * gg * gg <= 2 * p:
            gg *= 2
        gg = min(gg, p)
    o, gl = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=13, steps=None)
    S = o.slots
    ng = -(-p // gg)
    steps = sorted(set(list(range(1, max(p, 2))) + [S - gg * i for i in range(1, ng)]))
    o.keygen(steps)
    gl.keygen(steps)
    rng = np.random.default_rng(m * 11 + n + p)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    oa, ga = encrypt_both(o, gl, encode_columns(o, layouts.matrix_a_columns(A, S)), ct_id_base=0)
    ob, gb = encrypt_both(o, gl, encode_columns(o, layouts.matrix_b_rows(Bm, S)), ct_id_base=60)
    gd = gl.matmul_bsgs(ga, gb, m, p, g)
    assert np.array_equal(gd.export(), o.matmul_bsgs(oa, ob, p, gg))
    C = gl.decrypt_matrix(gd, m, p)
    assert np.abs(C - A @ Bm).max() < 1e-5
    assert np.abs(C - gl.decrypt_matrix(gl.matmul(ga, gb, m, p), m, p)).max() < 1e-5


@pytest.mark.parametrize("log_n,m,n,p", [(13, 4, 8, 4), (10, 20, 3, 32), (10, 1, 5, 2), (10, 16, 9, 1)])
def test_matmul_volley_matches_oracle_and_fp64(lib, log_n, m, n, p):
    """Zero-rotation matmul: bit-exact with the oracle from the same plaintexts, decrypts to
    A @ B; the (20, 3, 32) case splits the positions into several groups."""
    if log_n == 13:
        o, g = pair_from_preset(synthetic.MATMUL_SMALL, seed=101, steps=[])
        A, Bm = synthetic.matmul_operands(m, n, p, seed=101)
    else:
        o, g = make_pair(log_n, (60, 40, 40), 1, 60, 1, 40.0, seed=12, steps=[])
        rng = np.random.default_rng(m * 7 + n + p)
        A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    M, per, G, _ = layouts.volley_geometry(o.slots, m, p)
    if (m, p) == (20, 32):
        assert G == 3
    Ah = layouts.matrix_a_volley(A, o.slots, p).reshape(G * n, o.slots)
    oa, ga = encrypt_both(o, g, encode_columns(o, Ah), ct_id_base=0)
    ob, gb = encrypt_both(o, g, encode_columns(o, layouts.matrix_b_rows(Bm, o.slots)), ct_id_base=500)
    gd = g.matmul_volley(ga, gb)
    od = o.matmul_volley(oa.reshape(G, n, *oa.shape[1:]), ob)
    assert np.array_equal(gd.export(), od)
    assert np.abs(g.decrypt_matrix_volley(gd, m, p) - A @ Bm).max() < 1e-5
    # the library's own encoder of the volley layout
    C2 = g.decrypt_matrix_volley(g.matmul_volley(g.encrypt_matrix_a_volley(A, p, 0), g.encrypt_matrix_b(Bm, 500)),
                                 m, p)
    assert np.abs(C2 - A @ Bm).max() < 1e-5
    # the same product through the revolver path (rotations) decrypts to the same matrix
    if p > 1:
        g.keygen(list(range(1, p)))
        C3 = g.decrypt_matrix(g.matmul(g.encrypt_matrix_a(A, 0), g.encrypt_matrix_b(Bm, 500), m, p), m, p)
        assert np.abs(C3 - C2).max() < 1e-5


@pytest.mark.parametrize("stride,c_in,k,side", [(1, 1, 3, 9), (2, 3, 3, 11), (2, 1, 5, 13), (1, 2, 1, 6)])
def test_conv2d_matches_oracle_and_fp64(lib, stride, c_in, k, side):
    H = 16
    o, g = make_pair(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=7, steps=list(range(1, k)))
    rng = np.random.default_rng(stride * 10 + c_in)
    imgs = rng.uniform(0, 1, (3, c_in, side, side - 1))
    K = rng.normal(0, 0.3, (4, c_in, k, k))
    bias = rng.normal(0, 0.3, 4)
    ox, gx = image_columns_both(o, g, imgs, H, ct_id_base=1000)
    gy = g.conv2d(gx, c_in, 1, K, bias, stride)
    oy = o.conv2d(ox, 1, K, bias, stride, o.scale)
    assert np.array_equal(gy.export(), oy)
    ref = fp64_ref.conv2d(imgs, K, bias, stride)
    got = g.decrypt_image(gy, 3, H, stride, ref.shape[2])  # [B][o*w'][h']
    got = got.reshape(3, 4, ref.shape[3], ref.shape[2]).transpose(0, 1, 3, 2)
    assert np.abs(got - ref).max() < 1e-5


@pytest.mark.parametrize("c_out,polys", [(16, 2), (11, 3)])
def test_conv2d_96bit_sums_reduce_mid_sum_and_run_two_channel_passes(lib, c_out, polys):
    """The second convolution's shape with 45-bit working primes: c_in = 8, k = 3 gives 72 terms per
    output, more than the 63 products a 96-bit sum of 45-bit residues holds, so the multiply-
    accumulate reduces in the middle of each sum; 16 (and a ragged 11) output channels run as two
    passes of 8 over the same rotated inputs. Gap 2 and stride 2 as after a strided first layer;
    the three-component case is the square's unrelinearised output. Bit-exact with the oracle."""
    o, g = make_pair(10, (60,) + (45,) * 6, 2, 60, 2, 45.0, seed=41, steps=[2, 4])
    H, side, Bn, c_in, k, stride, gap = 32, 13, 3, 8, 3, 2, 2
    rng = np.random.default_rng(41 + c_out)
    imgs = rng.uniform(-1, 1, (Bn, c_in, side, side))
    K = rng.normal(0, 0.2, (c_out, c_in, k, k))
    bias = rng.normal(0, 0.2, c_out)
    z = np.concatenate([layouts.image_columns(imgs[:, c], o.slots, H, gap) for c in range(c_in)])
    ox, gx = encrypt_both(o, g, encode_columns(o, z), ct_id_base=2000)
    sc = o.scale
    if polys == 3:
        ox = o.square(ox)
        g.square(gx)
        sc = sc * sc / o.q[o.L1 - 1]
        assert gx.scale == sc and gx.polys == 3
    ox = ox.reshape(c_in, side, *ox.shape[1:])
    gy = g.conv2d(gx, c_in, gap, K, bias, stride)
    oy = o.conv2d(ox, gap, K, bias, stride, sc)
    assert oy.shape[0] == c_out * ((side - k) // stride + 1)
    assert np.array_equal(gy.export(), oy)
    x = imgs ** 2 if polys == 3 else imgs
    ref = fp64_ref.conv2d(x, K, bias, stride)
    got = g.decrypt_image(gy, Bn, H, gap * stride, ref.shape[2])
    got = got.reshape(Bn, c_out, ref.shape[3], ref.shape[2]).transpose(0, 1, 3, 2)
    assert np.abs(got - ref).max() < 1e-4


@pytest.mark.parametrize("c_in,k,stride,c_out,polys", [(8, 3, 2, 16, 3), (1, 5, 2, 8, 2), (2, 3, 1, 8, 2),
                                                        (8, 3, 2, 11, 2), (9, 3, 1, 4, 2), (10, 3, 2, 3, 2),
                                                        (2, 3, 1, 5, 2)])
def test_conv_tensor_cores_equal_cuda_cores_and_oracle(lib, c_in, k, stride, c_out, polys):
    """The convolution's multiply-accumulate on the tensor cores (residues cut into bytes (45-bit
    primes) or 7-bit chunks (60-bit primes) whose products the tensor cores sum exactly in fp32,
    recombined modulo q) and on the CUDA cores give the same words, bit-exact with the oracle:
    8, 16 and ragged channel counts, 72, 25 and 18 terms, 81 (the last term count the byte chunks
    take) and 90 (past it: the CUDA cores), a layer too small for the tensor path (5 channels of 18
    terms: the CUDA cores), two- and three-component inputs."""
    o, g = make_pair(10, (60,) + (45,) * 6, 2, 60, 2, 45.0, seed=47, steps=list(range(1, k)))
    H, side, Bn, gap = 32, 13, 3, 1
    rng = np.random.default_rng(47 + c_out + c_in)
    imgs = rng.uniform(-1, 1, (Bn, c_in, side, side))
    K = rng.normal(0, 0.2, (c_out, c_in, k, k))
    bias = rng.normal(0, 0.2, c_out)
    z = np.concatenate([layouts.image_columns(imgs[:, c], o.slots, H, gap) for c in range(c_in)])
    ox, gx = encrypt_both(o, g, encode_columns(o, z), ct_id_base=3000)
    sc = o.scale
    if polys == 3:
        ox = o.square(ox)
        g.square(gx)
        sc = sc * sc / o.q[o.L1 - 1]
    ox = ox.reshape(c_in, side, *ox.shape[1:])
    got = {}
    for tc in (True, False):
        g.set_tensor_cores(tc)
        got[tc] = g.conv2d(gx, c_in, gap, K, bias, stride).export()
    g.set_tensor_cores(True)
    assert np.array_equal(got[True], got[False])
    assert np.array_equal(got[True], o.conv2d(ox, gap, K, bias, stride, sc))


def test_three_digits_and_five_special_primes_match_oracle(lib):
    """The CNN's prime chain with dnum = 3 (digits of five primes) and five 60-bit special primes:
    hoisted rotations, the square with its deferred relinearisation and a strided convolution over
    it, bit-exact with the oracle, and decrypting to the FP64 convolution."""
    o, g = make_pair(10, (60,) + (45,) * 12, 5, 60, 5, 45.0, seed=51, steps=[1, 2, 3])
    assert len(o.primes) == 18
    H, side, Bn, c_in, k, c_out = 32, 11, 3, 2, 3, 4
    rng = np.random.default_rng(51)
    imgs = rng.uniform(-1, 1, (Bn, c_in, side, side))
    z = np.concatenate([layouts.image_columns(imgs[:, c], o.slots, H) for c in range(c_in)])
    ox, gx = encrypt_both(o, g, encode_columns(o, z), ct_id_base=0)
    r = g.rotate(gx.slice(0, 2), [1, 3]).export().reshape(2, 2, 2, o.L1, o.N)
    for c in range(2):
        want = o.rotate(ox[c], [1, 3])
        assert np.array_equal(r[c], want), c
    K = rng.normal(0, 0.2, (c_out, c_in, k, k))
    bias = rng.normal(0, 0.2, c_out)
    g.square(gx)
    sq = o.square(ox)
    sc = o.scale * o.scale / o.q[o.L1 - 1]
    gy = g.conv2d(gx, c_in, 1, K, bias, 2)
    oy = o.conv2d(sq.reshape(c_in, side, *sq.shape[1:]), 1, K, bias, 2, sc)
    assert np.array_equal(gy.export(), oy)
    ref = fp64_ref.conv2d(imgs ** 2, K, bias, 2)
    got = g.decrypt_image(gy, Bn, H, 2, ref.shape[2])
    got = got.reshape(Bn, c_out, ref.shape[3], ref.shape[2]).transpose(0, 1, 3, 2)
    assert np.abs(got - ref).max() < 1e-4


def test_fc_96bit_sums_over_480_columns(lib):
    """The dense layer's shape (16 channels x 30 columns = 480 input ciphertexts, rows at gap 4 in
    blocks of 128) with 45-bit working primes: the 96-bit sums are reduced every ~63 columns, several
    times per output, and the 10 outputs run as two passes. Bit-exact with the oracle, FP64 within 1e-4."""
    o, g = make_pair(10, (60,) + (45,) * 4, 2, 60, 2, 45.0, seed=43, steps=[4, 8, 16, 32, 64])
    c_in, hv, w_in, gap, H, out_dim = 16, 30, 30, 4, 128, 10
    Bn = o.slots // H
    rng = np.random.default_rng(43)
    x = rng.uniform(-1, 1, (Bn, c_in, hv, w_in))
    W = rng.normal(0, 0.05, (out_dim, c_in * hv * w_in))
    b = rng.normal(0, 0.05, out_dim)
    z = np.concatenate([layouts.image_columns(x[:, c], o.slots, H, gap) for c in range(c_in)])
    ox, gx = encrypt_both(o, g, encode_columns(o, z), ct_id_base=0)
    ox = ox.reshape(c_in, w_in, *ox.shape[1:])
    lp = o.L1
    pts = o.fc_plaintexts(lp, c_in, hv, w_in, gap, H, Bn, W, list(range(out_dim)))
    oz = o.fc(ox, gap, H, pts, b, o.scale, list(range(out_dim)))
    gz = g.fc_apply(gx, g.fc_prepare_coeffs(pts, gap, H, lp), b)
    assert np.array_equal(gz.export(), oz)
    logits = layouts.logits_from_fc(g.decrypt_slots(gz), Bn, H)
    assert np.abs(logits - fp64_ref.dense(x, W, b)).max() < 1e-4


@pytest.mark.parametrize("stride,c_in,k", [(1, 1, 3), (2, 3, 3), (2, 2, 5)])
def test_conv2d_encrypted_kernels_matches_oracle_and_fp64(lib, stride, c_in, k):
    """Encrypted kernels (the model provider's ciphertexts): bit-exact with the oracle from the same
    kernel plaintexts and seeds, decrypting to the FP64 convolution; the library's own kernel
    encryption (he_encrypt_conv_weights) encodes the same integers, so it is bit-exact too."""
    H, side, c_out = 16, 11, 3
    o, g = make_pair(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=17, steps=list(range(1, k)))
    rng = np.random.default_rng(30 + stride * 10 + c_in)
    imgs = rng.uniform(0, 1, (3, c_in, side, side - 1))
    K = rng.normal(0, 0.3, (c_out, c_in, k, k))
    bias = rng.normal(0, 0.3, c_out)
    ox, gx = image_columns_both(o, g, imgs, H, ct_id_base=1000)
    lp = o.L1
    m = o.conv_weight_plaintexts(K, lp)
    ow, gw = encrypt_both(o, g, m, ct_id_base=7000, scale=float(o.q[lp - 1]))
    gy = g.conv2d_enc(gx, c_in, 1, gw, bias, c_out, k, stride)
    oy = o.conv2d_enc(ox, 1, ow, bias, c_out, k, stride, o.scale)
    assert np.array_equal(gy.export(), oy)
    gw2 = g.encrypt_conv_weights(K, lp, 7000)
    assert np.array_equal(gw2.export(), ow)
    ref = fp64_ref.conv2d(imgs, K, bias, stride)
    got = g.decrypt_image(gy, 3, H, stride, ref.shape[2])
    got = got.reshape(3, c_out, ref.shape[3], ref.shape[2]).transpose(0, 1, 3, 2)
    assert np.abs(got - ref).max() < 1e-5


@pytest.mark.parametrize("gap,h,H", [(2, 5, 16), (4, 3, 16), (2, 31, 64)])
def test_reform_matches_oracle(lib, gap, h, H):
    """ReForm: bit-exact with the oracle from the same mask plaintexts; the library's own mask
    encoder decrypts to the same compacted rows."""
    o, g = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=27, steps=None)
    steps = [(gap - 1) * i for i in range(1, h)]
    o.keygen(steps)
    g.keygen(steps)
    rng = np.random.default_rng(gap + h)
    B = o.slots // H
    rows = rng.uniform(-1, 1, (2, B, h))
    z = np.zeros((2, o.slots))
    for c in range(2):
        for b in range(B):
            z[c, b * H + gap * np.arange(h)] = rows[c, b]
    ox, gx = encrypt_both(o, g, encode_columns(o, z), ct_id_base=40)
    masks = o.reform_masks(h, H, o.L1)
    gy = g.reform_coeffs(gx, gap, h, masks)
    assert np.array_equal(gy.export(), o.reform(ox, gap, h, masks))
    want = np.zeros((2, o.slots))
    for c in range(2):
        for b in range(B):
            want[c, b * H: b * H + h] = rows[c, b]
    assert np.abs(g.decrypt_slots(g.reform(gx, gap, h, H)) - want).max() < 1e-5


@pytest.mark.parametrize("h,w,k,Hb,Wb", [(6, 6, 3, 8, 8), (7, 5, 2, 8, 8), (12, 10, 3, 16, 16)])
def test_vr_conv2d_matches_oracle_and_fp64(lib, h, w, k, Hb, Wb):
    """The paper's single-ciphertext convolution (Alg. 4 with Kernelspanner and SumForConv) over
    virtual image blocks: bit-exact with the oracle from the same plaintexts and seeds, decrypting to
    FP64; the library's own encoders agree within tolerance."""
    o, g = make_pair(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=29,
                     steps=list(range(1, k)) + [Wb * p for p in range(1, k)])
    S = o.slots
    rng = np.random.default_rng(h * 100 + k)
    B = 2 * (S // (Hb * Wb))  # two ciphertexts of images
    imgs = rng.uniform(0, 1, (B, h, w))
    K = rng.normal(0, 0.4, (k, k))
    k0 = 0.15
    lp = o.L1
    mx = encode_columns(o, layouts.vr_images(imgs, S, Hb, Wb))
    ox, gx = encrypt_both(o, g, mx, ct_id_base=0)
    ql = float(o.q[lp - 1])
    ms = np.stack([o.encode(v, ql) for v in layouts.vr_kernelspanner(K, h, w, S, Hb, Wb)])
    os_, gs = encrypt_both(o, g, ms, ct_id_base=20, scale=ql)
    mb = o.encode(layouts.vr_bias(k0, k, h, w, S, Hb, Wb))[None]
    ob, gb = encrypt_both(o, g, mb, limbs=lp - 2, ct_id_base=90)
    masks = np.stack([o.encode(v, float(o.q[lp - 2])) for v in layouts.vr_masks(k, h, w, S, Hb, Wb)])
    gy = g.vr_conv2d_coeffs(gx, gs, gb, k, Wb, masks)
    oy = o.vr_conv2d(ox, os_, ob[0], k, Wb, masks)
    assert np.array_equal(gy.export(), oy)
    ref = fp64_ref.conv2d(imgs[:, None], K[None, None], np.array([k0]), 1)[:, 0]
    ho, wo = h - k + 1, w - k + 1
    got = layouts.vr_images_from(g.decrypt_slots(gy), B, h, w, Hb, Wb)
    assert np.abs(got[:, :ho, :wo] - ref).max() < 1e-5
    # the library's own encoders (images, Kernelspanner, bias, masks)
    gx2 = g.vr_encrypt_images(imgs, Hb, Wb, 0)
    gk2, gb2 = g.vr_encrypt_kernels(K, k0, h, w, Hb, Wb, lp, 20)
    got2 = layouts.vr_images_from(g.decrypt_slots(g.vr_conv2d(gx2, gk2, gb2, h, w, k, Hb, Wb)), B, h, w, Hb, Wb)
    assert np.abs(got2[:, :ho, :wo] - ref).max() < 1e-5


@pytest.mark.parametrize("m,n,p", [(4, 8, 4), (8, 4, 2), (16, 16, 8)])
def test_vr_matmul_matches_oracle_and_fp64(lib, m, n, p):
    """The paper's single-ciphertext matmul (Alg. 3: tau_a, tau_b, RowShifter, SumColVec, mask F):
    bit-exact with the oracle from the same plaintexts and seeds, decrypting to A @ B; the library's
    own encoders agree within tolerance."""
    steps = [idx * n for idx in range(1, p)] + [t for t in (1, 2, 4, 8, 16) if t < n] + \
            [-t for t in (1, 2, 4, 8, 16) if t < n]
    o, g = make_pair(10, (60, 40, 40, 40, 40), 1, 60, 1, 40.0, seed=31, steps=steps)
    S = o.slots
    rng = np.random.default_rng(m + n * 10 + p)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    lp = o.L1
    oa, ga = encrypt_both(o, g, encode_columns(o, layouts.vr_matrix_a(A, S)[None]), ct_id_base=3)
    ob, gb = encrypt_both(o, g, encode_columns(o, layouts.vr_matrix_b(Bm, S)[None]), ct_id_base=4)
    mv = layouts.vr_matmul_masks(m, n, p, S)
    masks = np.stack([o.encode(mv[0], float(o.q[lp - 2]))] + [o.encode(v, float(o.q[lp - 3])) for v in mv[1:]])
    gd = g.vr_matmul_coeffs(ga, gb, m, n, p, masks)
    od = o.vr_matmul(oa[0], ob[0], n, p, masks)
    assert np.array_equal(gd.export()[0], od)
    sc = o.scale ** 2 / o.q[lp - 1]
    assert np.abs(layouts.vr_matmul_from(g.decrypt_slots(gd)[0], m, n, p) - A @ Bm).max() < 1e-5
    gd2 = g.vr_matmul(g.vr_encrypt_matrix_a(A, 3), g.vr_encrypt_matrix_b(Bm, 4), m, n, p)
    assert np.abs(layouts.vr_matmul_from(g.decrypt_slots(gd2)[0], m, n, p) - A @ Bm).max() < 1e-5
    assert gd.scale == sc


@pytest.mark.parametrize("n,hw,r", [(16, 12, 5), (32, 20, 19), (64, 64, 3)])
def test_vrot_matches_oracle(lib, n, hw, r):
    """vRot (Alg. 5): bit-exact with the oracle from the same mask plaintexts; the library's own
    masks decrypt to every virtual ciphertext rotated left by r."""
    o, g = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=33, steps=None)
    S = o.slots
    o.keygen([r, S - hw + r])
    g.keygen([r, S - hw + r])
    v = np.random.default_rng(n + r).uniform(-1, 1, (2, S))
    ox, gx = encrypt_both(o, g, encode_columns(o, v), ct_id_base=11)
    masks = np.stack([o.encode(f, float(o.q[o.L1 - 1])) for f in layouts.vrot_masks(n, hw, r, S)])
    assert np.array_equal(g.vrot_coeffs(gx, r, hw, masks).export(), o.vrot(ox, r, hw, masks))
    want = np.stack([layouts.vrot_slots(v[t], n, hw, r) for t in range(2)])
    assert np.abs(g.decrypt_slots(g.vrot(gx, r, n, hw)) - want).max() < 1e-5


def _act_polynomials():
    from tests.test_oracle_pins import act_polynomials
    return act_polynomials()


@pytest.mark.parametrize("name", ["ACT-1", "ACT-2", "deg2"])
def test_poly_act_degree3_matches_oracle_and_fp64(lib, name):
    """The paper's ACT-1 / ACT-2 (Table I) and a general degree-2 polynomial: bit-exact with the
    oracle (two- and three-component inputs), decrypting to f(x) in FP64."""
    c = _act_polynomials()[name] if name != "deg2" else [0.3, -0.7, 1.1, 0.0]
    o, g = make_pair(10, (60,) + (45,) * 4, 2, 60, 2, 45.0, seed=23, steps=[])
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (3, o.slots))
    ox, gx = encrypt_both(o, g, encode_columns(o, x), ct_id_base=70)
    coeffs = c if name != "deg2" else c[:3]
    gy = g.poly_act(gx, coeffs)
    oy, sy = o.poly_act3(ox, c, o.scale)
    assert gy.polys == 3 and gy.limbs == o.L1 - 2 and gy.scale == sy
    assert np.array_equal(gy.export(), oy)
    want = c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3
    got = g.decrypt_slots(gy)
    assert np.abs(got - want).max() < 1e-5
    # three-component input: x^2 (unrelinearised) through the activation
    gs = g.poly_act(encrypt_both(o, g, encode_columns(o, x), ct_id_base=70)[1], [0.0, 0.0, 1.0])
    os_ = np.stack([o.rescale(o.tensor(ox[t], ox[t])) for t in range(3)])
    g2 = g.poly_act(gs, coeffs)
    o2, s2 = o.poly_act3(os_, c, o.scale * o.scale / o.q[o.L1 - 1])
    assert np.array_equal(g2.export(), o2) and g2.scale == s2
    x2 = x ** 2
    assert np.abs(g.decrypt_slots(g2) - (c[0] + c[1] * x2 + c[2] * x2 ** 2 + c[3] * x2 ** 3)).max() < 1e-5


def test_fc_matches_oracle(lib):
    o, g = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=8, steps=[2, 4, 8])
    rng = np.random.default_rng(8)
    c_in, hv, w_in, gap, H, Bn, out_dim = 3, 5, 4, 2, 16, 4, 6
    x = rng.uniform(-1, 1, (Bn, c_in, hv, w_in))
    W = rng.normal(0, 0.3, (out_dim, c_in * hv * w_in))
    b = rng.normal(0, 0.3, out_dim)
    z = np.concatenate([layouts.image_columns(x[:, c], o.slots, H, gap) for c in range(c_in)])
    ox, gx = encrypt_both(o, g, encode_columns(o, z), ct_id_base=0)
    ox = ox.reshape(c_in, w_in, *ox.shape[1:])
    lp = o.L1
    pts = o.fc_plaintexts(lp, c_in, hv, w_in, gap, H, Bn, W, list(range(out_dim)))
    oz = o.fc(ox, gap, H, pts, b, o.scale, list(range(out_dim)))
    gp = g.fc_prepare_coeffs(pts, gap, H, lp)
    gz = g.fc_apply(gx, gp, b)
    assert np.array_equal(gz.export(), oz)
    logits = layouts.logits_from_fc(g.decrypt_slots(gz), Bn, H)
    assert np.abs(logits - fp64_ref.dense(x, W, b)).max() < 1e-5
    # the library's own weight encoder agrees within tolerance
    gp2 = g.fc_prepare(W, c_in, hv, w_in, gap, H, Bn, lp)
    logits2 = layouts.logits_from_fc(g.decrypt_slots(g.fc_apply(gx, gp2, b)), Bn, H)
    assert np.abs(logits2 - fp64_ref.dense(x, W, b)).max() < 1e-5


def test_cnn_small_matches_oracle(lib):
    """conv 5x5 s2 -> x^2 -> conv 3x3 s2 -> x^2 -> FC, CNN prime shape, reduced ring and image."""
    o, g = make_pair(10, (60,) + (45,) * 6, 2, 60, 2, 45.0, seed=31, steps=[1, 2, 3, 4, 8, 16])
    side, H, Bn = 17, 32, 3
    h1 = (side - 5) // 2 + 1
    h2 = (h1 - 3) // 2 + 1
    rng = np.random.default_rng(31)
    imgs = rng.uniform(0, 1, (Bn, 1, side, side))
    c1w, c1b = rng.normal(0, 0.2, (2, 1, 5, 5)), rng.normal(0, 0.2, 2)
    c2w, c2b = rng.normal(0, 0.2, (3, 2, 3, 3)), rng.normal(0, 0.2, 3)
    fw, fb = rng.normal(0, 0.2, (4, 3 * h2 * h2)), rng.normal(0, 0.2, 4)
    ox, gx = image_columns_both(o, g, imgs, H)
    sc = o.scale
    gy = g.conv2d(gx, 1, 1, c1w, c1b, 2)
    oy = o.conv2d(ox, 1, c1w, c1b, 2, sc)
    assert np.array_equal(gy.export(), oy)
    g.square(gy)
    oy = o.square(oy)
    assert np.array_equal(gy.export(), oy)
    sc = sc * sc / o.q[o.L1 - 2]
    assert gy.scale == sc
    oy = oy.reshape(2, h1, *oy.shape[1:])
    gy2 = g.conv2d(gy, 2, 2, c2w, c2b, 2)
    oy2 = o.conv2d(oy, 2, c2w, c2b, 2, sc)
    assert np.array_equal(gy2.export(), oy2)
    g.square(gy2)
    oy2 = o.square(oy2)
    lp = oy2.shape[2]
    sc = sc * sc / o.q[lp]
    oy2 = oy2.reshape(3, h2, *oy2.shape[1:])
    pts = o.fc_plaintexts(lp, 3, h2, h2, 4, H, Bn, fw, list(range(4)))
    oz = o.fc(oy2, 4, H, pts, fb, sc, list(range(4)))
    gz = g.fc_apply(gy2, g.fc_prepare_coeffs(pts, 4, H, lp), fb)
    assert np.array_equal(gz.export(), oz)
    logits = layouts.logits_from_fc(g.decrypt_slots(gz), Bn, H)
    x = fp64_ref.conv2d(imgs, c1w, c1b, 2) ** 2
    x = fp64_ref.conv2d(x, c2w, c2b, 2) ** 2
    assert np.abs(logits - fp64_ref.dense(x, fw, fb)).max() < 1e-4


# ---------------------------------------------------------------------------
# errors and degenerate cases
# ---------------------------------------------------------------------------
def test_errors(lib):
    from paper_2512_18646_gb300 import HeError, api
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_E_LEVEL, HE_E_NOKEY, HE_E_STATE
    g = api.Context(8, (60, 40), 1, 60, 1, 40.0)
    with pytest.raises(HeError) as e:
        g.encrypt_matrix_a(np.ones((2, 2)))
    assert e.value.code == HE_E_STATE
    g.keygen([1])
    x = g.encrypt_matrix_a(np.ones((2, 3)))
    with pytest.raises(HeError) as e:
        g.rotate(x, [2])
    assert e.value.code == HE_E_NOKEY
    y = g.mul(x, x)
    with pytest.raises(HeError) as e:
        g.mul(y, y)
    assert e.value.code == HE_E_LEVEL
    with pytest.raises(HeError) as e:
        g.encrypt_matrix_b(np.ones((2, 3)))  # 3 does not divide the slot count
    assert e.value.code == HE_E_ARG
    with pytest.raises(HeError) as e:
        g.encrypt_image(np.ones((1, 5, 5)), 4)  # block smaller than the image
    assert e.value.code == HE_E_ARG
    with pytest.raises(HeError) as e:
        api.Context(20, (60,), 1, 60, 1, 40.0)
    assert e.value.code == HE_E_ARG


def test_errors_of_the_layer_variants(lib):
    """Argument, level and state errors of the matmul variants, activations, ReForm, the
    single-ciphertext layers, graphs and the transform geometry (no GPU fault on any path)."""
    import torch
    from paper_2512_18646_gb300 import HeError, api
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_E_LEVEL, HE_E_STATE, HE_E_UNIMPL

    def code(fn):
        with pytest.raises(HeError) as e:
            fn()
        return e.value.code

    g = api.Context(8, (60, 40, 40), 1, 60, 1, 40.0, stream=torch.cuda.Stream().cuda_stream)
    g.keygen([1, 2, 3])
    assert code(lambda: api.volley_geometry(128, 5, 3)) == HE_E_ARG  # p does not divide the slots
    assert code(lambda: api.volley_geometry(16, 20, 4)) == HE_E_ARG  # no block fits
    A = g.encrypt_matrix_a(np.ones((2, 4)), 0)
    B = g.encrypt_matrix_b(np.ones((4, 4)), 10)
    assert code(lambda: g.matmul_bsgs(A, B, 2, 4, 5)) == HE_E_ARG  # baby step larger than p
    Ahat = g.encrypt_matrix_a_volley(np.ones((2, 4)), 4, 0)
    B3 = g.encrypt_matrix_b(np.ones((3, 4)), 20)
    assert code(lambda: g.matmul_volley(Ahat, B3)) == HE_E_ARG  # 4 ciphertexts of A, 3 of B
    x = g.encrypt_matrix_a(np.ones((2, 2)), 30)
    assert code(lambda: g.poly_act(x, [0, 1, 0, 0, 1])) == HE_E_UNIMPL  # degree 4
    low = g.mul(x, x)  # one level left
    assert code(lambda: g.poly_act(low, [0.1, 0.2, 0.3, 0.4])) == HE_E_LEVEL  # two levels needed
    assert code(lambda: g.reform(x, 1, 2, 8)) == HE_E_ARG  # gap 1
    assert code(lambda: g.reform(x, 2, 5, 8)) == HE_E_ARG  # rows do not fit the block
    xi = g.vr_encrypt_images(np.ones((2, 4, 4)), 4, 4, 0)
    assert code(lambda: g.vr_encrypt_kernels(np.ones((5, 5)), 0.0, 4, 4, 4, 4)) == HE_E_ARG  # kernel > image
    kk, bb = g.vr_encrypt_kernels(np.ones((2, 2)), 0.0, 4, 4, 4, 4)
    assert code(lambda: g.vr_conv2d(xi, bb, bb, 4, 4, 2, 4, 4)) == HE_E_ARG  # one kernel ciphertext, k^2 = 4 needed
    assert code(lambda: g.vr_conv2d(low, kk, bb, 4, 4, 2, 4, 4)) == HE_E_LEVEL  # input one level from the bottom
    assert code(lambda: g.vr_encrypt_matrix_b(np.ones((4, 3)), 0)) == HE_E_ARG  # p does not divide the rows
    assert code(lambda: g.ntt_set_geometry(9, 16)) == HE_E_ARG
    assert code(lambda: g.ntt_autotune(0)) == HE_E_ARG
    assert code(lambda: g.graph_end()) == HE_E_STATE  # no capture open
    g.graph_begin()
    assert code(lambda: g.graph_begin()) == HE_E_STATE  # already capturing
    A2 = g.add(A, A)  # made during the capture
    assert code(lambda: g.assign(A, A2)) == HE_E_STATE  # into a set made before the capture
    y = g.add(x, x)
    graph = g.graph_end()
    graph.launch()
    g.synchronize()
    assert np.array_equal(y.export(), g.add(x, x).export())
    graph.destroy()
    del xi


def test_degenerate_cases(lib):
    """Empty and one-element inputs of the layer variants: an empty batch, ReForm of one row, vRot by 0
    (the image part of every row kept, the rest cleared), the identity polynomial."""
    from paper_2512_18646_gb300 import api
    o, g = make_pair(8, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=34, steps=[128 - 12])  # vRot by 0 wraps by -12
    assert g.matmul_batched([], [], [], []) == []
    S = o.slots
    v = np.random.default_rng(1).uniform(-1, 1, (1, S))
    ox, gx = encrypt_both(o, g, encode_columns(o, v), ct_id_base=0)
    # ReForm of a single row is the row mask itself
    masks = o.reform_masks(1, 16, o.L1)
    assert np.array_equal(g.reform_coeffs(gx, 2, 1, masks).export(), o.reform(ox, 2, 1, masks))
    want = np.zeros(S)
    want[::16] = v[0, ::16]
    assert np.abs(g.decrypt_slots(g.reform(gx, 2, 1, 16))[0] - want).max() < 1e-5
    # vRot by 0: F2 is empty, every row keeps its image part
    got = g.decrypt_slots(g.vrot(gx, 0, 16, 12))[0]
    assert np.abs(got - layouts.vrot_slots(v[0], 16, 12, 0)).max() < 1e-5
    # f(x) = x through the degree-3 schedule
    y = g.poly_act(g.encrypt_coeffs(encode_columns(o, v), o.L1, o.scale, 5), [0.0, 1.0, 0.0, 0.0])
    assert np.abs(g.decrypt_slots(y)[0] - v[0]).max() < 1e-5


def test_matmul_batched_equals_single_matmuls(lib):
    """Mixed shapes (some sharing p): batched results equal he_matmul's bit for bit, and GEMM."""
    o, g = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=12, steps=list(range(1, 8)))
    rng = np.random.default_rng(12)
    shapes = [(4, 3, 8), (8, 5, 4), (2, 2, 8), (16, 1, 1), (5, 7, 4)]
    As, Bs, ref = [], [], []
    for t, (m, n, p) in enumerate(shapes):
        A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
        As.append(g.encrypt_matrix_a(A, 1000 * t))
        Bs.append(g.encrypt_matrix_b(Bm, 1000 * t + 500))
        ref.append(A @ Bm)
    outs = g.matmul_batched(As, Bs, [s[0] for s in shapes], [s[2] for s in shapes])
    for t, (m, n, p) in enumerate(shapes):
        single = g.matmul(As[t], Bs[t], m, p)
        assert np.array_equal(outs[t].export(), single.export()), t
        assert np.abs(g.decrypt_matrix(outs[t], m, p) - ref[t]).max() < 1e-5



def test_matmul_batched_matches_oracle_on_ragged_shapes(lib):
    """he_matmul_batched over ragged shapes (some sharing p, so their B operands share launches),
    each product bit-exact against the oracle's revolver matmul on the same ciphertexts."""
    o, g = make_pair(10, (60, 40, 40), 1, 60, 1, 40.0, seed=17, steps=list(range(1, 8)))
    rng = np.random.default_rng(17)
    shapes = [(5, 3, 8), (8, 5, 4), (3, 2, 8), (16, 1, 1), (7, 6, 4), (1, 4, 2)]
    ga_s, gb_s, oa_s, ob_s, mats = [], [], [], [], []
    for t, (m, n, p) in enumerate(shapes):
        A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
        oa, ga = encrypt_both(o, g, encode_columns(o, layouts.matrix_a_columns(A, o.slots)), ct_id_base=1000 * t)
        ob, gb = encrypt_both(o, g, encode_columns(o, layouts.matrix_b_rows(Bm, o.slots)), ct_id_base=1000 * t + 500)
        ga_s.append(ga), gb_s.append(gb), oa_s.append(oa), ob_s.append(ob), mats.append(A @ Bm)
    outs = g.matmul_batched(ga_s, gb_s, [s[0] for s in shapes], [s[2] for s in shapes])
    for t, (m, n, p) in enumerate(shapes):
        assert np.array_equal(outs[t].export(), o.matmul(oa_s[t], ob_s[t], p)), t
        assert np.abs(g.decrypt_matrix(outs[t], m, p) - mats[t]).max() < 1e-5


def test_graph_replays_batched_matmuls(lib):
    """A batched call captured into a CUDA graph: each replay recomputes the products from the
    current contents of the input sets, bit-identical to eager calls; in-place calls on sets made
    before the capture are refused inside it."""
    import torch
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HE_E_STATE, HeError
    stream = torch.cuda.Stream()
    pre = synthetic.MATMUL_SMALL
    g = api.Context.from_preset(pre, seed=77, stream=stream.cuda_stream)
    g.keygen([1, 2, 3, 4, 5, 6, 7])
    shapes = [(4, 8, 4), (4, 8, 4), (3, 5, 8), (4, 8, 4), (2, 3, 2)]

    def operands(seed):
        rng = np.random.default_rng(seed)
        ops = [(rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))) for m, n, p in shapes]
        return ([g.encrypt_matrix_a(A, 10 * t) for t, (A, _) in enumerate(ops)],
                [g.encrypt_matrix_b(B, 10 * t + 5) for t, (_, B) in enumerate(ops)], ops)

    A1, B1, ops1 = operands(1)
    A2, B2, ops2 = operands(2)
    ms, ps = [s[0] for s in shapes], [s[2] for s in shapes]
    eager1 = [c.export() for c in g.matmul_batched(A1, B1, ms, ps)]
    eager2 = [c.export() for c in g.matmul_batched(A2, B2, ms, ps)]
    # graph inputs: sets made before the capture, holding the first operands
    Ain, Bin, _ = operands(1)
    g.graph_begin()
    outs = g.matmul_batched(Ain, Bin, ms, ps)
    with pytest.raises(HeError) as e:
        g.rescale(Ain[0])
    assert e.value.code == HE_E_STATE
    graph = g.graph_end()
    assert graph.kernel_nodes > 0
    graph.launch()
    g.synchronize()
    for t in range(len(shapes)):
        assert np.array_equal(outs[t].export(), eager1[t])
        assert np.abs(g.decrypt_matrix(outs[t], ms[t], ps[t]) - ops1[t][0] @ ops1[t][1]).max() < 1e-5
    for t in range(len(shapes)):
        g.assign(Ain[t], A2[t])
        g.assign(Bin[t], B2[t])
    graph.launch()
    graph.launch()  # a replay over the same inputs gives the same results
    g.synchronize()
    for t in range(len(shapes)):
        assert np.array_equal(outs[t].export(), eager2[t])
    graph.destroy()


def test_graph_capture_failure_leaves_context_usable(lib):
    """A call that uploads host data cannot be captured: the capture reports HE_E_CUDA and the
    context keeps working eagerly."""
    import torch
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HE_E_CUDA, HeError
    stream = torch.cuda.Stream()
    g = api.Context(10, (60, 40, 40), 1, 60, 1, 40.0, seed=78, stream=stream.cuda_stream)
    g.keygen([1])
    g.graph_begin()
    failed = False
    try:
        g.encrypt_matrix_a(np.ones((2, 2)), 0)
    except HeError:
        failed = True
    with pytest.raises(HeError) as e:
        g.graph_end()
    assert e.value.code == HE_E_CUDA or failed
    A, Bm = np.arange(6.0).reshape(2, 3) / 6, np.arange(6.0).reshape(3, 2) / 6
    C = g.decrypt_matrix(g.matmul(g.encrypt_matrix_a(A, 0), g.encrypt_matrix_b(Bm, 5), 2, 2), 2, 2)
    assert np.abs(C - A @ Bm).max() < 1e-5


def test_device_wait_that_runs_out_is_reported_and_the_context_stays_usable(lib):
    """A device-side wait that nothing ends (he_debug_wait_timeout: a barrier no thread arrives on)
    gives up after its limit and records the failure in the context's status word; the next
    synchronisation reports HE_E_TIMEOUT once, and the context keeps computing exact results."""
    from paper_2512_18646_gb300 import HeError, load
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_E_TIMEOUT, check
    o, g = make_pair(10, (60, 45, 45), 2, 60, 2, 45.0, seed=9, steps=[1])
    rng = np.random.default_rng(9)
    m = rng.integers(-(1 << 30), 1 << 30, size=(2, o.N), dtype=np.int64)
    oc, gc = encrypt_both(o, g, m)
    check(load().he_debug_wait_timeout(g.h, 2000))  # 2 ms
    with pytest.raises(HeError) as e:
        g.synchronize()
    assert e.value.code == HE_E_TIMEOUT
    g.synchronize()  # reported once
    assert np.array_equal(g.rotate(gc, [1]).export(), np.stack([o.rotate(c, [1])[0] for c in oc]))
    for bad in (0, 2000001):
        assert load().he_debug_wait_timeout(g.h, bad) == HE_E_ARG


def test_overlapped_import_equals_import_and_reports_bad_residues_later(lib):
    """he_ctset_import_async (the copy on a stream of its own, two staging buffers taken in turn)
    gives the same words as he_ctset_import over three imports interleaved with computation; an
    out-of-range residue is reported as HE_E_ARG by the next synchronisation, after which the
    context keeps working."""
    import torch
    from paper_2512_18646_gb300 import HeError
    from paper_2512_18646_gb300._lib import HE_E_ARG
    o, g = make_pair(10, (60, 45, 45), 2, 60, 2, 45.0, seed=13, steps=[1])
    rng = np.random.default_rng(13)
    hosts = []
    for t in range(3):
        a = np.stack([np.stack([rng.integers(0, q, g.N, dtype=np.uint64) for q in g.primes[:3]]) for _ in range(2)])
        buf = torch.empty(a.size, dtype=torch.int64).pin_memory().numpy().view(np.uint64).reshape(1, 2, 3, g.N)
        buf[...] = a[None]
        hosts.append(buf)
    outs = []
    for t in range(3):
        x = g.import_coeffs_async(hosts[t], g.scale)
        outs.append((x, g.rotate(x, [1])))  # computation queued behind the import
    for t in range(3):
        ref = g.import_coeffs(hosts[t], g.scale)
        assert np.array_equal(outs[t][0].export_raw(), ref.export_raw())
        assert np.array_equal(outs[t][1].export_raw(), g.rotate(ref, [1]).export_raw())
    for at in ((0, 1, 2, 5), (0, 1, 2, g.N - 1), (0, 0, 0, 0)):
        bad = hosts[0].copy()
        bad[at] = np.uint64(g.primes[at[2]])  # a residue equal to its prime
        g.import_coeffs_async(bad, g.scale)
        with pytest.raises(HeError) as e:
            g.synchronize()
        assert e.value.code == HE_E_ARG
        g.synchronize()  # reported once
        with pytest.raises(HeError) as e:
            g.import_coeffs(bad, g.scale)
        assert e.value.code == HE_E_ARG
    assert np.array_equal(g.import_coeffs_async(hosts[1], g.scale).export_raw(), outs[1][0].export_raw())


def test_export_async_equals_export_and_waits_by_ticket(lib):
    """he_ctset_export_async queued behind computation writes the words he_ctset_export gives; six
    exports (more than the context's four event slots) from sets freed right after the call are
    waited by ticket, the oldest first; tickets grow; 0 and a ticket not yet issued are refused; the
    call is refused inside a capture of the context's stream, which stays usable."""
    import torch
    from paper_2512_18646_gb300 import HeError, api
    from paper_2512_18646_gb300._lib import HE_E_ARG
    _, g = make_pair(10, (60, 45, 45), 2, 60, 2, 45.0, seed=14, steps=[1])
    m = np.random.default_rng(14).integers(-(1 << 40), 1 << 40, size=(3, g.N), dtype=np.int64)
    x = g.encrypt_coeffs(m, 3, g.scale)
    ops = (lambda: g.add(x, x), lambda: g.rotate(x, [1]))
    want = [op().export() for op in ops]

    def pinned(shape):
        n = int(np.prod(shape))
        return torch.empty(n, dtype=torch.int64).pin_memory().numpy().view(np.uint64).reshape(shape)

    bufs, tickets = [], []
    for t in range(6):
        y = ops[t % 2]()
        bufs.append(pinned(want[t % 2].shape))
        tickets.append(y.export_async(bufs[-1]))
        y.free()  # its release is ordered after the copy
    assert tickets[0] > 0 and all(b > a for a, b in zip(tickets, tickets[1:]))
    g.export_wait(tickets[0])  # its event slot was re-recorded by a later export
    assert np.array_equal(bufs[0], want[0])
    g.export_wait(tickets[4])
    for t in range(1, 5):
        assert np.array_equal(bufs[t], want[t % 2]), t
    g.export_wait(tickets[2])  # already complete
    g.export_wait(tickets[5])
    assert np.array_equal(bufs[5], want[1])
    for bad in (0, tickets[-1] + 1):
        with pytest.raises(HeError) as e:
            g.export_wait(bad)
        assert e.value.code == HE_E_ARG

    s = torch.cuda.Stream()
    g2 = api.Context(10, (60, 45, 45), 2, 60, 2, 45.0, seed=15, stream=s.cuda_stream)
    g2.keygen([])
    x2 = g2.encrypt_coeffs(m, 3, g2.scale)
    g2.synchronize()
    refused = False
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gr.capture_begin()
        try:
            x2.export_async(bufs[0])
        except HeError:
            refused = True
        finally:
            try:
                gr.capture_end()
            except RuntimeError:
                refused = True
    assert refused
    t2 = x2.export_async(bufs[0])
    g2.export_wait(t2)
    assert np.array_equal(bufs[0], x2.export())


def test_direct_capture_of_the_context_stream_is_refused_loudly(lib):
    """A capture the caller opens on the context's stream itself (torch's CUDA graph on that stream,
    not he_graph_begin) must not record a copy from the context's page-locked staging slots, which
    later calls reuse: a call that uploads host data (a convolution's weights) fails the capture
    with an error instead, calls without uploads capture and replay like eager calls, and the
    context keeps giving its eager results afterwards."""
    import torch
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HeError
    s = torch.cuda.Stream()
    g = api.Context(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=79, stream=s.cuda_stream)
    g.keygen([1, 2])
    rng = np.random.default_rng(79)
    imgs = rng.uniform(0, 1, (2, 8, 8))
    K, bias = rng.normal(0, 0.3, (2, 1, 3, 3)), rng.normal(0, 0.3, 2)
    x = g.encrypt_image(imgs, 16, ct_id_base=0)
    eager = g.conv2d(x, 1, 1, K, bias, 1).export()
    g.synchronize()
    # many uploads before the capture so that every staging slot holds some other call's data
    for _ in range(20):
        g.conv2d(x, 1, 1, K * 0.5, bias, 1)
    g.synchronize()
    refused = False
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gr.capture_begin()
        try:
            g.conv2d(x, 1, 1, K, bias, 1)
        except HeError:
            refused = True
        finally:
            try:
                gr.capture_end()
            except RuntimeError:
                refused = True
    assert refused
    # the overlapped import is refused inside such a capture too (its copy reads host memory)
    host = np.ascontiguousarray(x.export())
    refused = False
    gr1 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gr1.capture_begin()
        try:
            g.import_coeffs_async(host, g.scale)
        except HeError:
            refused = True
        finally:
            try:
                gr1.capture_end()
            except RuntimeError:
                refused = True
    assert refused
    assert np.array_equal(g.import_coeffs_async(host, g.scale).export(), host)  # usable afterwards
    # a call without host uploads captures and replays bit-identically
    y = g.conv2d(x, 1, 1, K, bias, 1)
    g.synchronize()
    want = g.add(y, y).export()
    gr2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gr2.capture_begin()
        z = g.add(y, y)
        gr2.capture_end()
    for _ in range(20):
        g.conv2d(x, 1, 1, K * 0.25, bias, 1)
    gr2.replay()
    torch.cuda.synchronize()
    assert np.array_equal(z.export(), want)
    assert np.array_equal(g.conv2d(x, 1, 1, K, bias, 1).export(), eager)


def test_work_budget_chunks_are_bit_identical(lib):
    """Chunked convolutions, relinearisations, products and rescales (a 1-byte work budget: one
    column or ciphertext per chunk) give the same words as the unchunked path; the chunked conv
    layer matches the oracle."""
    from paper_2512_18646_gb300 import api
    pre = synthetic.small_preset(11, q_bits=(60, 40, 40, 40, 40))
    o = Oracle.from_preset(pre, seed=17)
    o.keygen([1, 2])
    imgs = np.random.default_rng(18).uniform(0, 1, (2, 12, 12))
    z = layouts.image_columns(imgs, o.slots, 16)
    m = np.stack([o.encode(v) for v in z])
    rng = np.random.default_rng(19)
    K1, b1 = rng.normal(0, 0.3, (3, 1, 3, 3)), rng.normal(0, 0.3, 3)
    K2, b2 = rng.normal(0, 0.3, (2, 3, 3, 3)), rng.normal(0, 0.3, 2)
    X = np.stack([o.encrypt(m[j], o.L1, j) for j in range(len(m))])[None]
    oy1 = o.conv2d(X, 1, K1, b1, 1, o.scale)
    outs = []
    for budget in (0, 1):
        g = api.Context.from_preset(pre, seed=17)
        g.keygen([1, 2])
        g.set_work_budget(budget)
        x = g.encrypt_coeffs(m, o.L1, o.scale, 0)
        y1 = g.conv2d(x, 1, 1, K1, b1, 1)
        e1 = y1.export()
        assert np.array_equal(e1, oy1)
        g.square(y1)                       # three components, rescaled
        y2 = g.conv2d(y1, 3, 1, K2, b2, 2)  # relinearises its input first
        y3 = g.mul(y2, y2)
        outs.append([e1, y1.export(), y2.export(), y3.export()])
        del x, y1, y2, y3
        g.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_destroy_returns_cached_pool_memory(lib):
    """Freed ciphertexts stay cached in the device's memory pool while their context lives; destroying
    the context hands that memory back to the driver, so a later process or context can use it."""
    import torch
    from paper_2512_18646_gb300 import api
    torch.cuda.init()
    api.Context(14, (60, 45, 45, 45), 2, 60, 2, 45.0, seed=3).close()  # start from a trimmed pool
    free0, _ = torch.cuda.mem_get_info()
    g = api.Context(14, (60, 45, 45, 45), 2, 60, 2, 45.0, seed=3)
    g.keygen([])
    x = g.encrypt_coeffs(np.zeros((256, g.N), np.int64), 4, g.scale)   # 256 MiB of ciphertexts
    x.free()
    g.synchronize()
    held, _ = torch.cuda.mem_get_info()
    assert held < free0 - (200 << 20)       # still cached after the free
    g.close()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 > held + (200 << 20)
    assert free1 > free0 - (64 << 20)


def test_table1_network_single_ciphertext(lib):
    """Table I's CNN (CONV, ACT-1, FC-1, ACT-2, FC-2) in the paper's single-ciphertext layout at a
    reduced size (N = 2^11: 16 images of 6 x 6 in 8 x 8 blocks, 2 kernels 3 x 3, FC-1 from 2 x 4 x 4
    inputs to 32 outputs in two groups of 16, FC-2 to 4 outputs), twelve levels: every stage
    bit-exact with the oracle from the same plaintexts and seeds (CONV per kernel after ACT-1, each
    FC-1 group, FC-1 with its bias, ACT-2, FC-2 with its bias), the logits within 1e-3 of FP64;
    then the network from the library's own encoders (table1.encrypt_model / forward) against
    FP64."""
    from paper_2512_18646_gb300 import table1
    geo = table1.Geometry(h=6, w=6, k=3, Hb=8, Wb=8, channels=2, fc1_out=32, fc2_out=4, slots=1024)
    o, g = make_pair(11, (60,) + (40,) * 12, 1, 60, 1, 40.0, seed=43, steps=table1.rotation_steps(geo))
    S, n, m, p1, p2 = o.slots, geo.n, geo.images, geo.p1, geo.p2
    assert (n, m, p1, p2) == (64, 16, 16, 4)
    wts = synthetic.table1_weights(h=6, w=6, c=2, k=3, fc1_out=32, fc2_out=4, seed=44)
    imgs = synthetic.images(m, 6, 6, seed=45)
    lp = o.L1

    def mm_masks(limbs, p):
        mv = layouts.vr_matmul_masks(m, n, p, S)
        return np.stack([o.encode(mv[0], float(o.q[limbs - 2]))] +
                        [o.encode(v, float(o.q[limbs - 3])) for v in mv[1:]])

    ox, gx = encrypt_both(o, g, encode_columns(o, layouts.vr_images(imgs, S, 8, 8)), ct_id_base=0)
    cmasks = np.stack([o.encode(v, float(o.q[lp - 2])) for v in layouts.vr_masks(3, 6, 6, S, 8, 8)])
    ys_o, ys_g = [], []
    s1 = None
    for c in range(2):
        ks = layouts.vr_kernelspanner(wts.conv_w[c], 6, 6, S, 8, 8)
        ms = np.stack([o.encode(v, float(o.q[lp - 1])) for v in ks])
        os_, gs = encrypt_both(o, g, ms, ct_id_base=20 + 10 * c, scale=float(o.q[lp - 1]))
        mb = o.encode(layouts.vr_bias(float(wts.conv_b[c]), 3, 6, 6, S, 8, 8))[None]
        ob, gb = encrypt_both(o, g, mb, limbs=lp - 2, ct_id_base=90 + c)
        gy = g.vr_conv2d_coeffs(gx, gs, gb, 3, 8, cmasks)
        g.relinearize(g.poly_act(gy, table1.ACT1))
        oy3, s1 = o.poly_act3(o.vr_conv2d(ox, os_, ob[0], 3, 8, cmasks), table1.ACT1, o.scale)
        oy = o.relin(oy3[0])
        assert np.array_equal(gy.export()[0], oy), c
        ys_o.append(oy)
        ys_g.append(gy)
    l1 = lp - 4
    B1 = table1.fc1_blocks(geo, wts.fc1_w)
    masks1 = mm_masks(l1, p1)
    oz, gz = None, None
    for t in range(B1.shape[1]):
        ozt, gzt = None, None
        for c in range(2):
            obb, gbb = encrypt_both(o, g, encode_columns(o, layouts.vr_matrix_b(B1[c, t], S)[None]),
                                    ct_id_base=200 + 10 * c + t)
            gbd = g.drop_levels(gbb, l1)
            assert gbd.limbs == l1 and gbd.scale == gbb.scale
            op = o.vr_matmul(ys_o[c], obb[0][:, :l1], n, p1, masks1)
            gp = g.vr_matmul_coeffs(ys_g[c], gbd, m, n, p1, masks1)
            ozt = op if ozt is None else o.add(ozt, op)
            gzt = gp if gzt is None else g.add(gzt, gp)
        if t > 0:
            ozt = o.rotate(ozt, [-t * p1])[0]
            gzt = g.rotate(gzt, [-t * p1])
        assert np.array_equal(gzt.export()[0], ozt), t
        oz = ozt if oz is None else o.add(oz, ozt)
        gz = gzt if gz is None else g.add(gz, gzt)
    sz = (s1 * o.scale) / float(o.q[l1 - 1])
    assert gz.scale == sz
    mb1 = o.encode(table1.row_vector(geo, wts.fc1_b), sz)
    oz = o.add_plain(oz, mb1)
    g.add_plain_coeffs(gz, mb1)
    assert np.array_equal(gz.export()[0], oz)
    oa3, s2 = o.poly_act3(oz[None], table1.ACT2, sz)
    oa = o.relin(oa3[0])
    g.relinearize(g.poly_act(gz, table1.ACT2))
    assert np.array_equal(gz.export()[0], oa)
    l2 = l1 - 5
    ob2, gb2 = encrypt_both(o, g, encode_columns(o, layouts.vr_matrix_b(table1.fc2_block(geo, wts.fc2_w), S)[None]),
                            ct_id_base=300)
    masks2 = mm_masks(l2, p2)
    oo = o.vr_matmul(oa, ob2[0][:, :l2], n, p2, masks2)
    go = g.vr_matmul_coeffs(gz, g.drop_levels(gb2, l2), m, n, p2, masks2)
    so = (s2 * o.scale) / float(o.q[l2 - 1])
    mb2 = o.encode(table1.row_vector(geo, wts.fc2_b), so)
    oo = o.add_plain(oo, mb2)
    g.add_plain_coeffs(go, mb2)
    assert go.limbs == 1
    assert np.array_equal(go.export()[0], oo)
    ref = fp64_ref.table1_cnn(imgs, wts, table1.ACT1, table1.ACT2)
    assert np.abs(table1.logits(g, geo, go) - ref).max() < 1e-3
    # the library's own encoders end to end
    model = table1.encrypt_model(g, geo, wts)
    out = table1.forward(g, geo, g.vr_encrypt_images(imgs, 8, 8, 0), model)
    assert np.abs(table1.logits(g, geo, out) - ref).max() < 1e-3


def test_plaintext_add_and_drop_levels(lib):
    """Add with a plaintext operand and modulus dropping: bit-exact with the oracle from the same
    plaintexts and seeds (two and three components, one plaintext for the set or one per
    ciphertext), the slots decrypting to the sums; dropped sets keep their scale and decrypt to the
    same values; argument and level errors."""
    from paper_2512_18646_gb300 import HeError
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_E_LEVEL
    o, g = make_pair(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=47, steps=())
    S = o.slots
    rng = np.random.default_rng(48)
    x, v = rng.uniform(-1, 1, (3, S)), rng.uniform(-1, 1, (3, S))
    ox, gx = encrypt_both(o, g, encode_columns(o, x), ct_id_base=5)
    mv = encode_columns(o, v)
    # one plaintext per ciphertext
    g.add_plain_coeffs(gx, mv)
    want = np.stack([o.add_plain(ox[i], mv[i]) for i in range(3)])
    assert np.array_equal(gx.export(), want)
    assert np.abs(g.decrypt_slots(gx) - (x + v)).max() < 1e-6
    # one plaintext for the set, on a three-component product
    d = g.mul(gx, gx)
    od = np.stack([o.rescale(o.tensor(want[i], want[i])) for i in range(3)])
    assert np.array_equal(d.export(), od)
    g.add_plain_coeffs(d, mv[0])
    assert np.array_equal(d.export(), np.stack([o.add_plain(od[i], mv[0]) for i in range(3)]))
    # the library's own encoding at the set's scale
    y = g.encrypt_coeffs(encode_columns(o, x), o.L1, o.scale, 40)
    g.add_slots(y, v[1])
    assert np.abs(g.decrypt_slots(y) - (x + v[1])).max() < 1e-6
    # dropping primes: the same residues, the same scale, the same values
    low = g.drop_levels(y, 2)
    assert low.limbs == 2 and low.scale == y.scale
    full = y.export().reshape(3, 2, o.L1, o.N)
    assert np.array_equal(low.export().reshape(3, 2, 2, o.N), full[:, :, :2])
    assert np.abs(g.decrypt_slots(low) - (x + v[1])).max() < 1e-6
    for bad in (0, o.L1 + 1):
        with pytest.raises(HeError) as e:
            g.drop_levels(y, bad)
        assert e.value.code == HE_E_LEVEL
    with pytest.raises(HeError) as e:
        g.add_plain_coeffs(y, mv[:2])  # two plaintexts for three ciphertexts
    assert e.value.code == HE_E_ARG


def test_key_checkpoint_moves_keys_between_contexts(lib):
    """he_keys_export / he_keys_import: a context with the same parameters but another seed takes the
    first one's keys from the checkpoint, then decrypts the first one's ciphertexts and rotates and
    multiplies them to the same words. Other parameters, a truncated checkpoint and a residue out of
    range are refused (HE_E_ARG), and the refused context keeps its own keys."""
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_E_STATE, HeError
    params = (10, (60, 45, 45, 45), 2, 60, 2, 45.0)
    a = api.Context(*params, seed=61)
    with pytest.raises(HeError) as e:
        a.export_keys()
    assert e.value.code == HE_E_STATE
    a.keygen([1, 5])
    words = a.export_keys()
    b = api.Context(*params, seed=62)
    b.import_keys(words)
    assert np.array_equal(b.export_keys(), words)
    A = np.random.default_rng(61).uniform(-1, 1, (7, 3))
    xa = a.encrypt_matrix_a(A, 0)
    xb = b.import_coeffs(xa.export(), xa.scale)
    assert np.abs(b.decrypt_slots(xb)[:, :7] - A.T).max() < 1e-6
    assert np.array_equal(b.rotate(xb, [1, 5]).export(), a.rotate(xa, [1, 5]).export())
    assert np.array_equal(b.relinearize(b.mul(xb, xb)).export(), a.relinearize(a.mul(xa, xa)).export())
    # refusals
    c = api.Context(10, (60, 45, 45, 45), 2, 60, 1, 45.0, seed=63)
    c.keygen([])
    own = c.export_keys()
    for bad in (words, words[:-5]):
        with pytest.raises(HeError) as e:
            c.import_keys(bad)
        assert e.value.code == HE_E_ARG
    bad = words.copy()
    bad[6 + len(a.primes) + 3] = np.uint64(1 << 63)  # a secret-key residue above its prime
    with pytest.raises(HeError) as e:
        b.import_keys(bad)
    assert e.value.code == HE_E_ARG
    assert np.array_equal(c.export_keys(), own)
