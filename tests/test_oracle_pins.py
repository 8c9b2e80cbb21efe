"""Pins of the CPU oracle against what the paper and the mathematics fix.

These run without a GPU. Each test checks the oracle against something other
than itself: textbook definitions evaluated with Python integers (schoolbook
negacyclic product, the NTT's defining sum, CRT lifts), closed forms (the
canonical-embedding sum), invariants (rotation = slot shift after decryption,
automorphisms are ring maps), the paper's worked examples
(tests/golden/*.txt) and the FP64 results the encrypted layers must decrypt to.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import sympy

from inputs import synthetic
from oracle import Oracle, fp64_ref, layouts, slot_sim
from tests.conftest import golden_path


def brv(x: int, bits: int) -> int:
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.fixture(scope="module")
def small():
    o = Oracle(5, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=11)
    o.keygen([1, 2, 3, 5, -1, 7])
    return o


@pytest.fixture(scope="module")
def hybrid():
    # two special primes, digits of two primes (the CNN parameter shape), small ring
    o = Oracle(6, (60, 45, 45, 45, 45), 2, 60, 2, 45.0, seed=5)
    o.keygen([1, 2, 4])
    return o


# ---------------------------------------------------------------------------
# Prime chain and roots
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log_n,q_bits,K,sb", [(13, (60, 40, 40), 1, 60), (16, (60,) + (45,) * 12, 2, 60),
                                               (15, (60,) + (40,) * 8, 1, 60)])
def test_prime_chain_rule(log_n, q_bits, K, sb):
    o = Oracle(log_n, q_bits, K, sb, 1 if K == 1 else 2, 40.0)
    two_n = 2 * (1 << log_n)
    assert len(set(o.primes)) == len(o.primes)
    for q, b in zip(o.primes, list(q_bits) + [sb] * K):
        assert sympy.isprime(q)
        assert q % two_n == 1
        assert q.bit_length() == b
    # the specials are the largest candidates of their size, q_0 the next one
    cands = [(1 << sb) - t * two_n + 1 for t in range(1, 2000)]
    primes_sb = [c for c in cands if sympy.isprime(c)]
    assert o.p == primes_sb[:K]
    if q_bits[0] == sb:
        assert o.q[0] == primes_sb[K]
    # q_1..q_L: the largest unused candidates of their size, in order
    b = q_bits[1]
    cands_b = [c for c in ((1 << b) - t * two_n + 1 for t in range(1, 4000)) if sympy.isprime(c)]
    same = [q for q, bb in zip(o.q[1:], q_bits[1:]) if bb == b]
    assert b != sb and same == cands_b[: len(same)]


def test_psi_is_primitive_2n_root(small):
    for pi, q in enumerate(small.primes):
        psi = small.psi(pi)
        assert pow(psi, small.N, q) == q - 1
        # the root comes from the smallest quadratic non-residue
        x = next(x for x in range(2, 1000) if pow(x, (q - 1) // 2, q) == q - 1)
        assert psi == pow(x, (q - 1) // (2 * small.N), q)


# ---------------------------------------------------------------------------
# P1: NTT against its defining sum and against the schoolbook product
# ---------------------------------------------------------------------------
def test_ntt_matches_definition(small):
    rng = np.random.default_rng(0)
    N, bits = small.N, small.log_n
    for pi, q in enumerate(small.primes):
        a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
        psi = small.psi(pi)
        ref = [sum(a[i] * pow(psi, (2 * brv(j, bits) + 1) * i, q) for i in range(N)) % q for j in range(N)]
        got = small.ntt(np.array(a, dtype=np.uint64), pi)
        assert [int(x) for x in got] == ref
        assert [int(x) for x in small.ntt(got, pi, inverse=True)] == a


def schoolbook_negacyclic(a, b, q):
    N = len(a)
    r = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                r[k] += a[i] * b[j]
            else:
                r[k - N] -= a[i] * b[j]
    return [x % q for x in r]


@pytest.mark.parametrize("log_n", [4, 6])
def test_polymul_matches_schoolbook(log_n):
    o = Oracle(log_n, (60, 40, 45), 2, 60, 1, 40.0)
    rng = np.random.default_rng(log_n)
    for pi, q in enumerate(o.primes):
        a = [int(x) for x in rng.integers(0, q, o.N, dtype=np.uint64)]
        b = [int(x) for x in rng.integers(0, q, o.N, dtype=np.uint64)]
        got = o.polymul(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64), pi)
        assert [int(x) for x in got] == schoolbook_negacyclic(a, b, q)


def test_automorphism_is_ring_map(small):
    rng = np.random.default_rng(3)
    q = small.q[1]
    a = rng.integers(0, q, small.N, dtype=np.uint64)
    b = rng.integers(0, q, small.N, dtype=np.uint64)
    for step in (1, 2, 5):
        k = small.galois_elt(step)
        assert k == pow(5, step, 2 * small.N)
        lhs = small.automorph(small.polymul(a, b, 1), k, 1)
        rhs = small.polymul(small.automorph(a, k, 1), small.automorph(b, k, 1), 1)
        assert np.array_equal(lhs, rhs)
    k1, k2 = small.galois_elt(1), small.galois_elt(2)
    assert np.array_equal(small.automorph(small.automorph(a, k1, 1), k2, 1),
                          small.automorph(a, (k1 * k2) % (2 * small.N), 1))
    # definition on X: X -> X^k, with X^N = -1
    x = np.zeros(small.N, np.uint64)
    x[1] = 1
    k = small.galois_elt(3)
    e = k % (2 * small.N)
    y = small.automorph(x, k, 1)
    exp = np.zeros(small.N, np.uint64)
    if e < small.N:
        exp[e] = 1
    else:
        exp[e - small.N] = q - 1
    assert np.array_equal(y, exp)


# ---------------------------------------------------------------------------
# P2: base conversion, ModDown and rescale against big-integer CRT lifts
# ---------------------------------------------------------------------------
def crt(res, mods):
    M = math.prod(mods)
    x = 0
    for r, m in zip(res, mods):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M


def test_modup_is_crt_lift_plus_small_multiple(hybrid):
    o = hybrid
    rng = np.random.default_rng(7)
    lp = 4  # three digits at alpha = 2: {q0,q1}, {q2,q3}
    x = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.q[:lp]])
    basis = o.q[:lp] + o.p
    for j in range(2):
        I = list(range(2 * j, min(2 * j + 2, lp)))
        D = math.prod(o.q[i] for i in I)
        ext = o.modup(x, j)
        for n in range(0, o.N, 7):
            X = crt([x[i][n] for i in I], [o.q[i] for i in I])
            ok = False
            for u in range(len(I)):
                if all(int(ext[pos][n]) == (X + u * D) % t for pos, t in enumerate(basis)):
                    ok = True
            assert ok, (j, n)


def test_moddown_is_division_by_p(hybrid):
    o = hybrid
    rng = np.random.default_rng(8)
    lp = 3
    basis = o.q[:lp] + o.p
    u = np.stack([rng.integers(0, t, o.N, dtype=np.uint64) for t in basis])
    out = o.moddown(u)
    Q = math.prod(o.q[:lp])
    P = math.prod(o.p)
    for n in range(0, o.N, 5):
        U = crt([u[i][n] for i in range(len(basis))], basis)
        UP = U % P
        ok = False
        for e in range(o.K):
            V = ((U - UP) // P - e) % Q
            if all(int(out[i][n]) == V % q for i, q in enumerate(o.q[:lp])):
                ok = True
        assert ok, n


def test_rescale_rounds_half_up(small):
    o = small
    rng = np.random.default_rng(9)
    lp = 4
    ct = np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.q[:lp]]) for _ in range(2)])
    out = o.rescale(ct)
    ql = o.q[lp - 1]
    Q = math.prod(o.q[:lp])
    for t in range(2):
        for n in range(o.N):
            X = crt([ct[t][i][n] for i in range(lp)], o.q[:lp])
            V = ((X + ql // 2) // ql) % (Q // ql)
            assert [int(out[t][i][n]) for i in range(lp - 1)] == [V % q for q in o.q[: lp - 1]]


# ---------------------------------------------------------------------------
# P3: encoding (canonical embedding) and encryption
# ---------------------------------------------------------------------------
def test_encode_matches_embedding_sum():
    o = Oracle(5, (60, 40), 1, 60, 1, 30.0)
    N, S = o.N, o.slots
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, S)
    m = o.encode(z)
    zeta = np.exp(1j * np.pi / N)
    e = [pow(5, j, 2 * N) for j in range(S)]
    for k in range(N):
        val = o.scale * (2.0 / N) * sum(z[j] * zeta ** (-e[j] * k) for j in range(S)).real
        assert abs(m[k] - val) <= 0.5 + 1e-6
    # m(zeta^(5^j)) = scale * z_j
    for j in range(S):
        ev = sum(int(m[k]) * zeta ** (e[j] * k) for k in range(N))
        assert abs(ev / o.scale - z[j]) < 1e-8


def test_decode_inverts_encode():
    o = Oracle(12, (60, 40), 1, 60, 1, 40.0)
    z = np.random.default_rng(2).uniform(-1, 1, o.slots)
    assert np.abs(o.decode(o.encode(z).astype(float)) - z).max() < 1e-9


def test_secret_is_ternary(small):
    s = small.secret()
    assert set(np.unique(s)).issubset({-1, 0, 1})
    counts = [int((s == v).sum()) for v in (-1, 0, 1)]
    assert min(counts) > 0


def test_encrypt_decrypt(small):
    z = np.random.default_rng(3).uniform(-1, 1, small.slots)
    m = small.encode(z)
    for limbs in (4, 2, 1):
        ct = small.encrypt(m, limbs, ct_id=limbs)
        assert np.abs(small.decrypt(ct) - z).max() < 1e-6
        # the error in the coefficient domain is small and not zero
        err = small.decrypt_coeffs(ct) - m
        assert 0 < np.abs(err).max() < 200
    # distinct ciphertext ids draw distinct randomness
    a, b = small.encrypt(m, 4, 1), small.encrypt(m, 4, 2)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, small.encrypt(m, 4, 1))


# ---------------------------------------------------------------------------
# P4 / P5: Rot, key switching, Mul, cMul (Sec. II-A)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fx", ["small", "hybrid"])
def test_rotation_is_left_shift(fx, request):
    o = request.getfixturevalue(fx)
    z = np.random.default_rng(4).uniform(-1, 1, o.slots)
    ct = o.encrypt(o.encode(z), ct_id=3)
    steps = [0, 1, 2] if fx == "hybrid" else [0, 1, 3, 5, -1, 7]
    r = o.rotate(ct, steps)
    for t, s in enumerate(steps):
        assert np.abs(o.decrypt(r[t]) - np.roll(z, -s)).max() < 1e-6, s
    # a wrong direction would fail
    assert np.abs(o.decrypt(r[1]) - np.roll(z, steps[1])).max() > 1e-2


@pytest.mark.parametrize("fx", ["small", "hybrid"])
def test_keyswitch_noise_is_small(fx, request):
    o = request.getfixturevalue(fx)
    rng = np.random.default_rng(6)
    for lp in (o.L1, 2):
        x = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.q[:lp]])
        negx = np.stack([(np.uint64(q) - x[i]) % np.uint64(q) for i, q in enumerate(o.q[:lp])])
        v = o.keyswitch(x, 0)
        e = o.decrypt_coeffs(np.stack([v[0], v[1], negx]))  # v0 + v1 s - x s^2
        assert np.abs(e).max() < 2000


def test_tensor_relin_rescale(small):
    rng = np.random.default_rng(5)
    x, y = rng.uniform(-1, 1, small.slots), rng.uniform(-1, 1, small.slots)
    a = small.encrypt(small.encode(x), ct_id=10)
    b = small.encrypt(small.encode(y), ct_id=11)
    d = small.tensor(a, b)
    assert np.abs(small.decrypt(d, small.scale ** 2) - x * y).max() < 1e-6
    r = small.relin(d)
    assert np.abs(small.decrypt(r, small.scale ** 2) - x * y).max() < 1e-6
    s = small.rescale(r)
    assert np.abs(small.decrypt(s, small.scale ** 2 / small.q[-1]) - x * y).max() < 1e-6
    # Add
    assert np.abs(small.decrypt(small.add(a, b)) - (x + y)).max() < 1e-6


def test_cmul_scalar_and_plain(small):
    rng = np.random.default_rng(12)
    x, w = rng.uniform(-1, 1, small.slots), rng.uniform(-1, 1, small.slots)
    a = small.encrypt(small.encode(x), ct_id=20)
    ql = small.q[-1]
    r = small.rescale(small.mul_scalar(a, round(0.37 * ql)))
    assert np.abs(small.decrypt(r) - 0.37 * x).max() < 1e-6
    r = small.rescale(small.mul_plain(a, small.encode(w, float(ql))))
    assert np.abs(small.decrypt(r) - w * x).max() < 1e-6


def test_add_plain_adds_slots(small):
    """Add with a plaintext operand decrypts to the slotwise sum; a plaintext that is not reduced
    modulo the primes (a negative constant) is taken modulo each prime."""
    rng = np.random.default_rng(13)
    x, v = rng.uniform(-1, 1, small.slots), rng.uniform(-1, 1, small.slots)
    a = small.encrypt(small.encode(x), ct_id=21)
    assert np.abs(small.decrypt(small.add_plain(a, small.encode(v))) - (x + v)).max() < 1e-6
    c = np.full(small.slots, -0.75)
    assert np.abs(small.decrypt(small.add_plain(a, small.encode(c))) - (x - 0.75)).max() < 1e-6
    # adding to component 1 instead would not decrypt to the sum: the pin sees the component
    wrong = a.copy()
    wrong[1] = small.add_plain(a[1:2], small.encode(v))[0]
    assert np.abs(small.decrypt(wrong) - (x + v)).max() > 1e-2


# ---------------------------------------------------------------------------
# Paper's worked examples in the plaintext slot simulator (P8, P9)
# ---------------------------------------------------------------------------
def read_blocks(name):
    blocks, cur, tag = [], None, None
    for line in open(golden_path(name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("matrix", "bias"):
            cur = []
            blocks.append((line, cur))
            continue
        row = [int(v) for v in line.split()]
        if cur is None:
            cur = []
            blocks.append(("matrix", cur))
        cur.append(row)
    return [(t, np.array(m)) for t, m in blocks]


def test_sumforconv_worked_example():
    flags = read_blocks("sumforconv_h4_w4_k3.txt")[0][1]
    Z = np.random.default_rng(0).uniform(-1, 1, (4, 4))
    got = (slot_sim.sum_for_conv(Z.reshape(-1), 4, 4, 3) * slot_sim.valid_mask(4, 4, 3)).reshape(4, 4)
    for i in range(4):
        for j in range(4):
            exp = Z[i:i + 3, j:j + 3].sum() if flags[i, j] else 0.0
            assert abs(got[i, j] - exp) < 1e-12
    # the literal text (row pass on the input) does not give the printed box sums
    lit = (slot_sim.sum_for_conv(Z.reshape(-1), 4, 4, 3, separable=False) * slot_sim.valid_mask(4, 4, 3)).reshape(4, 4)
    assert abs(lit[0, 0] - Z[0:3, 0:3].sum()) > 1e-6


def test_kernelspanner_worked_example():
    blocks = read_blocks("kernelspanner_h4_w4_k2.txt")
    kv = {1: 2.0, 2: 3.0, 3: 5.0, 4: 7.0, 5: 11.0}
    K = np.array([[kv[1], kv[2]], [kv[3], kv[4]]])
    sim = slot_sim.kernelspanner(K, 4, 4)
    expect = [np.vectorize(lambda e: kv.get(e, 0.0))(m) for t, m in blocks if t == "matrix"]
    assert len(expect) == len(sim) == 4
    for E in expect:
        assert any(np.array_equal(E, P) for P in sim.values())
    bias = [np.vectorize(lambda e: kv.get(e, 0.0))(m) for t, m in blocks if t == "bias"][0]
    assert np.array_equal(slot_sim.bias_block(kv[5], 4, 4, 2), bias)


@pytest.mark.parametrize("h,w,k", [(4, 4, 2), (6, 5, 3), (7, 7, 3), (9, 8, 4)])
def test_alg4_slot_simulation_is_convolution(h, w, k):
    rng = np.random.default_rng(h * 100 + w * 10 + k)
    I = rng.uniform(0, 1, (h, w))
    K = rng.normal(0, 1, (k, k))
    out = slot_sim.conv_alg4(I, K, 0.3)
    ref = fp64_ref.conv2d(I[None, None], K[None, None], [0.3], 1)[0, 0]
    assert np.abs(out[: h - k + 1, : w - k + 1] - ref).max() < 1e-12
    assert np.abs(out[h - k + 1:, :]).max() == 0 and np.abs(out[:, w - k + 1:]).max() == 0


def test_multi_ct_layouts_in_slot_simulator():
    rng = np.random.default_rng(2)
    A = rng.uniform(-1, 1, (6, 5))
    Bm = rng.uniform(-1, 1, (5, 4))
    D = slot_sim.matmul_multi_ct(A, Bm, 64)
    assert np.abs(layouts.matmul_from_diagonals(D, 6, 4) - A @ Bm).max() < 1e-12
    imgs = rng.uniform(0, 1, (2, 3, 11, 9))
    K = rng.normal(0, 1, (4, 3, 3, 3))
    bias = rng.normal(0, 1, 4)
    for stride in (1, 2):
        Y = slot_sim.conv_columns(imgs, K, bias, stride, 64, 16)
        ref = fp64_ref.conv2d(imgs, K, bias, stride)
        got = np.moveaxis(layouts.image_from_columns(Y, 2, 16, stride, ref.shape[2]), 0, 1)
        # [O][B][h][w] -> [B][O][h][w]
        assert np.abs(got - ref).max() < 1e-12


# ---------------------------------------------------------------------------
# P6 / P7: encrypted layers decrypt to the FP64 results
# ---------------------------------------------------------------------------
def test_matmul_config_small_matches_fp64():
    pre = synthetic.MATMUL_SMALL
    o = Oracle.from_preset(pre, seed=101)
    A, Bm = synthetic.matmul_operands(4, 8, 4, seed=101)
    o.keygen(list(range(1, 4)))
    Ac = np.stack([o.encrypt(o.encode(v), ct_id=i) for i, v in enumerate(layouts.matrix_a_columns(A, o.slots))])
    Bc = np.stack([o.encrypt(o.encode(v), ct_id=100 + i) for i, v in enumerate(layouts.matrix_b_rows(Bm, o.slots))])
    o.reset_counters()
    D = o.matmul(Ac, Bc, 4)
    sc = o.scale ** 2 / o.q[-1]
    C = layouts.matmul_from_diagonals(np.stack([o.decrypt(d, sc) for d in D]), 4, 4)
    assert np.abs(C - A @ Bm).max() < 1e-4
    assert np.abs(C - A @ Bm).max() < 1e-6
    # P10: n (p-1) rotations from n hoisted ModUps, n p tensors, p relins, p rescales
    c = o.counters()
    assert c["rotations"] == 8 * 3 and c["tensors"] == 32 and c["relins"] == 4 and c["rescales"] == 4
    assert c["modups"] == 8 + 4  # one per B~_k, one per relinearisation


def test_matmul_rectangular_detects_transposition():
    o = Oracle(8, (60, 40, 40), 1, 60, 1, 40.0, seed=3)
    o.keygen(list(range(1, 8)))
    rng = np.random.default_rng(4)
    A, Bm = rng.uniform(-1, 1, (5, 3)), rng.uniform(-1, 1, (3, 8))
    Ac = np.stack([o.encrypt(o.encode(v), ct_id=i) for i, v in enumerate(layouts.matrix_a_columns(A, o.slots))])
    Bc = np.stack([o.encrypt(o.encode(v), ct_id=50 + i) for i, v in enumerate(layouts.matrix_b_rows(Bm, o.slots))])
    D = o.matmul(Ac, Bc, 8)
    C = layouts.matmul_from_diagonals(np.stack([o.decrypt(d, o.scale ** 2 / o.q[-1]) for d in D]), 5, 8)
    assert np.abs(C - A @ Bm).max() < 1e-6


@pytest.mark.parametrize("slots,m,n,p", [(64, 5, 3, 8), (64, 4, 2, 4), (32, 3, 5, 16), (64, 9, 2, 1),
                                          (4096, 17, 4, 64), (32768, 256, 3, 256), (32768, 16, 2, 256)])
def test_volley_layout_is_gemm_in_slots(slots, m, n, p):
    """Zero-rotation matmul layout: block geometry, and the slotwise sum of products of A's
    volley encoding with B's period-p rows decodes to A @ B (plaintext slots, exact up to fp)."""
    M, per, G, off = layouts.volley_geometry(slots, m, p)
    assert M >= m and (M - 1) % p == 0 and G == -(-p // per)
    covered = []
    for g in range(G):
        cnt = min(per, p - g * per)
        assert cnt >= 1 and (cnt - 1) * M + off[g] + m <= slots
        assert off[g] == (g * per) % p
        covered += [g * per + t for t in range(cnt)]
    assert covered == list(range(p))
    rng = np.random.default_rng(slots + m + p)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    Ah = layouts.matrix_a_volley(A, slots, p)
    Bt = layouts.matrix_b_rows(Bm, slots)
    assert Ah.shape == (G, n, slots)
    # each group holds m * cnt nonzero slots per column ciphertext, nothing else
    assert all(np.count_nonzero(Ah[g, 0]) == m * min(per, p - g * per) for g in range(G))
    d = np.stack([(Ah[g] * Bt).sum(0) for g in range(G)])
    assert np.abs(layouts.matmul_from_volley(d, m, p) - A @ Bm).max() < 1e-12
    # a transposed operand is caught
    if m == n and m > 1:
        d2 = np.stack([(layouts.matrix_a_volley(A.T, slots, p)[g] * Bt).sum(0) for g in range(G)])
        assert np.abs(layouts.matmul_from_volley(d2, m, p) - A @ Bm).max() > 1e-3


@pytest.mark.parametrize("m,n,p", [(5, 3, 8), (20, 2, 16)])
def test_matmul_volley_encrypted_matches_fp64_without_rotations(m, n, p):
    """Encrypted zero-rotation matmul: decrypts to A @ B; G n tensors, G relins, no rotation."""
    o = Oracle(8, (60, 40, 40), 1, 60, 1, 40.0, seed=5)
    o.keygen([])
    rng = np.random.default_rng(m + n + p)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    M, per, G, off = layouts.volley_geometry(o.slots, m, p)
    Ah = layouts.matrix_a_volley(A, o.slots, p)
    Ac = np.stack([[o.encrypt(o.encode(Ah[g, k]), ct_id=g * n + k) for k in range(n)] for g in range(G)])
    Bc = np.stack([o.encrypt(o.encode(v), ct_id=50 + i) for i, v in enumerate(layouts.matrix_b_rows(Bm, o.slots))])
    o.reset_counters()
    D = o.matmul_volley(Ac, Bc)
    c = o.counters()
    assert c["rotations"] == 0 and c["tensors"] == G * n and c["relins"] == G and c["rescales"] == G
    C = layouts.matmul_from_volley(np.stack([o.decrypt(d, o.scale ** 2 / o.q[-1]) for d in D]), m, p)
    assert np.abs(C - A @ Bm).max() < 1e-6
    if m == 20:
        assert G > 1  # the second case splits the positions into groups


def act_polynomials():
    """Table I's ACT-1 / ACT-2 coefficients from the golden fixture: {name: [c0, c1, c2, c3]}."""
    out = {}
    for line in open(golden_path("act_polynomials_table1.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out[f[0]] = [float(v) for v in f[1:]]
    return out


def test_act_fixture_matches_table1():
    acts = act_polynomials()
    assert set(acts) == {"ACT-1", "ACT-2"} and all(len(c) == 4 for c in acts.values())
    assert acts["ACT-1"][2] == 2.0225089 and acts["ACT-2"][0] == -1.5650465


@pytest.mark.parametrize("name,coeffs", [("ACT-1", None), ("ACT-2", None), ("x^2", [0, 0, 1, 0]),
                                         ("const", [0.75, 0, 0, 0]), ("identity", [0, 1, 0, 0]),
                                         ("cube", [0, 0, 0, 1])])
def test_poly_act3_decrypts_to_polynomial(name, coeffs):
    """Degree-3 activation (Table I's ACT layers): decrypts to c0 + c1 x + c2 x^2 + c3 x^3 at every
    slot, two levels consumed, three components out; also from a three-component input."""
    c = act_polynomials()[name] if coeffs is None else coeffs
    o = Oracle(10, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=21)
    o.keygen([])
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (2, o.slots))
    X = np.stack([o.encrypt(o.encode(v), ct_id=i) for i, v in enumerate(x)])
    o.reset_counters()
    Y, sy = o.poly_act3(X, c, o.scale)
    cnt = o.counters()
    assert Y.shape == (2, 3, o.L1 - 2, o.N)
    assert cnt["tensors"] == 4 and cnt["rescales"] == 8 and cnt["relins"] == 2 and cnt["ct_scalar"] == 4
    want = c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3
    got = np.stack([o.decrypt(o.relin(y), sy) for y in Y])
    assert np.abs(got - want).max() < 1e-6
    # a three-component input (an unrelinearised product) is relinearised first
    sq = o.rescale(o.tensor(X[0], X[0]))
    s2 = o.scale * o.scale / o.q[o.L1 - 1]
    Y2, sy2 = o.poly_act3(sq[None], c, s2)
    x2 = x[0] ** 2
    got2 = o.decrypt(o.relin(Y2[0]), sy2)
    assert np.abs(got2 - (c[0] + c[1] * x2 + c[2] * x2 ** 2 + c[3] * x2 ** 3)).max() < 1e-5


def test_poly_act3_dropped_term_is_caught():
    """Planted mistake check: a wrong coefficient order (c3 <-> c2) changes the result."""
    o = Oracle(9, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=22)
    o.keygen([])
    x = np.random.default_rng(4).uniform(-1, 1, o.slots)
    X = o.encrypt(o.encode(x), ct_id=0)[None]
    c = act_polynomials()["ACT-1"]
    Y, sy = o.poly_act3(X, [c[0], c[1], c[3], c[2]], o.scale)
    got = o.decrypt(o.relin(Y[0]), sy)
    assert np.abs(got - (c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3)).max() > 1e-2


@pytest.mark.parametrize("m,n,p,g", [(5, 3, 8, 4), (6, 2, 8, 3), (4, 4, 4, 1), (3, 2, 4, 4)])
def test_matmul_bsgs_matches_fp64_with_fewer_rotations(m, n, p, g):
    """Baby-step giant-step revolver: decrypts to A @ B and to the revolver's diagonals, with
    n(g-1) + n(ceil(p/g)-1) + (p - g) rotations (all outputs rotated back but the first g)."""
    o = Oracle(8, (60, 40, 40), 1, 60, 1, 40.0, seed=6)
    S = o.slots
    ng = -(-p // g)
    o.keygen(sorted(set(list(range(1, p)) + [S - g * i for i in range(1, ng)])))
    rng = np.random.default_rng(m * 10 + p + g)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    Ac = np.stack([o.encrypt(o.encode(v), ct_id=i) for i, v in enumerate(layouts.matrix_a_columns(A, S))])
    Bc = np.stack([o.encrypt(o.encode(v), ct_id=50 + i) for i, v in enumerate(layouts.matrix_b_rows(Bm, S))])
    o.reset_counters()
    D = o.matmul_bsgs(Ac, Bc, p, g)
    c = o.counters()
    assert c["rotations"] == n * (g - 1) + n * (ng - 1) + (p - min(g, p))
    assert c["tensors"] == n * p and c["relins"] == p
    sc = o.scale ** 2 / o.q[-1]
    C = layouts.matmul_from_diagonals(np.stack([o.decrypt(d, sc) for d in D]), m, p)
    assert np.abs(C - A @ Bm).max() < 1e-6


@pytest.mark.parametrize("gap,h,H", [(2, 5, 16), (4, 3, 16), (2, 8, 16)])
def test_reform_compacts_rows(gap, h, H):
    """ReForm (Sec. IV-C) in the column layout: rows at slots b H + gap i move to b H + i, every other
    slot becomes 0; h - 1 rotations (one hoisted ModUp), h plaintext products, one rescale."""
    o = Oracle(8, (60, 40, 40), 1, 60, 1, 40.0, seed=26)
    steps = [(gap - 1) * i for i in range(1, h)]
    o.keygen(steps)
    rng = np.random.default_rng(gap * 10 + h)
    B = o.slots // H
    rows = rng.uniform(-1, 1, (B, h))
    z = np.zeros(o.slots)
    for b in range(B):
        z[b * H + gap * np.arange(h)] = rows[b]
        z[b * H + gap * h - 1] = 5.0  # an invalid slot (between rows) must not leak
    X = o.encrypt(o.encode(z), ct_id=0)[None]
    masks = o.reform_masks(h, H, o.L1)
    o.reset_counters()
    Y = o.reform(X, gap, h, masks)
    c = o.counters()
    assert c["rotations"] == h - 1 and c["modups"] == 1 and c["ct_plain"] == h and c["rescales"] == 1
    got = o.decrypt(Y[0])
    want = np.zeros(o.slots)
    for b in range(B):
        want[b * H: b * H + h] = rows[b]
    assert np.abs(got - want).max() < 1e-6


def _vr_conv_slots(x, P, F, bias_v, k, Wb):
    """Alg. 4 on slot vectors (the slot simulator's steps, several image blocks at once)."""
    acc = bias_v.copy()
    for t in range(k * k):
        acc = acc + slot_sim.sum_for_conv(x * P[t], 0, Wb, k) * F[t]
    return acc


@pytest.mark.parametrize("h,w,k,Hb,Wb", [(6, 5, 3, 8, 8), (7, 7, 2, 8, 8), (5, 6, 3, 8, 16)])
def test_vr_layout_alg4_over_virtual_images(h, w, k, Hb, Wb):
    """Alg. 4 over several images in one slot vector (row-major blocks of Hb x Wb, Sec. III-D):
    every image's valid output equals its FP64 convolution plus the bias; invalid positions hold 0."""
    slots = 256
    rng = np.random.default_rng(h * 10 + k)
    B = slots // (Hb * Wb)
    imgs = rng.uniform(0, 1, (B, h, w))
    K = rng.normal(0, 0.5, (k, k))
    k0 = 0.3
    x = layouts.vr_images(imgs, slots, Hb, Wb)[0]
    P = layouts.vr_kernelspanner(K, h, w, slots, Hb, Wb)
    F = layouts.vr_masks(k, h, w, slots, Hb, Wb)
    bias_v = layouts.vr_bias(k0, k, h, w, slots, Hb, Wb)
    out = _vr_conv_slots(x, P, F, bias_v, k, Wb)
    got = layouts.vr_images_from(out[None], B, h, w, Hb, Wb)
    ref = fp64_ref.conv2d(imgs[:, None], K[None, None], np.array([k0]), 1)[:, 0]
    ho, wo = h - k + 1, w - k + 1
    assert np.abs(got[:, :ho, :wo] - ref).max() < 1e-12
    assert np.abs(got[:, ho:, :]).max() < 1e-12 and np.abs(got[:, :, wo:]).max() < 1e-12


def test_vr_conv2d_encrypted_matches_fp64():
    """Alg. 4 encrypted over virtual images (the paper's single-ciphertext convolution): kernel
    ciphertexts at scale q_l, masks at scale q_{l-1}, encrypted bias; decrypts to FP64; k^2 tensor
    products and relinearisations, 2 k^2 (k-1) rotations from 2 k^2 hoisted ModUps."""
    o = Oracle(9, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=28)
    h, w, k, Hb, Wb = 6, 6, 3, 8, 8
    o.keygen(list(range(1, k)) + [Wb * p for p in range(1, k)])
    S = o.slots
    rng = np.random.default_rng(5)
    B = S // (Hb * Wb)
    imgs = rng.uniform(0, 1, (B, h, w))
    K = rng.normal(0, 0.5, (k, k))
    k0 = -0.2
    lp = o.L1
    X = o.encrypt(o.encode(layouts.vr_images(imgs, S, Hb, Wb)[0]), lp, 0)[None]
    Sct = np.stack([o.encrypt(o.encode(v, float(o.q[lp - 1])), lp, 10 + t)
                    for t, v in enumerate(layouts.vr_kernelspanner(K, h, w, S, Hb, Wb))])
    bias = o.encrypt(o.encode(layouts.vr_bias(k0, k, h, w, S, Hb, Wb)), lp - 2, 99)
    masks = np.stack([o.encode(v, float(o.q[lp - 2])) for v in layouts.vr_masks(k, h, w, S, Hb, Wb)])
    o.reset_counters()
    Y = o.vr_conv2d(X, Sct, bias, k, Wb, masks)
    c = o.counters()
    assert c["tensors"] == k * k and c["relins"] == k * k and c["ct_plain"] == k * k
    assert c["rotations"] == 2 * k * k * (k - 1) and c["modups"] == 2 * k * k + k * k
    got = layouts.vr_images_from(o.decrypt(Y[0])[None], B, h, w, Hb, Wb)
    ref = fp64_ref.conv2d(imgs[:, None], K[None, None], np.array([k0]), 1)[:, 0]
    assert np.abs(got[:, : h - k + 1, : w - k + 1] - ref).max() < 1e-5


@pytest.mark.parametrize("m,n,p", [(4, 8, 4), (8, 4, 2), (3, 8, 8), (16, 4, 4)])
def test_vr_matmul_single_ciphertext_matches_fp64(m, n, p):
    """Alg. 3 with one ciphertext per operand (tau_a, tau_b, RowShifter as Rot(., idx n), SumColVec by
    log-rotations with a column-0 mask, Alg. 3's mask F): decrypts to A @ B with C[i][c] at slot
    i n + c; p products, 2 p log2(n) + (p - 1) rotations, 2 p plaintext products (tab2's counts
    with log2 n for SumColVec)."""
    o = Oracle(9, (60, 40, 40, 40, 40), 1, 60, 1, 40.0, seed=30)
    S = o.slots
    steps = [idx * n for idx in range(1, p)] + [t for t in (1, 2, 4, 8, 16) if t < n] + \
            [-t for t in (1, 2, 4, 8, 16) if t < n]
    o.keygen(steps)
    rng = np.random.default_rng(m * 100 + n + p)
    A, Bm = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (n, p))
    lp = o.L1
    Ac = o.encrypt(o.encode(layouts.vr_matrix_a(A, S)), lp, 0)
    Bc = o.encrypt(o.encode(layouts.vr_matrix_b(Bm, S)), lp, 1)
    mv = layouts.vr_matmul_masks(m, n, p, S)
    masks = np.stack([o.encode(mv[0], float(o.q[lp - 2]))] + [o.encode(v, float(o.q[lp - 3])) for v in mv[1:]])
    o.reset_counters()
    D = o.vr_matmul(Ac, Bc, n, p, masks)
    c = o.counters()
    lg = int(math.log2(n))
    assert c["tensors"] == p and c["relins"] == p and c["ct_plain"] == 2 * p
    assert c["rotations"] == (p - 1) + 2 * p * lg
    C = layouts.vr_matmul_from(o.decrypt(D, o.scale ** 2 / o.q[lp - 1]), m, n, p)
    assert np.abs(C - A @ Bm).max() < 1e-5


@pytest.mark.parametrize("n,hw,r", [(16, 12, 5), (16, 16, 1), (32, 20, 19), (8, 8, 7)])
def test_vrot_rotates_every_virtual_ciphertext(n, hw, r):
    """vRot (Alg. 5, with F2 applied to every row): every row's image of hw slots rotates left by r,
    the rest of the row becomes 0; two rotations from one ModUp, two masks, one rescale."""
    o = Oracle(8, (60, 40, 40), 1, 60, 1, 40.0, seed=32)
    S = o.slots
    o.keygen([r, S - hw + r])
    v = np.random.default_rng(n + hw + r).uniform(-1, 1, S)
    X = o.encrypt(o.encode(v), ct_id=0)[None]
    masks = np.stack([o.encode(f, float(o.q[o.L1 - 1])) for f in layouts.vrot_masks(n, hw, r, S)])
    o.reset_counters()
    Y = o.vrot(X, r, hw, masks)
    c = o.counters()
    assert c["rotations"] == 2 and c["modups"] == 1 and c["ct_plain"] == 2 and c["rescales"] == 1
    assert np.abs(o.decrypt(Y[0]) - layouts.vrot_slots(v, n, hw, r)).max() < 1e-6
    # the literal F2[m][j] (last row only) would leave the wrapped part of the other rows empty
    if S // n > 1:
        wrong = layouts.vrot_slots(v, n, hw, r).copy()
        wrong[: n * (S // n - 1)] *= layouts.vrot_masks(n, hw, r, S)[0][: n * (S // n - 1)]
        assert np.abs(o.decrypt(Y[0]) - wrong).max() > 1e-3


def encrypt_images(o, imgs, H, limbs=None, base_id=0):
    """imgs [B][C][h][w] -> X [C][w][2][limbs][N]."""
    Bn, C, h, w = imgs.shape
    out = []
    for c in range(C):
        z = layouts.image_columns(imgs[:, c], o.slots, H)
        out.append(np.stack([o.encrypt(o.encode(z[j]), limbs, base_id + c * w + j) for j in range(w)]))
    return np.stack(out)


@pytest.mark.parametrize("stride,c_in", [(1, 1), (2, 2)])
def test_conv2d_matches_fp64_and_schedules_agree(stride, c_in):
    o = Oracle(8, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=21)
    k, c_out, H = 3, 2, 16
    o.keygen([1, 2])
    rng = np.random.default_rng(stride)
    imgs = rng.uniform(0, 1, (3, c_in, 9, 8))
    K = rng.normal(0, 0.3, (c_out, c_in, k, k))
    bias = rng.normal(0, 0.3, c_out)
    X = encrypt_images(o, imgs, H)
    o.reset_counters()
    Y = o.conv2d(X, 1, K, bias, stride, o.scale)
    c = o.counters()
    w_out = (8 - k) // stride + 1
    ref = fp64_ref.conv2d(imgs, K, bias, stride)
    z = np.stack([o.decrypt(y) for y in Y]).reshape(c_out, w_out, o.slots)
    got = np.moveaxis(layouts.image_from_columns(z, 3, H, stride, ref.shape[2]), 0, 1)
    assert np.abs(got - ref).max() < 1e-6
    # P10: (k-1) rotations of every used input column, one ModUp each
    used = min(8, stride * (w_out - 1) + k)
    assert c["rotations"] == c_in * used * (k - 1) and c["modups"] == c_in * used
    assert c["rescales"] == c_out * w_out and c["ct_scalar"] == c_out * w_out * c_in * k * k
    # P12: the SumForConv order (multiply, then rotate partial sums) decrypts the same
    Y2 = o.conv2d(X, 1, K, bias, stride, o.scale, schedule=1)
    z2 = np.stack([o.decrypt(y) for y in Y2]).reshape(c_out, w_out, o.slots)
    got2 = np.moveaxis(layouts.image_from_columns(z2, 3, H, stride, ref.shape[2]), 0, 1)
    assert np.abs(got2 - got).max() < 1e-6
    assert not np.array_equal(Y, Y2)  # different key switches, same decryption


@pytest.mark.parametrize("stride,c_in", [(1, 1), (2, 2)])
def test_conv2d_encrypted_kernels_matches_fp64(stride, c_in):
    """Convolution with encrypted kernels (the model provider's role, Sec. V): kernel ciphertexts
    encrypt the constant K at scale q_l; decrypts to the FP64 convolution and to the plaintext-weight
    schedule; c_out w' c_in k^2 tensor products, one relinearisation per output."""
    o = Oracle(8, (60, 40, 40, 40), 1, 60, 1, 40.0, seed=24)
    k, c_out, H = 3, 2, 16
    o.keygen([1, 2])
    rng = np.random.default_rng(10 + stride)
    imgs = rng.uniform(0, 1, (3, c_in, 9, 8))
    K = rng.normal(0, 0.3, (c_out, c_in, k, k))
    bias = rng.normal(0, 0.3, c_out)
    X = encrypt_images(o, imgs, H)
    lp = o.L1
    m = o.conv_weight_plaintexts(K, lp)
    assert m.shape == (K.size, o.N) and not m[:, 1:].any()
    Wct = np.stack([o.encrypt(m[i], lp, 5000 + i) for i in range(len(m))])
    # each kernel ciphertext holds K at every slot
    assert np.abs(o.decrypt(Wct[1], float(o.q[lp - 1])) - K.reshape(-1)[1]).max() < 1e-6
    o.reset_counters()
    Y = o.conv2d_enc(X, 1, Wct, bias, c_out, k, stride, o.scale)
    c = o.counters()
    w_out = (8 - k) // stride + 1
    assert c["tensors"] == c_out * w_out * c_in * k * k and c["relins"] == c_out * w_out
    assert c["rescales"] == c_out * w_out and c["ct_scalar"] == 0
    ref = fp64_ref.conv2d(imgs, K, bias, stride)
    z = np.stack([o.decrypt(y) for y in Y]).reshape(c_out, w_out, o.slots)
    got = np.moveaxis(layouts.image_from_columns(z, 3, H, stride, ref.shape[2]), 0, 1)
    assert np.abs(got - ref).max() < 1e-6
    Yp = o.conv2d(X, 1, K, bias, stride, o.scale)
    zp = np.stack([o.decrypt(y) for y in Yp]).reshape(c_out, w_out, o.slots)
    assert np.abs(zp - z).max() < 1e-6


def test_cnn_small_matches_fp64():
    """conv(5x5,s2) -> x^2 -> conv(3x3,s2) -> x^2 -> FC on a reduced ring and image."""
    o = Oracle(9, (60,) + (45,) * 6, 2, 60, 2, 45.0, seed=31)
    side, H, Bn = 17, 32, 2
    h1 = (side - 5) // 2 + 1   # 7
    h2 = (h1 - 3) // 2 + 1     # 3
    rng = np.random.default_rng(31)
    imgs = rng.uniform(0, 1, (Bn, side, side))
    c1w, c1b = rng.normal(0, 0.2, (2, 1, 5, 5)), rng.normal(0, 0.2, 2)
    c2w, c2b = rng.normal(0, 0.2, (3, 2, 3, 3)), rng.normal(0, 0.2, 3)
    fw, fb = rng.normal(0, 0.2, (4, 3 * h2 * h2)), rng.normal(0, 0.2, 4)
    o.keygen([1, 2, 3, 4, 6, 8, 16])
    X = encrypt_images(o, imgs[:, None], H)
    sc = o.scale
    Y = o.conv2d(X, 1, c1w, c1b, 2, sc).reshape(2, h1, 2, -1, o.N)
    Y = o.square(Y.reshape(-1, 2, Y.shape[-2], o.N)).reshape(2, h1, 3, -1, o.N)  # three components
    sc = sc * sc / o.q[X.shape[3] - 2]
    Y = o.conv2d(Y, 2, c2w, c2b, 2, sc).reshape(3, h2, 2, -1, o.N)
    lp = Y.shape[3]
    Y = o.square(Y.reshape(-1, 2, lp, o.N)).reshape(3, h2, 3, lp - 1, o.N)
    sc = sc * sc / o.q[lp - 1]
    pts = o.fc_plaintexts(lp - 1, 3, h2, h2, 4, H, Bn, fw, list(range(4)))
    Z = o.fc(Y, 4, H, pts, fb, sc, list(range(4)))
    z = np.stack([o.decrypt(zz, sc) for zz in Z])
    logits = layouts.logits_from_fc(z, Bn, H)
    x = imgs[:, None]
    x = fp64_ref.conv2d(x, c1w, c1b, 2) ** 2
    x = fp64_ref.conv2d(x, c2w, c2b, 2) ** 2
    ref = fp64_ref.dense(x, fw, fb)
    assert np.abs(logits - ref).max() < 1e-4


@pytest.mark.parametrize("K,alpha,decrypts", [(2, 5, False), (5, 5, True), (2, 2, True)])
def test_three_digits_need_a_special_modulus_above_the_digit(K, alpha, decrypts):
    """The CNN configuration names 2 special primes and dnum = 3. With its 13 Q primes, three digits
    hold 5 primes each (up to 60 + 4 x 45 = 240 bits) while P = 2 x 60 = 120 bits, and the key-switch
    noise, about (digit / P) sigma sqrt(N) per coefficient, swamps the 2^45 scale: a rotation decrypts
    with an error far above 1e-4. Five special primes (P = 300 bits, dnum = 3) or digits of two primes
    with the two stated special primes (7 digits, the reading the CNN runs) decrypt within 1e-6."""
    o = Oracle(11, (60,) + (45,) * 12, K, 60, alpha, 45.0, seed=9)
    o.keygen([1])
    z = np.random.default_rng(9).uniform(-1, 1, o.slots)
    ct = o.encrypt(o.encode(z), o.L1, 0)
    err = float(np.abs(o.decrypt(o.rotate(ct, [1])[0]) - np.roll(z, -1)).max())
    if decrypts:
        assert err < 1e-6
    else:
        assert err > 1e-4
