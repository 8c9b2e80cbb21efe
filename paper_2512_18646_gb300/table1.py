"""Table I's CNN (Sec. V) in the paper's single-ciphertext layout, composed from library calls.

Images sit in blocks of Hb x Wb slots, one image per block and N / (2 Hb Wb) images per
ciphertext (the virtual ciphertexts of Sec. III-D: 32 images of 28 x 28 in 32 x 32 blocks at
N = 2^16). Read as a matrix of N / (2 n) rows of n = Hb Wb slots, such a ciphertext is exactly
Alg. 3's tau_a layout with one image per row, which is what lets the dense layers run as
Volley Revolver products:

- CONV: per kernel o, Alg. 4 (he_vr_conv2d) with the model provider's Kernelspanner ciphertexts
  and bias; the valid (h - k + 1) x (w - k + 1) outputs stay at block positions r Wb + c;
- ACT-1: the degree-3 polynomial of Table I (he_poly_act), then one relinearisation;
- FC-1: sum over kernels o of Alg. 3 (he_vr_matmul) with A = channel o's ciphertext and
  B = the rows of FC-1's weights that belong to channel o, placed at the block positions
  r Wb + c (zero rows elsewhere) and tau_b-encoded by the model provider (Sec. V). A product
  yields p1 outputs, p1 dividing the N / (2 n) rows (reading of Sec. III-B's RowShifter as a
  rotation by idx n); FC-1's outputs come as fc1_out / p1 such products, output group t moved
  to columns t p1 .. t p1 + p1 - 1 by a rotation of -t p1 and added; the bias is a plaintext
  added to the result (Alg. 3 starts its accumulator from it);
- ACT-2, then FC-2 the same way with p2 >= fc2_out outputs (zero-padded).

Output c of image i sits at slot i n + c. Depth: 2 (CONV) + 2 (ACT-1) + 3 (FC-1) + 2 (ACT-2)
+ 3 (FC-2) = 12 levels, the CNN parameter set's 13 primes. Every operand of a product is brought
to its partner's level by dropping primes (he_ctset_drop_levels).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

# Table I's activation polynomials, coefficients of x^0 .. x^3
ACT1 = (-0.00015120704, 0.4610149, 2.0225089, -1.4511951)
ACT2 = (-1.5650465, -0.9943767, 1.6794522, 0.5350255)


@dataclasses.dataclass
class Geometry:
    h: int
    w: int
    k: int
    Hb: int
    Wb: int
    channels: int
    fc1_out: int
    fc2_out: int
    slots: int

    @property
    def n(self) -> int:
        return self.Hb * self.Wb

    @property
    def images(self) -> int:
        return self.slots // self.n

    @property
    def p1(self) -> int:
        """outputs of one FC-1 product: the largest power of two dividing both fc1_out and the rows"""
        p = 1
        while p * 2 <= min(self.fc1_out, self.images) and self.fc1_out % (p * 2) == 0 and self.images % (p * 2) == 0:
            p *= 2
        return p

    @property
    def p2(self) -> int:
        """outputs of the FC-2 product: the smallest power of two >= fc2_out (zero-padded)"""
        p = 1
        while p < self.fc2_out:
            p *= 2
        if self.images % p or p > self.n:
            raise ValueError("FC-2's padded output count must divide the rows")
        return p

    def check(self):
        ho, wo = self.h - self.k + 1, self.w - self.k + 1
        if self.h > self.Hb or self.w > self.Wb or ho < 1 or wo < 1:
            raise ValueError("images do not fit the blocks")
        if self.slots % self.n or self.n & (self.n - 1):
            raise ValueError("the block size must be a power of two dividing the slots")
        if self.fc1_out > self.n or self.fc1_out % self.p1:
            raise ValueError("FC-1's outputs must fit a row")


def rotation_steps(geo: Geometry) -> List[int]:
    """Every rotation the network takes: Alg. 4's column and row shifts, Alg. 3's RowShifter
    (idx n) and SumColVec (+-1, +-2, .., +-n/2), and the moves of FC-1's output groups."""
    k, Wb, n = geo.k, geo.Wb, geo.n
    steps = set(range(1, k)) | {Wb * a for a in range(1, k)}
    steps |= {idx * n for idx in range(1, max(geo.p1, geo.p2))}
    t = 1
    while t < n:
        steps |= {t, -t}
        t *= 2
    steps |= {-g * geo.p1 for g in range(1, geo.fc1_out // geo.p1)}
    return sorted(steps)


def fc1_blocks(geo: Geometry, W1: np.ndarray) -> np.ndarray:
    """FC-1's weights [c][ho][wo][fc1_out] as Alg. 3 right operands: [c][group][n][p1], row
    r Wb + c' of channel c holding W1[c][r][c'] (zero rows elsewhere)."""
    ho, wo = geo.h - geo.k + 1, geo.w - geo.k + 1
    G = geo.fc1_out // geo.p1
    out = np.zeros((geo.channels, G, geo.n, geo.p1))
    for ch in range(geo.channels):
        for r in range(ho):
            for c in range(wo):
                out[ch, :, r * geo.Wb + c, :] = W1[ch, r, c].reshape(G, geo.p1)
    return out


def fc2_block(geo: Geometry, W2: np.ndarray) -> np.ndarray:
    """FC-2's weights [fc1_out][fc2_out] as an Alg. 3 right operand [n][p2] (zero-padded)."""
    out = np.zeros((geo.n, geo.p2))
    out[: geo.fc1_out, : geo.fc2_out] = W2
    return out


def row_vector(geo: Geometry, b: Sequence[float]) -> np.ndarray:
    """A bias as a slot vector: b[c] at slot i n + c of every row i."""
    v = np.zeros(geo.slots)
    for i in range(geo.images):
        v[i * geo.n: i * geo.n + len(b)] = b
    return v


@dataclasses.dataclass
class EncryptedModel:
    kernels: list   # per channel: (Kernelspanner set, bias set)
    fc1: list       # [c][group]: tau_b set (top level)
    fc2: object     # tau_b set (top level)
    fc1_b: np.ndarray
    fc2_b: np.ndarray


def encrypt_model(g, geo: Geometry, wts) -> EncryptedModel:
    """The model provider's ciphertexts: Kernelspanner sets per kernel and tau_b-encoded dense
    weights (Sec. V); the dense biases stay plaintexts."""
    geo.check()
    L1 = g.L1
    kernels = [g.vr_encrypt_kernels(wts.conv_w[o], float(wts.conv_b[o]), geo.h, geo.w, geo.Hb, geo.Wb, L1,
                                    1000 + 100 * o) for o in range(geo.channels)]
    B1 = fc1_blocks(geo, wts.fc1_w)
    fc1 = [[g.vr_encrypt_matrix_b(B1[o, t], 2000 + 10 * o + t) for t in range(B1.shape[1])]
           for o in range(geo.channels)]
    fc2 = g.vr_encrypt_matrix_b(fc2_block(geo, wts.fc2_w), 3000)
    return EncryptedModel(kernels, fc1, fc2, np.asarray(wts.fc1_b), np.asarray(wts.fc2_b))


def forward(g, geo: Geometry, x, model: EncryptedModel):
    """One encrypted inference of x (one ciphertext of geo.images images) -> the FC-2
    ciphertext (logit c of image i at slot i n + c)."""
    n, m = geo.n, geo.images
    ys = []
    for o in range(geo.channels):
        S, b = model.kernels[o]
        y = g.vr_conv2d(x, S, b, geo.h, geo.w, geo.k, geo.Hb, geo.Wb)
        g.poly_act(y, ACT1)
        ys.append(g.relinearize(y))
    z = None
    for t in range(geo.fc1_out // geo.p1):
        zt = None
        for o in range(geo.channels):
            Bo = g.drop_levels(model.fc1[o][t], ys[o].limbs)
            part = g.vr_matmul(ys[o], Bo, m, n, geo.p1)
            zt = part if zt is None else g.add(zt, part)
        if t > 0:
            zt = g.rotate(zt, [-t * geo.p1])
        z = zt if z is None else g.add(z, zt)
    g.add_slots(z, row_vector(geo, model.fc1_b))
    g.poly_act(z, ACT2)
    g.relinearize(z)
    out = g.vr_matmul(z, g.drop_levels(model.fc2, z.limbs), m, n, geo.p2)
    g.add_slots(out, row_vector(geo, model.fc2_b))
    return out


def logits(g, geo: Geometry, out) -> np.ndarray:
    """The decrypted logits [images][fc2_out]."""
    z = g.decrypt_slots(out)[0]
    return np.stack([z[i * geo.n: i * geo.n + geo.fc2_out] for i in range(geo.images)])

