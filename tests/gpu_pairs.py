"""Helpers for the GPU parity tests: an oracle context and a library context
built from the same parameters and seed, and their layout glue."""
from __future__ import annotations

import numpy as np

from oracle import Oracle, layouts


def make_pair(log_n, q_bits, n_special, special_bits, alpha, log_scale, seed=1, steps=()):
    from paper_2512_18646_gb300 import api
    o = Oracle(log_n, q_bits, n_special, special_bits, alpha, log_scale, seed=seed)
    g = api.Context(log_n, q_bits, n_special, special_bits, alpha, log_scale, seed=seed)
    assert o.primes == g.primes
    if steps is not None:
        o.keygen(list(steps))
        g.keygen(list(steps))
    return o, g


def pair_from_preset(preset, seed=1, steps=(), log_n=None):
    return make_pair(preset.log_n if log_n is None else log_n, preset.q_bits, preset.n_special,
                     preset.special_bits, preset.alpha, preset.log_scale, seed, steps)


def encode_columns(o, z):
    """slot vectors [n][S] -> oracle-encoded integer plaintexts [n][N]."""
    return np.stack([o.encode(v) for v in z])


def encrypt_both(o, g, m, limbs=None, ct_id_base=0, scale=None):
    """Encrypt the same integer plaintexts on both sides.

    Returns (oracle ciphertexts [n][2][limbs][N], library CtSet)."""
    limbs = o.L1 if limbs is None else limbs
    sc = o.scale if scale is None else scale
    oc = np.stack([o.encrypt(m[i], limbs, ct_id_base + i) for i in range(len(m))])
    gc = g.encrypt_coeffs(m, limbs, sc, ct_id_base)
    return oc, gc


def image_columns_both(o, g, imgs, H, ct_id_base=0):
    """imgs [B][C][h][w] -> (oracle X [C][w][2][L][N], library set of C*w ciphertexts)."""
    Bn, C, h, w = imgs.shape
    z = np.concatenate([layouts.image_columns(imgs[:, c], o.slots, H) for c in range(C)])
    m = encode_columns(o, z)
    oc, gc = encrypt_both(o, g, m, ct_id_base=ct_id_base)
    return oc.reshape(C, w, *oc.shape[1:]), gc
