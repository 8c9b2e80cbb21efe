"""CPU oracle for the encrypted matmul / convolution path (TEST INFRASTRUCTURE).

A plain, slow RNS-CKKS implementation (C++ in this folder, loaded through
ctypes) and the paper's multi-ciphertext layouts, written from the paper and
the scheme's textbook definitions. Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may import it; the CUDA library never does, and
this package imports nothing from the library.

Ciphertexts cross this interface as numpy uint64 arrays [n_polys][limbs][N]
in the coefficient domain (residues in [0, q_i)).
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        V = ctypes.c_void_p
        sig = {
            "oc_create": (V, [ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_double, ctypes.c_uint64]),
            "oc_free": (None, [V]),
            "oc_last_error": (ctypes.c_char_p, []),
            "ol_last_error": (ctypes.c_char_p, []),
            "oc_n_primes": (ctypes.c_int, [V]),
            "oc_primes": (None, [V, _u64p]),
            "oc_psi": (ctypes.c_uint64, [V, ctypes.c_int]),
            "oc_ntt": (ctypes.c_int, [V, ctypes.c_int, _u64p, ctypes.c_int]),
            "oc_polymul": (ctypes.c_int, [V, ctypes.c_int, _u64p, _u64p, _u64p]),
            "oc_automorph": (ctypes.c_int, [V, ctypes.c_int, _u64p, ctypes.c_uint64, _u64p]),
            "oc_galois_elt": (ctypes.c_uint64, [V, ctypes.c_long]),
            "oc_modup": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, _u64p]),
            "oc_moddown": (ctypes.c_int, [V, _u64p, ctypes.c_int, _u64p]),
            "oc_encode": (ctypes.c_int, [V, _dp, ctypes.c_size_t, ctypes.c_double, _i64p]),
            "oc_decode": (ctypes.c_int, [V, _dp, ctypes.c_double, _dp]),
            "oc_keygen": (ctypes.c_int, [V, _lp, ctypes.c_int]),
            "oc_secret": (ctypes.c_int, [V, _i64p]),
            "oc_export_key": (ctypes.c_int, [V, ctypes.c_uint64, _u64p]),
            "oc_encrypt": (ctypes.c_int, [V, _i64p, ctypes.c_int, ctypes.c_uint64, _u64p]),
            "oc_decrypt_coeffs": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, _dp]),
            "oc_decrypt_slots": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]),
            "oc_add": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_int, ctypes.c_int, _u64p]),
            "oc_tensor": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_int, _u64p]),
            "oc_relin": (ctypes.c_int, [V, _u64p, ctypes.c_int, _u64p]),
            "oc_keyswitch": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_uint64, _u64p]),
            "oc_rotate_hoisted": (ctypes.c_int, [V, _u64p, ctypes.c_int, _lp, ctypes.c_int, _u64p]),
            "oc_rescale": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, _u64p]),
            "oc_mul_scalar": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int64, _u64p]),
            "oc_mul_plain": (ctypes.c_int, [V, _u64p, ctypes.c_int, _i64p, _u64p]),
            "oc_counters": (None, [V, _lp]),
            "oc_reset_counters": (None, [V]),
            "oc_matmul": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p]),
            "oc_matmul_volley": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p]),
            "oc_vrot": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long, ctypes.c_int,
                                       _i64p, _u64p]),
            "oc_vr_matmul": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p,
                                            _u64p]),
            "oc_vr_conv2d": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, _u64p,
                                            ctypes.c_int, ctypes.c_int, _i64p, _u64p]),
            "oc_reform": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         _i64p, _u64p]),
            "oc_matmul_bsgs": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              _u64p]),
            "oc_conv2d_enc": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _u64p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int, _ip, _u64p]),
            "oc_poly_act3": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                            _u64p, _dp]),
            "oc_conv2d": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip,
                                         ctypes.c_int, _u64p]),
            "oc_square": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, _u64p]),
            "oc_fc_plaintexts": (ctypes.c_int, [V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _ip, _i64p]),
            "oc_fc": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _i64p, _dp, ctypes.c_double, ctypes.c_int, _ip, _u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def round_half_away(x: float) -> int:
    """Nearest integer to the double x, ties away from zero (C's llround): the
    fraction |x| - floor(|x|) is exact in double precision."""
    a = abs(x)
    f = math.floor(a)
    r = int(f) + (1 if a - f >= 0.5 else 0)
    return -r if x < 0 else r


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _check(rc: int):
    if rc != 0:
        lib = _lib()
        msg = (lib.oc_last_error() or b"") + b" " + (lib.ol_last_error() or b"")
        raise RuntimeError("oracle: " + msg.decode().strip())


class Oracle:
    """RNS-CKKS context on the CPU: prime chain, keys, and the operations."""

    def __init__(self, log_n: int, q_bits: Sequence[int], n_special: int, special_bits: int,
                 alpha: int, log_scale: float, sigma: float = 3.2, seed: int = 1):
        self.lib = _lib()
        qb = (ctypes.c_int * len(q_bits))(*q_bits)
        self.h = self.lib.oc_create(log_n, len(q_bits), qb, n_special, special_bits, alpha, sigma, seed)
        if not self.h:
            raise RuntimeError("oracle: " + self.lib.oc_last_error().decode())
        self.log_n = log_n
        self.N = 1 << log_n
        self.slots = self.N // 2
        self.L1 = len(q_bits)
        self.K = n_special
        self.alpha = alpha
        self.scale = float(2.0 ** log_scale)
        self.seed = seed
        pr = np.zeros(self.L1 + self.K, dtype=np.uint64)
        self.lib.oc_primes(self.h, _p(pr, _u64p))
        self.primes = [int(x) for x in pr]
        self.q = self.primes[: self.L1]
        self.p = self.primes[self.L1:]

    @classmethod
    def from_preset(cls, preset, seed: int = 1):
        return cls(preset.log_n, preset.q_bits, preset.n_special, preset.special_bits, preset.alpha,
                   preset.log_scale, preset.sigma, seed)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oc_free(h)
            self.h = None

    # ---- transforms ----
    def psi(self, pi: int) -> int:
        return int(self.lib.oc_psi(self.h, pi))

    def ntt(self, a, pi: int, inverse: bool = False) -> np.ndarray:
        x = _u64(a).copy()
        _check(self.lib.oc_ntt(self.h, pi, _p(x, _u64p), int(inverse)))
        return x

    def polymul(self, a, b, pi: int) -> np.ndarray:
        a, b = _u64(a), _u64(b)
        out = np.zeros(self.N, np.uint64)
        _check(self.lib.oc_polymul(self.h, pi, _p(a, _u64p), _p(b, _u64p), _p(out, _u64p)))
        return out

    def automorph(self, a, k: int, pi: int) -> np.ndarray:
        a = _u64(a)
        out = np.zeros(self.N, np.uint64)
        _check(self.lib.oc_automorph(self.h, pi, _p(a, _u64p), k, _p(out, _u64p)))
        return out

    def galois_elt(self, step: int) -> int:
        return int(self.lib.oc_galois_elt(self.h, step))

    def modup(self, x, j: int) -> np.ndarray:
        x = _u64(x)
        lp = x.shape[0]
        out = np.zeros((lp + self.K, self.N), np.uint64)
        _check(self.lib.oc_modup(self.h, _p(x, _u64p), lp, j, _p(out, _u64p)))
        return out

    def moddown(self, u) -> np.ndarray:
        u = _u64(u)
        lp = u.shape[0] - self.K
        out = np.zeros((lp, self.N), np.uint64)
        _check(self.lib.oc_moddown(self.h, _p(u, _u64p), lp, _p(out, _u64p)))
        return out

    # ---- encoding ----
    def encode(self, z, scale: Optional[float] = None) -> np.ndarray:
        z = np.ascontiguousarray(z, dtype=np.float64)
        out = np.zeros(self.N, np.int64)
        _check(self.lib.oc_encode(self.h, _p(z, _dp), z.size, self.scale if scale is None else scale,
                                  _p(out, _i64p)))
        return out

    def decode(self, m, scale: Optional[float] = None) -> np.ndarray:
        m = np.ascontiguousarray(m, dtype=np.float64)
        z = np.zeros(self.slots, np.float64)
        _check(self.lib.oc_decode(self.h, _p(m, _dp), self.scale if scale is None else scale, _p(z, _dp)))
        return z

    # ---- keys / encryption ----
    def keygen(self, rot_steps: Sequence[int] = ()):
        st = (ctypes.c_long * max(1, len(rot_steps)))(*rot_steps)
        _check(self.lib.oc_keygen(self.h, st, len(rot_steps)))

    def secret(self) -> np.ndarray:
        s = np.zeros(self.N, np.int64)
        _check(self.lib.oc_secret(self.h, _p(s, _i64p)))
        return s

    def export_key(self, key_id: int) -> np.ndarray:
        beta = -(-self.L1 // self.alpha)
        out = np.zeros((beta, 2, self.L1 + self.K, self.N), np.uint64)
        _check(self.lib.oc_export_key(self.h, key_id, _p(out, _u64p)))
        return out

    def encrypt(self, m, limbs: Optional[int] = None, ct_id: int = 0) -> np.ndarray:
        m = np.ascontiguousarray(m, dtype=np.int64)
        limbs = self.L1 if limbs is None else limbs
        out = np.zeros((2, limbs, self.N), np.uint64)
        _check(self.lib.oc_encrypt(self.h, _p(m, _i64p), limbs, ct_id, _p(out, _u64p)))
        return out

    def decrypt_coeffs(self, ct) -> np.ndarray:
        ct = _u64(ct)
        out = np.zeros(self.N, np.float64)
        _check(self.lib.oc_decrypt_coeffs(self.h, _p(ct, _u64p), ct.shape[0], ct.shape[1], _p(out, _dp)))
        return out

    def decrypt(self, ct, scale: Optional[float] = None) -> np.ndarray:
        ct = _u64(ct)
        z = np.zeros(self.slots, np.float64)
        _check(self.lib.oc_decrypt_slots(self.h, _p(ct, _u64p), ct.shape[0], ct.shape[1],
                                         self.scale if scale is None else scale, _p(z, _dp)))
        return z

    # ---- operations ----
    def add(self, a, b) -> np.ndarray:
        a, b = _u64(a), _u64(b)
        out = np.zeros_like(a)
        _check(self.lib.oc_add(self.h, _p(a, _u64p), _p(b, _u64p), a.shape[0], a.shape[1], _p(out, _u64p)))
        return out

    def add_plain(self, ct, m) -> np.ndarray:
        """Add with a plaintext operand (Sec. II-A's Add): ct [polys][lp][N] (coefficient domain)
        plus the encoded integer plaintext m [N] on component 0, limb i taken modulo q_i."""
        ct = _u64(ct).copy()
        m = np.asarray(m, dtype=np.int64)
        for i in range(ct.shape[1]):
            q = int(self.q[i])
            r = np.mod(m, np.int64(q)).astype(np.uint64)
            ct[0, i] = (ct[0, i] + r) % np.uint64(q)
        return ct

    def tensor(self, a, b) -> np.ndarray:
        a, b = _u64(a), _u64(b)
        out = np.zeros((3,) + a.shape[1:], np.uint64)
        _check(self.lib.oc_tensor(self.h, _p(a, _u64p), _p(b, _u64p), a.shape[1], _p(out, _u64p)))
        return out

    def relin(self, d) -> np.ndarray:
        d = _u64(d)
        out = np.zeros((2,) + d.shape[1:], np.uint64)
        _check(self.lib.oc_relin(self.h, _p(d, _u64p), d.shape[1], _p(out, _u64p)))
        return out

    def keyswitch(self, x, key_id: int) -> np.ndarray:
        x = _u64(x)
        out = np.zeros((2,) + x.shape, np.uint64)
        _check(self.lib.oc_keyswitch(self.h, _p(x, _u64p), x.shape[0], key_id, _p(out, _u64p)))
        return out

    def rotate(self, ct, steps: Sequence[int]) -> np.ndarray:
        ct = _u64(ct)
        st = (ctypes.c_long * len(steps))(*steps)
        out = np.zeros((len(steps),) + ct.shape, np.uint64)
        _check(self.lib.oc_rotate_hoisted(self.h, _p(ct, _u64p), ct.shape[1], st, len(steps), _p(out, _u64p)))
        return out

    def rescale(self, ct) -> np.ndarray:
        ct = _u64(ct)
        out = np.zeros((ct.shape[0], ct.shape[1] - 1, self.N), np.uint64)
        _check(self.lib.oc_rescale(self.h, _p(ct, _u64p), ct.shape[0], ct.shape[1], _p(out, _u64p)))
        return out

    def mul_scalar(self, ct, w: int) -> np.ndarray:
        ct = _u64(ct)
        out = np.zeros_like(ct)
        _check(self.lib.oc_mul_scalar(self.h, _p(ct, _u64p), ct.shape[1], int(w), _p(out, _u64p)))
        return out

    def mul_plain(self, ct, pt) -> np.ndarray:
        ct = _u64(ct)
        pt = np.ascontiguousarray(pt, dtype=np.int64)
        out = np.zeros_like(ct)
        _check(self.lib.oc_mul_plain(self.h, _p(ct, _u64p), ct.shape[1], _p(pt, _i64p), _p(out, _u64p)))
        return out

    def counters(self) -> dict:
        c = (ctypes.c_long * 7)()
        self.lib.oc_counters(self.h, c)
        keys = ["rotations", "modups", "tensors", "relins", "rescales", "ct_scalar", "ct_plain"]
        return dict(zip(keys, list(c)))

    def reset_counters(self):
        self.lib.oc_reset_counters(self.h)

    # ---- layers ----
    def matmul(self, A, B, p: int) -> np.ndarray:
        """A, B: [n][2][lp][N] -> D [p][2][lp-1][N] (diagonal layout)."""
        A, B = _u64(A), _u64(B)
        n, _, lp, _ = A.shape
        out = np.zeros((p, 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_matmul(self.h, _p(A, _u64p), _p(B, _u64p), n, p, lp, _p(out, _u64p)))
        return out

    def matmul_bsgs(self, A, B, p: int, g: int) -> np.ndarray:
        """A, B: [n][2][lp][N] -> D [p][2][lp-1][N] (diagonal layout), baby-step size g."""
        A, B = _u64(A), _u64(B)
        n, _, lp, _ = A.shape
        out = np.zeros((p, 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_matmul_bsgs(self.h, _p(A, _u64p), _p(B, _u64p), n, p, g, lp, _p(out, _u64p)))
        return out

    def vrot(self, X, r: int, hw: int, masks) -> np.ndarray:
        """vRot (Alg. 5) of X [n_ct][2 or 3][lp][N] by r inside rows of images of hw slots; masks
        [2][N] (F1, F2 encoded at scale q_{lp-1}) -> [n_ct][2][lp-1][N]."""
        X = _u64(X)
        n_ct, polys, lp, _ = X.shape
        masks = np.ascontiguousarray(masks, dtype=np.int64)
        out = np.zeros((n_ct, 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_vrot(self.h, _p(X, _u64p), n_ct, polys, lp, r, hw, _p(masks, _i64p), _p(out, _u64p)))
        return out

    def vr_matmul(self, A, Bbar, n: int, p: int, masks) -> np.ndarray:
        """Alg. 3 on one ciphertext per operand: A, Bbar [2][lp][N] -> [2][lp-3][N]. masks [1 + p][N]:
        the column-0 mask of SumColVec encoded at scale q_{lp-2}, then the masks F_idx at scale
        q_{lp-3} (layouts.vr_matmul_masks)."""
        A, Bbar = _u64(A), _u64(Bbar)
        lp = A.shape[1]
        masks = np.ascontiguousarray(masks, dtype=np.int64)
        out = np.zeros((2, lp - 3, self.N), np.uint64)
        _check(self.lib.oc_vr_matmul(self.h, _p(A, _u64p), _p(Bbar, _u64p), lp, n, p, _p(masks, _i64p),
                                     _p(out, _u64p)))
        return out

    def vr_conv2d(self, X, S, bias, k: int, Wb: int, masks) -> np.ndarray:
        """Alg. 4 over one-ciphertext image blocks: X [n][2 or 3][lp][N], kernel ciphertexts
        S [k*k][2][lp][N] (scale q_{lp-1}), bias ciphertext [2][lp-2][N], mask plaintexts
        [k*k][N] (scale q_{lp-2}) -> [n][2][lp-2][N]."""
        X, S, bias = _u64(X), _u64(S), _u64(bias)
        n, polys, lp, _ = X.shape
        masks = np.ascontiguousarray(masks, dtype=np.int64)
        out = np.zeros((n, 2, lp - 2, self.N), np.uint64)
        _check(self.lib.oc_vr_conv2d(self.h, _p(X, _u64p), n, polys, lp, _p(S, _u64p), _p(bias, _u64p), k, Wb,
                                     _p(masks, _i64p), _p(out, _u64p)))
        return out

    def reform_masks(self, h: int, H: int, lp: int) -> np.ndarray:
        """ReForm's plaintexts: mask_i (1 at slots b H + i of every block, else 0) encoded at
        scale q_{lp-1} -> [h][N] int64."""
        out = np.zeros((h, self.N), np.int64)
        for i in range(h):
            z = np.zeros(self.slots)
            z[i::H] = 1.0
            out[i] = self.encode(z, float(self.q[lp - 1]))
        return out

    def reform(self, X, gap: int, h: int, masks) -> np.ndarray:
        """ReForm: X [n][2 or 3][lp][N] with rows at gap `gap` -> [n][2][lp-1][N] with rows at gap 1."""
        X = _u64(X)
        n, polys, lp, _ = X.shape
        masks = np.ascontiguousarray(masks, dtype=np.int64)
        out = np.zeros((n, 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_reform(self.h, _p(X, _u64p), n, polys, lp, gap, h, _p(masks, _i64p), _p(out, _u64p)))
        return out

    def matmul_volley(self, Ahat, B) -> np.ndarray:
        """Ahat [G][n][2][lp][N] (volley encoding of A), B [n][2][lp][N] -> D [G][2][lp-1][N]."""
        Ahat, B = _u64(Ahat), _u64(B)
        G, n, _, lp, _ = Ahat.shape
        out = np.zeros((G, 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_matmul_volley(self.h, _p(Ahat, _u64p), _p(B, _u64p), n, G, lp, _p(out, _u64p)))
        return out

    def conv2d(self, X, gap: int, K, bias, stride: int, scale: float, sel=None, schedule: int = 0) -> np.ndarray:
        """X [c_in][w_in][2 or 3][lp][N]; K [c_out][c_in][k][k] -> [n_sel][2][lp-1][N].

        Three-component inputs (unrelinearised products) are relinearised first."""
        X = _u64(X)
        c_in, w_in, polys, lp, _ = X.shape
        K = np.ascontiguousarray(K, dtype=np.float64)
        c_out, _, k, _ = K.shape
        w_out = (w_in - k) // stride + 1
        if sel is None:
            sel = [(o, j) for o in range(c_out) for j in range(w_out)]
        sel_a = np.ascontiguousarray(np.array(sel, dtype=np.int32).reshape(-1, 2))
        b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
        out = np.zeros((len(sel), 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_conv2d(self.h, _p(X, _u64p), polys, lp, c_in, w_in, gap, _p(K, _dp),
                                  None if b is None else _p(b, _dp), c_out, k, stride, scale, len(sel),
                                  _p(sel_a, _ip), schedule, _p(out, _u64p)))
        return out

    def conv_weight_plaintexts(self, K, lp: int) -> np.ndarray:
        """Constant plaintexts of encrypted kernels: K [c_out][c_in][k][k] -> [c_out*c_in*k*k][N]
        int64, coefficient 0 = round(K q_{lp-1}) (every slot K at scale q_{lp-1}), others 0."""
        K = np.asarray(K, dtype=np.float64)
        m = np.zeros((K.size, self.N), np.int64)
        ql = float(self.q[lp - 1])
        m[:, 0] = [int(round_half_away(w * ql)) for w in K.reshape(-1)]
        return m

    def conv2d_enc(self, X, gap: int, Wct, bias, c_out: int, k: int, stride: int, scale: float,
                   sel=None) -> np.ndarray:
        """X [c_in][w_in][2 or 3][lp][N]; Wct [c_out*c_in*k*k][2][lp][N] kernel ciphertexts
        -> [n_sel][2][lp-1][N]."""
        X, Wct = _u64(X), _u64(Wct)
        c_in, w_in, polys, lp, _ = X.shape
        w_out = (w_in - k) // stride + 1
        if sel is None:
            sel = [(o, j) for o in range(c_out) for j in range(w_out)]
        sel_a = np.ascontiguousarray(np.array(sel, dtype=np.int32).reshape(-1, 2))
        b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
        out = np.zeros((len(sel), 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_conv2d_enc(self.h, _p(X, _u64p), polys, lp, c_in, w_in, gap, _p(Wct, _u64p),
                                      None if b is None else _p(b, _dp), c_out, k, stride, scale, len(sel),
                                      _p(sel_a, _ip), _p(out, _u64p)))
        return out

    def square(self, X) -> np.ndarray:
        """Tensor product and rescale: [n][2][lp][N] -> [n][3][lp-1][N] (relinearised later)."""
        X = _u64(X)
        n, _, lp, _ = X.shape
        out = np.zeros((n, 3, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_square(self.h, _p(X, _u64p), n, lp, _p(out, _u64p)))
        return out

    def poly_act3(self, X, coeffs, scale: float):
        """Degree-3 activation c0 + c1 x + c2 x^2 + c3 x^3 of X [n][2 or 3][lp][N]
        -> ([n][3][lp-2][N], output scale)."""
        X = _u64(X)
        n, polys, lp, _ = X.shape
        c = np.ascontiguousarray(np.zeros(4) if coeffs is None else coeffs, dtype=np.float64)
        assert c.shape == (4,)
        out = np.zeros((n, 3, lp - 2, self.N), np.uint64)
        so = ctypes.c_double()
        _check(self.lib.oc_poly_act3(self.h, _p(X, _u64p), n, polys, lp, _p(c, _dp), scale, _p(out, _u64p),
                                     ctypes.byref(so)))
        return out, so.value

    def fc_plaintexts(self, lp: int, c_in: int, hv: int, w_in: int, gap: int, H: int, B: int, W, sel_o) -> np.ndarray:
        W = np.ascontiguousarray(W, dtype=np.float64)
        sel = np.ascontiguousarray(sel_o, dtype=np.int32)
        out = np.zeros((len(sel), c_in, w_in, self.N), np.int64)
        _check(self.lib.oc_fc_plaintexts(self.h, lp, c_in, hv, w_in, gap, H, B, _p(W, _dp), len(sel),
                                         _p(sel, _ip), _p(out, _i64p)))
        return out

    def fc(self, X, gap: int, H: int, pts, bias, scale: float, sel_o) -> np.ndarray:
        """X [c_in][w_in][2 or 3][lp][N] -> [n_sel][2][lp-1][N]."""
        X = _u64(X)
        c_in, w_in, polys, lp, _ = X.shape
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        sel = np.ascontiguousarray(sel_o, dtype=np.int32)
        b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
        out = np.zeros((len(sel), 2, lp - 1, self.N), np.uint64)
        _check(self.lib.oc_fc(self.h, _p(X, _u64p), polys, lp, c_in, w_in, gap, H, _p(pts, _i64p),
                              None if b is None else _p(b, _dp), scale, len(sel), _p(sel, _ip), _p(out, _u64p)))
        return out
