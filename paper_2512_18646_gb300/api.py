"""Python face of the C ABI (include/he_gb300.h): same operations, numpy in
and out, handles freed when their Python objects die. Marshalling only."""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from ._lib import HE_E_TIMEOUT, P_D, P_I, P_I32, P_I64, P_U64, ParamsDesc, ServerDesc, check, load


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _words_buffer(buf):
    """(pointer, on_device, words) of a uint64 numpy array or a 64-bit torch tensor."""
    if isinstance(buf, np.ndarray):
        assert buf.dtype == np.uint64 and buf.flags.c_contiguous
        return _ptr(buf, P_U64), 0, buf.size
    assert buf.element_size() == 8 and buf.is_contiguous(), "64-bit contiguous tensor expected"
    return ctypes.cast(ctypes.c_void_p(buf.data_ptr()), P_U64), int(buf.is_cuda), buf.numel()


def volley_geometry(slots: int, m: int, p: int):
    """(M, per, groups) of the zero-rotation matmul layout (he_volley_geometry)."""
    M, per, G = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(load().he_volley_geometry(slots, m, p, ctypes.byref(M), ctypes.byref(per), ctypes.byref(G)))
    return M.value, per.value, G.value


class CtSet:
    """n ciphertexts at one level and scale, in device memory (NTT domain)."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.h = ctypes.c_void_p(handle)

    def free(self):
        if self.h:
            load().he_ctset_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        """(n, limbs, scale)."""
        return self.info4()[:3]

    def info4(self):
        """(n, limbs, scale, polys)."""
        n, limbs, sc, pol = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        check(load().he_ctset_info(self.h, ctypes.byref(n), ctypes.byref(limbs), ctypes.byref(sc), ctypes.byref(pol)))
        return n.value, limbs.value, sc.value, pol.value

    @property
    def polys(self):
        return self.info4()[3]

    @property
    def n(self):
        return self.info()[0]

    @property
    def limbs(self):
        return self.info()[1]

    @property
    def scale(self):
        return self.info()[2]

    def export(self) -> np.ndarray:
        """Coefficient-domain limbs [n][polys][limbs][N] (uint64)."""
        n, limbs, _, polys = self.info4()
        out = np.zeros((n, polys, limbs, self.ctx.N), np.uint64)
        check(load().he_ctset_export(self.h, _ptr(out, P_U64), out.size))
        return out

    def export_async(self, out: np.ndarray) -> int:
        """Queue export() into `out` ([n][polys][limbs][N] uint64, page-locked for overlap) without
        waiting (he_ctset_export_async); returns the ticket Context.export_wait takes. `out` must
        not be read before that wait."""
        n, limbs, _, polys = self.info4()
        assert out.dtype == np.uint64 and out.flags.c_contiguous and out.size >= n * polys * limbs * self.ctx.N
        t = ctypes.c_uint64()
        check(load().he_ctset_export_async(self.h, _ptr(out, P_U64), out.size, ctypes.byref(t)))
        return t.value

    def export_raw(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """The device words as held, [n][polys][limbs][N] uint64 in the NTT domain."""
        n, limbs, _, polys = self.info4()
        if out is None:
            out = np.zeros((n, polys, limbs, self.ctx.N), np.uint64)
        assert out.dtype == np.uint64 and out.flags.c_contiguous and out.size >= n * polys * limbs * self.ctx.N
        check(load().he_ctset_export_raw(self.h, _ptr(out, P_U64), out.size))
        return out

    def export_words(self, dst) -> None:
        """The words as held, [n][polys][limbs][N] in the NTT domain, into `dst`: a C-contiguous
        numpy uint64 array (host) or a contiguous 64-bit torch CUDA tensor on the context's GPU."""
        n, limbs, _, polys = self.info4()
        need = n * polys * limbs * self.ctx.N
        ptr, on_dev, size = _words_buffer(dst)
        assert size >= need, "destination too small"
        check(load().he_ctset_export_words(self.h, ptr, on_dev, size))

    def device_ptr(self) -> int:
        p = P_U64()
        check(load().he_ctset_device_ptr(self.h, ctypes.byref(p)))
        return ctypes.cast(p, ctypes.c_void_p).value

    def slice(self, first: int, n: int) -> "CtSet":
        out = ctypes.c_void_p()
        check(load().he_ctset_slice(self.ctx.h, self.h, first, n, ctypes.byref(out)))
        return CtSet(self.ctx, out.value)


class PtSet:
    def __init__(self, handle: int):
        self.h = ctypes.c_void_p(handle)

    def __del__(self):
        try:
            if self.h:
                load().he_ptset_free(self.h)
                self.h = None
        except Exception:
            pass


class Graph:
    """A captured sequence of library calls (he_graph_*); replay with launch()."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.h = ctypes.c_void_p(handle)

    def launch(self):
        check(load().he_graph_launch(self.h))

    @property
    def kernel_nodes(self) -> int:
        n = ctypes.c_uint64()
        check(load().he_graph_info(self.h, ctypes.byref(n)))
        return n.value

    def destroy(self):
        if self.h:
            load().he_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Context:
    """he_ctx: parameters, NTT tables and keys on the current CUDA device."""

    def __init__(self, log_n: int, q_bits: Sequence[int], n_special: int, special_bits: int, alpha: int,
                 log_scale: float, sigma: float = 3.2, seed: int = 1, stream: Optional[int] = None):
        lib = load()
        qb = (ctypes.c_int * len(q_bits))(*q_bits)
        self._qb = qb
        d = ParamsDesc(log_n, len(q_bits), qb, n_special, special_bits, alpha, float(log_scale), float(sigma))
        h = ctypes.c_void_p()
        check(lib.he_ctx_create(ctypes.byref(d), seed, ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        self.log_n = log_n
        self.N = 1 << log_n
        self.slots = self.N // 2
        self.L1 = len(q_bits)
        self.K = n_special
        self.alpha = alpha
        self.scale = float(2.0 ** log_scale)
        pr = np.zeros(self.L1 + self.K, np.uint64)
        check(lib.he_ctx_primes(h, _ptr(pr, P_U64), pr.size))
        self.primes = [int(x) for x in pr]
        self.q = self.primes[: self.L1]
        self.p = self.primes[self.L1:]

    @classmethod
    def from_preset(cls, preset, seed: int = 1, stream: Optional[int] = None):
        return cls(preset.log_n, preset.q_bits, preset.n_special, preset.special_bits, preset.alpha,
                   preset.log_scale, preset.sigma, seed, stream)

    def set_work_budget(self, nbytes: int):
        """Bound the device temporaries of one operation (0 = none); results do not change."""
        check(load().he_ctx_set_work_budget(self.h, int(nbytes)))

    def set_tensor_cores(self, on: bool):
        check(load().he_ctx_set_tensor_cores(self.h, int(bool(on))))

    def synchronize(self):
        check(load().he_ctx_synchronize(self.h))

    def export_wait(self, ticket: int):
        """Block until CtSet.export_async's copy with this ticket (and every earlier one) is on the host."""
        check(load().he_ctset_export_wait(self.h, int(ticket)))

    def close(self):
        if getattr(self, "h", None):
            load().he_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _set(self, fn, *args) -> CtSet:
        out = ctypes.c_void_p()
        check(fn(*args, ctypes.byref(out)))
        return CtSet(self, out.value)

    # ---- keys / encryption ----
    def keygen(self, steps: Sequence[int] = ()):
        st = (ctypes.c_int32 * max(1, len(steps)))(*steps)
        check(load().he_keygen(self.h, st, len(steps)))

    def export_keys(self) -> np.ndarray:
        """The key checkpoint (include/he_gb300.h he_keys_export) as uint64 words."""
        n = ctypes.c_size_t()
        check(load().he_keys_export(self.h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, np.uint64)
        check(load().he_keys_export(self.h, _ptr(out, P_U64), out.size, None))
        return out

    def import_keys(self, words):
        words = np.ascontiguousarray(words, dtype=np.uint64)
        check(load().he_keys_import(self.h, _ptr(words, P_U64), words.size))

    def encrypt_image(self, px, block_stride: int, ct_id_base: int = 0) -> CtSet:
        px = _f64(px)
        b, h, w = px.shape
        return self._set(load().he_encrypt_image, self.h, _ptr(px, P_D), b, h, w, block_stride, ct_id_base)

    def encrypt_matrix_a(self, A, ct_id_base: int = 0) -> CtSet:
        A = _f64(A)
        return self._set(load().he_encrypt_matrix_a, self.h, _ptr(A, P_D), A.shape[0], A.shape[1], ct_id_base)

    def ntt_set_geometry(self, n1: int, cols: int):
        check(load().he_ntt_set_geometry(self.h, n1, cols))

    def ntt_autotune(self, rows: int):
        """-> (n1, cols, microseconds of a forward + inverse transform of `rows` limbs)."""
        n1, c, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(load().he_ntt_autotune(self.h, rows, ctypes.byref(n1), ctypes.byref(c), ctypes.byref(us)))
        return n1.value, c.value, us.value

    def graph_begin(self):
        check(load().he_graph_begin(self.h))

    def graph_end(self) -> Graph:
        out = ctypes.c_void_p()
        check(load().he_graph_end(self.h, ctypes.byref(out)))
        return Graph(self, out.value)

    def assign(self, dst: CtSet, src: CtSet):
        check(load().he_ctset_assign(self.h, dst.h, src.h))

    def encrypt_matrix_a_volley(self, A, p: int, ct_id_base: int = 0) -> CtSet:
        A = _f64(A)
        return self._set(load().he_encrypt_matrix_a_volley, self.h, _ptr(A, P_D), A.shape[0], A.shape[1], p,
                         ct_id_base)

    def encrypt_matrix_b(self, B, ct_id_base: int = 0) -> CtSet:
        B = _f64(B)
        return self._set(load().he_encrypt_matrix_b, self.h, _ptr(B, P_D), B.shape[0], B.shape[1], ct_id_base)

    def encrypt_coeffs(self, m, limbs: Optional[int] = None, scale: Optional[float] = None,
                       ct_id_base: int = 0) -> CtSet:
        m = np.ascontiguousarray(m, dtype=np.int64).reshape(-1, self.N)
        return self._set(load().he_encrypt_coeffs, self.h, _ptr(m, P_I64), m.shape[0],
                         self.L1 if limbs is None else limbs, self.scale if scale is None else scale, ct_id_base)

    def import_coeffs(self, host, scale: float) -> CtSet:
        host = np.ascontiguousarray(host, dtype=np.uint64)
        n, _, limbs, _ = host.shape
        return self._set(load().he_ctset_import, self.h, _ptr(host, P_U64), n, limbs, scale)

    def import_coeffs_async(self, host, scale: float) -> CtSet:
        """import_coeffs without waiting for the copy (he_ctset_import_async): `host` (page-locked
        for overlap) must stay unchanged until the context is next synchronised."""
        assert host.dtype == np.uint64 and host.flags.c_contiguous
        n, _, limbs, _ = host.shape
        return self._set(load().he_ctset_import_async, self.h, _ptr(host, P_U64), n, limbs, scale)

    # ---- evaluation ----
    def matmul(self, A: CtSet, B: CtSet, m: int, p: int) -> CtSet:
        return self._set(load().he_matmul, self.h, A.h, B.h, m, p)

    def matmul_range(self, A: CtSet, B: CtSet, m: int, p: int, lo: int, hi: int) -> CtSet:
        """Diagonals lo .. hi - 1 of matmul(A, B, m, p)."""
        return self._set(load().he_matmul_range, self.h, A.h, B.h, m, p, lo, hi)

    def matmul_bsgs(self, A: CtSet, B: CtSet, m: int, p: int, g: int = 0) -> CtSet:
        return self._set(load().he_matmul_bsgs, self.h, A.h, B.h, m, p, g)

    def matmul_volley(self, A: CtSet, B: CtSet) -> CtSet:
        return self._set(load().he_matmul_volley, self.h, A.h, B.h)

    def matmul_batched(self, As, Bs, ms, ps):
        n = len(As)
        arrA = (ctypes.c_void_p * n)(*[a.h.value for a in As])
        arrB = (ctypes.c_void_p * n)(*[b.h.value for b in Bs])
        mm = (ctypes.c_int * n)(*ms)
        pp = (ctypes.c_int * n)(*ps)
        out = (ctypes.c_void_p * n)()
        check(load().he_matmul_batched(self.h, n, arrA, arrB, mm, pp, out))
        return [CtSet(self, out[i]) for i in range(n)]

    def conv2d(self, x: CtSet, c_in: int, gap: int, W, bias, stride: int) -> CtSet:
        W = _f64(W)
        c_out, _, k, _ = W.shape
        b = None if bias is None else _f64(bias)
        return self._set(load().he_conv2d, self.h, x.h, c_in, gap, _ptr(W, P_D), None if b is None else _ptr(b, P_D),
                         c_out, k, stride)

    def vrot(self, x: CtSet, r: int, row_len: int, img_len: int) -> CtSet:
        return self._set(load().he_vrot, self.h, x.h, r, row_len, img_len)

    def vrot_coeffs(self, x: CtSet, r: int, img_len: int, masks) -> CtSet:
        m = np.ascontiguousarray(masks, dtype=np.int64)
        return self._set(load().he_vrot_coeffs, self.h, x.h, r, img_len, _ptr(m, P_I64))

    def vr_encrypt_matrix_a(self, A, ct_id_base: int = 0) -> CtSet:
        A = _f64(A)
        return self._set(load().he_vr_encrypt_matrix_a, self.h, _ptr(A, P_D), A.shape[0], A.shape[1], ct_id_base)

    def vr_encrypt_matrix_b(self, B, ct_id_base: int = 0) -> CtSet:
        B = _f64(B)
        return self._set(load().he_vr_encrypt_matrix_b, self.h, _ptr(B, P_D), B.shape[0], B.shape[1], ct_id_base)

    def vr_matmul(self, A: CtSet, Bbar: CtSet, m: int, n: int, p: int) -> CtSet:
        return self._set(load().he_vr_matmul, self.h, A.h, Bbar.h, m, n, p)

    def vr_matmul_coeffs(self, A: CtSet, Bbar: CtSet, m: int, n: int, p: int, masks) -> CtSet:
        mm = np.ascontiguousarray(masks, dtype=np.int64)
        return self._set(load().he_vr_matmul_coeffs, self.h, A.h, Bbar.h, m, n, p, _ptr(mm, P_I64))

    def vr_encrypt_images(self, px, block_h: int, block_w: int, ct_id_base: int = 0) -> CtSet:
        px = _f64(px)
        b, h, w = px.shape
        return self._set(load().he_vr_encrypt_images, self.h, _ptr(px, P_D), b, h, w, block_h, block_w, ct_id_base)

    def vr_encrypt_kernels(self, K, k0: float, h: int, w: int, block_h: int, block_w: int,
                           limbs: Optional[int] = None, ct_id_base: int = 0):
        K = _f64(K)
        ks, bs = ctypes.c_void_p(), ctypes.c_void_p()
        check(load().he_vr_encrypt_kernels(self.h, _ptr(K, P_D), K.shape[0], float(k0), h, w, block_h, block_w,
                                           self.L1 if limbs is None else limbs, ct_id_base, ctypes.byref(ks),
                                           ctypes.byref(bs)))
        return CtSet(self, ks.value), CtSet(self, bs.value)

    def vr_conv2d(self, x: CtSet, kernels: CtSet, bias: CtSet, h: int, w: int, k: int, block_h: int,
                  block_w: int) -> CtSet:
        return self._set(load().he_vr_conv2d, self.h, x.h, kernels.h, bias.h, h, w, k, block_h, block_w)

    def vr_conv2d_coeffs(self, x: CtSet, kernels: CtSet, bias: CtSet, k: int, block_w: int, masks) -> CtSet:
        m = np.ascontiguousarray(masks, dtype=np.int64)
        return self._set(load().he_vr_conv2d_coeffs, self.h, x.h, kernels.h, bias.h, k, block_w, _ptr(m, P_I64))

    def reform(self, x: CtSet, gap: int, h_valid: int, block_stride: int) -> CtSet:
        return self._set(load().he_reform, self.h, x.h, gap, h_valid, block_stride)

    def reform_coeffs(self, x: CtSet, gap: int, h_valid: int, masks) -> CtSet:
        m = np.ascontiguousarray(masks, dtype=np.int64)
        return self._set(load().he_reform_coeffs, self.h, x.h, gap, h_valid, _ptr(m, P_I64))

    def encrypt_conv_weights(self, K, limbs: Optional[int] = None, ct_id_base: int = 0) -> CtSet:
        K = _f64(K)
        c_out, c_in, k, _ = K.shape
        return self._set(load().he_encrypt_conv_weights, self.h, _ptr(K, P_D), c_out, c_in, k,
                         self.L1 if limbs is None else limbs, ct_id_base)

    def conv2d_enc(self, x: CtSet, c_in: int, gap: int, Wct: CtSet, bias, c_out: int, k: int, stride: int) -> CtSet:
        b = None if bias is None else _f64(bias)
        return self._set(load().he_conv2d_enc, self.h, x.h, c_in, gap, Wct.h, None if b is None else _ptr(b, P_D),
                         c_out, k, stride)

    def poly_act(self, x: CtSet, coeffs: Sequence[float]):
        c = _f64(coeffs)
        check(load().he_poly_act(self.h, x.h, _ptr(c, P_D), len(coeffs) - 1))
        return x

    def square(self, x: CtSet) -> CtSet:
        return self.poly_act(x, [0.0, 0.0, 1.0])

    def fc_prepare(self, W, c_in: int, h_valid: int, w_in: int, gap: int, block_stride: int, batch: int,
                   limbs: int) -> PtSet:
        W = _f64(W)
        out = ctypes.c_void_p()
        check(load().he_fc_prepare(self.h, _ptr(W, P_D), W.shape[0], c_in, h_valid, w_in, gap, block_stride, batch,
                                   limbs, ctypes.byref(out)))
        return PtSet(out.value)

    def fc_prepare_coeffs(self, pts, gap: int, block_stride: int, limbs: int) -> PtSet:
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        out_dim, c_in, w_in, _ = pts.shape
        out = ctypes.c_void_p()
        check(load().he_fc_prepare_coeffs(self.h, _ptr(pts, P_I64), out_dim, c_in, w_in, gap, block_stride, limbs,
                                          ctypes.byref(out)))
        return PtSet(out.value)

    def fc_apply(self, x: CtSet, pts: PtSet, bias) -> CtSet:
        b = None if bias is None else _f64(bias)
        return self._set(load().he_fc_apply, self.h, x.h, pts.h, None if b is None else _ptr(b, P_D))

    def fc_partial(self, x: CtSet, pts: PtSet, first: int) -> CtSet:
        """Sums over input columns first .. first + x.n - 1, before the rescale (he_fc_partial)."""
        return self._set(load().he_fc_partial, self.h, x.h, pts.h, first)

    def fc_finish(self, sums: CtSet, pts: PtSet, bias) -> CtSet:
        """Rescale, relinearisation, rotate-and-add and bias of full sums (he_fc_finish)."""
        b = None if bias is None else _f64(bias)
        return self._set(load().he_fc_finish, self.h, sums.h, pts.h, None if b is None else _ptr(b, P_D))

    def pack_blocks(self, sets: Sequence[CtSet], masks: PtSet) -> CtSet:
        """rescale(sum_t masks_t * sets_t) (he_pack_blocks)."""
        arr = (ctypes.c_void_p * len(sets))(*[s.h.value for s in sets])
        return self._set(load().he_pack_blocks, self.h, arr, len(sets), masks.h)

    def rotate(self, x: CtSet, steps: Sequence[int]) -> CtSet:
        st = (ctypes.c_int32 * len(steps))(*steps)
        return self._set(load().he_rotate, self.h, x.h, st, len(steps))

    def mul(self, a: CtSet, b: CtSet) -> CtSet:
        return self._set(load().he_mul, self.h, a.h, b.h)

    def add(self, a: CtSet, b: CtSet) -> CtSet:
        return self._set(load().he_add, self.h, a.h, b.h)

    def add_slots(self, x: CtSet, v) -> CtSet:
        """In place: component 0 of every ciphertext gains the slot vector(s) v ([N/2] for all,
        or [n][N/2] one per ciphertext), encoded at x's scale."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        n_vec = 1 if v.ndim == 1 else v.shape[0]
        full = np.zeros((n_vec, self.N // 2))
        full[:, : v.shape[-1]] = v.reshape(n_vec, -1)
        check(load().he_add_slots(self.h, x.h, _ptr(full, P_D), n_vec))
        return x

    def add_plain_coeffs(self, x: CtSet, m) -> CtSet:
        """In place: component 0 of every ciphertext gains the encoded plaintext(s) m ([N] or [n][N])."""
        mm = np.ascontiguousarray(m, dtype=np.int64)
        n_vec = 1 if mm.ndim == 1 else mm.shape[0]
        check(load().he_add_plain_coeffs(self.h, x.h, _ptr(mm, P_I64), n_vec))
        return x

    def drop_levels(self, x: CtSet, limbs: int) -> CtSet:
        """A new set: x modulo its first `limbs` primes (scale unchanged)."""
        return self._set(load().he_ctset_drop_levels, self.h, x.h, limbs)

    def relinearize(self, x: CtSet) -> CtSet:
        check(load().he_relinearize(self.h, x.h))
        return x

    def rescale(self, x: CtSet) -> CtSet:
        check(load().he_rescale(self.h, x.h))
        return x

    # ---- decryption ----
    def decrypt_slots(self, x: CtSet) -> np.ndarray:
        n = x.n
        out = np.zeros((n, self.slots), np.float64)
        check(load().he_decrypt_slots(self.h, x.h, _ptr(out, P_D), out.size))
        return out

    def import_raw(self, words, limbs: int, scale: float) -> CtSet:
        """A set from NTT-domain words [n][2][limbs][N] (as CtSet.export_raw writes them)."""
        a = np.ascontiguousarray(words, dtype=np.uint64)
        n = a.size // (2 * limbs * self.N)
        return self._set(load().he_ctset_import_raw, self.h, _ptr(a, P_U64), n, limbs, float(scale))

    def concat(self, sets: Sequence[CtSet]) -> CtSet:
        """One set of the given sets' ciphertexts in order (same level, scale and components)."""
        arr = (ctypes.c_void_p * len(sets))(*[s.h.value for s in sets])
        return self._set(load().he_ctset_concat, self.h, arr, len(sets))

    def import_words(self, src, n: int, polys: int, limbs: int, scale: float) -> CtSet:
        """A set of n ciphertexts of `polys` components from NTT-domain words [n][polys][limbs][N]
        in a numpy uint64 array or a 64-bit torch tensor (host or the context's GPU)."""
        ptr, on_dev, size = _words_buffer(src)
        assert size >= n * polys * limbs * self.N, "source too small"
        return self._set(load().he_ctset_import_words, self.h, ptr, on_dev, n, polys, limbs, float(scale))

    def decrypt_matrix(self, C: CtSet, m: int, p: int) -> np.ndarray:
        out = np.zeros((m, p), np.float64)
        check(load().he_decrypt_matrix(self.h, C.h, m, p, _ptr(out, P_D)))
        return out

    def decrypt_matrix_volley(self, C: CtSet, m: int, p: int) -> np.ndarray:
        out = np.zeros((m, p), np.float64)
        check(load().he_decrypt_matrix_volley(self.h, C.h, m, p, _ptr(out, P_D)))
        return out

    def decrypt_image(self, x: CtSet, batch: int, block_stride: int, gap: int, h_valid: int) -> np.ndarray:
        """[batch][n_ct][h_valid]: per ciphertext (column), the valid rows."""
        out = np.zeros((batch, x.n, h_valid), np.float64)
        check(load().he_decrypt_image(self.h, x.h, batch, block_stride, gap, h_valid, _ptr(out, P_D), out.size))
        return out

    def ntt(self, host, first_prime: int = 0, inverse: bool = False) -> np.ndarray:
        a = np.ascontiguousarray(host, dtype=np.uint64).copy()
        shp = a.shape
        a3 = a.reshape(-1, shp[-2] if a.ndim >= 2 else 1, self.N)
        check(load().he_ntt(self.h, _ptr(a3, P_U64), a3.shape[0], a3.shape[1], first_prime, int(inverse)))
        return a3.reshape(shp)


class Server:
    """he_server: continuous batching of encrypted CNN requests (include/he_gb300.h).

    Requests are host arrays of uint64 words (page-locked ones let the upload
    overlap the running batch); each must stay alive until its request is
    done, which this class guarantees by holding a reference until take()."""

    def __init__(self, ctx: Context, weights_by_side, hbm_budget_bytes: int, max_blocks: int,
                 start_paused: bool = False):
        """weights_by_side: {side: CnnWeights}; the conv layers of the first entry serve every side."""
        sides = sorted(weights_by_side)
        w0 = weights_by_side[sides[0]]
        self._keep = [_f64(w0.conv1_w), _f64(w0.conv1_b), _f64(w0.conv2_w), _f64(w0.conv2_b)]
        fcw = [_f64(weights_by_side[s].fc_w) for s in sides]
        fcb = [_f64(weights_by_side[s].fc_b) for s in sides]
        self._keep += fcw + fcb
        PD = ctypes.POINTER(ctypes.c_double)
        self._fcw = (PD * len(sides))(*[_ptr(a, PD) for a in fcw])
        self._fcb = (PD * len(sides))(*[_ptr(a, PD) for a in fcb])
        self._sides = (ctypes.c_int * len(sides))(*sides)
        d = ServerDesc(_ptr(self._keep[0], PD), _ptr(self._keep[1], PD), _ptr(self._keep[2], PD),
                       _ptr(self._keep[3], PD), len(sides), self._sides, self._fcw, self._fcb,
                       int(hbm_budget_bytes), int(max_blocks), int(start_paused))
        h = ctypes.c_void_p()
        check(load().he_server_create(ctx.h, ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.ctx = ctx
        self.sides = sides
        self._held = {}

    def request_words(self, side: int) -> int:
        n = ctypes.c_size_t()
        check(load().he_server_request_words(self.h, side, ctypes.byref(n)))
        return n.value

    def submit(self, words: np.ndarray, side: int) -> int:
        assert words.dtype == np.uint64 and words.flags.c_contiguous
        rid = ctypes.c_uint64()
        check(load().he_server_submit(self.h, ctypes.c_void_p(words.ctypes.data), words.size, side,
                                      ctypes.byref(rid)))
        self._held[rid.value] = words
        return rid.value

    def submit_ptr(self, ptr: int, n_words: int, side: int) -> int:
        """Submit from a raw host address (e.g. page-locked memory); the caller keeps it alive."""
        rid = ctypes.c_uint64()
        check(load().he_server_submit(self.h, ctypes.c_void_p(ptr), n_words, side, ctypes.byref(rid)))
        return rid.value

    def poll(self, rid: int) -> int:
        st = ctypes.c_int()
        check(load().he_server_poll(self.h, rid, ctypes.byref(st)))
        return st.value

    def wait(self, rid: int, timeout_ms: int) -> bool:
        """True once the request is done or failed, False if timeout_ms passed first."""
        st = ctypes.c_int()
        rc = load().he_server_wait(self.h, rid, int(timeout_ms), ctypes.byref(st))
        if rc == HE_E_TIMEOUT:
            return False
        check(rc)
        return True

    def take(self, rid: int):
        """(logits CtSet, slot block, times_ms [submit, admit, start, done])."""
        out = ctypes.c_void_p()
        blk = ctypes.c_int()
        t = np.zeros(4, np.float64)
        try:
            check(load().he_server_take(self.h, rid, ctypes.byref(out), ctypes.byref(blk), _ptr(t, P_D)))
        finally:
            self._held.pop(rid, None)
        return CtSet(self.ctx, out.value), blk.value, t

    def result_words(self) -> int:
        n = ctypes.c_size_t()
        check(load().he_server_result_words(self.h, ctypes.byref(n)))
        return n.value

    def take_host(self, rid: int, out: np.ndarray):
        """Result words into `out` (uint64, page-locked for a direct copy): (slot block, times_ms)."""
        assert out.dtype == np.uint64 and out.flags.c_contiguous
        blk = ctypes.c_int()
        t = np.zeros(4, np.float64)
        try:
            check(load().he_server_take_host(self.h, rid, ctypes.c_void_p(out.ctypes.data), out.size,
                                             ctypes.byref(blk), _ptr(t, P_D)))
        finally:
            self._held.pop(rid, None)
        return blk.value, t

    def pause(self, on: bool):
        check(load().he_server_pause(self.h, int(on)))

    def cancel(self, rid: int):
        """Withdraw a request (include/he_gb300.h he_server_cancel); its host words may be reused
        once it reads HE_REQ_CANCELLED and is not running."""
        check(load().he_server_cancel(self.h, rid))

    def stats(self):
        c = np.zeros(7, np.uint64)
        b = (ctypes.c_size_t * 4)()
        check(load().he_server_stats(self.h, _ptr(c, P_U64), b))
        keys = ("submitted", "waiting", "admitted", "done", "failed", "batches", "cancelled")
        out = {k: int(v) for k, v in zip(keys, c)}
        out.update(held_bytes=b[0], max_held_bytes=b[1], reserve_bytes=b[2], pool_high_bytes=b[3])
        return out

    def close(self):
        if getattr(self, "h", None):
            load().he_server_destroy(self.h)
            self.h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sched_simulate(arrival_ms, side, nbytes, sides, base_ms, per_request_ms, budget: int, reserve: int,
                   max_blocks: int, out_bytes: int = 0):
    """he_sched_simulate: the server's scheduler on a simulated GPU. Returns a dict of per-request arrays."""
    n = len(arrival_ms)
    arr = _f64(arrival_ms)
    sd = np.ascontiguousarray(side, dtype=np.int32)
    nb = np.ascontiguousarray(nbytes, dtype=np.uint64)
    ss = np.ascontiguousarray(sides, dtype=np.int32)
    bm, pm = _f64(base_ms), _f64(per_request_ms)
    batch = np.zeros(n, np.int64)
    block = np.zeros(n, np.int32)
    adm, st, dn = np.zeros(n), np.zeros(n), np.zeros(n)
    mh = ctypes.c_size_t()
    SZP = ctypes.POINTER(ctypes.c_size_t)
    check(load().he_sched_simulate(n, _ptr(arr, P_D), _ptr(sd, P_I), _ptr(nb, SZP), len(ss), _ptr(ss, P_I),
                                   _ptr(bm, P_D), _ptr(pm, P_D), int(budget), int(reserve), int(max_blocks),
                                   int(out_bytes), _ptr(batch, P_I64), _ptr(block, P_I), _ptr(adm, P_D),
                                   _ptr(st, P_D), _ptr(dn, P_D), ctypes.byref(mh)))
    return dict(batch=batch, block=block, admit_ms=adm, start_ms=st, done_ms=dn, max_held=mh.value)
