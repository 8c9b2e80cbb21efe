"""ctypes binding of libhegb300.so (the C ABI in include/he_gb300.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Loading fails loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhegb300.so")

HE_OK, HE_E_ARG, HE_E_LEVEL, HE_E_NOKEY, HE_E_SCALE, HE_E_OOM, HE_E_TIMEOUT, HE_E_CUDA, HE_E_UNIMPL, HE_E_STATE = range(10)
ERROR_NAMES = {1: "HE_E_ARG", 2: "HE_E_LEVEL", 3: "HE_E_NOKEY", 4: "HE_E_SCALE", 5: "HE_E_OOM", 6: "HE_E_TIMEOUT",
               7: "HE_E_CUDA", 8: "HE_E_UNIMPL", 9: "HE_E_STATE"}


class HeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class ParamsDesc(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int), ("n_q", ctypes.c_int), ("q_bits", ctypes.POINTER(ctypes.c_int)),
                ("n_special", ctypes.c_int), ("special_bits", ctypes.c_int), ("alpha", ctypes.c_int),
                ("log_scale", ctypes.c_double), ("sigma", ctypes.c_double)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("conv1_w", ctypes.POINTER(ctypes.c_double)), ("conv1_b", ctypes.POINTER(ctypes.c_double)),
                ("conv2_w", ctypes.POINTER(ctypes.c_double)), ("conv2_b", ctypes.POINTER(ctypes.c_double)),
                ("n_sides", ctypes.c_int), ("sides", ctypes.POINTER(ctypes.c_int)),
                ("fc_w", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("fc_b", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("hbm_budget_bytes", ctypes.c_size_t), ("max_blocks", ctypes.c_int), ("start_paused", ctypes.c_int)]


HE_REQ_WAITING, HE_REQ_ADMITTED, HE_REQ_RUNNING, HE_REQ_DONE, HE_REQ_FAILED, HE_REQ_CANCELLED = range(6)

V = ctypes.c_void_p
PV = ctypes.POINTER(ctypes.c_void_p)
I = ctypes.c_int
U64 = ctypes.c_uint64
D = ctypes.c_double
SZ = ctypes.c_size_t
P_U64 = ctypes.POINTER(ctypes.c_uint64)
P_I64 = ctypes.POINTER(ctypes.c_int64)
P_I32 = ctypes.POINTER(ctypes.c_int32)
P_I = ctypes.POINTER(ctypes.c_int)
P_D = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every entry point declared in include/he_gb300.h
SIGNATURES = {
    "he_ctx_create": (I, [ctypes.POINTER(ParamsDesc), U64, V, PV]),
    "he_ctx_destroy": (None, [V]),
    "he_ctx_synchronize": (I, [V]),
    "he_ctx_primes": (I, [V, P_U64, I]),
    "he_ctx_info": (I, [V, P_I, P_I, P_I, P_I, P_D]),
    "he_ctx_set_work_budget": (I, [V, SZ]),
    "he_ctx_set_tensor_cores": (I, [V, I]),
    "he_keygen": (I, [V, P_I32, I]),
    "he_keys_export": (I, [V, P_U64, SZ, ctypes.POINTER(SZ)]),
    "he_keys_import": (I, [V, P_U64, SZ]),
    "he_encrypt_image": (I, [V, P_D, I, I, I, I, U64, PV]),
    "he_encrypt_matrix_a": (I, [V, P_D, I, I, U64, PV]),
    "he_encrypt_matrix_b": (I, [V, P_D, I, I, U64, PV]),
    "he_volley_geometry": (I, [I, I, I, P_I, P_I, P_I]),
    "he_encrypt_matrix_a_volley": (I, [V, P_D, I, I, I, U64, PV]),
    "he_encrypt_coeffs": (I, [V, P_I64, I, I, D, U64, PV]),
    "he_matmul": (I, [V, V, V, I, I, PV]),
    "he_matmul_range": (I, [V, V, V, I, I, I, I, PV]),
    "he_matmul_batched": (I, [V, I, PV, PV, P_I, P_I, PV]),
    "he_matmul_volley": (I, [V, V, V, PV]),
    "he_matmul_bsgs": (I, [V, V, V, I, I, I, PV]),
    "he_conv2d": (I, [V, V, I, I, P_D, P_D, I, I, I, PV]),
    "he_vrot": (I, [V, V, I, I, I, PV]),
    "he_vrot_coeffs": (I, [V, V, I, I, P_I64, PV]),
    "he_vr_encrypt_matrix_a": (I, [V, P_D, I, I, U64, PV]),
    "he_vr_encrypt_matrix_b": (I, [V, P_D, I, I, U64, PV]),
    "he_vr_matmul": (I, [V, V, V, I, I, I, PV]),
    "he_vr_matmul_coeffs": (I, [V, V, V, I, I, I, P_I64, PV]),
    "he_vr_encrypt_images": (I, [V, P_D, I, I, I, I, I, U64, PV]),
    "he_vr_encrypt_kernels": (I, [V, P_D, I, D, I, I, I, I, I, U64, PV, PV]),
    "he_vr_conv2d": (I, [V, V, V, V, I, I, I, I, I, PV]),
    "he_vr_conv2d_coeffs": (I, [V, V, V, V, I, I, P_I64, PV]),
    "he_reform": (I, [V, V, I, I, I, PV]),
    "he_reform_coeffs": (I, [V, V, I, I, P_I64, PV]),
    "he_encrypt_conv_weights": (I, [V, P_D, I, I, I, I, U64, PV]),
    "he_conv2d_enc": (I, [V, V, I, I, V, P_D, I, I, I, PV]),
    "he_poly_act": (I, [V, V, P_D, I]),
    "he_fc_prepare": (I, [V, P_D, I, I, I, I, I, I, I, I, PV]),
    "he_fc_prepare_coeffs": (I, [V, P_I64, I, I, I, I, I, I, PV]),
    "he_ptset_free": (None, [V]),
    "he_fc_apply": (I, [V, V, V, P_D, PV]),
    "he_fc_partial": (I, [V, V, V, I, PV]),
    "he_fc_finish": (I, [V, V, V, P_D, PV]),
    "he_fc": (I, [V, V, P_D, P_D, I, I, I, I, I, I, I, PV]),
    "he_pack_blocks": (I, [V, PV, I, V, PV]),
    "he_rotate": (I, [V, V, P_I32, I, PV]),
    "he_mul": (I, [V, V, V, PV]),
    "he_relinearize": (I, [V, V]),
    "he_rescale": (I, [V, V]),
    "he_add": (I, [V, V, V, PV]),
    "he_add_slots": (I, [V, V, P_D, I]),
    "he_add_plain_coeffs": (I, [V, V, P_I64, I]),
    "he_ctset_drop_levels": (I, [V, V, I, PV]),
    "he_decrypt_slots": (I, [V, V, P_D, SZ]),
    "he_decrypt_matrix": (I, [V, V, I, I, P_D]),
    "he_decrypt_matrix_volley": (I, [V, V, I, I, P_D]),
    "he_decrypt_image": (I, [V, V, I, I, I, I, P_D, SZ]),
    "he_ctset_export": (I, [V, P_U64, SZ]),
    "he_ctset_export_async": (I, [V, P_U64, SZ, P_U64]),
    "he_ctset_export_wait": (I, [V, U64]),
    "he_ctset_import": (I, [V, P_U64, I, I, D, PV]),
    "he_ctset_export_raw": (I, [V, P_U64, SZ]),
    "he_ctset_import_raw": (I, [V, P_U64, I, I, D, PV]),
    "he_ctset_info": (I, [V, P_I, P_I, P_D, P_I]),
    "he_ctset_device_ptr": (I, [V, ctypes.POINTER(P_U64)]),
    "he_ctset_import_async": (I, [V, P_U64, I, I, D, PV]),
    "he_ctset_export_words": (I, [V, P_U64, I, SZ]),
    "he_ctset_import_words": (I, [V, P_U64, I, I, I, I, D, PV]),
    "he_ctset_slice": (I, [V, V, I, I, PV]),
    "he_ctset_concat": (I, [V, PV, I, PV]),
    "he_ctset_free": (None, [V]),
    "he_graph_begin": (I, [V]),
    "he_graph_end": (I, [V, PV]),
    "he_graph_launch": (I, [V]),
    "he_graph_info": (I, [V, P_U64]),
    "he_graph_destroy": (None, [V]),
    "he_ctset_assign": (I, [V, V, V]),
    "he_rescale_noalloc": (I, [V, V, I, I, D, V, P_D]),
    "he_server_create": (I, [V, ctypes.POINTER(ServerDesc), PV]),
    "he_server_request_words": (I, [V, I, ctypes.POINTER(SZ)]),
    "he_server_submit": (I, [V, V, SZ, I, P_U64]),
    "he_server_poll": (I, [V, U64, P_I]),
    "he_server_wait": (I, [V, U64, I, P_I]),
    "he_server_take": (I, [V, U64, PV, P_I, P_D]),
    "he_server_result_words": (I, [V, ctypes.POINTER(SZ)]),
    "he_server_take_host": (I, [V, U64, V, SZ, P_I, P_D]),
    "he_server_pause": (I, [V, I]),
    "he_server_stats": (I, [V, P_U64, ctypes.POINTER(SZ)]),
    "he_server_cancel": (I, [V, U64]),
    "he_debug_fail_allocations": (I, [I]),
    "he_debug_wait_timeout": (I, [V, I]),
    "he_server_destroy": (None, [V]),
    "he_sched_simulate": (I, [I, P_D, P_I, ctypes.POINTER(SZ), I, P_I, P_D, P_D, SZ, SZ, I, SZ, P_I64, P_I, P_D,
                              P_D, P_D, ctypes.POINTER(SZ)]),
    "he_ntt": (I, [V, P_U64, I, I, I, I]),
    "he_ntt_set_geometry": (I, [V, I, I]),
    "he_ntt_autotune": (I, [V, I, P_I, P_I, P_D]),
    "he_calibrate_modmul": (I, [V, P_D]),
    "he_calibrate_mac96": (I, [V, P_D]),
    "he_calibrate_butterfly": (I, [V, I, P_D]),
    "he_kernel_launches": (U64, []),
    "he_profile_enable": (I, [I]),
    "he_profile_read": (I, [ctypes.c_char_p, SZ, P_D, P_U64, P_D, P_D, I, P_I]),
    "he_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (once). Raises if it is missing: there is no CPU fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libhegb300.so not built at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def check(rc: int):
    if rc != HE_OK:
        raise HeError(rc, (load().he_last_error() or b"").decode())
