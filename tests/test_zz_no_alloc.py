"""he_rescale_noalloc: the rescale for callers that cannot allocate device
memory during the call (a serving loop with a fixed footprint, a framework
that owns every device allocation, an exhausted memory quota).

The caller provides the output buffer; the library's scratch is a fixed
16 MiB array held on the GPU. Its results must equal he_rescale's, bit for bit
(the integer-exact bar of every parity test here), on two calls in a row --
the second call runs on scratch that still holds the first call's data.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rescale_noalloc_matches_rescale_on_two_calls():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2512_18646_gb300 import api, load
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_OK, check

    lib = load()
    torch.cuda.init()
    g = api.Context(12, (60, 45, 45, 45, 45), 2, 60, 2, 45.0, seed=17)
    g.keygen([])
    rng = np.random.default_rng(17)
    for call, (n_ct, limbs) in enumerate([(3, 5), (2, 4)]):
        m = rng.integers(-(1 << 44), 1 << 44, size=(n_ct, g.N), dtype=np.int64)
        x = g.encrypt_coeffs(m, limbs, g.scale, ct_id_base=100 * call)
        _, _, sc = x.info()
        ref = x.slice(0, n_ct)
        g.rescale(ref)
        # caller-owned output buffer (this test allocates it; the entry point does not)
        out = torch.zeros(n_ct * 2 * (limbs - 1) * g.N, dtype=torch.int64, device="cuda")
        out_scale = ctypes.c_double()
        rc = lib.he_rescale_noalloc(g.h, ctypes.c_void_p(x.device_ptr()), n_ct, limbs, sc,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.byref(out_scale))
        check(rc)
        g.synchronize()
        torch.cuda.synchronize()
        got_ntt = out.cpu().numpy().view(np.uint64).reshape(n_ct * 2, limbs - 1, g.N)
        got = g.ntt(got_ntt, 0, inverse=True).reshape(n_ct, 2, limbs - 1, g.N)
        assert np.array_equal(got, ref.export()), f"call {call}"
        assert out_scale.value == ref.scale

    # sizes beyond the 16 MiB scratch are rejected with a clear error
    big = g.encrypt_coeffs(np.zeros((1, g.N), np.int64), 5, g.scale)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.he_rescale_noalloc(g.h, ctypes.c_void_p(big.device_ptr()), 1 << 10, 5, g.scale,
                                ctypes.c_void_p(out.data_ptr()), None)
    assert rc == HE_E_ARG
    assert b"exceeds the scratch" in lib.he_last_error()
    assert rc != HE_OK
