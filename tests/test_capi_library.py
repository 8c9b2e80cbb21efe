"""The CUDA library builds for sm_103a and exports every entry point that
include/he_gb300.h declares (no GPU needed: nothing here calls into CUDA)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

from tests.conftest import ROOT


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "he_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 30
    for s in syms:
        assert hasattr(lib, s), s
    # the Python binding covers exactly the declared entry points
    assert sorted(_lib.SIGNATURES) == syms
    # exported dynamic symbols of the library, for the record
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    for s in syms:
        assert re.search(rf"\bT {s}\b", out), s
    assert lib.he_last_error is not None


def test_library_is_built_for_sm_103a_only():
    from paper_2512_18646_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path):
    import pytest
    from paper_2512_18646_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_volley_geometry_matches_oracle_layout():
    """Host-only arithmetic of the library (no CUDA call): the zero-rotation matmul
    geometry equals the oracle layout's, and misfits are rejected."""
    import pytest
    import __graft_entry__
    __graft_entry__.build()
    from oracle import layouts
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HeError
    for slots, m, p in [(64, 5, 8), (64, 4, 4), (32, 3, 16), (64, 9, 1), (512, 20, 32), (32768, 256, 256),
                        (32768, 16, 256), (32768, 128, 128), (32768, 255, 2), (32768, 100, 64)]:
        M, per, G, _ = layouts.volley_geometry(slots, m, p)
        assert api.volley_geometry(slots, m, p) == (M, per, G)
    for slots, m, p in [(64, 5, 3), (16, 20, 4), (16, 10, 8)]:  # p does not divide, or no block fits
        with pytest.raises(HeError):
            api.volley_geometry(slots, m, p)


def test_corrupted_or_freed_handles_are_refused_without_touching_them():
    """Every entry point checks its handle arguments against the library's registry of live handles
    before it reads them: a pointer that is no handle (here a zeroed host buffer, and a stray address)
    gets HE_E_ARG, and the free / destroy calls ignore it. No CUDA call is reached."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import _lib
    lib = _lib.load()
    fake = ctypes.create_string_buffer(4096)
    for bogus in (ctypes.cast(fake, ctypes.c_void_p), ctypes.c_void_p(0x1000)):
        n, lv, polys = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sc = ctypes.c_double()
        assert lib.he_ctset_info(bogus, ctypes.byref(n), ctypes.byref(lv), ctypes.byref(sc),
                                 ctypes.byref(polys)) == _lib.HE_E_ARG
        assert b"invalid handle" in lib.he_last_error()
        assert lib.he_ctx_synchronize(bogus) == _lib.HE_E_ARG
        assert lib.he_keygen(bogus, None, 0) == _lib.HE_E_ARG
        st = ctypes.c_int()
        assert lib.he_server_poll(bogus, ctypes.c_uint64(1), ctypes.byref(st)) == _lib.HE_E_ARG
        assert lib.he_server_wait(bogus, ctypes.c_uint64(1), 10, ctypes.byref(st)) == _lib.HE_E_ARG
        out = ctypes.c_void_p()
        assert lib.he_rotate(bogus, bogus, None, 0, ctypes.byref(out)) == _lib.HE_E_ARG
        # freeing what is no handle does nothing
        lib.he_ctset_free(bogus)
        lib.he_ptset_free(bogus)
        lib.he_graph_destroy(bogus)
        lib.he_server_destroy(bogus)
        lib.he_ctx_destroy(bogus)
    assert fake.raw == b"\0" * 4096  # never written
