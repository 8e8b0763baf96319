"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/kclique.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kclique.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:kclique|kc_server)_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["kclique_prepare", "kclique_count", "kclique_list", "kclique_info", "kclique_release",
                 "kclique_status_string", "kclique_count_batch", "kclique_edge_data"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2311_13798_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    lib.kclique_status_string.restype = ctypes.c_char_p
    assert lib.kclique_status_string(0) == b"ok"
    assert b"2^128" in lib.kclique_status_string(-6)


def test_binding_names_match_the_abi():
    from paper_2311_13798_gb300 import kclique
    for name in _declared():
        if name in ("kclique_release", "kclique_last_error") or name.startswith("kc_server_"):
            continue  # the server's calls are wrapped by serve.KCliqueServer
        assert hasattr(kclique, name), name


def test_binding_rejects_bad_arguments_without_gpu():
    from paper_2311_13798_gb300 import kclique
    lib = kclique.library()
    r = kclique.KcResult()
    # null graph handle: rejected on the host before any CUDA call
    assert lib.kclique_count(None, 4, None, None, ctypes.byref(r)) == kclique.KC_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.kclique_prepare(None, None, 0, 0, 0, None, ctypes.byref(h)) == kclique.KC_ERR_INVALID_ARG


def test_server_structs_match_the_header():
    """The binding's server structs have the sizes of the C ones (fields of 8-byte
    alignment in the order the header gives)."""
    from paper_2311_13798_gb300 import kclique as K
    assert ctypes.sizeof(K.KcRequest) == 4 + 4 + 8 + 8 + 8 + 8 + 8 + 4 + 4 + 8 + 4 * 4
    assert ctypes.sizeof(K.KcCompletion) == 8 + 8 + 4 + 4 + 4 + 4 + 8 * 4 + 8 + 8
    assert ctypes.sizeof(K.KcServerBackend) == 5 * 8
    assert ctypes.sizeof(K.KcServerConfig) == 8 + 4 + 4 + 4 + 4 + 4 + 4 + ctypes.sizeof(K.KcParams) + 8


def test_server_rejects_bad_requests_without_gpu():
    from paper_2311_13798_gb300 import kclique as K
    lib = K.library()
    t = ctypes.c_uint64()
    assert lib.kc_server_submit(None, None, ctypes.byref(t), None) == K.KC_ERR_INVALID_ARG
    assert lib.kc_server_create(None, None) == K.KC_ERR_INVALID_ARG


def test_flag_and_limit_constants_match_the_header():
    """Every numeric #define of include/kclique.h has the same value in the binding."""
    import re
    from paper_2311_13798_gb300 import kclique
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "kclique.h")).read()
    found = re.findall(r"#define (KC_[A-Z0-9_]+) (0x[0-9a-fA-F]+|\d+)u?\b", hdr)
    assert len(found) >= 7
    for name, val in found:
        assert getattr(kclique, name) == int(val, 0), name
