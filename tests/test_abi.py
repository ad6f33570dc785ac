"""The C-ABI library loads and exports every entry point include/spamm.h declares
(no GPU needed; compute calls are not made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"SPAMM_API\s+[\w\s\*]+?\b(spamm_\w+)\s*\(", txt))
    return names


def test_header_declares_entry_points():
    names = declared()
    assert {"spamm_tree_build", "spamm_multiply", "spamm_stats", "spamm_triples"} <= names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build_library()
    from paper_1011_3534_gb300 import spamm as S
    lib = ctypes.CDLL(S.lib_path())
    for name in declared():
        assert hasattr(lib, name), name
    assert set(S.EXPORTS) >= declared()


def test_internal_symbols_hidden():
    from paper_1011_3534_gb300 import spamm as S
    lib = ctypes.CDLL(S.lib_path())
    assert not hasattr(lib, "_Z11launch_cullP12spamm_tree_sS0_S0_dPjiP11CUstream_stPi")


def test_errors_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1011_3534_gb300 import spamm as S
    h = ctypes.c_void_p()
    assert S.LIB.spamm_ctx_create(0, None, 0, ctypes.byref(h)) == S.SPAMM_ECUDA
    assert S.LIB.spamm_ctx_create(0, None, 0, None) == S.SPAMM_EINVAL
    assert S.LIB.spamm_multiply(None, None, None, 0.0, 0, 0, None) == S.SPAMM_EINVAL
    assert S.LIB.spamm_tree_free(None) == S.SPAMM_EINVAL
    assert S.LIB.spamm_stats(None, None) == S.SPAMM_EINVAL


def test_every_entry_point_refuses_null_arguments():
    # each entry point, called with null handles and pointers and zero sizes, returns
    # SPAMM_EINVAL (or -1 / a message for the queries) and touches no memory or device
    from paper_1011_3534_gb300 import spamm as S
    for name in sorted(declared()):
        f = getattr(S.LIB, name)
        assert f.argtypes is not None, f"{name}: the binding declares no argument types"
        args = []
        for t in f.argtypes:
            if t in (ctypes.c_double, ctypes.c_float):
                args.append(0.0)
            elif t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64):
                args.append(0)
            else:
                args.append(None)
        r = f(*args)
        if name == "spamm_last_error":
            assert isinstance(r, bytes) and r
        elif name in ("spamm_kernel_launches", "spamm_mlp_num_params"):
            assert r == -1, name
        else:
            assert r == S.SPAMM_EINVAL, (name, r)
