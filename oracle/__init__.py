"""SpAMM oracle: TEST INFRASTRUCTURE ONLY.

Python access to the plain FP64 CPU SpAMM in `spamm_oracle.c` (Eq. 1 quadtree, Eq. 4
recursion, brute-force leaf triples, naive product) and to the small oracles written
in numpy beside it. Only the test suite, the smoke check and the benchmark's CPU
baseline import this package; the CUDA library never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spamm_oracle.c")
BUILD = os.path.join(HERE, "_build")
MAX_LEVELS = 24


def build(mutant: int = 0, out_dir: str | None = None) -> str:
    """Compile the C oracle with gcc (OpenMP when available); returns the .so path."""
    out_dir = out_dir or BUILD
    os.makedirs(out_dir, exist_ok=True)
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    so = os.path.join(out_dir, name)
    if os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(SRC):
        return so
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
            f"-DORACLE_MUTANT={mutant}", SRC, "-o", so + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(so + ".tmp", so)
    return so


class _Stats(ctypes.Structure):
    _fields_ = [("tested", ctypes.c_int64 * MAX_LEVELS),
                ("culled", ctypes.c_int64 * MAX_LEVELS),
                ("culled_bound", ctypes.c_double * MAX_LEVELS),
                ("leaf_products", ctypes.c_int64)]


@dataclass
class Stats:
    tested: list
    culled: list
    culled_bound: list
    leaf_products: int


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)


def _load(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    lib.oracle_tree_build.argtypes = [_D, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_P)]
    lib.oracle_tree_build.restype = ctypes.c_int
    lib.oracle_tree_free.argtypes = [_P]
    lib.oracle_tree_kmax.argtypes = [_P]
    lib.oracle_tree_kmax.restype = ctypes.c_int32
    lib.oracle_tree_NB.argtypes = [_P]
    lib.oracle_tree_NB.restype = ctypes.c_int32
    lib.oracle_tree_level_norm2.argtypes = [_P, ctypes.c_int32, _D]
    lib.oracle_tree_level_norm2.restype = ctypes.c_int
    lib.oracle_spamm.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int32, _D, _U32,
                                 ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(_Stats)]
    lib.oracle_spamm.restype = ctypes.c_int
    lib.oracle_spamm_ex.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _D, _U32,
                                    ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_Stats)]
    lib.oracle_spamm_ex.restype = ctypes.c_int
    lib.oracle_spamm_values.argtypes = [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, _D]
    lib.oracle_spamm_values.restype = ctypes.c_int
    lib.oracle_spamm_block.argtypes = [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _D]
    lib.oracle_spamm_block.restype = ctypes.c_int
    lib.oracle_triples_flat.argtypes = [_P, _P, ctypes.c_double, _U32, ctypes.c_int64]
    lib.oracle_triples_flat.restype = ctypes.c_int64
    lib.oracle_flat_bound.argtypes = [_P, _P, ctypes.c_double]
    lib.oracle_flat_bound.restype = ctypes.c_double
    lib.oracle_matmul_naive.argtypes = [_D, _D, ctypes.c_int64, _D, ctypes.c_int32]
    lib.oracle_mutant.restype = ctypes.c_int32
    lib.oracle_max_threads.restype = ctypes.c_int32
    return lib


_LIBS: dict[str, ctypes.CDLL] = {}


def lib(mutant: int = 0, out_dir: str | None = None) -> ctypes.CDLL:
    path = build(mutant, out_dir)
    if path not in _LIBS:
        _LIBS[path] = _load(path)
    return _LIBS[path]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


class Tree:
    """Padded quadtree of one FP64 matrix with its per-tier squared Frobenius norms."""

    def __init__(self, A: np.ndarray, leaf: int, L: ctypes.CDLL | None = None):
        A = np.ascontiguousarray(A, dtype=np.float64)
        assert A.ndim == 2 and A.shape[0] == A.shape[1]
        self.L = L or lib()
        self.n = A.shape[0]
        self.leaf = leaf
        h = _P()
        rc = self.L.oracle_tree_build(_dptr(A), self.n, leaf, ctypes.byref(h))
        if rc:
            raise RuntimeError(f"oracle_tree_build failed ({rc})")
        self.h = h
        self.kmax = self.L.oracle_tree_kmax(h)
        self.NB = self.L.oracle_tree_NB(h)

    def norm2(self, level: int) -> np.ndarray:
        d = 1 << level
        out = np.empty((d, d), dtype=np.float64)
        if self.L.oracle_tree_level_norm2(self.h, level, _dptr(out)):
            raise ValueError(level)
        return out

    def __del__(self):
        if getattr(self, "h", None):
            self.L.oracle_tree_free(self.h)
            self.h = None


def spamm(A: Tree, B: Tree, tau: float, *, product: bool = True, triples: bool = False,
          stats: bool = False, threads: int = 1, depth_scaled: bool = False):
    """Eq. 4 from the root. Returns dict(C, triples (recursion order), count, stats).
    depth_scaled: tier k tests against tau * 8^-k (the rigorous variant of Sec. II)."""
    L = A.L
    C = np.empty((A.n, A.n), dtype=np.float64) if product else None
    cnt = ctypes.c_int64(0)
    st = _Stats() if stats else None
    trip = None
    if triples:
        # size the buffer with a norm-only pass first
        rc = L.oracle_spamm_ex(A.h, B.h, tau, int(depth_scaled), 1, None, None, 0, ctypes.byref(cnt), None)
        if rc:
            raise RuntimeError(rc)
        trip = np.empty((max(cnt.value, 1), 3), dtype=np.uint32)
    rc = L.oracle_spamm_ex(A.h, B.h, tau, int(depth_scaled), threads if not (triples or stats) else 1,
                        _dptr(C) if C is not None else None,
                        trip.ctypes.data_as(_U32) if trip is not None else None,
                        trip.shape[0] if trip is not None else 0, ctypes.byref(cnt),
                        ctypes.byref(st) if st is not None else None)
    if rc:
        raise RuntimeError(f"oracle_spamm failed ({rc})")
    out = {"C": C, "count": cnt.value}
    if trip is not None:
        out["triples"] = trip[:cnt.value]
    if st is not None:
        kk = A.kmax + 1
        out["stats"] = Stats(list(st.tested[:kk]), list(st.culled[:kk]),
                             list(st.culled_bound[:kk]), st.leaf_products)
    return out


def spamm_values(A: Tree, B: Tree, Av: Tree, Bv: Tree, tau: float, threads: int = 1) -> np.ndarray:
    """SpAMM with the tier tests of A, B and the leaf products of Av, Bv."""
    C = np.empty((A.n, A.n), dtype=np.float64)
    if A.L.oracle_spamm_values(A.h, B.h, Av.h, Bv.h, tau, threads, _dptr(C)):
        raise RuntimeError("oracle_spamm_values failed")
    return C


def spamm_block(A: Tree, B: Tree, tau: float, i: int, j: int, Av: Tree | None = None,
                Bv: Tree | None = None) -> np.ndarray:
    out = np.empty((A.leaf, A.leaf), dtype=np.float64)
    if A.L.oracle_spamm_block(A.h, B.h, Av.h if Av else None, Bv.h if Bv else None, tau, i, j,
                              _dptr(out)):
        raise ValueError((i, j))
    return out


def triples_flat(A: Tree, B: Tree, tau: float) -> np.ndarray:
    cnt = A.L.oracle_triples_flat(A.h, B.h, tau, None, 0)
    trip = np.empty((max(cnt, 1), 3), dtype=np.uint32)
    A.L.oracle_triples_flat(A.h, B.h, tau, trip.ctypes.data_as(_U32), cnt)
    return trip[:cnt]


def flat_bound(A: Tree, B: Tree, tau: float) -> float:
    return A.L.oracle_flat_bound(A.h, B.h, tau)


def matmul_naive(A: np.ndarray, B: np.ndarray, threads: int = 1, L=None) -> np.ndarray:
    L = L or lib()
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    C = np.empty_like(A)
    L.oracle_matmul_naive(_dptr(A), _dptr(B), A.shape[0], _dptr(C), threads)
    return C


def sort_triples(t: np.ndarray) -> np.ndarray:
    """Triples ordered by (i, j, k)."""
    if t.size == 0:
        return t.reshape(0, 3)
    o = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    return t[o]


def max_threads() -> int:
    return lib().oracle_max_threads()


def mutant_lib(mutant: int) -> ctypes.CDLL:
    """A copy of the oracle built with one planted mistake (for the pin tests)."""
    d = os.path.join(tempfile.gettempdir(), "spamm_oracle_mutants")
    return lib(mutant, d)
