"""Thin Python binding of the C ABI in include/spamm.h (argument marshalling only).

Every function here forwards to the entry point of the same name in libspamm.so; all
computation runs in the library's CUDA kernels. Device buffers may be given as torch
CUDA tensors (their data_ptr is passed), host buffers as numpy arrays. The module fails
loudly at import if the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SPAMM_OK, SPAMM_EINVAL, SPAMM_ENOMEM, SPAMM_ECUDA, SPAMM_ERANGE, SPAMM_ETIMEOUT, SPAMM_EUNSUPPORTED = range(7)
SPAMM_FP64, SPAMM_TF32, SPAMM_BF16, SPAMM_FP16, SPAMM_BF16X3, SPAMM_TF32X3 = range(6)
PRECISIONS = {"fp64": SPAMM_FP64, "tf32": SPAMM_TF32, "bf16": SPAMM_BF16, "fp16": SPAMM_FP16,
              "bf16x3": SPAMM_BF16X3, "tf32x3": SPAMM_TF32X3}

SPAMM_HOST_INPUT = 0x0001
SPAMM_SYMMETRIC = 0x0002
SPAMM_KEEP_FP64 = 0x0004
SPAMM_COPY_TF32 = 0x0010
SPAMM_COPY_BF16 = 0x0020
SPAMM_COPY_FP16 = 0x0040
SPAMM_COPY_BF16X3 = 0x0080
SPAMM_NO_RIGHT = 0x0100
SPAMM_GRAPH = 0x0200
SPAMM_COPY_TF32X3 = 0x0400
SPAMM_SYM_PRODUCT = 0x0800
SPAMM_DEPTH_TAU = 0x1000
SPAMM_WARP_TILES = 0x2000
COPY_FLAG = {SPAMM_FP64: SPAMM_KEEP_FP64, SPAMM_TF32: SPAMM_COPY_TF32, SPAMM_BF16: SPAMM_COPY_BF16,
             SPAMM_FP16: SPAMM_COPY_FP16, SPAMM_BF16X3: SPAMM_COPY_BF16X3, SPAMM_TF32X3: SPAMM_COPY_TF32X3}
MLP_FEATURES = 69
MAX_LEVELS = 24

# Every entry point declared in include/spamm.h.
EXPORTS = ("spamm_ctx_create", "spamm_ctx_destroy", "spamm_sync", "spamm_last_error",
           "spamm_kernel_launches", "spamm_tree_build", "spamm_tree_update", "spamm_tree_free", "spamm_tree_info",
           "spamm_tree_build_ms",
           "spamm_tree_norms", "spamm_tree_to_dense", "spamm_tree_to_dense_f32", "spamm_tree_leaf_copy", "spamm_multiply", "spamm_stats",
           "spamm_triples", "spamm_cull_noalloc", "spamm_sp2", "spamm_multiply_batched",
           "spamm_tune_leaf", "spamm_tune_shape", "spamm_mlp_create", "spamm_mlp_free", "spamm_mlp_num_params",
           "spamm_mlp_get_params", "spamm_mlp_set_params", "spamm_mlp_forward", "spamm_mlp_gradient",
           "spamm_mlp_adam_step", "spamm_mlp_adam_apply", "spamm_mlp_train", "spamm_features", "spamm_tau_select",
           "spamm_tree_distance", "spamm_sp2_begin", "spamm_sp2_step", "spamm_sp2_step_learned",
           "spamm_sp2_iterate", "spamm_sp2_end", "spamm_sp2_learned", "spamm_sp2_step_learned_margin",
           "spamm_sp2_learned_margin", "spamm_drop_blocks",
           "spamm_sp2_step_drop", "spamm_sp2_dropping", "spamm_tree_update_batched")


class SpammError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class StatsT(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("leaf", ctypes.c_int32), ("n", ctypes.c_int64),
                ("tested", ctypes.c_int64 * MAX_LEVELS), ("culled", ctypes.c_int64 * MAX_LEVELS),
                ("culled_bound", ctypes.c_double * MAX_LEVELS),
                ("leaf_products", ctypes.c_int64), ("mirrored_products", ctypes.c_int64),
                ("output_blocks", ctypes.c_int64),
                ("leaf_flops", ctypes.c_double), ("dense_equiv_flops", ctypes.c_double),
                ("mma_flops", ctypes.c_double), ("ms_cull", ctypes.c_double),
                ("ms_leaf", ctypes.c_double), ("prec", ctypes.c_int32), ("tau", ctypes.c_double)]


SP2_MAX_STEPS = 128


class Sp2ResultT(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double),
                ("steps", ctypes.c_int32), ("trace", ctypes.c_double * (SP2_MAX_STEPS + 1)),
                ("branch", ctypes.c_int32 * SP2_MAX_STEPS), ("leaf_products", ctypes.c_int64 * SP2_MAX_STEPS),
                ("tau", ctypes.c_double * SP2_MAX_STEPS), ("ms", ctypes.c_double)]


_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


def lib_path() -> str:
    return _build.LIB


def _declare(L: ctypes.CDLL) -> ctypes.CDLL:
    st = ctypes.c_int
    L.spamm_ctx_create.argtypes = [ctypes.c_int, _P, _I32, ctypes.POINTER(_P)]
    L.spamm_ctx_destroy.argtypes = [_P]
    L.spamm_sync.argtypes = [_P]
    L.spamm_last_error.argtypes = [_P]
    L.spamm_last_error.restype = ctypes.c_char_p
    L.spamm_kernel_launches.argtypes = [_P]
    L.spamm_kernel_launches.restype = _I64
    L.spamm_tree_build.argtypes = [_P, _P, _I64, _I32, _I32, ctypes.POINTER(_P)]
    L.spamm_tree_free.argtypes = [_P]
    L.spamm_tree_update.argtypes = [_P, _P, _I32]
    L.spamm_tree_build_ms.argtypes = [_P, ctypes.POINTER(ctypes.c_float)]
    L.spamm_tree_info.argtypes = [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                                  ctypes.POINTER(_I32), ctypes.POINTER(_I32)]
    L.spamm_tree_norms.argtypes = [_P, _I32, _P]
    L.spamm_tree_to_dense.argtypes = [_P, _P, _I32]
    L.spamm_tree_to_dense_f32.argtypes = [_P, _P, _I32]
    L.spamm_tree_leaf_copy.argtypes = [_P, _I32, _P, _I64, _I32]
    L.spamm_multiply.argtypes = [_P, _P, _P, _D, ctypes.c_int, _I32, ctypes.POINTER(_P)]
    L.spamm_stats.argtypes = [_P, ctypes.POINTER(StatsT)]
    L.spamm_triples.argtypes = [_P, _P, _I64, ctypes.POINTER(_I64)]
    L.spamm_cull_noalloc.argtypes = [_P, _P, _I32, _D, _P, _I64, _P, _P]
    L.spamm_multiply_batched.argtypes = [_P, _P, _P, _P, _I32, ctypes.c_int, _I32, _P]
    L.spamm_tune_leaf.argtypes = [_P, _P, _I64, _D, ctypes.c_int, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_D)]
    L.spamm_tune_shape.argtypes = [_P, _P, _I64, _D, ctypes.c_int, _I32, ctypes.POINTER(_I32),
                                   ctypes.POINTER(_I32), ctypes.POINTER(_D)]
    L.spamm_sp2.argtypes = [_P, _I64, _P, _P, _P, _D, _I32, _I32, ctypes.c_int, _P, ctypes.POINTER(Sp2ResultT)]
    L.spamm_sp2_learned.argtypes = [_P, _I64, _P, _P, _P, _D, _I32, _I32, ctypes.c_int, _P, _D, _D, _D,
                                    ctypes.POINTER(Sp2ResultT)]
    L.spamm_sp2_begin.argtypes = [_P, _I64, _P, _P, _P, _D, _I32, ctypes.c_int, ctypes.POINTER(_P)]
    L.spamm_sp2_step.argtypes = [_P, _D]
    L.spamm_sp2_step_drop.argtypes = [_P, _D]
    L.spamm_sp2_dropping.argtypes = [_P, _I64, _P, _P, _P, _D, _I32, _I32, ctypes.c_int, _D,
                                     ctypes.POINTER(Sp2ResultT)]
    L.spamm_drop_blocks.argtypes = [_P, _D, ctypes.POINTER(_I64)]
    L.spamm_tree_update_batched.argtypes = [_P, _I32, _P, _P, _I32]
    L.spamm_sp2_step_learned.argtypes = [_P, _P, _D, _D, _D]
    L.spamm_sp2_step_learned_margin.argtypes = [_P, _P, _D, _D, _D, _D, _D]
    L.spamm_sp2_learned_margin.argtypes = [_P, _I64, _P, _P, _P, _D, _I32, _I32, ctypes.c_int, _P, _D, _D, _D, _D,
                                           _D, ctypes.POINTER(Sp2ResultT)]
    L.spamm_sp2_iterate.argtypes = [_P, ctypes.POINTER(_P)]
    L.spamm_sp2_end.argtypes = [_P, ctypes.POINTER(Sp2ResultT)]
    L.spamm_mlp_create.argtypes = [_P, _I32, _I32, ctypes.c_uint64, ctypes.POINTER(_P)]
    L.spamm_mlp_free.argtypes = [_P]
    L.spamm_mlp_num_params.argtypes = [_P]
    L.spamm_mlp_get_params.argtypes = [_P, _P, _I32]
    L.spamm_mlp_set_params.argtypes = [_P, _P, _I32]
    L.spamm_mlp_forward.argtypes = [_P, _P, _I32, _P]
    L.spamm_mlp_gradient.argtypes = [_P, _P, _P, _I32, _P, _P]
    L.spamm_mlp_adam_step.argtypes = [_P, _P, _P, _I32, ctypes.c_float, _P]
    L.spamm_mlp_adam_apply.argtypes = [_P, _P, ctypes.c_float]
    L.spamm_mlp_train.argtypes = [_P, _P, _P, _I32, _I32, _I32, ctypes.c_float, ctypes.c_uint64, _P]
    L.spamm_features.argtypes = [_P, _P, _D, _P]
    L.spamm_tau_select.argtypes = [_P, _P, _P, _D, _D, _D, ctypes.POINTER(_D)]
    L.spamm_tree_distance.argtypes = [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]
    for name in EXPORTS:
        if name not in ("spamm_last_error", "spamm_kernel_launches", "spamm_mlp_num_params"):
            getattr(L, name).restype = st
    L.spamm_mlp_num_params.restype = _I32
    return L


def _load() -> ctypes.CDLL:
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libspamm.so is not built ({path}); run __graft_entry__.build()")
    return _declare(ctypes.CDLL(path))


LIB = _load()


def _ptr(x) -> int:
    """Raw address of a torch tensor (device or host) or a numpy array."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


def _matrix(x, n: int, what: str, device: int | None = None, writable: bool = False,
            dtype: str = "float64") -> tuple[int, bool]:
    """Address of an n x n row-major matrix of `dtype` (FP64 unless stated) and whether
    it is in host memory: a numpy array or torch CPU tensor (host, pageable or
    page-locked) or a torch CUDA tensor on the context's device. Any other type, dtype,
    size or layout raises here, before the library sees the pointer."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.dtype(dtype) or not x.flags.c_contiguous or (n >= 1 and x.size != n * n):
            raise ValueError(f"{what}: need a C-contiguous {dtype} array of {n} x {n} elements, "
                             f"got {x.dtype} {x.shape}")
        if writable and not x.flags.writeable:
            raise ValueError(f"{what}: the output array is read-only")
        return x.ctypes.data, True
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if str(x.dtype) != f"torch.{dtype}" or not x.is_contiguous() or (n >= 1 and x.numel() != n * n):
            raise ValueError(f"{what}: need a contiguous torch.{dtype} tensor of {n} x {n} elements, "
                             f"got {x.dtype} {tuple(x.shape)}")
        if not x.is_cuda:
            return x.data_ptr(), True
        if device is not None and x.device.index is not None and x.device.index != device:
            raise ValueError(f"{what}: tensor on cuda:{x.device.index}, context on cuda:{device}")
        return x.data_ptr(), False
    raise TypeError(f"{what}: expected a numpy array or a torch CUDA tensor, got {type(x).__name__}")


def _device_buf(x, dtypes: tuple, min_numel: int, what: str) -> int:
    """Address of a contiguous torch CUDA tensor of one of `dtypes` holding at least
    `min_numel` elements; anything else raises before the library sees the pointer."""
    if not (hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)):
        raise TypeError(f"{what}: expected a torch CUDA tensor, got {type(x).__name__}")
    if str(x.dtype) not in dtypes or not x.is_contiguous() or x.numel() < min_numel:
        raise ValueError(f"{what}: need a contiguous {' or '.join(dtypes)} tensor of at least {min_numel} "
                         f"elements, got {x.dtype} {tuple(x.shape)}")
    return x.data_ptr()


class Ctx:
    def __init__(self, handle: int, device: int | None = None):
        self.h = handle
        self.device = device

    def check(self, status: int, what: str = ""):
        if status != SPAMM_OK:
            raise SpammError(status, f"{what}: {LIB.spamm_last_error(self.h).decode()}")


class Tree:
    def __init__(self, ctx: Ctx, handle: int):
        self.ctx = ctx
        self.h = handle
        n, leaf, nbp, kmax = _I64(), _I32(), _I32(), _I32()
        LIB.spamm_tree_info(handle, ctypes.byref(n), ctypes.byref(leaf), ctypes.byref(nbp), ctypes.byref(kmax))
        self.n, self.leaf, self.NB, self.kmax = n.value, leaf.value, nbp.value, kmax.value


def spamm_ctx_create(device: int = 0, stream=None, timing: bool = False) -> Ctx:
    h = _P()
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = LIB.spamm_ctx_create(device, s, 1 if timing else 0, ctypes.byref(h))
    if rc != SPAMM_OK:
        raise SpammError(rc, "spamm_ctx_create failed (is a CUDA device present?)")
    return Ctx(h.value, device)


def spamm_ctx_destroy(ctx: Ctx):
    if ctx.h:
        LIB.spamm_ctx_destroy(ctx.h)
        ctx.h = None


def spamm_sync(ctx: Ctx):
    ctx.check(LIB.spamm_sync(ctx.h), "spamm_sync")


def spamm_last_error(ctx: Ctx) -> str:
    return LIB.spamm_last_error(ctx.h).decode()


def spamm_kernel_launches(ctx: Ctx) -> int:
    return LIB.spamm_kernel_launches(ctx.h)


def spamm_tree_build(ctx: Ctx, A, n: int, leaf: int, flags: int) -> Tree:
    """A: torch CUDA tensor (device) or numpy array (host; SPAMM_HOST_INPUT is added)."""
    addr, host = _matrix(A, n, "spamm_tree_build", ctx.device)
    if host:
        flags |= SPAMM_HOST_INPUT
    h = _P()
    ctx.check(LIB.spamm_tree_build(ctx.h, addr, n, leaf, flags, ctypes.byref(h)), "spamm_tree_build")
    return Tree(ctx, h.value)


def spamm_tree_update(t: Tree, A) -> Tree:
    """Rebuild t in place from A (torch CUDA tensor, or numpy host array)."""
    addr, host = _matrix(A, t.n, "spamm_tree_update", t.ctx.device)
    t.ctx.check(LIB.spamm_tree_update(t.h, addr, SPAMM_HOST_INPUT if host else 0), "spamm_tree_update")
    return t


def spamm_tree_update_batched(ctx: Ctx, trees: list, inputs: list):
    """Rebuild trees[p] from the torch CUDA tensors inputs[p], the rebuilds spread over
    the context's side streams."""
    count = len(trees)
    if len(inputs) != count:
        raise ValueError("spamm_tree_update_batched: one input per tree")
    addrs = []
    for t, a in zip(trees, inputs):
        addr, host = _matrix(a, t.n, "spamm_tree_update_batched", ctx.device)
        if host:
            raise ValueError("spamm_tree_update_batched: inputs must be torch CUDA tensors")
        addrs.append(addr)
    pt = (ctypes.c_void_p * count)(*[t.h for t in trees])
    pa = (ctypes.c_void_p * count)(*addrs)
    ctx.check(LIB.spamm_tree_update_batched(ctx.h, count, ctypes.addressof(pt), ctypes.addressof(pa), 0),
              "spamm_tree_update_batched")


def spamm_tree_build_ms(t: Tree) -> float:
    """Device time (ms) of the leaf-block kernel in t's last build or update (timing contexts)."""
    ms = ctypes.c_float()
    t.ctx.check(LIB.spamm_tree_build_ms(t.h, ctypes.byref(ms)), "spamm_tree_build_ms")
    return ms.value


def spamm_tree_free(t: Tree):
    if t.h:
        LIB.spamm_tree_free(t.h)
        t.h = None


def spamm_tree_norms(t: Tree, level: int) -> np.ndarray:
    d = 1 << level
    out = np.empty((d, d), dtype=np.float64)
    t.ctx.check(LIB.spamm_tree_norms(t.h, level, out.ctypes.data), "spamm_tree_norms")
    return out


def spamm_tree_to_dense(t: Tree, out=None, asynchronous: bool = False):
    """Dense n x n FP64 copy: into `out` (numpy host or torch device), or a new numpy array.
    asynchronous (host output only): return once queued; `out` is complete after spamm_sync."""
    if out is None:
        out = np.empty((t.n, t.n), dtype=np.float64)
    addr, host = _matrix(out, t.n, "spamm_tree_to_dense", t.ctx.device, writable=True)
    mode = (2 if asynchronous else 1) if host else 0
    t.ctx.check(LIB.spamm_tree_to_dense(t.h, addr, mode), "spamm_tree_to_dense")
    return out


def spamm_tree_to_dense_f32(t: Tree, out=None, asynchronous: bool = False):
    """Dense n x n FP32 copy (FP32 tiles as they are, FP64 tiles rounded to nearest):
    into `out` (numpy float32 host or torch float32 device), or a new numpy array.
    asynchronous (host output only): return once queued; `out` is complete after spamm_sync."""
    if out is None:
        out = np.empty((t.n, t.n), dtype=np.float32)
    addr, host = _matrix(out, t.n, "spamm_tree_to_dense_f32", t.ctx.device, writable=True, dtype="float32")
    mode = (2 if asynchronous else 1) if host else 0
    t.ctx.check(LIB.spamm_tree_to_dense_f32(t.h, addr, mode), "spamm_tree_to_dense_f32")
    return out


SPAMM_LEAF = {"f64": 0, "f32": 1, "tf32": 2, "tf32_t": 3, "bf16": 4, "bf16_t": 5, "fp16": 6, "fp16_t": 7,
              "bf16lo": 8, "bf16lo_t": 9, "tf32lo": 10, "tf32lo_t": 11}
_LEAF_DTYPE = {"f64": np.float64, "f32": np.float32, "tf32": np.float32, "tf32lo": np.float32,
               "bf16": np.uint16, "fp16": np.uint16, "bf16lo": np.uint16}


def spamm_tree_leaf_copy(t: Tree, which: str) -> np.ndarray:
    """One stored leaf copy of a tree as a host array of shape (nb, nb, leaf, leaf) (leaf
    (r, c) at [r, c]; BF16 and FP16 copies as their uint16 bit patterns)."""
    nb = -(-t.n // t.leaf)
    out = np.empty((nb, nb, t.leaf, t.leaf), dtype=_LEAF_DTYPE[which.replace("_t", "")])
    t.ctx.check(LIB.spamm_tree_leaf_copy(t.h, SPAMM_LEAF[which], out.ctypes.data, out.nbytes, 1),
                "spamm_tree_leaf_copy")
    return out


def spamm_multiply(ctx: Ctx, A: Tree, B: Tree, tau: float, prec: int = SPAMM_FP64, flags: int = 0,
                   C: Tree | None = None) -> Tree:
    h = _P(C.h if C is not None else None)
    ctx.check(LIB.spamm_multiply(ctx.h, A.h, B.h, float(tau), int(prec), flags, ctypes.byref(h)),
              "spamm_multiply")
    return C if C is not None else Tree(ctx, h.value)


def spamm_stats(C: Tree) -> dict:
    s = StatsT()
    C.ctx.check(LIB.spamm_stats(C.h, ctypes.byref(s)), "spamm_stats")
    L = s.levels
    return dict(levels=L, leaf=s.leaf, n=s.n, tested=list(s.tested[:L]), culled=list(s.culled[:L]),
                culled_bound=list(s.culled_bound[:L]), leaf_products=s.leaf_products,
                mirrored_products=s.mirrored_products,
                output_blocks=s.output_blocks, leaf_flops=s.leaf_flops,
                dense_equiv_flops=s.dense_equiv_flops, mma_flops=s.mma_flops, ms_cull=s.ms_cull,
                ms_leaf=s.ms_leaf, prec=s.prec, tau=s.tau)


def spamm_triples(C: Tree) -> np.ndarray:
    """Surviving leaf triples (i, j, k), sorted, as a (count, 3) uint32 array."""
    cnt = _I64()
    C.ctx.check(LIB.spamm_triples(C.h, None, 0, ctypes.byref(cnt)), "spamm_triples")
    out = np.empty((max(cnt.value, 1), 3), dtype=np.uint32)
    C.ctx.check(LIB.spamm_triples(C.h, out.ctypes.data, out.shape[0], ctypes.byref(cnt)), "spamm_triples")
    return out[:cnt.value]


def spamm_cull_noalloc(normA2, normB2, nb_padded: int, tau: float, triples, cap: int, count, stream=None):
    """Forward to the allocation-free cull: all buffers are device tensors the caller owns
    (the norms FP64, NB x NB; the triples int32 or uint32, 3 per slot; the count int64).
    A block count the library refuses (not a power of two, above 128) goes through for
    the library to report."""
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    nn = nb_padded * nb_padded if 1 <= nb_padded <= 128 and nb_padded & (nb_padded - 1) == 0 else 0
    f64, u32 = ("torch.float64",), ("torch.int32", "torch.uint32")
    pa = _device_buf(normA2, f64, nn, "spamm_cull_noalloc normA2")
    pb = _device_buf(normB2, f64, nn, "spamm_cull_noalloc normB2")
    pt = _device_buf(triples, u32, 3 * max(cap, 0), "spamm_cull_noalloc triples") if triples is not None else None
    if triples is None and cap > 0:
        raise ValueError("spamm_cull_noalloc: cap > 0 without a triples buffer")
    pc = _device_buf(count, ("torch.int64",), 1, "spamm_cull_noalloc count")
    rc = LIB.spamm_cull_noalloc(pa, pb, nb_padded, float(tau), pt, cap, pc, s)
    if rc != SPAMM_OK:
        raise SpammError(rc, "spamm_cull_noalloc failed")


def spamm_sp2(ctx: Ctx, indptr, indices, data, n_occ: float, steps: int, leaf: int, prec: int, tau) -> dict:
    """SP2 purification of the symmetric CSR matrix H (host numpy arrays)."""
    indptr, indices, data = _csr(indptr, indices, data)
    tau = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, dtype=np.float64), (steps,)))
    n = indptr.size - 1
    r = Sp2ResultT()
    ctx.check(LIB.spamm_sp2(ctx.h, n, indptr.ctypes.data, indices.ctypes.data, data.ctypes.data, float(n_occ),
                            steps, leaf, int(prec), tau.ctypes.data if steps else None, ctypes.byref(r)),
              "spamm_sp2")
    return _sp2_dict(r)


def _sp2_dict(r: Sp2ResultT) -> dict:
    k = r.steps
    return dict(energy=r.energy, eps_min=r.eps_min, eps_max=r.eps_max, steps=k,
                traces=list(r.trace[:k + 1]), branches=list(r.branch[:k]),
                leaf_products=list(r.leaf_products[:k]), taus=list(r.tau[:k]), ms=r.ms)


def _csr(indptr, indices, data):
    """Host CSR arrays as int64 / int64 / FP64, with as many column indices and values as
    indptr[-1] says (the library reads that many; it checks the index ranges itself)."""
    ip = np.ascontiguousarray(indptr, dtype=np.int64).reshape(-1)
    ix = np.ascontiguousarray(indices, dtype=np.int64).reshape(-1)
    dv = np.ascontiguousarray(data, dtype=np.float64).reshape(-1)
    if ip.size < 1 or ip[-1] != ix.size or ix.size != dv.size:
        raise ValueError(f"CSR: indptr[-1] must equal the number of indices and values, got "
                         f"{ip[-1] if ip.size else None}, {ix.size}, {dv.size}")
    return ip, ix, dv


def spamm_sp2_learned_margin(ctx: Ctx, indptr, indices, data, n_occ: float, steps: int, leaf: int, prec: int,
                             mlp: "Mlp", err_budget: float, tau_min: float, tau_max: float, mu_ref: float,
                             gain_max: float) -> dict:
    """SP2 with every step's tolerance chosen on the device by the controller, each step's
    budget loosened by the margin of its branch decision (clamp(margin / mu_ref, 1, gain_max))."""
    ip, ix, dv = _csr(indptr, indices, data)
    r = Sp2ResultT()
    ctx.check(LIB.spamm_sp2_learned_margin(ctx.h, ip.size - 1, ip.ctypes.data, ix.ctypes.data, dv.ctypes.data,
                                           float(n_occ), steps, leaf, int(prec), mlp.h, float(err_budget),
                                           float(tau_min), float(tau_max), float(mu_ref), float(gain_max),
                                           ctypes.byref(r)), "spamm_sp2_learned_margin")
    return _sp2_dict(r)


def spamm_sp2_learned(ctx: Ctx, indptr, indices, data, n_occ: float, steps: int, leaf: int, prec: int,
                      mlp: "Mlp", err_budget: float, tau_min: float, tau_max: float) -> dict:
    """SP2 with every step's tolerance chosen on the device by the controller."""
    ip, ix, dv = _csr(indptr, indices, data)
    r = Sp2ResultT()
    ctx.check(LIB.spamm_sp2_learned(ctx.h, ip.size - 1, ip.ctypes.data, ix.ctypes.data, dv.ctypes.data,
                                    float(n_occ), steps, leaf, int(prec), mlp.h, float(err_budget),
                                    float(tau_min), float(tau_max), ctypes.byref(r)), "spamm_sp2_learned")
    return _sp2_dict(r)


def spamm_sp2_dropping(ctx: Ctx, indptr, indices, data, n_occ: float, steps: int, leaf: int, prec: int,
                       tau_drop: float) -> dict:
    """SP2 by the paper's scheme (I): exact products, each filtered by spamm_drop_blocks."""
    ip, ix, dv = _csr(indptr, indices, data)
    r = Sp2ResultT()
    ctx.check(LIB.spamm_sp2_dropping(ctx.h, ip.size - 1, ip.ctypes.data, ix.ctypes.data, dv.ctypes.data,
                                     float(n_occ), steps, leaf, int(prec), float(tau_drop), ctypes.byref(r)),
              "spamm_sp2_dropping")
    return _sp2_dict(r)


def spamm_drop_blocks(t: Tree, tau: float, count: bool = True):
    """Drop the leaf blocks of t with Frobenius norm below tau; the number kept (or None)."""
    kept = _I64()
    t.ctx.check(LIB.spamm_drop_blocks(t.h, float(tau), ctypes.byref(kept) if count else None), "spamm_drop_blocks")
    return kept.value if count else None


class Sp2Run:
    """spamm_sp2_begin .. spamm_sp2_end: the SP2 loop one step at a time."""

    def __init__(self, ctx: Ctx, indptr, indices, data, n_occ: float, leaf: int, prec: int):
        self.ctx = ctx
        ip, ix, dv = _csr(indptr, indices, data)
        h = _P()
        ctx.check(LIB.spamm_sp2_begin(ctx.h, ip.size - 1, ip.ctypes.data, ix.ctypes.data, dv.ctypes.data,
                                      float(n_occ), leaf, int(prec), ctypes.byref(h)), "spamm_sp2_begin")
        self.h = h.value

    def step(self, tau: float):
        self.ctx.check(LIB.spamm_sp2_step(self.h, float(tau)), "spamm_sp2_step")

    def step_drop(self, tau_drop: float):
        self.ctx.check(LIB.spamm_sp2_step_drop(self.h, float(tau_drop)), "spamm_sp2_step_drop")

    def step_learned(self, mlp: "Mlp", err_budget: float, tau_min: float, tau_max: float):
        self.ctx.check(LIB.spamm_sp2_step_learned(self.h, mlp.h, float(err_budget), float(tau_min), float(tau_max)),
                       "spamm_sp2_step_learned")

    def iterate(self) -> Tree:
        """The current iterate (borrowed: valid until the next step or end; never freed here)."""
        x = _P()
        self.ctx.check(LIB.spamm_sp2_iterate(self.h, ctypes.byref(x)), "spamm_sp2_iterate")
        return Tree(self.ctx, x.value)

    def end(self) -> dict:
        r = Sp2ResultT()
        h, self.h = self.h, None
        self.ctx.check(LIB.spamm_sp2_end(h, ctypes.byref(r)), "spamm_sp2_end")
        return _sp2_dict(r)


# ---- tolerance controller ----
class Mlp:
    def __init__(self, ctx: Ctx, inputs: int, hidden: int, seed: int = 0):
        self.ctx = ctx
        h = _P()
        ctx.check(LIB.spamm_mlp_create(ctx.h, inputs, hidden, seed, ctypes.byref(h)), "spamm_mlp_create")
        self.h = h.value
        self.inputs, self.hidden = inputs, hidden
        self.P = LIB.spamm_mlp_num_params(self.h)

    def free(self):
        if self.h:
            LIB.spamm_mlp_free(self.h)
            self.h = None

    def get_params(self) -> np.ndarray:
        out = np.empty(self.P, dtype=np.float32)
        self.ctx.check(LIB.spamm_mlp_get_params(self.h, out.ctypes.data, self.P), "spamm_mlp_get_params")
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        self.ctx.check(LIB.spamm_mlp_set_params(self.h, th.ctypes.data, th.size), "spamm_mlp_set_params")

    def _samples(self, X, y=None):
        """X as (samples, inputs) FP32 rows and y as one FP32 label per sample."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != self.inputs:
            raise ValueError(f"Mlp: X must be (samples, {self.inputs}), got {X.shape}")
        if y is not None:
            y = np.ascontiguousarray(y, dtype=np.float32)
            if y.shape != (X.shape[0],):
                raise ValueError(f"Mlp: y must hold one label per sample ({X.shape[0]}), got {y.shape}")
        return X, y

    def forward(self, X) -> np.ndarray:
        X, _ = self._samples(X)
        y = np.empty(X.shape[0], dtype=np.float32)
        self.ctx.check(LIB.spamm_mlp_forward(self.h, X.ctypes.data, X.shape[0], y.ctypes.data), "spamm_mlp_forward")
        return y

    def gradient(self, X, y) -> tuple[float, np.ndarray]:
        X, y = self._samples(X, y)
        g = np.empty(self.P, dtype=np.float32)
        L = np.zeros(1, dtype=np.float32)
        self.ctx.check(LIB.spamm_mlp_gradient(self.h, X.ctypes.data, y.ctypes.data, X.shape[0], g.ctypes.data,
                                              L.ctypes.data), "spamm_mlp_gradient")
        return float(L[0]), g

    def adam_step(self, X, y, lr: float) -> float:
        X, y = self._samples(X, y)
        L = np.zeros(1, dtype=np.float32)
        self.ctx.check(LIB.spamm_mlp_adam_step(self.h, X.ctypes.data, y.ctypes.data, X.shape[0], float(lr),
                                               L.ctypes.data), "spamm_mlp_adam_step")
        return float(L[0])

    def adam_apply(self, grad, lr: float):
        g = np.ascontiguousarray(grad, dtype=np.float32)
        if g.size != self.P:
            raise ValueError(f"Mlp: gradient of {g.size} entries, the network has {self.P} parameters")
        self.ctx.check(LIB.spamm_mlp_adam_apply(self.h, g.ctypes.data, float(lr)), "spamm_mlp_adam_apply")

    def train(self, X, y, epochs: int, batch: int, lr: float, seed: int = 0) -> float:
        X, y = self._samples(X, y)
        L = np.zeros(1, dtype=np.float32)
        self.ctx.check(LIB.spamm_mlp_train(self.h, X.ctypes.data, y.ctypes.data, X.shape[0], epochs, batch,
                                           float(lr), seed, L.ctypes.data), "spamm_mlp_train")
        return float(L[0])


def spamm_features(A: Tree, B: Tree, tau: float) -> np.ndarray:
    out = np.empty(MLP_FEATURES, dtype=np.float32)
    A.ctx.check(LIB.spamm_features(A.h, B.h, float(tau), out.ctypes.data), "spamm_features")
    return out


def spamm_tau_select(mlp: Mlp, A: Tree, B: Tree, err_budget: float, tau_min: float, tau_max: float) -> float:
    t = _D()
    A.ctx.check(LIB.spamm_tau_select(mlp.h, A.h, B.h, float(err_budget), float(tau_min), float(tau_max),
                                     ctypes.byref(t)), "spamm_tau_select")
    return t.value


def spamm_tree_distance(X: Tree, Y: Tree) -> tuple[float, float]:
    """(||X - Y||_F, ||Y||_F)."""
    d, r = _D(), _D()
    X.ctx.check(LIB.spamm_tree_distance(X.h, Y.h, ctypes.byref(d), ctypes.byref(r)), "spamm_tree_distance")
    return d.value, r.value


def spamm_multiply_batched(ctx: Ctx, A: list, B: list, tau, prec: int, flags: int = 0, C: list | None = None) -> list:
    """C[p] ~ A[p] B[p] with tolerance tau[p]; returns the list of product trees."""
    count = len(A)
    if len(B) != count or (C is not None and len(C) != count):
        raise ValueError("spamm_multiply_batched: A, B (and C) must have one entry per product")
    pa = (ctypes.c_void_p * count)(*[t.h for t in A])
    pb = (ctypes.c_void_p * count)(*[t.h for t in B])
    pc = (ctypes.c_void_p * count)(*[(c.h if c is not None else None) for c in (C or [None] * count)])
    tv = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, dtype=np.float64), (count,)))
    ctx.check(LIB.spamm_multiply_batched(ctx.h, ctypes.addressof(pa), ctypes.addressof(pb), tv.ctypes.data, count,
                                         int(prec), flags, ctypes.addressof(pc)), "spamm_multiply_batched")
    if C is not None:
        return C
    return [Tree(ctx, pc[p]) for p in range(count)]


def spamm_tune_leaf(ctx: Ctx, A, n: int, tau: float, prec: int, flags: int = 0) -> tuple[int, float]:
    """Fastest leaf size for the product A A (A: torch CUDA tensor or numpy host array)."""
    addr, host = _matrix(A, n, "spamm_tune_leaf", ctx.device)
    if host:
        flags |= SPAMM_HOST_INPUT
    leaf, ms = _I32(), _D()
    ctx.check(LIB.spamm_tune_leaf(ctx.h, addr, n, float(tau), int(prec), flags, ctypes.byref(leaf),
                                  ctypes.byref(ms)), "spamm_tune_leaf")
    return leaf.value, ms.value


def spamm_tune_shape(ctx: Ctx, A, n: int, tau: float, prec: int, flags: int = 0) -> tuple[int, int, float]:
    """Fastest (leaf size, tile-shape multiply flags, ms) for the product A A."""
    addr, host = _matrix(A, n, "spamm_tune_shape", ctx.device)
    if host:
        flags |= SPAMM_HOST_INPUT
    leaf, tf, ms = _I32(), _I32(), _D()
    ctx.check(LIB.spamm_tune_shape(ctx.h, addr, n, float(tau), int(prec), flags, ctypes.byref(leaf), ctypes.byref(tf),
                                   ctypes.byref(ms)), "spamm_tune_shape")
    return leaf.value, tf.value, ms.value
