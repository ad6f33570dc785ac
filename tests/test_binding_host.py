"""Operand checks of the Python binding (no GPU): every matrix handed to the library is
an n x n row-major FP64 buffer, host (numpy or torch CPU) or CUDA; anything else is
refused in Python before the library sees the pointer."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
S = pytest.importorskip("paper_1011_3534_gb300.spamm")


def test_host_arrays():
    A = np.zeros((5, 5))
    addr, host = S._matrix(A, 5, "t")
    assert host and addr == A.ctypes.data
    T = torch.zeros((5, 5), dtype=torch.float64)
    addr, host = S._matrix(T, 5, "t")
    assert host and addr == T.data_ptr()


@pytest.mark.parametrize("bad", [
    np.zeros((5, 5), dtype=np.float32),               # another dtype
    np.zeros((5, 6)),                                 # another size
    np.asfortranarray(np.arange(25.0).reshape(5, 5)),  # column-major
    np.zeros((10, 10))[::2, ::2],                     # strided view
])
def test_bad_numpy(bad):
    with pytest.raises(ValueError):
        S._matrix(bad, 5, "t")


@pytest.mark.parametrize("bad", [
    torch.zeros((5, 5), dtype=torch.float32),
    torch.zeros((4, 4), dtype=torch.float64),
    torch.arange(25.0, dtype=torch.float64).reshape(5, 5).t(),
])
def test_bad_tensors(bad):
    with pytest.raises(ValueError):
        S._matrix(bad, 5, "t")


def test_read_only_output():
    A = np.zeros((3, 3))
    A.flags.writeable = False
    S._matrix(A, 3, "t")
    with pytest.raises(ValueError):
        S._matrix(A, 3, "t", writable=True)


def test_other_types():
    with pytest.raises(TypeError):
        S._matrix([[0.0]], 1, "t")


def _fake_cuda(index):
    return types.SimpleNamespace(data_ptr=lambda: 4096, is_cuda=True, dtype="torch.float64", shape=(2, 2),
                                 is_contiguous=lambda: True, numel=lambda: 4,
                                 device=types.SimpleNamespace(index=index))


def test_device_must_match_the_context():
    assert S._matrix(_fake_cuda(0), 2, "t", device=0) == (4096, False)
    with pytest.raises(ValueError):
        S._matrix(_fake_cuda(1), 2, "t", device=0)


def test_refused_before_the_library_call():
    ctx = S.Ctx(0)   # a null context: any call reaching the library would fail differently
    with pytest.raises(ValueError):
        S.spamm_tree_build(ctx, np.zeros((3, 3), dtype=np.float32), 3, 16, 0)
    with pytest.raises(ValueError):
        S.spamm_tune_leaf(ctx, np.zeros((2, 3)), 3, 1e-6, S.SPAMM_FP64)


def _fake_dev(dtype, numel, contiguous=True):
    return types.SimpleNamespace(data_ptr=lambda: 8192, is_cuda=True, dtype=dtype, shape=(numel,),
                                 is_contiguous=lambda: contiguous, numel=lambda: numel)


def test_device_buffers():
    assert S._device_buf(_fake_dev("torch.float64", 16), ("torch.float64",), 16, "t") == 8192
    with pytest.raises(ValueError):
        S._device_buf(_fake_dev("torch.float64", 15), ("torch.float64",), 16, "t")
    with pytest.raises(ValueError):
        S._device_buf(_fake_dev("torch.float32", 16), ("torch.float64",), 16, "t")
    with pytest.raises(ValueError):
        S._device_buf(_fake_dev("torch.float64", 16, contiguous=False), ("torch.float64",), 16, "t")
    with pytest.raises(TypeError):
        S._device_buf(np.zeros(16), ("torch.float64",), 16, "t")
    with pytest.raises(TypeError):
        S._device_buf(torch.zeros(16, dtype=torch.float64), ("torch.float64",), 16, "t")


def test_noalloc_cull_buffers_checked_before_the_call():
    n2 = _fake_dev("torch.float64", 64 * 64)
    cnt = _fake_dev("torch.int64", 1)
    with pytest.raises(ValueError):   # norms of 32 x 32 blocks for NB = 64
        S.spamm_cull_noalloc(_fake_dev("torch.float64", 32 * 32), n2, 64, 1e-6, None, 0, cnt)
    with pytest.raises(ValueError):   # room for 9 triples, cap 10
        S.spamm_cull_noalloc(n2, n2, 64, 1e-6, _fake_dev("torch.int32", 27), 10, cnt)
    with pytest.raises(ValueError):   # a 32-bit count
        S.spamm_cull_noalloc(n2, n2, 64, 1e-6, None, 0, _fake_dev("torch.int32", 1))
    with pytest.raises(ValueError):   # cap without a buffer
        S.spamm_cull_noalloc(n2, n2, 64, 1e-6, None, 4, cnt)


def test_mlp_samples_shape():
    m = object.__new__(S.Mlp)   # the shape checks only, no network on a device
    m.inputs = 3
    X, y = m._samples(np.zeros((5, 3)), np.zeros(5))
    assert X.dtype == np.float32 and X.shape == (5, 3) and y.dtype == np.float32
    with pytest.raises(ValueError):
        m._samples(np.zeros((5, 4)))
    with pytest.raises(ValueError):
        m._samples(np.zeros(3))
    with pytest.raises(ValueError):
        m._samples(np.zeros((5, 3)), np.zeros(4))


def test_csr_lengths():
    ip, ix, d = S._csr([0, 1, 3], [0, 0, 1], [1.0, 2.0, 3.0])
    assert ip.dtype == np.int64 and ix.dtype == np.int64 and d.dtype == np.float64
    with pytest.raises(ValueError):   # indptr promises 3 entries, 2 given
        S._csr([0, 1, 3], [0, 0], [1.0, 2.0])
    with pytest.raises(ValueError):   # values and indices disagree
        S._csr([0, 1, 2], [0, 1], [1.0])
    with pytest.raises(ValueError):
        S._csr([], [], [])


def test_batched_lists_must_match():
    ctx = S.Ctx(0)
    with pytest.raises(ValueError):
        S.spamm_multiply_batched(ctx, [None, None], [None], 1e-6, S.SPAMM_BF16)
    with pytest.raises(ValueError):
        S.spamm_multiply_batched(ctx, [None], [None], 1e-6, S.SPAMM_BF16, C=[None, None])
