"""The allocation-free cull entry point against the regular multiply.

spamm_cull_noalloc serves callers that cannot allocate device memory (work inside a
stream capture, foreign allocators, raw-pointer embedders). Here it gets the leaf norms
of the regular trees and must return the same surviving leaf triples as
spamm_multiply / spamm_triples (integers: exactly), on two calls in a row, since every
call reuses the same static scratch array. This file is collected last.
"""
import numpy as np
import pytest

from paper_1011_3534_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1011_3534_gb300 import spamm
    return spamm


def sort_rows(t):
    t = np.asarray(t)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))] if len(t) else t.reshape(0, 3)


@pytest.mark.parametrize("n,leaf,tau", [(8192, 64, 1e-8), (1000, 16, 1e-6), (40, 64, 0.0)])
def test_noalloc_cull_matches_multiply(S, n, leaf, tau):
    stream = torch.cuda.current_stream()
    ctx = S.spamm_ctx_create(0, stream)
    A = W.algebraic_decay(n, 2, 0)
    B = W.exp_decay(n, 0.9, 1, 0)
    tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, S.SPAMM_KEEP_FP64)
    tB = S.spamm_tree_build(ctx, torch.from_numpy(B).cuda(), n, leaf, S.SPAMM_KEEP_FP64)
    tC = S.spamm_multiply(ctx, tA, tB, tau, S.SPAMM_FP64)
    ref = S.spamm_triples(tC)
    nA2 = torch.from_numpy(S.spamm_tree_norms(tA, tA.kmax)).cuda()
    nB2 = torch.from_numpy(S.spamm_tree_norms(tB, tB.kmax)).cuda()
    cap = len(ref) + 16
    for call in range(2):
        out = torch.full((cap, 3), 0xFFFFFFFF, dtype=torch.int64).to(torch.int32).cuda()
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        S.spamm_cull_noalloc(nA2, nB2, tA.NB, tau, out, cap, cnt, stream)
        torch.cuda.synchronize()
        c = int(cnt.item())
        assert c == len(ref), (call, c, len(ref))
        got = out[:c].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        assert np.array_equal(sort_rows(got), ref.astype(np.int64)), call
    for t in (tC, tB, tA):
        S.spamm_tree_free(t)
    S.spamm_ctx_destroy(ctx)


def test_noalloc_rejects_oversize(S):
    buf = torch.zeros((256, 256), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(S.SpammError) as e:
        S.spamm_cull_noalloc(buf, buf, 256, 1e-6, None, 0, cnt)
    assert e.value.status == S.SPAMM_ERANGE
    with pytest.raises(S.SpammError) as e:
        S.spamm_cull_noalloc(buf, buf, 96, 1e-6, None, 0, cnt)
    assert e.value.status == S.SPAMM_EINVAL
