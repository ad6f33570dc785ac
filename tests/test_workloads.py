"""Pins of the input generators (CPU): the SplitMix64 stream against its published
outputs, exact symmetry, and the site orderings of the lattice workloads."""
import numpy as np
import pytest

from oracle import sp2 as O
from paper_1011_3534_gb300 import workloads as W


def cube(bits):
    g = np.arange(1 << bits)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


@pytest.mark.parametrize("bits", [1, 2, 3, 4, 5])
def test_hilbert_curve_is_a_continuous_bijection(bits):
    # a Hilbert curve visits every point of the 2^bits cube once, and consecutive points
    # are lattice neighbours (one unit step); it starts at the origin and, in three
    # dimensions, ends one edge away at (2^bits - 1, 0, 0)
    x, y, z = cube(bits)
    h = W.hilbert3(x, y, z, bits)
    assert np.array_equal(np.sort(h), np.arange(8 ** bits))
    o = np.argsort(h)
    P = np.stack([x[o], y[o], z[o]], axis=1)
    assert np.all(np.abs(np.diff(P, axis=0)).sum(axis=1) == 1)
    assert tuple(P[0]) == (0, 0, 0) and tuple(P[-1]) == ((1 << bits) - 1, 0, 0)


@pytest.mark.parametrize("bits", [2, 3])
def test_hilbert_octants_are_contiguous(bits):
    # each aligned 2^k sub-cube is one contiguous run of the curve (the property that
    # makes the ordering align with the quadtree's power-of-two blocks)
    x, y, z = cube(bits)
    h = W.hilbert3(x, y, z, bits)
    for k in range(1, bits):
        key = (x >> k) * 64 + (y >> k) * 8 + (z >> k)
        for v in np.unique(key):
            run = np.sort(h[key == v])
            assert run[-1] - run[0] == run.size - 1


def test_orderings_permute_the_same_hamiltonian():
    # the Hilbert-ordered Hamiltonian is P H P^T of the Morton-ordered one: same
    # spectrum, same SP2 energy
    side = 8
    n = side ** 3
    Hm = W.csr_to_dense(n, *W.tight_binding(side))
    Hh = W.csr_to_dense(n, *W.tight_binding(side, order="hilbert"))
    perm = W.site_permutation(side, "hilbert")
    assert np.array_equal(Hh, Hm[np.ix_(perm, perm)])
    np.testing.assert_allclose(np.linalg.eigvalsh(Hh), np.linalg.eigvalsh(Hm), atol=1e-12)
    lo, hi = -9.0, 9.0
    em = O.sp2_spectral(np.linalg.eigvalsh(Hm), n / 2, 20, lo, hi)["energy"]
    eh = O.sp2_dense(Hh, n / 2, 20, lo, hi)["energy"]
    assert abs(em - eh) <= 1e-9 * abs(em)


def test_physical_decay_hilbert_is_a_site_permutation():
    A = W.physical_decay(side=4, per_site=2)
    Ah = W.physical_decay(side=4, per_site=2, order="hilbert")
    perm = W.site_permutation(4, "hilbert")
    pb = (perm[:, None] * 2 + np.arange(2)).ravel()
    assert np.array_equal(Ah, A[np.ix_(pb, pb)])
    assert np.array_equal(Ah, Ah.T)


def test_splitmix64_known_answers():
    # the first outputs of SplitMix64 from state 0 (Steele, Lea and Flood 2014; the
    # sequence Java's SplittableRandom and the authors' reference code produce)
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    u = W.uniform(0, np.arange(4, dtype=np.uint64))
    assert np.array_equal(u, np.array([(r >> 11) * 2.0 ** -53 for r in ref]))
    assert [W._mix64_int(W._GAMMA * (t + 1)) for t in range(4)] == ref


def test_symmetric_generators_are_exactly_symmetric():
    for A in (W.exp_decay(130, 0.85, 1, 0), W.algebraic_decay(130, 2, 0)):
        assert np.array_equal(A, A.T)
        assert A.dtype == np.float64 and A.flags.c_contiguous
