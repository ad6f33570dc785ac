"""Shared comparison helpers of the GPU parity tests (test-side only)."""
import numpy as np

import oracle

BAND = 1e-12   # near-tau band: triples whose product is within BAND * tau of tau


def keys(trip: np.ndarray, NB: int) -> np.ndarray:
    t = trip.astype(np.int64)
    return (t[:, 0] * NB + t[:, 1]) * NB + t[:, 2]


def products(trip: np.ndarray, nA2: np.ndarray, nB2: np.ndarray) -> np.ndarray:
    i, j, k = trip[:, 0], trip[:, 1], trip[:, 2]
    return np.sqrt(nA2[i, k]) * np.sqrt(nB2[k, j])


def compare_triples(gpu: np.ndarray, ora: np.ndarray, NB: int, nA2, nB2, tau):
    """Bit-exact equality of the sorted triple lists outside the near-tau band.
    Returns (gpu_only, oracle_only) triples, all of which lie inside the band."""
    kg, ko = keys(gpu, NB), keys(ora, NB)
    assert np.all(np.diff(kg) > 0), "GPU triples not sorted/unique"
    only_g = gpu[~np.isin(kg, ko)]
    only_o = ora[~np.isin(ko, kg)]
    for t in (only_g, only_o):
        if len(t):
            p = products(t, nA2, nB2)
            outside = np.abs(p - tau) > BAND * tau
            assert not np.any(outside), f"triples differ outside the band: {t[outside][:5]} p={p[outside][:5]}"
    if len(only_g) or len(only_o):
        print(f"near-tau triples logged: gpu-only {only_g.tolist()} oracle-only {only_o.tolist()}")
    return only_g, only_o


def padded(A: np.ndarray, NB: int, b: int) -> np.ndarray:
    P = np.zeros((NB * b, NB * b))
    P[:A.shape[0], :A.shape[0]] = A
    return P


def adjust_for_band(Cref, A, B, b, NB, only_g, only_o):
    """Oracle C plus the contributions of band triples the GPU kept (minus those it
    dropped), computed from the inputs on the host."""
    if not len(only_g) and not len(only_o):
        return Cref
    n = A.shape[0]
    PA, PB = padded(A, NB, b), padded(B, NB, b)
    C = padded(Cref, NB, b)
    for sgn, tt in ((1.0, only_g), (-1.0, only_o)):
        for i, j, k in tt:
            C[i*b:(i+1)*b, j*b:(j+1)*b] += sgn * (PA[i*b:(i+1)*b, k*b:(k+1)*b] @ PB[k*b:(k+1)*b, j*b:(j+1)*b])
    return C[:n, :n]


def rel_fro(X, R) -> float:
    d = np.linalg.norm(X - R)
    r = np.linalg.norm(R)
    return d / r if r > 0 else d


# products one tcgen05 MMA instruction sums: K = 32 bytes of each operand
MMA_K = {"bf16": 16, "fp16": 16, "bf16x3": 16, "tf32": 8, "tf32x3": 8}


def tc_units(products, prec: str):
    """Units of 2^-23 of the magnitude sum |A||B| that bound the FP32 accumulation
    error of `products` exact products on the tensor cores: one per product for the
    sequential FP32 sums, one more per MMA instruction (its Kq products are aligned to
    the largest magnitude taking part before the truncating add), and one instruction's
    Kq as margin for the first alignment and (split forms) the epilogue's sums of the
    passes in FP32."""
    kq = MMA_K[prec]
    return products + np.ceil(products / kq) + kq


FP32_MIN_NORMAL = 2.0 ** -126


def tc_bound(products, prec: str, cabs):
    """Elementwise bound of |C_gpu - C_ref| for tensor-core products: tc_units(...) units
    of 2^-23 of the magnitude sum, plus one FP32 minimum normal per product for results
    below FP32's normal range (subnormal sums flushed to zero by the accumulator)."""
    return tc_units(products, prec) * 2.0 ** -23 * cabs + products * FP32_MIN_NORMAL + 1e-300
