// Quadtree build (Eq. 1) with Frobenius norms (Sec. III), norm pyramid, and the
// tile -> dense conversion.
//
// Layout in HBM (one tree):
//   leaf copies : leaf (r, c), r, c < nb = ceil(n / b), stored contiguously at element
//                 offset (r * nb + c) * b * b, row-major inside the leaf (the transposed
//                 copies hold each leaf transposed, at the same offset). Leaves past
//                 nb are never stored; their norm is zero and nz = 0.
//   norm2, norm : every tier l = 0..kmax as a 2^l x 2^l row-major FP64 grid at offset
//                 (4^l - 1) / 3; norm = sqrt(norm2).
//   nz          : NB x NB bytes, 1 where the leaf's tile storage holds the block.
#include <type_traits>

#include "convert.cuh"
#include "f32x2.cuh"
#include "internal.cuh"

namespace {

struct BuildArgs {
  const double *A;
  int64_t n;
  int32_t b, nb, NB, kmax;
  double *leaf_norm2;      // tier kmax of norm2
  uint8_t *nz;
  double *f64;             // optional copies (nullptr = not written)
  float *f32;              // FP32 master (purification iterates)
  float *tf32, *tf32T, *tlo, *tloT;   // TF32 and the low part of the TF32 split
  uint16_t *bf16, *bf16T, *fp16, *fp16T, *lo, *loT;
};

// Leaf-block kernel (K1). A leaf is read as pairs of consecutive elements of a row
// (16-byte loads: a warp reads 512 contiguous bytes) by TPL threads, several leaves per
// CTA for small leaves; each thread streams its pairs in rounds of four. The FP64 pipe
// is kept idle: each round's squared norm is accumulated from an exact FP32 hi/lo split
// of its elements scaled by the round's largest exponent, with error-free (TwoSum)
// accumulation, rounds and threads are merged in double-float after rescaling to a
// common exponent (relative error of the squared norm about 2^-46 typically and at most
// 4e-13: 3 2^-46 from the dropped low bits, 1.25 2^-46 from the cross-term rounding,
// 2^-42 from the FP32 sums of a round's error terms, about 20 double-float merges of
// 2^-47; inside the 1e-12 near-tau band), and the leaf copies are rounded to nearest
// even from the FP64 bit pattern (integer arithmetic, or the FP32-pipe split round).
template <int B>
struct BuildCfg {
  // threads per CTA: a 64 x 64 leaf gets 64 threads, so that each streams eight rounds
  // and the leaf's coordinates stay CTA-uniform
  static constexpr int T = B == 64 ? 64 : 256;
  static constexpr int PAIRS = B * B / 2;          // element pairs per leaf
  static constexpr int TPL = PAIRS / 4 < T ? PAIRS / 4 : T;   // threads per leaf
  static constexpr int LPC = T / TPL;              // leaves per CTA
  static constexpr int RPT = PAIRS / TPL;          // pairs per thread
  static constexpr int ROUNDS = RPT / 4;
};

__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  float err = (h - (s - bb)) + (bh - bb);
  err += l + bl;
  h = s + err;
  l = err - (h - s);
}

// 2^(2d) as a float for d <= 0 (0 when it would not be a normal float)
__device__ __forceinline__ float pow4(int d) {
  const int ex = 2 * d + 127;
  return ex >= 1 ? __uint_as_float((uint32_t)ex << 23) : 0.f;
}

// Double-float accumulator (H + L) * 2^(2 (E - 1023)); E = 0 means empty.
struct NormAcc {
  float H = 0.f, L = 0.f;
  int E = 0;
  __device__ __forceinline__ void merge(float h, float l, int e) {
    if (e == 0) return;
    if (E == 0) { H = h; L = l; E = e; return; }
    if (e > E) {
      const float f = pow4(E - e);
      H *= f;
      L *= f;
      E = e;
    } else {
      const float f = pow4(e - E);
      h *= f;
      l *= f;
    }
    df_add(H, L, h, l);
  }
};


// BF16 pair of two FP64 values with FP32-normal results (exponent fields 897..1150):
// each value truncated to FP32 with the discarded low bits folded into the last bit
// (sticky), then the hardware FP32 -> BF16x2 round to nearest even. The sticky bit
// turns an FP64 value just above a BF16 tie into one above the tie in FP32 too, and is
// far below the BF16 rounding position otherwise, so the result is the correctly
// rounded BF16 of the FP64 value.
__device__ __forceinline__ uint32_t trunc_f32_sticky(uint32_t h, uint32_t l) {
  return (h & 0x80000000u) | ((((h & 0x7FFFFFFFu) - (896u << 20)) << 3) | (l >> 29)) |
         ((l & 0x1FFFFFFFu) != 0u ? 1u : 0u);
}

__device__ __forceinline__ uint32_t bf16x2_fast(uint32_t h0, uint32_t l0, uint32_t h1, uint32_t l1) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;"
      : "=r"(r)
      : "f"(__uint_as_float(trunc_f32_sticky(h1, l1))), "f"(__uint_as_float(trunc_f32_sticky(h0, l0))));
  return r;   // element 0 in the low half
}

// Leaf copies a kernel instance writes: one bit per output. The instance for kAllCopies
// checks every pointer at run time; the specialised instances (the copy sets of the
// common symmetric operands) compile only their own outputs, which keeps the kernel
// small enough for the instruction cache.
constexpr uint32_t kF64 = 1u << 0, kF32 = 1u << 1, kTF32 = 1u << 2, kTF32T = 1u << 3, kTLO = 1u << 4,
                   kTLOT = 1u << 5, kBF16 = 1u << 6, kBF16T = 1u << 7, kLO = 1u << 8, kLOT = 1u << 9,
                   kFP16 = 1u << 10, kFP16T = 1u << 11, kAllCopies = (1u << 12) - 1;

// One round of a split operand (copy set TF32 hi + lo, or BF16 hi + lo, one orientation)
// whose elements all have FP64 exponent fields 949..1149 within 60 binades of each
// other, on the FP32 pipe. Per element x (magnitude |x| handled, sign applied last):
//   a  = |x| truncated to 24 significant bits, m = the next 23 bits (an integer), and
//   j = 1 if any of the last 6 bits is set, so |x| = a + m 2^(p-46) + (last bits) with
//   p the exponent of x; all exact FP32 values.
//   norm: a and 2 m 2^(p-46), scaled by 2^(1023 - Er) (the round's largest exponent),
//   are the same hi and lo2 as the general path's, so the squared norm is the same bits.
//   hi = fmt(x): a with a sticky bit for the discarded bits, rounded to nearest even.
//   lo = fmt(x - hi): d = a - hi (exact), b = (2m + j) 2^(p-47) (the rest of |x|,
//   truncated with a sticky last bit, exact), s = d + b rounded toward zero and its exact
//   error e = b - (s - d); s with a sticky bit for e != 0, rounded to nearest even, is
//   fmt(d + b), and that equals fmt(|x| - hi) whenever fmt's rounding unit at |s| is at
//   least 2^(p-45), i.e. |s| >= 2^(p-34) (TF32) or 2^(p-37) (BF16). A remainder below
//   that (the low bits of x nearly cancel hi's rounding), rare, takes the integer route.
// TF32 round to nearest even of a positive FP32 pattern (the sticky-bit forms below), by
// the hardware conversion: the same bits as tf32_of_sticky for finite normal inputs.
__device__ __forceinline__ uint32_t tf32_rn(uint32_t f) {
  uint32_t r;
  asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(r) : "f"(__uint_as_float(f)));
  return r;
}

// The two norm chains of the round (even and odd elements of each pair) and the
// remainder arithmetic run as the two lanes of f32x2 instructions.
template <int B, bool TF>
__device__ __forceinline__ void k1_round_split(const BuildArgs &p, int64_t tile, const uint32_t (&hw)[8],
                                               const uint32_t (&lw)[8], const int (&rows)[4], const int (&cols)[4],
                                               int Er, NormAcc &acc) {
  const float scR = __uint_as_float((uint32_t)(1150 - Er) << 23);   // 2^(1023 - Er), Er <= 1149
  const uint64_t SCR = f2(scR, scR), NSCR = f2(-scR, -scR), SCR4 = f2(4.f * scR, 4.f * scR);
  const uint64_t TWO = f2(2.f, 2.f), THR = f2(TF ? 8192.f : 1024.f, TF ? 8192.f : 1024.f);
  uint64_t S = f2(0.f, 0.f), s2 = f2(0.f, 0.f);   // chains: even, odd elements
#pragma unroll
  for (int u = 0; u < 4; u++) {
    float a[2], m_f[2], jf[2], sc47[2], hif[2];
    uint32_t a_bits[2], himag[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const uint32_t h = hw[2 * u + k], l = lw[2 * u + k];
      const uint32_t E = (h >> 20) & 0x7FFu;
      a_bits[k] = __funnelshift_l(l, (h & 0x7FFFFFFFu) - (896u << 20), 3);
      a[k] = __uint_as_float(a_bits[k]);
      m_f[k] = u23_to_float((l >> 6) & 0x7FFFFFu);
      jf[k] = (l & 63u) ? 1.f : 0.f;
      sc47[k] = __uint_as_float((E - 943u) << 23);          // 2^(p - 47)
      // hi = fmt(|x|) from a and a sticky bit for the bits below it
      const uint32_t jam = a_bits[k] | ((l & 0x1FFFFFFFu) != 0u ? 1u : 0u);
      himag[k] = TF ? tf32_rn(jam) : (jam + 0x7FFFu + ((jam >> 16) & 1u)) & 0xFFFF0000u;
      hif[k] = __uint_as_float(himag[k]);
    }
    const uint64_t A = f2(a[0], a[1]), M = f2(m_f[0], m_f[1]), SC = f2(sc47[0], sc47[1]);
    // squared norm, both chains: hi_s = a 2^(1023-Er), lo2_s = 2 m 2^(p-46) 2^(1023-Er);
    // npp = -hi_s^2 rounded, cc = (hi_s^2 - pp) + hi_s lo2_s; TwoSum of S + pp
    const uint64_t hs = mul2(A, SCR), nhs = mul2(A, NSCR);
    const uint64_t l2s = mul2(M, mul2(SC, SCR4));
    const uint64_t npp = mul2(hs, nhs);
    const uint64_t cc = fma2(hs, l2s, fma2(hs, hs, npp));
    const uint64_t t = sub2(S, npp);
    const uint64_t tb = sub2(t, S);
    // (S - (t - tb)) + (pp - tb), with pp - tb = -(npp + tb)
    s2 = add2(s2, add2(sub2(sub2(S, sub2(t, tb)), add2(npp, tb)), cc));
    S = t;
    // lo: d = a - hi (exact), b = (2m + j) 2^(p-47), s = d + b toward zero, e = b - (s - d)
    const uint64_t d = sub2(A, f2(hif[0], hif[1]));
    const uint64_t bj = mul2(fma2(M, TWO, f2(jf[0], jf[1])), SC);
    const uint64_t sr2 = add2_rz(d, bj);
    const uint64_t ee2 = sub2(bj, sub2(sr2, d));
    const uint64_t thr2 = mul2(SC, THR);
    float srk[2], eek[2], thrk[2];
    f2_get(sr2, srk[0], srk[1]);
    f2_get(ee2, eek[0], eek[1]);
    f2_get(thr2, thrk[0], thrk[1]);
    uint32_t hb[2], lb[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const uint32_t h = hw[2 * u + k], l = lw[2 * u + k];
      const float sr = srk[k], ee = eek[k];
      uint32_t lo;
      if (fabsf(sr) >= thrk[k] || (sr == 0.f && ee == 0.f)) {
        const uint32_t sb = (__float_as_uint(sr) & 0x7FFFFFFFu) | (ee != 0.f ? 1u : 0u);
        const uint32_t lm = TF ? tf32_rn(sb) : ((sb + 0x7FFFu + ((sb >> 16) & 1u)) & 0xFFFF0000u);
        lo = lm ? lm | ((h ^ __float_as_uint(sr)) & 0x80000000u) : 0u;
      } else {
        lo = slow_split_lo(h, l, TF ? 11 : 8);
      }
      hb[k] = himag[k] | (h & 0x80000000u);
      lb[k] = lo;
    }
    const int64_t o = tile + (int64_t)rows[u] * B + cols[u];
    if (TF) {
      *reinterpret_cast<uint2 *>(p.tf32 + o) = make_uint2(hb[0], hb[1]);
      *reinterpret_cast<uint2 *>(p.tlo + o) = make_uint2(lb[0], lb[1]);
    } else {
      *reinterpret_cast<uint32_t *>(p.bf16 + o) = (hb[0] >> 16) | (hb[1] & 0xFFFF0000u);
      *reinterpret_cast<uint32_t *>(p.lo + o) = (lb[0] >> 16) | (lb[1] & 0xFFFF0000u);
    }
  }
  float S0, S1, e0, e1;
  f2_get(S, S0, S1);
  f2_get(s2, e0, e1);
  df_add(S0, e0, S1, e1);
  acc.merge(S0, e0, Er);
}

// Squared norm (into acc) and leaf copies of one round: the 8 elements of 4 pairs
// (row rows[u], columns cols[u] and cols[u] + 1 of the leaf at element offset `tile`),
// given as the high and low words of their FP64 patterns. Transposed copies go to
// shared-memory leaf images (nullptr: not written).
template <int B, uint32_t M>
__device__ __forceinline__ void k1_round(const BuildArgs &p, int64_t tile, const uint32_t (&hw)[8],
                                         const uint32_t (&lw)[8], const int (&rows)[4], const int (&cols)[4],
                                         NormAcc &acc, float *s_tf32T, float *s_tloT, uint16_t *s_bf16T,
                                         uint16_t *s_fp16T, uint16_t *s_loT) {
  // squared norm of the round, scaled by its largest exponent field Er
  int Er = 0, Emin = 0x7FF;
#pragma unroll
  for (int e = 0; e < 8; e++) {
    const int E = (int)((hw[e] >> 20) & 0x7FFu);
    Er = max(Er, E);
    Emin = min(Emin, E);
  }
  // a round whose 8 elements are all FP32-normal (exponent fields 897..1150) within 60
  // binades of each other needs no per-element range test in the norm or the copies
  const bool fast = Emin >= 897 && Er <= 1150 && Er - Emin <= 60;
  // ... and a round whose elements all have exponent fields 949..1150 splits on the fast path
  const bool fast_split = Emin >= 949 && Er <= 1150;
  if constexpr (M == (kTF32 | kTLO) || M == (kBF16 | kLO)) {   // split operands: norm and copies on the FP32 pipe
    if (Emin >= 949 && Er <= 1149 && Er - Emin <= 60) {
      k1_round_split<B, M == (kTF32 | kTLO)>(p, tile, hw, lw, rows, cols, Er, acc);
      return;
    }
  }
  if (Er > 0 && Er < 0x7FF) {
    // two independent double-float sums (even and odd elements) halve the dependency
    // chain; they are joined once per round
    float S[2] = {0.f, 0.f}, s2[2] = {0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int E = (int)((hw[e] >> 20) & 0x7FFu);
      const int es = E - Er;
      if (!fast && (E == 0 || es < -60)) continue;   // below 2^-120 of the round's largest square
      // hi: sign-free top 24 significand bits; lo: the bits below
      const float hi = __uint_as_float(((uint32_t)(es + 127) << 23) | (((hw[e] & 0xFFFFFu) << 3) | (lw[e] >> 29)));
      // (the next 23 bits, as an exact FP32 integer: their last 6 bits' share of the
      // square is below 2^-46), times two: lo2 = 2 lo for the cross term 2 hi lo
      const float lo2 = u23_to_float((lw[e] >> 6) & 0x7FFFFFu) * __uint_as_float((uint32_t)(es - 45 + 127) << 23);
      const float pp = hi * hi;
      float cc = fmaf(hi, hi, -pp);
      cc = fmaf(hi, lo2, cc);
      float &Sx = S[e & 1], &sx = s2[e & 1];
      const float t = Sx + pp;
      const float tb = t - Sx;
      sx += ((Sx - (t - tb)) + (pp - tb)) + cc;
      Sx = t;
    }
    df_add(S[0], s2[0], S[1], s2[1]);
    acc.merge(S[0], s2[0], Er);
  } else if (Er == 0x7FF) {
    acc.merge(__uint_as_float(0x7F800000u), 0.f, 0x7FE);
  }
  // leaf copies of the round
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int64_t o = tile + (int64_t)rows[u] * B + cols[u];
    const uint32_t h0 = hw[2 * u], l0 = lw[2 * u], h1 = hw[2 * u + 1], l1 = lw[2 * u + 1];
    const int E0 = (int)((h0 >> 20) & 0x7FFu), E1 = (int)((h1 >> 20) & 0x7FFu);
    if (p.f64)
      *reinterpret_cast<double2 *>(p.f64 + o) =
          make_double2(__hiloint2double((int)h0, (int)l0), __hiloint2double((int)h1, (int)l1));
    if (p.f32) {
      const uint32_t a0 = (E0 >= 897 && E0 <= 1150) ? f32_fast(h0, l0)
                                                   : slow_round_bits(h0, l0, 24, -126);
      const uint32_t a1 = (E1 >= 897 && E1 <= 1150) ? f32_fast(h1, l1)
                                                   : slow_round_bits(h1, l1, 24, -126);
      *reinterpret_cast<uint2 *>(p.f32 + o) = make_uint2(a0, a1);
    }
    if (p.bf16 || s_bf16T || p.lo || s_loT) {
      uint32_t b0, b1;
      if (fast || (E0 >= 897 && E0 <= 1150 && E1 >= 897 && E1 <= 1150)) {
        const uint32_t pk = bf16x2_fast(h0, l0, h1, l1);
        b0 = pk & 0xFFFFu;
        b1 = pk >> 16;
      } else {   // out of the FP32-normal range: out of line
        b0 = (E0 >= 897 && E0 <= 1150) ? bf16_fast(h0, l0) : (slow_round_bits(h0, l0, 8, -126) >> 16);
        b1 = (E1 >= 897 && E1 <= 1150) ? bf16_fast(h1, l1) : (slow_round_bits(h1, l1, 8, -126) >> 16);
      }
      if (p.bf16) *reinterpret_cast<uint32_t *>(p.bf16 + o) = b0 | (b1 << 16);
      if (s_bf16T) {
        s_bf16T[cols[u] * B + rows[u]] = (uint16_t)b0;
        s_bf16T[(cols[u] + 1) * B + rows[u]] = (uint16_t)b1;
      }
      if (p.lo || s_loT) {   // low parts of the split: bf16(x - hi)
        uint32_t q0, q1;
        if (fast_split || (E0 >= 949 && E0 <= 1150 && E1 >= 949 && E1 <= 1150)) {
          uint32_t pk;
          asm("cvt.rn.bf16x2.f32 %0, %1, %2;"
              : "=r"(pk)
              : "f"(__uint_as_float(split_lo_sticky<45>(h1, l1, E1))),
                "f"(__uint_as_float(split_lo_sticky<45>(h0, l0, E0))));
          q0 = pk & 0xFFFFu;
          q1 = pk >> 16;
        } else {
          q0 = slow_split_lo(h0, l0, 8) >> 16;
          q1 = slow_split_lo(h1, l1, 8) >> 16;
        }
        if (p.lo) *reinterpret_cast<uint32_t *>(p.lo + o) = q0 | (q1 << 16);
        if (s_loT) {
          s_loT[cols[u] * B + rows[u]] = (uint16_t)q0;
          s_loT[(cols[u] + 1) * B + rows[u]] = (uint16_t)q1;
        }
      }
    }
    if (p.tf32 || s_tf32T || p.tlo || s_tloT) {
      const uint32_t t0 = (E0 >= 897 && E0 <= 1150) ? tf32_fast(h0, l0) : slow_round_bits(h0, l0, 11, -126);
      const uint32_t t1 = (E1 >= 897 && E1 <= 1150) ? tf32_fast(h1, l1) : slow_round_bits(h1, l1, 11, -126);
      if (p.tf32) *reinterpret_cast<uint2 *>(p.tf32 + o) = make_uint2(t0, t1);
      if (s_tf32T) {
        s_tf32T[cols[u] * B + rows[u]] = __uint_as_float(t0);
        s_tf32T[(cols[u] + 1) * B + rows[u]] = __uint_as_float(t1);
      }
      if (p.tlo || s_tloT) {   // low parts of the split: tf32(x - hi)
        uint32_t q0, q1;
        if (fast_split || (E0 >= 949 && E0 <= 1150 && E1 >= 949 && E1 <= 1150)) {
          q0 = tf32_of_sticky(split_lo_sticky<42>(h0, l0, E0));
          q1 = tf32_of_sticky(split_lo_sticky<42>(h1, l1, E1));
        } else {
          q0 = slow_split_lo(h0, l0, 11);
          q1 = slow_split_lo(h1, l1, 11);
        }
        if (p.tlo) *reinterpret_cast<uint2 *>(p.tlo + o) = make_uint2(q0, q1);
        if (s_tloT) {
          s_tloT[cols[u] * B + rows[u]] = __uint_as_float(q0);
          s_tloT[(cols[u] + 1) * B + rows[u]] = __uint_as_float(q1);
        }
      }
    }
    if (p.fp16 || s_fp16T) {
      const uint32_t f0 = (E0 >= 985 && E0 <= 1038) ? fp16_fast(h0, l0, E0)
          : slow_fp16_bits(h0, l0);
      const uint32_t f1 = (E1 >= 985 && E1 <= 1038) ? fp16_fast(h1, l1, E1)
          : slow_fp16_bits(h1, l1);
      if (p.fp16) *reinterpret_cast<uint32_t *>(p.fp16 + o) = f0 | (f1 << 16);
      if (s_fp16T) {
        s_fp16T[cols[u] * B + rows[u]] = (uint16_t)f0;
        s_fp16T[(cols[u] + 1) * B + rows[u]] = (uint16_t)f1;
      }
    }
  }
}

template <uint32_t M>
__device__ __forceinline__ BuildArgs masked(const BuildArgs &in) {
  BuildArgs p = in;
  if (!(M & kF64)) p.f64 = nullptr;
  if (!(M & kF32)) p.f32 = nullptr;
  if (!(M & kTF32)) p.tf32 = nullptr;
  if (!(M & kTF32T)) p.tf32T = nullptr;
  if (!(M & kTLO)) p.tlo = nullptr;
  if (!(M & kTLOT)) p.tloT = nullptr;
  if (!(M & kBF16)) p.bf16 = nullptr;
  if (!(M & kBF16T)) p.bf16T = nullptr;
  if (!(M & kLO)) p.lo = nullptr;
  if (!(M & kLOT)) p.loT = nullptr;
  if (!(M & kFP16)) p.fp16 = nullptr;
  if (!(M & kFP16T)) p.fp16T = nullptr;
  return p;
}

// The squared norm of a leaf from its warps' double-float partials (each scaled by
// 2^(-2 (e - 1023))): merged in order in double-float, converted to FP64 once.
__device__ __forceinline__ double merge_warps(const float *h, const float *l, const int *e, int count) {
  NormAcc m;
  for (int w = 0; w < count; w++) m.merge(h[w], l[w], e[w]);
  return m.E ? ldexp((double)m.H + (double)m.L, 2 * (m.E - 1023)) : 0.0;
}

template <int B, bool VEC, uint32_t M>
__global__ void __launch_bounds__(BuildCfg<B>::T, 1024 / BuildCfg<B>::T) k_tree_build(BuildArgs p_in) {
  const BuildArgs p = masked<M>(p_in);
  using Cfg = BuildCfg<B>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_h[8], s_l[8];
  __shared__ int s_e[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = threadIdx.x / Cfg::TPL, tl = threadIdx.x % Cfg::TPL;
  const int64_t leaf = (int64_t)blockIdx.x * Cfg::LPC + li;
  const bool inrange = leaf < (int64_t)p.NB * p.NB;
  const int32_t r = inrange ? (int32_t)(leaf / p.NB) : 0, c = inrange ? (int32_t)(leaf % p.NB) : 0;
  const bool stored = inrange && r < p.nb && c < p.nb;
  const int64_t tile = ((int64_t)r * p.nb + c) * (int64_t)B * B;
  const size_t bb = (size_t)B * B;
  const bool any_t = p.tf32T || p.bf16T || p.fp16T || p.loT || p.tloT;
  float *s_tf32T = nullptr, *s_tloT = nullptr;
  uint16_t *s_bf16T = nullptr, *s_fp16T = nullptr, *s_loT = nullptr;
  {
    unsigned char *q = smem;
    if (p.tf32T) { s_tf32T = (float *)q + li * bb; q += Cfg::LPC * bb * 4; }
    if (p.tloT) { s_tloT = (float *)q + li * bb; q += Cfg::LPC * bb * 4; }
    if (p.bf16T) { s_bf16T = (uint16_t *)q + li * bb; q += Cfg::LPC * bb * 2; }
    if (p.fp16T) { s_fp16T = (uint16_t *)q + li * bb; q += Cfg::LPC * bb * 2; }
    if (p.loT) { s_loT = (uint16_t *)q + li * bb; q += Cfg::LPC * bb * 2; }
  }
  // a leaf wholly inside the matrix loads without bounds checks
  const bool full = stored && (int64_t)(r + 1) * B <= p.n && (int64_t)(c + 1) * B <= p.n;
  NormAcc acc;
  if (stored) {
#pragma unroll 1
    for (int rd = 0; rd < Cfg::ROUNDS; rd++) {
      uint32_t hw[8], lw[8];   // high and low words of the round's 8 elements
      int rows[4], cols[4];
      if (VEC && full && rd + 1 < Cfg::ROUNDS) {
        // the next round's lines into L2 while this round's arithmetic runs
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int q = tl + Cfg::TPL * (4 * (rd + 1) + u);
          const int64_t gr = (int64_t)r * B + q / (B / 2), gc = (int64_t)c * B + 2 * (q % (B / 2));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p.A + gr * p.n + gc));
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int q = tl + Cfg::TPL * (4 * rd + u);
        rows[u] = q / (B / 2);
        cols[u] = 2 * (q % (B / 2));
        const int64_t gr = (int64_t)r * B + rows[u], gc = (int64_t)c * B + cols[u];
        double2 d = make_double2(0.0, 0.0);
        if (VEC && full) {
          d = __ldcs(reinterpret_cast<const double2 *>(p.A + gr * p.n + gc));
        } else if (gr < p.n) {
          const double *src = p.A + gr * p.n + gc;
          if (VEC && gc + 1 < p.n) {
            d = __ldcs(reinterpret_cast<const double2 *>(src));
          } else {
            if (gc < p.n) d.x = __ldcs(src);
            if (gc + 1 < p.n) d.y = __ldcs(src + 1);
          }
        }
        hw[2 * u] = (uint32_t)__double2hiint(d.x);
        lw[2 * u] = (uint32_t)__double2loint(d.x);
        hw[2 * u + 1] = (uint32_t)__double2hiint(d.y);
        lw[2 * u + 1] = (uint32_t)__double2loint(d.y);
      }
      k1_round<B, M>(p, tile, hw, lw, rows, cols, acc, s_tf32T, s_tloT, s_bf16T, s_fp16T, s_loT);
    }
  }
  // leaf norm: threads -> warp (rescale to the warp's largest exponent) -> leaf
  const int Ew = __reduce_max_sync(0xffffffffu, acc.E);
  float H = 0.f, L = 0.f;
  if (acc.E) {
    const float f = pow4(acc.E - Ew);
    H = acc.H * f;
    L = acc.L * f;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, H, off), l2 = __shfl_xor_sync(0xffffffffu, L, off);
    df_add(H, L, h2, l2);
  }
  if (lane == 0) {
    s_h[warp] = H;
    s_l[warp] = L;
    s_e[warp] = Ew;
  }
  __syncthreads();
  constexpr int WPL = Cfg::TPL >= 32 ? Cfg::TPL / 32 : 1;
  if (tl == 0 && inrange) {
    if (stored) {
      p.leaf_norm2[leaf] = merge_warps(s_h + li * WPL, s_l + li * WPL, s_e + li * WPL, WPL);
      p.nz[leaf] = 1;
    } else {
      p.leaf_norm2[leaf] = 0.0;
      p.nz[leaf] = 0;
    }
  }
  if (!any_t) return;
  __syncthreads();
  if (!stored) return;
  // transposed copies: shared -> global, 16-byte vectors
  if (s_tf32T)
    for (int q = tl; q < (int)(bb / 4); q += Cfg::TPL)
      reinterpret_cast<float4 *>(p.tf32T + tile)[q] = reinterpret_cast<const float4 *>(s_tf32T)[q];
  if (s_tloT)
    for (int q = tl; q < (int)(bb / 4); q += Cfg::TPL)
      reinterpret_cast<float4 *>(p.tloT + tile)[q] = reinterpret_cast<const float4 *>(s_tloT)[q];
  if (s_bf16T)
    for (int q = tl; q < (int)(bb / 8); q += Cfg::TPL)
      reinterpret_cast<uint4 *>(p.bf16T + tile)[q] = reinterpret_cast<const uint4 *>(s_bf16T)[q];
  if (s_fp16T)
    for (int q = tl; q < (int)(bb / 8); q += Cfg::TPL)
      reinterpret_cast<uint4 *>(p.fp16T + tile)[q] = reinterpret_cast<const uint4 *>(s_fp16T)[q];
  if (s_loT)
    for (int q = tl; q < (int)(bb / 8); q += Cfg::TPL)
      reinterpret_cast<uint4 *>(p.loT + tile)[q] = reinterpret_cast<const uint4 *>(s_loT)[q];
}

// Norm pyramid, parent^2 = ((n11 + n12) + n21) + n22 of the children's squared norms,
// and norm = sqrt(norm^2) on every tier (IEEE sqrt, as the cull test needs). One CTA
// per 16 x 16 region of leaves builds the four tiers above them inside shared memory,
// spreading the FP64 work over many SMs; a single CTA finishes the tiers above.
constexpr int kPyrR = 16;   // region side (leaves)
constexpr int kPyrL = 4;    // tiers built per region: log2(kPyrR)

// Tiers top .. 0 from tier top + 1 (used by the last region CTA and by k_pyramid_top).
__device__ __forceinline__ void pyramid_top_tiers(double *norm2, double *norm, int32_t top_tier) {
  for (int l = top_tier; l >= 0; l--) {
    const int64_t d = int64_t(1) << l, dc = 2 * d;
    const double *c2 = norm2 + level_offset(l + 1);
    double *p2 = norm2 + level_offset(l);
    double *p1 = norm + level_offset(l);
    for (int64_t t = threadIdx.x; t < d * d; t += blockDim.x) {
      const int64_t I = t / d, K = t % d;
      const int64_t i11 = (2 * I) * dc + 2 * K, i21 = (2 * I + 1) * dc + 2 * K;
      const double s = ((__ldcg(c2 + i11) + __ldcg(c2 + i11 + 1)) + __ldcg(c2 + i21)) + __ldcg(c2 + i21 + 1);
      p2[t] = s;
      p1[t] = sqrt(s);
    }
    __syncthreads();
  }
}

// With `ctr` set, the region CTA that arrives last also builds the tiers above the
// regions (top_tier .. 0) and resets the counter for the next launch.
__global__ void __launch_bounds__(256) k_pyramid_region(double *norm2, double *norm, int32_t kmax,
                                                        unsigned int *ctr, int32_t top_tier) {
  __shared__ double s0[kPyrR * kPyrR], s1[kPyrR * kPyrR / 4];
  __shared__ bool s_last;
  const int R = min(kPyrR, 1 << kmax);          // region side for small trees
  const int levels = min(kPyrL, kmax);
  const int64_t NB = int64_t(1) << kmax;
  const int64_t per_side = NB / R;
  const int64_t RI = blockIdx.x / per_side, RK = blockIdx.x % per_side;
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    const int li = t / R, lk = t % R;
    const int64_t idx = level_offset(kmax) + (RI * R + li) * NB + (RK * R + lk);
    const double v = norm2[idx];
    norm[idx] = sqrt(v);
    s0[t] = v;
  }
  __syncthreads();
  double *cur = s0, *nxt = s1;
  int d = R;
  for (int lev = 1; lev <= levels; lev++) {
    const int dp = d / 2;
    const int tier = kmax - lev;
    const int64_t W = NB >> lev;
    for (int t = threadIdx.x; t < dp * dp; t += blockDim.x) {
      const int li = t / dp, lk = t % dp;
      const double n11 = cur[(2 * li) * d + 2 * lk], n12 = cur[(2 * li) * d + 2 * lk + 1];
      const double n21 = cur[(2 * li + 1) * d + 2 * lk], n22 = cur[(2 * li + 1) * d + 2 * lk + 1];
      const double sum = ((n11 + n12) + n21) + n22;
      const int64_t idx = level_offset(tier) + (RI * dp + li) * W + (RK * dp + lk);
      norm2[idx] = sum;
      norm[idx] = sqrt(sum);
      nxt[t] = sum;
    }
    __syncthreads();
    double *tmp = cur;
    cur = nxt;
    nxt = tmp;
    d = dp;
  }
  if (!ctr) return;
  __threadfence();   // this CTA's tiers are visible before it is counted
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  pyramid_top_tiers(norm2, norm, top_tier);
  if (threadIdx.x == 0) *ctr = 0u;
}

// Tiers kmax - 5 .. 0 (above the regions) in one CTA, for trees without a counter.
__global__ void __launch_bounds__(1024) k_pyramid_top(double *norm2, double *norm, int32_t top_tier) {
  pyramid_top_tiers(norm2, norm, top_tier);
}

// Dense row-major image (FP64, or FP32 rounded to nearest) of a tree's master tiles. A
// thread writes four consecutive columns of one row (they lie in one leaf: b is a
// multiple of 4), rows are spread over grid.y; 16-byte stores when the output rows are
// 16-byte aligned. The output may be device memory or mapped page-locked host memory.
template <typename T, typename O>
__global__ void __launch_bounds__(256) k_to_dense(const T *tiles, const uint8_t *nz, int64_t n, int32_t lb,
                                                  int32_t nb, int32_t NB, O *out, int vec) {
  const int32_t b = 1 << lb;
  const int64_t groups = (n + 3) / 4;   // four-column groups per row
  for (int64_t row = blockIdx.y; row < n; row += gridDim.y) {
    const int64_t r = row >> lb, rr = row & (b - 1);
    O *orow = out + row * n;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
      const int64_t col = 4 * g, c = col >> lb, cc = col & (b - 1);
      O v[4] = {O(0), O(0), O(0), O(0)};
      if (nz[r * NB + c]) {
        const T *src = tiles + ((r * nb + c) * b + rr) * b + cc;
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] = (O)src[q];   // col + q < b: same leaf, stored
      }
      if (vec && col + 3 < n) {
        if constexpr (sizeof(O) == 8) {
          reinterpret_cast<double2 *>(orow + col)[0] = make_double2(v[0], v[1]);
          reinterpret_cast<double2 *>(orow + col)[1] = make_double2(v[2], v[3]);
        } else {
          *reinterpret_cast<float4 *>(orow + col) = make_float4(v[0], v[1], v[2], v[3]);
        }
      } else {
        for (int q = 0; q < 4 && col + q < n; q++) orow[col + q] = v[q];
      }
    }
  }
}

}  // namespace

template <int B, bool VEC, uint32_t M>
static cudaError_t run_build_m(const BuildArgs &p, size_t sm, cudaStream_t s) {
  using Cfg = BuildCfg<B>;
  const int64_t leaves = (int64_t)p.NB * p.NB;
  const unsigned grid = (unsigned)((leaves + Cfg::LPC - 1) / Cfg::LPC);
  auto k = k_tree_build<B, VEC, M>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, Cfg::T, sm, s>>>(p);
  return cudaGetLastError();
}

template <int B>
static cudaError_t run_build(const BuildArgs &p, size_t bytes_per_leaf_T, bool vec, cudaStream_t s) {
  using Cfg = BuildCfg<B>;
  const size_t sm = bytes_per_leaf_T * Cfg::LPC;
  const uint32_t m = (p.f64 ? kF64 : 0u) | (p.f32 ? kF32 : 0u) | (p.tf32 ? kTF32 : 0u) | (p.tf32T ? kTF32T : 0u) |
                     (p.tlo ? kTLO : 0u) | (p.tloT ? kTLOT : 0u) | (p.bf16 ? kBF16 : 0u) | (p.bf16T ? kBF16T : 0u) |
                     (p.lo ? kLO : 0u) | (p.loT ? kLOT : 0u) | (p.fp16 ? kFP16 : 0u) | (p.fp16T ? kFP16T : 0u);
  if constexpr (B == 64 || B == 128) {
    if (vec) switch (m) {
      case 0: return run_build_m<B, true, 0>(p, sm, s);
      case kF64: return run_build_m<B, true, kF64>(p, sm, s);
      case kBF16: return run_build_m<B, true, kBF16>(p, sm, s);
      case kBF16 | kLO: return run_build_m<B, true, kBF16 | kLO>(p, sm, s);
      case kTF32: return run_build_m<B, true, kTF32>(p, sm, s);
      case kTF32 | kTLO: return run_build_m<B, true, kTF32 | kTLO>(p, sm, s);
      case kFP16: return run_build_m<B, true, kFP16>(p, sm, s);
      default: break;
    }
  }
  return vec ? run_build_m<B, true, kAllCopies>(p, sm, s) : run_build_m<B, false, kAllCopies>(p, sm, s);
}

cudaError_t launch_tree_build(spamm_tree t, const double *A, cudaStream_t s) {
  BuildArgs p{};
  p.A = A;
  p.n = t->n;
  p.b = t->b;
  p.nb = t->nb;
  p.NB = t->NB;
  p.kmax = t->kmax;
  p.leaf_norm2 = t->norm2 + level_offset(t->kmax);
  p.nz = t->nz;
  p.f64 = (double *)t->copy[CK_F64];
  p.f32 = (float *)t->copy[CK_F32];
  p.tf32 = (float *)t->copy[CK_TF32];
  p.tf32T = (float *)t->copy[CK_TF32_T];
  p.tlo = (float *)t->copy[CK_TF32LO];
  p.tloT = (float *)t->copy[CK_TF32LO_T];
  p.bf16 = (uint16_t *)t->copy[CK_BF16];
  p.bf16T = (uint16_t *)t->copy[CK_BF16_T];
  p.fp16 = (uint16_t *)t->copy[CK_FP16];
  p.fp16T = (uint16_t *)t->copy[CK_FP16_T];
  p.lo = (uint16_t *)t->copy[CK_BF16LO];
  p.loT = (uint16_t *)t->copy[CK_BF16LO_T];
  size_t per_leaf = 0;
  const size_t bb = (size_t)t->b * t->b;
  if (p.tf32T) per_leaf += bb * 4;
  if (p.tloT) per_leaf += bb * 4;
  if (p.bf16T) per_leaf += bb * 2;
  if (p.fp16T) per_leaf += bb * 2;
  if (p.loT) per_leaf += bb * 2;
  const bool vec = (t->n % 2) == 0 && (((uintptr_t)A) % 16) == 0;
  switch (t->b) {
    case 16: return run_build<16>(p, per_leaf, vec, s);
    case 32: return run_build<32>(p, per_leaf, vec, s);
    case 64: return run_build<64>(p, per_leaf, vec, s);
    case 128: return run_build<128>(p, per_leaf, vec, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pyramid(spamm_tree t, cudaStream_t s) {
  const int R = std::min(kPyrR, 1 << t->kmax);
  const int64_t per_side = (int64_t(1) << t->kmax) / R;
  const int top = t->kmax - kPyrL - 1;
  unsigned int *ctr = top >= 0 ? t->pyr_ctr : nullptr;
  k_pyramid_region<<<(unsigned)(per_side * per_side), 256, 0, s>>>(t->norm2, t->norm, t->kmax, ctr, top);
  if (top >= 0 && !ctr) k_pyramid_top<<<1, 1024, 0, s>>>(t->norm2, t->norm, top);
  return cudaGetLastError();
}

// kernels launch_pyramid issues for this tree
int pyramid_launches(spamm_tree t) { return 1 + (t->kmax - kPyrL - 1 >= 0 && !t->pyr_ctr ? 1 : 0); }


// C_ji := C_ij^T for every stored block i < j of a symmetric product (master tiles,
// squared leaf norm, presence byte). Work item w is sub-tile w % S (E x E elements,
// S = (b / E)^2) of block w / S in row-major block order; a CTA of 256 threads first
// tests 256 of its items at once and then moves the sub-tiles of stored blocks above the
// diagonal, one per iteration, with 16-byte loads and stores (V elements each) through a
// padded shared-memory tile.
template <typename T, int E, int V>
__global__ void __launch_bounds__(256) k_mirror(T *tiles, uint8_t *nz, double *leaf_norm2, int32_t b, int32_t nb,
                                                int32_t NB) {
  static_assert((E * E) % (256 * V) == 0, "whole vectors per thread");
  constexpr int VR = E / V;                     // vectors per tile row
  constexpr int PER = E * E / (256 * V);        // vectors per thread
  constexpr int RSTEP = 256 / VR;               // tile rows covered by one pass of the CTA
  using Vec = typename std::conditional<V * sizeof(T) == 16, uint4,
              typename std::conditional<V * sizeof(T) == 8, uint2, uint32_t>::type>::type;
  __shared__ T s[E][E + 1];
  __shared__ int64_t s_list[256];   // this CTA's items that need moving, from one parallel scan
  __shared__ int s_cnt;
  const int sub = b / E, S = sub * sub;
  const int vc = threadIdx.x % VR, vr = threadIdx.x / VR;
  const int64_t items = (int64_t)nb * nb * S;
  // the CTA's items are blockIdx.x + m * gridDim.x; 256 of them are tested at once (one
  // presence byte each) and only the blocks above the diagonal that are stored are moved
  for (int64_t m0 = 0; (int64_t)blockIdx.x + m0 * gridDim.x < items; m0 += 256) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    {
      const int64_t w = (int64_t)blockIdx.x + (m0 + threadIdx.x) * gridDim.x;
      if (w < items) {
        const int64_t t = w / S;
        const int32_t i = (int32_t)(t / nb), j = (int32_t)(t % nb);
        if (i < j && nz[(int64_t)i * NB + j]) s_list[atomicAdd(&s_cnt, 1)] = w;
      }
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int m = 0; m < cnt; m++) {
      const int64_t w = s_list[m];
      const int64_t t = w / S;
      const int q = (int)(w % S);
      const int32_t i = (int32_t)(t / nb), j = (int32_t)(t % nb);
      const int64_t uij = (int64_t)i * NB + j, uji = (int64_t)j * NB + i;
      const int r0 = (q / sub) * E, c0 = (q % sub) * E;   // sub-tile origin in block (i, j)
      const T *src = tiles + ((int64_t)i * nb + j) * b * b;
      T *dst = tiles + ((int64_t)j * nb + i) * b * b;
      __syncthreads();   // the previous item's reads of s are done
#pragma unroll
      for (int k = 0; k < PER; k++) {
        const int y = vr + k * RSTEP;
        union { Vec v; T e[V]; } u;
        u.v = *reinterpret_cast<const Vec *>(src + (int64_t)(r0 + y) * b + c0 + vc * V);
#pragma unroll
        for (int e = 0; e < V; e++) s[y][vc * V + e] = u.e[e];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < PER; k++) {
        const int y = vr + k * RSTEP;   // row c0 + y of block (j, i) = column c0 + y of (i, j)
        union { Vec v; T e[V]; } u;
#pragma unroll
        for (int e = 0; e < V; e++) u.e[e] = s[vc * V + e][y];
        *reinterpret_cast<Vec *>(dst + (int64_t)(c0 + y) * b + r0 + vc * V) = u.v;
      }
      if (q == 0 && threadIdx.x == 0) {
        leaf_norm2[uji] = leaf_norm2[uij];
        nz[uji] = 1;
      }
    }
    __syncthreads();   // s_list and s_cnt are reused
  }
}

template <typename T, int E, int V>
static void run_mirror(spamm_tree C, T *tiles, double *ln2, cudaStream_t s) {
  const int64_t S = (C->b / E) * (C->b / E);
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)C->nb * C->nb * S, (int64_t)C->ctx->sm_count * 8);
  k_mirror<T, E, V><<<grid, 256, 0, s>>>(tiles, C->nz, ln2, C->b, C->nb, C->NB);
}

cudaError_t launch_mirror(spamm_tree C, cudaStream_t s) {
  double *ln2 = C->norm2 + level_offset(C->kmax);
  if (C->copy[CK_F64]) {
    double *t = (double *)C->copy[CK_F64];
    if (C->b >= 32) run_mirror<double, 32, 2>(C, t, ln2, s);
    else if (C->b == 16) run_mirror<double, 16, 1>(C, t, ln2, s);
    else return cudaErrorInvalidValue;
  } else if (C->copy[CK_F32]) {
    float *t = (float *)C->copy[CK_F32];
    if (C->b >= 64) run_mirror<float, 64, 4>(C, t, ln2, s);
    else if (C->b == 32) run_mirror<float, 32, 4>(C, t, ln2, s);
    else if (C->b == 16) run_mirror<float, 16, 1>(C, t, ln2, s);
    else return cudaErrorInvalidValue;
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The dropping filter of the paper's scheme (I) (Sec. III, after each multiplication):
// a stored leaf block whose Frobenius norm sqrt(norm^2) is below tau is no longer stored
// (presence byte and squared norm cleared; readers never load the tile of an absent
// block). Counts the blocks that stay.
__global__ void __launch_bounds__(256) k_drop_blocks(uint8_t *nz, double *leaf_norm2, int32_t nb, int32_t NB,
                                                     double tau, unsigned long long *kept) {
  unsigned int mine = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nb * nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t li = (t / nb) * NB + (t % nb);
    if (!nz[li]) continue;
    if (sqrt(leaf_norm2[li]) < tau) {
      nz[li] = 0;
      leaf_norm2[li] = 0.0;
    } else {
      mine++;
    }
  }
  if (!kept) return;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, off);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(kept, (unsigned long long)mine);
}

cudaError_t launch_drop(spamm_tree t, double tau, unsigned long long *kept, cudaStream_t s) {
  const int64_t blocks = (int64_t)t->nb * t->nb;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((blocks + 255) / 256, 4096));
  k_drop_blocks<<<grid, 256, 0, s>>>(t->nz, t->norm2 + level_offset(t->kmax), t->nb, t->NB, tau, kept);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pyramid(t, s);
}

template <typename O>
static cudaError_t to_dense_as(spamm_tree t, O *out, cudaStream_t s) {
  int lb = 0;
  while ((1 << lb) < t->b) lb++;
  const int64_t groups = (t->n + 3) / 4;
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((groups + 255) / 256, 8)),
                  (unsigned)std::min<int64_t>(t->n, 8192));
  // 16-byte stores need 16-byte aligned rows
  const int vec = (t->n * (int64_t)sizeof(O)) % 16 == 0 && ((uintptr_t)out % 16) == 0;
  if (t->copy[CK_F64]) {
    k_to_dense<double, O><<<grid, 256, 0, s>>>((const double *)t->copy[CK_F64], t->nz, t->n, lb, t->nb, t->NB,
                                               out, vec);
  } else if (t->copy[CK_F32]) {
    k_to_dense<float, O><<<grid, 256, 0, s>>>((const float *)t->copy[CK_F32], t->nz, t->n, lb, t->nb, t->NB,
                                              out, vec);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_dense(spamm_tree t, double *out, cudaStream_t s) { return to_dense_as<double>(t, out, s); }

cudaError_t launch_to_dense_f32(spamm_tree t, float *out, cudaStream_t s) { return to_dense_as<float>(t, out, s); }

// ---- leaf copies of a product tree, from its master tiles (FP64 or FP32) ----
namespace {

struct ConvertArgs {
  const void *src;
  int src_f64;
  const uint8_t *nz;
  int32_t b, nb, NB;
  float *tf32, *tf32T, *tlo, *tloT;
  uint16_t *bf16, *bf16T, *fp16, *fp16T, *lo, *loT;
};

__global__ void __launch_bounds__(256) k_tile_convert(ConvertArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t b = p.b;
  const int64_t leaf = blockIdx.x;
  const int32_t r = (int32_t)(leaf / p.nb), c = (int32_t)(leaf % p.nb);
  if (!p.nz[(int64_t)r * p.NB + c]) return;   // never read: zero blocks load as zero fill
  const int64_t tile = leaf * (int64_t)b * b;
  float *s_tf32T = nullptr, *s_tloT = nullptr;
  uint16_t *s_bf16T = nullptr, *s_fp16T = nullptr, *s_loT = nullptr;
  {
    unsigned char *q = smem;
    if (p.tf32T) { s_tf32T = (float *)q; q += (size_t)b * b * 4; }
    if (p.tloT) { s_tloT = (float *)q; q += (size_t)b * b * 4; }
    if (p.bf16T) { s_bf16T = (uint16_t *)q; q += (size_t)b * b * 2; }
    if (p.fp16T) { s_fp16T = (uint16_t *)q; q += (size_t)b * b * 2; }
    if (p.loT) { s_loT = (uint16_t *)q; q += (size_t)b * b * 2; }
  }
  const int32_t bb = b * b;
  for (int32_t e = threadIdx.x; e < bb; e += blockDim.x) {
    const int32_t row = e / b, col = e % b;
    Rounded hb, tb, fb;
    uint32_t lb = 0, tl = 0;
    const bool want_tlo = p.tlo || s_tloT;
    if (p.src_f64) {
      const uint64_t bits = (uint64_t)__double_as_longlong(((const double *)p.src)[tile + e]);
      hb = round_f64bits(bits, 8, -126);
      tb = round_f64bits(bits, 11, -126);
      fb = round_f64bits(bits, 11, -14);
      if (p.lo || s_loT) lb = bf16_lo_bits(bits, hb);
      if (want_tlo) tl = split_lo_bits(bits, tb, 11);
    } else {
      const float f = ((const float *)p.src)[tile + e];
      hb = round_f32(f, 8, -126);
      tb = round_f32(f, 11, -126);
      fb = round_f32(f, 11, -14);
      if (p.lo || s_loT) lb = bf16_lo_bits_f32(f, hb);
      if (want_tlo) tl = split_lo_bits_f32(f, tb, 11);
    }
    if (p.tf32) p.tf32[tile + e] = __uint_as_float(tb.bits);
    if (s_tf32T) s_tf32T[col * b + row] = __uint_as_float(tb.bits);
    if (p.tlo) p.tlo[tile + e] = __uint_as_float(tl);
    if (s_tloT) s_tloT[col * b + row] = __uint_as_float(tl);
    if (p.bf16) p.bf16[tile + e] = bf16_from_f32bits(hb.bits);
    if (s_bf16T) s_bf16T[col * b + row] = bf16_from_f32bits(hb.bits);
    if (p.lo) p.lo[tile + e] = bf16_from_f32bits(lb);
    if (s_loT) s_loT[col * b + row] = bf16_from_f32bits(lb);
    if (p.fp16 || s_fp16T) {
      const uint16_t h = fp16_from_f32bits(fb.bits);
      if (p.fp16) p.fp16[tile + e] = h;
      if (s_fp16T) s_fp16T[col * b + row] = h;
    }
  }
  __syncthreads();
  for (int32_t e = threadIdx.x; e < bb; e += blockDim.x) {
    if (s_tf32T) p.tf32T[tile + e] = s_tf32T[e];
    if (s_tloT) p.tloT[tile + e] = s_tloT[e];
    if (s_bf16T) p.bf16T[tile + e] = s_bf16T[e];
    if (s_fp16T) p.fp16T[tile + e] = s_fp16T[e];
    if (s_loT) p.loT[tile + e] = s_loT[e];
  }
}

}  // namespace

cudaError_t launch_tile_convert(spamm_tree t, cudaStream_t s) {
  ConvertArgs p{};
  p.src_f64 = t->copy[CK_F64] != nullptr;
  p.src = p.src_f64 ? t->copy[CK_F64] : t->copy[CK_F32];
  if (!p.src) return cudaErrorInvalidValue;
  p.nz = t->nz;
  p.b = t->b;
  p.nb = t->nb;
  p.NB = t->NB;
  p.tf32 = (float *)t->copy[CK_TF32];
  p.tf32T = (float *)t->copy[CK_TF32_T];
  p.tlo = (float *)t->copy[CK_TF32LO];
  p.tloT = (float *)t->copy[CK_TF32LO_T];
  p.bf16 = (uint16_t *)t->copy[CK_BF16];
  p.bf16T = (uint16_t *)t->copy[CK_BF16_T];
  p.fp16 = (uint16_t *)t->copy[CK_FP16];
  p.fp16T = (uint16_t *)t->copy[CK_FP16_T];
  p.lo = (uint16_t *)t->copy[CK_BF16LO];
  p.loT = (uint16_t *)t->copy[CK_BF16LO_T];
  if (!p.tf32 && !p.tf32T && !p.bf16 && !p.bf16T && !p.fp16 && !p.fp16T && !p.lo && !p.loT && !p.tlo && !p.tloT)
    return cudaSuccess;
  size_t sm = 0;
  const size_t bb = (size_t)t->b * t->b;
  if (p.tf32T) sm += bb * 4;
  if (p.tloT) sm += bb * 4;
  if (p.bf16T) sm += bb * 2;
  if (p.fp16T) sm += bb * 2;
  if (p.loT) sm += bb * 2;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tile_convert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_tile_convert<<<(unsigned)((int64_t)t->nb * t->nb), 256, sm, s>>>(p);
  return cudaGetLastError();
}
