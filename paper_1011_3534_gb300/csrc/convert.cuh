// Round-to-nearest-even conversions from FP64 (or FP32) to the leaf operand formats,
// in integer arithmetic on the bit pattern.
//
// A format with p significant bits and minimum normal exponent emin represents a value
// as r * 2^q, q = max(e, emin) - (p - 1), e the exponent of its leading bit; rounding
// is to nearest with ties to even (IEEE 754). BF16: p = 8, emin = -126; FP16: p = 11,
// emin = -14; TF32: p = 11, emin = -126. Every result is returned as the FP32 bit
// pattern of the rounded value, which all three formats fit in exactly.
//
// The integer route keeps these conversions off the FP64 pipe, which on this GPU
// issues a small fraction of the FP32/INT32 rate; it rounds once, from the full
// significand, so there is no double rounding.
#pragma once
#ifndef __CUDA_BF16_H__
#include <cuda_bf16.h>
#endif
#ifndef __CUDA_FP16_H__
#include <cuda_fp16.h>
#endif
#include <stdint.h>

struct Rounded {
  uint32_t bits;   // FP32 bit pattern of the rounded value
  uint32_t r;      // rounded significand: value = r * 2^q
  int q;
};

// (-1)^sign * M * 2^x with M > 0 and leading bit of M at position `top`.
__device__ __forceinline__ Rounded round_core(uint32_t sign, uint64_t M, int x, int top, int p, int emin) {
  Rounded o;
  const int e = x + top;
  const int q = (e > emin ? e : emin) - (p - 1);
  const int shift = q - x;
  uint64_t r;
  if (shift <= 0) {
    r = M << (-shift);
  } else if (shift > 64) {
    r = 0;
  } else if (shift == 64) {
    r = M > (1ull << 63) ? 1 : 0;
  } else {
    r = M >> shift;
    const uint64_t rem = M & ((1ull << shift) - 1), half = 1ull << (shift - 1);
    r += (rem > half || (rem == half && (r & 1ull))) ? 1ull : 0ull;
  }
  o.r = (uint32_t)r;
  o.q = q;
  if (r == 0) {
    o.bits = sign;
    return o;
  }
  const uint32_t r32 = (uint32_t)r;                 // r <= 2^p <= 2^24
  const int t = 31 - __clz((int)r32);
  const int e32 = q + t;
  if (e32 > 127) o.bits = sign | 0x7F800000u;
  else if (e32 >= -126) o.bits = sign | ((uint32_t)(e32 + 127) << 23) | ((r32 << (23 - t)) & 0x7FFFFFu);
  else o.bits = sign | (r32 << (q + 149));          // FP32 subnormal, q >= -149
  return o;
}

// FP64 bit pattern -> rounded value (FP64 zero and subnormals, far below every
// format's range, give signed zero; infinities and NaN pass through).
__device__ __forceinline__ Rounded round_f64bits(uint64_t bits, int p, int emin) {
  const uint32_t sign = (uint32_t)(bits >> 32) & 0x80000000u;
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) {
    Rounded o;
    o.r = 0;
    o.q = 0;
    o.bits = E == 0 ? sign : (sign | 0x7F800000u | ((bits & 0xFFFFFFFFFFFFFull) ? 0x400000u : 0u));
    return o;
  }
  const uint64_t sig = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  return round_core(sign, sig, E - 1075, 52, p, emin);
}

// The low part of a split pair: fmt(x - hi), hi = fmt(x), from the exact integer
// remainder of the significand, rounded to p significant bits (8: BF16, 11: TF32).
__device__ __forceinline__ uint32_t split_lo_bits(uint64_t bits, const Rounded &hi, int p) {
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) return 0;
  const uint64_t sig = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int x = E - 1075;
  const int shift = hi.q - x;                        // >= 42
  int64_t R = (int64_t)sig;
  if (shift < 64) R -= (int64_t)((uint64_t)hi.r << shift);
  if (R == 0) return 0;
  uint32_t sign = (uint32_t)(bits >> 32) & 0x80000000u;
  uint64_t M = (uint64_t)R;
  if (R < 0) {
    sign ^= 0x80000000u;
    M = (uint64_t)(-R);
  }
  return round_core(sign, M, x, 63 - __clzll((long long)M), p, -126).bits;
}

__device__ __forceinline__ uint32_t bf16_lo_bits(uint64_t bits, const Rounded &hi) { return split_lo_bits(bits, hi, 8); }

__device__ __forceinline__ uint16_t bf16_from_f32bits(uint32_t b) { return (uint16_t)(b >> 16); }

__device__ __forceinline__ uint16_t fp16_from_f32bits(uint32_t b) {
  return __half_as_ushort(__float2half_rn(__uint_as_float(b)));   // exact: the value is an FP16 value
}

// FP32 input (product trees of tensor-core precisions): same rounding from the FP32
// significand.
__device__ __forceinline__ Rounded round_f32(float f, int p, int emin) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const int E = (int)((u >> 23) & 0xFF);
  if (E == 0xFF) {
    Rounded o;
    o.r = 0;
    o.q = 0;
    o.bits = u;
    return o;
  }
  if (E == 0) {
    const uint32_t m = u & 0x7FFFFFu;
    if (!m) {
      Rounded o;
      o.r = 0;
      o.q = 0;
      o.bits = sign;
      return o;
    }
    return round_core(sign, m, -149, 31 - __clz((int)m), p, emin);
  }
  return round_core(sign, (u & 0x7FFFFFu) | 0x800000u, E - 150, 23, p, emin);
}

__device__ __forceinline__ uint32_t split_lo_bits_f32(float f, const Rounded &hi, int p) {
  const uint32_t u = __float_as_uint(f);
  const int E = (int)((u >> 23) & 0xFF);
  if (E == 0xFF || (u & 0x7FFFFFFFu) == 0) return 0;
  const uint64_t sig = E ? ((u & 0x7FFFFFu) | 0x800000u) : (u & 0x7FFFFFu);
  const int x = E ? E - 150 : -149;
  const int shift = hi.q - x;
  int64_t R = (int64_t)sig;
  if (shift >= 0 && shift < 64) R -= (int64_t)((uint64_t)hi.r << shift);
  else if (shift < 0) R -= (int64_t)((uint64_t)hi.r >> (-shift));   // not reached: hi.q >= x
  if (R == 0) return 0;
  uint32_t sign = u & 0x80000000u;
  uint64_t M = (uint64_t)R;
  if (R < 0) {
    sign ^= 0x80000000u;
    M = (uint64_t)(-R);
  }
  return round_core(sign, M, x, 63 - __clzll((long long)M), p, -126).bits;
}

__device__ __forceinline__ uint32_t bf16_lo_bits_f32(float f, const Rounded &hi) { return split_lo_bits_f32(f, hi, 8); }

// ---- fast paths on the high and low 32-bit words of an FP64 value ----
// Round to nearest even at bit k = 45 (BF16) or k = 42 (TF32, FP16) of the 64-bit
// pattern: adding (2^(k-1) - 1) + (bit k) rounds the magnitude. Only the high word is
// kept; the low word's all-ones part plus bit k carries into it exactly when the low
// word is nonzero or bit k is set. Valid when the result is a
// normal number of the target format; other inputs take round_f64bits.

// BF16 bits, E (FP64 exponent field) in [897, 1150].
__device__ __forceinline__ uint32_t bf16_fast(uint32_t h, uint32_t l) {
  const uint32_t h2 = h + 0xFFFu + ((((h >> 13) & 1u) | l) != 0u ? 1u : 0u);
  return ((h2 >> 16) & 0x8000u) | ((((h2 >> 20) & 0x7FFu) - 896u) << 7) | ((h2 >> 13) & 0x7Fu);
}

// TF32 (as FP32 bits), E in [897, 1150].
__device__ __forceinline__ uint32_t tf32_fast(uint32_t h, uint32_t l) {
  const uint32_t h2 = h + 0x1FFu + ((((h >> 10) & 1u) | l) != 0u ? 1u : 0u);
  return (h2 & 0x80000000u) | ((((h2 >> 20) & 0x7FFu) - 896u) << 23) | (((h2 >> 10) & 0x3FFu) << 13);
}

// FP16 bits for FP64 exponent fields E in [985, 1038]: normal results (E >= 1009) by
// the bias trick, overflow to infinity, subnormal results (quantum 2^-24) from the
// high significand word with the low word as sticky bit.
__device__ __forceinline__ uint32_t fp16_fast(uint32_t h, uint32_t l, int E) {
  const uint32_t sign = (h >> 16) & 0x8000u;
  if (E >= 1009) {
    const uint32_t h2 = h + 0x1FFu + ((((h >> 10) & 1u) | l) != 0u ? 1u : 0u);
    const uint32_t ex = ((h2 >> 20) & 0x7FFu) - 1008u;
    if (ex >= 31u) return sign | 0x7C00u;
    return sign | (ex << 10) | ((h2 >> 10) & 0x3FFu);
  }
  const uint32_t hs = (h & 0xFFFFFu) | 0x100000u;   // significand bits 52..32
  const int s2 = 1019 - E;                          // 11 .. 34 here
  if (s2 >= 22) return sign;                        // below half the least subnormal
  const uint32_t r = hs >> s2, rem = hs & ((1u << s2) - 1u), half = 1u << (s2 - 1);
  const bool up = rem > half || (rem == half && (l != 0u || (r & 1u)));
  return sign | (r + (up ? 1u : 0u));
}

// FP32 round to nearest even from the FP64 pattern, E in [897, 1150] (normal FP32
// results): the rounding position (bit 29) lies in the low word, so the bias is added
// to the full 64-bit pattern.
__device__ __forceinline__ uint32_t f32_fast(uint32_t h, uint32_t l) {
  const uint64_t u = (((uint64_t)h << 32) | l) + 0x0FFFFFFFull + ((l >> 29) & 1u);
  const uint32_t uh = (uint32_t)(u >> 32);
  return (uh & 0x80000000u) | ((((uh >> 20) & 0x7FFu) - 896u) << 23) | ((uint32_t)(u >> 29) & 0x7FFFFFu);
}

// Low part of the split pair of an FP64 value, hi = fmt(x) rounded at bit K of the
// 64-bit pattern (K = 45: BF16, K = 42: TF32): x - hi = (-1)^s M 2^(E - 1075) exactly,
// M the integer formed by the K discarded significand bits (or 2^K minus them when hi
// rounded up). M is normalised with a count of leading zeros and returned as an FP32
// pattern whose last bit also holds every bit of M below the FP32 significand (sticky),
// so that one round to nearest even at 8 or 11 significant bits gives the correctly
// rounded fmt(x - hi). Zero when x = hi. Valid for FP64 exponent fields E in
// [949, 1150]: a nonzero x - hi is then at least 2^-126, an FP32-normal value.
template <int K>
__device__ __forceinline__ uint32_t split_lo_sticky(uint32_t h, uint32_t l, int E) {
  constexpr uint32_t mask = (1u << (K - 32)) - 1u, half = 1u << (K - 33);
  const uint32_t rh = h & mask;
  const bool lnz = l != 0u;
  const bool up = rh > half || (rh == half && (lnz || ((h >> (K - 32)) & 1u)));
  const uint32_t Mh = up ? mask + 1u - rh - (lnz ? 1u : 0u) : rh;
  const uint32_t Ml = up ? 0u - l : l;
  const uint32_t sign = (h ^ (up ? 0x80000000u : 0u)) & 0x80000000u;
  const bool hz = Mh == 0u;
  const uint32_t top = hz ? Ml : Mh, bot = hz ? 0u : Ml;
  if (top == 0u) return 0u;
  const int lz = __clz((int)top);                        // < 32: top != 0
  const uint32_t T = __funnelshift_lc(bot, top, lz);    // bits p .. p - 31 of M
  const uint32_t rest = bot << lz;
  const int be = E - 948 + (hz ? 31 : 63) - lz;          // FP32 biased exponent of M 2^(E - 1075)
  return sign | ((uint32_t)be << 23) | ((T >> 8) & 0x7FFFFFu) | (((T & 0xFFu) | rest) != 0u ? 1u : 0u);
}

// TF32 (as FP32 bits) of an FP32 pattern with a sticky last bit: round to nearest
// even at bit 13.
__device__ __forceinline__ uint32_t tf32_of_sticky(uint32_t f) {
  return (f + 0xFFFu + ((f >> 13) & 1u)) & 0xFFFFE000u;
}

// Out-of-line rounding for the rare inputs outside a fast path's range, so the fast
// paths stay short branches instead of predicated copies of the general code.
static __device__ __noinline__ uint32_t slow_round_bits(uint32_t h, uint32_t l, int p, int emin) {
  return round_f64bits(((uint64_t)h << 32) | l, p, emin).bits;
}

// fmt(x - fmt(x)) (BF16: p = 8, TF32: p = 11) as FP32 bits, for inputs outside the fast
// split's range.
static __device__ __noinline__ uint32_t slow_split_lo(uint32_t h, uint32_t l, int p) {
  const uint64_t bits = ((uint64_t)h << 32) | l;
  return split_lo_bits(bits, round_f64bits(bits, p, -126), p);
}

static __device__ __noinline__ uint32_t slow_fp16_bits(uint32_t h, uint32_t l) {
  return fp16_from_f32bits(round_f64bits(((uint64_t)h << 32) | l, 11, -14).bits);
}

// Exact FP32 value of an integer below 2^23, on the FP32 pipe: the integer is placed in
// the significand of 2^23 and 2^23 is subtracted.
__device__ __forceinline__ float u23_to_float(uint32_t m) {
  return __uint_as_float(0x4B000000u | m) - 8388608.0f;
}
