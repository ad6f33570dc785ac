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

// The low half of the split BF16 pair: bf16(x - hi), hi = bf16(x), from the exact
// integer remainder of the significand.
__device__ __forceinline__ uint32_t bf16_lo_bits(uint64_t bits, const Rounded &hi) {
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) return 0;
  const uint64_t sig = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int x = E - 1075;
  const int shift = hi.q - x;                        // >= 45
  int64_t R = (int64_t)sig;
  if (shift < 64) R -= (int64_t)((uint64_t)hi.r << shift);
  if (R == 0) return 0;
  uint32_t sign = (uint32_t)(bits >> 32) & 0x80000000u;
  uint64_t M = (uint64_t)R;
  if (R < 0) {
    sign ^= 0x80000000u;
    M = (uint64_t)(-R);
  }
  return round_core(sign, M, x, 63 - __clzll((long long)M), 8, -126).bits;
}

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

__device__ __forceinline__ uint32_t bf16_lo_bits_f32(float f, const Rounded &hi) {
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
  return round_core(sign, M, x, 63 - __clzll((long long)M), 8, -126).bits;
}
