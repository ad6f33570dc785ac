// Round-to-nearest-even conversions from FP64 to the leaf operand formats.
//
// Each conversion rounds once, from the FP64 value. A direct FP64 -> FP32 ->
// narrow chain with round-to-nearest at both steps can round twice; instead the
// FP64 -> FP32 step rounds to odd (truncate, then set the last bit when anything was
// cut off), which keeps the final round-to-nearest-even exact as long as FP32 has at
// least two more significand bits than the target (Boldo and Melquiond, "Emulation
// of FMA and correctly rounded sums: proved algorithms using rounding to odd",
// IEEE Trans. Computers 57(4), 2008).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

__device__ __forceinline__ float f64_to_f32_odd(double x) {
  float t = __double2float_rz(x);
  if ((double)t != x) {
    uint32_t u = __float_as_uint(t) | 1u;
    t = __uint_as_float(u);
  }
  return t;
}

// FP32 bits -> BF16 bits, round to nearest even (finite inputs).
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float f) {
  uint32_t u = __float_as_uint(f);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

__device__ __forceinline__ uint16_t f64_to_bf16_bits(double x) {
  return f32_to_bf16_bits(f64_to_f32_odd(x));
}

__device__ __forceinline__ double bf16_bits_to_f64(uint16_t h) {
  return (double)__uint_as_float(((uint32_t)h) << 16);
}

__device__ __forceinline__ uint16_t f64_to_fp16_bits(double x) {
  __half h = __float2half_rn(f64_to_f32_odd(x));
  return __half_as_ushort(h);
}

// TF32: FP32 storage with the low 13 significand bits zero, rounded to nearest even.
__device__ __forceinline__ float f64_to_tf32(double x) {
  uint32_t u = __float_as_uint(f64_to_f32_odd(x));
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= ~0x1FFFu;
  return __uint_as_float(u);
}

__device__ __forceinline__ float f32_to_tf32(float f) {
  uint32_t u = __float_as_uint(f);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= ~0x1FFFu;
  return __uint_as_float(u);
}
