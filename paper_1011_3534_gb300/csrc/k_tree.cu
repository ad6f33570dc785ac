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
#include "convert.cuh"
#include "internal.cuh"

namespace {

struct BuildArgs {
  const double *A;
  int64_t n;
  int32_t b, nb, NB, kmax;
  double *leaf_norm2;      // tier kmax of norm2
  uint8_t *nz;
  double *f64;             // optional copies (nullptr = not written)
  float *tf32, *tf32T;
  uint16_t *bf16, *bf16T, *fp16, *fp16T, *lo, *loT;
};

// One CTA per leaf block. Reads the leaf's b x b window of A once (double2 loads along
// rows, coalesced), sums squares in FP64 (per thread, then a warp shuffle tree, then
// the 8 warp sums in fixed order), and writes every requested copy. Transposed copies
// are staged in shared memory so their global writes stay coalesced.
template <bool VEC>
__global__ void __launch_bounds__(256) k_tree_build(BuildArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t b = p.b;
  const int64_t leaf = blockIdx.x;
  const int32_t r = (int32_t)(leaf / p.NB), c = (int32_t)(leaf % p.NB);
  if (r >= p.nb || c >= p.nb) {
    if (threadIdx.x == 0) {
      p.leaf_norm2[leaf] = 0.0;
      p.nz[leaf] = 0;
    }
    return;
  }
  const int64_t tile = ((int64_t)r * p.nb + c) * (int64_t)b * b;
  const int32_t half = b / 2;
  const int32_t pairs = b * half;
  // transposed staging areas, in the order tf32T, bf16T, fp16T, loT
  float *s_tf32T = nullptr;
  uint16_t *s_bf16T = nullptr, *s_fp16T = nullptr, *s_loT = nullptr;
  {
    unsigned char *q = smem;
    if (p.tf32T) { s_tf32T = (float *)q; q += (size_t)b * b * 4; }
    if (p.bf16T) { s_bf16T = (uint16_t *)q; q += (size_t)b * b * 2; }
    if (p.fp16T) { s_fp16T = (uint16_t *)q; q += (size_t)b * b * 2; }
    if (p.loT) { s_loT = (uint16_t *)q; q += (size_t)b * b * 2; }
  }
  double ss = 0.0;
  for (int32_t q = threadIdx.x; q < pairs; q += blockDim.x) {
    const int32_t row = q / half, col = 2 * (q % half);
    const int64_t gr = (int64_t)r * b + row, gc = (int64_t)c * b + col;
    double v0 = 0.0, v1 = 0.0;
    if (gr < p.n) {
      const double *src = p.A + gr * p.n + gc;
      if (VEC && gc + 1 < p.n) {
        double2 v = __ldcs(reinterpret_cast<const double2 *>(src));
        v0 = v.x;
        v1 = v.y;
      } else {
        if (gc < p.n) v0 = __ldcs(src);
        if (gc + 1 < p.n) v1 = __ldcs(src + 1);
      }
    }
    ss = fma(v0, v0, ss);
    ss = fma(v1, v1, ss);
    const int64_t o = tile + (int64_t)row * b + col;
    if (p.f64) *reinterpret_cast<double2 *>(p.f64 + o) = make_double2(v0, v1);
    if (p.tf32 || s_tf32T) {
      float t0 = f64_to_tf32(v0), t1 = f64_to_tf32(v1);
      if (p.tf32) *reinterpret_cast<float2 *>(p.tf32 + o) = make_float2(t0, t1);
      if (s_tf32T) { s_tf32T[col * b + row] = t0; s_tf32T[(col + 1) * b + row] = t1; }
    }
    if (p.bf16 || s_bf16T || p.lo || s_loT) {
      uint16_t h0 = f64_to_bf16_bits(v0), h1 = f64_to_bf16_bits(v1);
      if (p.bf16) *reinterpret_cast<uint32_t *>(p.bf16 + o) = (uint32_t)h0 | ((uint32_t)h1 << 16);
      if (s_bf16T) { s_bf16T[col * b + row] = h0; s_bf16T[(col + 1) * b + row] = h1; }
      if (p.lo || s_loT) {
        uint16_t l0 = f64_to_bf16_bits(v0 - bf16_bits_to_f64(h0));
        uint16_t l1 = f64_to_bf16_bits(v1 - bf16_bits_to_f64(h1));
        if (p.lo) *reinterpret_cast<uint32_t *>(p.lo + o) = (uint32_t)l0 | ((uint32_t)l1 << 16);
        if (s_loT) { s_loT[col * b + row] = l0; s_loT[(col + 1) * b + row] = l1; }
      }
    }
    if (p.fp16 || s_fp16T) {
      uint16_t h0 = f64_to_fp16_bits(v0), h1 = f64_to_fp16_bits(v1);
      if (p.fp16) *reinterpret_cast<uint32_t *>(p.fp16 + o) = (uint32_t)h0 | ((uint32_t)h1 << 16);
      if (s_fp16T) { s_fp16T[col * b + row] = h0; s_fp16T[(col + 1) * b + row] = h1; }
    }
  }
  // squared Frobenius norm of the leaf
  for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  __shared__ double wsum[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) wsum[warp] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += wsum[w];
    p.leaf_norm2[leaf] = s;
    p.nz[leaf] = 1;
  }
  // transposed copies: shared -> global, 16-byte vectors
  if (s_tf32T) {
    const int32_t v4 = b * b / 4;
    for (int32_t q = threadIdx.x; q < v4; q += blockDim.x)
      reinterpret_cast<float4 *>(p.tf32T + tile)[q] = reinterpret_cast<const float4 *>(s_tf32T)[q];
  }
  const int32_t v8 = b * b / 8;
  if (s_bf16T)
    for (int32_t q = threadIdx.x; q < v8; q += blockDim.x)
      reinterpret_cast<uint4 *>(p.bf16T + tile)[q] = reinterpret_cast<const uint4 *>(s_bf16T)[q];
  if (s_fp16T)
    for (int32_t q = threadIdx.x; q < v8; q += blockDim.x)
      reinterpret_cast<uint4 *>(p.fp16T + tile)[q] = reinterpret_cast<const uint4 *>(s_fp16T)[q];
  if (s_loT)
    for (int32_t q = threadIdx.x; q < v8; q += blockDim.x)
      reinterpret_cast<uint4 *>(p.loT + tile)[q] = reinterpret_cast<const uint4 *>(s_loT)[q];
}

// Leaf tier sqrt plus tier kmax - 1 (one thread per parent): parent^2 =
// ((n11 + n12) + n21) + n22 of the children's squared norms.
__global__ void k_pyramid_low(double *norm2, double *norm, int32_t kmax) {
  const int64_t dl = int64_t(1) << kmax;
  double *c2 = norm2 + level_offset(kmax);
  double *c1 = norm + level_offset(kmax);
  if (kmax == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) c1[0] = sqrt(c2[0]);
    return;
  }
  const int64_t dp = dl / 2;
  double *p2 = norm2 + level_offset(kmax - 1);
  double *p1 = norm + level_offset(kmax - 1);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dp * dp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = t / dp, K = t % dp;
    const int64_t i11 = (2 * I) * dl + 2 * K, i21 = (2 * I + 1) * dl + 2 * K;
    const double n11 = c2[i11], n12 = c2[i11 + 1], n21 = c2[i21], n22 = c2[i21 + 1];
    c1[i11] = sqrt(n11);
    c1[i11 + 1] = sqrt(n12);
    c1[i21] = sqrt(n21);
    c1[i21 + 1] = sqrt(n22);
    const double s = ((n11 + n12) + n21) + n22;
    p2[t] = s;
    p1[t] = sqrt(s);
  }
}

// Tiers kmax - 2 .. 0 in one CTA.
__global__ void __launch_bounds__(1024) k_pyramid_top(double *norm2, double *norm, int32_t kmax) {
  for (int l = kmax - 2; l >= 0; l--) {
    const int64_t d = int64_t(1) << l, dc = 2 * d;
    const double *c2 = norm2 + level_offset(l + 1);
    double *p2 = norm2 + level_offset(l);
    double *p1 = norm + level_offset(l);
    for (int64_t t = threadIdx.x; t < d * d; t += blockDim.x) {
      const int64_t I = t / d, K = t % d;
      const int64_t i11 = (2 * I) * dc + 2 * K, i21 = (2 * I + 1) * dc + 2 * K;
      const double s = ((c2[i11] + c2[i11 + 1]) + c2[i21]) + c2[i21 + 1];
      p2[t] = s;
      p1[t] = sqrt(s);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_to_dense(const T *tiles, const uint8_t *nz, int64_t n, int32_t b, int32_t nb,
                           int32_t NB, double *out) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / n, col = e % n;
    const int64_t r = row / b, c = col / b;
    double v = 0.0;
    if (nz[r * NB + c]) v = (double)tiles[((r * nb + c) * b + (row % b)) * b + (col % b)];
    out[e] = v;
  }
}

}  // namespace

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
  p.tf32 = (float *)t->copy[CK_TF32];
  p.tf32T = (float *)t->copy[CK_TF32_T];
  p.bf16 = (uint16_t *)t->copy[CK_BF16];
  p.bf16T = (uint16_t *)t->copy[CK_BF16_T];
  p.fp16 = (uint16_t *)t->copy[CK_FP16];
  p.fp16T = (uint16_t *)t->copy[CK_FP16_T];
  p.lo = (uint16_t *)t->copy[CK_BF16LO];
  p.loT = (uint16_t *)t->copy[CK_BF16LO_T];
  size_t sm = 0;
  const size_t bb = (size_t)t->b * t->b;
  if (p.tf32T) sm += bb * 4;
  if (p.bf16T) sm += bb * 2;
  if (p.fp16T) sm += bb * 2;
  if (p.loT) sm += bb * 2;
  const bool vec = (t->n % 2) == 0 && (((uintptr_t)A) % 16) == 0;
  const unsigned grid = (unsigned)((int64_t)t->NB * t->NB);
  cudaError_t e;
  if (vec) {
    if (sm > 48 * 1024) {
      e = cudaFuncSetAttribute(k_tree_build<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_tree_build<true><<<grid, 256, sm, s>>>(p);
  } else {
    if (sm > 48 * 1024) {
      e = cudaFuncSetAttribute(k_tree_build<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_tree_build<false><<<grid, 256, sm, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_pyramid(spamm_tree t, cudaStream_t s) {
  const int64_t dp = t->kmax > 0 ? (int64_t(1) << (t->kmax - 1)) : 1;
  const int64_t work = dp * dp;
  const unsigned grid = (unsigned)std::min<int64_t>((work + 255) / 256, 4096);
  k_pyramid_low<<<grid, 256, 0, s>>>(t->norm2, t->norm, t->kmax);
  if (t->kmax >= 2) k_pyramid_top<<<1, 1024, 0, s>>>(t->norm2, t->norm, t->kmax);
  return cudaGetLastError();
}

cudaError_t launch_to_dense(spamm_tree t, double *out, cudaStream_t s) {
  const int64_t total = t->n * t->n;
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 64);
  if (t->copy[CK_F64]) {
    k_to_dense<double><<<grid, 256, 0, s>>>((const double *)t->copy[CK_F64], t->nz, t->n, t->b,
                                            t->nb, t->NB, out);
  } else if (t->copy[CK_F32]) {
    k_to_dense<float><<<grid, 256, 0, s>>>((const float *)t->copy[CK_F32], t->nz, t->n, t->b,
                                           t->nb, t->NB, out);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---- leaf copies of a product tree, from its master tiles (FP64 or FP32) ----
namespace {

struct ConvertArgs {
  const void *src;
  int src_f64;
  const uint8_t *nz;
  int32_t b, nb, NB;
  float *tf32, *tf32T;
  uint16_t *bf16, *bf16T, *fp16, *fp16T, *lo, *loT;
};

__global__ void __launch_bounds__(256) k_tile_convert(ConvertArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t b = p.b;
  const int64_t leaf = blockIdx.x;
  const int32_t r = (int32_t)(leaf / p.nb), c = (int32_t)(leaf % p.nb);
  if (!p.nz[(int64_t)r * p.NB + c]) return;   // never read: zero blocks load as zero fill
  const int64_t tile = leaf * (int64_t)b * b;
  float *s_tf32T = nullptr;
  uint16_t *s_bf16T = nullptr, *s_fp16T = nullptr, *s_loT = nullptr;
  {
    unsigned char *q = smem;
    if (p.tf32T) { s_tf32T = (float *)q; q += (size_t)b * b * 4; }
    if (p.bf16T) { s_bf16T = (uint16_t *)q; q += (size_t)b * b * 2; }
    if (p.fp16T) { s_fp16T = (uint16_t *)q; q += (size_t)b * b * 2; }
    if (p.loT) { s_loT = (uint16_t *)q; q += (size_t)b * b * 2; }
  }
  const int32_t bb = b * b;
  for (int32_t e = threadIdx.x; e < bb; e += blockDim.x) {
    const int32_t row = e / b, col = e % b;
    const double v = p.src_f64 ? ((const double *)p.src)[tile + e] : (double)((const float *)p.src)[tile + e];
    if (p.tf32 || s_tf32T) {
      const float t = f64_to_tf32(v);
      if (p.tf32) p.tf32[tile + e] = t;
      if (s_tf32T) s_tf32T[col * b + row] = t;
    }
    if (p.bf16 || s_bf16T || p.lo || s_loT) {
      const uint16_t h = f64_to_bf16_bits(v);
      if (p.bf16) p.bf16[tile + e] = h;
      if (s_bf16T) s_bf16T[col * b + row] = h;
      if (p.lo || s_loT) {
        const uint16_t l = f64_to_bf16_bits(v - bf16_bits_to_f64(h));
        if (p.lo) p.lo[tile + e] = l;
        if (s_loT) s_loT[col * b + row] = l;
      }
    }
    if (p.fp16 || s_fp16T) {
      const uint16_t h = f64_to_fp16_bits(v);
      if (p.fp16) p.fp16[tile + e] = h;
      if (s_fp16T) s_fp16T[col * b + row] = h;
    }
  }
  __syncthreads();
  for (int32_t e = threadIdx.x; e < bb; e += blockDim.x) {
    if (s_tf32T) p.tf32T[tile + e] = s_tf32T[e];
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
  p.bf16 = (uint16_t *)t->copy[CK_BF16];
  p.bf16T = (uint16_t *)t->copy[CK_BF16_T];
  p.fp16 = (uint16_t *)t->copy[CK_FP16];
  p.fp16T = (uint16_t *)t->copy[CK_FP16_T];
  p.lo = (uint16_t *)t->copy[CK_BF16LO];
  p.loT = (uint16_t *)t->copy[CK_BF16LO_T];
  if (!p.tf32 && !p.tf32T && !p.bf16 && !p.bf16T && !p.fp16 && !p.fp16T && !p.lo && !p.loT)
    return cudaSuccess;
  size_t sm = 0;
  const size_t bb = (size_t)t->b * t->b;
  if (p.tf32T) sm += bb * 4;
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
