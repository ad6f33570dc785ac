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

// Leaf-block kernel (K1). Each leaf is split into groups of 8 consecutive elements of
// one row; a leaf is handled by TPL threads (several leaves per CTA for small leaves),
// each thread loading its groups as 64-byte runs (four 16-byte loads, coalesced along
// rows). The FP64 pipe is kept idle: the squared Frobenius norm is accumulated from an
// exact FP32 hi/lo split of each element, scaled by the leaf's largest exponent, with
// error-free (TwoSum) accumulation and a double-float reduction (relative error ~2^-46, far
// inside the 1e-12 near-tau band), and the leaf copies are rounded in integer
// arithmetic from the FP64 bit pattern.
template <int B>
struct BuildCfg {
  static constexpr int T = B == 128 ? 1024 : 256;   // threads per CTA
  static constexpr int GROUPS = B * B / 8;           // 8-element groups per leaf
  static constexpr int TPL = GROUPS < T ? GROUPS : T;
  static constexpr int LPC = T / TPL;                // leaves per CTA
  static constexpr int ROUNDS = GROUPS / TPL;
  static constexpr int EPT = ROUNDS * 8;             // elements per thread
};

__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  float err = (h - (s - bb)) + (bh - bb);
  err += l + bl;
  h = s + err;
  l = err - (h - s);
}

template <int B, bool VEC>
__global__ void __launch_bounds__(BuildCfg<B>::T) k_tree_build(BuildArgs p) {
  using Cfg = BuildCfg<B>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_emax[Cfg::T / 32];
  __shared__ float s_h[Cfg::T / 32], s_l[Cfg::T / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = threadIdx.x / Cfg::TPL, tl = threadIdx.x % Cfg::TPL;
  const int64_t leaf = (int64_t)blockIdx.x * Cfg::LPC + li;
  const bool inrange = leaf < (int64_t)p.NB * p.NB;
  const int32_t r = inrange ? (int32_t)(leaf / p.NB) : 0, c = inrange ? (int32_t)(leaf % p.NB) : 0;
  const bool stored = inrange && r < p.nb && c < p.nb;

  uint64_t v[Cfg::EPT];
  int emax = 0;
#pragma unroll
  for (int j = 0; j < Cfg::ROUNDS; j++) {
    const int g = tl + Cfg::TPL * j;
    const int row = (8 * g) / B, col0 = (8 * g) % B;
    const int64_t gr = (int64_t)r * B + row, gc = (int64_t)c * B + col0;
    if (stored && gr < p.n) {
      const double *src = p.A + gr * p.n + gc;
      if (VEC && gc + 8 <= p.n) {
#pragma unroll
        for (int h = 0; h < 4; h++) {
          const double2 d = __ldcs(reinterpret_cast<const double2 *>(src) + h);
          v[8 * j + 2 * h] = (uint64_t)__double_as_longlong(d.x);
          v[8 * j + 2 * h + 1] = (uint64_t)__double_as_longlong(d.y);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; e++)
          v[8 * j + e] = gc + e < p.n ? (uint64_t)__double_as_longlong(__ldcs(src + e)) : 0ull;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; e++) v[8 * j + e] = 0ull;
    }
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int E = (int)((v[8 * j + e] >> 52) & 0x7FF);
      emax = E > emax ? E : emax;
    }
  }
  // largest exponent field of the leaf (its threads span whole warps)
  emax = __reduce_max_sync(0xffffffffu, emax);
  if (lane == 0) s_emax[warp] = emax;
  __syncthreads();
  constexpr int WPL = Cfg::TPL / 32;   // warps per leaf
  int Emax = 0;
#pragma unroll
  for (int w = 0; w < WPL; w++) Emax = max(Emax, s_emax[li * WPL + w]);

  // squared norm of the leaf scaled by 2^(-2 (Emax - 1023))
  float S = 0.f, s2 = 0.f;
  if (Emax > 0 && Emax < 0x7FF) {
#pragma unroll
    for (int e = 0; e < Cfg::EPT; e++) {
      const uint64_t bits = v[e];
      const int E = (int)((bits >> 52) & 0x7FF);
      const int es = E - Emax;
      if (E == 0 || es < -100) continue;   // below 2^-200 of the largest square: negligible
      const float hi = __uint_as_float(((uint32_t)(es + 127) << 23) | (uint32_t)((bits >> 29) & 0x7FFFFFu));
      const float lo = es >= -74 ? __uint2float_rn((uint32_t)(bits & 0x1FFFFFFFu)) *
                                       __uint_as_float((uint32_t)(es - 52 + 127) << 23)
                                 : 0.f;
      const float pp = hi * hi;
      float cc = fmaf(hi, hi, -pp);
      cc = fmaf(2.f * hi, lo, cc);
      cc = fmaf(lo, lo, cc);
      // TwoSum (Knuth): S + pp = t + err exactly, whatever their magnitudes
      const float t = S + pp;
      const float bb = t - S;
      const float err = (S - (t - bb)) + (pp - bb);
      S = t;
      s2 += err + cc;
    }
  }
  float H = S, L = s2;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, H, off), l2 = __shfl_xor_sync(0xffffffffu, L, off);
    df_add(H, L, h2, l2);
  }
  if (lane == 0) {
    s_h[warp] = H;
    s_l[warp] = L;
  }
  __syncthreads();
  if (tl == 0 && inrange) {
    if (stored) {
      double acc = 0.0;
      for (int w = 0; w < WPL; w++) acc += (double)s_h[li * WPL + w] + (double)s_l[li * WPL + w];
      p.leaf_norm2[leaf] = (Emax > 0 && Emax < 0x7FF) ? ldexp(acc, 2 * (Emax - 1023))
                                                       : (Emax == 0x7FF ? __longlong_as_double(0x7FF0000000000000ll) : 0.0);
      p.nz[leaf] = 1;
    } else {
      p.leaf_norm2[leaf] = 0.0;
      p.nz[leaf] = 0;
    }
  }
  if (!stored && !(p.tf32T || p.bf16T || p.fp16T || p.loT)) return;

  // leaf copies
  const int64_t tile = ((int64_t)r * p.nb + c) * (int64_t)B * B;
  const size_t bb = (size_t)B * B;
  float *s_tf32T = nullptr;
  uint16_t *s_bf16T = nullptr, *s_fp16T = nullptr, *s_loT = nullptr;
  {
    unsigned char *q = smem;
    if (p.tf32T) { s_tf32T = (float *)q + li * bb; q += Cfg::LPC * bb * 4; }
    if (p.bf16T) { s_bf16T = (uint16_t *)q + li * bb; q += Cfg::LPC * bb * 2; }
    if (p.fp16T) { s_fp16T = (uint16_t *)q + li * bb; q += Cfg::LPC * bb * 2; }
    if (p.loT) { s_loT = (uint16_t *)q + li * bb; q += Cfg::LPC * bb * 2; }
  }
  if (stored) {
#pragma unroll
    for (int j = 0; j < Cfg::ROUNDS; j++) {
      const int g = tl + Cfg::TPL * j;
      const int row = (8 * g) / B, col0 = (8 * g) % B;
      const int64_t o = tile + (int64_t)row * B + col0;
      if (p.f64) {
#pragma unroll
        for (int h = 0; h < 4; h++)
          reinterpret_cast<double2 *>(p.f64 + o)[h] =
              make_double2(__longlong_as_double((long long)v[8 * j + 2 * h]),
                           __longlong_as_double((long long)v[8 * j + 2 * h + 1]));
      }
      if (p.bf16 || s_bf16T || p.lo || s_loT) {
        uint32_t hb[8], lb[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const Rounded h = round_f64bits(v[8 * j + e], 8, -126);
          hb[e] = h.bits;
          lb[e] = (p.lo || s_loT) ? bf16_lo_bits(v[8 * j + e], h) : 0u;
        }
        if (p.bf16) {
          uint4 w;
          w.x = (hb[0] >> 16) | (hb[1] & 0xFFFF0000u);
          w.y = (hb[2] >> 16) | (hb[3] & 0xFFFF0000u);
          w.z = (hb[4] >> 16) | (hb[5] & 0xFFFF0000u);
          w.w = (hb[6] >> 16) | (hb[7] & 0xFFFF0000u);
          *reinterpret_cast<uint4 *>(p.bf16 + o) = w;
        }
        if (p.lo) {
          uint4 w;
          w.x = (lb[0] >> 16) | (lb[1] & 0xFFFF0000u);
          w.y = (lb[2] >> 16) | (lb[3] & 0xFFFF0000u);
          w.z = (lb[4] >> 16) | (lb[5] & 0xFFFF0000u);
          w.w = (lb[6] >> 16) | (lb[7] & 0xFFFF0000u);
          *reinterpret_cast<uint4 *>(p.lo + o) = w;
        }
#pragma unroll
        for (int e = 0; e < 8; e++) {
          if (s_bf16T) s_bf16T[(col0 + e) * B + row] = bf16_from_f32bits(hb[e]);
          if (s_loT) s_loT[(col0 + e) * B + row] = bf16_from_f32bits(lb[e]);
        }
      }
      if (p.tf32 || s_tf32T) {
        uint32_t tb[8];
#pragma unroll
        for (int e = 0; e < 8; e++) tb[e] = round_f64bits(v[8 * j + e], 11, -126).bits;
        if (p.tf32) {
          reinterpret_cast<uint4 *>(p.tf32 + o)[0] = make_uint4(tb[0], tb[1], tb[2], tb[3]);
          reinterpret_cast<uint4 *>(p.tf32 + o)[1] = make_uint4(tb[4], tb[5], tb[6], tb[7]);
        }
        if (s_tf32T)
#pragma unroll
          for (int e = 0; e < 8; e++) s_tf32T[(col0 + e) * B + row] = __uint_as_float(tb[e]);
      }
      if (p.fp16 || s_fp16T) {
        uint16_t hh[8];
#pragma unroll
        for (int e = 0; e < 8; e++) hh[e] = fp16_from_f32bits(round_f64bits(v[8 * j + e], 11, -14).bits);
        if (p.fp16) {
          uint4 w;
          w.x = hh[0] | ((uint32_t)hh[1] << 16);
          w.y = hh[2] | ((uint32_t)hh[3] << 16);
          w.z = hh[4] | ((uint32_t)hh[5] << 16);
          w.w = hh[6] | ((uint32_t)hh[7] << 16);
          *reinterpret_cast<uint4 *>(p.fp16 + o) = w;
        }
        if (s_fp16T)
#pragma unroll
          for (int e = 0; e < 8; e++) s_fp16T[(col0 + e) * B + row] = hh[e];
      }
    }
  }
  if (!(p.tf32T || p.bf16T || p.fp16T || p.loT)) return;
  __syncthreads();
  if (!stored) return;
  // transposed copies: shared -> global, 16-byte vectors
  if (s_tf32T)
    for (int q = tl; q < (int)(bb / 4); q += Cfg::TPL)
      reinterpret_cast<float4 *>(p.tf32T + tile)[q] = reinterpret_cast<const float4 *>(s_tf32T)[q];
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

__global__ void __launch_bounds__(256) k_pyramid_region(double *norm2, double *norm, int32_t kmax) {
  __shared__ double s0[kPyrR * kPyrR], s1[kPyrR * kPyrR / 4];
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
}

// Tiers kmax - 5 .. 0 (above the regions) in one CTA.
__global__ void __launch_bounds__(1024) k_pyramid_top(double *norm2, double *norm, int32_t top_tier) {
  for (int l = top_tier; l >= 0; l--) {
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

template <int B>
static cudaError_t run_build(const BuildArgs &p, size_t bytes_per_leaf_T, bool vec, cudaStream_t s) {
  using Cfg = BuildCfg<B>;
  const size_t sm = bytes_per_leaf_T * Cfg::LPC;
  const int64_t leaves = (int64_t)p.NB * p.NB;
  const unsigned grid = (unsigned)((leaves + Cfg::LPC - 1) / Cfg::LPC);
  auto k = vec ? k_tree_build<B, true> : k_tree_build<B, false>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, Cfg::T, sm, s>>>(p);
  return cudaGetLastError();
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
  p.tf32 = (float *)t->copy[CK_TF32];
  p.tf32T = (float *)t->copy[CK_TF32_T];
  p.bf16 = (uint16_t *)t->copy[CK_BF16];
  p.bf16T = (uint16_t *)t->copy[CK_BF16_T];
  p.fp16 = (uint16_t *)t->copy[CK_FP16];
  p.fp16T = (uint16_t *)t->copy[CK_FP16_T];
  p.lo = (uint16_t *)t->copy[CK_BF16LO];
  p.loT = (uint16_t *)t->copy[CK_BF16LO_T];
  size_t per_leaf = 0;
  const size_t bb = (size_t)t->b * t->b;
  if (p.tf32T) per_leaf += bb * 4;
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
  k_pyramid_region<<<(unsigned)(per_side * per_side), 256, 0, s>>>(t->norm2, t->norm, t->kmax);
  const int top = t->kmax - kPyrL - 1;
  if (top >= 0) k_pyramid_top<<<1, 1024, 0, s>>>(t->norm2, t->norm, top);
  return cudaGetLastError();
}

// kernels launch_pyramid issues for a tree of this depth
int pyramid_launches(int kmax) { return 1 + (kmax - kPyrL - 1 >= 0 ? 1 : 0); }

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
    Rounded hb, tb, fb;
    uint32_t lb = 0;
    if (p.src_f64) {
      const uint64_t bits = (uint64_t)__double_as_longlong(((const double *)p.src)[tile + e]);
      hb = round_f64bits(bits, 8, -126);
      tb = round_f64bits(bits, 11, -126);
      fb = round_f64bits(bits, 11, -14);
      if (p.lo || s_loT) lb = bf16_lo_bits(bits, hb);
    } else {
      const float f = ((const float *)p.src)[tile + e];
      hb = round_f32(f, 8, -126);
      tb = round_f32(f, 11, -126);
      fb = round_f32(f, 11, -14);
      if (p.lo || s_loT) lb = bf16_lo_bits_f32(f, hb);
    }
    if (p.tf32) p.tf32[tile + e] = __uint_as_float(tb.bits);
    if (s_tf32T) s_tf32T[col * b + row] = __uint_as_float(tb.bits);
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
