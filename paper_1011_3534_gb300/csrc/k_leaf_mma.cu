// Tensor-core leaf products for small leaves (b = 16, 32), the k = k_max case of Eq. 4,
// with warp-level mma.sync (m16n8k16 for BF16 and FP16, m16n8k8 for TF32).
//
// A b x b leaf is below the tcgen05 MMA shape (M = 128), so each output block is the
// work of one warp: work item = one output leaf block (i, j) = (2I + a, 2J + c) of a
// tier kmax-1 group (I, J); its surviving k are 2K + e for the group's K ascending and e
// ascending where mask bit ((a*2 + c)*2 + e) is set. A persistent grid of 4-warp CTAs
// takes items from a counter. Per k the warp stages A_ik (rows) and the right operand's
// leaf in N x K orientation (B_kj^T: the row copy of a symmetric tree, the transposed
// copy otherwise) in its own padded shared-memory tiles, forms the fragments with plain
// shared loads and issues the MMAs with a zero accumulator input; every MMA result is
// added to the block's FP32 sum in registers with round to nearest, in k order (split
// forms: hi lo + lo hi first, then hi hi, per K-step). No atomics; C is FP32 with its
// squared Frobenius norm (FP64, fixed-order reduction) and presence byte.
#include "internal.cuh"
#include "sync.cuh"

namespace {


struct MmaArgs {
  const void *A, *Alo;          // left operand rows (hi, lo of a split)
  const void *B, *Blo;          // right operand leaves in N x K orientation
  const uint8_t *nzA, *nzB;
  int32_t bsym;                 // right operand symmetric: leaf (k, j) read as (j, k)
  float *C;
  uint8_t *nzC;
  double *leaf_norm2C;
  const uint32_t *gij, *gstart, *glen;
  const uint16_t *K;
  const uint8_t *mask;
  const unsigned long long *ngroups;
  int64_t cap_entries, cap_groups;
  int32_t nb, NB;
  unsigned int *work_ctr;
  unsigned long long *mma_count;   // MMA instructions issued
  uint32_t *status;
};

// Element type of a format: 16-bit patterns (BF16, FP16) or 32-bit TF32 in FP32 storage.
template <int FMT>
struct Fmt {
  static constexpr int bytes = FMT == 2 ? 4 : 2;
  static constexpr int kstep = FMT == 2 ? 8 : 16;   // K of one MMA instruction
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %10, %10, %10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f));
}

__device__ __forceinline__ void mma_fp16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %10, %10, %10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f));
}

__device__ __forceinline__ void mma_tf32x(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %10, %10, %10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f));
}

template <int FMT>
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  if (FMT == 0) mma_bf16(d, a, b);
  else if (FMT == 1) mma_fp16(d, a, b);
  else mma_tf32x(d, a, b);
}

// Shared-memory tile of one leaf: b rows of b elements, rows padded so that the
// fragment loads of a warp (8 rows x 4 words) fall in distinct banks.
template <int B, int FMT>
struct Tile {
  static constexpr int row_words = B * Fmt<FMT>::bytes / 4 + 4;
  static constexpr int words = B * row_words;
};

// Copy one leaf (b x b contiguous elements at src) into a padded tile, 16-byte loads.
template <int B, int FMT>
__device__ __forceinline__ void stage(uint32_t *dst, const void *src, int lane) {
  constexpr int rw = B * Fmt<FMT>::bytes / 4;          // words of one leaf row
  constexpr int vecs = B * rw / 4;                     // 16-byte vectors of the leaf
  const uint4 *s = reinterpret_cast<const uint4 *>(src);
#pragma unroll
  for (int v = lane; v < vecs; v += 32) {
    const uint4 x = __ldg(s + v);
    const int r = (4 * v) / rw, c = (4 * v) % rw;
    *reinterpret_cast<uint4 *>(dst + r * Tile<B, FMT>::row_words + c) = x;   // rows 16-byte aligned
  }
}

// Warps of a CTA: four, or three where four warps' tiles would not fit in shared memory
// (leaf 64 split TF32: 4 tiles of 17 KB per warp).
template <int B, int FMT, bool SPLIT>
struct Cta {
  static constexpr size_t warp_bytes = (size_t)(SPLIT ? 4 : 2) * Tile<B, FMT>::words * 4;
  static constexpr int warps = 4 * warp_bytes <= 200 * 1024 ? 4 : 3;
  static_assert(warps * warp_bytes <= 227 * 1024, "leaf tiles exceed shared memory");
};

template <int B, int FMT, bool SPLIT>
__global__ void __launch_bounds__(Cta<B, FMT, SPLIT>::warps * 32) k_leaf_mma(MmaArgs p) {
  using F = Fmt<FMT>;
  using TL = Tile<B, FMT>;
  constexpr int RW = TL::row_words;
  constexpr int MT = B / 16, NT = B / 8, KS = B / F::kstep;
  constexpr int NTILES = SPLIT ? 4 : 2;            // A hi, B hi (, A lo, B lo)
  extern __shared__ __align__(16) uint32_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tig = lane & 3;
  uint32_t *tA = smem + (size_t)warp * NTILES * TL::words, *tB = tA + TL::words;
  uint32_t *tAl = tB + TL::words, *tBl = tAl + TL::words;   // split forms only
  const unsigned long long ngroups = *p.ngroups;
  const unsigned long long nitems = 4ull * (ngroups < (unsigned long long)p.cap_groups ? ngroups : p.cap_groups);
  const size_t bytes = (size_t)B * B * F::bytes;   // one leaf
  auto leaf = [&](const void *base, int64_t idx) {
    return reinterpret_cast<const unsigned char *>(base) + (size_t)idx * bytes;
  };

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(p.work_ctr, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const unsigned long long gq = item >> 2;
    const int q = (int)(item & 3);
    const uint32_t ij = p.gij[gq];
    const int32_t i = 2 * (int32_t)(ij >> 16) + (q >> 1);
    const int32_t j = 2 * (int32_t)(ij & 0xFFFFu) + (q & 1);
    if (i >= p.nb || j >= p.nb) continue;        // padding block: never stored
    const uint32_t start = p.gstart[gq];
    uint32_t len = p.glen[gq];
    if ((int64_t)start + len > p.cap_entries) {
      if (lane == 0) flag_error(p.status, DEV_BADARG);
      len = 0;
    }
    float run[MT][NT][4];
#pragma unroll
    for (int m = 0; m < MT; m++)
#pragma unroll
      for (int n = 0; n < NT; n++)
#pragma unroll
        for (int x = 0; x < 4; x++) run[m][n][x] = 0.f;
    bool any = false;
    unsigned long long nmma = 0;
    for (uint32_t e0 = 0; e0 < len; e0++) {
      const uint32_t bits = (p.mask[start + e0] >> (2 * q)) & 3u;
      if (!bits) continue;
      const int32_t K2 = 2 * (int32_t)p.K[start + e0];
      for (int e = 0; e < 2; e++) {
        if (!((bits >> e) & 1u)) continue;
        const int32_t k = K2 + e;
        if (k >= p.nb || !p.nzA[(int64_t)i * p.NB + k] || !p.nzB[(int64_t)k * p.NB + j]) continue;
        any = true;
        const int64_t ia = (int64_t)i * p.nb + k;
        const int64_t ib = p.bsym ? (int64_t)j * p.nb + k : (int64_t)k * p.nb + j;
        __syncwarp();   // the previous k's fragment loads are done
        stage<B, FMT>(tA, leaf(p.A, ia), lane);
        stage<B, FMT>(tB, leaf(p.B, ib), lane);
        if (SPLIT) {
          stage<B, FMT>(tAl, leaf(p.Alo, ia), lane);
          stage<B, FMT>(tBl, leaf(p.Blo, ib), lane);
        }
        __syncwarp();
        // (leaf 64: one K-step at a time keeps its 128 sums and one step's fragments in
        // registers)
#pragma unroll(B <= 32 ? KS : 1)
        for (int ks = 0; ks < KS; ks++) {
          // word offset of the K-step inside a row
          constexpr int kw = F::kstep * F::bytes / 4;
          uint32_t a[MT][4], al[MT][4], bh[NT][2], bl[NT][2];
#pragma unroll
          for (int m = 0; m < MT; m++) {
            const uint32_t *r0 = tA + (m * 16 + g) * RW + ks * kw, *r8 = r0 + 8 * RW;
            const uint32_t *s0 = tAl + (m * 16 + g) * RW + ks * kw, *s8 = s0 + 8 * RW;
            // BF16/FP16: 2 elements per word, columns 2 tig (+8); TF32: columns tig (+4);
            // either way words tig and tig + 4 of the K-step
            constexpr int c1 = 4;
            a[m][0] = r0[tig];
            a[m][1] = r8[tig];
            a[m][2] = r0[tig + c1];
            a[m][3] = r8[tig + c1];
            if (SPLIT) {
              al[m][0] = s0[tig];
              al[m][1] = s8[tig];
              al[m][2] = s0[tig + c1];
              al[m][3] = s8[tig + c1];
            }
          }
#pragma unroll
          for (int n = 0; n < NT; n++) {
            const uint32_t *r = tB + (n * 8 + g) * RW + ks * kw, *s = tBl + (n * 8 + g) * RW + ks * kw;
            bh[n][0] = r[tig];
            bh[n][1] = r[tig + 4];
            if (SPLIT) {
              bl[n][0] = s[tig];
              bl[n][1] = s[tig + 4];
            }
          }
#pragma unroll
          for (int m = 0; m < MT; m++)
#pragma unroll
            for (int n = 0; n < NT; n++) {
              float d[4];
              mma<FMT>(d, a[m], bh[n]);
              if (SPLIT) {
                float d1[4], d2[4];
                mma<FMT>(d1, a[m], bl[n]);
                mma<FMT>(d2, al[m], bh[n]);
#pragma unroll
                for (int x = 0; x < 4; x++) run[m][n][x] += d[x] + (d1[x] + d2[x]);
              } else {
#pragma unroll
                for (int x = 0; x < 4; x++) run[m][n][x] += d[x];
              }
            }
        }
        nmma += (unsigned long long)MT * NT * KS * (SPLIT ? 3 : 1);
      }
    }
    if (!any) continue;     // empty block: nz stays 0 and its norm 0
    float *Ct = p.C + ((int64_t)i * p.nb + j) * B * B;
    double ss = 0.0;
#pragma unroll
    for (int m = 0; m < MT; m++)
#pragma unroll
      for (int n = 0; n < NT; n++) {
        const int r = m * 16 + g, c = n * 8 + 2 * tig;
        *reinterpret_cast<float2 *>(Ct + (int64_t)r * B + c) = make_float2(run[m][n][0], run[m][n][1]);
        *reinterpret_cast<float2 *>(Ct + (int64_t)(r + 8) * B + c) = make_float2(run[m][n][2], run[m][n][3]);
#pragma unroll
        for (int x = 0; x < 4; x++) ss = fma((double)run[m][n][x], (double)run[m][n][x], ss);
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    if (lane == 0) {
      p.leaf_norm2C[(int64_t)i * p.NB + j] = ss;
      p.nzC[(int64_t)i * p.NB + j] = 1;
      atomicAdd(p.mma_count, nmma);
    }
  }
}

template <int B, int FMT, bool SPLIT>
cudaError_t run_mma(const MmaArgs &a, int sm_count, cudaStream_t s) {
  constexpr int warps = Cta<B, FMT, SPLIT>::warps;
  const size_t sm = (size_t)warps * Cta<B, FMT, SPLIT>::warp_bytes;
  auto k = k_leaf_mma<B, FMT, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, warps * 32, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  k<<<(unsigned)(sm_count * occ), warps * 32, sm, s>>>(a);
  return cudaGetLastError();
}

template <int B>
cudaError_t run_leaf(const MmaArgs &a, int prec, int sm_count, cudaStream_t s) {
  switch (prec) {
    case SPAMM_BF16: return run_mma<B, 0, false>(a, sm_count, s);
    case SPAMM_FP16: return run_mma<B, 1, false>(a, sm_count, s);
    case SPAMM_TF32: return run_mma<B, 2, false>(a, sm_count, s);
    case SPAMM_BF16X3: return run_mma<B, 0, true>(a, sm_count, s);
    case SPAMM_TF32X3: return run_mma<B, 2, true>(a, sm_count, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_leaf_mma(spamm_tree A, spamm_tree B, spamm_tree C, int prec, uint32_t *dev_status,
                            int sm_count, cudaStream_t s) {
  const bool tf32 = tf32_prec(prec);
  const int row = tf32 ? CK_TF32 : prec == SPAMM_FP16 ? CK_FP16 : CK_BF16;
  const bool bsym = (B->flags & SPAMM_SYMMETRIC) != 0;
  const int lo = tf32 ? CK_TF32LO : CK_BF16LO;
  const TierList &par = C->tiers[C->kmax];
  MmaArgs a{};
  a.A = A->copy[row];
  a.B = B->copy[bsym ? row : row + 1];
  a.Alo = split_prec(prec) ? A->copy[lo] : nullptr;
  a.Blo = split_prec(prec) ? B->copy[bsym ? lo : lo + 1] : nullptr;
  if (!a.A || !a.B || (split_prec(prec) && (!a.Alo || !a.Blo))) return cudaErrorInvalidValue;
  a.nzA = A->nz;
  a.nzB = B->nz;
  a.bsym = bsym ? 1 : 0;
  a.C = (float *)C->copy[CK_F32];
  a.nzC = C->nz;
  a.leaf_norm2C = C->norm2 + level_offset(C->kmax);
  a.gij = par.gij;
  a.gstart = par.gstart;
  a.glen = par.glen;
  a.K = par.K;
  a.mask = C->mask;
  a.ngroups = &C->counts->ngroups[C->kmax];
  a.cap_entries = par.cap_entries;
  a.cap_groups = par.cap_groups;
  a.nb = C->nb;
  a.NB = C->NB;
  a.work_ctr = &C->counts->work_ctr;
  a.mma_count = &C->counts->mma_small;
  a.status = dev_status;
  switch (C->b) {
    case 16: return run_leaf<16>(a, prec, sm_count, s);
    case 32: return run_leaf<32>(a, prec, sm_count, s);
    case 64: return run_leaf<64>(a, prec, sm_count, s);   // the warp-tile shape of leaf 64
    default: return cudaErrorInvalidValue;
  }
}
