// FP64 leaf products (the k = k_max case of Eq. 4) on CUDA cores, for every leaf size.
//
// Work item = one output leaf block (i, j) = (2I + a, 2J + c) of a tier kmax-1 group
// (I, J): its surviving k are 2K + e for the group's K ascending and e ascending where
// mask bit ((a*2 + c)*2 + e) is set, so C_ij is summed over k in ascending order by one
// CTA, with no atomics. Items are fetched dynamically by a persistent grid.
// Inside a leaf product the inner index is split into slices of KS staged in shared
// memory; each of 256 threads holds a (b/16) x (b/16) register tile of C_ij with rows
// ty + 16 r and columns tx + 16 q (conflict-free shared reads, coalesced stores).
// Epilogue: C_ij in FP64, its squared Frobenius norm (fixed-order reduction), nz = 1.
#include "internal.cuh"
#include "sync.cuh"

namespace {

struct LeafArgs {
  const double *A, *B;          // FP64 tiles
  const uint8_t *nzA, *nzB;
  double *C;
  uint8_t *nzC;
  double *leaf_norm2C;
  const uint32_t *gij, *gstart, *glen;
  const uint16_t *K;
  const uint8_t *mask;
  const unsigned long long *ngroups;
  int64_t cap_entries;
  int32_t b, nb, NB;
  unsigned int *work_ctr;
};

template <int B>
__global__ void __launch_bounds__(256) k_leaf_f64(LeafArgs p) {
  constexpr int KS = B <= 32 ? B : (B == 64 ? 32 : 16);   // inner slice (<= 48 KB smem)
  constexpr int T = B / 16;             // register tile side
  __shared__ __align__(16) double As[B][KS + 1];
  __shared__ __align__(16) double Bs[KS][B];
  __shared__ unsigned int s_item;
  __shared__ double s_red[8];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const unsigned long long nitems = 4ull * (*p.ngroups);
  const int64_t bb = (int64_t)B * B;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.work_ctr, 1u);
    __syncthreads();
    const unsigned long long item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    const unsigned long long g = item >> 2;
    const int q = (int)(item & 3);
    const uint32_t ij = p.gij[g];
    const int32_t i = 2 * (int32_t)(ij >> 16) + (q >> 1);
    const int32_t j = 2 * (int32_t)(ij & 0xFFFFu) + (q & 1);
    if (i >= p.nb || j >= p.nb) continue;        // padding block: never stored
    uint32_t start = p.gstart[g], len = p.glen[g];
    if ((int64_t)start + len > p.cap_entries) len = 0;
    double acc[T][T];
#pragma unroll
    for (int r = 0; r < T; r++)
#pragma unroll
      for (int c = 0; c < T; c++) acc[r][c] = 0.0;
    bool any = false;
    for (uint32_t e0 = 0; e0 < len; e0++) {
      const uint32_t bits = (p.mask[start + e0] >> (2 * q)) & 3u;
      if (!bits) continue;
      const int32_t K2 = 2 * (int32_t)p.K[start + e0];
      for (int e = 0; e < 2; e++) {
        if (!((bits >> e) & 1u)) continue;
        const int32_t k = K2 + e;
        if (k >= p.nb || !p.nzA[(int64_t)i * p.NB + k] || !p.nzB[(int64_t)k * p.NB + j]) continue;
        any = true;
        const double *At = p.A + ((int64_t)i * p.nb + k) * bb;
        const double *Bt = p.B + ((int64_t)k * p.nb + j) * bb;
        for (int s0 = 0; s0 < B; s0 += KS) {
          for (int x = tid; x < B * KS; x += 256) {
            const int r = x / KS, c = x % KS;
            As[r][c] = At[(int64_t)r * B + s0 + c];
          }
          for (int x = tid; x < KS * B; x += 256) {
            const int r = x / B, c = x % B;
            Bs[r][c] = Bt[(int64_t)(s0 + r) * B + c];
          }
          __syncthreads();
          {
#pragma unroll 4
            for (int l = 0; l < KS; l++) {
              double av[T], bv[T];
#pragma unroll
              for (int r = 0; r < T; r++) av[r] = As[ty + 16 * r][l];
#pragma unroll
              for (int c = 0; c < T; c++) bv[c] = Bs[l][tx + 16 * c];
#pragma unroll
              for (int r = 0; r < T; r++)
#pragma unroll
                for (int c = 0; c < T; c++) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
            }
          }
          __syncthreads();
        }
      }
    }
    if (!any) continue;     // empty block: nz stays 0 and its norm 0
    double ss = 0.0;
    double *Ct = p.C + ((int64_t)i * p.nb + j) * bb;
    {
#pragma unroll
      for (int r = 0; r < T; r++)
#pragma unroll
        for (int c = 0; c < T; c++) {
          Ct[(int64_t)(ty + 16 * r) * B + tx + 16 * c] = acc[r][c];
          ss = fma(acc[r][c], acc[r][c], ss);
        }
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) s_red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; w++) s += s_red[w];
      p.leaf_norm2C[(int64_t)i * p.NB + j] = s;
      p.nzC[(int64_t)i * p.NB + j] = 1;
    }
  }
}

template <int B>
cudaError_t run(const LeafArgs &a, int sm_count, cudaStream_t s) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_leaf_f64<B>, 256, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  k_leaf_f64<B><<<(unsigned)(sm_count * occ), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_f64(spamm_tree A, spamm_tree B, spamm_tree C, uint32_t *dev_status,
                            int sm_count, cudaStream_t s) {
  (void)dev_status;
  const TierList &par = C->tiers[C->kmax];
  LeafArgs a{};
  a.A = (const double *)A->copy[CK_F64];
  a.B = (const double *)B->copy[CK_F64];
  a.nzA = A->nz;
  a.nzB = B->nz;
  a.C = (double *)C->copy[CK_F64];
  a.nzC = C->nz;
  a.leaf_norm2C = C->norm2 + level_offset(C->kmax);
  a.gij = par.gij;
  a.gstart = par.gstart;
  a.glen = par.glen;
  a.K = par.K;
  a.mask = C->mask;
  a.ngroups = &C->counts->ngroups[C->kmax];
  a.cap_entries = par.cap_entries;
  a.b = C->b;
  a.nb = C->nb;
  a.NB = C->NB;
  a.work_ctr = &C->counts->work_ctr;
  switch (C->b) {
    case 16: return run<16>(a, sm_count, s);
    case 32: return run<32>(a, sm_count, s);
    case 64: return run<64>(a, sm_count, s);
    case 128: return run<128>(a, sm_count, s);
    default: return cudaErrorInvalidValue;
  }
}
