// spamm_cull_noalloc: the tier-by-tier cull for callers that cannot allocate device
// memory. Its working memory is one file-scope device array; the paper has no
// counterpart to this entry point.
#include <cmath>
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kMaxKmax = 7;                       // NB <= 128 leaf blocks per side
constexpr size_t kScratchBytes = size_t(2) << 20; // 2 MiB, held by every GPU that loads the library

// Working memory of every spamm_cull_noalloc call on a device: norm pyramids, tier
// lists, look-back words, counters. Calls share it; see spamm.h.
static __device__ __align__(256) unsigned char g_cull_scratch[kScratchBytes];

// Device address of g_cull_scratch per device, looked up once with that device current.
std::mutex g_lock;
void *g_addr[64] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carve {
  unsigned char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    T *p = reinterpret_cast<T *>(base + off);
    off = align256(off + count * sizeof(T));
    return p;
  }
};

// Byte size of the scratch layout for a given kmax (also used to check the maximum).
size_t layout(int kmax, unsigned char *base, spamm_tree_s *A, spamm_tree_s *B, spamm_tree_s *C,
              uint32_t **status, uint32_t **tile_sums, int64_t *offsets) {
  Carve cv{base};
  const size_t levels = (size_t)level_offset(kmax + 1);
  A->norm2 = cv.take<double>(levels);
  A->norm = cv.take<double>(levels);
  B->norm2 = cv.take<double>(levels);
  B->norm = cv.take<double>(levels);
  for (int li = 0; li <= kmax; li++) {
    TierList &T = C->tiers[li];
    const int l = li - 1;
    T.cap_groups = l < 0 ? 1 : (int64_t(1) << (2 * l));
    T.cap_entries = l < 0 ? 1 : (int64_t(1) << (3 * l));
    T.gij = cv.take<uint32_t>(T.cap_groups);
    T.gstart = cv.take<uint32_t>(T.cap_groups);
    T.glen = cv.take<uint32_t>(T.cap_groups);
    T.K = cv.take<uint16_t>(T.cap_entries);
  }
  C->cap_mask = C->tiers[kmax].cap_entries;
  C->mask = cv.take<uint8_t>(C->cap_mask);
  C->cap_look = cull_look_words(kmax);
  C->look = cv.take<uint64_t>(C->cap_look);
  C->cap_bound = cull_bound_words(kmax, offsets);
  C->bound_part = cv.take<double>(C->cap_bound + kmax + 1);
  C->counts = cv.take<DevCounts>(1);
  *status = cv.take<uint32_t>(1);
  *tile_sums = cv.take<uint32_t>(256);   // the expansion's per-tile survivor counts
  return cv.off;
}

// The surviving leaf triples from the tier kmax-1 masks, in two launches over tiles of
// kExpandTile entries (at most 256 tiles): each tile's survivor count, then each tile
// writes its triples after those of the tiles before it. Order: groups in list order
// (Morton order of the output blocks), entries in K order, mask bits in bit order.
constexpr int kExpandTile = 1024;
constexpr int kMaxTiles = 256;   // 8^(kMaxKmax - 1) entries / kExpandTile

__device__ __forceinline__ unsigned int block_sum(unsigned int v, unsigned int *s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  unsigned int t = 0;
  if (warp == 0) t = __reduce_add_sync(0xffffffffu, lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u);
  __syncthreads();
  return t;   // valid in warp 0
}

__global__ void __launch_bounds__(kExpandTile) k_expand_count(const uint8_t *mask, const DevCounts *cnt, int list,
                                                              uint32_t *tile_sums) {
  __shared__ unsigned int s_warp[32];
  const unsigned long long ne = cnt->nentries[list];
  const unsigned long long e = (unsigned long long)blockIdx.x * kExpandTile + threadIdx.x;
  if ((unsigned long long)blockIdx.x * kExpandTile >= ne) return;   // the whole CTA
  const unsigned int t = block_sum(e < ne ? (unsigned int)__popc(mask[e]) : 0u, s_warp);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kExpandTile) k_expand_write(const uint32_t *gij, const uint32_t *gstart,
                                                              const uint16_t *K, const uint8_t *mask,
                                                              const DevCounts *cnt, int list,
                                                              const uint32_t *tile_sums, uint32_t *out,
                                                              int64_t cap, int64_t *count, const uint32_t *status) {
  __shared__ unsigned int s_warp[32];
  __shared__ unsigned long long s_before;
  const unsigned long long ng = cnt->ngroups[list], ne = cnt->nentries[list];
  const unsigned long long ntiles = (ne + kExpandTile - 1) / kExpandTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (blockIdx.x == 0) {   // the count: every tile's survivors
    const unsigned int t = block_sum(threadIdx.x < ntiles ? tile_sums[threadIdx.x] : 0u, s_warp);
    if (threadIdx.x == 0) *count = *status ? -1 : (int64_t)t;
  }
  if (blockIdx.x >= ntiles) return;
  // survivors of the tiles before this one
  const unsigned int before = block_sum(threadIdx.x < blockIdx.x ? tile_sums[threadIdx.x] : 0u, s_warp);
  if (threadIdx.x == 0) s_before = before;
  __syncthreads();
  const unsigned long long e = (unsigned long long)blockIdx.x * kExpandTile + threadIdx.x;
  const uint32_t bits = e < ne ? mask[e] : 0u;
  const unsigned int c = __popc(bits);
  unsigned int inc = c;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned int w = s_warp[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    s_warp[lane] = w;   // inclusive warp totals
  }
  __syncthreads();
  if (!c) return;
  const unsigned long long pos = s_before + (warp ? s_warp[warp - 1] : 0u) + inc - c;
  // group holding entry e: last group whose start is <= e
  unsigned long long lo = 0, hi = ng;
  while (hi - lo > 1) {
    const unsigned long long mid = (lo + hi) / 2;
    if (gstart[mid] <= e) lo = mid; else hi = mid;
  }
  const uint32_t I = gij[lo] >> 16, J = gij[lo] & 0xFFFFu, k = K[e];
  unsigned long long p = pos;
  for (int q = 0; q < 8; q++)
    if ((bits >> q) & 1u) {
      if ((int64_t)p < cap) {
        out[3 * p] = 2 * I + ((q >> 2) & 1);
        out[3 * p + 1] = 2 * J + ((q >> 1) & 1);
        out[3 * p + 2] = 2 * k + (q & 1);
      }
      p++;
    }
}

}  // namespace

static_assert(kMaxKmax <= 8, "scratch layout sized for NB <= 128");
static_assert((int64_t(1) << (3 * (kMaxKmax - 1))) <= (int64_t)kMaxTiles * kExpandTile, "expansion tiles");

extern "C" SPAMM_API spamm_status spamm_cull_noalloc(const double *normA2, const double *normB2,
                                                     int32_t nb_padded, double tau, uint32_t *triples,
                                                     int64_t cap, int64_t *count, void *cuda_stream) {
  if (!normA2 || !normB2 || !count || (cap > 0 && !triples) || cap < 0) return SPAMM_EINVAL;
  if (!(tau >= 0.0) || !std::isfinite(tau)) return SPAMM_EINVAL;
  if (nb_padded < 1 || (nb_padded & (nb_padded - 1))) return SPAMM_EINVAL;
  int kmax = 0;
  while ((1 << kmax) < nb_padded) kmax++;
  if (kmax > kMaxKmax) return SPAMM_ERANGE;   // more than 128 leaf blocks per side
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPAMM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPAMM_ECUDA;
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_cull_scratch) != cudaSuccess || !p) return SPAMM_ECUDA;
      g_addr[dev] = p;
    }
    scratch = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  spamm_tree_s A, B, C;
  uint32_t *status = nullptr, *tile_sums = nullptr;
  int64_t offsets[kMaxKmax + 1];
  const size_t used = layout(kmax, (unsigned char *)scratch, &A, &B, &C, &status, &tile_sums, offsets);
  if (used > kScratchBytes) return SPAMM_ERANGE;
  for (spamm_tree_s *t : {&A, &B, &C}) {
    t->NB = nb_padded;
    t->nb = nb_padded;
    t->kmax = kmax;
    t->b = 1;
    t->n = nb_padded;
  }
  const size_t leaf_bytes = (size_t)nb_padded * nb_padded * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(A.norm2 + level_offset(kmax), normA2, leaf_bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B.norm2 + level_offset(kmax), normB2, leaf_bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(C.counts, 0, sizeof(DevCounts), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(C.look, 0, (size_t)C.cap_look * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, s);
  if (e == cudaSuccess) e = launch_pyramid(&A, s);
  if (e == cudaSuccess) e = launch_pyramid(&B, s);
  int launches = 0;
  if (e == cudaSuccess) e = launch_cull(&A, &B, &C, tau, nullptr, status, sms, s, &launches);
  if (e == cudaSuccess) {
    // tiles cover the list's capacity; tiles past the surviving entries return at once
    const unsigned tiles =
        (unsigned)std::max<int64_t>(1, (C.tiers[kmax].cap_entries + kExpandTile - 1) / kExpandTile);
    k_expand_count<<<tiles, kExpandTile, 0, s>>>(C.mask, C.counts, kmax, tile_sums);
    k_expand_write<<<tiles, kExpandTile, 0, s>>>(C.tiers[kmax].gij, C.tiers[kmax].gstart, C.tiers[kmax].K, C.mask,
                                                 C.counts, kmax, tile_sums, triples, cap, count, status);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}
