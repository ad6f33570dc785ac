// Tier-by-tier cull of the product space (Eq. 4), with the surviving triples kept
// grouped by output block.
//
// Tier l holds the triples (I, J, K), I, J, K < 2^l, whose test
// ||A^l_IK||_F ||B^l_KJ||_F >= tau passed and whose ancestors all passed: exactly the
// calls of the Eq. 4 recursion that neither return 0 nor reach the leaves. A tier
// list is a sequence of groups, one per output block (I, J), each with its K in
// ascending order; groups follow the Morton order of (I, J).
//
// One launch expands tier l-1 into tier l: every parent entry (I, J, K) proposes the
// eight children (2I+a, 2J+c, 2K+e) and tests them with the tier-l norms. The children
// of parent group (I, J) form the four child groups (2I+a, 2J+c), each listing 2K+e
// for K ascending, then e ascending, so the new lists are again sorted by K. A warp
// handles one parent group; a CTA handles a tile of 8 parent groups, fetched
// dynamically, and places its 32 child groups after those of all earlier tiles with
// a decoupled look-back scan (Merrill and Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", NVIDIA tech report NVR-2016-002). The last tier
// (l = kmax) is not materialised: each entry of tier kmax-1 gets an 8-bit mask of its
// surviving leaf children instead, bit ((a*2 + c)*2 + e).
//
// Counters: tests, culls and the sum of culled norm products per tier. Integer
// counters use atomics (exact); the FP64 sums are written per parent group and summed
// in a fixed order afterwards, so they are reproducible run to run.
#include <cmath>

#include "internal.cuh"
#include "sync.cuh"

namespace {

constexpr int kWarps = 8;
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62, kFlagMask = 3ull << 62;
constexpr uint64_t kEntMask = (1ull << 31) - 1;

__device__ __forceinline__ uint64_t pack(uint64_t flag, uint64_t groups, uint64_t entries) {
  return flag | ((groups & ((1ull << 31) - 1)) << 31) | (entries & kEntMask);
}

// Decoupled look-back of one tile (called by a whole warp): publishes this tile's
// aggregates (entries, groups) and returns the exclusive prefix of all earlier tiles.
// Waits on predecessors are bounded; a wait that runs out flags DEV_TIMEOUT.
__device__ void tile_lookback(uint64_t *look, unsigned int tile, uint64_t agg_e, uint64_t agg_g,
                              uint64_t &ex_e, uint64_t &ex_g, uint32_t *status) {
  const int lane = threadIdx.x & 31;
  ex_e = 0;
  ex_g = 0;
  if (tile == 0) {
    if (lane == 0) st_release_u64(look + tile, pack(kFlagPrefix, agg_g, agg_e));
    return;
  }
  if (lane == 0) st_release_u64(look + tile, pack(kFlagAgg, agg_g, agg_e));
  int64_t base = (int64_t)tile - 1;
  const unsigned long long t0 = globaltimer_ns();
  bool timed_out = false;
  for (;;) {
    const int64_t idx = base - lane;
    uint64_t w = idx >= 0 ? ld_acquire_u64(look + idx) : kFlagPrefix;
    unsigned spins = 0;
    for (;;) {   // warp-uniform: every lane leaves together
      const bool pending = (w & kFlagMask) == 0;
      if (!__any_sync(0xffffffffu, pending)) break;
      if (pending) w = ld_acquire_u64(look + idx);
      if ((++spins & 255u) == 0 && __any_sync(0xffffffffu, globaltimer_ns() - t0 > kSpinLimitNs)) {
        timed_out = true;
        break;
      }
    }
    if (timed_out) {
      if (lane == 0) flag_error(status, DEV_TIMEOUT);
      break;
    }
    const unsigned pre = __ballot_sync(0xffffffffu, (w & kFlagMask) == kFlagPrefix);
    const int stop = pre ? __ffs(pre) - 1 : 31;   // nearest tile with a full prefix
    const uint64_t e = lane <= stop ? (w & kEntMask) : 0;
    const uint64_t gg = lane <= stop ? ((w >> 31) & ((1ull << 31) - 1)) : 0;
    ex_e += warp_sum(e);
    ex_g += warp_sum(gg);
    if (pre) break;
    base -= 32;
  }
  if (lane == 0) st_release_u64(look + tile, pack(kFlagPrefix, ex_g + agg_g, ex_e + agg_e));
}

// Entry (r, c) of a 2^l x 2^l tier grid; a symmetric tree is read on and above the
// diagonal only, so ||A_rc|| and ||A_cr|| are the same number (the entries below it sum
// the same squares in another order and may differ in the last bit).
__device__ __forceinline__ int64_t tier_at(uint32_t r, uint32_t c, int32_t D, int32_t sym) {
  return sym && r > c ? (int64_t)c * D + r : (int64_t)r * D + c;
}

struct CullArgs {
  const double *nA, *nB;    // norms (not squared) of tier l, 2^l x 2^l
  int32_t symA, symB;       // operand trees of symmetric matrices
  int32_t l, D, nb, NB, final_tier;
  int32_t sym;              // symmetric product: output blocks below the diagonal are skipped
  double tau;
  double tau_scale;         // 8^-l with the depth-scaled threshold, else 1 (exact)
  const double *tau_dev;         // when set, tau is read from device memory at launch
  const uint32_t *pgij, *pgstart, *pglen;
  const uint16_t *pK;
  const unsigned long long *p_ngroups;
  int64_t p_cap_entries;
  uint32_t *cgij, *cgstart, *cglen;
  uint16_t *cK;
  int64_t cap_entries, cap_groups;
  unsigned long long *c_ngroups, *c_nentries;
  uint8_t *mask;
  uint64_t *look;
  unsigned int *tile_ctr;
  unsigned long long *tested, *culled, *leaf_products, *output_blocks, *mirror_products;
  double *bound_part;
  uint32_t *status;
  // task plan of the tensor-core leaf kernel (last tier only)
  int plan_mode;                 // 0: none; 1: leaf 64, one item per group (its 2 x 2 output
                                 // blocks); 2: leaf 128, one item per output block
  const uint8_t *nzA, *nzB;
  int bsym;                      // B leaf (k, j) read as leaf (j, k) of a symmetric tree
  int4 *plan;                    // per pass: leaf coordinates {A row 0, A row 1, B col 0, B col 1}
  int64_t cap_plan;
  uint2 *items;                  // per item: {first pass, passes | touched quadrants << 24}
  unsigned long long *npasses;
};

// Passes of one candidate k = 2K + e of a leaf-64 item: the 2 x 2 survival pattern over
// (a, c) taken as one outer product of a row and a column mask when it is one, else one
// pass per row. Returns the pass count; rm/cm get the masks.
__device__ __forceinline__ int passes64(uint32_t m, int e, uint32_t (&rm)[2], uint32_t (&cm)[2]) {
  const uint32_t r0 = ((m >> e) & 1u) | (((m >> (2 + e)) & 1u) << 1);   // a = 0: c = 0, 1
  const uint32_t r1 = ((m >> (4 + e)) & 1u) | (((m >> (6 + e)) & 1u) << 1);
  if (!r0 && !r1) return 0;
  if (!r0 || !r1 || r0 == r1) {
    rm[0] = (r0 ? 1u : 0u) | (r1 ? 2u : 0u);
    cm[0] = r0 | r1;
    return 1;
  }
  rm[0] = 1;
  cm[0] = r0;
  rm[1] = 2;
  cm[1] = r1;
  return 2;
}

// p < tau for a norm product p >= +0 and tau >= +0, on the integer ALU: nonnegative
// doubles order as their bit patterns (a NaN product compares not below, as in FP64),
// which keeps the test off the narrow FP64 pipe.
__device__ __forceinline__ bool below_tau(double p, double tau) {
  return (unsigned long long)__double_as_longlong(p) < (unsigned long long)__double_as_longlong(tau);
}

// Children of entry (I, J, K) tested at tier l: survival bits, test count, and the
// culled norm products summed in a fixed order.
__device__ __forceinline__ uint32_t child_bits(const CullArgs &a, double tau, uint32_t I, uint32_t J,
                                               uint32_t K, int &tests, double &bound) {
  uint32_t bits = 0;
#pragma unroll
  for (int e = 0; e < 2; e++) {
    const uint32_t k = 2 * K + e;
    if (k >= (uint32_t)a.D) continue;
#pragma unroll
    for (int ai = 0; ai < 2; ai++) {
      const uint32_t i = 2 * I + ai;
      if (i >= (uint32_t)a.D) continue;
      const double na = a.nA[tier_at(i, k, a.D, a.symA)];
#pragma unroll
      for (int c = 0; c < 2; c++) {
        const uint32_t j = 2 * J + c;
        if (j >= (uint32_t)a.D) continue;
        if (a.sym && i > j) continue;   // below the diagonal: the mirror of (j, i)
        const double p = na * a.nB[tier_at(k, j, a.D, a.symB)];
        tests++;
        if (below_tau(p, tau)) bound += p;
        else bits |= 1u << (((ai * 2 + c) * 2) + e);
      }
    }
  }
  return bits;
}

// Last tier: the task plan of the tensor-core leaf kernel. Items of the tile (8 groups;
// one item per group at leaf 64, four at leaf 128) are placed after all earlier tiles
// by the same look-back scan, each with its passes in k order (entries ascending, then
// e, then rows): the leaf coordinates of every box the pass loads, or one past the last
// leaf for a box that must be zero (a culled product, a padding or absent leaf).
__device__ void final_plan(const CullArgs &a, unsigned int tile, int warp, int lane, bool has, uint32_t g,
                           uint32_t I, uint32_t J, uint32_t start, uint32_t len, unsigned int (&npq)[4],
                           uint32_t touched, unsigned long long ngroups, unsigned int *s_cnt,
                           unsigned int *s_off) {
#pragma unroll
  for (int q = 0; q < 4; q++) npq[q] = warp_sum(npq[q]);
  touched = __reduce_or_sync(0xffffffffu, touched);
  if (lane < 4) s_cnt[warp * 4 + lane] = has ? npq[lane] : 0u;
  __syncthreads();
  if (warp == 0) {
    const unsigned int v = s_cnt[lane];
    const unsigned int inc = warp_inclusive_scan(v);
    const uint64_t agg = __shfl_sync(0xffffffffu, inc, 31);
    uint64_t ex = 0, exg = 0;
    tile_lookback(a.look, tile, agg, 0, ex, exg, a.status);
    s_off[lane] = (unsigned int)(ex + inc - v);
    if (lane == 0 && (unsigned long long)(tile + 1) * 8 >= ngroups) {
      *a.npasses = ex + agg;
      if ((int64_t)(ex + agg) > a.cap_plan) flag_error(a.status, DEV_OVERFLOW);
    }
  }
  __syncthreads();
  if (!has) return;
  const int oob = a.nb * a.nb;
  if (lane == 0) {
    if (a.plan_mode == 1) {
      a.items[g] = make_uint2(s_off[warp * 4], npq[0] | (touched << 24));
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++)
        a.items[4 * (uint64_t)g + q] = make_uint2(s_off[warp * 4 + q], npq[q] | (((touched >> q) & 1u) << 24));
    }
  }
  unsigned int run[4];
#pragma unroll
  for (int q = 0; q < 4; q++) run[q] = s_off[warp * 4 + q];
  __syncwarp();
  for (uint32_t p0 = 0; p0 < len; p0 += 32) {
    const uint32_t pe = p0 + lane;
    uint32_t bits = 0;
    int K2 = 0;
    if (pe < len) {
      bits = a.mask[start + pe];
      K2 = 2 * (int)a.pK[start + pe];
    }
    if (a.plan_mode == 1) {
      uint32_t rm0[2], cm0[2], rm1[2], cm1[2];
      const int n0 = passes64(bits, 0, rm0, cm0), n1 = passes64(bits, 1, rm1, cm1);
      const unsigned int m = (unsigned int)(n0 + n1);
      const unsigned int inc = warp_inclusive_scan(m);
      int64_t pos = (int64_t)run[0] + inc - m;
      for (int e = 0; e < 2; e++) {
        const int np = e ? n1 : n0;
        const int k = K2 + e;
        for (int ps = 0; ps < np; ps++) {
          const uint32_t rmask = e ? rm1[ps] : rm0[ps], cmask = e ? cm1[ps] : cm0[ps];
          int4 d = make_int4(oob, oob, oob, oob);
          const int i0 = 2 * (int)I, j0 = 2 * (int)J;
          if ((rmask & 1u) && i0 < a.nb && k < a.nb && a.nzA[(int64_t)i0 * a.NB + k]) d.x = i0 * a.nb + k;
          if ((rmask & 2u) && i0 + 1 < a.nb && k < a.nb && a.nzA[(int64_t)(i0 + 1) * a.NB + k]) d.y = (i0 + 1) * a.nb + k;
          if ((cmask & 1u) && j0 < a.nb && k < a.nb && a.nzB[(int64_t)k * a.NB + j0])
            d.z = a.bsym ? j0 * a.nb + k : k * a.nb + j0;
          if ((cmask & 2u) && j0 + 1 < a.nb && k < a.nb && a.nzB[(int64_t)k * a.NB + j0 + 1])
            d.w = a.bsym ? (j0 + 1) * a.nb + k : k * a.nb + j0 + 1;
          if (pos < a.cap_plan) a.plan[pos] = d;
          pos++;
        }
      }
      run[0] += __shfl_sync(0xffffffffu, inc, 31);
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const uint32_t two = (bits >> (2 * q)) & 3u;
        const unsigned int m = __popc(two);
        const unsigned int inc = warp_inclusive_scan(m);
        int64_t pos = (int64_t)run[q] + inc - m;
        const int i = 2 * (int)I + (q >> 1), j = 2 * (int)J + (q & 1);
        for (int e = 0; e < 2; e++) {
          if (!((two >> e) & 1u)) continue;
          const int k = K2 + e;
          int4 d = make_int4(oob, oob, oob, oob);
          if (i < a.nb && k < a.nb && a.nzA[(int64_t)i * a.NB + k]) d.x = i * a.nb + k;
          if (j < a.nb && k < a.nb && a.nzB[(int64_t)k * a.NB + j]) d.z = a.bsym ? j * a.nb + k : k * a.nb + j;
          if (pos < a.cap_plan) a.plan[pos] = d;
          pos++;
        }
        run[q] += __shfl_sync(0xffffffffu, inc, 31);
      }
    }
  }
}

__global__ void __launch_bounds__(kWarps * 32) k_cull_tier(CullArgs a) {
  __shared__ unsigned int s_tile;
  __shared__ unsigned int s_cnt[kWarps * 4];
  __shared__ unsigned int s_off[kWarps * 4];
  __shared__ unsigned int s_gix[kWarps * 4];
  // the CTA's counter sums (tested, culled, leaf products, output blocks, mirrored
  // products), added to the product's counters once at the end
  __shared__ unsigned long long s_acc[5];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long ngroups = *a.p_ngroups;
  const double tau = (a.tau_dev ? *a.tau_dev : a.tau) * a.tau_scale;
  if (threadIdx.x < 5) s_acc[threadIdx.x] = 0ull;
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const unsigned int tile = s_tile;
    __syncthreads();
    if ((unsigned long long)tile * kWarps >= ngroups) break;
    const unsigned long long g = (unsigned long long)tile * kWarps + warp;
    const bool has = g < ngroups;
    uint32_t I = 0, J = 0, start = 0, len = 0;
    if (has) {
      const uint32_t ij = a.pgij[g];
      I = ij >> 16;
      J = ij & 0xFFFFu;
      start = a.pgstart[g];
      len = a.pglen[g];
      // an overflowed parent tier (already flagged) is read only inside its buffer
      if ((int64_t)start >= a.p_cap_entries) len = 0;
      else if ((int64_t)start + len > a.p_cap_entries) len = (uint32_t)(a.p_cap_entries - start);
    }
    // pass 1: per child-quadrant counts (and, on the last tier, the masks)
    unsigned int cnt[4] = {0, 0, 0, 0};
    unsigned int npq[4] = {0, 0, 0, 0};   // passes per item (plan)
    uint32_t touched = 0;
    int tests = 0;
    double bound = 0.0;
    uint32_t keep0 = 0, keep1 = 0, keep2 = 0, keep3 = 0;   // survival bits of the first 128 entries
    for (uint32_t p0 = 0; p0 < len; p0 += 32) {
      const uint32_t p = p0 + lane;
      uint32_t bits = 0;
      if (p < len) {
        const uint32_t K = a.pK[start + p];
        bits = child_bits(a, tau, I, J, K, tests, bound);
        if (a.final_tier) a.mask[start + p] = (uint8_t)bits;
      }
      const uint32_t it = p0 >> 5;
      if (it == 0) keep0 = bits;
      else if (it == 1) keep1 = bits;
      else if (it == 2) keep2 = bits;
      else if (it == 3) keep3 = bits;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        cnt[q] += __popc((bits >> (2 * q)) & 3u);
        if ((bits >> (2 * q)) & 3u) touched |= 1u << q;
      }
      if (a.plan_mode == 1) {
        uint32_t rm[2], cm[2];
        npq[0] += passes64(bits, 0, rm, cm) + passes64(bits, 1, rm, cm);
      } else if (a.plan_mode == 2) {
#pragma unroll
        for (int q = 0; q < 4; q++) npq[q] += __popc((bits >> (2 * q)) & 3u);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) cnt[q] = warp_sum(cnt[q]);
    tests = warp_sum(tests);
    bound = warp_sum(bound);
    if (has && lane == 0) {
      const unsigned int surv = cnt[0] + cnt[1] + cnt[2] + cnt[3];
      atomicAdd(&s_acc[0], (unsigned long long)tests);
      atomicAdd(&s_acc[1], (unsigned long long)(tests - (int)surv));
      a.bound_part[g] = bound;
      if (a.final_tier) {
        atomicAdd(&s_acc[2], (unsigned long long)surv);
        unsigned int blocks = 0, mir = 0;
        for (int q = 0; q < 4; q++) {
          const uint32_t bi = 2 * I + (q >> 1), bj = 2 * J + (q & 1);
          if (cnt[q] && bi < (uint32_t)a.nb && bj < (uint32_t)a.nb) blocks += (a.sym && bi < bj) ? 2 : 1;
          if (a.sym && bi < bj) mir += cnt[q];
        }
        if (blocks) atomicAdd(&s_acc[3], (unsigned long long)blocks);
        if (mir) atomicAdd(&s_acc[4], (unsigned long long)mir);
      }
    }
    if (a.final_tier) {
      if (a.plan_mode) final_plan(a, tile, warp, lane, has, (uint32_t)g, I, J, start, len, npq, touched,
                                  ngroups, s_cnt, s_off);
      continue;
    }

    // tile scan of the 32 child groups (warp w, quadrant q) in order
    if (lane < 4) s_cnt[warp * 4 + lane] = has ? cnt[lane] : 0u;
    __syncthreads();
    if (warp == 0) {
      const unsigned int v = s_cnt[lane];
      const unsigned int f = v ? 1u : 0u;
      const unsigned int inc_v = warp_inclusive_scan(v);
      const unsigned int inc_f = warp_inclusive_scan(f);
      const uint64_t agg_e = __shfl_sync(0xffffffffu, inc_v, 31);
      const uint64_t agg_g = __shfl_sync(0xffffffffu, inc_f, 31);
      uint64_t ex_e = 0, ex_g = 0;
      tile_lookback(a.look, tile, agg_e, agg_g, ex_e, ex_g, a.status);
      s_off[lane] = (unsigned int)(ex_e + inc_v - v);
      s_gix[lane] = (unsigned int)(ex_g + inc_f - f);
      if (lane == 0 && (unsigned long long)(tile + 1) * kWarps >= ngroups) {
        *a.c_nentries = ex_e + agg_e;
        *a.c_ngroups = ex_g + agg_g;
        if ((int64_t)(ex_e + agg_e) > a.cap_entries) flag_error(a.status, DEV_OVERFLOW);
      }
    }
    __syncthreads();
    if (!has) continue;

    // pass 2: child group records and child entries
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (lane == 0 && cnt[q]) {
        const unsigned int gi = s_gix[warp * 4 + q];
        if ((int64_t)gi < a.cap_groups) {
          a.cgij[gi] = ((2 * I + (q >> 1)) << 16) | (2 * J + (q & 1));
          a.cgstart[gi] = s_off[warp * 4 + q];
          a.cglen[gi] = cnt[q];
        }
      }
    }
    unsigned int run[4];
#pragma unroll
    for (int q = 0; q < 4; q++) run[q] = s_off[warp * 4 + q];
    for (uint32_t p0 = 0; p0 < len; p0 += 32) {
      const uint32_t p = p0 + lane;
      uint32_t bits = 0, K = 0;
      if (p < len) {
        K = a.pK[start + p];
        const uint32_t it = p0 >> 5;
        if (it < 4) {
          bits = it == 0 ? keep0 : it == 1 ? keep1 : it == 2 ? keep2 : keep3;
        } else {   // beyond the kept entries: test again (the same deterministic result)
          int dummy_t = 0;
          double dummy_b = 0.0;
          bits = child_bits(a, tau, I, J, K, dummy_t, dummy_b);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const uint32_t two = (bits >> (2 * q)) & 3u;
        const unsigned int m = __popc(two);
        const unsigned int inc = warp_inclusive_scan(m);
        unsigned int pos = run[q] + inc - m;
        if (two & 1u) {
          if ((int64_t)pos < a.cap_entries) a.cK[pos] = (uint16_t)(2 * K);
          pos++;
        }
        if (two & 2u) {
          if ((int64_t)pos < a.cap_entries) a.cK[pos] = (uint16_t)(2 * K + 1);
        }
        run[q] += __shfl_sync(0xffffffffu, inc, 31);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long *dst[5] = {a.tested, a.culled, a.leaf_products, a.output_blocks, a.mirror_products};
    for (int q = 0; q < 5; q++)
      if (s_acc[q]) atomicAdd(dst[q], s_acc[q]);
  }
}

// The upper tiers in one CTA. Tiers 0..T (T < k_max, at most kTopTiers of them) hold at
// most 8^T triples, far too little work for a launch per tier. Tier l is evaluated for
// all its 4^l output blocks at once, a thread per block (I, J) in Morton order (so the
// parent block is index >> 2), each over its K < 2^l: the triple (I, J, K) is tested
// when its parent (I/2, J/2, K/2) survived tier l-1 (and, for a symmetric product,
// I <= J) and survives when ||A^l_IK||_F ||B^l_KJ||_F >= tau: exactly the calls of the
// Eq. 4 recursion, as in k_cull_tier. A block's survivors form a bit mask over K, which
// is the next tier's parent test. Only the tier-T list (groups in Morton order, K
// ascending) and the counters of tiers 0..T are written; the culled bound of tier l
// (summed per thread over K, per warp and then over warps by fixed trees) goes
// to the first parent-group slot of the tier and zeros to the others, so the fixed-
// order reduction of the slots returns it unchanged.
constexpr int kTopTiers = 6;                 // tiers 0..5
constexpr int kTopBlocks = 1024;             // output blocks of tier 5 (4^5), a thread each
constexpr int kTopThreads = 1024;
constexpr int kTopWarps = kTopThreads / 32;
constexpr int kTopNorms = ((1 << (2 * kTopTiers)) - 1) / 3;   // norms of tiers 0..5 per operand
static_assert(kTopBlocks == 1 << (2 * (kTopTiers - 1)) && kTopBlocks <= kTopThreads, "a thread per tier-T block");

struct TopArgs {
  const double *nA[kTopTiers], *nB[kTopTiers];   // tier norms (not squared)
  int64_t bound_off[kTopTiers];                  // this tier's block of bound_part
  int32_t T;                                     // last tier run here
  int32_t sym;                                   // symmetric product
  int32_t symA, symB;                            // operand trees of symmetric matrices
  int32_t depth_tau;                             // tier l tests against tau * 8^-l
  double tau;
  const double *tau_dev;
  uint32_t *gij, *gstart, *glen;                 // the tier-T list (C->tiers[T + 1])
  uint16_t *K;
  int64_t cap_groups, cap_entries;
  DevCounts *cnt;
  double *bound_part;
  uint32_t *status;
  // the product's prologue, done by the other CTAs of the launch: look-back words and
  // the product's leaf norms and presence bytes zeroed
  uint64_t *look;
  int64_t nlook;
  double *leaf_norm2C;
  uint8_t *nzC;
  int64_t nleaves;
};

// (I, J) of Morton index m: bit 2b of m is bit b of J, bit 2b + 1 is bit b of I.
__device__ __forceinline__ void morton_ij(uint32_t m, uint32_t &I, uint32_t &J) {
  I = 0;
  J = 0;
#pragma unroll
  for (int b = 0; b < kTopTiers; b++) {
    J |= ((m >> (2 * b)) & 1u) << b;
    I |= ((m >> (2 * b + 1)) & 1u) << b;
  }
}

__global__ void __launch_bounds__(kTopThreads, 1) k_cull_top(TopArgs t) {
  if (blockIdx.x > 0) {   // the prologue's zeroing, spread over CTAs 1 ..
    const int64_t t0 = (blockIdx.x - 1) * (int64_t)blockDim.x + threadIdx.x;
    const int64_t st = (int64_t)(gridDim.x - 1) * blockDim.x;
    for (int64_t q = t0; q < t.nlook; q += st) t.look[q] = 0ull;
    if (t.leaf_norm2C)
      for (int64_t q = t0; q < t.nleaves; q += st) t.leaf_norm2C[q] = 0.0;
    if (t.nzC)
      for (int64_t q = t0; q < t.nleaves; q += st) t.nzC[q] = 0;
    return;
  }
  __shared__ double s_nA[kTopNorms], s_nB[kTopNorms];   // the tier norms, read once
  {   // counters zeroed (no other CTA touches them); tier 0's parent list is the root group
    uint32_t *cw = reinterpret_cast<uint32_t *>(t.cnt);
    for (int q = threadIdx.x; q < (int)(sizeof(DevCounts) / 4); q += blockDim.x) cw[q] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
      t.cnt->ngroups[0] = 1;
      t.cnt->nentries[0] = 1;
    }
  }
  __shared__ uint32_t s_mask[2][kTopBlocks];            // survivors over K per block: tiers l-1, l
  __shared__ double s_wb[kTopWarps];                    // per-warp culled bounds
  __shared__ uint32_t s_wg[kTopWarps], s_we[kTopWarps];
  __shared__ uint32_t s_wt[kTopWarps], s_ws[kTopWarps];   // per-warp tests and survivors
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double tau = t.tau_dev ? *t.tau_dev : t.tau;
  for (int l = 0; l <= t.T; l++) {
    const int64_t off = level_offset(l);
    for (int q = threadIdx.x; q < (1 << (2 * l)); q += blockDim.x) {
      s_nA[off + q] = t.nA[l][q];
      s_nB[off + q] = t.nB[l][q];
    }
  }
  __syncthreads();
  const uint32_t m = threadIdx.x;
  uint32_t I = 0, J = 0;
  morton_ij(m, I, J);
  int cur = 0;                 // s_mask[cur]: the tier just evaluated
  uint32_t parent_groups = 1;  // groups of the tier l-1 list (tier -1: the root group)
  double tl = tau;             // this tier's threshold
  for (int l = 0; l <= t.T; l++) {
    if (l && t.depth_tau) tl *= 0.125;
    const uint32_t D = 1u << l, nblk = D * D;
    const double *nA = s_nA + level_offset(l), *nB = s_nB + level_offset(l);
    uint32_t mask = 0;
    int tests = 0;
    double bound = 0.0;
    if (m < nblk && !(t.sym && I > J)) {   // below the diagonal: the mirror of (J, I)
      // the parent's surviving K' (tier 0's parent: K' = 0 of the root); only their
      // children 2K' + e are calls, visited in ascending K, so that the FP64 products
      // (a narrow pipe on this GPU) are issued for the warp's calls only
      for (uint32_t pend = l ? s_mask[cur][m >> 2] : 1u; pend; pend &= pend - 1u) {
        const uint32_t Kp = (uint32_t)(__ffs(pend) - 1);
#pragma unroll
        for (uint32_t e = 0; e < 2; e++) {
          const uint32_t K = 2 * Kp + e;
          if (K >= D) continue;
          const double p = nA[tier_at(I, K, D, t.symA)] * nB[tier_at(K, J, D, t.symB)];
          tests++;
          if (below_tau(p, tl)) bound += p;
          else mask |= 1u << K;
        }
      }
    }
    const int nx = l ? cur ^ 1 : 0;
    if (m < nblk) s_mask[nx][m] = mask;
    tests = warp_sum(tests);
    const unsigned int surv = warp_sum((unsigned int)__popc(mask));
    if (__any_sync(0xffffffffu, bound != 0.0)) bound = warp_sum(bound);   // else every lane holds +0
    if (lane == 0) {
      s_wb[warp] = bound;
      s_wt[warp] = (uint32_t)tests;
      s_ws[warp] = surv;
    }
    const uint32_t groups = (uint32_t)__syncthreads_count(m < nblk && mask != 0u);
    if (warp == 0) {   // the warps' bounds by a fixed shuffle tree (warps without blocks hold +0)
      double b = s_wb[lane];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) b += __shfl_down_sync(0xffffffffu, b, off);
      const unsigned long long tested = warp_sum((unsigned long long)s_wt[lane]);
      const unsigned long long survived = warp_sum((unsigned long long)s_ws[lane]);
      if (lane == 0) {
        t.bound_part[t.bound_off[l]] = b;
        t.cnt->tested[l] = tested;
        t.cnt->culled[l] = tested - survived;
        t.cnt->ngroups[l + 1] = groups;
        t.cnt->nentries[l + 1] = survived;
      }
    }
    for (uint32_t g = 1 + threadIdx.x; g < parent_groups; g += blockDim.x) t.bound_part[t.bound_off[l] + g] = 0.0;
    parent_groups = groups;
    cur = nx;
    __syncthreads();
  }
  // the tier-T list, for the launch of tier T + 1: groups and entries placed by a
  // block-wide exclusive scan over the blocks in Morton order
  const uint32_t DT = 1u << t.T;
  const uint32_t mask = m < DT * DT ? s_mask[cur][m] : 0u;
  const uint32_t has = mask ? 1u : 0u, cntK = (uint32_t)__popc(mask);
  const uint32_t ig = warp_inclusive_scan(has), ie = warp_inclusive_scan(cntK);
  if (lane == 31) {
    s_wg[warp] = ig;
    s_we[warp] = ie;
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t vg = s_wg[lane], ve = s_we[lane];
    const uint32_t sg = warp_inclusive_scan(vg), se = warp_inclusive_scan(ve);
    s_wg[lane] = sg - vg;
    s_we[lane] = se - ve;
  }
  __syncthreads();
  if (has) {
    const uint32_t gi = s_wg[warp] + ig - 1u, e0 = s_we[warp] + ie - cntK;
    if ((int64_t)gi < t.cap_groups) {
      t.gij[gi] = (I << 16) | J;
      t.gstart[gi] = e0;
      t.glen[gi] = cntK;
    }
    uint32_t r = 0;
    for (uint32_t K = 0; K < DT; K++)
      if ((mask >> K) & 1u) {
        if ((int64_t)(e0 + r) < t.cap_entries) t.K[e0 + r] = (uint16_t)K;
        r++;
      }
  }
}

// Prologue of a product: zeroes the counters, the look-back words and the product's
// leaf norms / presence bytes, and seeds the virtual tier -1: one group (0, 0) holding
// K = 0, whose only in-range child is the root triple (0, 0, 0).
__global__ void __launch_bounds__(256) k_cull_prologue(uint32_t *gij, uint32_t *gstart, uint32_t *glen,
                                                       uint16_t *K, DevCounts *cnt, uint64_t *look,
                                                       int64_t nlook, double *leaf_norm2, uint8_t *nz,
                                                       int64_t nleaves) {
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = t0; t < nlook; t += st) look[t] = 0ull;
  if (leaf_norm2)
    for (int64_t t = t0; t < nleaves; t += st) leaf_norm2[t] = 0.0;
  if (nz)
    for (int64_t t = t0; t < nleaves; t += st) nz[t] = 0;
  if (blockIdx.x != 0) return;
  // the counters are zeroed and seeded by block 0 alone, so no other block can race
  uint32_t *cw = reinterpret_cast<uint32_t *>(cnt);
  for (int t = threadIdx.x; t < (int)(sizeof(DevCounts) / 4); t += blockDim.x) cw[t] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    gij[0] = 0;
    gstart[0] = 0;
    glen[0] = 1;
    K[0] = 0;
    cnt->ngroups[0] = 1;
    cnt->nentries[0] = 1;
  }
}

// Fixed-order sum of the per-group culled bounds of every tier, one CTA per tier.
__global__ void __launch_bounds__(256) k_bound_reduce(const double *part, const int64_t *off,
                                                      DevCounts *cnt) {
  const int l = blockIdx.x;
  const unsigned long long ng = cnt->ngroups[l];   // parent groups of tier l
  const double *p = part + off[l];
  double s = 0.0;
  for (unsigned long long g = threadIdx.x; g < ng; g += blockDim.x) s += p[g];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt->culled_bound[l] = sh[0];
}

}  // namespace

// Offsets of each tier's per-group bound partials (tier l uses the parent groups of
// list l, at most 4^(l-1) of them, 1 for l = 0).
static int64_t bound_groups_cap(int l) { return l == 0 ? 1 : (int64_t(1) << (2 * (l - 1))); }

cudaError_t launch_cull(spamm_tree A, spamm_tree B, spamm_tree C, double tau, const double *tau_dev,
                        uint32_t *dev_status, int sm_count, cudaStream_t s, int *launches) {
  const int kmax = A->kmax;
  DevCounts *cnt = C->counts;
  const TierList &root = C->tiers[0];
  const int64_t nleaves = (int64_t)C->NB * C->NB;
  const int64_t work = std::max<int64_t>(nleaves, C->cap_look);
  if (kmax < 2) {   // with k_cull_top, its other CTAs do this
    const unsigned pg = (unsigned)std::min<int64_t>((work + 255) / 256, 1024);
    k_cull_prologue<<<pg, 256, 0, s>>>(root.gij, root.gstart, root.glen, root.K, cnt, C->look, C->cap_look,
                                       C->norm2 ? C->norm2 + level_offset(C->kmax) : nullptr, C->nz, nleaves);
    (*launches)++;
  }
  int64_t look_off = 0, bound_off = 0;
  int l0 = 0;   // first tier launched on its own
  if (kmax >= 2) {
    TopArgs ta{};
    ta.T = std::min(kTopTiers, kmax) - 1;   // the last tier always runs in k_cull_tier
    for (int l = 0; l <= ta.T; l++) {
      ta.nA[l] = A->norm + level_offset(l);
      ta.nB[l] = B->norm + level_offset(l);
      ta.bound_off[l] = bound_off;
      look_off += (bound_groups_cap(l) + kWarps - 1) / kWarps;
      bound_off += bound_groups_cap(l);
    }
    ta.tau = tau;
    ta.tau_dev = tau_dev;
    ta.sym = C->sym_product ? 1 : 0;
    ta.symA = (A->flags & SPAMM_SYMMETRIC) ? 1 : 0;
    ta.depth_tau = C->depth_tau ? 1 : 0;
    ta.symB = (B->flags & SPAMM_SYMMETRIC) ? 1 : 0;
    const TierList &out = C->tiers[ta.T + 1];
    ta.gij = out.gij;
    ta.gstart = out.gstart;
    ta.glen = out.glen;
    ta.K = out.K;
    ta.cap_groups = out.cap_groups;
    ta.cap_entries = out.cap_entries;
    ta.cnt = cnt;
    ta.bound_part = C->bound_part;
    ta.status = dev_status;
    ta.look = C->look;
    ta.nlook = C->cap_look;
    ta.leaf_norm2C = C->norm2 ? C->norm2 + level_offset(C->kmax) : nullptr;
    ta.nzC = C->nz;
    ta.nleaves = nleaves;
    const unsigned zc = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + kTopThreads - 1) / kTopThreads, 4 * sm_count));
    k_cull_top<<<1 + zc, kTopThreads, 0, s>>>(ta);
    (*launches)++;
    l0 = ta.T + 1;
  }
  for (int l = l0; l <= kmax; l++) {
    CullArgs a{};
    a.nA = A->norm + level_offset(l);
    a.nB = B->norm + level_offset(l);
    a.l = l;
    a.D = 1 << l;
    a.nb = A->nb;
    a.NB = A->NB;
    a.final_tier = (l == kmax);
    a.sym = C->sym_product ? 1 : 0;
    a.symA = (A->flags & SPAMM_SYMMETRIC) ? 1 : 0;
    a.symB = (B->flags & SPAMM_SYMMETRIC) ? 1 : 0;
    a.tau = tau;
    a.tau_scale = C->depth_tau ? std::ldexp(1.0, -3 * l) : 1.0;
    a.tau_dev = tau_dev;
    const TierList &par = C->tiers[l];
    a.pgij = par.gij;
    a.pgstart = par.gstart;
    a.pglen = par.glen;
    a.pK = par.K;
    a.p_ngroups = &cnt->ngroups[l];
    a.p_cap_entries = par.cap_entries;
    if (!a.final_tier) {
      const TierList &ch = C->tiers[l + 1];
      a.cgij = ch.gij;
      a.cgstart = ch.gstart;
      a.cglen = ch.glen;
      a.cK = ch.K;
      a.cap_entries = ch.cap_entries;
      a.cap_groups = ch.cap_groups;
      a.c_ngroups = &cnt->ngroups[l + 1];
      a.c_nentries = &cnt->nentries[l + 1];
    } else {
      a.mask = C->mask;
      a.plan_mode = C->warp_tiles ? 0 : C->plan_mode;   // the warp-tile kernel reads the tier lists
      a.nzA = A->nz;
      a.nzB = B->nz;
      a.bsym = (B->flags & SPAMM_SYMMETRIC) != 0;
      a.plan = C->plan;
      a.cap_plan = C->cap_plan;
      a.items = C->items;
      a.npasses = &cnt->npasses;
    }
    const int64_t pg = bound_groups_cap(l);
    const int64_t tiles = (pg + kWarps - 1) / kWarps;
    a.look = C->look + look_off;
    a.tile_ctr = &cnt->tile_ctr[l];
    a.tested = &cnt->tested[l];
    a.culled = &cnt->culled[l];
    a.leaf_products = &cnt->leaf_products;
    a.output_blocks = &cnt->output_blocks;
    a.mirror_products = &cnt->mirror_products;
    a.bound_part = C->bound_part + bound_off;
    a.status = dev_status;
    look_off += tiles;
    bound_off += pg;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)sm_count * 8);
    k_cull_tier<<<(unsigned)grid, kWarps * 32, 0, s>>>(a);
    (*launches)++;
  }
  return cudaGetLastError();
}

cudaError_t launch_finish_stats(spamm_tree C, cudaStream_t s) {
  // bound offsets table lives in the tail of bound_part's allocation
  const int kmax = C->kmax;
  int64_t *off = reinterpret_cast<int64_t *>(C->bound_part + C->cap_bound);
  k_bound_reduce<<<kmax + 1, 256, 0, s>>>(C->bound_part, off, C->counts);
  return cudaGetLastError();
}

int64_t cull_look_words(int kmax) {
  int64_t t = 0;
  for (int l = 0; l <= kmax; l++) t += (bound_groups_cap(l) + kWarps - 1) / kWarps;
  return t;
}

int64_t cull_bound_words(int kmax, int64_t *offsets) {
  int64_t t = 0;
  for (int l = 0; l <= kmax; l++) {
    if (offsets) offsets[l] = t;
    t += bound_groups_cap(l);
  }
  return t;
}
