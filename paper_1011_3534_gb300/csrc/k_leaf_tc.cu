// Tensor-core leaf products (the k = k_max case of Eq. 4) with tcgen05, TMA and TMEM.
//
// Work item. Leaf 64: one tier kmax-1 group (I, J), i.e. the 2 x 2 output blocks
// (2I + a, 2J + c), a 128 x 128 FP32 accumulator in TMEM. Leaf 128: one output block
// (2I + a, 2J + c), also 128 x 128. A persistent grid of one CTA per SM takes items in
// Morton order of the output blocks from one counter, each CTA the next item when its
// producer gets to it, so that the SMs finish together however uneven the items are.
//
// Candidates. For each entry K of the group (ascending) and e = 0, 1, the surviving
// children form a 2 x 2 pattern over (a, c). A pattern that is an outer product of a
// row mask and a column mask is one pass: the A leaves (2I + a, k) of unmasked rows and
// the B leaves (k, 2J + c) of unmasked columns are loaded, the others are zero-filled
// by the TMA (a leaf coordinate past the end of the tensor), and one 128 x N x b MMA
// chain adds exactly the surviving products: N = 128, or N = 64 on the one column half
// a single-column pass touches (leaf 64). Other patterns take one pass per row. Each
// output block therefore sums its surviving k in ascending order, in FP32.
//
// Pipeline (one CTA, 320 threads): warp 0 issues TMA loads into a ring of stages, one
// 128-byte K chunk of every operand per stage (plain forms: 6 stages of A 128 x 128 B +
// B 128 x 128 B; split forms: 3 stages of A hi, B hi, A lo, B lo, each hi and lo box
// loaded once per chunk and read by the three products), 128-byte swizzle; warp 1
// issues tcgen05.mma (4 K-steps of 32 bytes per operand pair and stage) and commits to
// the stage's empty barrier; warps 2-9 (two per TMEM lane quarter, each on 64 of the
// 128 accumulator columns) drain finished accumulators with tcgen05.ld, store C (FP32
// tiles, and the transposed block of a symmetric product) and its squared Frobenius
// norms (double-float, fixed-order sums) while later work accumulates in the other TMEM
// buffers.
//
// Accumulation. The tensor cores of this GPU truncate each MMA's FP32 sum (measured
// bias about -0.5 unit in the last place per instruction), so the error of one
// accumulator grows with the instructions it takes at its own magnitude. Plain forms:
// one accumulator per item (four in TMEM). Split forms (hi hi + hi lo + lo hi): the
// large hi hi products of every pass go to a fresh accumulator (two in TMEM, alternating)
// and the epilogue adds the passes in FP32 registers with round to nearest, in the order
// of the plan; the small corrections hi lo + lo hi, 2^-11 of the products and so of the
// truncation bias, accumulate over the whole item in one accumulator (two in TMEM, one
// item ahead), added once at the end.
// Every wait is bounded; a wait that runs out sets an error bit and the CTA unwinds.
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "f32x2.cuh"
#include "tc_ptx.cuh"

// Optional per-role cycle counters (build with -DSPAMM_LEAF_ROLE_CYCLES; the library's
// own build compiles none of this): per CTA, the cycles each role spends waiting and
// working, read back by spamm_leaf_role_cycles (paper_1011_3534_gb300/leaf_role_cycles.py).
#ifdef SPAMM_LEAF_ROLE_CYCLES
__device__ unsigned long long g_role_cycles[1024][16];
#define ROLE_T0(v) const long long v = clock64()
#define ROLE_ADD(slot, v)                                                                               \
  do {                                                                                                  \
    if ((threadIdx.x & 31) == 0)                                                                        \
      atomicAdd(&g_role_cycles[blockIdx.x & 1023][slot], (unsigned long long)(clock64() - (v)));       \
  } while (0)
#define ROLE_COUNT(slot)                                                                                \
  do {                                                                                                  \
    if ((threadIdx.x & 31) == 0) atomicAdd(&g_role_cycles[blockIdx.x & 1023][slot], 1ull);            \
  } while (0)
#else
#define ROLE_T0(v)
#define ROLE_ADD(slot, v)
#define ROLE_COUNT(slot)
#endif

namespace {

constexpr int kThreads = 320;   // producer, MMA issuer, eight epilogue warps
constexpr uint32_t kTmemCols = 512;   // four 128-column FP32 accumulators
constexpr int kBoxBytes = 16384;      // one operand of one stage: 128 rows x 128 bytes
constexpr size_t kSmemBytes = (size_t)6 * 32768 + 1024;   // the ring (either form) + alignment

// Stage ring of the plain (one operand pair) and split (hi and lo of both operands) forms.
template <bool SPLIT>
struct Ring {
  static constexpr int kStages = SPLIT ? 3 : 6;
  static constexpr int kStageBytes = SPLIT ? 4 * kBoxBytes : 2 * kBoxBytes;
  // byte offsets inside a stage
  static constexpr int kAhi = 0, kBhi = kBoxBytes, kAlo = 2 * kBoxBytes, kBlo = 3 * kBoxBytes;
  // accumulator slots of 128 columns: plain, one per item (four); split, one per pass
  // for hi hi (two) and one per item for the corrections hi lo + lo hi (two, from
  // column 256)
  static constexpr int kAcc = SPLIT ? 2 : 4;
  static constexpr int kSmall = SPLIT ? 2 : 1;
  static constexpr uint32_t kSmallCol = 256u;
};
static_assert((size_t)Ring<true>::kStages * Ring<true>::kStageBytes + 1024 <= kSmemBytes, "split ring");
static_assert((size_t)Ring<false>::kStages * Ring<false>::kStageBytes + 1024 <= kSmemBytes, "plain ring");

// One product of a launch. The table lives in device memory (64-byte aligned for the
// tensor maps); a single product and a batch use the same kernel.
struct __align__(64) ProdDesc {
  CUtensorMap mA, mB, mAlo, mBlo;          // leaf copies: A rows, B (rows if symmetric, else
                                           // transposed leaves), and the lows of a split
  const uint2 *items;                      // per item: {first pass, passes | touched << 24}
  const int4 *plan;                        // per pass: leaf coordinates of the four boxes
  int64_t cap_plan;
  int64_t cap_items;
  const uint32_t *gij;                     // groups of the last tier list: (I << 16) | J
  const unsigned long long *ngroups;       // number of those groups (device)
  float *C;                                // FP32 tiles of the product
  uint8_t *nzC;
  double *leaf_norm2C;
  unsigned long long *mma_stages;
  unsigned int *work_ctr;                  // item counter of a launch (the first product's, zeroed by its cull)
  int32_t nb, NB;
  int32_t sym;                             // symmetric product: blocks i < j also written as C_ji = C_ij^T
};

struct TcCommon {
  uint32_t idesc;        // M = 128, N = 128
  uint32_t idesc64;      // M = 128, N = 64
  int32_t chunks;        // 128-byte K chunks per leaf
  int32_t chunk_elems;   // elements per chunk
  uint32_t *status;
};

constexpr int kMaxProd = 1024;   // products per launch

__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  float err = (h - (s - bb)) + (bh - bb);
  err += l + bl;
  h = s + err;
  l = err - (h - s);
}

// Product holding global item g: offsets s_off[0..nprod] in shared memory.
__device__ __forceinline__ int find_prod(const unsigned long long *s_off, int nprod, unsigned long long g) {
  int lo = 0, hi = nprod;   // s_off[lo] <= g < s_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_off[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Column halves a pass multiplies (leaf 64): bit c set when the B leaf of column c is
// loaded (a coordinate below nb^2); a pass with neither (absent leaves, tau = 0) is
// treated as a full one. Leaf 128 items have one column: always 3 (N = 128).
template <int LEAF>
__device__ __forceinline__ uint32_t pass_cols(const int4 &d, int oob) {
  if (LEAF != 64) return 3u;
  const uint32_t cm = (d.z < oob ? 1u : 0u) | (d.w < oob ? 2u : 0u);
  return cm ? cm : 3u;
}

// Passes of an item that the kernel may read: the plan's count, cut at its capacity
// (an overflowing plan is also flagged by the cull).
__device__ __forceinline__ uint32_t item_passes(const ProdDesc &P, uint2 meta, uint32_t *status) {
  const uint32_t first = meta.x;
  uint32_t np = meta.y & 0xFFFFFFu;
  if ((int64_t)first + np > P.cap_plan) {
    flag_error(status, DEV_BADARG);
    np = (int64_t)first >= P.cap_plan ? 0u : (uint32_t)(P.cap_plan - first);
  }
  return np;
}

template <int LEAF, bool TF32, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_leaf_tc(const ProdDesc *__restrict__ prods, int nprod, TcCommon cm) {
  using R = Ring<SPLIT>;
  constexpr int kStages = R::kStages;
  constexpr int kAcc = R::kAcc;
  extern __shared__ uint8_t smem_raw[];
  constexpr int kSmall = R::kSmall;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf[kAcc], acce[kAcc], smf[kSmall], sme[kSmall];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ double s_norm[4][2];
  __shared__ int4 s_desc[32];                    // producer: the chunk of passes being issued
  __shared__ uint8_t s_cols[kStages];            // producer -> MMA: column halves of a stage
  __shared__ float s_epi[8][32][17];             // epilogue: one 32 x 16 piece per warp, transposed out
  __shared__ unsigned long long s_off[kMaxProd + 1];   // first global item of each product
  constexpr int kQ = 4;                          // item ring: producer -> MMA and epilogue warps
  __shared__ __align__(8) uint64_t qfull[kQ], qempty[kQ];
  __shared__ int4 s_qe[kQ];                      // {product, index in it, first pass, passes | touched << 24}
  __shared__ uint32_t s_qij[kQ];                 // the item's group (I << 16) | J
  constexpr int RA = LEAF == 64 ? 2 : 1;        // A leaves stacked along M
  constexpr int RC = LEAF == 64 ? 2 : 1;        // B leaves stacked along N
  constexpr uint32_t kBox = LEAF * 128;         // bytes of one leaf box (LEAF rows x 128 B)
  constexpr unsigned long long kPer = LEAF == 64 ? 1ull : 4ull;   // items per group

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ROLE_T0(t_kernel);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < kAcc; a++) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 256);
    }
    for (int a = 0; a < kSmall; a++) {
      mbar_init(&smf[a], 1);
      mbar_init(&sme[a], 256);
    }
    for (int q = 0; q < kQ; q++) {
      mbar_init(&qfull[q], 1);
      mbar_init(&qempty[q], 9);   // the MMA warp and the eight epilogue warps
    }
    s_abort = 0;
    mbar_fence_init();
  }
  for (int q = threadIdx.x; q < nprod; q += blockDim.x) s_off[q + 1] = kPer * (*prods[q].ngroups);
  if (warp == 1) tmem_alloc(&s_tmem, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) {   // item offsets of the products (nprod <= kMaxProd)
    s_off[0] = 0;
    for (int q = 1; q <= nprod; q++) s_off[q] += s_off[q - 1];
  }
  __syncthreads();
  const uint32_t tmem = s_tmem;
  const unsigned long long nitems = s_off[nprod];
  // Items are taken from a counter shared by all CTAs (the product's work counter,
  // zeroed by its cull) as the producer gets to them, so that every SM keeps working
  // until the list is empty; the producer hands each item to the MMA warp and the
  // epilogue warps through a ring of kQ slots in shared memory (a negative product
  // index ends the list).
  unsigned int *const ctr = prods[0].work_ctr;
  // the item after this CTA's current one: its product, index in the product and
  // metadata {first pass, passes | touched << 24}, and its group (I << 16) | J
  auto claim = [&]() -> unsigned int { return lane == 0 ? atomicAdd(ctr, 1u) : 0u; };
  auto describe = [&](unsigned int g, int4 &e, uint32_t &ij) {
    g = __shfl_sync(0xffffffffu, g, 0);
    e = make_int4(-1, 0, 0, 0);
    ij = 0u;
    if ((unsigned long long)g >= nitems) return;
    const int prod = find_prod(s_off, nprod, g);
    const unsigned long long local = g - s_off[prod];
    const unsigned long long gq = LEAF == 64 ? local : (local >> 2);
    if ((int64_t)local >= prods[prod].cap_items || (int64_t)gq >= prods[prod].cap_items) {
      flag_error(cm.status, DEV_BADARG);   // cannot happen for a well-formed list
      return;
    }
    const uint2 meta = prods[prod].items[local];
    e = make_int4(prod, (int)local, (int)meta.x, (int)meta.y);
    ij = prods[prod].gij[gq];
  };
  // consumers: the next slot of the ring (lane 0 waits; every lane reads it)
  auto take = [&](int &qs, uint32_t &qp, int4 &e, uint32_t &ij) -> bool {
    bool ok = true;
    if (lane == 0) ok = mbar_wait(&qfull[qs], qp, &s_abort);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (!ok) {
      if (lane == 0) {
        s_abort = 1;
        flag_error(cm.status, DEV_TIMEOUT);
      }
      return false;
    }
    e = s_qe[qs];
    ij = s_qij[qs];
    __syncwarp();
    if (lane == 0) mbar_arrive(&qempty[qs]);
    if (++qs == kQ) {
      qs = 0;
      qp ^= 1u;
    }
    return e.x >= 0;
  };

  // whole-warp bounded wait: every lane polls, the outcome is made warp-uniform, and a
  // wait that ran out sets the abort flag and the error bit
  auto wwait = [&](uint64_t *bar, uint32_t parity) -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, parity, &s_abort));
    if (!ok && lane == 0) {
      s_abort = 1;
      flag_error(cm.status, DEV_TIMEOUT);
    }
    return ok;
  };
  auto aborted = [&]() -> bool { return __any_sync(0xffffffffu, s_abort != 0); };

  if (warp == 0) {
    // ---------------- TMA producer (warp 0) ----------------
    // Each item's passes are loaded 32 at a time, the next chunk while lane 0 issues
    // the current one.
    if (lane == 0 && nprod == 1) {
      tma_prefetch_desc(&prods[0].mA);
      tma_prefetch_desc(&prods[0].mB);
      if (SPLIT) {
        tma_prefetch_desc(&prods[0].mAlo);
        tma_prefetch_desc(&prods[0].mBlo);
      }
    }
    int stage = 0;
    uint32_t phase = 0;
    int qs = 0;
    uint32_t qp = 0;
    int4 cur_e;
    uint32_t cur_ij;
    describe(claim(), cur_e, cur_ij);
    for (;;) {
      ROLE_T0(t_pub);
      // publish the item to the other roles
      if (lane == 0) {
        if (!mbar_wait(&qempty[qs], qp ^ 1u, &s_abort)) {
          s_abort = 1;
          flag_error(cm.status, DEV_TIMEOUT);
        }
        s_qe[qs] = s_abort ? make_int4(-1, 0, 0, 0) : cur_e;
        s_qij[qs] = cur_ij;
        mbar_arrive(&qfull[qs]);
      }
      if (++qs == kQ) {
        qs = 0;
        qp ^= 1u;
      }
      ROLE_ADD(11, t_pub);
      if (cur_e.x < 0 || __shfl_sync(0xffffffffu, s_abort ? 1 : 0, 0)) break;
      // the next item is claimed and its description read two passes before this one's
      // loads end (the replies arrive while they go out): late enough that a CTA does not
      // hold an unstarted item while others run dry at the end of the list
      int4 nxt_e;
      uint32_t nxt_ij;
      bool claimed = false;
      {
        const ProdDesc &P = prods[cur_e.x];
        const uint2 mt = make_uint2((uint32_t)cur_e.z, (uint32_t)cur_e.w);
        const uint32_t first = mt.x;
        const uint32_t np = item_passes(P, mt, cm.status);
        const int oob = P.nb * P.nb;
        const int4 *plan = P.plan;
        int4 cur = make_int4(0, 0, 0, 0);
        if ((uint32_t)lane < np) cur = plan[(int64_t)first + lane];
        for (uint32_t c0 = 0; c0 < np; c0 += 32) {
          s_desc[lane] = cur;
          __syncwarp();
          if (c0 + 32 < np && c0 + 32 + lane < np) cur = plan[(int64_t)first + c0 + 32 + lane];
          // the whole warp walks the passes and waits; one elected lane issues each
          // stage's copies
          const int nl = (int)min(32u, np - c0);
          for (int l = 0; l < nl && !aborted(); l++) {
            if (!claimed && c0 + (uint32_t)l + 2u >= np) {
              describe(claim(), nxt_e, nxt_ij);
              claimed = true;
            }
            const int4 d = s_desc[l];
            // the first pass of an item initialises both column halves (N = 128) of the
            // item's accumulator (plain) or correction accumulator (split)
            const uint32_t cols = c0 + l == 0 ? 3u : pass_cols<LEAF>(d, oob);
            const int boxes = (SPLIT ? 2 : 1) * (RA + (RC == 2 ? __popc(cols) : 1));
            for (int ch = 0; ch < cm.chunks; ch++) {
              ROLE_T0(t_we);
              const bool ok_e = wwait(&empty[stage], phase ^ 1u);
              ROLE_ADD(0, t_we);
              if (!ok_e) break;
              if (elect_one()) {
                s_cols[stage] = (uint8_t)cols;   // read by the MMA warp after the full barrier
                mbar_expect_tx(&full[stage], (uint32_t)boxes * kBox);
                const uint32_t st = base + stage * R::kStageBytes;
                const int x = ch * cm.chunk_elems;
#pragma unroll
                for (int h = 0; h < (SPLIT ? 2 : 1); h++) {   // hi, then (split) lo
                  const CUtensorMap *ma = h ? &P.mAlo : &P.mA;
                  const CUtensorMap *mb = h ? &P.mBlo : &P.mB;
                  const uint32_t sa = st + (h ? R::kAlo : R::kAhi), sb = st + (h ? R::kBlo : R::kBhi);
                  tma_load_3d(sa, ma, &full[stage], x, 0, d.x);
                  if (RA == 2) tma_load_3d(sa + kBox, ma, &full[stage], x, 0, d.y);
                  if (cols & 1u) tma_load_3d(sb, mb, &full[stage], x, 0, d.z);
                  if (RC == 2 && (cols & 2u)) tma_load_3d(sb + kBox, mb, &full[stage], x, 0, d.w);
                }
              }
              __syncwarp();
              if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
              }
            }
          }
          __syncwarp();
        }
      }
      ROLE_T0(t_ds);
      if (!claimed) describe(claim(), nxt_e, nxt_ij);   // no passes, or an abort before the claim point
      cur_e = nxt_e;
      cur_ij = nxt_ij;
      ROLE_ADD(12, t_ds);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (warp 1) ----------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0, sm_idx = 0;
    uint32_t acc_phase = 0, sm_phase = 0;
    unsigned long long nst = 0;
    int last_prod = -1;
    // All MMAs of a stage (4 K-steps of 32 bytes; split: hi lo and lo hi into the
    // correction accumulator ds, then hi hi into d) and the stage's commit, issued back
    // to back by one elected lane: N = 128, or N = 64 on the column half c. The
    // descriptors of the stage's boxes are formed once; a K-step adds 2 (32 bytes >> 4)
    // to the address field, which stays below 2^14 for every stage of the ring. Issuing
    // each MMA under its own election and warp sync cost ~115 cycles per 128 x 128 MMA
    // against 64 for this form (measured on this GPU).
    auto stage_mmas = [&](uint32_t st, uint32_t cols, uint32_t d, uint32_t ds, uint32_t accb, uint32_t accs,
                          uint64_t *done) {
      const bool both = cols == 3u;
      const uint32_t c = cols == 2u ? 1u : 0u;
      const uint32_t boff = both ? 0u : c * kBox, doff = both ? 0u : 64u * c;
      const uint32_t id = both ? cm.idesc : cm.idesc64;
      const uint64_t dAhi = desc_sw128(st + R::kAhi), dBhi = desc_sw128(st + R::kBhi + boff);
      const uint64_t dAlo = SPLIT ? desc_sw128(st + R::kAlo) : 0ull;
      const uint64_t dBlo = SPLIT ? desc_sw128(st + R::kBlo + boff) : 0ull;
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
          if (SPLIT) {
            if (TF32) {
              mma_tf32(ds + doff, dAhi + 2 * kk, dBlo + 2 * kk, id, kk ? 1u : accs);
              mma_tf32(ds + doff, dAlo + 2 * kk, dBhi + 2 * kk, id, 1u);
            } else {
              mma_f16(ds + doff, dAhi + 2 * kk, dBlo + 2 * kk, id, kk ? 1u : accs);
              mma_f16(ds + doff, dAlo + 2 * kk, dBhi + 2 * kk, id, 1u);
            }
          }
          if (TF32) mma_tf32(d + doff, dAhi + 2 * kk, dBhi + 2 * kk, id, kk ? 1u : accb);
          else mma_f16(d + doff, dAhi + 2 * kk, dBhi + 2 * kk, id, kk ? 1u : accb);
        }
        mma_commit(done);
      }
      __syncwarp();
    };
    auto commit = [&](uint64_t *bar) {
      if (elect_one()) mma_commit(bar);
      __syncwarp();
    };
    int qs = 0;
    uint32_t qp = 0;
    for (;;) {
      int4 e;
      uint32_t ij_unused;
      ROLE_T0(t_tk);
      const bool more = take(qs, qp, e, ij_unused);
      ROLE_ADD(10, t_tk);
      if (!more) break;
      {
        const int pr = e.x;
        const uint2 mt = make_uint2((uint32_t)e.z, (uint32_t)e.w);
        const uint32_t np = item_passes(prods[pr], mt, cm.status);
        if (lane == 0 && pr != last_prod) {
          // stage counts are kept per product: flush this CTA's count of the previous one
          if (last_prod >= 0 && nst) atomicAdd(prods[last_prod].mma_stages, nst);
          nst = 0;
          last_prod = pr;
        }
        // plain: one accumulator per item; split: a fresh hi hi accumulator for every
        // pass and one correction accumulator for the item
        const int chains = SPLIT ? (int)np : 1;
        const int per_chain = SPLIT ? cm.chunks : (int)np * cm.chunks;
        bool small_ok = true;
        if (SPLIT && !aborted()) {
          ROLE_T0(t_ws);
          small_ok = wwait(&sme[sm_idx], sm_phase ^ 1u);
          ROLE_ADD(3, t_ws);
          tc_fence_after();
        }
        const uint32_t ds = tmem + R::kSmallCol + (uint32_t)sm_idx * 128u;   // split: hi lo + lo hi
        uint32_t acc_small = 0;
        ROLE_COUNT(8);
        for (int p = 0; p < chains && !aborted(); p++) {
          ROLE_T0(t_wa);
          const bool ok_a = wwait(&acce[acc], acc_phase ^ 1u);
          ROLE_ADD(3, t_wa);
          if (ok_a) {
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)acc * 128u;   // plain, or split hi hi
            uint32_t acc_big = 0;
            for (int t = 0; t < per_chain; t++) {
              ROLE_T0(t_wf);
              const bool ok_f = wwait(&full[stage], phase);
              ROLE_ADD(2, t_wf);
              if (!ok_f) break;
              tc_fence_after();
              const uint32_t cols = s_cols[stage];
              const uint32_t st = base + stage * R::kStageBytes;
              ROLE_T0(t_is);
              stage_mmas(st, cols, d, ds, acc_big, acc_small, &empty[stage]);
              acc_big = 1;
              acc_small = 1;
              ROLE_ADD(4, t_is);
              ROLE_COUNT(9);
              nst += (SPLIT ? 3u : 1u) * (cols == 3u ? 2u : 1u);   // 128 x 64 x chunk MMA chains
              if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
              }
            }
            commit(&accf[acc]);
          }
          if (SPLIT && ++acc == kAcc) {
            acc = 0;
            acc_phase ^= 1u;
          }
        }
        if (SPLIT) {
          if (small_ok) commit(&smf[sm_idx]);   // after the item's last MMA
          if (++sm_idx == kSmall) {
            sm_idx = 0;
            sm_phase ^= 1u;
          }
        }
        __syncwarp();
        if (!SPLIT && ++acc == kAcc) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
    }
    if (lane == 0 && last_prod >= 0 && nst) atomicAdd(prods[last_prod].mma_stages, nst);
  } else if (warp >= 2) {
    // ---------------- epilogue (warps 2-9) ----------------
    // Two warps per TMEM lane quarter: warp w reads lanes 32 (w % 4) .. + 31 (the rows
    // it may access) and the 64 accumulator columns of its half, (w - 2) / 4: leaf 64,
    // output block column c = half; leaf 128, columns 64 half .. + 63 of the block.
    const int ew = warp - 2;
    const int slice = warp & 3;            // TMEM lanes 32 * slice .. + 31
    const int half = ew >> 2;              // accumulator columns 64 * half .. + 63
    const int row = 32 * slice + lane;     // accumulator row
    const uint32_t lanes = (uint32_t)(32 * slice) << 16;
    int acc = 0, sm_idx = 0;
    uint32_t acc_phase = 0, sm_phase = 0;
    int qs = 0;
    uint32_t qp = 0;
    for (;;) {
      int4 e;
      uint32_t ij;
      ROLE_T0(t_tk);
      const bool more = take(qs, qp, e, ij);
      if (warp == 2) ROLE_ADD(14, t_tk);
      if (!more) break;
      {
        const int pr = e.x;
        const ProdDesc &P = prods[pr];
        const int qd = LEAF == 64 ? 0 : (e.y & 3);
        const uint32_t I = ij >> 16, J = ij & 0xFFFFu;
        const uint2 mt = make_uint2((uint32_t)e.z, (uint32_t)e.w);
        uint32_t touched = mt.y >> 24;   // quadrants with a product
        if (LEAF == 128) touched = touched ? (1u << qd) : 0u;
        // split: the hi hi products of each pass arrive in an accumulator of their own and
        // are summed here in FP32 (round to nearest) in the order of the plan, then the
        // item's corrections are added
        float run[64];
        if (SPLIT) {
          const uint32_t first = mt.x;
          const uint32_t np = item_passes(P, mt, cm.status);
          const int oob = P.nb * P.nb;
#pragma unroll
          for (int x = 0; x < 64; x++) run[x] = 0.f;
          bool all_ok = true;
          // this warp's 64 columns x 32 lanes from two TMEM column chunks, one wait for both
          auto add2 = [&](uint32_t d) {
            uint32_t v[32], w[32];
            tmem_ld32_nowait(d + (uint32_t)(half * 64), v);
            tmem_ld32_nowait(d + (uint32_t)(half * 64 + 32), w);
            tmem_wait_ld();
#pragma unroll
            for (int x = 0; x < 32; x++) {
              run[x] += __uint_as_float(v[x]);
              run[32 + x] += __uint_as_float(w[x]);
            }
          };
          int4 pl = make_int4(0, 0, 0, 0);
          for (uint32_t p = 0; p < np; p++) {
            if ((p & 31u) == 0u && p + lane < np) pl = P.plan[(int64_t)first + p + lane];
            const uint32_t cols = p == 0 ? 3u : __shfl_sync(0xffffffffu, pass_cols<LEAF>(pl, oob), p & 31u);
            ROLE_T0(t_ep);
            bool ok = mbar_wait(&accf[acc], acc_phase, &s_abort);
            if (warp == 2 && lane == 0) ROLE_ADD(6, t_ep);
            if (!ok) {
              s_abort = 1;
              flag_error(cm.status, DEV_TIMEOUT);
            }
            ok = __all_sync(0xffffffffu, ok);
            all_ok = all_ok && ok;
            if (ok) {
              tc_fence_after();
              // a column half this pass left alone is skipped (leaf 128 passes cover both)
              if ((cols >> half) & 1u) add2(tmem + lanes + (uint32_t)acc * 128u);
            }
            tc_fence_before();
            mbar_arrive(&acce[acc]);
            if (++acc == kAcc) {
              acc = 0;
              acc_phase ^= 1u;
            }
          }
          ROLE_T0(t_es);
          bool ok = mbar_wait(&smf[sm_idx], sm_phase, &s_abort);
          if (warp == 2 && lane == 0) ROLE_ADD(6, t_es);
          if (!ok) {
            s_abort = 1;
            flag_error(cm.status, DEV_TIMEOUT);
          }
          ok = __all_sync(0xffffffffu, ok);
          all_ok = all_ok && ok;
          if (ok && np > 0) {
            tc_fence_after();
            add2(tmem + lanes + R::kSmallCol + (uint32_t)sm_idx * 128u);
          }
          tc_fence_before();
          mbar_arrive(&sme[sm_idx]);
          if (++sm_idx == kSmall) {
            sm_idx = 0;
            sm_phase ^= 1u;
          }
          if (!all_ok) touched = 0;
        } else {
          ROLE_T0(t_ea);
          bool ok = mbar_wait(&accf[acc], acc_phase, &s_abort);
          if (warp == 2 && lane == 0) ROLE_ADD(6, t_ea);
          if (!ok) {
            s_abort = 1;
            flag_error(cm.status, DEV_TIMEOUT);
          }
          ok = __all_sync(0xffffffffu, ok);   // warp-uniform: the TMEM loads are warp-collective
          if (!ok) touched = 0;
          tc_fence_after();
        }
        ROLE_T0(t_fin);
        const int a = LEAF == 64 ? row / 64 : (qd >> 1);
        const int c = LEAF == 64 ? half : (qd & 1);
        const int r = LEAF == 64 ? row % 64 : row;
        const int i = (int)(2 * I) + a, j = (int)(2 * J) + c;
        const int col0 = LEAF == 64 ? 0 : half * 64;   // this warp's first column of block (i, j)
        // squared norm of the warp's part in double-float: f^2 = pp + e exactly, TwoSum
        // accumulation
        // the warp's 64 columns in registers; plain forms: both TMEM chunks behind one
        // wait, and the accumulator handed back to the MMA warp before the stores
        uint32_t v[2][32];
        if (SPLIT) {
#pragma unroll
          for (int x = 0; x < 32; x++) {
            v[0][x] = __float_as_uint(run[x]);
            v[1][x] = __float_as_uint(run[32 + x]);
          }
        } else {
          const uint32_t d = tmem + lanes + (uint32_t)acc * 128u + (uint32_t)(half * 64);
          tmem_ld32_nowait(d, v[0]);
          tmem_ld32_nowait(d + 32u, v[1]);
          tmem_wait_ld();
          tc_fence_before();
          mbar_arrive(&acce[acc]);
        }
        // squared norm: two TwoSum chains (even and odd columns) as the lanes of f32x2
        uint64_t Sh = f2(0.f, 0.f), Sl = f2(0.f, 0.f);
        const uint64_t kNeg1 = f2(-1.f, -1.f);
        if (((touched >> (a * 2 + c)) & 1u) && i < P.nb && j < P.nb) {   // warp-uniform
          // the warp's 32 rows of block (i, j) go through shared memory 16 columns at a
          // time, so that each store instruction covers whole 64-byte row pieces
          float *blk = P.C + ((int64_t)i * P.nb + j) * LEAF * LEAF + (int64_t)(r - lane) * LEAF;
          float(*sb)[17] = s_epi[ew];
          // symmetric product: block (j, i) = (i, j)^T from the same staged piece
          const bool mir = P.sym && i < j;
          float *blkT = P.C + ((int64_t)j * P.nb + i) * LEAF * LEAF + (r - lane);
#pragma unroll
          for (int hh = 0; hh < 2; hh++) {   // 32-column units of the warp's 64 columns
#pragma unroll
            for (int g = 0; g < 2; g++) {
              const int cb = col0 + hh * 32 + g * 16;   // first column of the piece
#pragma unroll
              for (int x = 0; x < 16; x++) sb[lane][x] = __uint_as_float(v[hh][g * 16 + x]);
              __syncwarp();
#pragma unroll
              for (int it = 0; it < 4; it++) {   // rows rl, columns cb + c4 .. + 3
                const int rl = it * 8 + (lane >> 2), c4 = (lane & 3) * 4;
                *reinterpret_cast<float4 *>(blk + (int64_t)rl * LEAF + cb + c4) =
                    make_float4(sb[rl][c4], sb[rl][c4 + 1], sb[rl][c4 + 2], sb[rl][c4 + 3]);
              }
              if (mir) {   // row cb + cl of block (j, i), its 32 columns r - lane ..
#pragma unroll
                for (int it = 0; it < 4; it++) {
                  const int cl = it * 4 + (lane >> 3), r4 = (lane & 7) * 4;
                  *reinterpret_cast<float4 *>(blkT + (int64_t)(cb + cl) * LEAF + r4) =
                      make_float4(sb[r4][cl], sb[r4 + 1][cl], sb[r4 + 2][cl], sb[r4 + 3][cl]);
                }
              }
              __syncwarp();
            }
#pragma unroll
            for (int x = 0; x < 32; x += 2) {
              // f^2 = pp + e exactly (npp = -pp); TwoSum of Sh + pp, (Sh - (t - bb)) + (pp - bb)
              // with pp - bb = -(npp + bb)
              const uint64_t fv = f2(__uint_as_float(v[hh][x]), __uint_as_float(v[hh][x + 1]));
              const uint64_t npp = mul2(fv, mul2(fv, kNeg1));
              const uint64_t ee = fma2(fv, fv, npp);
              const uint64_t t = sub2(Sh, npp);
              const uint64_t bb = sub2(t, Sh);
              Sl = add2(Sl, add2(sub2(sub2(Sh, sub2(t, bb)), add2(npp, bb)), ee));
              Sh = t;
            }
          }
        }
        float sh[2], sl[2];
        f2_get(Sh, sh[0], sh[1]);
        f2_get(Sl, sl[0], sl[1]);
        df_add(sh[0], sl[0], sh[1], sl[1]);
        // squared Frobenius norms of the written blocks: rows -> warp -> fixed order
        {
          float H = sh[0], L = sl[0];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, H, off), l2 = __shfl_xor_sync(0xffffffffu, L, off);
            df_add(H, L, h2, l2);
          }
          if (lane == 0) s_norm[slice][half] = (double)H + (double)L;
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (warp == 2 && lane < 4) {
          if (LEAF == 64) {
            const int aa = lane >> 1, cc = lane & 1;
            const int ii = (int)(2 * I) + aa, jj = (int)(2 * J) + cc;
            if (((touched >> (aa * 2 + cc)) & 1u) && ii < P.nb && jj < P.nb) {
              const double v2 = s_norm[2 * aa][cc] + s_norm[2 * aa + 1][cc];
              P.leaf_norm2C[(int64_t)ii * P.NB + jj] = v2;
              P.nzC[(int64_t)ii * P.NB + jj] = 1;
              if (P.sym && ii < jj) {
                P.leaf_norm2C[(int64_t)jj * P.NB + ii] = v2;
                P.nzC[(int64_t)jj * P.NB + ii] = 1;
              }
            }
          } else if (lane == 0) {
            if (((touched >> qd) & 1u) && i < P.nb && j < P.nb) {
              const double v2 = ((s_norm[0][0] + s_norm[0][1]) + (s_norm[1][0] + s_norm[1][1])) +
                                ((s_norm[2][0] + s_norm[2][1]) + (s_norm[3][0] + s_norm[3][1]));
              P.leaf_norm2C[(int64_t)i * P.NB + j] = v2;
              P.nzC[(int64_t)i * P.NB + j] = 1;
              if (P.sym && i < j) {
                P.leaf_norm2C[(int64_t)j * P.NB + i] = v2;
                P.nzC[(int64_t)j * P.NB + i] = 1;
              }
            }
          }
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (warp == 2) ROLE_ADD(13, t_fin);
        if (!SPLIT && ++acc == kAcc) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
    }
  }
  if (lane == 0 && warp <= 2) ROLE_ADD(warp == 0 ? 1 : warp == 1 ? 5 : 7, t_kernel);
  tc_fence_before();
  __syncthreads();
  if (s_abort) {
    // error path only: give copies and MMAs already issued time to land before the
    // shared memory and TMEM are released
    const unsigned long long t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) __nanosleep(1000);
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// 3-D view [leaf][row][col] of a tree's leaf copy; boxes of one 128-byte K chunk.
bool make_map(CUtensorMap *m, const void *data, int elem, int b, int nb) {
  auto fn = encode_fn();
  if (!fn || !data) return false;
  const CUtensorMapDataType dt = elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  cuuint64_t dims[3] = {(cuuint64_t)b, (cuuint64_t)b, (cuuint64_t)nb * nb};
  cuuint64_t strides[2] = {(cuuint64_t)b * elem, (cuuint64_t)b * b * elem};
  cuuint32_t box[3] = {(cuuint32_t)(128 / elem), (cuuint32_t)b, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, dt, 3, const_cast<void *>(data), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int LEAF, bool TF32, bool SPLIT>
cudaError_t run(const ProdDesc *table, int nprod, const TcCommon &cm, int sm_count, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_leaf_tc<LEAF, TF32, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  k_leaf_tc<LEAF, TF32, SPLIT><<<sm_count, kThreads, kSmemBytes, s>>>(table, nprod, cm);
  return cudaGetLastError();
}

// Host image of one product's descriptor.
bool fill_desc(ProdDesc *d, spamm_tree A, spamm_tree B, spamm_tree C, int prec) {
  const bool tf32 = tf32_prec(prec);
  const int elem = tf32 ? 4 : 2;
  const int row = tf32 ? CK_TF32 : prec == SPAMM_FP16 ? CK_FP16 : CK_BF16;
  const bool bsym = (B->flags & SPAMM_SYMMETRIC) != 0;
  const int brow = bsym ? row : row + 1;
  const int alo = tf32 ? CK_TF32LO : CK_BF16LO;
  const int blo = bsym ? alo : alo + 1;
  memset(d, 0, sizeof *d);
  if (!make_map(&d->mA, A->copy[row], elem, A->b, A->nb) || !make_map(&d->mB, B->copy[brow], elem, B->b, B->nb))
    return false;
  if (split_prec(prec)) {
    if (!make_map(&d->mAlo, A->copy[alo], elem, A->b, A->nb) || !make_map(&d->mBlo, B->copy[blo], elem, B->b, B->nb))
      return false;
  } else {
    d->mAlo = d->mA;
    d->mBlo = d->mB;
  }
  d->items = C->items;
  d->plan = C->plan;
  d->cap_plan = C->cap_plan;
  d->cap_items = C->cap_items;
  d->gij = C->tiers[C->kmax].gij;
  d->ngroups = &C->counts->ngroups[C->kmax];
  d->C = (float *)C->copy[CK_F32];
  d->nzC = C->nz;
  d->leaf_norm2C = C->norm2 + level_offset(C->kmax);
  d->mma_stages = &C->counts->mma_tiles;
  d->work_ctr = &C->counts->work_ctr;
  d->nb = C->nb;
  d->NB = C->NB;
  d->sym = C->sym_product ? 1 : 0;
  return true;
}

TcCommon common_of(int prec, int b, uint32_t *status) {
  const bool tf32 = tf32_prec(prec);
  const int elem = tf32 ? 4 : 2;
  TcCommon cm{};
  const uint32_t fmt = tf32 ? kFmtTF32 : prec == SPAMM_FP16 ? kFmtF16 : kFmtBF16;
  cm.idesc = make_idesc(fmt, 128, 128);
  cm.idesc64 = make_idesc(fmt, 128, 64);
  cm.chunks = b * elem / 128;
  cm.chunk_elems = 128 / elem;
  cm.status = status;
  return cm;
}

cudaError_t run_table(const ProdDesc *table, int nprod, int b, int prec, uint32_t *status, int sm_count,
                      cudaStream_t s) {
  const TcCommon cm = common_of(prec, b, status);
  const bool tf32 = tf32_prec(prec), pp = split_prec(prec);
  if (b == 64) {
    if (pp) return tf32 ? run<64, true, true>(table, nprod, cm, sm_count, s) : run<64, false, true>(table, nprod, cm, sm_count, s);
    return tf32 ? run<64, true, false>(table, nprod, cm, sm_count, s) : run<64, false, false>(table, nprod, cm, sm_count, s);
  }
  if (b == 128) {
    if (pp) return tf32 ? run<128, true, true>(table, nprod, cm, sm_count, s) : run<128, false, true>(table, nprod, cm, sm_count, s);
    return tf32 ? run<128, true, false>(table, nprod, cm, sm_count, s) : run<128, false, false>(table, nprod, cm, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

static_assert(sizeof(ProdDesc) <= kTcDescBytes, "descriptor storage of a tree");

size_t tc_desc_bytes() { return sizeof(ProdDesc); }

cudaError_t launch_leaf_tc(spamm_tree A, spamm_tree B, spamm_tree C, int prec, uint32_t *dev_status,
                           int sm_count, cudaStream_t s) {
  ProdDesc d;
  if (!fill_desc(&d, A, B, C, prec)) return cudaErrorInvalidValue;
  if (!C->tc_desc_dev) {
    cudaError_t e = cudaMalloc(&C->tc_desc_dev, sizeof(ProdDesc));
    if (e != cudaSuccess) return e;
    C->tc_desc_valid = false;
  }
  // upload only when the descriptor changed (other operands or a new tree)
  if (!C->tc_desc_valid || memcmp(C->tc_desc_host, &d, sizeof d) != 0) {
    memcpy(C->tc_desc_host, &d, sizeof d);
    cudaError_t e = cudaMemcpyAsync(C->tc_desc_dev, C->tc_desc_host, sizeof d, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    C->tc_desc_valid = true;
  }
  return run_table((const ProdDesc *)C->tc_desc_dev, 1, C->b, prec, dev_status, sm_count, s);
}

// Batched products: host descriptors of `count` products (same leaf size and
// precision) are written to `host_table` (pinned); the caller copies them to a device
// table and launches over it.
cudaError_t fill_leaf_tc_table(const spamm_tree *A, const spamm_tree *B, const spamm_tree *C, int count, int prec,
                               void *host_table) {
  if (count < 1 || count > kMaxProd) return cudaErrorInvalidValue;
  ProdDesc *h = (ProdDesc *)host_table;
  for (int q = 0; q < count; q++)
    if (!fill_desc(&h[q], A[q], B[q], C[q], prec)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_leaf_tc_table(const void *dev_table, int count, int b, int prec, uint32_t *dev_status,
                                 int sm_count, cudaStream_t s) {
  if (count < 1 || count > kMaxProd) return cudaErrorInvalidValue;
  return run_table((const ProdDesc *)dev_table, count, b, prec, dev_status, sm_count, s);
}

#ifdef SPAMM_LEAF_ROLE_CYCLES
// The per-role counters of the probe build: copy them to `host` (1024 x 10 unsigned
// 64-bit values, row = CTA) or, with reset != 0, zero them.
extern "C" __attribute__((visibility("default"))) int spamm_leaf_role_cycles(void *host, int reset) {
  if (reset) {
    static unsigned long long zero[1024][16] = {};
    return (int)cudaMemcpyToSymbol(g_role_cycles, zero, sizeof zero);
  }
  return (int)cudaMemcpyFromSymbol(host, g_role_cycles, sizeof(unsigned long long) * 1024 * 16);
}
#endif
