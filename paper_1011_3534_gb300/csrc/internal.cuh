// Internal declarations of the SpAMM CUDA library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <list>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/spamm.h"

// Device-side status bits (ctx->dev_status), set with atomicOr by kernels.
enum : uint32_t {
  DEV_TIMEOUT = 1u << 0,    // a bounded spin-wait ran out
  DEV_OVERFLOW = 1u << 1,   // a tier's entry list exceeded its capacity
  DEV_BADARG = 1u << 2,     // a kernel found an index outside its buffers
};

// Internal tree flag: the product tree keeps an FP32 master (tensor-core precisions).
#define SPAMM_INTERNAL_F32 0x10000
// flag groups of the public API
constexpr int32_t kCopyFlags = SPAMM_KEEP_FP64 | SPAMM_COPY_TF32 | SPAMM_COPY_BF16 | SPAMM_COPY_FP16 |
                               SPAMM_COPY_BF16X3 | SPAMM_COPY_TF32X3;
constexpr int32_t kTreeFlags = SPAMM_HOST_INPUT | SPAMM_SYMMETRIC | SPAMM_NO_RIGHT | kCopyFlags;
constexpr int32_t kLowCopyFlags = kCopyFlags & ~SPAMM_KEEP_FP64;
inline bool split_prec(int prec) { return prec == SPAMM_BF16X3 || prec == SPAMM_TF32X3; }
inline bool tf32_prec(int prec) { return prec == SPAMM_TF32 || prec == SPAMM_TF32X3; }

// Bytes reserved in a product tree for its tensor-core launch descriptor (host image).
constexpr size_t kTcDescBytes = 1024;
constexpr int kBuildEvents = 64;

// Bounded waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kSpinLimitNs = 2000000000ull;

// Maximum entries of one tier's triple list (uint32 offsets, 31 bits).
constexpr int64_t kEntryCap = int64_t(1) << 30;

constexpr int kSideStreams = 8;   // concurrent per-product work of a batch

struct BatchGraph {                // a captured batched product, replayed with new taus
  std::vector<uintptr_t> key;      // precision and the trees it was captured for
  int count = 0;
  double *tau_host = nullptr, *tau_dev = nullptr;
  void *table_host = nullptr, *table_dev = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  cudaEvent_t tau_copied = nullptr;   // the last copy out of tau_host has run
};

struct spamm_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  bool timing = false;
  std::string err;
  uint32_t *dev_status = nullptr;   // device word of DEV_* bits
  unsigned long long *dev_count = nullptr;   // one device counter (spamm_drop_blocks)
  int64_t launches = 0;
  // staging buffer for host input / output (device)
  void *stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // batched products
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t side_ev[kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr;
  // dense host output: a staging buffer and a copy stream, so that the device-to-host
  // copy of one result overlaps the context's later work
  void *stage_out = nullptr;
  size_t stage_out_bytes = 0;
  cudaStream_t d2h = nullptr;
  cudaEvent_t d2h_staged = nullptr, d2h_done = nullptr;
  bool d2h_pending = false;
  // page-locked host input: a staging buffer filled on a copy stream, so that the
  // transfer of the next input overlaps the context's work on the previous one
  // the norm pyramid of a spamm_multiply product runs on its own stream, overlapping
  // whatever the caller queues next that does not read the product (the next operand
  // rebuild, say); every call that may read a product waits for it first (settle)
  cudaStream_t pyr_stream = nullptr;
  cudaEvent_t pyr_ready = nullptr, pyr_done = nullptr;
  bool pyr_pending = false;
  void *stage_in = nullptr;
  size_t stage_in_bytes = 0;
  cudaStream_t h2d = nullptr;
  cudaEvent_t h2d_done = nullptr, stage_in_free = nullptr;
  bool stage_in_used = false;
  void *batch_host = nullptr, *batch_dev = nullptr;   // descriptor tables (pinned / device)
  cudaEvent_t batch_copied = nullptr;   // the last copy out of batch_host has run
  size_t batch_cap = 0;
  std::list<BatchGraph> graphs;
  std::map<int64_t, std::pair<int, double>> tuned;     // autotuner cache: leaf, ms
};

// Leaf copies a tree can hold. Index into spamm_tree_s::copy.
enum CopyKind : int {
  CK_F64 = 0,     // FP64 tiles (row orientation)
  CK_F32,         // FP32 tiles (product trees of tensor-core precisions)
  CK_TF32,        // TF32-rounded values in FP32 storage
  CK_TF32_T,      // ... transposed leaves
  CK_BF16,
  CK_BF16_T,
  CK_FP16,
  CK_FP16_T,
  CK_BF16LO,      // low half of the BF16 split
  CK_BF16LO_T,
  CK_TF32LO,      // low part of the TF32 split, in FP32 storage
  CK_TF32LO_T,
  CK_COUNT
};

inline int copy_elem_bytes(int ck) {
  switch (ck) {
    case CK_F64: return 8;
    case CK_F32: case CK_TF32: case CK_TF32_T: case CK_TF32LO: case CK_TF32LO_T: return 4;
    default: return 2;
  }
}

// Surviving triples of one tier: a group per output block (I, J) of the tier, each
// with its ascending list of K (uint16).
struct TierList {
  uint32_t *gij = nullptr;     // (I << 16) | J
  uint32_t *gstart = nullptr;  // first entry of the group
  uint32_t *glen = nullptr;    // number of entries
  uint16_t *K = nullptr;       // entries
  int64_t cap_groups = 0, cap_entries = 0;
};

struct DevCounts {                     // device-resident counters of one product
  unsigned long long ngroups[SPAMM_MAX_LEVELS + 1];   // groups per tier list (index l+1)
  unsigned long long nentries[SPAMM_MAX_LEVELS + 1];  // entries per tier list (index l+1)
  unsigned long long tested[SPAMM_MAX_LEVELS];
  unsigned long long culled[SPAMM_MAX_LEVELS];
  unsigned long long leaf_products;
  unsigned long long mirror_products;  // triples of blocks i < j (mirrored to j > i)
  unsigned long long output_blocks;
  unsigned long long mma_tiles;        // leaf-kernel MMA chains issued, in 128 x 64 x chunk units
  unsigned long long npasses;          // passes of the tensor-core task plan
  unsigned long long mma_small;        // warp-level MMA instructions of the small-leaf kernel
  unsigned int tile_ctr[SPAMM_MAX_LEVELS + 2];        // dynamic tile counters
  unsigned int work_ctr;
  double culled_bound[SPAMM_MAX_LEVELS];
};

struct spamm_tree_s {
  spamm_ctx ctx = nullptr;
  int64_t n = 0;
  int32_t b = 0, nb = 0, NB = 0, kmax = 0;
  int32_t flags = 0;
  double *norm2 = nullptr;   // every tier: tier l at offset (4^l - 1) / 3, 2^l x 2^l
  double *norm = nullptr;    // sqrt of norm2, same layout
  uint8_t *nz = nullptr;     // NB x NB: 1 if tile storage holds leaf (i, j)
  unsigned int *pyr_ctr = nullptr;   // arrivals of the norm pyramid's region CTAs (0 between launches)
  void *copy[CK_COUNT] = {};
  // product trees
  bool is_product = false;
  bool sym_product = false;               // C = A A of a symmetric A, blocks i <= j computed
  bool depth_tau = false;                 // tier l of the cull tests against tau * 8^-l
  bool warp_tiles = false;                // leaf 64 tensor-core product in warp tiles (k_leaf_mma)
  int32_t prec = 0;
  double tau = 0;
  TierList tiers[SPAMM_MAX_LEVELS + 1];   // tiers[l + 1] lists tier l; tiers[0] the virtual root
  uint8_t *mask = nullptr;                // 8 child bits per entry of tier kmax - 1
  int64_t cap_mask = 0;
  double *bound_part = nullptr;           // per parent group partial culled bounds
  int64_t cap_bound = 0;
  uint64_t *look = nullptr;               // look-back tile status words
  int64_t cap_look = 0;
  DevCounts *counts = nullptr;            // device
  // task plan of the tensor-core leaf kernel (set by the last cull tier)
  int plan_mode = 0;                      // 0 none, 1 leaf 64, 2 leaf 128
  int4 *plan = nullptr;
  int64_t cap_plan = 0;
  uint2 *items = nullptr;
  int64_t cap_items = 0;
  void *tc_desc_dev = nullptr;            // device copy of the leaf kernel's descriptor
  alignas(64) unsigned char tc_desc_host[kTcDescBytes] = {};
  bool tc_desc_valid = false;
  spamm_stats_t host_stats{};
  bool stats_valid = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  // timing contexts: event pairs around the leaf-block kernel of the last kBuildEvents
  // builds (a ring), and how many were recorded since spamm_tree_build_ms last read them
  cudaEvent_t ev_build[kBuildEvents][2] = {};
  int build_pos = 0, build_count = 0;
};

// A symmetric product whose blocks j > i are written by k_mirror after the leaf kernel:
// FP64 and the warp-tile kernel (the tcgen05 forms write them in their epilogue).
inline bool mirror_after_leaf(const spamm_tree_s *C) {
  return C->prec == SPAMM_FP64 || C->b < 64 || C->warp_tiles;
}

__host__ __device__ inline int64_t level_offset(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }

// ---- launchers (each returns a cudaError_t from the launch) ----
cudaError_t launch_tree_build(spamm_tree t, const double *A, cudaStream_t s);
cudaError_t launch_pyramid(spamm_tree t, cudaStream_t s);
cudaError_t launch_mirror(spamm_tree C, cudaStream_t s);       // C_ji := C_ij^T for i < j
// Leaf blocks with ||T_ij||_F < tau dropped (presence and norm cleared; kept counted into
// *kept when not null), then the norm pyramid rebuilt.
cudaError_t launch_drop(spamm_tree t, double tau, unsigned long long *kept, cudaStream_t s);
cudaError_t launch_to_dense(spamm_tree t, double *out, cudaStream_t s);
cudaError_t launch_to_dense_f32(spamm_tree t, float *out, cudaStream_t s);
cudaError_t launch_cull(spamm_tree A, spamm_tree B, spamm_tree C, double tau, const double *tau_dev,
                        uint32_t *dev_status, int sm_count, cudaStream_t s, int *launches);
cudaError_t launch_leaf_f64(spamm_tree A, spamm_tree B, spamm_tree C, uint32_t *dev_status,
                            int sm_count, cudaStream_t s);
// Tensor-core leaf products of leaf 16 and 32 (warp-level MMA), any tensor-core precision.
cudaError_t launch_leaf_mma(spamm_tree A, spamm_tree B, spamm_tree C, int prec, uint32_t *dev_status,
                            int sm_count, cudaStream_t s);
cudaError_t launch_leaf_tc(spamm_tree A, spamm_tree B, spamm_tree C, int prec,
                           uint32_t *dev_status, int sm_count, cudaStream_t s);
cudaError_t launch_finish_stats(spamm_tree C, cudaStream_t s);
cudaError_t launch_tile_convert(spamm_tree t, cudaStream_t s);
int64_t cull_look_words(int kmax);
int64_t cull_bound_words(int kmax, int64_t *offsets);
int pyramid_launches(spamm_tree t);
// The context stream waits for a product's pyramid still running on its own stream.
spamm_status settle(spamm_ctx ctx);
cudaError_t sp2_x0(int64_t n, const int64_t *indptr, const int64_t *indices, const double *data, double emin,
                   double emax, double *X, cudaStream_t s);
size_t sp2_record_bytes();
cudaError_t sp2_step_finish(spamm_tree X, spamm_tree C, double n_occ, int step, void *rec, cudaStream_t s);
cudaError_t sp2_trace_only(spamm_tree X, int idx, void *rec, cudaStream_t s);
cudaError_t sp2_energy(spamm_tree X, int64_t n, const int64_t *indptr, const int64_t *indices,
                       const double *data, double *partial, void *rec, cudaStream_t s);
void sp2_read_record(const void *host_rec, int steps, spamm_sp2_result *out);
double *sp2_tau_slot(void *rec, int step);   // device address of the record's tau of a step
// log10 of a step's error budget, loosened by its branch margin (into *out, device)
cudaError_t sp2_margin_budget(spamm_tree X, int step, void *rec, double n_occ, double mu_ref, double gain_max,
                              double log10_budget, double *out, cudaStream_t s);
constexpr int kTreeFeatures = 34;            // per-tree part of the controller's features
size_t tc_desc_bytes();
// Batched tensor-core products: host descriptors of `count` products (same leaf size
// and precision) written to `host_table`, then one launch over a device copy of them.
cudaError_t fill_leaf_tc_table(const spamm_tree *A, const spamm_tree *B, const spamm_tree *C, int count, int prec,
                               void *host_table);
cudaError_t launch_leaf_tc_table(const void *dev_table, int count, int b, int prec, uint32_t *dev_status,
                                 int sm_count, cudaStream_t s);
spamm_status product_prepare(spamm_ctx ctx, spamm_tree A, spamm_tree B, double tau, spamm_prec prec,
                             int32_t flags, spamm_tree *C);
cudaError_t launch_feat_hist(spamm_tree t, float *out, cudaStream_t s);
cudaError_t launch_tau_select(spamm_mlp mm, const float *fa, const float *fb, const double *grid, const double *bound,
                              double log10_budget, double *tau_out, cudaStream_t s,
                              const double *log10_budget_dev = nullptr);
cudaError_t launch_flat_bound(spamm_tree A, spamm_tree B, const double *grid, int G, double *work, double *bound,
                              cudaStream_t s);
size_t bound_workspace_doubles(spamm_tree A);   // work + bound of launch_flat_bound on the 37-point grid
void tau_grid(double tau_min, double tau_max, double *grid);   // the 37 log-spaced tolerances
constexpr int kTauGrid = 37;
int mlp_inputs(spamm_mlp mm);
