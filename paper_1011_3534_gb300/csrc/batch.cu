// Batched products and the leaf-size autotuner (host side).
//
// spamm_multiply_batched runs the culls of all products concurrently on the context's
// side streams, then one persistent tensor-core launch per leaf size over every
// product's task plan (the kernel resolves each global item to its product through a
// descriptor table), then the products' norm pyramids. With SPAMM_GRAPH the whole
// sequence is captured once into a CUDA graph per set of trees and replayed; the cull
// kernels then read each product's tau from a device array refreshed before each replay.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "internal.cuh"

namespace {

spamm_status bfail(spamm_ctx ctx, spamm_status st, const char *msg) {
  ctx->err = msg;
  return st;
}

spamm_status bcuda(spamm_ctx ctx, cudaError_t e, const char *what) {
  ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SPAMM_ENOMEM : SPAMM_ECUDA;
}

#define BCK(call, what)                                  \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return bcuda(ctx, _e, what);  \
  } while (0)

spamm_status ensure_side_streams(spamm_ctx ctx) {
  if (ctx->side[0]) return SPAMM_OK;
  for (int i = 0; i < kSideStreams; i++) {
    BCK(cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking), "side stream");
    BCK(cudaEventCreateWithFlags(&ctx->side_ev[i], cudaEventDisableTiming), "side event");
  }
  BCK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "fork event");
  BCK(cudaEventCreateWithFlags(&ctx->batch_copied, cudaEventDisableTiming), "batch table event");
  return SPAMM_OK;
}

// fork: side streams wait for the main stream; join: the main stream waits for them
spamm_status fork(spamm_ctx ctx, int used) {
  BCK(cudaEventRecord(ctx->fork_ev, ctx->stream), "fork");
  for (int i = 0; i < used; i++) BCK(cudaStreamWaitEvent(ctx->side[i], ctx->fork_ev, 0), "fork");
  return SPAMM_OK;
}

spamm_status join(spamm_ctx ctx, int used) {
  for (int i = 0; i < used; i++) {
    BCK(cudaEventRecord(ctx->side_ev[i], ctx->side[i]), "join");
    BCK(cudaStreamWaitEvent(ctx->stream, ctx->side_ev[i], 0), "join");
  }
  return SPAMM_OK;
}

spamm_status ensure_batch_tables(spamm_ctx ctx, int count) {
  const size_t need = tc_desc_bytes() * (size_t)count;
  if (ctx->batch_cap >= need) return SPAMM_OK;
  if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
  if (ctx->batch_dev) cudaFree(ctx->batch_dev);
  ctx->batch_host = nullptr;
  ctx->batch_dev = nullptr;
  ctx->batch_cap = 0;
  BCK(cudaStreamSynchronize(ctx->stream), "batch tables");
  BCK(cudaMallocHost(&ctx->batch_host, need), "batch tables");
  BCK(cudaMalloc(&ctx->batch_dev, need), "batch tables");
  ctx->batch_cap = need;
  return SPAMM_OK;
}

}  // namespace

// The launch sequence of a batch: culls (side streams), tensor-core launches per leaf
// size, FP64 leaf kernels, pyramids (side streams). tau_dev may be null (host taus).
static spamm_status batch_sequence(spamm_ctx ctx, const spamm_tree *A, const spamm_tree *B, const double *tau,
                                   const double *tau_dev, int count, spamm_prec prec, spamm_tree *C,
                                   void *host_table, void *dev_table, cudaEvent_t copied) {
  const bool tc = prec != SPAMM_FP64;
  const int used = std::min(count, kSideStreams);
  spamm_status st = fork(ctx, used);
  if (st != SPAMM_OK) return st;
  for (int p = 0; p < count; p++) {
    int launches = 0;
    BCK(launch_cull(A[p], B[p], C[p], tau ? tau[p] : 0.0, tau_dev ? tau_dev + p : nullptr, ctx->dev_status,
                    ctx->sm_count, ctx->side[p % used], &launches),
        "batch: cull");
    ctx->launches += launches;
  }
  st = join(ctx, used);
  if (st != SPAMM_OK) return st;
  if (tc) {
    // one persistent launch per leaf size over all products of that size; the
    // descriptors of all launches go over in one copy
    struct Chunk { size_t off; int m, leaf; };
    std::vector<Chunk> chunks;
    size_t off = 0;
    for (int leaf : {64, 128}) {
      std::vector<spamm_tree> a, b, c;
      for (int p = 0; p < count; p++)
        if (C[p]->b == leaf && !C[p]->warp_tiles) {
          a.push_back(A[p]);
          b.push_back(B[p]);
          c.push_back(C[p]);
        }
      for (size_t s0 = 0; s0 < c.size(); s0 += 1024) {
        const int m = (int)std::min<size_t>(1024, c.size() - s0);
        BCK(fill_leaf_tc_table(a.data() + s0, b.data() + s0, c.data() + s0, m, prec,
                               (unsigned char *)host_table + off),
            "batch: descriptors");
        chunks.push_back({off, m, leaf});
        off += tc_desc_bytes() * m;
      }
    }
    BCK(cudaMemcpyAsync(dev_table, host_table, off, cudaMemcpyHostToDevice, ctx->stream), "batch: descriptors");
    if (copied) BCK(cudaEventRecord(copied, ctx->stream), "batch: descriptors");
    for (const Chunk &k : chunks) {
      BCK(launch_leaf_tc_table((unsigned char *)dev_table + k.off, k.m, k.leaf, prec, ctx->dev_status, ctx->sm_count,
                               ctx->stream),
          "batch: leaf launch");
      ctx->launches++;
    }
    for (int p = 0; p < count; p++)   // warp tiles (leaves 16, 32, and 64 on request): one launch per product
      if (C[p]->b < 64 || C[p]->warp_tiles) {
        BCK(launch_leaf_mma(A[p], B[p], C[p], prec, ctx->dev_status, ctx->sm_count, ctx->stream), "batch: leaf launch");
        ctx->launches++;
      }
  } else {
    for (int p = 0; p < count; p++) {
      BCK(launch_leaf_f64(A[p], B[p], C[p], ctx->dev_status, ctx->sm_count, ctx->stream), "batch: leaf launch");
      ctx->launches++;
    }
  }
  st = fork(ctx, used);
  if (st != SPAMM_OK) return st;
  for (int p = 0; p < count; p++) {
    BCK(launch_pyramid(C[p], ctx->side[p % used]), "batch: pyramid");
    ctx->launches += pyramid_launches(C[p]);
  }
  return join(ctx, used);
}

extern "C" spamm_status spamm_tree_update_batched(spamm_ctx ctx, int32_t count, const spamm_tree *trees,
                                                  const double *const *A, int32_t flags) {
  if (!ctx) return SPAMM_EINVAL;
  if (count < 1 || !trees || !A) return bfail(ctx, SPAMM_EINVAL, "update_batched: bad arguments");
  if (flags != 0) return bfail(ctx, SPAMM_EINVAL, "update_batched: flags must be 0 (device inputs)");
  for (int p = 0; p < count; p++) {
    if (!trees[p] || !A[p]) return bfail(ctx, SPAMM_EINVAL, "update_batched: null tree or input");
    if (trees[p]->ctx != ctx) return bfail(ctx, SPAMM_EINVAL, "update_batched: a tree of another context");
    if (trees[p]->is_product) return bfail(ctx, SPAMM_EINVAL, "update_batched: a product tree");
  }
  spamm_status st = ensure_side_streams(ctx);
  if (st != SPAMM_OK) return st;
  const int used = std::min(count, kSideStreams);
  // largest first, each to the stream with the least work so far (elements)
  std::vector<int> order(count);
  for (int p = 0; p < count; p++) order[p] = p;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return trees[a]->n > trees[b]->n; });
  std::vector<double> load(used, 0.0);
  st = fork(ctx, used);
  if (st != SPAMM_OK) return st;
  for (int p : order) {
    const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[q] += (double)trees[p]->n * (double)trees[p]->n;
    BCK(launch_tree_build(trees[p], A[p], ctx->side[q]), "update_batched: launch");
    BCK(launch_pyramid(trees[p], ctx->side[q]), "update_batched: launch");
    ctx->launches += 1 + pyramid_launches(trees[p]);
  }
  return join(ctx, used);
}

extern "C" spamm_status spamm_multiply_batched(spamm_ctx ctx, const spamm_tree *A, const spamm_tree *B,
                                               const double *tau, int32_t count, spamm_prec prec, int32_t flags,
                                               spamm_tree *C) {
  if (!ctx) return SPAMM_EINVAL;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!A || !B || !tau || !C || count < 1) return bfail(ctx, SPAMM_EINVAL, "batched: bad arguments");
  if (flags & ~(kLowCopyFlags | SPAMM_SYMMETRIC | SPAMM_NO_RIGHT | SPAMM_GRAPH | SPAMM_WARP_TILES))
    return bfail(ctx, SPAMM_EINVAL, "batched: unknown flag bits");
  if (flags & kLowCopyFlags) return bfail(ctx, SPAMM_EUNSUPPORTED, "batched: leaf copies of the products are not produced");
  spamm_status st = ensure_side_streams(ctx);
  if (st != SPAMM_OK) return st;
  // every product validated, created or checked, workspace allocated (before any capture)
  for (int p = 0; p < count; p++) {
    st = product_prepare(ctx, A[p], B[p], tau[p], prec, flags & (SPAMM_SYMMETRIC | SPAMM_NO_RIGHT | SPAMM_WARP_TILES),
                         &C[p]);
    if (st != SPAMM_OK) return st;
  }
  st = ensure_batch_tables(ctx, count);
  if (st != SPAMM_OK) return st;
  if (!(flags & SPAMM_GRAPH)) {
    // the pinned table is rewritten only after the previous call's copy out of it ran
    BCK(cudaEventSynchronize(ctx->batch_copied), "batched: descriptor table");
    return batch_sequence(ctx, A, B, tau, nullptr, count, prec, C, ctx->batch_host, ctx->batch_dev,
                          ctx->batch_copied);
  }

  // CUDA graph: one per (precision, trees) set, replayed with fresh taus
  std::vector<uintptr_t> key;
  key.push_back((uintptr_t)prec);
  for (int p = 0; p < count; p++) {
    key.push_back((uintptr_t)A[p]);
    key.push_back((uintptr_t)B[p]);
    key.push_back((uintptr_t)C[p]);
  }
  BatchGraph *g = nullptr;
  for (BatchGraph &bg : ctx->graphs)
    if (bg.key == key) g = &bg;
  if (!g) {
    if (ctx->stream == nullptr) return bfail(ctx, SPAMM_EUNSUPPORTED, "batched: graphs need a non-default context stream");
    ctx->graphs.emplace_back();
    g = &ctx->graphs.back();
    g->key = key;
    g->count = count;
    BCK(cudaMallocHost(&g->tau_host, sizeof(double) * count), "batched: graph taus");
    BCK(cudaMalloc(&g->tau_dev, sizeof(double) * count), "batched: graph taus");
    BCK(cudaMallocHost(&g->table_host, tc_desc_bytes() * count), "batched: graph table");
    BCK(cudaMalloc(&g->table_dev, tc_desc_bytes() * count), "batched: graph table");
    BCK(cudaEventCreateWithFlags(&g->tau_copied, cudaEventDisableTiming), "batched: graph taus");
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "batched: capture");
    const int64_t l0 = ctx->launches;
    // the captured copy reads table_host at every replay; it is written once, here
    st = batch_sequence(ctx, A, B, nullptr, g->tau_dev, count, prec, C, g->table_host, g->table_dev, nullptr);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != SPAMM_OK) {
      if (graph) cudaGraphDestroy(graph);
      ctx->graphs.pop_back();
      return st;
    }
    if (e != cudaSuccess) {
      ctx->graphs.pop_back();
      return bcuda(ctx, e, "batched: capture");
    }
    g->launches = ctx->launches - l0;
    ctx->launches = l0;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->graphs.pop_back();
      return bcuda(ctx, e, "batched: instantiate");
    }
  }
  BCK(cudaEventSynchronize(g->tau_copied), "batched: taus");   // the previous replay's taus were copied
  memcpy(g->tau_host, tau, sizeof(double) * count);
  BCK(cudaMemcpyAsync(g->tau_dev, g->tau_host, sizeof(double) * count, cudaMemcpyHostToDevice, ctx->stream),
      "batched: taus");
  BCK(cudaEventRecord(g->tau_copied, ctx->stream), "batched: taus");
  BCK(cudaGraphLaunch(g->exec, ctx->stream), "batched: graph launch");
  ctx->launches += g->launches;
  for (int p = 0; p < count; p++) {
    C[p]->is_product = true;
    C[p]->prec = prec;
    C[p]->tau = tau[p];
    C[p]->stats_valid = false;
  }
  return SPAMM_OK;
}

// Leaf-size autotuner: builds the tree of A at every candidate leaf size, times the
// product A A (tree build included) with CUDA events, and keeps the fastest; results are
// cached per (log2 n, precision, decade of tau).
namespace {

// Times spamm_tree_update + spamm_multiply of A A for each (leaf, multiply flags)
// candidate (the best of three repetitions after a first one) and returns the fastest.
spamm_status tune_candidates(spamm_ctx ctx, const double *A, int64_t n, double tau, spamm_prec prec, int32_t flags,
                             const std::vector<std::pair<int, int32_t>> &cand, int *best_leaf, int32_t *best_flags,
                             double *best_ms) {
  const bool tc = prec != SPAMM_FP64;
  const int32_t copy = tc ? (prec == SPAMM_TF32 ? SPAMM_COPY_TF32 : prec == SPAMM_FP16 ? SPAMM_COPY_FP16
                             : prec == SPAMM_BF16X3 ? SPAMM_COPY_BF16X3
                             : prec == SPAMM_TF32X3 ? SPAMM_COPY_TF32X3 : SPAMM_COPY_BF16)
                          : SPAMM_KEEP_FP64;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "tune: event");
  BCK(cudaEventCreate(&e1), "tune: event");
  int best = -1;
  int32_t bflags = 0;
  double bms = 0;
  for (const auto &cf : cand) {
    const int leaf = cf.first;
    spamm_tree t = nullptr, c = nullptr;
    spamm_status st = spamm_tree_build(ctx, A, n, leaf, copy | (flags & (SPAMM_SYMMETRIC | SPAMM_HOST_INPUT)), &t);
    if (st != SPAMM_OK) continue;
    double ms = 1e30;
    for (int rep = 0; rep < 4 && st == SPAMM_OK; rep++) {
      cudaEventRecord(e0, ctx->stream);
      st = spamm_tree_update(t, A, flags & SPAMM_HOST_INPUT);
      if (st == SPAMM_OK) st = spamm_multiply(ctx, t, t, tau, prec, cf.second, &c);
      cudaEventRecord(e1, ctx->stream);
      if (st == SPAMM_OK && cudaEventSynchronize(e1) == cudaSuccess && rep > 0) {
        float v = 0;
        cudaEventElapsedTime(&v, e0, e1);
        ms = std::min(ms, (double)v);
      }
    }
    if (c) spamm_tree_free(c);
    spamm_tree_free(t);
    if (st == SPAMM_OK && (best < 0 || ms < bms)) {
      best = leaf;
      bflags = cf.second;
      bms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return bfail(ctx, SPAMM_EUNSUPPORTED, "tune: no candidate ran");
  *best_leaf = best;
  *best_flags = bflags;
  *best_ms = bms;
  return SPAMM_OK;
}

int64_t tune_key(int64_t n, double tau, spamm_prec prec, int shape) {
  int lg = 0;
  while ((int64_t(1) << lg) < n) lg++;
  const int tdec = tau > 0 ? (int)std::floor(std::log10(tau)) : -400;
  return (((int64_t)lg * 16 + (int)prec) * 1000 + (tdec + 500)) * 2 + shape;
}

}  // namespace

extern "C" spamm_status spamm_tune_leaf(spamm_ctx ctx, const double *A, int64_t n, double tau, spamm_prec prec,
                                        int32_t flags, int32_t *leaf_out, double *ms_out) {
  if (!ctx) return SPAMM_EINVAL;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!A || !leaf_out || n < 1 || !(tau >= 0.0)) return bfail(ctx, SPAMM_EINVAL, "tune: bad arguments");
  const int64_t key = tune_key(n, tau, prec, 0);
  auto it = ctx->tuned.find(key);
  if (it == ctx->tuned.end()) {
    int leaf = 0;
    int32_t f = 0;
    double ms = 0;
    spamm_status st = tune_candidates(ctx, A, n, tau, prec, flags, {{16, 0}, {32, 0}, {64, 0}, {128, 0}}, &leaf, &f, &ms);
    if (st != SPAMM_OK) return st;
    it = ctx->tuned.emplace(key, std::make_pair(leaf, ms)).first;
  }
  *leaf_out = it->second.first;
  if (ms_out) *ms_out = it->second.second;
  return SPAMM_OK;
}

extern "C" spamm_status spamm_tune_shape(spamm_ctx ctx, const double *A, int64_t n, double tau, spamm_prec prec,
                                         int32_t flags, int32_t *leaf_out, int32_t *tile_flags_out, double *ms_out) {
  if (!ctx) return SPAMM_EINVAL;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!A || !leaf_out || !tile_flags_out || n < 1 || !(tau >= 0.0)) return bfail(ctx, SPAMM_EINVAL, "tune: bad arguments");
  const int64_t key = tune_key(n, tau, prec, 1);
  auto it = ctx->tuned.find(key);
  if (it == ctx->tuned.end()) {
    std::vector<std::pair<int, int32_t>> cand = {{16, 0}, {32, 0}, {64, 0}, {128, 0}};
    if (prec != SPAMM_FP64) cand.insert(cand.begin() + 3, {64, SPAMM_WARP_TILES});
    int leaf = 0;
    int32_t f = 0;
    double ms = 0;
    spamm_status st = tune_candidates(ctx, A, n, tau, prec, flags, cand, &leaf, &f, &ms);
    if (st != SPAMM_OK) return st;
    // the shape is kept in the leaf slot's sign: negative = warp tiles
    it = ctx->tuned.emplace(key, std::make_pair(f ? -leaf : leaf, ms)).first;
  }
  const int v = it->second.first;
  *leaf_out = v < 0 ? -v : v;
  *tile_flags_out = v < 0 ? SPAMM_WARP_TILES : 0;
  if (ms_out) *ms_out = it->second.second;
  return SPAMM_OK;
}
