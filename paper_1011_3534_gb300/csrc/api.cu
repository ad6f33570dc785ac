// C ABI of the SpAMM library: contexts, trees, the product, counters, exports.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

spamm_status fail(spamm_ctx ctx, spamm_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

spamm_status cuda_fail(spamm_ctx ctx, cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(ctx, SPAMM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(ctx, SPAMM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                              \
  do {                                              \
    cudaError_t _e = (call);                        \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, what); \
  } while (0)

bool valid_leaf(int32_t b) { return b == 16 || b == 32 || b == 64 || b == 128; }

template <typename T>
cudaError_t dmalloc(T **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  return cudaMalloc((void **)p, bytes);
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

// Which leaf copies a flag word asks for; transposed copies only when the tree may be a
// right operand and is not declared symmetric.
void wanted_copies(int32_t flags, bool want[CK_COUNT]) {
  for (int k = 0; k < CK_COUNT; k++) want[k] = false;
  const bool right_t = !(flags & SPAMM_SYMMETRIC) && !(flags & SPAMM_NO_RIGHT);
  if (flags & SPAMM_KEEP_FP64) want[CK_F64] = true;
  if (flags & SPAMM_COPY_TF32) { want[CK_TF32] = true; want[CK_TF32_T] = right_t; }
  if (flags & SPAMM_COPY_BF16) { want[CK_BF16] = true; want[CK_BF16_T] = right_t; }
  if (flags & SPAMM_COPY_FP16) { want[CK_FP16] = true; want[CK_FP16_T] = right_t; }
  if (flags & SPAMM_COPY_BF16X3) {
    want[CK_BF16] = true;
    want[CK_BF16LO] = true;
    want[CK_BF16_T] = right_t;
    want[CK_BF16LO_T] = right_t;
  }
  if (flags & SPAMM_COPY_TF32X3) {
    want[CK_TF32] = true;
    want[CK_TF32LO] = true;
    want[CK_TF32_T] = right_t;
    want[CK_TF32LO_T] = right_t;
  }
}

void shape(int64_t n, int32_t b, int32_t *nb, int32_t *NB, int32_t *kmax) {
  *nb = (int32_t)((n + b - 1) / b);
  *NB = 1;
  *kmax = 0;
  while (*NB < *nb) {
    *NB *= 2;
    (*kmax)++;
  }
}

void free_tree_memory(spamm_tree t) {
  dfree(t->norm2);
  dfree(t->norm);
  dfree(t->nz);
  dfree(t->pyr_ctr);
  for (int k = 0; k < CK_COUNT; k++) dfree(t->copy[k]);
  for (int l = 0; l <= SPAMM_MAX_LEVELS; l++) {
    dfree(t->tiers[l].gij);
    dfree(t->tiers[l].gstart);
    dfree(t->tiers[l].glen);
    dfree(t->tiers[l].K);
  }
  dfree(t->mask);
  dfree(t->bound_part);
  dfree(t->look);
  dfree(t->counts);
  dfree(t->plan);
  dfree(t->items);
  dfree(t->tc_desc_dev);
  for (int k = 0; k < 3; k++)
    if (t->ev[k]) cudaEventDestroy(t->ev[k]);
  for (int q = 0; q < kBuildEvents; q++)
    for (int k = 0; k < 2; k++)
      if (t->ev_build[q][k]) cudaEventDestroy(t->ev_build[q][k]);
}

spamm_status alloc_tree(spamm_ctx ctx, int64_t n, int32_t b, int32_t flags, spamm_tree *out) {
  spamm_tree t = new (std::nothrow) spamm_tree_s();
  if (!t) return fail(ctx, SPAMM_ENOMEM, "host allocation failed");
  t->ctx = ctx;
  t->n = n;
  t->b = b;
  t->flags = flags;
  shape(n, b, &t->nb, &t->NB, &t->kmax);
  if (t->kmax >= SPAMM_MAX_LEVELS - 1 || t->NB > 65536) {
    const int32_t NB = t->NB;
    delete t;
    return fail(ctx, SPAMM_EUNSUPPORTED, "n / leaf too large (NB = %d)", NB);
  }
  const size_t levels = (size_t)level_offset(t->kmax + 1);
  cudaError_t e = dmalloc(&t->norm2, levels * sizeof(double));
  if (e == cudaSuccess) e = dmalloc(&t->norm, levels * sizeof(double));
  if (e == cudaSuccess) e = dmalloc(&t->nz, (size_t)t->NB * t->NB);
  if (e == cudaSuccess) e = dmalloc(&t->pyr_ctr, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(t->pyr_ctr, 0, sizeof(unsigned int), ctx->stream);
  bool want[CK_COUNT];
  wanted_copies(flags, want);
  const size_t elems = (size_t)t->nb * t->nb * (size_t)b * b;
  for (int k = 0; k < CK_COUNT && e == cudaSuccess; k++)
    if (want[k]) e = dmalloc(&t->copy[k], elems * copy_elem_bytes(k));
  if (e != cudaSuccess) {
    free_tree_memory(t);
    delete t;
    return cuda_fail(ctx, e, "tree allocation");
  }
  *out = t;
  return SPAMM_OK;
}

// Worst-case workspace of a product tree: tier l holds at most 4^l groups and
// min(8^l, kEntryCap) entries, so no product can overflow it below that cap.
spamm_status alloc_product_workspace(spamm_ctx ctx, spamm_tree C) {
  if (C->counts) return SPAMM_OK;
  cudaError_t e = cudaSuccess;
  // tiers[0]: the virtual tier -1 (one group, one entry)
  for (int li = 0; li <= C->kmax && e == cudaSuccess; li++) {
    TierList &T = C->tiers[li];
    const int l = li - 1;
    T.cap_groups = l < 0 ? 1 : (int64_t(1) << (2 * l));
    T.cap_entries = l < 0 ? 1 : std::min<int64_t>(int64_t(1) << (3 * l), kEntryCap);
    e = dmalloc(&T.gij, T.cap_groups * 4);
    if (e == cudaSuccess) e = dmalloc(&T.gstart, T.cap_groups * 4);
    if (e == cudaSuccess) e = dmalloc(&T.glen, T.cap_groups * 4);
    if (e == cudaSuccess) e = dmalloc(&T.K, T.cap_entries * 2);
  }
  if (e == cudaSuccess) {
    C->cap_mask = C->tiers[C->kmax].cap_entries;
    e = dmalloc(&C->mask, (size_t)C->cap_mask);
  }
  std::vector<int64_t> offs(C->kmax + 1);
  if (e == cudaSuccess) {
    C->cap_bound = cull_bound_words(C->kmax, offs.data());
    e = dmalloc(&C->bound_part, (size_t)C->cap_bound * 8 + (C->kmax + 1) * sizeof(int64_t));
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(C->bound_part + C->cap_bound, offs.data(), (C->kmax + 1) * sizeof(int64_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    C->cap_look = cull_look_words(C->kmax);
    e = dmalloc(&C->look, (size_t)C->cap_look * 8);
  }
  if (e == cudaSuccess) e = dmalloc(&C->counts, sizeof(DevCounts));
  if (e == cudaSuccess && (C->flags & SPAMM_INTERNAL_F32) && (C->b == 64 || C->b == 128)) {
    // task plan of the tensor-core leaf kernel: at most 4 passes per tier kmax-1 entry at
    // leaf 64 (two per child k), 8 at leaf 128; one item per group or per output block
    const int64_t ent = C->tiers[C->kmax].cap_entries;
    C->cap_plan = std::min<int64_t>(ent * (C->b == 64 ? 4 : 8), int64_t(1) << 31);
    C->cap_items = C->tiers[C->kmax].cap_groups * (C->b == 64 ? 1 : 4);
    e = dmalloc(&C->plan, (size_t)C->cap_plan * sizeof(int4));
    if (e == cudaSuccess) e = dmalloc(&C->items, (size_t)C->cap_items * sizeof(uint2));
    C->plan_mode = C->b == 64 ? 1 : 2;
  }
  if (e == cudaSuccess && ctx->timing)
    for (int k = 0; k < 3 && e == cudaSuccess; k++) e = cudaEventCreate(&C->ev[k]);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "product workspace allocation");
  return SPAMM_OK;
}

spamm_status check_device_status(spamm_ctx ctx) {
  spamm_status sst = settle(ctx);
  if (sst != SPAMM_OK) return sst;
  if (ctx->d2h_pending) {   // an asynchronous dense output is part of the context's work
    CK(cudaStreamWaitEvent(ctx->stream, ctx->d2h_done, 0), "output copy wait");
    ctx->d2h_pending = false;
  }
  uint32_t st = 0;
  CK(cudaMemcpyAsync(&st, ctx->dev_status, 4, cudaMemcpyDeviceToHost, ctx->stream), "status read");
  CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  if (st) {
    CK(cudaMemsetAsync(ctx->dev_status, 0, 4, ctx->stream), "status reset");
    if (st & DEV_TIMEOUT) return fail(ctx, SPAMM_ETIMEOUT, "a device-side wait timed out");
    if (st & DEV_OVERFLOW) return fail(ctx, SPAMM_ERANGE, "a tier list exceeded its capacity");
    return fail(ctx, SPAMM_ECUDA, "device-side argument check failed (0x%x)", st);
  }
  return SPAMM_OK;
}

// Device address of a page-locked, mapped host array (cudaMallocHost, cudaHostAlloc,
// cudaHostRegister); nullptr for pageable memory.
void *mapped_view(const void *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Page-locked host input: copied on the context's input stream into the input staging
// buffer once the kernel that read the previous input is done with it; the context
// stream waits for the copy. The caller records stage_in_free after the reading kernel.
spamm_status stage_pinned_input(spamm_ctx ctx, const double *A, size_t bytes, const double **src) {
  if (!ctx->h2d) {
    CK(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking), "input copy stream");
    CK(cudaEventCreateWithFlags(&ctx->h2d_done, cudaEventDisableTiming), "input copy event");
    CK(cudaEventCreateWithFlags(&ctx->stage_in_free, cudaEventDisableTiming), "input copy event");
  }
  if (ctx->stage_in_bytes < bytes) {
    CK(cudaStreamSynchronize(ctx->h2d), "input copy stream");
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    if (ctx->stage_in) cudaFree(ctx->stage_in);
    ctx->stage_in = nullptr;
    ctx->stage_in_bytes = 0;
    ctx->stage_in_used = false;
    CK(cudaMalloc(&ctx->stage_in, bytes), "input staging buffer");
    ctx->stage_in_bytes = bytes;
  }
  if (ctx->stage_in_used) CK(cudaStreamWaitEvent(ctx->h2d, ctx->stage_in_free, 0), "input copy wait");
  CK(cudaMemcpyAsync(ctx->stage_in, A, bytes, cudaMemcpyHostToDevice, ctx->h2d), "host to device copy");
  CK(cudaEventRecord(ctx->h2d_done, ctx->h2d), "input copy event");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->h2d_done, 0), "input copy wait");
  ctx->stage_in_used = true;
  *src = (const double *)ctx->stage_in;
  return SPAMM_OK;
}

spamm_status ensure_stage(spamm_ctx ctx, size_t bytes) {
  if (ctx->stage_bytes >= bytes) return SPAMM_OK;
  if (ctx->stage) {
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
  }
  CK(cudaMalloc(&ctx->stage, bytes), "staging buffer");
  ctx->stage_bytes = bytes;
  return SPAMM_OK;
}

}  // namespace

spamm_status settle(spamm_ctx ctx) {
  if (!ctx->pyr_pending) return SPAMM_OK;
  CK(cudaStreamWaitEvent(ctx->stream, ctx->pyr_done, 0), "pyramid wait");
  ctx->pyr_pending = false;
  return SPAMM_OK;
}



static int32_t COPY_FLAG_OF(spamm_prec p) {
  switch (p) {
    case SPAMM_TF32: return SPAMM_COPY_TF32;
    case SPAMM_BF16: return SPAMM_COPY_BF16;
    case SPAMM_FP16: return SPAMM_COPY_FP16;
    case SPAMM_BF16X3: return SPAMM_COPY_BF16X3;
    case SPAMM_TF32X3: return SPAMM_COPY_TF32X3;
    default: return SPAMM_KEEP_FP64;
  }
}

extern "C" {

spamm_status spamm_ctx_create(int device, void *cuda_stream, int32_t timing, spamm_ctx *out) {
  if (!out) return SPAMM_EINVAL;
  *out = nullptr;
  spamm_ctx ctx = new (std::nothrow) spamm_ctx_s();
  if (!ctx) return SPAMM_ENOMEM;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->dev_status, 4);
  if (e == cudaSuccess) e = cudaMemset(ctx->dev_status, 0, 4);
  if (e != cudaSuccess) {
    if (ctx->dev_status) cudaFree(ctx->dev_status);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? SPAMM_ENOMEM : SPAMM_ECUDA;
  }
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->timing = timing != 0;
  *out = ctx;
  return SPAMM_OK;
}

spamm_status spamm_ctx_destroy(spamm_ctx ctx) {
  if (!ctx) return SPAMM_EINVAL;
  settle(ctx);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pyr_stream) {
    cudaStreamSynchronize(ctx->pyr_stream);
    cudaStreamDestroy(ctx->pyr_stream);
  }
  if (ctx->pyr_ready) cudaEventDestroy(ctx->pyr_ready);
  if (ctx->pyr_done) cudaEventDestroy(ctx->pyr_done);
  for (BatchGraph &g : ctx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.tau_host) cudaFreeHost(g.tau_host);
    if (g.table_host) cudaFreeHost(g.table_host);
    if (g.tau_dev) cudaFree(g.tau_dev);
    if (g.table_dev) cudaFree(g.table_dev);
    if (g.tau_copied) cudaEventDestroy(g.tau_copied);
  }
  for (int i = 0; i < kSideStreams; i++) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->side_ev[i]) cudaEventDestroy(ctx->side_ev[i]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->d2h) {
    cudaStreamSynchronize(ctx->d2h);
    cudaStreamDestroy(ctx->d2h);
  }
  if (ctx->d2h_staged) cudaEventDestroy(ctx->d2h_staged);
  if (ctx->h2d) {
    cudaStreamSynchronize(ctx->h2d);
    cudaStreamDestroy(ctx->h2d);
  }
  if (ctx->h2d_done) cudaEventDestroy(ctx->h2d_done);
  if (ctx->stage_in_free) cudaEventDestroy(ctx->stage_in_free);
  if (ctx->stage_in) cudaFree(ctx->stage_in);
  if (ctx->d2h_done) cudaEventDestroy(ctx->d2h_done);
  if (ctx->stage_out) cudaFree(ctx->stage_out);
  if (ctx->batch_copied) cudaEventDestroy(ctx->batch_copied);
  if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
  if (ctx->batch_dev) cudaFree(ctx->batch_dev);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->dev_count) cudaFree(ctx->dev_count);
  if (ctx->dev_status) cudaFree(ctx->dev_status);
  delete ctx;
  return SPAMM_OK;
}

spamm_status spamm_sync(spamm_ctx ctx) {
  if (!ctx) return SPAMM_EINVAL;
  return check_device_status(ctx);
}

const char *spamm_last_error(spamm_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t spamm_kernel_launches(spamm_ctx ctx) { return ctx ? ctx->launches : -1; }

// The leaf-block kernel, bracketed by the next event pair of the tree's ring on a
// timing context.
static cudaError_t timed_tree_build(spamm_tree t, const double *src, cudaStream_t s) {
  if (!t->ctx->timing) return launch_tree_build(t, src, s);
  cudaEvent_t *ev = t->ev_build[t->build_pos];
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; k++)
    if (!ev[k]) e = cudaEventCreate(&ev[k]);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = launch_tree_build(t, src, s);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) {
    t->build_pos = (t->build_pos + 1) % kBuildEvents;
    t->build_count = std::min(t->build_count + 1, kBuildEvents);
  }
  return e;
}

spamm_status spamm_tree_build(spamm_ctx ctx, const double *A, int64_t n, int32_t leaf,
                              int32_t flags, spamm_tree *out) {
  if (!ctx) return SPAMM_EINVAL;
  if (!A || !out) return fail(ctx, SPAMM_EINVAL, "tree_build: null pointer");
  if (n < 1) return fail(ctx, SPAMM_EINVAL, "tree_build: n = %lld < 1", (long long)n);
  if (!valid_leaf(leaf)) return fail(ctx, SPAMM_EINVAL, "tree_build: leaf %d not in {16,32,64,128}", leaf);
  if (flags & ~kTreeFlags) return fail(ctx, SPAMM_EINVAL, "tree_build: unknown flag bits 0x%x", flags);
  *out = nullptr;
  spamm_tree t = nullptr;
  spamm_status st = alloc_tree(ctx, n, leaf, flags, &t);
  if (st != SPAMM_OK) return st;
  const double *src = A;
  const bool pinned = (flags & SPAMM_HOST_INPUT) && mapped_view(A) != nullptr;
  if (pinned) {
    st = stage_pinned_input(ctx, A, (size_t)n * n * sizeof(double), &src);
    if (st != SPAMM_OK) {
      free_tree_memory(t);
      delete t;
      return st;
    }
  } else if (flags & SPAMM_HOST_INPUT) {
    st = ensure_stage(ctx, (size_t)n * n * sizeof(double));
    if (st != SPAMM_OK) {
      free_tree_memory(t);
      delete t;
      return st;
    }
    cudaError_t e = cudaMemcpyAsync(ctx->stage, A, (size_t)n * n * sizeof(double),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      free_tree_memory(t);
      delete t;
      return cuda_fail(ctx, e, "tree_build: host to device copy");
    }
    src = (const double *)ctx->stage;
  }
  cudaError_t e = timed_tree_build(t, src, ctx->stream);
  if (e == cudaSuccess && pinned) e = cudaEventRecord(ctx->stage_in_free, ctx->stream);
  if (e == cudaSuccess) e = launch_pyramid(t, ctx->stream);
  ctx->launches += 1 + pyramid_launches(t);
  if (e != cudaSuccess) {
    free_tree_memory(t);
    delete t;
    return cuda_fail(ctx, e, "tree_build: launch");
  }
  *out = t;
  return SPAMM_OK;
}

spamm_status spamm_tree_update(spamm_tree t, const double *A, int32_t flags) {
  if (!t) return SPAMM_EINVAL;
  spamm_ctx ctx = t->ctx;
  if (!A) return fail(ctx, SPAMM_EINVAL, "tree_update: null input");
  if (t->is_product) return fail(ctx, SPAMM_EINVAL, "tree_update: product trees cannot be rebuilt");
  if (flags & ~SPAMM_HOST_INPUT) return fail(ctx, SPAMM_EINVAL, "tree_update: only SPAMM_HOST_INPUT is accepted");
  const double *src = A;
  const bool pinned = (flags & SPAMM_HOST_INPUT) && mapped_view(A) != nullptr;
  if (pinned) {
    spamm_status st = stage_pinned_input(ctx, A, (size_t)t->n * t->n * sizeof(double), &src);
    if (st != SPAMM_OK) return st;
  } else if (flags & SPAMM_HOST_INPUT) {
    spamm_status st = ensure_stage(ctx, (size_t)t->n * t->n * sizeof(double));
    if (st != SPAMM_OK) return st;
    CK(cudaMemcpyAsync(ctx->stage, A, (size_t)t->n * t->n * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream), "tree_update: host to device copy");
    src = (const double *)ctx->stage;
  }
  CK(timed_tree_build(t, src, ctx->stream), "tree_update: launch");
  if (pinned) CK(cudaEventRecord(ctx->stage_in_free, ctx->stream), "tree_update: event");
  CK(launch_pyramid(t, ctx->stream), "tree_update: launch");
  ctx->launches += 1 + pyramid_launches(t);
  return SPAMM_OK;
}

spamm_status spamm_tree_free(spamm_tree t) {
  if (!t) return SPAMM_EINVAL;
  settle(t->ctx);
  cudaStreamSynchronize(t->ctx->stream);
  free_tree_memory(t);
  delete t;
  return SPAMM_OK;
}

spamm_status spamm_tree_build_ms(spamm_tree t, float *ms) {
  if (!t) return SPAMM_EINVAL;
  spamm_ctx ctx = t->ctx;
  if (!ms) return fail(ctx, SPAMM_EINVAL, "tree_build_ms: null output");
  if (t->build_count == 0) return fail(ctx, SPAMM_EINVAL, "tree_build_ms: no timed build of this tree since the last read");
  double sum = 0.0;
  for (int k = 1; k <= t->build_count; k++) {
    cudaEvent_t *ev = t->ev_build[(t->build_pos - k + kBuildEvents) % kBuildEvents];
    float one = 0.f;
    CK(cudaEventSynchronize(ev[1]), "tree_build_ms: event");
    CK(cudaEventElapsedTime(&one, ev[0], ev[1]), "tree_build_ms: event");
    sum += one;
  }
  *ms = (float)(sum / t->build_count);
  t->build_count = 0;
  return SPAMM_OK;
}

spamm_status spamm_drop_blocks(spamm_tree t, double tau, int64_t *kept) {
  if (!t) return SPAMM_EINVAL;
  spamm_ctx ctx = t->ctx;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(ctx, SPAMM_EINVAL, "drop_blocks: tau must be finite and >= 0");
  if (kept) {
    if (!ctx->dev_count) CK(cudaMalloc(&ctx->dev_count, sizeof(unsigned long long)), "drop_blocks: counter");
    CK(cudaMemsetAsync(ctx->dev_count, 0, sizeof(unsigned long long), ctx->stream), "drop_blocks: counter");
  }
  CK(launch_drop(t, tau, kept ? ctx->dev_count : nullptr, ctx->stream), "drop_blocks: launch");
  ctx->launches += 1 + pyramid_launches(t);
  t->stats_valid = false;
  if (kept) {
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, ctx->dev_count, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "drop_blocks: copy");
    spamm_status st = check_device_status(ctx);
    if (st != SPAMM_OK) return st;
    *kept = (int64_t)h;
  }
  return SPAMM_OK;
}

spamm_status spamm_tree_info(spamm_tree t, int64_t *n, int32_t *leaf, int32_t *nb_padded,
                             int32_t *kmax) {
  if (!t) return SPAMM_EINVAL;
  if (n) *n = t->n;
  if (leaf) *leaf = t->b;
  if (nb_padded) *nb_padded = t->NB;
  if (kmax) *kmax = t->kmax;
  return SPAMM_OK;
}

spamm_status spamm_tree_norms(spamm_tree t, int32_t level, double *out) {
  if (!t) return SPAMM_EINVAL;
  spamm_ctx ctx = t->ctx;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!out || level < 0 || level > t->kmax)
    return fail(ctx, SPAMM_EINVAL, "tree_norms: level %d outside 0..%d", level, t->kmax);
  const size_t cnt = (size_t)1 << (2 * level);
  CK(cudaMemcpyAsync(out, t->norm2 + level_offset(level), cnt * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream), "tree_norms: copy");
  return check_device_status(ctx);
}

spamm_status spamm_tree_leaf_copy(spamm_tree t, int32_t which, void *out, int64_t bytes, int32_t out_is_host) {
  if (!t) return SPAMM_EINVAL;
  spamm_ctx ctx = t->ctx;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!out || which < 0 || which >= CK_COUNT || (out_is_host != 0 && out_is_host != 1))
    return fail(ctx, SPAMM_EINVAL, "tree_leaf_copy: bad arguments");
  if (!t->copy[which]) return fail(ctx, SPAMM_EINVAL, "tree_leaf_copy: the tree holds no copy %d", which);
  const int64_t need = (int64_t)t->nb * t->nb * t->b * t->b * copy_elem_bytes(which);
  if (bytes < need) return fail(ctx, SPAMM_ERANGE, "tree_leaf_copy: %lld bytes needed", (long long)need);
  CK(cudaMemcpyAsync(out, t->copy[which], (size_t)need, out_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     ctx->stream), "tree_leaf_copy: copy");
  return out_is_host ? check_device_status(ctx) : SPAMM_OK;
}

}  // extern "C"

namespace {

// Dense image of a tree in FP64 (f32 = false) or FP32: on the context's stream into
// device memory, or through the output staging buffer and the context's copy stream
// into host memory (the staging buffer is reused only after the previous copy out of it
// finished).
spamm_status to_dense_impl(spamm_tree t, void *out, int32_t out_is_host, bool f32, const char *name) {
  if (!t) return SPAMM_EINVAL;
  spamm_ctx ctx = t->ctx;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!out) return fail(ctx, SPAMM_EINVAL, "%s: null output", name);
  if (!t->copy[CK_F64] && !t->copy[CK_F32])
    return fail(ctx, SPAMM_EINVAL, "%s: the tree keeps no FP64/FP32 tiles (SPAMM_KEEP_FP64)", name);
  if (out_is_host < 0 || out_is_host > 2) return fail(ctx, SPAMM_EINVAL, "%s: out_is_host must be 0, 1 or 2", name);
  const size_t bytes = (size_t)t->n * t->n * (f32 ? sizeof(float) : sizeof(double));
  auto launch = [&](void *dst) {
    return f32 ? launch_to_dense_f32(t, (float *)dst, ctx->stream) : launch_to_dense(t, (double *)dst, ctx->stream);
  };
  if (!out_is_host) {
    CK(launch(out), "tree_to_dense: launch");
    ctx->launches++;
    return SPAMM_OK;
  }
  if (!ctx->d2h) {
    CK(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking), "tree_to_dense: copy stream");
    CK(cudaEventCreateWithFlags(&ctx->d2h_staged, cudaEventDisableTiming), "tree_to_dense: event");
    CK(cudaEventCreateWithFlags(&ctx->d2h_done, cudaEventDisableTiming), "tree_to_dense: event");
  }
  if (ctx->stage_out_bytes < bytes) {
    CK(cudaStreamSynchronize(ctx->d2h), "tree_to_dense: copy stream");
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    if (ctx->stage_out) cudaFree(ctx->stage_out);
    ctx->stage_out = nullptr;
    ctx->stage_out_bytes = 0;
    CK(cudaMalloc(&ctx->stage_out, bytes), "tree_to_dense: staging buffer");
    ctx->stage_out_bytes = bytes;
  }
  if (ctx->d2h_pending) CK(cudaStreamWaitEvent(ctx->stream, ctx->d2h_done, 0), "tree_to_dense: wait");
  CK(launch(ctx->stage_out), "tree_to_dense: launch");
  ctx->launches++;
  CK(cudaEventRecord(ctx->d2h_staged, ctx->stream), "tree_to_dense: event");
  CK(cudaStreamWaitEvent(ctx->d2h, ctx->d2h_staged, 0), "tree_to_dense: wait");
  CK(cudaMemcpyAsync(out, ctx->stage_out, bytes, cudaMemcpyDeviceToHost, ctx->d2h), "tree_to_dense: copy");
  CK(cudaEventRecord(ctx->d2h_done, ctx->d2h), "tree_to_dense: event");
  ctx->d2h_pending = true;
  if (out_is_host == 1) return check_device_status(ctx);
  return SPAMM_OK;
}

}  // namespace

extern "C" {

spamm_status spamm_tree_to_dense(spamm_tree t, double *out, int32_t out_is_host) {
  return to_dense_impl(t, out, out_is_host, false, "tree_to_dense");
}

spamm_status spamm_tree_to_dense_f32(spamm_tree t, float *out, int32_t out_is_host) {
  return to_dense_impl(t, out, out_is_host, true, "tree_to_dense_f32");
}

spamm_status multiply_impl(spamm_ctx ctx, spamm_tree A, spamm_tree B, double tau, const double *tau_dev,
                           spamm_prec prec, int32_t flags, spamm_tree *C, bool async_pyramid = false);

spamm_status spamm_multiply(spamm_ctx ctx, spamm_tree A, spamm_tree B, double tau,
                            spamm_prec prec, int32_t flags, spamm_tree *C) {
  return multiply_impl(ctx, A, B, tau, nullptr, prec, flags, C, true);
}

}  // extern "C"

// The product with tau either given on the host or read by the cull kernels from device
// memory (tau_dev, e.g. chosen on the device by the tolerance controller).
// Validates a product, creates or checks the output tree and its workspace, and marks it
// as the product of (A, B, tau, prec). No device work is queued.
spamm_status product_prepare(spamm_ctx ctx, spamm_tree A, spamm_tree B, double tau, spamm_prec prec,
                             int32_t flags, spamm_tree *C) {
  if (!ctx) return SPAMM_EINVAL;
  if (!A || !B || !C) return fail(ctx, SPAMM_EINVAL, "multiply: null handle");
  if (A->n != B->n || A->b != B->b)
    return fail(ctx, SPAMM_EINVAL, "multiply: operands differ (n %lld/%lld, leaf %d/%d)",
                (long long)A->n, (long long)B->n, A->b, B->b);
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(ctx, SPAMM_EINVAL, "multiply: tau must be finite and >= 0");
  if (flags & ~((kTreeFlags & ~SPAMM_HOST_INPUT) | SPAMM_SYM_PRODUCT | SPAMM_DEPTH_TAU | SPAMM_WARP_TILES))
    return fail(ctx, SPAMM_EINVAL, "multiply: unknown flag bits 0x%x", flags);
  if ((flags & SPAMM_WARP_TILES) && prec == SPAMM_FP64)
    return fail(ctx, SPAMM_EINVAL, "multiply: SPAMM_WARP_TILES is a tile shape of the tensor-core precisions");
  if ((flags & SPAMM_WARP_TILES) && A->b > 64)
    return fail(ctx, SPAMM_EUNSUPPORTED, "multiply: leaf %d has no warp-tile shape", A->b);
  const bool symp = (flags & SPAMM_SYM_PRODUCT) != 0;
  if (symp && (A != B || !(A->flags & SPAMM_SYMMETRIC)))
    return fail(ctx, SPAMM_EINVAL, "multiply: SPAMM_SYM_PRODUCT needs B == A built with SPAMM_SYMMETRIC");
  const bool tc = prec != SPAMM_FP64;
  if (prec < SPAMM_FP64 || prec > SPAMM_TF32X3) return fail(ctx, SPAMM_EINVAL, "multiply: unknown precision %d", (int)prec);
  if (!tc) {
    if (!A->copy[CK_F64] || !B->copy[CK_F64])
      return fail(ctx, SPAMM_EINVAL, "multiply: SPAMM_FP64 needs SPAMM_KEEP_FP64 operands");
  } else {
    int row = tf32_prec(prec) ? CK_TF32 : prec == SPAMM_FP16 ? CK_FP16 : CK_BF16;
    int rowT = row + 1;
    const int lo = prec == SPAMM_TF32X3 ? CK_TF32LO : CK_BF16LO;
    if (!A->copy[row] || (split_prec(prec) && !A->copy[lo]))
      return fail(ctx, SPAMM_EINVAL, "multiply: left operand lacks the leaf copy for this precision");
    const bool bsym = (B->flags & SPAMM_SYMMETRIC) != 0;
    if (bsym ? !B->copy[row] : !B->copy[rowT])
      return fail(ctx, SPAMM_EINVAL, "multiply: right operand lacks the leaf copy for this precision");
    if (split_prec(prec) && (bsym ? !B->copy[lo] : !B->copy[lo + 1]))
      return fail(ctx, SPAMM_EINVAL, "multiply: right operand lacks the lo copy of the split");
  }
  spamm_tree Ct = *C;
  const int32_t cflags = (flags & (kLowCopyFlags | SPAMM_SYMMETRIC | SPAMM_NO_RIGHT)) | (symp ? SPAMM_SYMMETRIC : 0) |
                         (tc ? SPAMM_INTERNAL_F32 : SPAMM_KEEP_FP64);
  if (!Ct) {
    spamm_status st = alloc_tree(ctx, A->n, A->b, cflags & kTreeFlags, &Ct);
    if (st != SPAMM_OK) return st;
    if (tc) {
      cudaError_t e = dmalloc(&Ct->copy[CK_F32], (size_t)Ct->nb * Ct->nb * Ct->b * Ct->b * 4);
      if (e != cudaSuccess) {
        free_tree_memory(Ct);
        delete Ct;
        return cuda_fail(ctx, e, "multiply: product allocation");
      }
    }
    Ct->flags = cflags;
  } else {
    if (Ct == A || Ct == B) return fail(ctx, SPAMM_EINVAL, "multiply: output aliases an operand");
    if (Ct->n != A->n || Ct->b != A->b) return fail(ctx, SPAMM_EINVAL, "multiply: reused output has another shape");
    bool want[CK_COUNT];
    wanted_copies(cflags & kTreeFlags, want);
    for (int k = 0; k < CK_COUNT; k++)
      if (want[k] && !Ct->copy[k]) return fail(ctx, SPAMM_EINVAL, "multiply: reused output lacks a requested copy");
    if (tc ? !Ct->copy[CK_F32] : !Ct->copy[CK_F64])
      return fail(ctx, SPAMM_EINVAL, "multiply: reused output was made for another precision class");
  }
  spamm_status st = alloc_product_workspace(ctx, Ct);
  if (st != SPAMM_OK) {
    if (!*C) { free_tree_memory(Ct); delete Ct; }
    return st;
  }
  *C = Ct;
  Ct->is_product = true;
  Ct->sym_product = symp;
  Ct->depth_tau = (flags & SPAMM_DEPTH_TAU) != 0;
  Ct->warp_tiles = (flags & SPAMM_WARP_TILES) != 0 && Ct->b == 64;
  if (symp) Ct->flags |= SPAMM_SYMMETRIC;
  Ct->prec = prec;
  Ct->tau = tau;
  Ct->stats_valid = false;
  return SPAMM_OK;
}

spamm_status multiply_impl(spamm_ctx ctx, spamm_tree A, spamm_tree B, double tau, const double *tau_dev,
                           spamm_prec prec, int32_t flags, spamm_tree *C, bool async_pyramid) {
  if (!ctx) return SPAMM_EINVAL;
  spamm_status pst = settle(ctx);
  if (pst != SPAMM_OK) return pst;
  pst = product_prepare(ctx, A, B, tau, prec, flags, C);
  if (pst != SPAMM_OK) return pst;
  spamm_tree Ct = *C;
  const bool tc = prec != SPAMM_FP64;
  const int32_t cflags = (flags & (kLowCopyFlags | SPAMM_SYMMETRIC | SPAMM_NO_RIGHT)) | (tc ? SPAMM_INTERNAL_F32 : SPAMM_KEEP_FP64);
  cudaStream_t s = ctx->stream;
  if (ctx->timing) CK(cudaEventRecord(Ct->ev[0], s), "event");
  int launches = 0;
  CK(launch_cull(A, B, Ct, tau, tau_dev, ctx->dev_status, ctx->sm_count, s, &launches), "multiply: cull launch");
  if (ctx->timing) CK(cudaEventRecord(Ct->ev[1], s), "event");
  if (tc && Ct->b >= 64 && !Ct->warp_tiles) {
    CK(launch_leaf_tc(A, B, Ct, prec, ctx->dev_status, ctx->sm_count, s), "multiply: leaf launch");
  } else if (tc) {
    CK(launch_leaf_mma(A, B, Ct, prec, ctx->dev_status, ctx->sm_count, s), "multiply: leaf launch");
  } else {
    CK(launch_leaf_f64(A, B, Ct, ctx->dev_status, ctx->sm_count, s), "multiply: leaf launch");
  }
  launches++;
  if (ctx->timing) CK(cudaEventRecord(Ct->ev[2], s), "event");
  if (Ct->sym_product && mirror_after_leaf(Ct)) {   // the tcgen05 forms mirror in their epilogue
    CK(launch_mirror(Ct, s), "multiply: mirror launch");
    launches++;
  }
  if (async_pyramid) {
    if (!ctx->pyr_stream) {
      CK(cudaStreamCreateWithFlags(&ctx->pyr_stream, cudaStreamNonBlocking), "multiply: pyramid stream");
      CK(cudaEventCreateWithFlags(&ctx->pyr_ready, cudaEventDisableTiming), "multiply: pyramid event");
      CK(cudaEventCreateWithFlags(&ctx->pyr_done, cudaEventDisableTiming), "multiply: pyramid event");
    }
    CK(cudaEventRecord(ctx->pyr_ready, s), "multiply: pyramid event");
    CK(cudaStreamWaitEvent(ctx->pyr_stream, ctx->pyr_ready, 0), "multiply: pyramid wait");
    CK(launch_pyramid(Ct, ctx->pyr_stream), "multiply: pyramid launch");
    CK(cudaEventRecord(ctx->pyr_done, ctx->pyr_stream), "multiply: pyramid event");
    ctx->pyr_pending = true;
  } else {
    CK(launch_pyramid(Ct, s), "multiply: pyramid launch");
  }
  launches += pyramid_launches(Ct);
  bool want[CK_COUNT];
  wanted_copies(cflags & kTreeFlags, want);
  bool any_copy = false;
  for (int k = CK_TF32; k < CK_COUNT; k++) any_copy |= want[k];
  if (any_copy) {
    CK(launch_tile_convert(Ct, s), "multiply: copy launch");
    launches++;
  }
  ctx->launches += launches;
  return SPAMM_OK;
}

extern "C" {

spamm_status spamm_stats(spamm_tree C, spamm_stats_t *out) {
  if (!C) return SPAMM_EINVAL;
  spamm_ctx ctx = C->ctx;
  if (settle(ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!out) return fail(ctx, SPAMM_EINVAL, "stats: null output");
  if (!C->is_product) return fail(ctx, SPAMM_EINVAL, "stats: not a product tree");
  if (!C->stats_valid) {
    // the culled-bound partials of the last product are summed here, on demand
    CK(launch_finish_stats(C, ctx->stream), "stats: reduce launch");
    ctx->launches++;
    DevCounts h;
    CK(cudaMemcpyAsync(&h, C->counts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "stats: copy");
    spamm_status st = check_device_status(ctx);
    if (st != SPAMM_OK) return st;
    spamm_stats_t &S = C->host_stats;
    memset(&S, 0, sizeof S);
    S.levels = C->kmax + 1;
    S.leaf = C->b;
    S.n = C->n;
    for (int l = 0; l <= C->kmax; l++) {
      S.tested[l] = (int64_t)h.tested[l];
      S.culled[l] = (int64_t)h.culled[l];
      S.culled_bound[l] = h.culled_bound[l];
    }
    S.leaf_products = (int64_t)h.leaf_products;
    S.mirrored_products = (int64_t)h.mirror_products;
    S.output_blocks = (int64_t)h.output_blocks;
    const double b = C->b;
    S.leaf_flops = 2.0 * b * b * b * (double)h.leaf_products;
    S.dense_equiv_flops = 2.0 * (double)C->n * (double)C->n * (double)C->n;
    // tensor-core kernel: counted in 128 x 64 x (128-byte K chunk) MMA chains (an N = 128
    // MMA of one operand pair is two, a split stage's three products three times that)
    const double chunk_k = tf32_prec(C->prec) ? 32.0 : 64.0;
    S.mma_flops = C->prec == SPAMM_FP64 ? S.leaf_flops : (double)h.mma_tiles * 2.0 * 128.0 * 64.0 * chunk_k;
    // small leaves: warp-level m16n8k16 (BF16, FP16) or m16n8k8 (TF32) instructions
    if (C->prec != SPAMM_FP64) S.mma_flops += (double)h.mma_small * 2.0 * 16.0 * 8.0 * (tf32_prec(C->prec) ? 8.0 : 16.0);
    S.prec = C->prec;
    S.tau = C->tau;
    if (ctx->timing && C->ev[0]) {
      float a = 0, c = 0;
      cudaEventElapsedTime(&a, C->ev[0], C->ev[1]);
      cudaEventElapsedTime(&c, C->ev[1], C->ev[2]);
      S.ms_cull = a;
      S.ms_leaf = c;
    }
    C->stats_valid = true;
  }
  *out = C->host_stats;
  return SPAMM_OK;
}

spamm_status spamm_triples(spamm_tree C, uint32_t *ijk, int64_t cap, int64_t *count) {
  if (C && settle(C->ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!C) return SPAMM_EINVAL;
  spamm_ctx ctx = C->ctx;
  if (!count) return fail(ctx, SPAMM_EINVAL, "triples: null count");
  if (!C->is_product) return fail(ctx, SPAMM_EINVAL, "triples: not a product tree");
  DevCounts h;
  CK(cudaMemcpyAsync(&h, C->counts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "triples: copy");
  spamm_status st = check_device_status(ctx);
  if (st != SPAMM_OK) return st;
  const TierList &T = C->tiers[C->kmax];
  const int64_t ng = (int64_t)h.ngroups[C->kmax];
  const int64_t ne = (int64_t)h.nentries[C->kmax];
  // a symmetric product lists the mirror (j, i, k) of every triple of a block i < j
  *count = (int64_t)h.leaf_products + (C->sym_product ? (int64_t)h.mirror_products : 0);
  if (!ijk) return SPAMM_OK;
  if (*count > cap) return fail(ctx, SPAMM_ERANGE, "triples: %lld needed, cap %lld", (long long)*count, (long long)cap);
  std::vector<uint32_t> gij(ng), gs(ng), gl(ng);
  std::vector<uint16_t> K(ne);
  std::vector<uint8_t> m(ne);
  if (ng) {
    CK(cudaMemcpyAsync(gij.data(), T.gij, ng * 4, cudaMemcpyDeviceToHost, ctx->stream), "triples: copy");
    CK(cudaMemcpyAsync(gs.data(), T.gstart, ng * 4, cudaMemcpyDeviceToHost, ctx->stream), "triples: copy");
    CK(cudaMemcpyAsync(gl.data(), T.glen, ng * 4, cudaMemcpyDeviceToHost, ctx->stream), "triples: copy");
  }
  if (ne) {
    CK(cudaMemcpyAsync(K.data(), T.K, ne * 2, cudaMemcpyDeviceToHost, ctx->stream), "triples: copy");
    CK(cudaMemcpyAsync(m.data(), C->mask, ne, cudaMemcpyDeviceToHost, ctx->stream), "triples: copy");
  }
  CK(cudaStreamSynchronize(ctx->stream), "triples: synchronize");
  std::vector<uint64_t> keys;
  keys.reserve((size_t)*count);
  const int sh = 21;
  for (int64_t g = 0; g < ng; g++) {
    const uint64_t I = gij[g] >> 16, J = gij[g] & 0xFFFF;
    for (uint32_t p = 0; p < gl[g]; p++) {
      const uint64_t e = gs[g] + p;
      if ((int64_t)e >= ne) break;
      const uint32_t bits = m[e];
      for (int q = 0; q < 8; q++)
        if ((bits >> q) & 1u) {
          const uint64_t a = (q >> 2) & 1, c = (q >> 1) & 1, ee = q & 1;
          const uint64_t i = 2 * I + a, j = 2 * J + c, k = 2 * (uint64_t)K[e] + ee;
          keys.push_back((i << (2 * sh)) | (j << sh) | k);
          if (C->sym_product && i < j) keys.push_back((j << (2 * sh)) | (i << sh) | k);
        }
    }
  }
  if ((int64_t)keys.size() != *count)
    return fail(ctx, SPAMM_ECUDA, "triples: mask count %zu != counter %lld", keys.size(), (long long)*count);
  std::sort(keys.begin(), keys.end());
  const uint64_t mk = (1ull << sh) - 1;
  for (size_t t = 0; t < keys.size(); t++) {
    ijk[3 * t] = (uint32_t)(keys[t] >> (2 * sh));
    ijk[3 * t + 1] = (uint32_t)((keys[t] >> sh) & mk);
    ijk[3 * t + 2] = (uint32_t)(keys[t] & mk);
  }
  return SPAMM_OK;
}

}  // extern "C"

// ---- SP2 purification: a run object stepping on the context stream ----
struct spamm_sp2_s {
  spamm_ctx ctx = nullptr;
  int64_t n = 0, nnz = 0;
  double n_occ = 0, emin = 0, emax = 0;
  spamm_prec prec = SPAMM_FP64;
  int steps = 0;
  int64_t *d_ip = nullptr, *d_ix = nullptr;
  double *d_v = nullptr, *d_part = nullptr;
  void *d_rec = nullptr;
  float *d_feat = nullptr;
  double *d_ctrl = nullptr;   // controller: bound workspace, then the tolerance grid
  double grid_lo = 0, grid_hi = 0;
  spamm_tree X = nullptr, C = nullptr;
  double tau_host[SPAMM_SP2_MAX_STEPS] = {};
  bool learned[SPAMM_SP2_MAX_STEPS] = {};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

void sp2_release(spamm_sp2_run r) {
  if (!r) return;
  if (r->X) { free_tree_memory(r->X); delete r->X; }
  if (r->C) { free_tree_memory(r->C); delete r->C; }
  dfree(r->d_ip); dfree(r->d_ix); dfree(r->d_v); dfree(r->d_part); dfree(r->d_rec); dfree(r->d_feat);
  dfree(r->d_ctrl);
  if (r->e0) cudaEventDestroy(r->e0);
  if (r->e1) cudaEventDestroy(r->e1);
  delete r;
}

}  // namespace

extern "C" spamm_status spamm_sp2_begin(spamm_ctx ctx, int64_t n, const int64_t *indptr, const int64_t *indices,
                                        const double *data, double n_occ, int32_t leaf, spamm_prec prec,
                                        spamm_sp2_run *out) {
  if (!ctx) return SPAMM_EINVAL;
  if (!indptr || !indices || !data || !out) return fail(ctx, SPAMM_EINVAL, "sp2: null pointer");
  if (n < 1 || !valid_leaf(leaf)) return fail(ctx, SPAMM_EINVAL, "sp2: bad n / leaf");
  if (prec < SPAMM_FP64 || prec > SPAMM_TF32X3) return fail(ctx, SPAMM_EINVAL, "sp2: unknown precision");
  const bool tc = prec != SPAMM_FP64;
  if (tc && leaf != 64 && leaf != 128) return fail(ctx, SPAMM_EUNSUPPORTED, "sp2: tensor-core precisions need leaf 64 or 128");
  const int64_t nnz = indptr[n];
  if (nnz < 0 || indptr[0] != 0) return fail(ctx, SPAMM_EINVAL, "sp2: bad CSR");
  // Gershgorin interval on the host
  double emin = INFINITY, emax = -INFINITY;
  for (int64_t i = 0; i < n; i++) {
    if (indptr[i + 1] < indptr[i]) return fail(ctx, SPAMM_EINVAL, "sp2: bad CSR");
    double d = 0.0, rad = 0.0;
    for (int64_t q = indptr[i]; q < indptr[i + 1]; q++) {
      if (indices[q] < 0 || indices[q] >= n) return fail(ctx, SPAMM_EINVAL, "sp2: column index out of range");
      if (indices[q] == i) d += data[q];
      else rad += std::fabs(data[q]);
    }
    emin = std::min(emin, d - rad);
    emax = std::max(emax, d + rad);
  }
  if (!(emax > emin)) return fail(ctx, SPAMM_EINVAL, "sp2: empty spectral interval");
  spamm_sp2_run r = new (std::nothrow) spamm_sp2_s();
  if (!r) return SPAMM_ENOMEM;
  r->ctx = ctx;
  r->n = n;
  r->nnz = nnz;
  r->n_occ = n_occ;
  r->emin = emin;
  r->emax = emax;
  r->prec = prec;
  cudaStream_t s = ctx->stream;
  const int32_t flags = tc ? (COPY_FLAG_OF(prec) | SPAMM_SYMMETRIC | SPAMM_NO_RIGHT)
                           : (SPAMM_KEEP_FP64 | SPAMM_SYMMETRIC | SPAMM_NO_RIGHT);
#define SP2CK(call, what)                                  \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) { sp2_release(r); return cuda_fail(ctx, _e, what); } \
  } while (0)
  SP2CK(dmalloc(&r->d_ip, (n + 1) * 8), "sp2: allocation");
  SP2CK(dmalloc(&r->d_ix, std::max<int64_t>(nnz, 1) * 8), "sp2: allocation");
  SP2CK(dmalloc(&r->d_v, std::max<int64_t>(nnz, 1) * 8), "sp2: allocation");
  SP2CK(dmalloc(&r->d_part, ((n + 255) / 256) * 8), "sp2: allocation");
  SP2CK(dmalloc((unsigned char **)&r->d_rec, sp2_record_bytes()), "sp2: allocation");
  SP2CK(dmalloc(&r->d_feat, sizeof(float) * kTreeFeatures), "sp2: allocation");
  SP2CK(cudaMemsetAsync(r->d_rec, 0, sp2_record_bytes(), s), "sp2: memset");
  SP2CK(cudaMemcpyAsync(r->d_ip, indptr, (n + 1) * 8, cudaMemcpyHostToDevice, s), "sp2: copy");
  if (nnz) {
    SP2CK(cudaMemcpyAsync(r->d_ix, indices, nnz * 8, cudaMemcpyHostToDevice, s), "sp2: copy");
    SP2CK(cudaMemcpyAsync(r->d_v, data, nnz * 8, cudaMemcpyHostToDevice, s), "sp2: copy");
  }
  spamm_status st = alloc_tree(ctx, n, leaf, flags, &r->X);
  if (st == SPAMM_OK) st = alloc_tree(ctx, n, leaf, flags, &r->C);
  if (st != SPAMM_OK) { sp2_release(r); return st; }
  if (tc) {
    const size_t elems = (size_t)r->X->nb * r->X->nb * (size_t)leaf * leaf;
    SP2CK(dmalloc(&r->X->copy[CK_F32], elems * 4), "sp2: allocation");
    SP2CK(dmalloc(&r->C->copy[CK_F32], elems * 4), "sp2: allocation");
    r->X->flags |= SPAMM_INTERNAL_F32;
    r->C->flags |= SPAMM_INTERNAL_F32;
  }
  st = ensure_stage(ctx, (size_t)n * n * sizeof(double));
  if (st != SPAMM_OK) { sp2_release(r); return st; }
  SP2CK(sp2_x0(n, r->d_ip, r->d_ix, r->d_v, emin, emax, (double *)ctx->stage, s), "sp2: X0");
  SP2CK(launch_tree_build(r->X, (const double *)ctx->stage, s), "sp2: X0 tree");
  SP2CK(launch_pyramid(r->X, s), "sp2: X0 pyramid");
  SP2CK(cudaEventCreate(&r->e0), "sp2: event");
  SP2CK(cudaEventCreate(&r->e1), "sp2: event");
  SP2CK(cudaEventRecord(r->e0, s), "sp2: event");
#undef SP2CK
  ctx->launches += 2 + pyramid_launches(r->X);
  *out = r;
  return SPAMM_OK;
}

namespace {

// One step with tau on the host, or read from the record slot the controller wrote.
spamm_status sp2_advance(spamm_sp2_run r, double tau, bool from_record) {
  spamm_ctx ctx = r->ctx;
  const int step = r->steps;
  spamm_tree out_tree = r->C;
  const double *tau_dev = from_record ? sp2_tau_slot(r->d_rec, step) : nullptr;
  spamm_status st = multiply_impl(ctx, r->X, r->X, from_record ? 0.0 : tau, tau_dev, r->prec, SPAMM_SYM_PRODUCT,
                                  &out_tree);
  if (st != SPAMM_OK) return st;
  CK(sp2_step_finish(r->X, r->C, r->n_occ, step, r->d_rec, ctx->stream), "sp2: step");
  ctx->launches += 4 + pyramid_launches(r->C);
  r->tau_host[step] = tau;
  r->learned[step] = from_record;
  std::swap(r->X, r->C);
  r->steps++;
  return SPAMM_OK;
}

}  // namespace

// Scheme (I) of Sec. III: the product at the smallest positive tau (exact: only products
// with an absent or zero block are skipped), then the dropping filter on it, then the
// trace-correcting step on the filtered product.
static spamm_status sp2_advance_drop(spamm_sp2_run r, double tau_drop) {
  spamm_ctx ctx = r->ctx;
  const int step = r->steps;
  spamm_tree out_tree = r->C;
  spamm_status st = multiply_impl(ctx, r->X, r->X, std::numeric_limits<double>::denorm_min(), nullptr, r->prec,
                                  SPAMM_SYM_PRODUCT, &out_tree);
  if (st != SPAMM_OK) return st;
  CK(launch_drop(r->C, tau_drop, nullptr, ctx->stream), "sp2: dropping filter");
  ctx->launches += 1 + pyramid_launches(r->C);
  CK(sp2_step_finish(r->X, r->C, r->n_occ, step, r->d_rec, ctx->stream), "sp2: step");
  ctx->launches += 4 + pyramid_launches(r->C);
  r->tau_host[step] = tau_drop;
  r->learned[step] = false;
  std::swap(r->X, r->C);
  r->steps++;
  return SPAMM_OK;
}

extern "C" spamm_status spamm_sp2_step(spamm_sp2_run r, double tau) {
  if (!r) return SPAMM_EINVAL;
  if (r->steps >= SPAMM_SP2_MAX_STEPS) return fail(r->ctx, SPAMM_ERANGE, "sp2: more than %d steps", SPAMM_SP2_MAX_STEPS);
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(r->ctx, SPAMM_EINVAL, "sp2: tau invalid");
  return sp2_advance(r, tau, false);
}

extern "C" spamm_status spamm_sp2_step_drop(spamm_sp2_run r, double tau_drop) {
  if (!r) return SPAMM_EINVAL;
  if (r->steps >= SPAMM_SP2_MAX_STEPS) return fail(r->ctx, SPAMM_ERANGE, "sp2: more than %d steps", SPAMM_SP2_MAX_STEPS);
  if (!(tau_drop >= 0.0) || !std::isfinite(tau_drop)) return fail(r->ctx, SPAMM_EINVAL, "sp2: tau invalid");
  return sp2_advance_drop(r, tau_drop);
}

extern "C" spamm_status spamm_sp2_dropping(spamm_ctx ctx, int64_t n, const int64_t *indptr, const int64_t *indices,
                                           const double *data, double n_occ, int32_t steps, int32_t leaf,
                                           spamm_prec prec, double tau_drop, spamm_sp2_result *out) {
  if (!ctx) return SPAMM_EINVAL;
  if (!out) return fail(ctx, SPAMM_EINVAL, "sp2: null pointer");
  if (steps < 0 || steps > SPAMM_SP2_MAX_STEPS) return fail(ctx, SPAMM_EINVAL, "sp2: bad steps");
  spamm_sp2_run r = nullptr;
  spamm_status st = spamm_sp2_begin(ctx, n, indptr, indices, data, n_occ, leaf, prec, &r);
  if (st != SPAMM_OK) return st;
  for (int q = 0; q < steps && st == SPAMM_OK; q++) st = spamm_sp2_step_drop(r, tau_drop);
  if (st != SPAMM_OK) {
    spamm_sp2_end(r, nullptr);
    return st;
  }
  return spamm_sp2_end(r, out);
}

// One learned step; mu_ref > 0 loosens the step's budget by its branch margin on the device.
static spamm_status sp2_step_learned_impl(spamm_sp2_run r, spamm_mlp m, double err_budget, double tau_min,
                                          double tau_max, double mu_ref, double gain_max) {
  if (!r || !m) return SPAMM_EINVAL;
  spamm_ctx ctx = r->ctx;
  if (r->steps >= SPAMM_SP2_MAX_STEPS) return fail(ctx, SPAMM_ERANGE, "sp2: more than %d steps", SPAMM_SP2_MAX_STEPS);
  if (!(err_budget > 0.0) || !(tau_min > 0.0) || !(tau_max >= tau_min) || !std::isfinite(tau_max))
    return fail(ctx, SPAMM_EINVAL, "sp2: bad budget or tau range");
  if (mu_ref < 0.0 || !std::isfinite(mu_ref) || (mu_ref > 0.0 && !(gain_max >= 1.0 && std::isfinite(gain_max))))
    return fail(ctx, SPAMM_EINVAL, "sp2: bad margin reference or gain");
  if (mlp_inputs(m) != SPAMM_MLP_FEATURES) return fail(ctx, SPAMM_EINVAL, "sp2: network has the wrong input width");
  cudaStream_t s = ctx->stream;
  const size_t nw = bound_workspace_doubles(r->X);
  // the bound workspace, the tolerance grid, then the step's device budget
  if (!r->d_ctrl) CK(dmalloc(&r->d_ctrl, sizeof(double) * (nw + kTauGrid + 1)), "sp2: allocation");
  double *grid = r->d_ctrl + nw, *bound = r->d_ctrl + (nw - kTauGrid), *budget_dev = r->d_ctrl + nw + kTauGrid;
  if (r->grid_lo != tau_min || r->grid_hi != tau_max) {   // the grid, uploaded once per range
    double h[kTauGrid];
    tau_grid(tau_min, tau_max, h);
    CK(cudaMemcpyAsync(grid, h, sizeof h, cudaMemcpyHostToDevice, s), "sp2: grid");
    CK(cudaStreamSynchronize(s), "sp2: grid");
    r->grid_lo = tau_min;
    r->grid_hi = tau_max;
  }
  CK(launch_feat_hist(r->X, r->d_feat, s), "sp2: features");
  CK(launch_flat_bound(r->X, r->X, grid, kTauGrid, r->d_ctrl, bound, s), "sp2: flat bound");
  if (mu_ref > 0.0) {
    CK(sp2_margin_budget(r->X, r->steps, r->d_rec, r->n_occ, mu_ref, gain_max, std::log10(err_budget), budget_dev, s),
       "sp2: margin budget");
    ctx->launches++;
  }
  CK(launch_tau_select(m, r->d_feat, r->d_feat, grid, bound, std::log10(err_budget), sp2_tau_slot(r->d_rec, r->steps), s,
                       mu_ref > 0.0 ? budget_dev : nullptr),
     "sp2: tau selection");
  ctx->launches += 4;
  return sp2_advance(r, 0.0, true);
}

extern "C" spamm_status spamm_sp2_step_learned(spamm_sp2_run r, spamm_mlp m, double err_budget, double tau_min,
                                               double tau_max) {
  return sp2_step_learned_impl(r, m, err_budget, tau_min, tau_max, 0.0, 1.0);
}

extern "C" spamm_status spamm_sp2_step_learned_margin(spamm_sp2_run r, spamm_mlp m, double err_budget,
                                                      double tau_min, double tau_max, double mu_ref,
                                                      double gain_max) {
  if (r && !(mu_ref > 0.0)) return fail(r->ctx, SPAMM_EINVAL, "sp2: the margin reference must be positive");
  return sp2_step_learned_impl(r, m, err_budget, tau_min, tau_max, mu_ref, gain_max);
}

extern "C" spamm_status spamm_sp2_iterate(spamm_sp2_run r, spamm_tree *X) {
  if (!r || !X) return SPAMM_EINVAL;
  *X = r->X;
  return SPAMM_OK;
}

extern "C" spamm_status spamm_sp2_end(spamm_sp2_run r, spamm_sp2_result *out) {
  if (!r) return SPAMM_EINVAL;
  spamm_ctx ctx = r->ctx;
  cudaStream_t s = ctx->stream;
  std::vector<unsigned char> host_rec(sp2_record_bytes());
  spamm_status st = SPAMM_OK;
  cudaError_t e = sp2_trace_only(r->X, r->steps, r->d_rec, s);
  if (e == cudaSuccess) e = sp2_energy(r->X, r->n, r->d_ip, r->d_ix, r->d_v, r->d_part, r->d_rec, s);
  if (e == cudaSuccess) e = cudaEventRecord(r->e1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_rec.data(), r->d_rec, sp2_record_bytes(), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) st = cuda_fail(ctx, e, "sp2: finish");
  if (st == SPAMM_OK) st = check_device_status(ctx);
  if (st == SPAMM_OK && out) {
    memset(out, 0, sizeof *out);
    sp2_read_record(host_rec.data(), r->steps, out);
    for (int q = 0; q < r->steps; q++)
      if (!r->learned[q]) out->tau[q] = r->tau_host[q];
    out->eps_min = r->emin;
    out->eps_max = r->emax;
    out->steps = r->steps;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r->e0, r->e1);
    out->ms = ms;
  }
  ctx->launches += 3;
  sp2_release(r);
  return st;
}

extern "C" spamm_status spamm_sp2(spamm_ctx ctx, int64_t n, const int64_t *indptr, const int64_t *indices,
                                  const double *data, double n_occ, int32_t steps, int32_t leaf, spamm_prec prec,
                                  const double *tau, spamm_sp2_result *out) {
  if (!ctx) return SPAMM_EINVAL;
  if (!tau || !out) return fail(ctx, SPAMM_EINVAL, "sp2: null pointer");
  if (steps < 0 || steps > SPAMM_SP2_MAX_STEPS) return fail(ctx, SPAMM_EINVAL, "sp2: bad steps");
  for (int q = 0; q < steps; q++)
    if (!(tau[q] >= 0.0) || !std::isfinite(tau[q])) return fail(ctx, SPAMM_EINVAL, "sp2: tau[%d] invalid", q);
  spamm_sp2_run r = nullptr;
  spamm_status st = spamm_sp2_begin(ctx, n, indptr, indices, data, n_occ, leaf, prec, &r);
  if (st != SPAMM_OK) return st;
  for (int q = 0; q < steps && st == SPAMM_OK; q++) st = spamm_sp2_step(r, tau[q]);
  if (st != SPAMM_OK) {
    spamm_sp2_end(r, nullptr);
    return st;
  }
  return spamm_sp2_end(r, out);
}

extern "C" spamm_status spamm_sp2_learned(spamm_ctx ctx, int64_t n, const int64_t *indptr, const int64_t *indices,
                                          const double *data, double n_occ, int32_t steps, int32_t leaf,
                                          spamm_prec prec, spamm_mlp m, double err_budget, double tau_min,
                                          double tau_max, spamm_sp2_result *out) {
  if (!ctx) return SPAMM_EINVAL;
  if (!m || !out) return fail(ctx, SPAMM_EINVAL, "sp2: null pointer");
  if (steps < 0 || steps > SPAMM_SP2_MAX_STEPS) return fail(ctx, SPAMM_EINVAL, "sp2: bad steps");
  spamm_sp2_run r = nullptr;
  spamm_status st = spamm_sp2_begin(ctx, n, indptr, indices, data, n_occ, leaf, prec, &r);
  if (st != SPAMM_OK) return st;
  for (int q = 0; q < steps && st == SPAMM_OK; q++) st = spamm_sp2_step_learned(r, m, err_budget, tau_min, tau_max);
  if (st != SPAMM_OK) {
    spamm_sp2_end(r, nullptr);
    return st;
  }
  return spamm_sp2_end(r, out);
}

extern "C" spamm_status spamm_sp2_learned_margin(spamm_ctx ctx, int64_t n, const int64_t *indptr,
                                                 const int64_t *indices, const double *data, double n_occ,
                                                 int32_t steps, int32_t leaf, spamm_prec prec, spamm_mlp m,
                                                 double err_budget, double tau_min, double tau_max, double mu_ref,
                                                 double gain_max, spamm_sp2_result *out) {
  if (!ctx) return SPAMM_EINVAL;
  if (!m || !out) return fail(ctx, SPAMM_EINVAL, "sp2: null pointer");
  if (steps < 0 || steps > SPAMM_SP2_MAX_STEPS) return fail(ctx, SPAMM_EINVAL, "sp2: bad steps");
  if (!(mu_ref > 0.0)) return fail(ctx, SPAMM_EINVAL, "sp2: the margin reference must be positive");
  spamm_sp2_run r = nullptr;
  spamm_status st = spamm_sp2_begin(ctx, n, indptr, indices, data, n_occ, leaf, prec, &r);
  if (st != SPAMM_OK) return st;
  for (int q = 0; q < steps && st == SPAMM_OK; q++)
    st = spamm_sp2_step_learned_margin(r, m, err_budget, tau_min, tau_max, mu_ref, gain_max);
  if (st != SPAMM_OK) {
    spamm_sp2_end(r, nullptr);
    return st;
  }
  return spamm_sp2_end(r, out);
}
