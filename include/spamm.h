/*
 * spamm.h: C ABI of the GB300 (sm_103a) Sparse Approximate Matrix Multiply library.
 *
 * SpAMM (Challacombe and Bock, "Fast Multiplication of Matrices with Decay") computes
 * C ~ A B for matrices whose elements decay away from the diagonal. Each operand is
 * held as a quadtree (Eq. 1) with the Frobenius norm of every block (Sec. III); the
 * product recursion of Eq. 4 drops every block sub-product A^k B^k with
 * ||A^k||_F ||B^k||_F < tau at any tier k, and the dense leaf-block products that
 * survive are summed into C.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a spamm_status. No C++ exception crosses this boundary.
 *     A failing call stores a message that spamm_last_error(ctx) returns.
 *   - Matrices cross the boundary as dense n x n FP64 row-major arrays, on the host or
 *     on the device as each call's flags say. The caller owns those arrays; the
 *     library copies what it needs and owns all device memory behind its handles.
 *   - All device work is ordered on the context's CUDA stream. Calls that return data
 *     to the host (spamm_stats, spamm_triples, spamm_tree_norms, spamm_tree_to_dense
 *     with a host destination, spamm_sync) synchronise that stream first.
 *   - Sizes: n >= 1; leaf in {16, 32, 64, 128}; tau >= 0 and finite. The padded
 *     quadtree has NB = 2^kmax leaf blocks per side, NB the smallest power of two with
 *     NB * leaf >= n; padding is zero.
 *   - A device-side failure (a bounded wait that ran out, an internal capacity
 *     overflow) is recorded in a status word on the device and returned by the next
 *     synchronising call on that context; the context stays usable.
 */
#ifndef SPAMM_H
#define SPAMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SPAMM_API __attribute__((visibility("default")))
#else
#define SPAMM_API
#endif

typedef struct spamm_ctx_s *spamm_ctx;
typedef struct spamm_tree_s *spamm_tree;

typedef enum {
  SPAMM_OK = 0,
  SPAMM_EINVAL = 1,        /* bad argument: null handle, n < 1, leaf not supported,
                              tau < 0 or not finite, operands of unequal n or leaf,
                              an operand without the copy the precision needs */
  SPAMM_ENOMEM = 2,        /* device or pinned host allocation failed */
  SPAMM_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  SPAMM_ERANGE = 4,        /* a caller buffer or an internal capacity is too small;
                              the size needed is returned where the call says */
  SPAMM_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  SPAMM_EUNSUPPORTED = 6   /* valid request the library does not implement */
} spamm_status;

/* Arithmetic of the dense leaf products. Culling always uses the FP64 norms of the
   FP64 operands, so every precision multiplies the same surviving leaf triples. */
typedef enum {
  SPAMM_FP64 = 0,    /* FP64 operands, FP64 accumulation (CUDA cores) */
  SPAMM_TF32 = 1,    /* operands rounded to TF32, FP32 accumulation (tensor cores) */
  SPAMM_BF16 = 2,    /* operands rounded to BF16, FP32 accumulation (tensor cores) */
  SPAMM_FP16 = 3,    /* operands rounded to FP16, FP32 accumulation (tensor cores) */
  SPAMM_BF16X3 = 4,  /* split BF16: a = hi + lo, hi = bf16(a), lo = bf16(a - hi);
                        A B ~ Ahi Bhi + Ahi Blo + Alo Bhi, FP32 accumulation */
  SPAMM_TF32X3 = 5   /* split TF32, the same three products of hi = tf32(a),
                        lo = tf32(a - hi): about 22 significant bits of each operand */
} spamm_prec;

/* ---- flags of spamm_tree_build and spamm_multiply ---- */
#define SPAMM_HOST_INPUT   0x0001  /* spamm_tree_build: A is a host pointer (else device) */
#define SPAMM_SYMMETRIC    0x0002  /* caller asserts A == A^T: one low-precision copy then
                                      serves both operand roles (leaf (k,j) of A^T is
                                      leaf (j,k) of A, transposed), and the cull reads
                                      the tree's norms on and above the diagonal only,
                                      so ||A_ki|| and ||A_ik|| are the same number */
#define SPAMM_KEEP_FP64    0x0004  /* keep FP64 leaf tiles (needed by SPAMM_FP64 products) */
#define SPAMM_COPY_TF32    0x0010  /* write TF32 leaf copies */
#define SPAMM_COPY_BF16    0x0020  /* write BF16 leaf copies */
#define SPAMM_COPY_FP16    0x0040  /* write FP16 leaf copies */
#define SPAMM_COPY_BF16X3  0x0080  /* write BF16 hi and lo leaf copies */
#define SPAMM_NO_RIGHT     0x0100  /* the tree is never a right operand: skip the
                                      transposed copies a non-symmetric tree needs */
#define SPAMM_GRAPH        0x0200  /* spamm_multiply_batched: capture the batch into a CUDA
                                      graph on first use and replay it afterwards */
#define SPAMM_COPY_TF32X3  0x0400  /* write TF32 hi and lo leaf copies */
#define SPAMM_SYM_PRODUCT  0x0800  /* spamm_multiply of a symmetric tree by itself (B == A,
                                      built with SPAMM_SYMMETRIC): C = A A is symmetric, so
                                      only the output blocks i <= j are culled and
                                      multiplied, and C_ji is written as C_ij^T. As the
                                      cull reads a symmetric tree's norms on and above the
                                      diagonal, the surviving triples of (i, j) and (j, i)
                                      are the mirror images of each other */
#define SPAMM_DEPTH_TAU    0x1000  /* spamm_multiply: tier k tests against tau * 8^-k, the
                                      depth-scaled threshold tau^{k+1} = tau^k / 8 of Sec. II
                                      (rigorous: ||C~ - AB||_F < (k_max + 1) tau), instead of
                                      tau at every tier */
#define SPAMM_WARP_TILES   0x2000  /* spamm_multiply, spamm_multiply_batched: the tile shape
                                      of tensor-core products at leaf 64. Set: one warp per
                                      64 x 64 output block (warp-level mma.sync, the block's
                                      surviving k only). Clear (default): tcgen05 items of
                                      2 x 2 output blocks, 128 x 128 tiles, whose passes
                                      zero-fill the halves a k does not reach. Leaves 16 and
                                      32 always run the warp shape (the flag is accepted);
                                      leaf 128 has only the tcgen05 shape
                                      (SPAMM_EUNSUPPORTED); SPAMM_FP64: SPAMM_EINVAL. The
                                      results agree within the tensor-core bar; the sum
                                      order inside a block differs. */

#define SPAMM_MAX_LEVELS 24

/* Per-product counters, as the recursion of Eq. 4 would count them. */
typedef struct {
  int32_t levels;                          /* kmax + 1 tiers, 0 = root */
  int32_t leaf;                            /* leaf block size b */
  int64_t n;                               /* matrix order */
  int64_t tested[SPAMM_MAX_LEVELS];        /* norm-product tests made at each tier */
  int64_t culled[SPAMM_MAX_LEVELS];        /* tests that dropped the sub-product */
  double culled_bound[SPAMM_MAX_LEVELS];   /* sum of ||A^k|| ||B^k|| over the dropped ones;
                                              their total bounds ||C~ - AB||_F (Eq. 3) */
  int64_t leaf_products;                   /* surviving leaf triples (i, j, k) multiplied */
  int64_t mirrored_products;               /* surviving triples of blocks i > j obtained by
                                              mirroring (SPAMM_SYM_PRODUCT; else 0) */
  int64_t output_blocks;                   /* output leaf blocks with a surviving k */
  double leaf_flops;                       /* 2 b^3 leaf_products */
  double dense_equiv_flops;                /* 2 n^3 */
  double mma_flops;                        /* flops issued by the leaf kernel, counting
                                              zero-filled operand halves and the three
                                              products of the split precisions */
  double ms_cull;                          /* phase times (ms), when the context was made
                                              with timing on; else 0 */
  double ms_leaf;
  int32_t prec;                            /* spamm_prec of the product */
  double tau;
} spamm_stats_t;

/* ---- context ---- */

/* Create a context on CUDA device `device`, ordering its work on `cuda_stream`
   (a cudaStream_t; NULL = the legacy default stream). `timing` != 0 records CUDA
   events around the cull and leaf phases of every multiply (spamm_stats ms_*).
   Errors: SPAMM_EINVAL (out == NULL), SPAMM_ECUDA (no such device). */
SPAMM_API spamm_status spamm_ctx_create(int device, void *cuda_stream, int32_t timing, spamm_ctx *out);
SPAMM_API spamm_status spamm_ctx_destroy(spamm_ctx ctx);
/* Wait for the context's stream and return the first device-side error, if any. */
SPAMM_API spamm_status spamm_sync(spamm_ctx ctx);
/* Message of the last failed call on this context ("" if none). Owned by the context. */
SPAMM_API const char *spamm_last_error(spamm_ctx ctx);
/* Number of kernels this context has launched since it was created. */
SPAMM_API int64_t spamm_kernel_launches(spamm_ctx ctx);

/* ---- quadtree build (Eq. 1, Frobenius norms of Sec. III) ----
   Builds the padded quadtree of the n x n FP64 row-major matrix A: the squared
   Frobenius norm of every leaf block (one FP64 pass over A), the norm of every upper
   tier as the sum of its four children's squared norms, and the leaf copies `flags`
   asks for (converted in the same pass, round-to-nearest-even from FP64).
   A is a device pointer unless SPAMM_HOST_INPUT is set. On success *out is a new
   tree. Errors: SPAMM_EINVAL, SPAMM_ENOMEM, SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_tree_build(spamm_ctx ctx, const double *A, int64_t n, int32_t leaf,
                              int32_t flags, spamm_tree *out);
SPAMM_API spamm_status spamm_tree_free(spamm_tree t);
/* Rebuild tree t in place from a new n x n FP64 row-major matrix A of the same order:
   the same leaf size and leaf copies, no allocation (a repeated build, e.g. of the
   iterate of a purification loop). A is a device pointer unless `flags` holds
   SPAMM_HOST_INPUT. Errors: SPAMM_EINVAL (t is a product tree, bad flags), SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_tree_update(spamm_tree t, const double *A, int32_t flags);
/* Mean device time in milliseconds of the leaf-block kernel (quadtree leaves, leaf
   norms and leaf copies; Eq. 1 and the norms of Sec. III) over the builds and updates
   of t since the previous call (the last 64 at most), from CUDA events recorded on the
   context's stream around each launch when the context was created with timing != 0.
   Waits for those launches to finish, then starts a new count.
   Errors: SPAMM_EINVAL (null argument, or no timed build since the last call), SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_tree_build_ms(spamm_tree t, float *ms);
/* The dropping filter of the paper's scheme (I) (Sec. III: after each multiplication,
   blocks with ||P^k||_F < tau are dropped), at leaf resolution: every stored leaf block
   of t whose Frobenius norm is below tau is no longer stored (its presence byte and
   norm are cleared; no reader loads an absent block's tile), and the norm pyramid is
   rebuilt. tau = 0 drops nothing. *kept (may be NULL; then the call is asynchronous)
   gets the number of blocks still stored. Errors: SPAMM_EINVAL (tau negative or not
   finite), SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_drop_blocks(spamm_tree t, double tau, int64_t *kept);
/* Shape of a tree: order n, leaf size, padded blocks per side NB, and kmax. */
SPAMM_API spamm_status spamm_tree_info(spamm_tree t, int64_t *n, int32_t *leaf, int32_t *nb_padded,
                             int32_t *kmax);
/* Copy the squared Frobenius norms of tier `level` (0 = root .. kmax), a
   2^level x 2^level row-major FP64 grid, to the host buffer `out`. */
SPAMM_API spamm_status spamm_tree_norms(spamm_tree t, int32_t level, double *out);
/* Write the tree as a dense n x n FP64 row-major matrix to `out`. out_is_host: 0 =
   `out` is a device pointer (queued on the context's stream); 1 = a host pointer,
   written when the call returns; 2 = a host pointer, asynchronously: the call returns
   once the copy is queued, the copy runs on the context's copy stream while later
   calls proceed (the next step's input transfer, say), and `out` is complete after
   spamm_sync or any other call that synchronizes the context. Product trees in the
   tensor-core precisions hold an FP32 C, widened to FP64 here.
   Errors: SPAMM_EINVAL (null out, out_is_host not 0/1/2, a tree without FP64/FP32
   tiles), SPAMM_ENOMEM, SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_tree_to_dense(spamm_tree t, double *out, int32_t out_is_host);
/* Leaf copies a tree may hold, as spamm_tree_leaf_copy names them: the FP64 tiles; the
   FP32 tiles of a tensor-core product; the values rounded to TF32 (FP32 storage), BF16
   and FP16; the low parts of the split forms, fmt(a - fmt(a)) (BF16 in 16 bits, TF32 in
   FP32 storage); each also transposed (_T: every leaf stored transposed in place), the
   orientation a non-symmetric right operand keeps. */
typedef enum {
  SPAMM_LEAF_F64 = 0, SPAMM_LEAF_F32 = 1, SPAMM_LEAF_TF32 = 2, SPAMM_LEAF_TF32_T = 3,
  SPAMM_LEAF_BF16 = 4, SPAMM_LEAF_BF16_T = 5, SPAMM_LEAF_FP16 = 6, SPAMM_LEAF_FP16_T = 7,
  SPAMM_LEAF_BF16LO = 8, SPAMM_LEAF_BF16LO_T = 9, SPAMM_LEAF_TF32LO = 10, SPAMM_LEAF_TF32LO_T = 11
} spamm_leaf_copy;
/* Copy one stored leaf copy (spamm_leaf_copy `which`) of a tree, in the library's tile
   layout, to `out`: the leaves of the quadtree's finest tier (Eq. 1), leaf (r, c) with
   r, c < ceil(n / leaf) at element (r * ceil(n / leaf) + c) * leaf^2, row-major inside
   the leaf; nb^2 leaf^2 elements of 8, 4 or 2 bytes. Padding rows and columns of the
   edge leaves hold zeros; leaves of a product tree that hold no block (no surviving
   triple) hold unspecified values. out_is_host: 1 = host pointer (the call
   synchronises), 0 = device pointer (queued on the context's stream). `bytes` is the
   capacity of `out`. Errors: SPAMM_EINVAL (null arguments, `which` not held by the
   tree), SPAMM_ERANGE (`bytes` too small; nothing copied), SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_tree_leaf_copy(spamm_tree t, int32_t which, void *out, int64_t bytes,
                                            int32_t out_is_host);
/* As spamm_tree_to_dense, into a dense n x n FP32 row-major matrix: FP32 tiles (the
   products in the tensor-core precisions) are copied as they are, FP64 tiles rounded
   to nearest FP32. Half the bytes of the FP64 image, for callers that read a
   tensor-core product back to the host. The paper has no counterpart (its C stays in
   the quadtree). Errors as spamm_tree_to_dense. */
SPAMM_API spamm_status spamm_tree_to_dense_f32(spamm_tree t, float *out, int32_t out_is_host);

/* ---- the product (Eq. 4) ----
   C ~ A B with tolerance tau: the tier-by-tier cull of Eq. 4 from the root
   (a sub-product survives iff ||A^k||_F ||B^k||_F >= tau), then the surviving leaf
   products in precision `prec`, each output block summed over its k in ascending
   order with no atomics. `flags` may request leaf copies of C (SPAMM_COPY_*,
   SPAMM_SYMMETRIC, SPAMM_NO_RIGHT) so that C can be the operand of a next product.
   *C == NULL creates the product tree; otherwise *C is reused and must have the
   same n and leaf. A and B must have equal n and leaf and hold the copies `prec`
   needs (SPAMM_KEEP_FP64 for SPAMM_FP64, SPAMM_COPY_<prec> otherwise, and for B
   either SPAMM_SYMMETRIC or no SPAMM_NO_RIGHT).
   Supported: every precision at every leaf (16, 32, 64, 128): tensor-core products
   run as warp tiles at leaf 16 and 32 (and at 64 with SPAMM_WARP_TILES), as tcgen05
   items of 2 x 2 blocks at leaf 64 and of one block at 128. Other flags:
   SPAMM_SYM_PRODUCT, SPAMM_DEPTH_TAU, SPAMM_WARP_TILES.
   The norm pyramid of C runs on an internal stream of the context, overlapping later
   calls that do not read C (spamm_tree_update of an operand, say); every call that
   may read a product (including spamm_sync) first makes the context stream wait for it.
   Errors: SPAMM_EINVAL, SPAMM_EUNSUPPORTED, SPAMM_ENOMEM, SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_multiply(spamm_ctx ctx, spamm_tree A, spamm_tree B, double tau,
                            spamm_prec prec, int32_t flags, spamm_tree *C);

/* Counters of the product that made tree C. Errors: SPAMM_EINVAL if C is not a product. */
SPAMM_API spamm_status spamm_stats(spamm_tree C, spamm_stats_t *out);

/* The surviving leaf triples (i, j, k) of the product that made C, sorted by
   (i, j, k), three uint32 per triple, into the host buffer ijk of `cap` triples.
   *count receives the number of triples; SPAMM_ERANGE if it exceeds cap. */
SPAMM_API spamm_status spamm_triples(spamm_tree C, uint32_t *ijk, int64_t cap, int64_t *count);

/* ---- batched products ----
   C[p] ~ A[p] B[p] with tolerance tau[p] for p < count, every product as in
   spamm_multiply (same precision for all; each pair of equal n and leaf; C[p] created
   when NULL, else reused). The culls of all products run concurrently; the leaf
   products of all tensor-core products of one leaf size run in ONE persistent launch
   over a global work list spanning the products; the FP64 leaf kernels run per product.
   With SPAMM_GRAPH the sequence is captured into a CUDA graph the first time a given
   (precision, A, B, C) set is seen and replayed on later calls, the taus being read
   from device memory; the context stream must then be a created (non-default) stream.
   Leaf copies of the products are not produced (no SPAMM_COPY_* flags).
   Errors: as spamm_multiply; SPAMM_EUNSUPPORTED for copy flags or graphs on the
   default stream. */
SPAMM_API spamm_status spamm_multiply_batched(spamm_ctx ctx, const spamm_tree *A, const spamm_tree *B,
                                              const double *tau, int32_t count, spamm_prec prec,
                                              int32_t flags, spamm_tree *C);
/* spamm_tree_update of trees[p] from the device matrix A[p] (row-major FP64, the
   tree's order) for p < count, the rebuilds spread over the context's side streams
   (largest first, each to the least loaded stream) so that small ones run side by
   side; the context stream waits for all of them. flags must be 0 (device inputs); the
   builds are not timed (spamm_tree_build_ms). Errors: SPAMM_EINVAL (null or product
   trees, trees of another context, flags), SPAMM_ECUDA. */
SPAMM_API spamm_status spamm_tree_update_batched(spamm_ctx ctx, int32_t count, const spamm_tree *trees,
                                                 const double *const *A, int32_t flags);

/* Leaf-size autotuner: times the tree build plus the product A A at every leaf size
   (16, 32, 64, 128; each in its default tile shape) on the n x n matrix A (device, or
   host with SPAMM_HOST_INPUT; SPAMM_SYMMETRIC honoured) and returns the fastest in
   *leaf_out (and its time in *ms_out if not NULL). Results are cached in the context per
   (ceil(log2 n), precision, decade of tau). */
SPAMM_API spamm_status spamm_tune_leaf(spamm_ctx ctx, const double *A, int64_t n, double tau,
                                       spamm_prec prec, int32_t flags, int32_t *leaf_out,
                                       double *ms_out);

/* Leaf-size and tile-shape autotuner: as spamm_tune_leaf, over (leaf, tile shape)
   candidates: for tensor-core precisions leaf 16 and 32 (warp tiles), leaf 64 with the
   tcgen05 items of 2 x 2 blocks and with warp tiles (SPAMM_WARP_TILES), leaf 128
   (tcgen05); for SPAMM_FP64 the leaf sizes alone. Returns the fastest leaf in *leaf_out,
   the spamm_multiply flags that select its tile shape (0 or SPAMM_WARP_TILES) in
   *tile_flags_out, and its time in *ms_out if not NULL. Cached per (ceil(log2 n),
   precision, decade of tau), apart from spamm_tune_leaf's results. */
SPAMM_API spamm_status spamm_tune_shape(spamm_ctx ctx, const double *A, int64_t n, double tau,
                                        spamm_prec prec, int32_t flags, int32_t *leaf_out,
                                        int32_t *tile_flags_out, double *ms_out);

/* ---- learned tolerance controller ----
   (The paper has no counterpart: it fixes tau by hand, Sec. III.) A small network
   predicts log10 of a product's relative Frobenius error from features of the
   operands' norm trees and tau; the controller picks, per product, the largest tau on a
   grid whose prediction meets an error budget. The network is a perceptron with two
   tanh hidden layers, trained on the GPU by the library's own forward, backward and
   Adam kernels (FP32, fixed-order reductions). Parameters are one float vector:
   W1 (hidden x inputs, row-major), b1, W2 (hidden x hidden), b2, W3 (1 x hidden), b3.
   All arrays of these calls are host arrays; calls synchronise the context stream. */
typedef struct spamm_mlp_s *spamm_mlp;
#define SPAMM_MLP_FEATURES 69   /* per operand: 16-bin decade histograms of the block norms
                                   of its leaf tier and the tier above, as fractions of
                                   nonzero blocks; then (log10 tau - log10 ||A||_F -
                                   log10 ||B||_F) / 8, (log10 ||A||_F + log10 ||B||_F) / 8,
                                   the nonzero-leaf fractions of A and B, and
                                   (log10 F(tau) - log10 ||A||_F - log10 ||B||_F) / 8 (at
                                   least -2) of the flat leaf bound F(tau): the sum of
                                   ||A_ik|| ||B_kj|| over leaf triples below tau (FP32) */
/* Network with `inputs` (1..128) and `hidden` (1..64) units, weights drawn
   U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64(seed), biases 0. */
SPAMM_API spamm_status spamm_mlp_create(spamm_ctx ctx, int32_t inputs, int32_t hidden, uint64_t seed,
                                        spamm_mlp *out);
/* Release the network's device memory (SPAMM_EINVAL for NULL). */
SPAMM_API spamm_status spamm_mlp_free(spamm_mlp m);
/* Number of parameters, hidden * (inputs + hidden + 3) + 1; -1 for NULL. */
SPAMM_API int32_t spamm_mlp_num_params(spamm_mlp m);
/* Copy the parameters into out[cap] (cap >= spamm_mlp_num_params, else SPAMM_EINVAL). */
SPAMM_API spamm_status spamm_mlp_get_params(spamm_mlp m, float *out, int32_t cap);
/* Set the parameters (count == spamm_mlp_num_params) and reset the Adam state. */
SPAMM_API spamm_status spamm_mlp_set_params(spamm_mlp m, const float *in, int32_t count);
/* y[N] = network(X[N x inputs]). */
SPAMM_API spamm_status spamm_mlp_forward(spamm_mlp m, const float *X, int32_t N, float *y);
/* Loss (1/2N) sum (y_hat - y)^2 and its gradient grad[num_params] (either may be NULL). */
SPAMM_API spamm_status spamm_mlp_gradient(spamm_mlp m, const float *X, const float *y, int32_t N,
                                          float *grad, float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on N samples. */
SPAMM_API spamm_status spamm_mlp_adam_step(spamm_mlp m, const float *X, const float *y, int32_t N,
                                           float lr, float *loss);
/* One Adam step with the caller's gradient grad[num_params]. */
SPAMM_API spamm_status spamm_mlp_adam_apply(spamm_mlp m, const float *grad, float lr);
/* `epochs` passes of mini-batch Adam over a SplitMix64(seed) permutation per epoch;
   *final_loss gets the full-data loss at the end. */
SPAMM_API spamm_status spamm_mlp_train(spamm_mlp m, const float *X, const float *y, int32_t N,
                                       int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                       float *final_loss);
/* Features of the product A B at tolerance tau > 0 (SPAMM_MLP_FEATURES floats). */
SPAMM_API spamm_status spamm_features(spamm_tree A, spamm_tree B, double tau, float *out);
/* Largest tau on the grid of 37 values log-spaced over [tau_min, tau_max]
   (10^(log10 tau_min + g (log10 tau_max - log10 tau_min) / 36), g = 0..36) whose predicted
   relative error is <= err_budget (tau_min when none is). */
SPAMM_API spamm_status spamm_tau_select(spamm_mlp m, spamm_tree A, spamm_tree B, double err_budget,
                                        double tau_min, double tau_max, double *tau_out);
/* ||X - Y||_F and ||Y||_F of two trees of equal n and leaf (FP64 or FP32 tiles). */
SPAMM_API spamm_status spamm_tree_distance(spamm_tree X, spamm_tree Y, double *diff_fro,
                                           double *ref_fro);

/* ---- SP2 density-matrix purification (Sec. III: TC2 purification, energy Tr(H X)) ----
   H is a symmetric n x n matrix given as host CSR (indptr[n+1], indices and data[nnz],
   column indices sorted per row). X0 = (eps_max I - H) / (eps_max - eps_min) with the
   Gershgorin bounds of H; each step s forms C = SpAMM(X, X) with tolerance tau[s] in
   precision prec, computes t1 = Tr X and t2 = Tr C in FP64, and sets X <- C if
   |t2 - n_occ| <= |2 t1 - t2 - n_occ| (ties to C), else X <- 2X - C; every product is
   a SPAMM_SYM_PRODUCT (X is symmetric). The iterate keeps
   an FP64 master for SPAMM_FP64 and an FP32 master otherwise. After `steps` steps the
   result holds E = Tr(H X), the trace of every iterate, the branch taken and the
   surviving leaf products of every product. Work is ordered on the context stream;
   the call synchronises once at the end. leaf in {16,32,64,128} for SPAMM_FP64, 64 or
   128 for the tensor-core precisions; 0 <= steps <= SPAMM_SP2_MAX_STEPS.
   Errors: SPAMM_EINVAL, SPAMM_EUNSUPPORTED, SPAMM_ENOMEM, SPAMM_ECUDA, SPAMM_ETIMEOUT. */
#define SPAMM_SP2_MAX_STEPS 128
typedef struct {
  double energy;                                /* Tr(H X_steps) */
  double eps_min, eps_max;                      /* Gershgorin interval of H */
  int32_t steps;
  double trace[SPAMM_SP2_MAX_STEPS + 1];        /* Tr X_s, s = 0 .. steps */
  int32_t branch[SPAMM_SP2_MAX_STEPS];          /* 1: X <- X^2, 0: X <- 2X - X^2 */
  int64_t leaf_products[SPAMM_SP2_MAX_STEPS];   /* leaf triples multiplied at step s (the
                                                   products are symmetric: blocks i <= j) */
  double tau[SPAMM_SP2_MAX_STEPS];              /* tolerance of step s (given, or chosen
                                                   by the controller) */
  double ms;                                    /* device time of the loop (ms) */
} spamm_sp2_result;

SPAMM_API spamm_status spamm_sp2(spamm_ctx ctx, int64_t n, const int64_t *indptr,
                                 const int64_t *indices, const double *data, double n_occ,
                                 int32_t steps, int32_t leaf, spamm_prec prec, const double *tau,
                                 spamm_sp2_result *out);

/* The same loop one step at a time. spamm_sp2_begin validates H, forms X0 and its tree
   (errors as above; *out owns device memory until spamm_sp2_end). spamm_sp2_step queues
   one step with tolerance tau; spamm_sp2_step_learned queues one step whose tolerance
   the controller m chooses on the device from the features of X (spamm_tau_select's
   rule: budget and grid [tau_min, tau_max]), without a host round trip. Both are
   asynchronous on the context stream; more than SPAMM_SP2_MAX_STEPS steps give
   SPAMM_ERANGE. spamm_sp2_iterate lends the current iterate X as a tree (valid until
   the next step or the end; the caller must not free it), e.g. to record features and
   errors for training. spamm_sp2_end computes E, fills *out (may be NULL), and frees
   the run whatever the status. */
typedef struct spamm_sp2_s *spamm_sp2_run;
SPAMM_API spamm_status spamm_sp2_begin(spamm_ctx ctx, int64_t n, const int64_t *indptr,
                                       const int64_t *indices, const double *data, double n_occ,
                                       int32_t leaf, spamm_prec prec, spamm_sp2_run *out);
SPAMM_API spamm_status spamm_sp2_step(spamm_sp2_run r, double tau);
SPAMM_API spamm_status spamm_sp2_step_learned(spamm_sp2_run r, spamm_mlp m, double err_budget,
                                              double tau_min, double tau_max);
/* spamm_sp2_step_learned with the step's budget loosened where its branch decision is
   far from a tie (not in the paper; the energy error of the trace-correcting loop is
   decided at near-tie steps): budget x clamp(m / mu_ref, 1, gain_max), with m the
   relative margin | |t2 - N| - |2 t1 - t2 - N| | / N of the step's decision, t1 = Tr X
   (from the previous step) and t2 = Tr X^2 = ||X||_F^2 (X symmetric: the root of its
   norm pyramid), computed on the device before the product. The first step keeps the
   base budget. Errors: as spamm_sp2_step_learned; SPAMM_EINVAL for mu_ref <= 0 or
   gain_max < 1 or not finite. */
SPAMM_API spamm_status spamm_sp2_step_learned_margin(spamm_sp2_run r, spamm_mlp m, double err_budget,
                                                     double tau_min, double tau_max, double mu_ref,
                                                     double gain_max);
/* One step of the paper's scheme (I) comparator (Sec. III): the product X X at the
   smallest positive tau (exact: only sub-products with an absent or zero block are
   skipped), then the dropping filter at leaf resolution with tau_drop
   (spamm_drop_blocks), then the trace-correcting step on the filtered product. The
   step's leaf products and tau_drop are recorded as for spamm_sp2_step. */
SPAMM_API spamm_status spamm_sp2_step_drop(spamm_sp2_run r, double tau_drop);
SPAMM_API spamm_status spamm_sp2_iterate(spamm_sp2_run r, spamm_tree *X);
SPAMM_API spamm_status spamm_sp2_end(spamm_sp2_run r, spamm_sp2_result *out);
/* spamm_sp2 with every step taken by scheme (I) (spamm_sp2_step_drop, tau_drop). */
SPAMM_API spamm_status spamm_sp2_dropping(spamm_ctx ctx, int64_t n, const int64_t *indptr,
                                          const int64_t *indices, const double *data, double n_occ,
                                          int32_t steps, int32_t leaf, spamm_prec prec, double tau_drop,
                                          spamm_sp2_result *out);
/* spamm_sp2 with every step's tolerance chosen by the controller. */
SPAMM_API spamm_status spamm_sp2_learned(spamm_ctx ctx, int64_t n, const int64_t *indptr,
                                         const int64_t *indices, const double *data,
                                         double n_occ, int32_t steps, int32_t leaf,
                                         spamm_prec prec, spamm_mlp m, double err_budget,
                                         double tau_min, double tau_max, spamm_sp2_result *out);
/* spamm_sp2 with every step taken by spamm_sp2_step_learned_margin. */
SPAMM_API spamm_status spamm_sp2_learned_margin(spamm_ctx ctx, int64_t n, const int64_t *indptr,
                                                const int64_t *indices, const double *data, double n_occ,
                                                int32_t steps, int32_t leaf, spamm_prec prec, spamm_mlp m,
                                                double err_budget, double tau_min, double tau_max,
                                                double mu_ref, double gain_max, spamm_sp2_result *out);

/* ---- cull without device allocation ----
   For callers that cannot allocate device memory: code running inside a CUDA graph
   capture or a real-time loop where cudaMalloc would synchronise or fail, embedders
   whose memory is owned by another allocator, or callers holding only raw device
   pointers and a stream. (The paper has no counterpart to this entry point.)
   Computes the surviving leaf triples of SpAMM(A, B) with tolerance tau from the
   squared Frobenius norms of the leaf blocks of A and B, with the same tier-by-tier
   cull as spamm_multiply, and allocates nothing: its working memory is one 2 MiB
   static device array of the library, held by every GPU that loads it until exit.
     normA2, normB2 : device, NB x NB row-major FP64 squared leaf norms (tier kmax of
                      spamm_tree_norms, or computed by the caller); not modified
     nb_padded      : NB, a power of two, 1 <= NB <= 128 (larger: SPAMM_ERANGE)
     triples        : device, room for `cap` triples (i, j, k) as 3 uint32 each, written
                      in the cull's order (output blocks in Morton order, then k
                      ascending); beyond cap nothing is written
     count          : device int64: the number of surviving triples (may exceed cap),
                      or -1 if a device-side wait timed out
     cuda_stream    : the stream all work is ordered on (a cudaStream_t; NULL = legacy)
   The call is asynchronous on the stream. The first call on each device looks up the
   device address of the static array (cudaGetSymbolAddress, with that device current);
   make that first call before any stream capture. Every call on a device shares the
   array and later calls overwrite it: calls that may overlap on the GPU (other streams,
   other host threads) race and must be serialised by the caller.
   Errors: SPAMM_EINVAL (null pointer, NB not a power of two, tau < 0 or not finite),
   SPAMM_ERANGE (NB > 128), SPAMM_ECUDA (a CUDA call failed). */
SPAMM_API spamm_status spamm_cull_noalloc(const double *normA2, const double *normB2,
                                          int32_t nb_padded, double tau, uint32_t *triples,
                                          int64_t cap, int64_t *count, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SPAMM_H */
