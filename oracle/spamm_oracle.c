/*
 * SpAMM oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the Sparse Approximate Matrix Multiply
 * of Challacombe and Bock, "Fast Multiplication of Matrices with Decay". It exists to
 * check the CUDA path; only the test suite, the smoke check and the benchmark's CPU
 * baseline call it, and it shares no code with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   - quadtree representation of a matrix, split 2 x 2 per tier down to a leaf
 *     size b (Eq. 1); the matrix is embedded with zeros in an NB*b square, NB the
 *     next power of two of ceil(n/b) (a reading: the paper assumes exact 2x2 splits);
 *   - the Frobenius norm of every quadtree block (Sec. III: the norm used is the
 *     Frobenius norm); leaf blocks sum squares row-major, and a parent's squared
 *     norm is the sum of its four children's, ((n11 + n12) + n21) + n22, so parent
 *     norms never fall below child norms, bit for bit;
 *   - the recursion of Eq. 4: a sub-product is dropped when ||A^k|| ||B^k|| < tau,
 *     computed densely at k = k_max, and split into the eight child sub-products
 *     otherwise, the two terms of each output quadrant taken in the order Eq. 4
 *     writes them (A_x1 B_1y before A_x2 B_2y);
 *   - the same surviving leaf triples by brute force over all NB^3 of them (the flat
 *     form that follows from Eq. 3 and the monotone norm tree);
 *   - the naive triple-loop product, which SpAMM at tau = 0 must reproduce
 *     (Sec. III: at tau = 0 SpAMM reverts to the ordinary O(n^3) product);
 *   - the depth-scaled threshold of Sec. II, tau^{k+1} = tau^k / 8 with tau^0 = tau at
 *     the root: tier k tests against tau * 8^-k (exactly, a power of two), the rigorous
 *     but pessimistic variant the paper mentions and does not use.
 *
 * Rounding order is fixed and documented: leaf norm^2 is a sequential row-major sum
 * of fl(a*a); the leaf product accumulates c += a*b in i-k-j order with no fused
 * multiply-add (this file is compiled with -ffp-contract=off); k runs in ascending
 * order for every output block. The cull test is sqrt(nA2) * sqrt(nB2) < tau.
 *
 * ORACLE_MUTANT (compile-time, 0 = none) plants one known mistake so the test suite
 * can show that its pins catch it. It is never set in the normal build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define ORACLE_MAX_LEVELS 24

typedef struct {
  int64_t n;      /* logical order of the matrix */
  int32_t b;      /* leaf block size */
  int32_t NB;     /* padded number of leaf blocks per side (power of two) */
  int32_t kmax;   /* log2(NB): leaves live at tier kmax */
  int64_t N;      /* NB * b */
  double *a;      /* N x N zero-padded copy, row-major */
  double *norm2;  /* squared Frobenius norms of every tier, tier l at offset (4^l-1)/3,
                     stored as a 2^l x 2^l row-major grid */
} oracle_tree;

typedef struct {
  int64_t tested[ORACLE_MAX_LEVELS];   /* norm-product tests made at tier l */
  int64_t culled[ORACLE_MAX_LEVELS];   /* tests that dropped the sub-product */
  double culled_bound[ORACLE_MAX_LEVELS]; /* sum of ||A^l|| ||B^l|| over dropped ones */
  int64_t leaf_products;               /* dense leaf products computed */
} oracle_stats;

static int64_t level_offset(int l) { return (((int64_t)1 << (2 * l)) - 1) / 3; }

static double *level_ptr(const oracle_tree *t, int l) { return t->norm2 + level_offset(l); }

/* ---- Eq. 1: padded quadtree and its Frobenius norm at every tier ---- */
int oracle_tree_build(const double *A, int64_t n, int32_t b, oracle_tree **out) {
  if (!A || !out || n < 1 || b < 1) return 1;
  int64_t nb = (n + b - 1) / b;
  int32_t NB = 1, kmax = 0;
  while (NB < nb) { NB *= 2; kmax++; }
  if (kmax >= ORACLE_MAX_LEVELS) return 1;
  oracle_tree *t = (oracle_tree *)calloc(1, sizeof(oracle_tree));
  if (!t) return 2;
  t->n = n; t->b = b; t->NB = NB; t->kmax = kmax; t->N = (int64_t)NB * b;
  t->a = (double *)calloc((size_t)(t->N * t->N), sizeof(double));
  t->norm2 = (double *)calloc((size_t)level_offset(kmax + 1), sizeof(double));
  if (!t->a || !t->norm2) { free(t->a); free(t->norm2); free(t); return 2; }
  for (int64_t i = 0; i < n; i++)
    memcpy(t->a + i * t->N, A + i * n, (size_t)n * sizeof(double));

  /* leaf tier: sequential row-major sum of squares over each b x b block */
  double *leaf = level_ptr(t, kmax);
  for (int32_t I = 0; I < NB; I++)
    for (int32_t K = 0; K < NB; K++) {
      double s = 0.0;
      for (int32_t r = 0; r < b; r++)
        for (int32_t c = 0; c < b; c++) {
          double v = t->a[((int64_t)I * b + r) * t->N + (int64_t)K * b + c];
#if ORACLE_MUTANT == 5
          s += fabs(v);
#else
          s += v * v;
#endif
        }
      leaf[(int64_t)I * NB + K] = s;
    }
  /* upper tiers: ((n11 + n12) + n21) + n22 of the four children */
  for (int l = kmax - 1; l >= 0; l--) {
    int64_t d = (int64_t)1 << l, dc = d * 2;
    const double *ch = level_ptr(t, l + 1);
    double *pa = level_ptr(t, l);
    for (int64_t I = 0; I < d; I++)
      for (int64_t K = 0; K < d; K++) {
        double n11 = ch[(2 * I) * dc + 2 * K], n12 = ch[(2 * I) * dc + 2 * K + 1];
        double n21 = ch[(2 * I + 1) * dc + 2 * K], n22 = ch[(2 * I + 1) * dc + 2 * K + 1];
#if ORACLE_MUTANT == 2
        (void)n22;
        pa[I * d + K] = (n11 + n12) + n21;
#else
        pa[I * d + K] = ((n11 + n12) + n21) + n22;
#endif
      }
  }
  *out = t;
  return 0;
}

void oracle_tree_free(oracle_tree *t) {
  if (!t) return;
  free(t->a); free(t->norm2); free(t);
}

int32_t oracle_tree_kmax(const oracle_tree *t) { return t->kmax; }
int32_t oracle_tree_NB(const oracle_tree *t) { return t->NB; }

/* copy the squared norms of tier l (2^l x 2^l, row-major) into out */
int oracle_tree_level_norm2(const oracle_tree *t, int32_t l, double *out) {
  if (l < 0 || l > t->kmax) return 1;
  memcpy(out, level_ptr(t, l), sizeof(double) * ((size_t)1 << (2 * l)));
  return 0;
}

/* ---- the Eq. 4 recursion ---- */
typedef struct {
  const oracle_tree *A, *B;
  const oracle_tree *Av, *Bv;  /* operands whose values the leaf products use (A, B) */
  double tau;
  int depth_scaled;     /* 1: tier l tests against tau * 8^-l (Sec. II) */
  double *C;            /* N x N padded accumulator, or NULL (norm tests only) */
  uint32_t *trip;       /* recorded leaf triples (i, j, k), or NULL */
  int64_t cap, ntrip;
  oracle_stats *st;     /* or NULL */
  int task_depth;       /* spawn OpenMP tasks for output quadrants above this tier */
  int target;           /* 1: follow only the output leaf block (ti, tj) */
  int32_t ti, tj;
  int64_t row0;         /* first padded row held by C (0 unless target mode) */
  int64_t col0;         /* first padded column held by C (0 unless target mode) */
  int64_t ldc;          /* row stride of C in elements; 0: N */
} rec_ctx;

static int cull(double nA2, double nB2, double tau) {
  double p = sqrt(nA2) * sqrt(nB2);
#if ORACLE_MUTANT == 1
  return p <= tau;
#else
  return p < tau;
#endif
}

static void leaf_product(const rec_ctx *c, int32_t I, int32_t J, int32_t K) {
  const oracle_tree *A = c->Av, *B = c->Bv;
  const int64_t N = A->N, b = A->b, ldc = c->ldc ? c->ldc : N;
  for (int64_t r = 0; r < b; r++) {
    double *crow = c->C + (I * b + r - c->row0) * ldc + (J * b - c->col0);
    for (int64_t l = 0; l < b; l++) {
      double a = A->a[(I * b + r) * N + K * b + l];
#if ORACLE_MUTANT == 3
      for (int64_t q = 0; q < b; q++) crow[q] += a * B->a[(J * b + q) * N + K * b + l];
#else
      const double *brow = B->a + (K * b + l) * N + J * b;
      for (int64_t q = 0; q < b; q++) crow[q] += a * brow[q];
#endif
    }
  }
}

static void rec(rec_ctx *c, int l, int32_t I, int32_t J, int32_t K) {
  const oracle_tree *A = c->A, *B = c->B;
  int64_t d = (int64_t)1 << l;
  double nA2 = level_ptr(A, l)[(int64_t)I * d + K];
#if ORACLE_MUTANT == 6
  double nB2 = level_ptr(B, l)[(int64_t)J * d + K];
#else
  double nB2 = level_ptr(B, l)[(int64_t)K * d + J];
#endif
  if (c->st) {
#pragma omp atomic
    c->st->tested[l]++;
  }
#if ORACLE_MUTANT == 7
  const double tl = c->depth_scaled ? ldexp(c->tau, -3 * (l + 1)) : c->tau;
#else
  const double tl = c->depth_scaled ? ldexp(c->tau, -3 * l) : c->tau;
#endif
  if (cull(nA2, nB2, tl)) {                     /* ||A^k|| ||B^k|| < tau: 0 */
    if (c->st) {
#pragma omp atomic
      c->st->culled[l]++;
      double p = sqrt(nA2) * sqrt(nB2);
#pragma omp atomic
      c->st->culled_bound[l] += p;
    }
    return;
  }
  if (l == A->kmax) {                          /* k = k_max: dense A^k B^k */
    if (c->C) leaf_product(c, I, J, K);
    if (c->st) {
#pragma omp atomic
      c->st->leaf_products++;
    }
    if (c->trip && c->ntrip < c->cap) {
      c->trip[3 * c->ntrip + 0] = (uint32_t)I;
      c->trip[3 * c->ntrip + 1] = (uint32_t)J;
      c->trip[3 * c->ntrip + 2] = (uint32_t)K;
    }
#pragma omp atomic
    c->ntrip++;
    return;
  }
  /* else: the 2x2 block of sums of eight child sub-products */
  int shift = A->kmax - (l + 1);
  for (int a = 0; a < 2; a++)
    for (int q = 0; q < 2; q++) {
      int32_t ci = 2 * I + a, cj = 2 * J + q;
      if (c->target && ((c->ti >> shift) != ci || (c->tj >> shift) != cj)) continue;
      if (l < c->task_depth) {
#pragma omp task firstprivate(ci, cj)
        {
#if ORACLE_MUTANT == 4
          if (!(a == 0 && q == 0)) rec(c, l + 1, ci, cj, 2 * K + 0);
#else
          rec(c, l + 1, ci, cj, 2 * K + 0);   /* A_x1 B_1y */
#endif
          rec(c, l + 1, ci, cj, 2 * K + 1);   /* + A_x2 B_2y */
        }
      } else {
#if ORACLE_MUTANT == 4
        if (!(a == 0 && q == 0)) rec(c, l + 1, ci, cj, 2 * K + 0);
#else
        rec(c, l + 1, ci, cj, 2 * K + 0);
#endif
        rec(c, l + 1, ci, cj, 2 * K + 1);
      }
    }
  if (l < c->task_depth) {
#pragma omp taskwait
  }
}

static int compatible(const oracle_tree *A, const oracle_tree *B) {
  return A && B && A->n == B->n && A->b == B->b;
}

/*
 * SpAMM(A, B) of Eq. 4 from the root tier.
 *   C        : n x n row-major output (padding cropped), or NULL for norm tests only
 *   triples  : room for `cap` triples (i, j, k), recorded in recursion order, or NULL
 *   ntriples : number of surviving leaf triples (even beyond cap)
 *   stats    : per-tier counts, or NULL
 *   threads  : > 1 runs output quadrants of the top tiers as OpenMP tasks (C only:
 *              triples and stats need threads == 1 so their order is fixed)
 * Returns 0, or 1 on bad arguments, 2 on allocation failure.
 */
int oracle_spamm_ex(const oracle_tree *A, const oracle_tree *B, double tau, int32_t depth_scaled,
                    int32_t threads, double *C, uint32_t *triples, int64_t cap, int64_t *ntriples,
                    oracle_stats *stats) {
  if (!compatible(A, B) || !(tau >= 0.0)) return 1;
  if (threads > 1 && (triples || stats)) return 1;
  rec_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.B = B; c.Av = A; c.Bv = B; c.tau = tau; c.trip = triples; c.cap = cap; c.st = stats;
  c.depth_scaled = depth_scaled != 0;
  if (stats) memset(stats, 0, sizeof *stats);
  double *Cp = NULL;
  if (C) {
    Cp = (double *)calloc((size_t)(A->N * A->N), sizeof(double));
    if (!Cp) return 2;
    c.C = Cp;
  }
  if (threads > 1) {
    c.task_depth = A->kmax < 4 ? A->kmax : 4;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#pragma omp single
#endif
    rec(&c, 0, 0, 0, 0);
  } else {
    c.task_depth = -1;
    rec(&c, 0, 0, 0, 0);
  }
  if (C) {
    for (int64_t i = 0; i < A->n; i++)
      memcpy(C + i * A->n, Cp + i * A->N, (size_t)A->n * sizeof(double));
    free(Cp);
  }
  if (ntriples) *ntriples = c.ntrip;
  return 0;
}

/* SpAMM(A, B) with the plain threshold (every tier tests against tau). */
int oracle_spamm(const oracle_tree *A, const oracle_tree *B, double tau, int32_t threads,
                 double *C, uint32_t *triples, int64_t cap, int64_t *ntriples,
                 oracle_stats *stats) {
  return oracle_spamm_ex(A, B, tau, 0, threads, C, triples, cap, ntriples, stats);
}

/*
 * SpAMM(A, B) with the tier tests of A and B (their FP64 norms) but the leaf products
 * A^k B^k taken from the values of Av and Bv (same n and leaf): the result of a leaf
 * arithmetic that rounds the operands first, e.g. to a narrower format, with every
 * surviving product then summed exactly as above in FP64.
 */
int oracle_spamm_values(const oracle_tree *A, const oracle_tree *B, const oracle_tree *Av,
                        const oracle_tree *Bv, double tau, int32_t threads, double *C) {
  if (!compatible(A, B) || !compatible(A, Av) || !compatible(B, Bv) || !(tau >= 0.0) || !C)
    return 1;
  rec_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.B = B; c.Av = Av; c.Bv = Bv; c.tau = tau;
  double *Cp = (double *)calloc((size_t)(A->N * A->N), sizeof(double));
  if (!Cp) return 2;
  c.C = Cp;
  if (threads > 1) {
    c.task_depth = A->kmax < 4 ? A->kmax : 4;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#pragma omp single
#endif
    rec(&c, 0, 0, 0, 0);
  } else {
    c.task_depth = -1;
    rec(&c, 0, 0, 0, 0);
  }
  for (int64_t i = 0; i < A->n; i++)
    memcpy(C + i * A->n, Cp + i * A->N, (size_t)A->n * sizeof(double));
  free(Cp);
  return 0;
}

/*
 * One output leaf block C_IJ (b x b, row-major) of SpAMM(A, B), with leaf products taken
 * from Av, Bv when given (NULL: from A, B): the same recursion,
 * followed only into the quadrants that contain block (I, J); every other output
 * block is independent of it, and its own sum runs in the same order as in the full
 * recursion.
 */
int oracle_spamm_block(const oracle_tree *A, const oracle_tree *B, const oracle_tree *Av,
                       const oracle_tree *Bv, double tau, int32_t I, int32_t J, double *out) {
  if (!Av) Av = A;
  if (!Bv) Bv = B;
  if (!compatible(A, B) || !compatible(A, Av) || !compatible(B, Bv) || !(tau >= 0.0) || I < 0 ||
      J < 0 || I >= A->NB || J >= A->NB)
    return 1;
  const int64_t b = A->b;
  /* accumulate straight into the b x b output block (I, J) */
  memset(out, 0, (size_t)(b * b) * sizeof(double));
  rec_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.B = B; c.Av = Av; c.Bv = Bv; c.tau = tau; c.task_depth = -1; c.target = 1; c.ti = I; c.tj = J;
  c.C = out;
  c.row0 = (int64_t)I * b; /* out row 0 is padded row I*b */
  c.col0 = (int64_t)J * b; /* out column 0 is padded column J*b */
  c.ldc = b;
  rec(&c, 0, 0, 0, 0);
  return 0;
}

/*
 * Brute force: every leaf triple (i, j, k) of the NB^3 product space, tested at the
 * leaf tier only, in lexicographic (i, j, k) order. Returns the count.
 */
int64_t oracle_triples_flat(const oracle_tree *A, const oracle_tree *B, double tau,
                            uint32_t *triples, int64_t cap) {
  if (!compatible(A, B)) return -1;
  const int64_t NB = A->NB;
  const double *na = level_ptr(A, A->kmax), *nb = level_ptr(B, B->kmax);
  int64_t cnt = 0;
  for (int64_t i = 0; i < NB; i++)
    for (int64_t j = 0; j < NB; j++)
      for (int64_t k = 0; k < NB; k++) {
        if (cull(na[i * NB + k], nb[k * NB + j], tau)) continue;
        if (triples && cnt < cap) {
          triples[3 * cnt] = (uint32_t)i;
          triples[3 * cnt + 1] = (uint32_t)j;
          triples[3 * cnt + 2] = (uint32_t)k;
        }
        cnt++;
      }
  return cnt;
}

/* Sum of ||A_ik|| ||B_kj|| over the leaf triples that fail the test: by the
   sub-multiplicative Frobenius norm (Eq. 3) and the triangle inequality, an upper
   bound on ||SpAMM(A,B) - AB||_F. */
double oracle_flat_bound(const oracle_tree *A, const oracle_tree *B, double tau) {
  const int64_t NB = A->NB;
  const double *na = level_ptr(A, A->kmax), *nb = level_ptr(B, B->kmax);
  double s = 0.0;
  for (int64_t i = 0; i < NB; i++)
    for (int64_t j = 0; j < NB; j++)
      for (int64_t k = 0; k < NB; k++)
        if (cull(na[i * NB + k], nb[k * NB + j], tau)) s += sqrt(na[i * NB + k]) * sqrt(nb[k * NB + j]);
  return s;
}

/* The ordinary product C = A B of n x n row-major matrices, i-k-j loop. */
void oracle_matmul_naive(const double *A, const double *B, int64_t n, double *C, int32_t threads) {
  (void)threads;
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads > 0 ? threads : 1) schedule(static)
#endif
  for (int64_t i = 0; i < n; i++) {
    double *c = C + i * n;
    for (int64_t q = 0; q < n; q++) c[q] = 0.0;
    for (int64_t l = 0; l < n; l++) {
      double a = A[i * n + l];
      const double *brow = B + l * n;
      for (int64_t q = 0; q < n; q++) c[q] += a * brow[q];
    }
  }
}

int32_t oracle_mutant(void) { return ORACLE_MUTANT; }

int32_t oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
