// SP2 density-matrix purification on SpAMM products (Sec. III: TC2 purification of the
// Fockian, energy Tr(H X) as the global error measure).
//
// X0 = (eps_max I - H) / (eps_max - eps_min) from Gershgorin bounds; each step forms
// C = SpAMM(X, X) with that step's tau, computes t1 = Tr X and t2 = Tr C in FP64 on the
// device, takes X <- C when |t2 - N_occ| <= |2 t1 - t2 - N_occ| and X <- 2X - C
// otherwise, and rebuilds the new iterate's leaf copies, norms and pyramid in place of
// C. The two trees then swap roles. The whole loop is ordered on the context stream;
// the host synchronises once, to read the result.
#include <cmath>
#include <vector>

#include "convert.cuh"
#include "internal.cuh"
#include "sync.cuh"

namespace {

struct StepRec {        // device record of a solve
  double trace[SPAMM_SP2_MAX_STEPS + 1];
  double trace2[SPAMM_SP2_MAX_STEPS + 1];
  int32_t branch[SPAMM_SP2_MAX_STEPS + 1];
  unsigned long long leaf_products[SPAMM_SP2_MAX_STEPS];
  double tau[SPAMM_SP2_MAX_STEPS];   // tolerances chosen on the device (learned steps)
  double energy;
};

// Dense X0 from the CSR of H: X0_ij = (eps_max delta_ij - H_ij) / (eps_max - eps_min).
__global__ void k_sp2_x0(int64_t n, const int64_t *indptr, const int64_t *indices, const double *data,
                         double emax, double inv_range, double *X) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double diag = emax;
    for (int64_t q = indptr[i]; q < indptr[i + 1]; q++) {
      const int64_t j = indices[q];
      if (j == i) diag -= data[q];
      else X[i * n + j] = -data[q] * inv_range;
    }
    X[i * n + i] = diag * inv_range;
  }
}

template <typename T>
__device__ __forceinline__ double diag_sum(const T *tiles, const uint8_t *nz, int64_t n, int32_t b, int32_t nb,
                                           int32_t NB, int32_t i) {
  if (!nz[(int64_t)i * NB + i]) return 0.0;
  const T *t = tiles + ((int64_t)i * nb + i) * b * b;
  double s = 0.0;
  const int64_t rest = n - (int64_t)i * b;
  const int lim = rest < b ? (int)rest : b;
  for (int r = 0; r < lim; r++) s += (double)t[r * b + r];
  return s;
}

// t1 = Tr X, t2 = Tr C (one CTA, fixed-order sums) and the branch of this step.
template <typename T>
__global__ void __launch_bounds__(1024) k_sp2_trace(const T *X, const uint8_t *nzX, const T *C, const uint8_t *nzC,
                                                    int64_t n, int32_t b, int32_t nb, int32_t NB, double n_occ,
                                                    int step, StepRec *rec) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += diag_sum(X, nzX, n, b, nb, NB, i);
    c += diag_sum(C, nzC, n, b, nb, NB, i);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = c;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double t1 = s1[0], t2 = s2[0];
    rec->trace[step] = t1;
    rec->trace2[step] = t2;
    rec->branch[step] = fabs(t2 - n_occ) <= fabs(2.0 * t1 - t2 - n_occ) ? 1 : 0;
  }
}

struct UpdArgs {
  const void *X;
  void *C;
  const uint8_t *nzX;
  uint8_t *nzC;
  double *leaf_norm2C;
  int32_t b, nb, NB;
  const StepRec *rec;
  int step;
  float *tf32, *tlo;
  uint16_t *bf16, *lo, *fp16;
};

__device__ __forceinline__ void df_add2(float &h, float &l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  float err = (h - (s - bb)) + (bh - bb);
  err += l + bl;
  h = s + err;
  l = err - (h - s);
}

// New iterate into C's tiles: C (branch X^2) or 2X - C; its leaf copies, squared norm
// and presence byte. One CTA per stored leaf; leaves absent from both X and C stay absent.
template <typename T>
__global__ void __launch_bounds__(256) k_sp2_update(UpdArgs p) {
  __shared__ double s_part[8];
  __shared__ float s_h[8], s_l[8];
  const int64_t leaf = blockIdx.x;
  const int32_t r = (int32_t)(leaf / p.nb), c = (int32_t)(leaf % p.nb);
  const int64_t li = (int64_t)r * p.NB + c;
  const bool sq = p.rec->branch[p.step] != 0;
  const bool hx = p.nzX[li] != 0, hc = p.nzC[li] != 0;
  const bool present = sq ? hc : (hx || hc);
  if (!present) {
    if (threadIdx.x == 0) {
      p.leaf_norm2C[li] = 0.0;
      p.nzC[li] = 0;
    }
    return;
  }
  const int64_t bb = (int64_t)p.b * p.b, base = leaf * bb;
  const T *X = (const T *)p.X;
  T *C = (T *)p.C;
  double sd = 0.0;
  float sh = 0.f, sl = 0.f;
  for (int64_t e = threadIdx.x; e < bb; e += blockDim.x) {
    const T cv = hc ? C[base + e] : (T)0;
    T v = cv;
    if (!sq) v = (T)2 * (hx ? X[base + e] : (T)0) - cv;
    if (!sq || !hc) C[base + e] = v;
    if (sizeof(T) == 8) {
      sd = fma((double)v, (double)v, sd);
    } else {
      const float f = (float)v;
      const float pp = f * f, er = fmaf(f, f, -pp);
      const float t = sh + pp, tb = t - sh;
      sl += ((sh - (t - tb)) + (pp - tb)) + er;
      sh = t;
    }
    if (p.bf16 || p.lo || p.tf32 || p.tlo || p.fp16) {
      Rounded h, t32, f16;
      uint32_t lo = 0, tl = 0;
      if (sizeof(T) == 8) {
        const uint64_t bits = (uint64_t)__double_as_longlong((double)v);
        h = round_f64bits(bits, 8, -126);
        if (p.lo) lo = bf16_lo_bits(bits, h);
        if (p.tf32 || p.tlo) t32 = round_f64bits(bits, 11, -126);
        if (p.tlo) tl = split_lo_bits(bits, t32, 11);
        if (p.fp16) f16 = round_f64bits(bits, 11, -14);
      } else {
        const float f = (float)v;
        h = round_f32(f, 8, -126);
        if (p.lo) lo = bf16_lo_bits_f32(f, h);
        if (p.tf32 || p.tlo) t32 = round_f32(f, 11, -126);
        if (p.tlo) tl = split_lo_bits_f32(f, t32, 11);
        if (p.fp16) f16 = round_f32(f, 11, -14);
      }
      if (p.bf16) p.bf16[base + e] = bf16_from_f32bits(h.bits);
      if (p.lo) p.lo[base + e] = bf16_from_f32bits(lo);
      if (p.tf32) p.tf32[base + e] = __uint_as_float(t32.bits);
      if (p.tlo) p.tlo[base + e] = __uint_as_float(tl);
      if (p.fp16) p.fp16[base + e] = fp16_from_f32bits(f16.bits);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (sizeof(T) == 8) {
    sd = warp_sum(sd);
    if (lane == 0) s_part[warp] = sd;
  } else {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, sh, off), l2 = __shfl_xor_sync(0xffffffffu, sl, off);
      df_add2(sh, sl, h2, l2);
    }
    if (lane == 0) {
      s_h[warp] = sh;
      s_l[warp] = sl;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; w++) s += sizeof(T) == 8 ? s_part[w] : ((double)s_h[w] + (double)s_l[w]);
    p.leaf_norm2C[li] = s;
    p.nzC[li] = 1;
  }
}

// E = Tr(H X) = sum over the nonzeros of H of H_ij X_ji; per-row FP64 sums, per-block
// partials, then a fixed-order total.
template <typename T>
__global__ void __launch_bounds__(256) k_sp2_energy(int64_t n, const int64_t *indptr, const int64_t *indices,
                                                    const double *data, const T *X, const uint8_t *nzX, int32_t b,
                                                    int32_t nb, int32_t NB, double *partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    for (int64_t q = indptr[i]; q < indptr[i + 1]; q++) {
      const int64_t j = indices[q];
      const int64_t lr = j / b, lc = i / b;
      if (!nzX[lr * NB + lc]) continue;
      acc += data[q] * (double)X[((lr * nb + lc) * b + (j % b)) * b + (i % b)];
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sp2_energy_total(const double *partial, int64_t np, StepRec *rec) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int64_t q = 0; q < np; q++) s += partial[q];
    rec->energy = s;
  }
}

__global__ void k_copy_counter(const unsigned long long *src, unsigned long long *dst) {
  if (threadIdx.x == 0) *dst = *src;
}

}  // namespace

// ---- host side (called from the C ABI in api.cu) ----
cudaError_t sp2_x0(int64_t n, const int64_t *indptr, const int64_t *indices, const double *data, double emin,
                   double emax, double *X, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(X, 0, (size_t)n * n * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_sp2_x0<<<grid, 256, 0, s>>>(n, indptr, indices, data, emax, 1.0 / (emax - emin), X);
  return cudaGetLastError();
}

size_t sp2_record_bytes() { return sizeof(StepRec); }

cudaError_t sp2_step_finish(spamm_tree X, spamm_tree C, double n_occ, int step, void *rec_v, cudaStream_t s) {
  StepRec *rec = (StepRec *)rec_v;
  k_copy_counter<<<1, 32, 0, s>>>(&C->counts->leaf_products, &rec->leaf_products[step]);
  const bool f64 = C->copy[CK_F64] != nullptr;
  if (f64)
    k_sp2_trace<double><<<1, 1024, 0, s>>>((const double *)X->copy[CK_F64], X->nz, (const double *)C->copy[CK_F64],
                                           C->nz, C->n, C->b, C->nb, C->NB, n_occ, step, rec);
  else
    k_sp2_trace<float><<<1, 1024, 0, s>>>((const float *)X->copy[CK_F32], X->nz, (const float *)C->copy[CK_F32],
                                          C->nz, C->n, C->b, C->nb, C->NB, n_occ, step, rec);
  UpdArgs u{};
  u.X = f64 ? X->copy[CK_F64] : X->copy[CK_F32];
  u.C = f64 ? C->copy[CK_F64] : C->copy[CK_F32];
  u.nzX = X->nz;
  u.nzC = C->nz;
  u.leaf_norm2C = C->norm2 + level_offset(C->kmax);
  u.b = C->b;
  u.nb = C->nb;
  u.NB = C->NB;
  u.rec = rec;
  u.step = step;
  u.tf32 = (float *)C->copy[CK_TF32];
  u.tlo = (float *)C->copy[CK_TF32LO];
  u.bf16 = (uint16_t *)C->copy[CK_BF16];
  u.lo = (uint16_t *)C->copy[CK_BF16LO];
  u.fp16 = (uint16_t *)C->copy[CK_FP16];
  const unsigned grid = (unsigned)((int64_t)C->nb * C->nb);
  if (f64) k_sp2_update<double><<<grid, 256, 0, s>>>(u);
  else k_sp2_update<float><<<grid, 256, 0, s>>>(u);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pyramid(C, s);   // the iterate is symmetric: the cull reads its upper triangle
}

cudaError_t sp2_trace_only(spamm_tree X, int idx, void *rec_v, cudaStream_t s) {
  // Tr X into trace[idx]: the trace kernel with X as both arguments (branch unused)
  StepRec *rec = (StepRec *)rec_v;
  const bool f64 = X->copy[CK_F64] != nullptr;
  if (f64)
    k_sp2_trace<double><<<1, 1024, 0, s>>>((const double *)X->copy[CK_F64], X->nz, (const double *)X->copy[CK_F64],
                                           X->nz, X->n, X->b, X->nb, X->NB, 0.0, idx, rec);
  else
    k_sp2_trace<float><<<1, 1024, 0, s>>>((const float *)X->copy[CK_F32], X->nz, (const float *)X->copy[CK_F32],
                                          X->nz, X->n, X->b, X->nb, X->NB, 0.0, idx, rec);
  return cudaGetLastError();
}

cudaError_t sp2_energy(spamm_tree X, int64_t n, const int64_t *indptr, const int64_t *indices,
                       const double *data, double *partial, void *rec_v, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  const bool f64 = X->copy[CK_F64] != nullptr;
  if (f64)
    k_sp2_energy<double><<<(unsigned)blocks, 256, 0, s>>>(n, indptr, indices, data, (const double *)X->copy[CK_F64],
                                                          X->nz, X->b, X->nb, X->NB, partial);
  else
    k_sp2_energy<float><<<(unsigned)blocks, 256, 0, s>>>(n, indptr, indices, data, (const float *)X->copy[CK_F32],
                                                         X->nz, X->b, X->nb, X->NB, partial);
  k_sp2_energy_total<<<1, 32, 0, s>>>(partial, blocks, (StepRec *)rec_v);
  return cudaGetLastError();
}

void sp2_read_record(const void *host_rec, int steps, spamm_sp2_result *out) {
  const StepRec *r = (const StepRec *)host_rec;
  out->energy = r->energy;
  for (int s = 0; s <= steps; s++) out->trace[s] = r->trace[s];
  for (int s = 0; s < steps; s++) {
    out->branch[s] = r->branch[s];
    out->leaf_products[s] = (int64_t)r->leaf_products[s];
    out->tau[s] = r->tau[s];
  }
}

double *sp2_tau_slot(void *rec, int step) { return &((StepRec *)rec)->tau[step]; }

namespace {

// log10 of the per-product error budget of step `step`: the base budget times
// clamp(m / mu_ref, 1, gain_max), m the relative margin of the step's branch decision,
// | |t2 - N| - |2 t1 - t2 - N| | / N, with t1 = Tr X (from the previous step's traces and
// branch) and t2 = Tr X^2 = ||X||_F^2 (X is symmetric: the root of its norm pyramid).
// Step 0 keeps the base budget.
__global__ void k_sp2_margin_budget(const StepRec *rec, int step, const double *x_norm2_root, double n_occ,
                                    double mu_ref, double gain_max, double log10_budget, double *out) {
  if (threadIdx.x != 0) return;
  double lb = log10_budget;
  if (step > 0) {
    const double tp = rec->trace[step - 1], tp2 = rec->trace2[step - 1];
    const double t1 = rec->branch[step - 1] ? tp2 : 2.0 * tp - tp2;
    const double t2 = *x_norm2_root;
    const double m = fabs(fabs(t2 - n_occ) - fabs(2.0 * t1 - t2 - n_occ)) / n_occ;
    lb += log10(fmin(gain_max, fmax(1.0, m / mu_ref)));
  }
  *out = lb;
}

}  // namespace

cudaError_t sp2_margin_budget(spamm_tree X, int step, void *rec, double n_occ, double mu_ref, double gain_max,
                              double log10_budget, double *out, cudaStream_t s) {
  k_sp2_margin_budget<<<1, 32, 0, s>>>((const StepRec *)rec, step, X->norm2, n_occ, mu_ref, gain_max, log10_budget,
                                       out);
  return cudaGetLastError();
}
