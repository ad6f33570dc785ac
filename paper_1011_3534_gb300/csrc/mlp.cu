// The tolerance controller's network on the GPU: a two-hidden-layer tanh perceptron
// with hand-written forward, backward and Adam kernels (FP32), features of a product
// read from the operands' norm trees, and the choice of the largest tolerance whose
// predicted error meets a budget. The paper has no counterpart; the controller serves
// the SP2 loop (Sec. III), where the error of each product feeds the energy error.
//
// Network: x (F) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) -> W3 h2 + b3 (1),
// parameters flat in the order W1 (H x F row-major), b1, W2 (H x H), b2, W3 (1 x H), b3.
// Loss (1 / 2N) sum (y_hat - y)^2; Adam with bias correction. Every reduction runs in a
// fixed order, so training is reproducible bit for bit.
#include <math.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "internal.cuh"
#include "sync.cuh"

namespace {

constexpr int kMaxF = 128, kMaxH = 64;

struct Net {
  int F, H;
  int oW1, ob1, oW2, ob2, oW3, ob3, P;
};

Net layout(int F, int H) {
  Net n;
  n.F = F;
  n.H = H;
  n.oW1 = 0;
  n.ob1 = n.oW1 + H * F;
  n.oW2 = n.ob1 + H;
  n.ob2 = n.oW2 + H * H;
  n.oW3 = n.ob2 + H;
  n.ob3 = n.oW3 + H;
  n.P = n.ob3 + 1;
  return n;
}

// One thread per sample: activations h1, h2 and the prediction.
__global__ void k_forward(Net n, const float *__restrict__ th, const float *__restrict__ X,
                          const int *__restrict__ idx, int N, float *h1, float *h2, float *yh) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const float *x = X + (int64_t)(idx ? idx[s] : s) * n.F;
  float a1[kMaxH], a2[kMaxH];
  for (int j = 0; j < n.H; j++) {
    float acc = th[n.ob1 + j];
    for (int k = 0; k < n.F; k++) acc = fmaf(th[n.oW1 + j * n.F + k], x[k], acc);
    a1[j] = tanhf(acc);
  }
  for (int j = 0; j < n.H; j++) {
    float acc = th[n.ob2 + j];
    for (int k = 0; k < n.H; k++) acc = fmaf(th[n.oW2 + j * n.H + k], a1[k], acc);
    a2[j] = tanhf(acc);
  }
  float o = th[n.ob3];
  for (int k = 0; k < n.H; k++) o = fmaf(th[n.oW3 + k], a2[k], o);
  yh[s] = o;
  if (h1)
    for (int j = 0; j < n.H; j++) {
      h1[(int64_t)s * n.H + j] = a1[j];
      h2[(int64_t)s * n.H + j] = a2[j];
    }
}

// One thread per sample: deltas d3 = (y_hat - y) / N, d2, d1 of back-propagation.
__global__ void k_deltas(Net n, const float *__restrict__ th, const float *__restrict__ y,
                         const int *__restrict__ idx, int N, const float *yh, const float *h1, const float *h2,
                         float *d3, float *d2, float *d1) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const float r = (yh[s] - y[idx ? idx[s] : s]) / (float)N;
  d3[s] = r;
  float e2[kMaxH];
  for (int j = 0; j < n.H; j++) {
    const float h = h2[(int64_t)s * n.H + j];
    e2[j] = r * th[n.oW3 + j] * (1.f - h * h);
    d2[(int64_t)s * n.H + j] = e2[j];
  }
  for (int k = 0; k < n.H; k++) {
    float acc = 0.f;
    for (int j = 0; j < n.H; j++) acc = fmaf(e2[j], th[n.oW2 + j * n.H + k], acc);
    const float h = h1[(int64_t)s * n.H + k];
    d1[(int64_t)s * n.H + k] = acc * (1.f - h * h);
  }
}

// One thread per parameter: its gradient summed over the samples in order.
__global__ void k_weight_grads(Net n, const float *__restrict__ X, const int *__restrict__ idx, int N,
                               const float *h1, const float *h2, const float *d3, const float *d2,
                               const float *d1, float *g) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n.P) return;
  float acc = 0.f;
  if (q < n.ob1) {                 // W1[j][k] = sum d1[j] x[k]
    const int j = q / n.F, k = q % n.F;
    for (int s = 0; s < N; s++) acc = fmaf(d1[(int64_t)s * n.H + j], X[(int64_t)(idx ? idx[s] : s) * n.F + k], acc);
  } else if (q < n.oW2) {          // b1[j]
    const int j = q - n.ob1;
    for (int s = 0; s < N; s++) acc += d1[(int64_t)s * n.H + j];
  } else if (q < n.ob2) {          // W2[j][k] = sum d2[j] h1[k]
    const int j = (q - n.oW2) / n.H, k = (q - n.oW2) % n.H;
    for (int s = 0; s < N; s++) acc = fmaf(d2[(int64_t)s * n.H + j], h1[(int64_t)s * n.H + k], acc);
  } else if (q < n.oW3) {          // b2[j]
    const int j = q - n.ob2;
    for (int s = 0; s < N; s++) acc += d2[(int64_t)s * n.H + j];
  } else if (q < n.ob3) {          // W3[k] = sum d3 h2[k]
    const int k = q - n.oW3;
    for (int s = 0; s < N; s++) acc = fmaf(d3[s], h2[(int64_t)s * n.H + k], acc);
  } else {                         // b3
    for (int s = 0; s < N; s++) acc += d3[s];
  }
  g[q] = acc;
}

__global__ void k_loss(const float *yh, const float *y, const int *idx, int N, float *out) {
  __shared__ float sh[256];
  float acc = 0.f;
  for (int s = threadIdx.x; s < N; s += blockDim.x) {
    const float r = yh[s] - y[idx ? idx[s] : s];
    acc = fmaf(r, r, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5f * sh[0] / (float)N;
}

__global__ void k_adam(int P, float *th, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.f - b1) * gq;
  const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  th[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + eps);
}

}  // namespace

struct spamm_mlp_s {
  spamm_ctx ctx = nullptr;
  Net net{};
  float *th = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  int t = 0;
  // batch buffers
  int cap = 0;
  float *X = nullptr, *y = nullptr, *h1 = nullptr, *h2 = nullptr, *yh = nullptr, *d1 = nullptr, *d2 = nullptr,
        *d3 = nullptr, *loss = nullptr;
  int *idx = nullptr;
};

namespace {

spamm_status mfail(spamm_ctx ctx, spamm_status st, const char *msg) {
  if (ctx) ctx->err = msg;
  return st;
}

cudaError_t ensure_cap(spamm_mlp mm, int N) {
  if (mm->cap >= N) return cudaSuccess;
  cudaFree(mm->X); cudaFree(mm->y); cudaFree(mm->h1); cudaFree(mm->h2); cudaFree(mm->yh);
  cudaFree(mm->d1); cudaFree(mm->d2); cudaFree(mm->d3); cudaFree(mm->idx);
  const int F = mm->net.F, H = mm->net.H;
  cudaError_t e = cudaMalloc(&mm->X, sizeof(float) * (size_t)N * F);
  if (e == cudaSuccess) e = cudaMalloc(&mm->y, sizeof(float) * N);
  if (e == cudaSuccess) e = cudaMalloc(&mm->h1, sizeof(float) * (size_t)N * H);
  if (e == cudaSuccess) e = cudaMalloc(&mm->h2, sizeof(float) * (size_t)N * H);
  if (e == cudaSuccess) e = cudaMalloc(&mm->yh, sizeof(float) * N);
  if (e == cudaSuccess) e = cudaMalloc(&mm->d1, sizeof(float) * (size_t)N * H);
  if (e == cudaSuccess) e = cudaMalloc(&mm->d2, sizeof(float) * (size_t)N * H);
  if (e == cudaSuccess) e = cudaMalloc(&mm->d3, sizeof(float) * N);
  if (e == cudaSuccess) e = cudaMalloc(&mm->idx, sizeof(int) * N);
  if (e == cudaSuccess) mm->cap = N;
  return e;
}

// forward + deltas + gradients (+ loss) of samples idx (or 0..N-1) of the uploaded data
cudaError_t run_grad(spamm_mlp mm, int N, const int *idx, cudaStream_t s) {
  const Net &n = mm->net;
  const unsigned gs = (unsigned)((N + 127) / 128);
  k_forward<<<gs, 128, 0, s>>>(n, mm->th, mm->X, idx, N, mm->h1, mm->h2, mm->yh);
  k_deltas<<<gs, 128, 0, s>>>(n, mm->th, mm->y, idx, N, mm->yh, mm->h1, mm->h2, mm->d3, mm->d2, mm->d1);
  k_weight_grads<<<(unsigned)((n.P + 127) / 128), 128, 0, s>>>(n, mm->X, idx, N, mm->h1, mm->h2, mm->d3, mm->d2,
                                                               mm->d1, mm->g);
  k_loss<<<1, 256, 0, s>>>(mm->yh, mm->y, idx, N, mm->loss);
  mm->ctx->launches += 4;
  return cudaGetLastError();
}

cudaError_t run_adam(spamm_mlp mm, float lr, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  mm->t++;
  const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, mm->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, mm->t)));
  k_adam<<<(unsigned)((mm->net.P + 255) / 256), 256, 0, s>>>(mm->net.P, mm->th, mm->g, mm->m, mm->v, lr, b1, b2,
                                                             eps, c1, c2);
  mm->ctx->launches++;
  return cudaGetLastError();
}

uint64_t smix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

spamm_status spamm_mlp_create(spamm_ctx ctx, int32_t inputs, int32_t hidden, uint64_t seed, spamm_mlp *out) {
  if (!ctx || !out) return SPAMM_EINVAL;
  if (inputs < 1 || inputs > kMaxF || hidden < 1 || hidden > kMaxH)
    return mfail(ctx, SPAMM_EINVAL, "mlp_create: 1 <= inputs <= 128, 1 <= hidden <= 64");
  spamm_mlp mm = new (std::nothrow) spamm_mlp_s();
  if (!mm) return SPAMM_ENOMEM;
  mm->ctx = ctx;
  mm->net = layout(inputs, hidden);
  const int P = mm->net.P;
  // weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64, biases 0
  std::vector<float> th(P, 0.f);
  uint64_t st = seed;
  auto uni = [&]() { st += 0x9E3779B97F4A7C15ull; return (double)(smix(st) >> 11) * (1.0 / 9007199254740992.0); };
  const Net &n = mm->net;
  for (int q = n.oW1; q < n.ob1; q++) th[q] = (float)((2 * uni() - 1) / std::sqrt((double)inputs));
  for (int q = n.oW2; q < n.ob2; q++) th[q] = (float)((2 * uni() - 1) / std::sqrt((double)hidden));
  for (int q = n.oW3; q < n.ob3; q++) th[q] = (float)((2 * uni() - 1) / std::sqrt((double)hidden));
  cudaError_t e = cudaMalloc(&mm->th, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMalloc(&mm->m, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMalloc(&mm->v, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMalloc(&mm->g, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMalloc(&mm->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(mm->th, th.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(mm->m, 0, sizeof(float) * P);
  if (e == cudaSuccess) e = cudaMemset(mm->v, 0, sizeof(float) * P);
  if (e != cudaSuccess) {
    spamm_mlp_free(mm);
    ctx->err = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SPAMM_ENOMEM : SPAMM_ECUDA;
  }
  *out = mm;
  return SPAMM_OK;
}

spamm_status spamm_mlp_free(spamm_mlp mm) {
  if (!mm) return SPAMM_EINVAL;
  cudaStreamSynchronize(mm->ctx->stream);
  for (void *p : {(void *)mm->th, (void *)mm->m, (void *)mm->v, (void *)mm->g, (void *)mm->X, (void *)mm->y,
                  (void *)mm->h1, (void *)mm->h2, (void *)mm->yh, (void *)mm->d1, (void *)mm->d2, (void *)mm->d3,
                  (void *)mm->loss, (void *)mm->idx})
    if (p) cudaFree(p);
  delete mm;
  return SPAMM_OK;
}

int32_t spamm_mlp_num_params(spamm_mlp mm) { return mm ? mm->net.P : -1; }

spamm_status spamm_mlp_get_params(spamm_mlp mm, float *out, int32_t cap) {
  if (!mm || !out || cap < mm->net.P) return SPAMM_EINVAL;
  if (cudaMemcpyAsync(out, mm->th, sizeof(float) * mm->net.P, cudaMemcpyDeviceToHost, mm->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(mm->ctx->stream) != cudaSuccess)
    return SPAMM_ECUDA;
  return SPAMM_OK;
}

spamm_status spamm_mlp_set_params(spamm_mlp mm, const float *in, int32_t count) {
  if (!mm || !in || count != mm->net.P) return SPAMM_EINVAL;
  if (cudaMemcpyAsync(mm->th, in, sizeof(float) * count, cudaMemcpyHostToDevice, mm->ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(mm->m, 0, sizeof(float) * count, mm->ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(mm->v, 0, sizeof(float) * count, mm->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(mm->ctx->stream) != cudaSuccess)
    return SPAMM_ECUDA;
  mm->t = 0;
  return SPAMM_OK;
}

// y = network(X) for N samples of F features (host arrays).
spamm_status spamm_mlp_forward(spamm_mlp mm, const float *X, int32_t N, float *y) {
  if (!mm || !X || !y || N < 1) return SPAMM_EINVAL;
  cudaStream_t s = mm->ctx->stream;
  if (ensure_cap(mm, N) != cudaSuccess) return SPAMM_ENOMEM;
  cudaMemcpyAsync(mm->X, X, sizeof(float) * (size_t)N * mm->net.F, cudaMemcpyHostToDevice, s);
  k_forward<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(mm->net, mm->th, mm->X, nullptr, N, nullptr, nullptr, mm->yh);
  mm->ctx->launches++;
  cudaMemcpyAsync(y, mm->yh, sizeof(float) * N, cudaMemcpyDeviceToHost, s);
  return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

// Loss and gradient of the parameters on N samples (host arrays), no update.
spamm_status spamm_mlp_gradient(spamm_mlp mm, const float *X, const float *y, int32_t N, float *grad, float *loss) {
  if (!mm || !X || !y || N < 1) return SPAMM_EINVAL;
  cudaStream_t s = mm->ctx->stream;
  if (ensure_cap(mm, N) != cudaSuccess) return SPAMM_ENOMEM;
  cudaMemcpyAsync(mm->X, X, sizeof(float) * (size_t)N * mm->net.F, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(mm->y, y, sizeof(float) * N, cudaMemcpyHostToDevice, s);
  if (run_grad(mm, N, nullptr, s) != cudaSuccess) return SPAMM_ECUDA;
  if (grad) cudaMemcpyAsync(grad, mm->g, sizeof(float) * mm->net.P, cudaMemcpyDeviceToHost, s);
  if (loss) cudaMemcpyAsync(loss, mm->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  return cudaStreamSynchronize(s) == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

// One Adam step (learning rate lr) on N samples (host arrays).
spamm_status spamm_mlp_adam_step(spamm_mlp mm, const float *X, const float *y, int32_t N, float lr, float *loss) {
  spamm_status st = spamm_mlp_gradient(mm, X, y, N, nullptr, loss);
  if (st != SPAMM_OK) return st;
  if (run_adam(mm, lr, mm->ctx->stream) != cudaSuccess) return SPAMM_ECUDA;
  return cudaStreamSynchronize(mm->ctx->stream) == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

// One Adam step with a caller-supplied gradient (host array of num_params floats).
spamm_status spamm_mlp_adam_apply(spamm_mlp mm, const float *grad, float lr) {
  if (!mm || !grad) return SPAMM_EINVAL;
  cudaStream_t s = mm->ctx->stream;
  if (cudaMemcpyAsync(mm->g, grad, sizeof(float) * mm->net.P, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SPAMM_ECUDA;
  if (run_adam(mm, lr, s) != cudaSuccess) return SPAMM_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

// Mini-batch Adam over N samples (host arrays, uploaded once): `epochs` passes, each over
// a SplitMix64 permutation of the samples in batches of `batch`. Returns the final
// full-data loss.
spamm_status spamm_mlp_train(spamm_mlp mm, const float *X, const float *y, int32_t N, int32_t epochs,
                             int32_t batch, float lr, uint64_t seed, float *final_loss) {
  if (!mm || !X || !y || N < 1 || epochs < 0 || batch < 1) return SPAMM_EINVAL;
  cudaStream_t s = mm->ctx->stream;
  if (ensure_cap(mm, N) != cudaSuccess) return SPAMM_ENOMEM;
  cudaMemcpyAsync(mm->X, X, sizeof(float) * (size_t)N * mm->net.F, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(mm->y, y, sizeof(float) * N, cudaMemcpyHostToDevice, s);
  std::vector<int> perm(N);
  int *hperm = nullptr;
  if (cudaMallocHost(&hperm, sizeof(int) * (size_t)N * 2) != cudaSuccess) return SPAMM_ENOMEM;
  uint64_t st = seed;
  for (int ep = 0; ep < epochs; ep++) {
    for (int q = 0; q < N; q++) perm[q] = q;
    for (int q = N - 1; q > 0; q--) {   // Fisher-Yates
      st += 0x9E3779B97F4A7C15ull;
      const int r = (int)(smix(st) % (uint64_t)(q + 1));
      std::swap(perm[q], perm[r]);
    }
    int *buf = hperm + (ep & 1) * N;   // alternate halves: the previous epoch may still read one
    cudaStreamSynchronize(s);
    memcpy(buf, perm.data(), sizeof(int) * N);
    cudaMemcpyAsync(mm->idx, buf, sizeof(int) * N, cudaMemcpyHostToDevice, s);
    for (int b0 = 0; b0 < N; b0 += batch) {
      const int nb = std::min(batch, N - b0);
      if (run_grad(mm, nb, mm->idx + b0, s) != cudaSuccess || run_adam(mm, lr, s) != cudaSuccess) {
        cudaFreeHost(hperm);
        return SPAMM_ECUDA;
      }
    }
  }
  cudaError_t e = run_grad(mm, N, nullptr, s);
  if (final_loss) cudaMemcpyAsync(final_loss, mm->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFreeHost(hperm);
  return e == cudaSuccess && e2 == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- controller features
// Features of a product A B at tolerance tau (SPAMM_MLP_FEATURES = 69). Per operand, for
// its leaf tier and the tier above: a 16-bin histogram of block norms in decades below
// the tier's largest norm (bin q holds the blocks with max * 10^-(q+1) <= norm <
// max * 10^-q, bin 15 everything further down), as fractions of the tier's nonzero
// blocks. Then (log10 tau - log10 ||A||_F - log10 ||B||_F) / 8, (log10 ||A||_F +
// log10 ||B||_F) / 8, the fraction of nonzero leaves of A and of B, and
// (log10 bound(tau) - log10 ||A||_F - log10 ||B||_F) / 8 of the flat leaf bound below
// (-2 when it is zero, the floor of the feature). The bin of a
// block is decided by FP64 comparisons of its squared norm against max^2 * 10^(-2q), so
// the histogram is exact integer work.
namespace {

constexpr int kHist = 16;
constexpr int kTreeFeat = kTreeFeatures;   // two histograms, nonzero fraction, log10 norm
static_assert(kTreeFeat == 2 * kHist + 2, "per-tree feature count");
static_assert(SPAMM_MLP_FEATURES == 2 * kTreeFeat + 1, "feature layout");

__device__ __constant__ double c_decade2[kHist] = {1e-2,  1e-4,  1e-6,  1e-8,  1e-10, 1e-12, 1e-14, 1e-16,
                                                   1e-18, 1e-20, 1e-22, 1e-24, 1e-26, 1e-28, 1e-30, 1e-32};

// Histogram of the side x side tier `t2` into out[0..15]; *nzc gets its nonzero count.
__device__ void tier_hist(const double *t2, int64_t cells, double *s_red, double *s_thr, int *s_hist,
                          int *s_cnt, float *out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double mx = 0.0;
  for (int64_t q = tid; q < cells; q += blockDim.x) mx = fmax(mx, t2[q]);
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) s_red[warp] = mx;
  if (tid < kHist) s_hist[tid] = 0;
  if (tid == 0) *s_cnt = 0;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; w++) m = fmax(m, s_red[w]);
    for (int q = 0; q < kHist - 1; q++) s_thr[q] = m * c_decade2[q];
  }
  __syncthreads();
  int cnz = 0;
  for (int64_t q = tid; q < cells; q += blockDim.x) {
    const double v = t2[q];
    if (!(v > 0.0)) continue;
    cnz++;
    int bin = 0;
    while (bin < kHist - 1 && v < s_thr[bin]) bin++;
    atomicAdd(&s_hist[bin], 1);
  }
  atomicAdd(s_cnt, cnz);
  __syncthreads();
  const int c = *s_cnt;
  if (tid < kHist) out[tid] = c ? (float)s_hist[tid] / (float)c : 0.f;
  __syncthreads();
}

// out[0..15] leaf-tier histogram, out[16..31] the tier above, out[32] fraction of the
// nb x nb leaves that are nonzero, out[33] log10 ||A||_F
__global__ void __launch_bounds__(1024) k_feat_hist(const double *norm2, int kmax, int nb, float *out) {
  __shared__ double s_red[32], s_thr[kHist];
  __shared__ int s_hist[kHist], s_cnt, s_leaf_nz;
  const int lp = kmax > 0 ? kmax - 1 : 0;
  tier_hist(norm2 + level_offset(kmax), (int64_t)1 << (2 * kmax), s_red, s_thr, s_hist, &s_cnt, out);
  if (threadIdx.x == 0) s_leaf_nz = s_cnt;
  tier_hist(norm2 + level_offset(lp), (int64_t)1 << (2 * lp), s_red, s_thr, s_hist, &s_cnt, out + kHist);
  if (threadIdx.x == 0) {
    out[2 * kHist] = (float)s_leaf_nz / (float)((int64_t)nb * nb);
    out[2 * kHist + 1] = norm2[0] > 0.0 ? (float)(0.5 * log10(norm2[0])) : -300.f;
  }
}

// Flat leaf bound of the product at each tolerance of a grid: the sum of
// p = ||A_ik||_F ||B_kj||_F over the leaf triples with p < tau_q, the norms and p in FP32
// (the decision p < tau_q is taken in FP32 against tau_q rounded to FP32). It bounds the
// Frobenius error of the product at tau_q (triangle inequality over the dropped
// triples). One CTA per leaf row i: row i of A's norms staged in shared memory, threads
// over columns j, per-thread FP32 sums, fixed-order reductions, FP64 partial per row.
constexpr int kGrid = 37;   // tolerance grid of the selection
constexpr int kBoundThreads = 256;
constexpr int kBoundChunk = 2048;   // k-chunk of A's row staged at a time

template <int G>
__global__ void __launch_bounds__(kBoundThreads) k_flat_bound(const double *nA, const double *nB, int NB,
                                                              const double *grid, double *partial) {
  __shared__ float s_a[kBoundChunk];
  __shared__ float s_thr[G];
  __shared__ float s_w[kBoundThreads / 32][G];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < G) s_thr[tid] = (float)grid[tid];
  float bins[G];
#pragma unroll
  for (int q = 0; q < G; q++) bins[q] = 0.f;
  for (int k0 = 0; k0 < NB; k0 += kBoundChunk) {
    const int kn = NB - k0 < kBoundChunk ? NB - k0 : kBoundChunk;
    __syncthreads();
    for (int k = tid; k < kn; k += kBoundThreads) s_a[k] = (float)nA[(int64_t)i * NB + k0 + k];
    __syncthreads();
    for (int j = tid; j < NB; j += kBoundThreads) {
      for (int k = 0; k < kn; k++) {
        const float a = s_a[k];
        if (a == 0.f) continue;
        const float pr = a * (float)nB[(int64_t)(k0 + k) * NB + j];
        if (pr == 0.f) continue;
#pragma unroll
        for (int q = 0; q < G; q++) bins[q] += pr < s_thr[q] ? pr : 0.f;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < G; q++) {
    float v = bins[q];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_w[warp][q] = v;
  }
  __syncthreads();
  if (tid < G) {
    double t = 0.0;
    for (int w = 0; w < kBoundThreads / 32; w++) t += (double)s_w[w][tid];
    partial[(int64_t)i * G + tid] = t;
  }
}

__global__ void k_bound_total(const double *partial, int NB, int G, double *bound) {
  const int q = threadIdx.x;
  if (q >= G) return;
  double t = 0.0;
  for (int i = 0; i < NB; i++) t += partial[(int64_t)i * G + q];
  bound[q] = t;
}

// The network's input for tolerance log10_tau with flat bound `bound`.
__device__ __forceinline__ void assemble(const float *fa, const float *fb, double log10_tau, double bound, float *f) {
  for (int q = 0; q < 2 * kHist; q++) {
    f[q] = fa[q];
    f[2 * kHist + q] = fb[q];
  }
  const double la = (double)fa[2 * kHist + 1], lb = (double)fb[2 * kHist + 1];
  f[4 * kHist] = (float)((log10_tau - la - lb) / 8.0);
  f[4 * kHist + 1] = (float)((la + lb) / 8.0);
  f[4 * kHist + 2] = fa[2 * kHist];
  f[4 * kHist + 3] = fb[2 * kHist];
  double lr = bound > 0.0 ? (log10(bound) - la - lb) / 8.0 : -2.0;
  f[4 * kHist + 4] = (float)(lr < -2.0 ? -2.0 : lr);
}

__device__ float net_eval(const Net &n, const float *th, const float *x) {
  float a1[kMaxH], a2[kMaxH];
  for (int j = 0; j < n.H; j++) {
    float acc = th[n.ob1 + j];
    for (int k = 0; k < n.F; k++) acc = fmaf(th[n.oW1 + j * n.F + k], x[k], acc);
    a1[j] = tanhf(acc);
  }
  for (int j = 0; j < n.H; j++) {
    float acc = th[n.ob2 + j];
    for (int k = 0; k < n.H; k++) acc = fmaf(th[n.oW2 + j * n.H + k], a1[k], acc);
    a2[j] = tanhf(acc);
  }
  float o = th[n.ob3];
  for (int k = 0; k < n.H; k++) o = fmaf(th[n.oW3 + k], a2[k], o);
  return o;
}

// Thread g scores grid[g] (ascending); the largest grid[g] whose predicted log10
// relative error is within the budget is written to *tau_out (grid[0] when none is).
__global__ void __launch_bounds__(128) k_tau_select(Net n, const float *th, const float *fa, const float *fb,
                                                    const double *grid, const double *bound, int G,
                                                    double log10_budget, const double *log10_budget_dev,
                                                    double *tau_out) {
  __shared__ int s_best;
  if (threadIdx.x == 0) s_best = -1;
  __syncthreads();
  const int g = threadIdx.x;
  const double lb = log10_budget_dev ? *log10_budget_dev : log10_budget;   // a budget chosen on the device
  if (g < G) {
    float f[SPAMM_MLP_FEATURES];
    assemble(fa, fb, log10(grid[g]), bound[g], f);
    const float pred = net_eval(n, th, f);
    if (pred <= (float)lb) atomicMax(&s_best, g);
  }
  __syncthreads();
  if (threadIdx.x == 0) *tau_out = grid[s_best < 0 ? 0 : s_best];
}

__global__ void k_feat_assemble(const float *fa, const float *fb, double log10_tau, const double *bound, float *f) {
  if (threadIdx.x == 0) assemble(fa, fb, log10_tau, bound[0], f);
}

}  // namespace

cudaError_t launch_feat_hist(spamm_tree t, float *out, cudaStream_t s) {
  k_feat_hist<<<1, 1024, 0, s>>>(t->norm2, t->kmax, t->nb, out);
  return cudaGetLastError();
}

size_t bound_workspace_doubles(spamm_tree A) { return (size_t)A->NB * kGrid + kGrid; }

cudaError_t launch_flat_bound(spamm_tree A, spamm_tree B, const double *grid, int G, double *work, double *bound,
                              cudaStream_t s) {
  const double *nA = A->norm + level_offset(A->kmax), *nB = B->norm + level_offset(B->kmax);
  if (G == 1) k_flat_bound<1><<<(unsigned)A->NB, kBoundThreads, 0, s>>>(nA, nB, A->NB, grid, work);
  else if (G == kGrid) k_flat_bound<kGrid><<<(unsigned)A->NB, kBoundThreads, 0, s>>>(nA, nB, A->NB, grid, work);
  else return cudaErrorInvalidValue;
  k_bound_total<<<1, 64, 0, s>>>(work, A->NB, G, bound);
  return cudaGetLastError();
}

cudaError_t launch_tau_select(spamm_mlp mm, const float *fa, const float *fb, const double *grid, const double *bound,
                              double log10_budget, double *tau_out, cudaStream_t s, const double *log10_budget_dev) {
  k_tau_select<<<1, 128, 0, s>>>(mm->net, mm->th, fa, fb, grid, bound, kGrid, log10_budget, log10_budget_dev, tau_out);
  return cudaGetLastError();
}

void tau_grid(double tau_min, double tau_max, double *grid) {
  const double l0 = std::log10(tau_min), l1 = std::log10(tau_max);
  for (int g = 0; g < kGrid; g++) grid[g] = std::pow(10.0, l0 + (l1 - l0) * g / (kGrid - 1));
}

int mlp_inputs(spamm_mlp mm) { return mm->net.F; }

extern "C" {

spamm_status spamm_features(spamm_tree A, spamm_tree B, double tau, float *out) {
  if (A && settle(A->ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!A || !B || !out || !(tau > 0.0) || !std::isfinite(tau)) return SPAMM_EINVAL;
  spamm_ctx ctx = A->ctx;
  if (A->n != B->n || A->b != B->b) return mfail(ctx, SPAMM_EINVAL, "features: shapes differ");
  float *d = nullptr;
  double *w = nullptr;
  const size_t nw = (size_t)A->NB + 4;
  if (cudaMalloc(&d, sizeof(float) * (2 * kTreeFeat + SPAMM_MLP_FEATURES)) != cudaSuccess) return SPAMM_ENOMEM;
  if (cudaMalloc(&w, sizeof(double) * nw) != cudaSuccess) { cudaFree(d); return SPAMM_ENOMEM; }
  cudaStream_t s = ctx->stream;
  double *grid = w + A->NB, *bound = w + A->NB + 1;
  cudaError_t e = cudaMemcpyAsync(grid, &tau, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_feat_hist(A, d, s);
  if (e == cudaSuccess) e = launch_feat_hist(B, d + kTreeFeat, s);
  if (e == cudaSuccess) e = launch_flat_bound(A, B, grid, 1, w, bound, s);
  if (e == cudaSuccess) {
    k_feat_assemble<<<1, 32, 0, s>>>(d, d + kTreeFeat, log10(tau), bound, d + 2 * kTreeFeat);
    e = cudaGetLastError();
  }
  ctx->launches += 5;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 2 * kTreeFeat, sizeof(float) * SPAMM_MLP_FEATURES, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  cudaFree(w);
  return e == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

spamm_status spamm_tau_select(spamm_mlp mm, spamm_tree A, spamm_tree B, double err_budget, double tau_min,
                              double tau_max, double *tau_out) {
  if (A && settle(A->ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!mm || !A || !B || !tau_out || !(err_budget > 0.0) || !(tau_min > 0.0) || !(tau_max >= tau_min) ||
      !std::isfinite(tau_max))
    return SPAMM_EINVAL;
  spamm_ctx ctx = A->ctx;
  if (mm->net.F != SPAMM_MLP_FEATURES) return mfail(ctx, SPAMM_EINVAL, "tau_select: network input width");
  if (A->n != B->n || A->b != B->b) return mfail(ctx, SPAMM_EINVAL, "tau_select: shapes differ");
  float *d = nullptr;
  double *w = nullptr;
  const size_t nw = bound_workspace_doubles(A) + kGrid + 1;
  if (cudaMalloc(&d, sizeof(float) * 2 * kTreeFeat) != cudaSuccess) return SPAMM_ENOMEM;
  if (cudaMalloc(&w, sizeof(double) * nw) != cudaSuccess) { cudaFree(d); return SPAMM_ENOMEM; }
  double hgrid[kGrid];
  tau_grid(tau_min, tau_max, hgrid);
  double *grid = w + bound_workspace_doubles(A), *dt = grid + kGrid, *bound = w + (size_t)A->NB * kGrid;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(grid, hgrid, sizeof hgrid, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_feat_hist(A, d, s);
  if (e == cudaSuccess) e = launch_feat_hist(B, d + kTreeFeat, s);
  if (e == cudaSuccess) e = launch_flat_bound(A, B, grid, kGrid, w, bound, s);
  if (e == cudaSuccess) e = launch_tau_select(mm, d, d + kTreeFeat, grid, bound, log10(err_budget), dt, s);
  ctx->launches += 5;
  if (e == cudaSuccess) e = cudaMemcpyAsync(tau_out, dt, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  cudaFree(w);
  return e == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- tree distance
// ||X - Y||_F and ||Y||_F of two trees of the same shape (FP64 or FP32 tiles), for the
// labels of the controller: one CTA per stored leaf, FP64 partials, fixed-order total.
namespace {

template <typename TX, typename TY>
__global__ void __launch_bounds__(256) k_dist(const TX *X, const uint8_t *nzX, const TY *Y, const uint8_t *nzY,
                                              int32_t b, int32_t nb, int32_t NB, double *part) {
  __shared__ double s1[256], s2[256];
  const int64_t leaf = blockIdx.x;
  const int32_t r = (int32_t)(leaf / nb), c = (int32_t)(leaf % nb);
  const bool hx = nzX[(int64_t)r * NB + c] != 0, hy = nzY[(int64_t)r * NB + c] != 0;
  double a = 0.0, q = 0.0;
  if (hx || hy) {
    const int64_t bb = (int64_t)b * b, base = leaf * bb;
    for (int64_t e = threadIdx.x; e < bb; e += blockDim.x) {
      const double x = hx ? (double)X[base + e] : 0.0, y = hy ? (double)Y[base + e] : 0.0;
      a = fma(x - y, x - y, a);
      q = fma(y, y, q);
    }
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = q;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * leaf] = s1[0];
    part[2 * leaf + 1] = s2[0];
  }
}

__global__ void k_dist_total(const double *part, int64_t nleaves, double *out) {
  if (threadIdx.x == 0) {
    double a = 0.0, q = 0.0;
    for (int64_t l = 0; l < nleaves; l++) {
      a += part[2 * l];
      q += part[2 * l + 1];
    }
    out[0] = sqrt(a);
    out[1] = sqrt(q);
  }
}

template <typename TX>
cudaError_t dist_y(const TX *X, spamm_tree x, spamm_tree y, double *part, cudaStream_t s) {
  const unsigned grid = (unsigned)((int64_t)x->nb * x->nb);
  if (y->copy[CK_F64])
    k_dist<TX, double><<<grid, 256, 0, s>>>(X, x->nz, (const double *)y->copy[CK_F64], y->nz, x->b, x->nb, x->NB, part);
  else
    k_dist<TX, float><<<grid, 256, 0, s>>>(X, x->nz, (const float *)y->copy[CK_F32], y->nz, x->b, x->nb, x->NB, part);
  return cudaGetLastError();
}

}  // namespace

extern "C" spamm_status spamm_tree_distance(spamm_tree X, spamm_tree Y, double *diff_fro, double *ref_fro) {
  if (X && settle(X->ctx) != SPAMM_OK) return SPAMM_ECUDA;
  if (!X || !Y || !diff_fro || !ref_fro) return SPAMM_EINVAL;
  spamm_ctx ctx = X->ctx;
  if (X->n != Y->n || X->b != Y->b) return mfail(ctx, SPAMM_EINVAL, "tree_distance: shapes differ");
  if ((!X->copy[CK_F64] && !X->copy[CK_F32]) || (!Y->copy[CK_F64] && !Y->copy[CK_F32]))
    return mfail(ctx, SPAMM_EINVAL, "tree_distance: a tree keeps no FP64/FP32 tiles");
  const int64_t nl = (int64_t)X->nb * X->nb;
  double *part = nullptr;
  if (cudaMalloc(&part, sizeof(double) * (2 * nl + 2)) != cudaSuccess) return SPAMM_ENOMEM;
  cudaStream_t s = ctx->stream;
  cudaError_t e = X->copy[CK_F64] ? dist_y((const double *)X->copy[CK_F64], X, Y, part, s)
                                  : dist_y((const float *)X->copy[CK_F32], X, Y, part, s);
  if (e == cudaSuccess) {
    k_dist_total<<<1, 32, 0, s>>>(part, nl, part + 2 * nl);
    e = cudaGetLastError();
  }
  ctx->launches += 2;
  double h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, part + 2 * nl, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return SPAMM_ECUDA;
  *diff_fro = h[0];
  *ref_fro = h[1];
  return SPAMM_OK;
}
