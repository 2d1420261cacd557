// Learned CDF bucketing: model sample, training loop, zone boundaries, and
// the C-ABI entry points of the model's kernels (for testing).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/dtsort.h"
#include "dtsort_launch.h"
#include "dtsort_learned.cuh"

namespace dts {

namespace {

__device__ __forceinline__ uint64_t lrn_sm64(uint64_t s, uint64_t i) {
  uint64_t z = s + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// out[i] = key at position (SplitMix64 output i of the stream `s`) mod n
template <typename K>
__global__ void lrn_gather_kernel(const K *__restrict__ keys, int64_t n, uint64_t s,
                                  uint64_t *__restrict__ out, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint64_t)keys[lrn_sm64(s, (uint64_t)i) % (uint64_t)n];
}

// features of the sorted sample and their empirical CDF targets
__global__ void lrn_features_kernel(const uint64_t *__restrict__ sorted, int64_t m, int w,
                                    float *__restrict__ x, float *__restrict__ t,
                                    const int *en) {
  if (en && !*en) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = mlp_feature(sorted[i], w);
    t[i] = (float)(((double)i + 0.5) / (double)m);
  }
}

int grid_for(int64_t n, int threads) {
  const int64_t g = (n + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 4096);
}

}  // namespace

cudaError_t lrn_gather(const void *keys, int kb, int64_t n, uint64_t seed, uint64_t *out,
                       int64_t m, cudaStream_t s) {
  if (kb == 4)
    lrn_gather_kernel<uint32_t><<<grid_for(m, 256), 256, 0, s>>>((const uint32_t *)keys, n,
                                                                 seed, out, m);
  else
    lrn_gather_kernel<uint64_t><<<grid_for(m, 256), 256, 0, s>>>((const uint64_t *)keys, n,
                                                                 seed, out, m);
  return cudaGetLastError();
}

cudaError_t lrn_features(const uint64_t *sorted, int64_t m, int w, float *x, float *t,
                         const int *en, cudaStream_t s) {
  lrn_features_kernel<<<grid_for(m, 256), 256, 0, s>>>(sorted, m, w, x, t, en);
  return cudaGetLastError();
}

cudaError_t lrn_init(float *params, float *mom, float *vel, uint64_t seed, const int *en,
                     cudaStream_t s) {
  mlp_init_kernel<<<1, 352, 0, s>>>(params, mom, vel, seed, en);
  return cudaGetLastError();
}

// `steps` Adam steps on batches of `batch` points strided over the m points
// (batch s uses points (s mod stride) + i * stride, stride = m / batch).
cudaError_t lrn_train(float *params, float *mom, float *vel, const float *x, const float *t,
                      int64_t m, int steps, int batch, float lr, float *part, const int *en,
                      cudaStream_t s) {
  const int64_t stride = std::max<int64_t>(1, m / batch);
  const int nb = (batch + MLP_BLK - 1) / MLP_BLK;
  for (int k = 1; k <= steps; ++k) {
    mlp_grad_kernel<<<nb, MLP_BLK, 0, s>>>(params, x, t, m, (k - 1) % stride, stride, batch,
                                           part, en);
    mlp_adam_kernel<<<1, 352, 0, s>>>(params, mom, vel, part, nb, batch, nullptr, k, lr, en);
  }
  return cudaGetLastError();
}

cudaError_t lrn_splitters(const float *params, int B, int kb, void *spl, float *tab,
                          const int *en, cudaStream_t s) {
  if (kb == 4)
    lrn_splitters_kernel<uint32_t><<<1, 512, 0, s>>>(params, B, 32, (uint32_t *)spl, tab, en);
  else
    lrn_splitters_kernel<uint64_t><<<1, 512, 0, s>>>(params, B, 64, (uint64_t *)spl, tab, en);
  return cudaGetLastError();
}

cudaError_t lrn_decide(const uint64_t *sorted, int64_t m, int64_t n, int kb, int B,
                       const void *spl, int cap, int64_t target, int gmax, double penalty,
                       int *on, double *est, const int *en, cudaStream_t s) {
  if (kb == 4)
    lrn_decide_kernel<uint32_t><<<1, 512, 0, s>>>(sorted, m, n, 32, B, (const uint32_t *)spl,
                                                  cap, target, gmax, penalty, on, est, en);
  else
    lrn_decide_kernel<uint64_t><<<1, 512, 0, s>>>(sorted, m, n, 64, B, (const uint64_t *)spl,
                                                  cap, target, gmax, penalty, on, est, en);
  return cudaGetLastError();
}

cudaError_t lrn_quantiles(const uint64_t *sorted, int64_t m, int kb, int B, void *spl,
                          cudaStream_t s) {
  if (kb == 4)
    lrn_quantile_kernel<uint32_t><<<grid_for(B, 256), 256, 0, s>>>(sorted, m, B, (uint32_t *)spl);
  else
    lrn_quantile_kernel<uint64_t><<<grid_for(B, 256), 256, 0, s>>>(sorted, m, B, (uint64_t *)spl);
  return cudaGetLastError();
}

}  // namespace dts

// ---- C-ABI: the model's kernels on given data ------------------------------
extern "C" {

dtsort_status dtsort_mlp_forward(const float *params, const float *x, int64_t n, float *y,
                                 dtsort_stream stream) {
  if (!params || n < 0 || (n > 0 && (!x || !y))) return DTSORT_ERR_INVALID_ARG;
  if (n == 0) return DTSORT_OK;
  dts::mlp_forward_kernel<<<dts::grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(params, x,
                                                                                  n, y);
  return cudaGetLastError() == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}

dtsort_status dtsort_mlp_grad(const float *params, const float *x, const float *t, int64_t n,
                              float *partial, float *grad_out, dtsort_stream stream) {
  if (!params || !x || !t || !partial || !grad_out || n <= 0 || n > ((int64_t)1 << 30))
    return DTSORT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)((n + dts::MLP_BLK - 1) / dts::MLP_BLK);
  dts::mlp_grad_kernel<<<nb, dts::MLP_BLK, 0, s>>>(params, x, t, n, 0, 1, n, partial, nullptr);
  dts::mlp_adam_kernel<<<1, 352, 0, s>>>(nullptr, nullptr, nullptr, partial, nb, n, grad_out,
                                         0, 0.f, nullptr);
  return cudaGetLastError() == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}

dtsort_status dtsort_mlp_adam(float *params, float *m, float *v, const float *grad, int step,
                              float lr, dtsort_stream stream) {
  if (!params || !m || !v || !grad || step < 1) return DTSORT_ERR_INVALID_ARG;
  // a single "partial" equal to the gradient, one block
  dts::mlp_adam_kernel<<<1, 352, 0, (cudaStream_t)stream>>>(params, m, v, grad, 1, 1, nullptr,
                                                            step, lr, nullptr);
  return cudaGetLastError() == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}

dtsort_status dtsort_mlp_train(float *params, float *m, float *v, const float *x, const float *t,
                               int64_t n, int steps, int batch, float lr, float *partial,
                               dtsort_stream stream) {
  if (!params || !m || !v || !x || !t || !partial || n <= 0 || steps < 0 || batch <= 0 ||
      batch > n)
    return DTSORT_ERR_INVALID_ARG;
  return dts::lrn_train(params, m, v, x, t, n, steps, batch, lr, partial, nullptr,
                        (cudaStream_t)stream) == cudaSuccess
             ? DTSORT_OK
             : DTSORT_ERR_CUDA;
}

}  // extern "C"
