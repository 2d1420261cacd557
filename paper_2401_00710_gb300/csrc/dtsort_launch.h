// Host-side launch entry points of the four (key, value) instantiations.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "dtsort_device.cuh"

namespace dts {

// Kernel shape of one instantiation: finisher capacity, scatter tile, shared
// memory, resident CTAs per SM for the cooperative launch.
struct KernelShape {
  int fin_cap;
  int tile;
  int blk;   // records per count-matrix row
  int ch;    // rows per look-back chunk
  size_t smem;
  int blocks_per_sm;
  int phase_blocks[12];  // CTAs per SM of each single-phase kernel (by phase id)
};

#define DTS_DECLARE(NAME)                                                      \
  cudaError_t launch_##NAME(const Params &P, int grid, int head, const KernelShape &ks, \
                            int nsm, cudaStream_t s);                          \
  cudaError_t launch_split_##NAME(const Params &P, int grid, cudaStream_t s,   \
                                  void *ctl_host, int *launches);              \
  cudaError_t shape_##NAME(KernelShape *out);
#define DTS_DECLARE_SAMPLE(NAME)                                               \
  cudaError_t launch_sample_##NAME(const void *keys, int64_t start,            \
                                   int64_t size, int hi, uint64_t seed,        \
                                   int64_t m, int64_t L, uint64_t *heavy,      \
                                   int64_t *nheavy, uint64_t *mx,              \
                                   cudaStream_t s);

DTS_DECLARE(u32)
DTS_DECLARE(u32kv)
DTS_DECLARE(u64)
DTS_DECLARE(u64kv)
DTS_DECLARE_SAMPLE(u32)
DTS_DECLARE_SAMPLE(u64)

#undef DTS_DECLARE
#undef DTS_DECLARE_SAMPLE

// learned bucketing (dtsort_learned.cu)
cudaError_t lrn_gather(const void *keys, int kb, int64_t n, uint64_t seed, uint64_t *out,
                       int64_t m, cudaStream_t s);
// en: NULL, or a device flag (0: the model is not wanted; the kernels return)
cudaError_t lrn_features(const uint64_t *sorted, int64_t m, int w, float *x, float *t,
                         const int *en, cudaStream_t s);
cudaError_t lrn_init(float *params, float *mom, float *vel, uint64_t seed, const int *en,
                     cudaStream_t s);
cudaError_t lrn_train(float *params, float *mom, float *vel, const float *x, const float *t,
                      int64_t m, int steps, int batch, float lr, float *part, const int *en,
                      cudaStream_t s);
cudaError_t lrn_splitters(const float *params, int B, int kb, void *spl, float *tab,
                          const int *en, cudaStream_t s);
// the device's decision whether learned zones pay (see lrn_decide_kernel);
// en: NULL, or an earlier decision that, when 0, stands
cudaError_t lrn_decide(const uint64_t *sorted, int64_t m, int64_t n, int kb, int B,
                       const void *spl, int cap, int64_t target, int gmax, double penalty,
                       int *on, double *est, const int *en, cudaStream_t s);
// zone lower bounds at the sorted sample's quantiles (lrn_quantile_kernel)
cudaError_t lrn_quantiles(const uint64_t *sorted, int64_t m, int kb, int B, void *spl,
                          cudaStream_t s);

}  // namespace dts
