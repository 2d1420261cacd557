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
};

#define DTS_DECLARE(NAME)                                                      \
  cudaError_t launch_##NAME(const Params &P, int grid, cudaStream_t s);        \
  cudaError_t launch_split_##NAME(const Params &P, int grid, cudaStream_t s,   \
                                  void *ctl_host);                             \
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

}  // namespace dts
