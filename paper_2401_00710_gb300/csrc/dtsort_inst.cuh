// One (key, value) instantiation of the persistent kernel and its launchers.
// Included by inst_*.cu with DTS_K, DTS_HV and DTS_NAME defined.
#include "dtsort_launch.h"
#include "dtsort_phases.cuh"

#define DTS_CAT2(a, b) a##b
#define DTS_CAT(a, b) DTS_CAT2(a, b)

namespace dts {

cudaError_t DTS_CAT(shape_, DTS_NAME)(KernelShape *out) {
  using S = Shape<DTS_K, DTS_HV>;
  auto *fn = dtsort_kernel<DTS_K, DTS_HV>;
  const size_t smem = smem_bytes<DTS_K, DTS_HV>();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, smem);
  if (e != cudaSuccess) return e;
  out->fin_cap = S::FIN_CAP;
  out->tile = S::TILE;
  out->blk = S::BLK;
  out->ch = S::CH;
  out->smem = smem;
  out->blocks_per_sm = nb;
  return cudaSuccess;
}

cudaError_t DTS_CAT(launch_, DTS_NAME)(const Params &P, int grid, cudaStream_t s) {
  auto *fn = dtsort_kernel<DTS_K, DTS_HV>;
  const size_t smem = smem_bytes<DTS_K, DTS_HV>();
  Params copy = P;
  void *args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(NT), args, smem, s);
}

#if !DTS_HV
cudaError_t DTS_CAT(launch_sample_, DTS_NAME)(const void *keys, int64_t start, int64_t size,
                                              int hi, uint64_t seed, int64_t m, int64_t L,
                                              uint64_t *heavy, int64_t *nheavy, uint64_t *mx,
                                              cudaStream_t s) {
  auto *fn = sample_debug_kernel<DTS_K>;
  const size_t smem = sizeof(DTS_K) * SMAX + 8 * (NWARP + 1) + 64;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<1, NT, smem, s>>>((const DTS_K *)keys, start, size, hi, seed, m, L, heavy, nheavy, mx);
  return cudaGetLastError();
}
#endif

}  // namespace dts
