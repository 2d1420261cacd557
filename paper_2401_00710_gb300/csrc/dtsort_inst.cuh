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
  // the per-phase kernels too, here and not at launch (launches may be
  // captured into a graph): the combined one with the largest shared memory,
  // each single-phase one with its own, and how many CTAs of it an SM holds
  e = cudaFuncSetAttribute(dtsort_phase_kernel<DTS_K, DTS_HV>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const void *pk[12] = {
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_SEED>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_SETUP>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_SAMPLE>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_HIST>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_MSCAN>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_SCAN>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_SCATTER>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_FINISH>,
      nullptr,  // KP_CLOSE: inside the persistent kernel only
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_MERGE_PREP>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_MERGE>,
      (const void *)dtsort_phase_one<DTS_K, DTS_HV, KP_STATS>};
  for (int ph = 0; ph < 12; ++ph) {
    if (!pk[ph]) {
      out->phase_blocks[ph] = 0;
      continue;
    }
    const size_t sm = phase_smem_bytes<DTS_K, DTS_HV>(ph);
    e = cudaFuncSetAttribute(pk[ph], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pk[ph], phase_threads(ph), sm);
    if (e != cudaSuccess) return e;
    out->phase_blocks[ph] = b < phase_min_blocks(ph) ? b : phase_min_blocks(ph);
  }
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, smem);
  if (e != cudaSuccess) return e;
  out->fin_cap = S::FIN_CAP;
  out->tile = S::TILE;
  out->blk = S::BLK;  // default block (BLK_TILES tiles)
  out->ch = S::CH;
  out->smem = smem;
  out->blocks_per_sm = nb;
  return cudaSuccess;
}

// The first `head` levels as separate phase launches (queued, no host
// synchronisation; each phase checks on the device whether it has work), then
// the persistent kernel for the remaining levels and the merges.  head = 0:
// the persistent kernel alone.
cudaError_t DTS_CAT(launch_, DTS_NAME)(const Params &P, int grid, int head, const KernelShape &ks,
                                       int nsm, cudaStream_t s) {
  const size_t smem = smem_bytes<DTS_K, DTS_HV>();
  cudaError_t e;
  // one kernel per phase (attributes set by shape_), each with its own
  // shared memory and as many CTAs as an SM holds of it
  auto run = [&](int phase, int level, int g0, int prev) {
    const int g = g0 == 1 ? 1 : nsm * (ks.phase_blocks[phase] > 0 ? ks.phase_blocks[phase] : 1);
    const size_t smem = phase_smem_bytes<DTS_K, DTS_HV>(phase);
    switch (phase) {
      case KP_SEED: dtsort_phase_one<DTS_K, DTS_HV, KP_SEED><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_SETUP: dtsort_phase_one<DTS_K, DTS_HV, KP_SETUP><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_SAMPLE: dtsort_phase_one<DTS_K, DTS_HV, KP_SAMPLE><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_HIST: dtsort_phase_one<DTS_K, DTS_HV, KP_HIST><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_MSCAN: dtsort_phase_one<DTS_K, DTS_HV, KP_MSCAN><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_SCAN: dtsort_phase_one<DTS_K, DTS_HV, KP_SCAN><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_SCATTER: dtsort_phase_one<DTS_K, DTS_HV, KP_SCATTER><<<g, SCATTER_NT, smem, s>>>(P, level, prev); break;
      case KP_MERGE_PREP: dtsort_phase_one<DTS_K, DTS_HV, KP_MERGE_PREP><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_MERGE: dtsort_phase_one<DTS_K, DTS_HV, KP_MERGE><<<g, NT, smem, s>>>(P, level, prev); break;
      case KP_STATS: dtsort_phase_one<DTS_K, DTS_HV, KP_STATS><<<g, NT, smem, s>>>(P, level, prev); break;
      default: dtsort_phase_one<DTS_K, DTS_HV, KP_FINISH><<<g, NT, smem, s>>>(P, level, prev); break;
    }
    return cudaGetLastError();
  };
  if (head > 0) {
    if ((e = run(KP_SEED, 0, grid, -1)) != cudaSuccess) return e;
    for (int l = 0; l < head; ++l) {
      if ((e = run(KP_SETUP, l, 1, l == 0 ? PH_SETUP : PH_FINISH)) != cudaSuccess ||
          (e = run(KP_SAMPLE, l, grid, PH_SETUP)) != cudaSuccess ||
          (e = run(KP_HIST, l, grid, PH_SAMPLE)) != cudaSuccess ||
          (e = run(KP_MSCAN, l, grid, PH_HIST)) != cudaSuccess ||
          (e = run(KP_SCAN, l, grid, PH_SCAN)) != cudaSuccess ||
          (e = run(KP_SCATTER, l, grid, PH_SCAN)) != cudaSuccess ||
          (e = run(KP_FINISH, l, grid, PH_SCATTER)) != cudaSuccess)
        return e;
    }
  }
  auto *fn = dtsort_kernel<DTS_K, DTS_HV>;
  Params copy = P;
  int lev0 = head;
  void *args[] = {&copy, &lev0};
  e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(NT), args, smem, s);
  if (e != cudaSuccess || head == 0) return e;
  // the queued levels' dovetail merges, deepest first (each returns at once
  // when its level has no merge zone), then the statistics
  for (int l = head - 1; l >= 0; --l) {
    if ((e = run(KP_MERGE_PREP, l, grid, PH_MERGE)) != cudaSuccess ||
        (e = run(KP_MERGE, l, grid, PH_MERGE)) != cudaSuccess)
      return e;
  }
  return run(KP_STATS, 0, 1, PH_MERGE);
}

// One launch per phase; the host reads the control block between levels.
// ctl_host: pinned host memory for sizeof(Ctl).
cudaError_t DTS_CAT(launch_split_, DTS_NAME)(const Params &P, int grid, cudaStream_t s,
                                             void *ctl_host, int *launches) {
  auto *fn = dtsort_phase_kernel<DTS_K, DTS_HV>;
  const size_t smem = smem_bytes<DTS_K, DTS_HV>();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  Ctl *h = (Ctl *)ctl_host;
  *launches = 0;
  auto run = [&](int phase, int level, int g) {
    fn<<<g, NT, smem, s>>>(P, phase, level, 0, -1);
    ++*launches;
    return cudaGetLastError();
  };
  auto fetch = [&]() {
    cudaError_t e2 = cudaMemcpyAsync(h, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (e2 != cudaSuccess) return e2;
    return cudaStreamSynchronize(s);
  };
  if ((e = run(KP_SEED, 0, grid)) != cudaSuccess) return e;
  int level = 0;
  for (; level < MAXLEV; ++level) {
    if ((e = fetch()) != cudaSuccess) return e;
    const long long nseg = h->nseg[level & 1];
    if ((level > 0 && nseg == 0) || h->error) break;
    if ((e = run(KP_SETUP, level, 1)) != cudaSuccess) return e;
    if ((e = fetch()) != cudaSuccess) return e;
    if (h->error) break;
    if (nseg > 0) {
      const int ph[] = {KP_SAMPLE, KP_HIST, KP_MSCAN, KP_SCAN, KP_SCATTER};
      for (int k = 0; k < 5; ++k) {
        if ((e = run(ph[k], level, grid)) != cudaSuccess) return e;
        if (ph[k] == KP_MSCAN) {
          if ((e = fetch()) != cudaSuccess) return e;
          if (h->error) break;
        }
      }
      if (h->error) break;
    }
    if ((e = run(KP_FINISH, level, grid)) != cudaSuccess) return e;
  }
  if ((e = run(KP_CLOSE, level, 1)) != cudaSuccess) return e;
  if ((e = fetch()) != cudaSuccess) return e;
  for (int l = level - 1; l >= 0 && !h->error; --l) {
    if (h->lvl_zone[l + 1] == h->lvl_zone[l]) continue;
    if ((e = run(KP_MERGE_PREP, l, grid)) != cudaSuccess) return e;
    if ((e = run(KP_MERGE, l, grid)) != cudaSuccess) return e;
  }
  return run(KP_STATS, 0, 1);
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
