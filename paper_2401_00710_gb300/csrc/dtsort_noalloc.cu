// dtsort_u32_kv_noalloc: the 32-bit key/value sort for callers that cannot
// allocate device memory and cannot hand over a workspace either -- for
// example plugin or callback code that receives a stream from a host
// framework owning all device memory, or real-time pipelines that forbid
// allocations after start-up.
//
// Everything the sort needs beyond the caller's keys and values (the second
// copy of keys and values, the per-level tables, the control block) lives in
// one file-scope static __device__ array of NOALLOC_SCRATCH_BYTES, which every
// GPU that loads this library holds until the process exits.  In host code the
// array's name is only a host-side stand-in, so its device address is looked
// up once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernel.  All calls share the array: the control block is
// cleared at the start of every call, and calls that overlap on the GPU (two
// streams, or two devices' work racing on one device) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/dtsort.h"
#include "dtsort_phases.cuh"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)12 << 20;  // 12 MiB
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

using Sh = dts::Shape<uint32_t, true>;

struct NoallocDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
  int grid = 0;
};

NoallocDevice g_devices[kMaxDevices];
std::mutex g_mutex;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Offsets inside the scratch array for n records (same tables as the
// workspace of dtsort_u32_kv with default options).
struct NoallocLayout {
  size_t tkeys, tvals, ctl, segs0, segs1, info, bcount, bstart, lid, heavy, hashk, hashid,
      cmat, status, tasks, zones, mhk, mhs, mhst, devstatus, stats, total;
  int64_t maxseg, bmax, hmax, zmax, hashmax, cwords, swords, tmax, mhmax, target;
};

NoallocLayout noalloc_layout(int64_t n) {
  NoallocLayout L{};
  const int64_t cap = Sh::FIN_CAP;
  L.target = std::max<int64_t>(16, cap * 85 / 100);  // bucket size the levels aim at
  const int64_t nt = n / L.target + 1;
  L.maxseg = n / (cap + 1) + 2;
  // per subproblem 2^gamma < 8 * size / target: buckets <= 1.5 * 2^gamma + 1,
  // heavy keys <= 2^(gamma-1), light-table entries 2^gamma + 1
  L.bmax = 12 * nt + L.maxseg + 1024;
  L.hmax = 4 * nt + L.maxseg + 1024;
  L.zmax = 8 * nt + 2 * L.maxseg + 1024;
  L.hashmax = 16 * nt + 2 * L.maxseg + 1024;  // 2^(gamma+1) slots per subproblem
  L.cwords = (int64_t)dts::NB_HW * (n / Sh::BLK + 1) + L.bmax;
  L.swords = (int64_t)dts::NB_HW * (n / ((int64_t)Sh::BLK * Sh::CH) + 1) + L.bmax;
  L.tmax = 2 * L.bmax + 2 * (n / dts::COPY_CHUNK + 1) + 1 + 4096;
  L.mhmax = 4 * L.hmax + 4096;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t r = off;
    off = up256(off + bytes);
    return r;
  };
  L.tkeys = take((size_t)n * 4);
  L.tvals = take((size_t)n * 4);
  L.ctl = take(sizeof(dts::Ctl));
  L.segs0 = take(sizeof(dts::Seg) * (size_t)L.maxseg);
  L.segs1 = take(sizeof(dts::Seg) * (size_t)L.maxseg);
  L.info = take(sizeof(dts::SegInfo) * (size_t)L.maxseg);
  L.bcount = take(8 * (size_t)L.bmax);
  L.bstart = take(8 * (size_t)L.bmax);
  L.lid = take(4 * (size_t)L.zmax);
  L.heavy = take(4 * (size_t)L.hmax);
  L.hashk = take(4 * (size_t)L.hashmax);
  L.hashid = take(2 * (size_t)L.hashmax);
  L.cmat = take(4 * (size_t)L.cwords);
  L.status = take(8 * (size_t)L.swords);
  L.tasks = take(sizeof(dts::Task) * (size_t)L.tmax);
  L.zones = take(sizeof(dts::MZone) * (size_t)L.mhmax);
  L.mhk = take(4 * (size_t)L.mhmax);
  L.mhs = take(8 * (size_t)L.mhmax);
  L.mhst = take(8 * (size_t)L.mhmax);
  L.devstatus = take(sizeof(int));
  L.stats = take(sizeof(dts::DevStats));
  L.total = off;
  return L;
}

// Once per device, with that device current: the scratch array's device
// address, the kernel's shared-memory limit and its resident grid.
dtsort_status noalloc_setup(int dev, NoallocDevice **out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  NoallocDevice &D = g_devices[dev];
  if (!D.ready) {
    int major = 0, minor = 0, nsm = 0, coop = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
      return DTSORT_ERR_CUDA;
    if (major != 10 || minor != 3 || !coop) return DTSORT_ERR_UNSUPPORTED;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return DTSORT_ERR_CUDA;
    auto *fn = dts::dtsort_kernel<uint32_t, true>;
    const size_t smem = dts::smem_bytes<uint32_t, true>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return DTSORT_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, dts::NT, smem) !=
        cudaSuccess)
      return DTSORT_ERR_CUDA;
    if (per_sm < 1) return DTSORT_ERR_UNSUPPORTED;
    D.scratch = (unsigned char *)p;
    D.grid = nsm * std::min(per_sm, 2);
    D.ready = true;
  }
  *out = &D;
  return DTSORT_OK;
}

}  // namespace

extern "C" dtsort_status dtsort_u32_kv_noalloc(uint32_t *keys, uint32_t *values, int64_t n,
                                               int32_t *device_status, dtsort_stream stream) {
  if (n < 0 || n > DTSORT_NOALLOC_MAX_N) return DTSORT_ERR_INVALID_ARG;
  if (n == 0) return DTSORT_OK;
  if (!keys || !values || ((uintptr_t)keys % 4) || ((uintptr_t)values % 4))
    return DTSORT_ERR_INVALID_ARG;
  const NoallocLayout L = noalloc_layout(n);
  if (L.total > NOALLOC_SCRATCH_BYTES) return DTSORT_ERR_INTERNAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DTSORT_ERR_UNSUPPORTED;
  NoallocDevice *D = nullptr;
  const dtsort_status st = noalloc_setup(dev, &D);
  if (st != DTSORT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *w = D->scratch;
  int *status_word = device_status ? (int *)device_status : (int *)(w + L.devstatus);
  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(w + L.ctl, 0, sizeof(dts::Ctl), s) != cudaSuccess ||
      cudaMemsetAsync(status_word, 0, sizeof(int), s) != cudaSuccess)
    return DTSORT_ERR_CUDA;
  dts::Params P{};
  P.keys[0] = keys;
  P.keys[1] = w + L.tkeys;
  P.vals[0] = values;
  P.vals[1] = w + L.tvals;
  P.n = n;
  P.offsets = nullptr;
  P.nsegs_in = 1;
  P.key_bits = 32;
  P.gamma_max = dts::GAMMA_HW;
  P.cap = Sh::FIN_CAP;
  P.heavy_on = 1;
  P.heavy_min_share = dts::HEAVY_MIN_SHARE;
  P.target = L.target;
  P.seed = 1;
  P.sample_factor = 1;
  P.debug_fault = 0;
  P.blk_tiles = Sh::BLK_TILES;
  P.wait_ns = 2000ull * 1000000ull;
  P.ctl = (dts::Ctl *)(w + L.ctl);
  P.segs[0] = (dts::Seg *)(w + L.segs0);
  P.segs[1] = (dts::Seg *)(w + L.segs1);
  P.info = (dts::SegInfo *)(w + L.info);
  P.bcount = (int64_t *)(w + L.bcount);
  P.bstart = (int64_t *)(w + L.bstart);
  P.lid = (int32_t *)(w + L.lid);
  P.heavy = w + L.heavy;
  P.hash_keys = w + L.hashk;
  P.hash_ids = (uint16_t *)(w + L.hashid);
  P.cmat = (unsigned *)(w + L.cmat);
  P.status = (unsigned long long *)(w + L.status);
  P.tasks = (dts::Task *)(w + L.tasks);
  P.zones = (dts::MZone *)(w + L.zones);
  P.mh_keys = w + L.mhk;
  P.mh_sizes = (int64_t *)(w + L.mhs);
  P.mh_start = (int64_t *)(w + L.mhst);
  P.maxseg = L.maxseg;
  P.bmax = L.bmax;
  P.hmax = L.hmax;
  P.zmax = L.zmax;
  P.hashmax = L.hashmax;
  P.cwords = L.cwords;
  P.swords = L.swords;
  P.tmax = L.tmax;
  P.mhmax = L.mhmax;
  P.dev_status = status_word;
  P.stats = (dts::DevStats *)(w + L.stats);
  int lev0 = 0;  // the persistent kernel alone
  void *args[] = {&P, &lev0};
  const cudaError_t e = cudaLaunchCooperativeKernel(
      (const void *)dts::dtsort_kernel<uint32_t, true>, dim3(D->grid), dim3(dts::NT), args,
      dts::smem_bytes<uint32_t, true>(), s);
  return e == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}
