// The rank-local steps of the one-exchange multi-GPU sort (include/dtsort.h,
// "sorting an array sharded over several GPUs").
//
// P ranks hold contiguous, index-ordered shards of one array.  The stable
// order of the whole array is the order of the pairs (key, global index)
// (Sec. 2.3's problem statement), so P-1 splitters drawn from a global sample
// of such pairs cut it into P consecutive ranges, and a record belongs to
// range #{splitters <= (key, global index)}.  The splitting is a stable
// distribution by range number -- the counting sort of the paper's
// preliminaries, with P buckets: per-block counts, a column scan, and a
// scatter that keeps index order within each range.  A heavily duplicated
// key that straddles a splitter is split by global index, which keeps the
// ranges balanced.  After one all-to-all (the caller's collective), rank p
// holds range p's runs in source-rank order, i.e. in global index order, and
// one stable sort of them gives the p-th part of the sorted array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/dtsort.h"
#include "dtsort_device.cuh"

namespace {

constexpr int SNT = 256;                 // threads per CTA of these kernels
constexpr int SNW = SNT / 32;
constexpr int SMAXP = DTSORT_SHARD_MAX_PARTS;
constexpr int64_t SMIN_BLK = 4096;       // records per count-matrix row, at least
constexpr int64_t SMAX_ROWS = 4096;      // rows of the count matrix, at most

// Records per row of the count matrix for a shard of n records: at most
// SMAX_ROWS rows, a multiple of SNT records each.
int64_t shard_blk(int64_t n) {
  int64_t b = std::max<int64_t>(SMIN_BLK, (n + SMAX_ROWS - 1) / SMAX_ROWS);
  return (b + SNT - 1) / SNT * SNT;
}

// Range of a record: the number of splitters (sk[j], sg[j]) <= (key, g);
// the splitters increase.
__device__ __forceinline__ int range_of(uint64_t key, int64_t g, const uint64_t *sk,
                                        const int64_t *sg, int ns) {
  int lo = 0, hi = ns;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const uint64_t k2 = sk[mid];
    if (k2 < key || (k2 == key && sg[mid] <= g)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <typename K>
__device__ __forceinline__ uint64_t key_u64(const K *p, int64_t i) {
  return (uint64_t)dts::ld_key<K>(p + i);
}

// Sample i of a shard: the record at position x_i mod n, x_i the i-th output
// of the SplitMix64 sequence started from seed ^ fmix(gidx0 + golden gamma).
template <typename K>
__global__ void __launch_bounds__(SNT) shard_sample_kernel(const K *keys, int64_t n,
                                                           int64_t gidx0, uint64_t seed,
                                                           int64_t count, uint64_t *sk,
                                                           int64_t *sg) {
  const uint64_t s = seed ^ dts::sm64_fmix((uint64_t)gidx0 + 0x9E3779B97F4A7C15ull);
  for (int64_t i = blockIdx.x * (int64_t)SNT + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * SNT) {
    const int64_t pos = (int64_t)(dts::sm64_at(s, (uint64_t)i) % (uint64_t)n);
    sk[i] = key_u64<K>(keys, pos);
    sg[i] = gidx0 + pos;
  }
}

// Loads the splitters into shared memory (all threads call).
__device__ __forceinline__ void load_splitters(const uint64_t *split_k, const int64_t *split_g,
                                               int ns, uint64_t *sk, int64_t *sg) {
  for (int j = threadIdx.x; j < ns; j += SNT) {
    sk[j] = __ldcg((const unsigned long long *)split_k + j);
    sg[j] = (int64_t)__ldcg((const unsigned long long *)split_g + j);
  }
  __syncthreads();
}

// Row b of the count matrix: how many records of block b (records
// [b blk, (b+1) blk)) fall into each range.  cmat: nblk x P.
template <typename K>
__global__ void __launch_bounds__(SNT) shard_count_kernel(const K *keys, int64_t n,
                                                          int64_t gidx0, const uint64_t *split_k,
                                                          const int64_t *split_g, int parts,
                                                          int64_t blk, int64_t *cmat) {
  __shared__ uint64_t sk[SMAXP];
  __shared__ int64_t sg[SMAXP];
  __shared__ unsigned cnt[SMAXP];
  const int ns = parts - 1;
  for (int p = threadIdx.x; p < parts; p += SNT) cnt[p] = 0u;
  load_splitters(split_k, split_g, ns, sk, sg);
  const int64_t s = blockIdx.x * blk;
  const int64_t e = s + blk < n ? s + blk : n;
  const unsigned lane = threadIdx.x & 31;
  // every lane takes the same number of rounds; lanes past the end carry the
  // dummy range `parts` so that the warp-wide match stays complete
  for (int64_t base = s; base < e; base += SNT) {
    const int64_t i = base + threadIdx.x;
    const int d = i < e ? range_of(key_u64<K>(keys, i), gidx0 + i, sk, sg, ns) : parts;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < parts && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&cnt[d], __popc(peers));
  }
  __syncthreads();
  for (int p = threadIdx.x; p < parts; p += SNT)
    cmat[blockIdx.x * (int64_t)parts + p] = (int64_t)cnt[p];
}

// Turns the count matrix into offsets in the partitioned output: entry
// (b, p) becomes the first output slot of block b's records of range p, i.e.
// the start of range p (the records of all lower ranges) plus block b's
// predecessors' records of range p.  counts[p] = records of range p.  One
// CTA of 1024 threads: the columns are split into groups of rows.
__global__ void __launch_bounds__(1024) shard_scan_kernel(int64_t *cmat, int64_t nblk,
                                                          int parts, int64_t *counts) {
  __shared__ int64_t part[1024];
  __shared__ int64_t start[SMAXP + 1];
  const int G = 1024 / parts;  // row groups per column
  const int t = threadIdx.x;
  const int p = t % parts, g = t / parts;
  const bool on = g < G;
  const int64_t R = (nblk + G - 1) / G;
  const int64_t r0 = on ? g * R : 0;
  const int64_t r1 = on ? (r0 + R < nblk ? r0 + R : nblk) : 0;
  int64_t sum = 0;
  for (int64_t r = r0; r < r1; ++r) sum += cmat[r * parts + p];
  if (on) part[g * parts + p] = sum;
  __syncthreads();
  if (t < parts) {  // exclusive scan of column t over its row groups
    int64_t run = 0;
    for (int q = 0; q < G; ++q) {
      const int64_t v = part[q * parts + t];
      part[q * parts + t] = run;
      run += v;
    }
    counts[t] = run;
    start[t] = run;
  }
  __syncthreads();
  if (t == 0) {  // range starts: exclusive scan over the ranges
    int64_t run = 0;
    for (int q = 0; q < parts; ++q) {
      const int64_t v = start[q];
      start[q] = run;
      run += v;
    }
    start[parts] = run;
  }
  __syncthreads();
  if (on) {
    int64_t run = start[p] + part[g * parts + p];
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t v = cmat[r * parts + p];
      cmat[r * parts + p] = run;
      run += v;
    }
  }
}

// Stable scatter of block b into the ranges: each warp takes a contiguous
// chunk of the block (warp order = index order), counts it per range, gets
// its first slot per range from the block's offsets (prefix over the warps),
// then walks the chunk in rounds of 32 records; records of one range in one
// round are ranked by lane (__match_any_sync), so index order is kept.
template <typename K, bool HV>
__global__ void __launch_bounds__(SNT) shard_scatter_kernel(
    const K *keys, const K *vals, int64_t n, int64_t gidx0, const uint64_t *split_k,
    const int64_t *split_g, int parts, int64_t blk, const int64_t *cmat, K *out_k, K *out_v,
    int *bad) {
  __shared__ uint64_t sk[SMAXP];
  __shared__ int64_t sg[SMAXP];
  __shared__ int64_t wbase[SNW][SMAXP];
  __shared__ unsigned wcnt[SNW][SMAXP];
  const int ns = parts - 1;
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int p = threadIdx.x; p < SNW * SMAXP; p += SNT) (&wcnt[0][0])[p] = 0u;
  load_splitters(split_k, split_g, ns, sk, sg);
  const int64_t s = blockIdx.x * blk;
  const int64_t e = s + blk < n ? s + blk : n;
  const int64_t chunk = ((e - s + SNW - 1) / SNW + 31) / 32 * 32;
  const int64_t cs = s + w * chunk < e ? s + w * chunk : e;
  const int64_t ce = cs + chunk < e ? cs + chunk : e;
  for (int64_t base = cs; base < ce; base += 32) {
    const int64_t i = base + lane;
    const int d = i < ce ? range_of(key_u64<K>(keys, i), gidx0 + i, sk, sg, ns) : parts;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < parts && lane == (unsigned)(__ffs(peers) - 1)) wcnt[w][d] += __popc(peers);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < parts; p += SNT) {
    int64_t run = cmat[blockIdx.x * (int64_t)parts + p];
    for (int q = 0; q < SNW; ++q) {
      wbase[q][p] = run;
      run += wcnt[q][p];
    }
  }
  __syncthreads();
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  for (int64_t base = cs; base < ce; base += 32) {
    const int64_t i = base + lane;
    K k = (K)0;
    int d = parts;
    if (i < ce) {
      k = dts::ld_key<K>(keys + i);
      d = range_of((uint64_t)k, gidx0 + i, sk, sg, ns);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < parts) {
      const int64_t pos = wbase[w][d] + __popc(peers & lt);
      if (pos >= 0 && pos < n) {
        out_k[pos] = k;
        if constexpr (HV) out_v[pos] = dts::ld_key<K>(vals + i);
      } else {
        atomicExch(bad, (int)DTSORT_ERR_INTERNAL);
      }
    }
    __syncwarp();
    if (d < parts && lane == (unsigned)(__ffs(peers) - 1)) wbase[w][d] += __popc(peers);
    __syncwarp();
  }
}

bool aligned(const void *p, int bytes) { return ((uintptr_t)p % (uintptr_t)bytes) == 0; }

}  // namespace

extern "C" dtsort_status dtsort_shard_sample(const void *keys, int key_bytes, int64_t n_local,
                                             int64_t gidx0, uint64_t seed, int64_t count,
                                             uint64_t *sample_keys, int64_t *sample_gidx,
                                             dtsort_stream stream) {
  if ((key_bytes != 4 && key_bytes != 8) || n_local < 0 || gidx0 < 0 || count < 0)
    return DTSORT_ERR_INVALID_ARG;
  if (count == 0) return DTSORT_OK;
  if (n_local == 0 || !keys || !sample_keys || !sample_gidx || !aligned(keys, key_bytes) ||
      !aligned(sample_keys, 8) || !aligned(sample_gidx, 8))
    return DTSORT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t g = std::min<int64_t>((count + SNT - 1) / SNT, 4096);
  if (key_bytes == 4)
    shard_sample_kernel<uint32_t><<<(unsigned)g, SNT, 0, s>>>(
        (const uint32_t *)keys, n_local, gidx0, seed, count, sample_keys, sample_gidx);
  else
    shard_sample_kernel<uint64_t><<<(unsigned)g, SNT, 0, s>>>(
        (const uint64_t *)keys, n_local, gidx0, seed, count, sample_keys, sample_gidx);
  return cudaGetLastError() == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}

extern "C" dtsort_status dtsort_shard_splitters(const uint64_t *sample_keys,
                                                const int64_t *sample_gidx, int64_t m, int parts,
                                                uint64_t *split_keys, int64_t *split_gidx) {
  if (parts < 1 || parts > DTSORT_SHARD_MAX_PARTS || m < 0) return DTSORT_ERR_INVALID_ARG;
  if (parts == 1) return DTSORT_OK;
  if (!split_keys || !split_gidx || (m > 0 && (!sample_keys || !sample_gidx)))
    return DTSORT_ERR_INVALID_ARG;
  std::vector<std::pair<uint64_t, int64_t>> v((size_t)m);
  for (int64_t i = 0; i < m; ++i) v[(size_t)i] = {sample_keys[i], sample_gidx[i]};
  std::sort(v.begin(), v.end());
  for (int j = 1; j < parts; ++j) {
    if (m == 0) {  // no sample: everything goes to range 0
      split_keys[j - 1] = ~0ull;
      split_gidx[j - 1] = INT64_MAX;
    } else {
      const auto &x = v[(size_t)(j * m / parts)];
      split_keys[j - 1] = x.first;
      split_gidx[j - 1] = x.second;
    }
  }
  return DTSORT_OK;
}

extern "C" dtsort_status dtsort_shard_partition_workspace_bytes(int64_t n_local, int parts,
                                                                size_t *bytes) {
  if (!bytes || n_local < 0 || parts < 1 || parts > DTSORT_SHARD_MAX_PARTS)
    return DTSORT_ERR_INVALID_ARG;
  const int64_t nblk = n_local == 0 ? 0 : (n_local + shard_blk(n_local) - 1) / shard_blk(n_local);
  *bytes = 256 + (size_t)nblk * (size_t)parts * sizeof(int64_t);
  return DTSORT_OK;
}

extern "C" dtsort_status dtsort_shard_partition(const void *keys, const void *values,
                                                int key_bytes, int64_t n_local, int64_t gidx0,
                                                const uint64_t *split_keys,
                                                const int64_t *split_gidx, int parts,
                                                void *out_keys, void *out_values,
                                                int64_t *counts, void *ws, size_t ws_bytes,
                                                int32_t *device_status, dtsort_stream stream) {
  if ((key_bytes != 4 && key_bytes != 8) || n_local < 0 || gidx0 < 0 || parts < 1 ||
      parts > DTSORT_SHARD_MAX_PARTS || !counts || !aligned(counts, 8))
    return DTSORT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_local == 0)
    return cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)parts, s) == cudaSuccess
               ? DTSORT_OK : DTSORT_ERR_CUDA;
  if (!keys || !out_keys || !ws || (values != nullptr) != (out_values != nullptr) ||
      (parts > 1 && (!split_keys || !split_gidx)) || !aligned(keys, key_bytes) ||
      !aligned(out_keys, key_bytes) || (values && (!aligned(values, key_bytes) ||
                                                   !aligned(out_values, key_bytes))) ||
      !aligned(ws, 256) || (split_keys && !aligned(split_keys, 8)) ||
      (split_gidx && !aligned(split_gidx, 8)) || (device_status && !aligned(device_status, 4)))
    return DTSORT_ERR_INVALID_ARG;
  size_t need = 0;
  dtsort_shard_partition_workspace_bytes(n_local, parts, &need);
  if (ws_bytes < need) return DTSORT_ERR_WORKSPACE_TOO_SMALL;
  const int64_t blk = shard_blk(n_local);
  const int64_t nblk = (n_local + blk - 1) / blk;
  int *status = device_status ? (int *)device_status : (int *)ws;
  int64_t *cmat = (int64_t *)((char *)ws + 256);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (key_bytes == 4) {
    using K = uint32_t;
    shard_count_kernel<K><<<(unsigned)nblk, SNT, 0, s>>>((const K *)keys, n_local, gidx0,
                                                         split_keys, split_gidx, parts, blk,
                                                         cmat);
    shard_scan_kernel<<<1, 1024, 0, s>>>(cmat, nblk, parts, counts);
    if (values)
      shard_scatter_kernel<K, true><<<(unsigned)nblk, SNT, 0, s>>>(
          (const K *)keys, (const K *)values, n_local, gidx0, split_keys, split_gidx, parts, blk,
          cmat, (K *)out_keys, (K *)out_values, status);
    else
      shard_scatter_kernel<K, false><<<(unsigned)nblk, SNT, 0, s>>>(
          (const K *)keys, nullptr, n_local, gidx0, split_keys, split_gidx, parts, blk, cmat,
          (K *)out_keys, nullptr, status);
  } else {
    using K = uint64_t;
    shard_count_kernel<K><<<(unsigned)nblk, SNT, 0, s>>>((const K *)keys, n_local, gidx0,
                                                         split_keys, split_gidx, parts, blk,
                                                         cmat);
    shard_scan_kernel<<<1, 1024, 0, s>>>(cmat, nblk, parts, counts);
    if (values)
      shard_scatter_kernel<K, true><<<(unsigned)nblk, SNT, 0, s>>>(
          (const K *)keys, (const K *)values, n_local, gidx0, split_keys, split_gidx, parts, blk,
          cmat, (K *)out_keys, (K *)out_values, status);
    else
      shard_scatter_kernel<K, false><<<(unsigned)nblk, SNT, 0, s>>>(
          (const K *)keys, nullptr, n_local, gidx0, split_keys, split_gidx, parts, blk, cmat,
          (K *)out_keys, nullptr, status);
  }
  return cudaGetLastError() == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}
