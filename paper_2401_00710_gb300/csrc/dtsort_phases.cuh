// Phases of the persistent dtsort kernel (see dtsort_device.cuh).
#pragma once

#include "dtsort_device.cuh"

namespace dts {

// Compile-time shape of one (key, value) instantiation.
template <typename K, bool HV>
struct Shape {
  static constexpr int KB = sizeof(K);
  static constexpr int VB = HV ? (int)sizeof(K) : 0;
  static constexpr int ITEMS = KB == 4 ? 16 : 8;        // scatter items / thread
  static constexpr int TILE = NT * ITEMS;
  // 9 items per thread with values or 32-bit keys (a uniform 10^9-record
  // sort's buckets hold about 3,800 records: two levels for 64-bit key/value
  // pairs too, and 8 live rounds of the unrolled loops instead of 8 of 12 for
  // 32-bit keys), 12 for 64-bit keys alone.  The LSD fallback's two key and
  // two 16-bit index buffers must fit the base-case area.
  static constexpr int CAP_MAX = (KB == 4 || HV) ? 9 * NT : 12 * NT;
  static constexpr int FIN_LSD_REC = KB + (HV ? 2 : 0);  // LSD bytes per record
  static constexpr int FIN_CAP = (96 * 1024) / (2 * FIN_LSD_REC) < CAP_MAX
                                      ? (96 * 1024) / (2 * FIN_LSD_REC) : CAP_MAX;
  // base-case area: the two record buffers of the LSD passes, or the one-pass
  // bins, placed composites and values (see fin_core)
  static constexpr int FIN_BYTES = 96 * 1024;
  static constexpr int FIN_IT = FIN_CAP / NT;           // base-case items / thread
  // largest bin sorted in place by its owner thread: without values a big
  // bin is mostly one key (insertion sort is linear on equal keys); with
  // values the composites all differ (10^9 u32 KV measured: 64 is slower)
  static constexpr int FIN_CMAX = HV ? 16 : 64;
  static constexpr int STAGE = TILE * KB;               // scatter staging (keys or values)
  static constexpr int BLK_TILES = 8;                   // tiles per count-matrix row
  static constexpr int BLK = BLK_TILES * TILE;          // records per block
  static constexpr int CH = 32;                         // rows per look-back chunk
};

// One record of the on-chip base case: key, and the value next to it, so that
// a pass moves each record with one shared-memory load and one store.
template <typename K, bool HV>
struct Rec {
  K k;
};
template <>
struct alignas(8) Rec<uint32_t, true> {
  uint32_t k, v;
};
template <>
struct alignas(16) Rec<uint64_t, true> {
  uint64_t k, v;
};

// Hands out 16-byte aligned arrays of the kernel's dynamic shared memory, by
// pointer arithmetic on dts_smem (the shared address space stays visible).
struct Carve {
  size_t off = 0;
  __device__ __forceinline__ Carve() {}
  template <typename T>
  __device__ __forceinline__ T *take(size_t n) {
    off = (off + 15) & ~(size_t)15;
    T *r = reinterpret_cast<T *>(dts_smem + off);
    off += n * sizeof(T);
    return r;
  }
};

// Copy runs whose task descriptors the whole CTA writes later (a heavy run
// can be 10^8 records: thousands of tasks for the one thread that finds it).
struct CopyReq {
  int64_t start, size, i0, k;
  int32_t src, dst;
};
constexpr int COPY_REQS = 128;
struct CopyList {
  CopyReq *req;
  int *n;
};

// Threads of the per-phase scatter kernel: one CTA of 1024 per SM, tiles of
// 1024 * ITEMS records.  Twice the records per tile give each bucket run of a
// tile twice the length, so half as many partly written 32-byte sectors per
// byte moved (each costs a DRAM read-modify-write when it leaves L2 before
// the next tile completes it).  The persistent kernel scatters with NT.
constexpr int SCATTER_NT = 1024;

// Bytes of the scatter's staged tile (keys with their destinations, or keys
// with their values) for CTAs of NTS threads.
template <typename K, bool HV, int NTS = NT>
__host__ __device__ constexpr int scatter_area() {
  using S = Shape<K, HV>;
  constexpr int tile = NTS * S::ITEMS;
  constexpr int kd = tile * (int)sizeof(K) + 4 * tile;
  constexpr int kv = HV ? 2 * tile * (int)sizeof(K) : 0;
  return kd > kv ? kd : kv;
}

// Dynamic shared memory of the scatter with CTAs of NTS threads (the arrays
// phase_scatter carves, in its order, each 16-byte aligned).
template <typename K, bool HV, int NTS = NT>
constexpr size_t scatter_smem() {
  constexpr int NWS = NTS / 32;
  size_t sc = 0;
  sc += 64 + sizeof(SegTables<K>);
  sc += 16 + 4 * ((1 << GAMMA_HW) + 1);            // lid
  sc += 16 + sizeof(K) * HASH_HW + 16 + 2 * HASH_HW;  // hash
  sc += 16 + sizeof(K) * HEAVY_HW;                 // heavy keys, sorted
  sc += 16 + 4 * (size_t)NWS * NB_PAIR;            // warp counters
  sc += 3 * (16 + 4 * NB_PAD);                     // tile offsets, bases
  sc += 16 + 4 * (NWS + 1);                        // warp sums
  sc += 16 + sizeof(K) * (1 << GAMMA_HW) + 16 + 4 * (LRN_TAB_N + 1);  // learned tables
  sc += 16 + (size_t)scatter_area<K, HV, NTS>();   // staged tile
  return sc + 256;
}

template <typename K, bool HV>
constexpr size_t smem_bytes() {
  using S = Shape<K, HV>;
  // scatter
  const size_t sc = scatter_smem<K, HV, NT>();
  // base case
  size_t fin = 0;
  fin += 16 + (size_t)S::FIN_BYTES;
  fin += 16 + 2 * (size_t)NWARP * FIN_NB;
  fin += 16 + 4 * FIN_NB * 2;
  fin += 16 + 4 * (NWARP + 1) + 16 + 4 * NWARP + 4 * 16 + 16 + 16 + 2 * sizeof(Task) + 256;
  // sampler
  size_t smp = 16 + sizeof(K) * SMAX + 16 + sizeof(K) * (SMAX / 2 + 8) + 16 + 4 * 1024 +
               16 + sizeof(K) * HASH_HW + 16 + 2 * HASH_HW + 6 * (16 + 4 * HEAVY_HW) + 16 + 512;
  size_t m = sc > fin ? sc : fin;
  return m > smp ? m : smp;
}

// Dynamic shared memory of one phase's own kernel (the queued levels launch
// each phase as its own kernel; the light phases then fit more CTAs per SM).
template <typename K, bool HV>
constexpr size_t phase_smem_bytes(int ph) {
  // histogram: tables + one count row
  const size_t hist = 64 + sizeof(SegTables<K>) + 16 + 4 * ((1 << GAMMA_HW) + 1) + 16 +
                      sizeof(K) * HASH_HW + 16 + 2 * HASH_HW + 16 + sizeof(K) * HEAVY_HW +
                      16 + 4 * NB_PAD + 16 +
                      sizeof(K) * (1 << GAMMA_HW) + 16 + 4 * (LRN_TAB_N + 1) + 256;
  // sample: the on-chip sample and its tables
  const size_t smp = 16 + sizeof(K) * SMAX + 16 + sizeof(K) * (SMAX / 2 + 8) + 16 + 4 * 1024 +
                     16 + sizeof(K) * HASH_HW + 16 + 2 * HASH_HW + 6 * (16 + 4 * HEAVY_HW) +
                     16 + 512;
  // bucket scan: counts, offsets, light table
  const size_t scan = 16 + 8 * NB_PAD + 16 + 8 * (NB_PAD + 1) + 16 + 4 * ((1 << GAMMA_HW) + 1) +
                      16 + 8 * (NWARP + 1) + 16 + sizeof(CopyReq) * COPY_REQS + 16 + 4 + 256;
  switch (ph) {
    case 2: return smp;                        // KP_SAMPLE
    case 3: return hist;                       // KP_HIST
    case 4: return 64 + sizeof(SegInfo) + 256;  // KP_MSCAN
    case 5: return scan;                       // KP_SCAN
    case 0:                                    // KP_SEED
    case 1: return 8 * (NWARP + 1) + 256;      // KP_SETUP
    case 9:                                    // KP_MERGE_PREP
    case 10: {                                 // KP_MERGE: heavy runs, warp sums;
      const size_t dov =                       // or the generic merge's sub-tile
          3 * (16 + 8 * (HASH_HW / 2 + 1)) + 16 + 8 * (NWARP + 1) + 16 + sizeof(MZone) + 16 + 8 +
          256;
      const size_t gen = 16 + sizeof(K) * MERGE_SUB + 16 + sizeof(K) * (HV ? MERGE_SUB : 1) +
                         16 + 2 * MERGE_SUB + 16 + 8 * (MERGE_CHUNK / MERGE_SUB + 1) + 16 +
                         sizeof(MZone) + 16 + 8 + 256;
      return dov > gen ? dov : gen;
    }
    case 11: return 256;                       // KP_STATS
    case 6: return scatter_smem<K, HV, SCATTER_NT>();  // KP_SCATTER
    default: return smem_bytes<K, HV>();       // base case
  }
}

// Threads per CTA of each per-phase kernel.
__host__ __device__ constexpr int phase_threads(int ph) { return ph == 6 ? SCATTER_NT : NT; }

// CTAs per SM the per-phase kernels are built for: the sample and the scans
// 3; the histogram 2 (64 registers: a thread's keys all loaded before the
// table lookups, no spills; 10^9 u32 key/value pairs, uniform keys: the two
// histograms 1.52 -> 1.35 ms against 3 CTAs of 40 registers); the base case 2;
// the scatter 1024 threads' worth (64 registers a thread; their shared memory
// allows no more).
__host__ __device__ constexpr int phase_min_blocks(int ph) {
  return (ph == 2 || ph == 4 || ph == 5) ? 3 : (ph == 6 ? 1024 / SCATTER_NT : 2);
}

// ----------------------------------------------------------------- queues
__device__ __forceinline__ void push_task(const Params &P, const Task &t) {
  long long i = atomic_add_ll(&P.ctl->ntasks, 1ll);
  if (i >= P.tmax) {
    latch(P, ERR_INTERNAL);
    return;
  }
  P.tasks[i] = t;
}

// Task q of the copy run [start, start + size) reserved at i0.
__device__ __forceinline__ void write_copy_task(const Params &P, int64_t start, int64_t size,
                                                int src, int dst, long long i0, long long q) {
  if (i0 + q >= P.tmax) {
    latch(P, ERR_INTERNAL);
    return;
  }
  const int64_t a = q * COPY_CHUNK;
  Task t;
  t.start = start + a;
  t.size = size - a < COPY_CHUNK ? size - a : COPY_CHUNK;
  t.base = 0;
  t.hi = 0;
  t.src = (uint8_t)src;
  t.dst = (uint8_t)dst;
  t.kind = TASK_COPY;
  P.tasks[i0 + q] = t;
}

// All of the run's tasks are reserved at once; with a list, a run of more
// than one task is left there for flush_copies.
__device__ __forceinline__ void push_copy(const Params &P, int64_t start, int64_t size,
                                          int src, int dst, const CopyList *L = nullptr) {
  if (size <= 0 || src == dst) return;
  const long long k = (size + COPY_CHUNK - 1) / COPY_CHUNK;
  const long long i0 = atomic_add_ll(&P.ctl->ntasks, k);
  if (L && k > 1) {
    const int r = atomicAdd(L->n, 1);
    if (r < COPY_REQS) {
      L->req[r] = CopyReq{start, size, i0, k, src, dst};
      return;
    }
  }
  for (long long q = 0; q < k; ++q) write_copy_task(P, start, size, src, dst, i0, q);
}

// The whole CTA writes the descriptors of the listed runs and empties the
// list (all threads call; the list's writers are done).
__device__ __forceinline__ void flush_copies(const Params &P, const CopyList &L) {
  __syncthreads();
  const int nr = min(*L.n, COPY_REQS);
  for (int r = 0; r < nr; ++r) {
    const CopyReq q = L.req[r];
    for (long long t = threadIdx.x; t < q.k; t += NT)
      write_copy_task(P, q.start, q.size, q.src, q.dst, q.i0, t);
  }
  __syncthreads();
  if (threadIdx.x == 0) *L.n = 0;
}

__device__ __forceinline__ void push_seg(const Params &P, int list, const Seg &s) {
  long long i = atomic_add_ll(&P.ctl->nseg[list], 1ll);
  if (i >= P.maxseg) {
    latch(P, ERR_INTERNAL);
    return;
  }
  P.segs[list][i] = s;
}

// A bucket that still needs work: recurse, sort on chip, or just move it.
__device__ __forceinline__ void emit_child(const Params &P, int next_list, int64_t start,
                                           int64_t size, int hi, uint64_t base, int data_buf,
                                           int res_buf, int64_t ntotal,
                                           const CopyList *L = nullptr) {
  if (size <= 0) return;
  if (hi == 0 || size == 1) {
    push_copy(P, start, size, data_buf, res_buf, L);
  } else if (size <= P.cap) {
    Task t;
    t.start = start;
    t.size = size;
    t.base = base;
    t.hi = hi;
    t.src = (uint8_t)data_buf;
    t.dst = (uint8_t)res_buf;
    t.kind = TASK_SORT;
    push_task(P, t);
  } else {
    Seg s;
    s.start = start;
    s.size = size;
    s.ntotal = ntotal;
    s.base = base;
    s.hi = hi;
    s.res = (uint8_t)res_buf;
    push_seg(P, next_list, s);
  }
}

// ------------------------------------------------------------------- seed
template <typename K, bool HV>
__device__ void phase_seed(const Params &P) {
  const int64_t S = P.offsets ? P.nsegs_in : 1;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < S;
       i += (int64_t)gridDim.x * NT) {
    int64_t a = 0, b = P.n;
    if (P.offsets) {
      a = (int64_t)__ldcg((const unsigned long long *)P.offsets + i);
      b = (int64_t)__ldcg((const unsigned long long *)P.offsets + i + 1);
      bool bad = b < a || a < 0 || b > P.n || (i == 0 && a != 0) || (i == S - 1 && b != P.n);
      if (bad) {
        latch(P, ERR_INVALID);
        continue;
      }
    }
    emit_child(P, 0, a, b - a, P.key_bits, 0, 0, 0, b - a);
  }
}

// ------------------------------------------------------------------ setup
template <typename K, bool HV>
__device__ void phase_setup(const Params &P, int level, unsigned char *smem) {
  using S = Shape<K, HV>;
  Ctl *c = P.ctl;
  const int p = level & 1;
  const int64_t nseg = min(ld_cg64(&c->nseg[p]), (long long)P.maxseg);
  long long *sh = (long long *)dts_smem;  // NWARP+1 scratch
  int64_t cr_blk = 0, cr_chk = 0, cr_b = 0, cr_h = 0, cr_z = 0, cr_hash = 0, cr_c = 0,
          cr_st = 0, cr_rec = 0;
  for (int64_t base = 0; base < nseg; base += NT) {
    const int64_t i = base + threadIdx.x;
    int64_t nblk = 0, nchk = 0, nbm = 0, hm = 0, zm = 0, hsm = 0, cm = 0, stm = 0, sz = 0;
    int g = 0;
    if (i < nseg) {
      const Seg s = ldcg_obj(&P.segs[p][i]);
      sz = s.size;
      g = plan_gamma(s.size, P.target, P.gamma_max, s.hi, FIN_DIG);
      if (learned_level(P, level)) g = 31 - __clz(P.lrn_B);  // learned zones
      const int64_t blk = (int64_t)P.blk_tiles * S::TILE;
      nblk = (s.size + blk - 1) / blk;
      nchk = (nblk + S::CH - 1) / S::CH;
      hm = (1 << (g - 1)) < HEAVY_HW ? (1 << (g - 1)) : HEAVY_HW;
      nbm = (1 << g) + hm + 1;
      zm = (1 << g) + 1;
      hsm = (1 << (g + 1)) < HASH_HW ? (1 << (g + 1)) : HASH_HW;  // load <= 1/4
      cm = nblk * nbm;
      stm = nchk * nbm;
    }
    long long tot;
    const int64_t o_blk = block_excl_scan<long long>(nblk, sh, tot) + cr_blk; cr_blk += tot;
    const int64_t o_chk = block_excl_scan<long long>(nchk, sh, tot) + cr_chk; cr_chk += tot;
    const int64_t o_b = block_excl_scan<long long>(nbm, sh, tot) + cr_b; cr_b += tot;
    const int64_t o_h = block_excl_scan<long long>(hm, sh, tot) + cr_h; cr_h += tot;
    const int64_t o_z = block_excl_scan<long long>(zm, sh, tot) + cr_z; cr_z += tot;
    const int64_t o_hs = block_excl_scan<long long>(hsm, sh, tot) + cr_hash; cr_hash += tot;
    const int64_t o_c = block_excl_scan<long long>(cm, sh, tot) + cr_c; cr_c += tot;
    const int64_t o_s = block_excl_scan<long long>(stm, sh, tot) + cr_st; cr_st += tot;
    block_excl_scan<long long>(sz, sh, tot); cr_rec += tot;
    if (i < nseg) {
      SegInfo I;
      I.gamma = g;
      I.lo = I.t = 0;
      I.nheavy = 0;
      I.nb = 0;
      I.hbits = 0;
      I.nblk = nblk;
      I.blk0 = o_blk;
      I.nchk = nchk;
      I.chk0 = o_chk;
      I.boff = o_b;
      I.hoff = o_h;
      I.zoff = o_z;
      I.hashoff = o_hs;
      I.coff = o_c;
      I.soff = o_s;
      I.mhoff = 0;
      I.learned = 0;
      I.pad_ = 0;
      P.info[i] = I;
    }
  }
  if (threadIdx.x == 0) {
    if (cr_b > P.bmax || cr_h > P.hmax || cr_z > P.zmax || cr_hash > P.hashmax ||
        cr_c > P.cwords || cr_st > P.swords) {
      latch(P, ERR_INTERNAL);
    }
    c->nblocks = cr_blk;
    c->nchunks = cr_chk;
    c->chunk_ctr = 0;
    c->task_ctr = 0;
    c->merge_ctr = 0;
    c->nseg[p ^ 1] = 0;
    if (level > 0) c->ntasks = 0;
    const unsigned long long za = __ldcg(&c->zone_alloc);
    c->lvl_zone[level] = (long long)(za >> 40);
    c->lvl_chunk[level] = za & ((1ull << 40) - 1);
    const int l = level < 15 ? level : 15;
    c->st_segments[l] += nseg;
    c->st_records[l] += cr_rec;
  }
}

// ----------------------------------------------------------------- sample
template <typename K, bool HV>
__device__ void phase_sample(const Params &P, int level, unsigned char *smem) {
  Ctl *c = P.ctl;
  const int p = level & 1;
  const int64_t nseg = min(ld_cg64(&c->nseg[p]), (long long)P.maxseg);
  const K *src = (const K *)P.keys[level & 1];
  Carve cv;
  K *Ssm = cv.take<K>(SMAX);
  K *hv = cv.take<K>(SMAX / 2 + 8);
  K *hk = cv.take<K>(HASH_HW);
  uint16_t *hid = cv.take<uint16_t>(HASH_HW);
  long long *sh = cv.take<long long>(NWARP + 1);
  long long *resv = cv.take<long long>(1);
  // per heavy key: its zone, its first sample index and occurrences, its
  // zone's sample index range, its class / its zone's layout; and the count
  // of heavy keys kept
  int *hzone = cv.take<int>(HEAVY_HW), *hlb = cv.take<int>(HEAVY_HW);
  int *hocc = cv.take<int>(HEAVY_HW), *hzs = cv.take<int>(HEAVY_HW);
  int *hze = cv.take<int>(HEAVY_HW), *hcls = cv.take<int>(HEAVY_HW);
  int *nkeep = cv.take<int>(1);
  for (int64_t si = blockIdx.x; si < nseg; si += gridDim.x) {
    const Seg S = ldcg_obj(&P.segs[p][si]);
    SegInfo I = ldcg_obj(&P.info[si]);
    const int g = I.gamma;
    const int hcap = (1 << (g - 1)) < HEAVY_HW ? (1 << (g - 1)) : HEAVY_HW;
    const int64_t nbm = (1 << g) + hcap + 1;
    const bool learned = learned_level(P, level);
    for (int64_t b = threadIdx.x; b < nbm; b += NT) P.bcount[I.boff + b] = 0;
    int L = 0;
    while (L < 63 && (1ll << L) < S.ntotal) ++L;
    if (L < 1) L = 1;
    int64_t m = ((int64_t)1 << g) * L * (int64_t)P.sample_factor;
    if (m > SMAX) m = SMAX;
    int M = 1;
    while (M < m) M <<= 1;
    const uint64_t st = P.seed ^ (uint64_t)S.start ^ ((uint64_t)S.size * 0x9E3779B97F4A7C15ull) ^
                        ((uint64_t)S.hi << 57);
    {
      // SMAX / NT draws per thread: all positions and loads first, then the
      // stores (the random loads overlap)
      constexpr int SB = SMAX / NT;
      K v[SB];
#pragma unroll
      for (int r = 0; r < SB; ++r) {
        const int k = threadIdx.x + r * NT;
        v[r] = (K)~(K)0;
        if (k < m) {
          const int64_t pos = S.start + (int64_t)(sm64_at(st, (uint64_t)k) % (uint64_t)S.size);
          v[r] = ld_key<K>(src + pos);
        }
      }
#pragma unroll
      for (int r = 0; r < SB; ++r) {
        const int k = threadIdx.x + r * NT;
        if (k < M) Ssm[k] = v[r];
      }
    }
    __syncthreads();
    // bitonic sort of the sample on chip: per stage every thread takes whole
    // compare-exchange pairs (i, i + j), i the pair's lower index
    for (int kk = 2; kk <= M; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int pr = threadIdx.x; pr < (M >> 1); pr += NT) {
          const int i = 2 * pr - (pr & (j - 1));
          const int ixj = i + j;
          const K a = Ssm[i], b = Ssm[ixj];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) {
            Ssm[i] = b;
            Ssm[ixj] = a;
          }
        }
        __syncthreads();
      }
    }
    // key range from the largest sample (overflow bucket above it)
    const uint64_t rmax = ((uint64_t)Ssm[m - 1] - S.base) & lowmask(S.hi);
    // learned zones cover the whole key range: no overflow bucket is used
    const int t = learned ? S.hi : bitlen64(rmax);
    const int lo = learned ? 0 : (t - g > 0 ? t - g : 0);
    const int geff = learned ? g : t - lo;
    const K *lspl = (const K *)P.lrn_spl;
    auto zone_of = [&](K key) -> uint64_t {
      return learned ? (uint64_t)learned_zone_exact<K>(key, lspl, 1 << g)
                     : ((((uint64_t)key - S.base) & lowmask(S.hi)) >> lo);
    };
    // heavy keys: seen at least twice among S[L-1], S[2L-1], ...
    int nh = 0;
    if (P.heavy_on) {
      const int64_t nsub = m / L;
      long long carry = 0;
      for (int64_t base = 0; base < nsub; base += NT) {
        const int64_t j = base + threadIdx.x;
        int first = 0;
        K a = 0;
        if (j + 1 < nsub) {
          a = Ssm[(j + 1) * L - 1];
          const K b = Ssm[(j + 2) * L - 1];
          first = (a == b) && (j == 0 || Ssm[j * L - 1] != a);
        }
        long long tot;
        const long long o = block_excl_scan<long long>(first, sh, tot) + carry;
        if (first && o < (SMAX / 2 + 8)) hv[o] = a;
        carry += tot;
      }
      nh = (int)carry;
      if (nh > hcap) nh = hcap;
      if (nh > 0) {
        // the layout of each zone's buckets (numbered in key order): heavy
        // keys below every light key of the zone's sample, the light bucket,
        // the other heavy keys.  A zone whose light keys all fall between
        // them needs no dovetail merge (checked on every light key by the
        // histogram).  Heavy keys with sampled light keys on both sides
        // ("interior") force the merge of the zone; when they hold less
        // than 1/8 of the rest of the zone's sample they are dropped
        // instead (their records stay light and are distributed once more).
        __syncthreads();  // hv, written after the last scan's barrier
        for (int j = threadIdx.x; j < nh; j += NT) {
          const K h = hv[j];
          const int zj = (int)zone_of(h);
          int a = 0, b = (int)m;
          while (a < b) {
            const int mid = (a + b) >> 1;
            if (Ssm[mid] < h) a = mid + 1;
            else b = mid;
          }
          const int lbj = a;
          b = (int)m;
          while (a < b) {
            const int mid = (a + b) >> 1;
            if (!(h < Ssm[mid])) a = mid + 1;
            else b = mid;
          }
          const int ubj = a;
          a = 0;
          b = lbj;
          while (a < b) {
            const int mid = (a + b) >> 1;
            if (zone_of(Ssm[mid]) < (uint64_t)zj) a = mid + 1;
            else b = mid;
          }
          const int zsj = a;
          a = ubj;
          b = (int)m;
          while (a < b) {
            const int mid = (a + b) >> 1;
            if (zone_of(Ssm[mid]) <= (uint64_t)zj) a = mid + 1;
            else b = mid;
          }
          hzone[j] = zj;
          hlb[j] = lbj;
          hocc[j] = ubj - lbj;
          hzs[j] = zsj;
          hze[j] = a;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          // classes: 0 below the zone's light sample keys, 1 above, 2 interior
          int kept = 0;
          long long wkept = 0;  // sample keys equal to a kept heavy key
          for (int j0 = 0; j0 < nh;) {
            int j1 = j0 + 1;
            while (j1 < nh && hzone[j1] == hzone[j0]) ++j1;
            int occ = 0;
            for (int j = j0; j < j1; ++j) occ += hocc[j];
            int below = 0, npre = 0, nint = 0, wint = 0;
            for (int j = j0; j < j1; ++j) {
              const int lbelow = (hlb[j] - hzs[j0]) - below;
              const int labove = (hze[j0] - hlb[j] - hocc[j]) - (occ - below - hocc[j]);
              const int cl = lbelow == 0 ? 0 : (labove == 0 ? 1 : 2);
              hcls[j] = cl;
              npre += cl == 0;
              if (cl == 2) {
                ++nint;
                wint += hocc[j];
              }
              below += hocc[j];
            }
            const int wrest = (hze[j0] - hzs[j0]) - wint;
            const bool drop = nint > 0 && 8 * wint < wrest;
            const bool force = nint > 0 && !drop;
            // layout code per kept key: heavy buckets before the light one
            // (bits 0-7), forced merge (bit 8)
            const int code = (force ? 0 : npre) | (force ? 256 : 0);
            for (int j = j0; j < j1; ++j) {
              if (drop && hcls[j] == 2) continue;
              wkept += hocc[j];
              hv[kept] = hv[j];
              hzone[kept] = hzone[j];
              hcls[kept] = code;
              ++kept;
            }
            j0 = j1;
          }
          // heavy keys that hold less than the minimum share of the sample
          // are not worth the table lookup every record of the subproblem
          // then pays: the digit alone distributes it
          if (1000 * wkept < (long long)P.heavy_min_share * m) kept = 0;
          *nkeep = kept;
        }
        __syncthreads();
        nh = *nkeep;
      }
      if (nh > 0) {
        // room for this subproblem's heavy buckets in the merge store
        if (threadIdx.x == 0) {
          const long long off = atomic_add_ll(&c->mh_alloc, (long long)nh);
          *resv = (off + nh > P.mhmax) ? -1 : off;
        }
        __syncthreads();
        const long long off = *resv;
        __syncthreads();
        if (off < 0) nh = 0;  // store full: plain digit buckets for this one
        else I.mhoff = off;
      }
    }
    // heavy list out; light table: zone z's buckets start at z + (heavy keys
    // in zones < z), its light bucket after the heavy keys placed before it
    for (int j = threadIdx.x; j < nh; j += NT) ((K *)P.heavy)[I.hoff + j] = hv[j];
    const int nz = 1 << geff;
    for (int z = threadIdx.x; z <= nz; z += NT) {
      int a = 0, b = nh;
      while (a < b) {
        const int mid = (a + b) >> 1;
        if (hzone[mid] < z) a = mid + 1;
        else b = mid;
      }
      int e = a;
      b = nh;
      while (e < b) {
        const int mid = (e + b) >> 1;
        if (hzone[mid] <= z) e = mid + 1;
        else b = mid;
      }
      const int mz = e - a;
      const int code = mz ? hcls[a] : 0;
      P.lid[I.zoff + z] = le_pack(z + a + (code & 255), a, mz, (code & 256) != 0);
    }
    int hbits = 0;
    if (nh > 0) {
      hbits = 1;
      while ((1 << hbits) < 4 * nh) ++hbits;  // load factor <= 1/4: light keys stop early
      const int cap = 1 << hbits;
      for (int i = threadIdx.x; i < cap; i += NT) hid[i] = HEMPTY;
      __syncthreads();
      if (threadIdx.x == 0) {
        int g0 = 0;  // first heavy key of the current zone
        for (int j = 0; j < nh; ++j) {
          const K key = hv[j];
          const int zone = hzone[j];
          if (j == 0 || zone != hzone[j - 1]) g0 = j;
          // bucket of the zone's (j - g0)-th heavy key: after the light
          // bucket unless among the ones placed before it
          const int id = zone + j + (j - g0 < (hcls[j] & 255) ? 0 : 1);
          uint32_t s = hash_slot<K>(key, hbits);
          while (hid[s] != HEMPTY) s = (s + 1) & (uint32_t)(cap - 1);
          hk[s] = key;
          hid[s] = (uint16_t)id;
        }
      }
      __syncthreads();
      K *HK = (K *)P.hash_keys + I.hashoff;
      for (int i = threadIdx.x; i < cap; i += NT) {
        HK[i] = hk[i];
        P.hash_ids[I.hashoff + i] = hid[i];
      }
    }
    if (threadIdx.x == 0) {
      I.lo = lo;
      I.t = t;
      I.nheavy = nh;
      I.nb = nz + nh + 1;
      I.hbits = hbits;
      I.learned = learned ? 1 : 0;
      P.info[si] = I;
      atomic_add_ll(&c->st_heavy_keys[level < 15 ? level : 15], (long long)nh);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- histogram
// Row r of a subproblem's count matrix = bucket counts of its block r (the
// blocked counting sort of App. B); blocks are split evenly over the CTAs.
template <typename K, bool HV>
__device__ void phase_hist(const Params &P, int level, unsigned char *smem) {
  using S = Shape<K, HV>;
  Ctl *c = P.ctl;
  const int64_t nseg = min(ld_cg64(&c->nseg[level & 1]), (long long)P.maxseg);
  const int64_t nblocks = ld_cg64(&c->nblocks);
  if (nblocks == 0) return;
  const K *src = (const K *)P.keys[level & 1];
  Carve cv;
  SegTables<K> &T = *cv.take<SegTables<K>>(1);
  int32_t *lid_s = cv.take<int32_t>((1 << GAMMA_HW) + 1);
  K *hk_s = cv.take<K>(HASH_HW);
  uint16_t *hid_s = cv.take<uint16_t>(HASH_HW);
  K *hl_s = cv.take<K>(HEAVY_HW);
  unsigned *cnt = cv.take<unsigned>(NB_PAD);
  K *spl_s = cv.take<K>(1 << GAMMA_HW);
  float *tab_s = cv.take<float>(LRN_TAB_N + 1);
  long long fix_recs = 0, fix_steps = 0;
  unsigned bad = 0;  // a bucket id out of range (self-check), reported once
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r0 = nblocks * blockIdx.x / gridDim.x;
  const int64_t r1 = nblocks * (blockIdx.x + 1) / gridDim.x;
  // the current subproblem and the end of its blocks, in registers: T is
  // rewritten by thread 0 when the next one is loaded
  int cur = -1;
  int64_t cur_end = 0;
  for (int64_t r = r0; r < r1; ++r) {
    if (cur < 0 || r >= cur_end) {
      const int s = find_blk_seg(P, nseg, r);
      if (s != cur) {
        load_tables<K>(P, s, level, T, lid_s, hk_s, hid_s, hl_s, spl_s, tab_s);
        cur = s;
      }
      cur_end = T.info.blk0 + T.info.nblk;
    }
    const int nb = T.info.nb;
    const int lo = T.info.lo;

    const unsigned gmask = (1u << (T.info.t - T.info.lo)) - 1u;
    const bool fast = T.info.hbits == 0 && T.info.t >= T.hi && !T.info.learned;
    const uint64_t kbase = T.base;
    const BucketCtx X = bucket_ctx<K>(T);
    const int64_t lr = r - T.info.blk0;
    if (lr % S::CH == 0) {  // this chunk's look-back status starts empty
      const int64_t row = T.info.soff + (lr / S::CH) * nb;
      for (int b = threadIdx.x; b < nb; b += NT) P.status[row + b] = 0ull;
    }
    for (int b = threadIdx.x; b < NB_PAD; b += NT) cnt[b] = 0;
    __syncthreads();
    const int64_t b0 = T.start + lr * (int64_t)P.blk_tiles * S::TILE;
    const int64_t brem = T.start + T.size - b0;
    for (int sub = 0; sub < P.blk_tiles; ++sub) {
      const int64_t tb = (int64_t)sub * S::TILE;
      if (tb >= brem) break;
      const int tn = brem - tb < S::TILE ? (int)(brem - tb) : S::TILE;
      const K *ts = src + b0 + tb;
      if (threadIdx.x == 0) prefetch_l2<K>(src, b0 + tb + S::TILE, S::TILE, P.n);
      if (fast) {
        // all of a thread's keys loaded before any is counted
        K key[S::ITEMS];
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          key[j] = i < tn ? ld_key<K>(ts + i) : (K)0;
        }
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          // b <= gmask < nb: the tables were checked when loaded
          if (i < tn) atomicAdd(&cnt[fast_digit<K>(key[j], kbase, lo, gmask)], 1u);
        }
      } else {
        // all of a thread's keys loaded before any is looked up
        constexpr int HC = S::ITEMS;
        static_assert(S::ITEMS % HC == 0, "whole key groups");
#pragma unroll
        for (int j0 = 0; j0 < S::ITEMS; j0 += HC) {
          K key[HC];
#pragma unroll
          for (int r = 0; r < HC; ++r) {
            const int i = w * 32 * S::ITEMS + (j0 + r) * 32 + lane;
            key[r] = i < tn ? ld_key<K>(ts + i) : (K)0;
          }
          if (X.learned) {
#pragma unroll
            for (int r = 0; r < HC; ++r) {
              const int i = w * 32 * S::ITEMS + (j0 + r) * 32 + lane;
              if (i < tn) {
                unsigned st = 0;
                const unsigned b = bucket_of<K, true>(X, lid_s, hk_s, hid_s, hl_s, key[r],
                                                      spl_s, tab_s, &st);
                if (b < (unsigned)nb) atomicAdd(&cnt[b], 1u);
                else bad = b;
                fix_recs += st != 0;
                fix_steps += st;
              }
            }
          } else {
#pragma unroll
            for (int r = 0; r < HC; ++r) {
              const int i = w * 32 * S::ITEMS + (j0 + r) * 32 + lane;
              if (i < tn) {
                const unsigned b = bucket_of<K, true>(X, lid_s, hk_s, hid_s, hl_s, key[r]);
                if (b < (unsigned)nb) atomicAdd(&cnt[b], 1u);
                else bad = b;
              }
            }
          }
        }
      }
    }
    __syncthreads();
    unsigned *row = P.cmat + T.info.coff + lr * nb;
    for (int b = threadIdx.x; b < nb; b += NT) row[b] = cnt[b];
    // zones whose layout a light key of this block broke (LE_MERGE in the
    // on-chip table) are marked in the global light table, which the bucket
    // scan reads
    if (T.info.hbits) {
      const int nzl = T.info.learned ? (1 << T.info.gamma) : (1 << (T.info.t - T.info.lo));
      for (int z = threadIdx.x; z < nzl; z += NT) {
        const int32_t e = lid_s[z];
        if ((e & LE_MERGE) && le_mz(e)) atomicOr(P.lid + T.info.zoff + z, LE_MERGE);
      }
    }
    __syncthreads();
  }
  if (fix_recs) {
    atomic_add_ll(&c->st_fix_records, fix_recs);
    atomic_add_ll(&c->st_fix_steps, fix_steps);
  }
  if (bad) check_failed(P, 3, bad, level);
}

// ------------------------------------------------- count-matrix scan
// Exclusive scan of every column of a subproblem's count matrix (offset of
// each bucket's records of block r among that bucket's records) as one pass
// over chunks of CH rows with decoupled look-back across chunks.  The last
// chunk of a subproblem also yields the bucket totals.
template <typename K, bool HV>
__device__ void phase_mscan(const Params &P, int level, unsigned char *smem) {
  using S = Shape<K, HV>;
  Ctl *c = P.ctl;
  const int64_t nseg = min(ld_cg64(&c->nseg[level & 1]), (long long)P.maxseg);
  const int64_t nchunks = ld_cg64(&c->nchunks);
  long long *chunk_sh = (long long *)dts_smem;
  SegInfo *Is = (SegInfo *)(dts_smem + 16);
  while (true) {
    if (threadIdx.x == 0) *chunk_sh = atomic_add_ll(&c->chunk_ctr, 1ll);
    __syncthreads();
    const int64_t ch = *chunk_sh;
    if (ch >= nchunks) break;
    if (threadIdx.x == 0) *Is = ldcg_obj(&P.info[find_chk_seg(P, nseg, ch)]);
    __syncthreads();
    const SegInfo I = *Is;
    const int nb = I.nb;
    const int64_t lc = ch - I.chk0;
    const int64_t rb = lc * S::CH;
    const int64_t re = rb + S::CH < I.nblk ? rb + S::CH : I.nblk;
    const bool mute = P.debug_fault == 1 && level == 0 && ch == 1;
    unsigned *C = P.cmat + I.coff;
    unsigned long long *st = P.status + I.soff;
    for (int b = threadIdx.x; b < nb; b += NT) {
      unsigned long long sum = 0;
      for (int64_t r = rb; r < re; ++r) sum += __ldcg(C + r * nb + b);
      unsigned long long excl = 0;
      if (lc == 0) {
        st_relaxed(&st[b], (2ull << 62) | sum);
      } else {
        if (!mute) st_relaxed(&st[lc * nb + b], (1ull << 62) | sum);
        int64_t q = lc - 1;
        const unsigned long long t0 = gtimer();
        unsigned ns = 32;
        bool timed_out = false;
        while (true) {
          const unsigned long long v = ld_relaxed(&st[q * nb + b]);
          const unsigned f = (unsigned)(v >> 62);
          if (f == 0) {
            if (gtimer() - t0 > P.wait_ns) {
              timed_out = true;
              break;
            }
            __nanosleep(ns);
            ns = ns < 512 ? ns * 2 : 512;
            continue;
          }
          excl += v & ((1ull << 62) - 1);
          if (f == 2) break;
          --q;
        }
        if (timed_out) {
          latch(P, ERR_TIMEOUT);
          __threadfence();
        }
        if (!mute) st_relaxed(&st[lc * nb + b], (2ull << 62) | (excl + sum));
      }
      unsigned long long run = excl;
      for (int64_t r = rb; r < re; ++r) {
        const unsigned v = __ldcg(C + r * nb + b);
        C[r * nb + b] = (unsigned)run;
        run += v;
      }
      if (re == I.nblk) P.bcount[I.boff + b] = (long long)run;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- scan
template <typename K, bool HV>
__device__ void phase_scan(const Params &P, int level, unsigned char *smem) {
  Ctl *c = P.ctl;
  const int p = level & 1;
  const int64_t nseg = min(ld_cg64(&c->nseg[p]), (long long)P.maxseg);
  const int srcb = level & 1, dstb = srcb ^ 1;
  Carve cv;
  long long *cntv = cv.take<long long>(NB_PAD);
  long long *excl = cv.take<long long>(NB_PAD + 1);
  int32_t *lid_s = cv.take<int32_t>((1 << GAMMA_HW) + 1);
  long long *sh = cv.take<long long>(NWARP + 1);
  CopyList CL{cv.take<CopyReq>(COPY_REQS), cv.take<int>(1)};
  if (threadIdx.x == 0) *CL.n = 0;
  __syncthreads();
  for (int64_t si = blockIdx.x; si < nseg; si += gridDim.x) {
    const Seg S = ldcg_obj(&P.segs[p][si]);
    const SegInfo I = ldcg_obj(&P.info[si]);
    const int nb = I.nb;
    // bucket starts: two buckets per thread, one CTA-wide scan
    for (int b = threadIdx.x; b < NB_PAD; b += NT)
      cntv[b] = b < nb ? (long long)__ldcg((const unsigned long long *)&P.bcount[I.boff + b]) : 0;
    __syncthreads();
    const int i0 = 2 * threadIdx.x, i1 = i0 + 1;
    const long long v0 = i0 < NB_PAD ? cntv[i0] : 0;
    const long long v1 = i1 < NB_PAD ? cntv[i1] : 0;
    long long tot;
    const long long o = block_excl_scan<long long>(v0 + v1, sh, tot);
    if (i0 < NB_PAD) excl[i0] = o;
    if (i1 < NB_PAD) excl[i1] = o + v0;
    if (threadIdx.x == 0) excl[NB_PAD] = tot;
    const int nz = I.learned ? (1 << I.gamma) : (1 << (I.t - I.lo));
    for (int z = threadIdx.x; z <= nz; z += NT) lid_s[z] = __ldcg(P.lid + I.zoff + z);
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += NT) P.bstart[I.boff + b] = S.start + excl[b];
    const int res = S.res;
    long long heavy_recs = 0;
    long long free_zones = 0;
    for (int z = threadIdx.x; z < nz; z += NT) {
      // zone z's buckets [zb, zb + m], its light bucket lb among them (mp
      // heavy buckets before it)
      const int32_t e = lid_s[z];
      const int lb = le_light(e), hf = le_hfirst(e), m = le_mz(e);
      const int zb = z + hf, mp = lb - zb;
      if (e < 0 || mp < 0 || mp > m || zb + m >= nb - 1 || hf + m > I.nheavy) {
        check_failed(P, 7, z, (long long)e);
        continue;
      }
      const int64_t zs = S.start + excl[zb];
      const int64_t ls = S.start + excl[lb];
      const int64_t b0 = cntv[lb];
      const int64_t ze = S.start + excl[zb + m + 1];
      int light_res = res;
      if (m > 0) {
        heavy_recs += ze - zs - b0;
        // the heavy runs: [zs, ls) before the light bucket, [ls + b0, ze) after
        if ((e & LE_MERGE) && b0 > 0) {
          light_res = res ^ 1;  // the merge reads from the other buffer
          const int64_t nch = (ze - zs + MERGE_CHUNK - 1) / MERGE_CHUNK;
          const unsigned long long old =
              atomicAdd(&c->zone_alloc, (1ull << 40) | (unsigned long long)nch);
          const int64_t zidx = (int64_t)(old >> 40);
          const int64_t mh = I.mhoff + hf;
          for (int q = 0; q < m; ++q) {
            ((K *)P.mh_keys)[mh + q] = ld_key<K>((const K *)P.heavy + I.hoff + hf + q);
            P.mh_sizes[mh + q] = cntv[zb + q + (q < mp ? 0 : 1)];
          }
          MZone Z;
          Z.zs = zs;
          Z.b0 = b0;
          Z.ze = ze;
          Z.mh = mh;
          Z.chunk0 = (int64_t)(old & ((1ull << 40) - 1));
          Z.m = m;
          Z.obuf = (uint8_t)res;
          Z.np = (uint8_t)mp;
          if (zidx < P.mhmax) P.zones[zidx] = Z;
          else latch(P, ERR_INTERNAL);
          // heavy runs must sit in the merge's input buffer
          if (dstb == res) {
            push_copy(P, zs, ls - zs, dstb, dstb ^ 1, &CL);
            push_copy(P, ls + b0, ze - ls - b0, dstb, dstb ^ 1, &CL);
          }
        } else {
          // the zone's runs are already in key order: the light bucket's
          // result and the heavy runs go straight to the required buffer
          free_zones += 1;
          if (dstb != res) {
            push_copy(P, zs, ls - zs, dstb, res, &CL);
            push_copy(P, ls + b0, ze - ls - b0, dstb, res, &CL);
          }
        }
      }
      // the light bucket's keys: digit zone z covers base + [z, z+1) * 2^lo;
      // learned zone z covers [spl[z], spl[z+1])
      int chi = I.lo;
      uint64_t cbase = S.base + ((uint64_t)z << I.lo);
      if (I.learned) {
        const K *spl = (const K *)P.lrn_spl;
        const uint64_t a = (uint64_t)ld_key<K>(spl + z);
        const uint64_t top = z + 1 < nz ? (uint64_t)ld_key<K>(spl + z + 1) - 1
                                        : (uint64_t)(K)~(K)0;
        cbase = a;
        chi = top >= a ? bitlen64(top - a) : 0;
      }
      emit_child(P, p ^ 1, ls, b0, chi, cbase, dstb, light_res, S.ntotal, &CL);
      if (level == 0 && si == 0) {
        atomicAdd(&c->st_bsum, (double)b0);
        atomicAdd(&c->st_bsq, (double)b0 * (double)b0);
        atomicMax((unsigned long long *)&c->st_bmax, (unsigned long long)b0);
      }
    }
    if (level == 0 && si == 0 && threadIdx.x == 0) c->st_bnz = nz;
    if (threadIdx.x == 0) {
      const int ob = nb - 1;
      const int64_t os = S.start + excl[ob], ol = cntv[ob];
      if (ol > 0) {
        emit_child(P, p ^ 1, os, ol, S.hi, S.base, dstb, res, S.ntotal, &CL);
        atomic_add_ll(&c->st_overflow[level < 15 ? level : 15], (long long)ol);
      }
    }
    if (heavy_recs) atomic_add_ll(&c->st_heavy_records[level < 15 ? level : 15], heavy_recs);
    if (free_zones) atomic_add_ll(&c->st_free_zones, free_zones);
    flush_copies(P, CL);
  }
}

// ---------------------------------------------------------------- scatter
// Stable counting-sort scatter: block r writes bucket b's records starting at
// bstart[b] + X[r][b]; inside the block, tiles of TILE records are ranked per
// warp in input order and staged in shared memory in bucket order so that
// each bucket's run is written contiguously.  A subproblem without heavy keys
// whose digit reaches its top unsorted bit needs no table: bucket = digit.
// Per tile: clear the peer slots | barrier | rank (warp counters) | barrier |
// tile scan, then each warp's first slot per bucket (one barrier inside) |
// barrier | stage | barrier | write-out (the warp counters are cleared
// meanwhile) | barrier.
template <typename K, bool HV, int NTS = NT>
__device__ void phase_scatter(const Params &P, int level, unsigned char *smem) {
  using S = Shape<K, HV>;
  constexpr int NWS = NTS / 32;           // warps of this CTA
  constexpr int TILE = NTS * S::ITEMS;    // records per tile
  Ctl *c = P.ctl;
  const int64_t nseg = min(ld_cg64(&c->nseg[level & 1]), (long long)P.maxseg);
  const int64_t nblocks = ld_cg64(&c->nblocks);
  const int srcb = level & 1, dstb = srcb ^ 1;
  const K *src = (const K *)P.keys[srcb];
  K *dst = (K *)P.keys[dstb];
  const K *vsrc = HV ? (const K *)P.vals[srcb] : nullptr;
  K *vdst = HV ? (K *)P.vals[dstb] : nullptr;
  Carve cv;
  SegTables<K> &T = *cv.take<SegTables<K>>(1);
  int32_t *lid_s = cv.take<int32_t>((1 << GAMMA_HW) + 1);
  K *hk_s = cv.take<K>(HASH_HW);
  uint16_t *hid_s = cv.take<uint16_t>(HASH_HW);
  K *hl_s = cv.take<K>(HEAVY_HW);
  unsigned *wc2 = cv.take<unsigned>(NWS * NB_PAIR);  // warp counters, 16-bit pairs
  // FOLD: the warps' counters become their first slots per bucket (tile
  // offset included), so staging reads one table instead of two (32-bit
  // key/value pairs with 1024-thread CTAs, 10^9 records: scatters 13.31 ->
  // 12.93 ms; with the earlier 512-thread CTAs it had lost to spills)
  constexpr bool FOLD = true;
  unsigned *toff = cv.take<unsigned>(FOLD ? 1 : NB_PAD);
  unsigned *gbase = cv.take<unsigned>(NB_PAD);
  unsigned *base = cv.take<unsigned>(NB_PAD);
  unsigned *sh = cv.take<unsigned>(NWS + 1);
  K *spl_s = cv.take<K>(1 << GAMMA_HW);
  float *tab_s = cv.take<float>(LRN_TAB_N + 1);
  // the staged tile: keys + destinations, or keys + values on the fast path
  constexpr int AREA = scatter_area<K, HV, NTS>();
  unsigned char *area = cv.take<unsigned char>(AREA);
  K *stage = (K *)area;
  unsigned *dest = (unsigned *)(area + TILE * sizeof(K));  // offset in the subproblem
  // the ranking's peer slots use the staging area too (cleared before each
  // tile is ranked, after the previous tile's write-out has finished)
  static_assert(AREA >= 4 * NWS * NB_PAD, "slots fit in the staging area");
  unsigned *slots = (unsigned *)area;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned bad = 0;  // self-check: a slot or destination out of range, reported once
  unsigned *mywc = wc2 + w * NB_PAIR;
  unsigned *myslot = slots + w * NB_PAD;
  for (int i = threadIdx.x; i < NWS * NB_PAIR; i += NTS) wc2[i] = 0u;
  __syncthreads();
  const int64_t r0 = nblocks * blockIdx.x / gridDim.x;
  const int64_t r1 = nblocks * (blockIdx.x + 1) / gridDim.x;
  // the current subproblem and the end of its blocks, in registers: T is
  // rewritten by thread 0 when the next one is loaded
  int cur = -1;
  int64_t cur_end = 0;
  for (int64_t r = r0; r < r1; ++r) {
    if (cur < 0 || r >= cur_end) {
      const int s = find_blk_seg(P, nseg, r);
      if (s != cur) {
        load_tables<K>(P, s, level, T, lid_s, hk_s, hid_s, hl_s, spl_s, tab_s);
        cur = s;
      }
      cur_end = T.info.blk0 + T.info.nblk;
    }
    const int nb = T.info.nb;
    const int npair = (nb + 2) / 2;  // pairs covering buckets 0..nb (nb: the dummy)
    const int lo = T.info.lo;
    const unsigned gmask = (1u << (T.info.t - T.info.lo)) - 1u;
    const bool fast = T.info.hbits == 0 && T.info.t >= T.hi && !T.info.learned;
    const uint64_t kbase = T.base;
    const BucketCtx X = bucket_ctx<K>(T);
    const int64_t lr = r - T.info.blk0;
    const unsigned *Xr = P.cmat + T.info.coff + lr * nb;  // this block's offsets
    for (int b = threadIdx.x; b < nb; b += NTS)
      base[b] = (unsigned)(__ldcg((const long long *)&P.bstart[T.info.boff + b]) - T.start) +
                __ldcg(Xr + b);
    const int64_t blkrec = (int64_t)P.blk_tiles * S::TILE;  // records per row
    const int64_t b0 = T.start + lr * blkrec;
    const int64_t brem = T.start + T.size - b0 < blkrec ? T.start + T.size - b0 : blkrec;
    K *dseg = dst + T.start;
    K *vdseg = HV ? vdst + T.start : nullptr;
    const unsigned seg_size = (unsigned)T.size;
    for (int64_t tb = 0; tb < brem; tb += TILE) {
      const int tn = brem - tb < TILE ? (int)(brem - tb) : TILE;
      const int64_t tbase = b0 + tb;
      K key[S::ITEMS];
      unsigned br[S::ITEMS];  // bucket << 16 | rank within warp, later the slot
#pragma unroll
      for (int j = 0; j < S::ITEMS; ++j) {
        const int i = w * 32 * S::ITEMS + j * 32 + lane;
        key[j] = i < tn ? ld_key<K>(src + tbase + i) : (K)0;
      }
      // L2 prefetches, by measurement (10^9 records, the two scatters): 64-bit
      // keys fetch the next tile's keys and this and the next tile's values
      // (key/value 26.0 -> 24.0 ms); 32-bit key/value pairs fetch this tile's
      // values, which are read only after the ranking (15.5 -> 14.7 ms; the
      // next tile's keys as well measured 14.9 ms); 32-bit keys alone fetch
      // the next tile's keys (9.8 -> 9.0 ms)
      if (threadIdx.x == 0) {
        if constexpr (sizeof(K) == 8) {
          prefetch_l2<K>(src, tbase + TILE, TILE, P.n);
          if constexpr (HV) prefetch_l2<K>(vsrc, tbase, 2 * TILE, P.n);
        } else if constexpr (HV) {
          prefetch_l2<K>(vsrc, tbase, TILE, P.n);
          // one CTA per SM: nothing else hides the next tile's key loads
          if (NTS > NT) prefetch_l2<K>(src, tbase + TILE, TILE, P.n);
        } else {
          prefetch_l2<K>(src, tbase + TILE, TILE, P.n);
        }
      }
      {
        uint4 *z = (uint4 *)slots;
        for (int i = threadIdx.x; i < NWS * NB_PAD / 4; i += NTS) z[i] = make_uint4(0, 0, 0, 0);
      }
      __syncthreads();
      if (fast) {
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          const unsigned b = i < tn ? fast_digit<K>(key[j], kbase, lo, gmask) : (unsigned)nb;
          br[j] = (b << 16) | warp_rank(b, myslot, mywc);
        }
      } else {
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          const unsigned b =
              i < tn ? bucket_of<K>(X, lid_s, hk_s, hid_s, hl_s, key[j], spl_s, tab_s)
                     : (unsigned)nb;
          br[j] = (b << 16) | warp_rank(b, myslot, mywc);
        }
      }
      __syncthreads();
      // per bucket pair (2p, 2p+1): tile counts, the tile offsets (exclusive
      // scan over buckets) and bases; then every warp's counter pair becomes
      // its first slots in the staged tile (tile offset + exclusive prefix
      // over warps; below TILE, so the 16-bit halves cannot carry)
      {
        const int p = threadIdx.x;
        unsigned tot2 = 0;
        if (p < npair) {
#pragma unroll
          for (int q = 0; q < NWS; ++q) {
            const unsigned y = wc2[q * NB_PAIR + p];
            if constexpr (!FOLD) wc2[q * NB_PAIR + p] = tot2;  // exclusive prefix
            tot2 += y;
          }
        }
        const unsigned c0 = tot2 & 0xFFFFu, c1 = tot2 >> 16;
        const unsigned v = c0 + c1;
        unsigned x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) sh[w] = x;
        __syncthreads();
        if (p < npair) {
          unsigned off = x - v;
          for (int q = 0; q < w; ++q) off += sh[q];
          const int b = 2 * p;
          if constexpr (FOLD) {
            unsigned run = off | ((off + c0) << 16);
#pragma unroll
            for (int q = 0; q < NWS; ++q) {
              const unsigned y = wc2[q * NB_PAIR + p];
              wc2[q * NB_PAIR + p] = run;
              run += y;
            }
          } else {
            toff[b] = off;
            toff[b + 1] = off + c0;
          }
          gbase[b] = base[b] - off;
          gbase[b + 1] = base[b + 1] - off - c0;
          base[b] += c0;
          base[b + 1] += c1;
        }
      }
      __syncthreads();
      if (fast) {
        // keys and values staged side by side in bucket order; the write-out
        // takes each record's bucket again from its key (a digit), so no
        // destination array is kept and both arrays go out in one pass
        K *stage_v = (K *)(area + TILE * sizeof(K));
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          if (i < tn) {
            const unsigned b = br[j] >> 16;
            const unsigned pj =
                (FOLD ? 0u : toff[b]) + half16(mywc[b >> 1], b) + (br[j] & 0xFFFFu);
            if (b >= (unsigned)nb || pj >= (unsigned)tn) {
              bad = 1u + pj;
              br[j] = 0xFFFFFFFFu;
              continue;
            }
            stage[pj] = key[j];
            br[j] = pj;
          }
        }
        if constexpr (HV) {
#pragma unroll
          for (int j = 0; j < S::ITEMS; ++j) {
            const int i = w * 32 * S::ITEMS + j * 32 + lane;
            if (i < tn && br[j] != 0xFFFFFFFFu)
              stage_v[br[j]] = ld_key<K>(vsrc + tbase + i);
          }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NWS * NB_PAIR; i += NTS) wc2[i] = 0u;
        for (int q = threadIdx.x; q < tn; q += NTS) {
          const K k = stage[q];
          const unsigned d = gbase[fast_digit<K>(k, kbase, lo, gmask)] + (unsigned)q;
          if (d < seg_size) {
            st_key_hint<K>(dseg + d, k, l2_policy_evict_last());
            if constexpr (HV) st_key_hint<K>(vdseg + d, stage_v[q], l2_policy_evict_last());
          } else {
            bad = 1u + d;
          }
        }
        __syncthreads();
        continue;
      }
      // stage keys in bucket order, then write each bucket's run contiguously;
      // br[j] becomes the item's slot in the staged tile
#pragma unroll
      for (int j = 0; j < S::ITEMS; ++j) {
        const int i = w * 32 * S::ITEMS + j * 32 + lane;
        if (i < tn) {
          const unsigned b = br[j] >> 16;
          const unsigned pj =
              (FOLD ? 0u : toff[b]) + half16(mywc[b >> 1], b) + (br[j] & 0xFFFFu);
          if (b >= (unsigned)nb || pj >= (unsigned)tn) {
            bad = 1u + pj;
            br[j] = 0;
            continue;
          }
          stage[pj] = key[j];
          dest[pj] = gbase[b] + pj;
          br[j] = pj;
        }
      }
      // value loads go out before the key stores so that both overlap
      K val[HV ? S::ITEMS : 1];
      if constexpr (HV) {
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          val[j] = i < tn ? ld_key<K>(vsrc + tbase + i) : (K)0;
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < NWS * NB_PAIR; i += NTS) wc2[i] = 0u;
      for (int q = threadIdx.x; q < tn; q += NTS) {
        const unsigned d = dest[q];
        if (d < seg_size) st_key_hint<K>(dseg + d, stage[q], l2_policy_evict_last());
        else bad = 1u + d;
      }
      if constexpr (HV) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < S::ITEMS; ++j) {
          const int i = w * 32 * S::ITEMS + j * 32 + lane;
          if (i < tn) stage[br[j]] = val[j];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < tn; q += NTS) {
          const unsigned d = dest[q];
          if (d < seg_size) st_key_hint<K>(vdseg + d, stage[q], l2_policy_evict_last());
        }
      }
      __syncthreads();
    }
  }
  if (bad) check_failed(P, 1, bad - 1u, level);
}

// ------------------------------------------------------- base case + copy
// Bins of the one-pass base case for composites of type CT: the most
// (2^9..2^13) whose padded counters fit in the base-case area beside the
// placed composites and, with values, the values in input order.
template <typename K, bool HV, typename CT>
__host__ __device__ constexpr int fin_fb() {
  using S = Shape<K, HV>;
  int fb = 13;
  while (fb > 9 && 4 * ((1 << fb) + NT) + 32 + S::FIN_CAP * ((int)sizeof(CT) + S::VB) >
                       S::FIN_BYTES)
    --fb;
  return fb;
}

// key - kb in the key's own width (32-bit arithmetic for 32-bit keys).
template <typename K>
using KOff = typename std::conditional<sizeof(K) == 4, uint32_t, uint64_t>::type;
template <typename K>
__device__ __forceinline__ KOff<K> key_off(K k, K kb) {
  return (KOff<K>)(k - kb);
}

// Bin of a record: the top fb bits of its composite (key - kb) << IB | i,
// whose key part has `bits` bits: ksh = max(bits - fb, 0) key bits are
// dropped, and when the key part is narrower than fb the top ish =
// max(fb - bits, 0) index bits fill in (so that the records of one key value
// spread over bins by position; without values there are no index bits and
// ish is 0).
template <typename K, bool HV>
__device__ __forceinline__ unsigned fin_bin(KOff<K> dk, int i, int ksh, int ish) {
  if constexpr (HV) return ((unsigned)(dk >> ksh) << ish) | ((unsigned)i >> (FIN_IB - ish));
  else return (unsigned)(dk >> ksh);
}

// Layout of the base-case area for composites of type CT: the bins (thread
// t's run of per bins at t (per + 1)), the placed composites, the values in
// input order.
template <typename K, bool HV, typename CT>
struct FinArea {
  static constexpr int FBM = fin_fb<K, HV, CT>();
  static constexpr int PC_OFF = (4 * ((1 << FBM) + NT) + 15) & ~15;
  static constexpr int V_OFF = PC_OFF + ((int)((sizeof(CT) * Shape<K, HV>::FIN_CAP + 15) & ~15));
  static_assert(V_OFF + Shape<K, HV>::VB * Shape<K, HV>::FIN_CAP <= Shape<K, HV>::FIN_BYTES,
                "bins, composites and values fit the base-case area");
};

// Histogram of a task's records (item j of thread t is record i = j NT + t,
// keys in [kb, kb + 2^bits), held in registers) on bins fin_bin(key - kb, i,
// ksh, ish), and the values (read again from vs) in input order; the bins
// must be zero.
template <typename K, bool HV, typename CT>
__device__ __forceinline__ void fin_hist(const K (&rk)[Shape<K, HV>::FIN_IT], const K *vs, int n,
                                         int R, K kb, int ksh, int ish, int psh,
                                         unsigned char *region) {
  using S = Shape<K, HV>;
  using A = FinArea<K, HV, CT>;
  unsigned *bins = (unsigned *)region;
  K *vst = (K *)(region + A::V_OFF);
#pragma unroll
  for (int j = 0; j < S::FIN_IT; ++j) {
    const int i = j * NT + threadIdx.x;
    if (j < R && i < n) {
      if constexpr (HV) vst[i] = ld_key<K>(vs + i);
      const unsigned b = fin_bin<K, HV>(key_off<K>(rk[j], kb), i, ksh, ish);
      atomicAdd(&bins[b + (b >> psh)], 1u);
    }
  }
}

// One-pass base case of a task of n <= FIN_CAP records whose keys are held in
// registers (item j of thread t is record i = j NT + t), keys in
// [kb, kb + 2^bits), values in the input-order copy,
// after fin_hist has counted its 2^fb bins (fin_bin with ksh, ish).  Each
// record is the composite c = (key - kb) << FIN_IB | i (without values
// c = key - kb): with values the composites are distinct and their order is
// the order of (key, original index), i.e. the stable order.  The bins'
// counts give their starts; the composites are placed by bin (in arbitrary
// order inside a bin); the thread that owns a run of bins then sorts each of
// its bins that holds more than one record (insertion sort: bins hold about
// half a record on average), and the write-out is a plain coalesced copy of
// the placed order, the value taken from the input-order copy by the
// composite's index.  Returns false, having written nothing to global
// memory, when a bin holds more than FIN_CMAX records.  Barriers: 4 (1 when
// it returns false).
template <typename K, bool HV, typename CT>
__device__ __forceinline__ bool fin_core(const K (&rk)[Shape<K, HV>::FIN_IT], int n,
                                         int R, K kb, int fb, int ksh, int ish,
                                         unsigned char *region,
                                         unsigned *wsum, unsigned *cmax, K *kd, K *vd,
                                         unsigned &bad) {
  using S = Shape<K, HV>;
  using A = FinArea<K, HV, CT>;
  constexpr int IB = HV ? FIN_IB : 0;
  constexpr int PERM = 1 << (A::FBM - 9);
  static_assert(A::FBM >= 9 && NT == 512, "one bin per thread at least");
  unsigned *bins = (unsigned *)region;
  CT *pc = (CT *)(region + A::PC_OFF);
  const K *vst = (const K *)(region + A::V_OFF);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int psh = fb - 9, per = 1 << psh;
  auto comp = [&](K k, int i) -> CT {
    if constexpr (HV) return ((CT)key_off<K>(k, kb) << IB) | (CT)i;
    else return (CT)key_off<K>(k, kb);
  };
  // thread t owns bins [t per, (t+1) per): bin starts = exclusive prefix
  unsigned *mb = bins + threadIdx.x * (per + 1);
  unsigned cnt[PERM];
  unsigned sum = 0, mx = 0, multi = 0;
#pragma unroll
  for (int q = 0; q < PERM; ++q) {
    cnt[q] = q < per ? mb[q] : 0u;
    sum += cnt[q];
    mx = max(mx, cnt[q]);
    multi |= (cnt[q] > 1u ? 1u : 0u) << q;
  }
  unsigned x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 31) wsum[w] = x;
  if (lane == 0) atomicMax(cmax, mx);
  __syncthreads();
  // without values, bins that hold one key value each need no sorting
  const bool presorted = !HV && ksh == 0;
  if (presorted) multi = 0;
  if (!presorted && *cmax > (unsigned)S::FIN_CMAX) return false;
  unsigned run = x - sum + __reduce_add_sync(0xffffffffu, lane < w ? wsum[lane] : 0u);
  const unsigned my0 = run;
#pragma unroll
  for (int q = 0; q < PERM; ++q) {
    if (q < per) mb[q] = run;
    run += cnt[q];
  }
  __syncthreads();
  // placement by bin; the bins then hold their ends
#pragma unroll
  for (int j = 0; j < S::FIN_IT; ++j) {
    const int i = j * NT + threadIdx.x;
    if (j < R && i < n) {
      const unsigned b = fin_bin<K, HV>(key_off<K>(rk[j], kb), i, ksh, ish);
      const unsigned p = atomicAdd(&bins[b + (b >> psh)], 1u);
      if (p < (unsigned)n) pc[p] = comp(rk[j], i);
      else bad = 1u + p;
    }
  }
  __syncthreads();
  // sort the own bins that hold more than one record
  while (multi) {
    const int q = __ffs(multi) - 1;
    multi &= multi - 1u;
    const unsigned s = q ? mb[q - 1] : my0;
    const unsigned e = mb[q];
    if (e > (unsigned)n || s >= e) {
      bad = 1u + e;
      continue;
    }
    const unsigned m = e - s;
    if (m == 2) {  // most multi-record bins: loads together, one exchange
      const CT v0 = pc[s], v1 = pc[s + 1];
      if (v1 < v0) {
        pc[s] = v1;
        pc[s + 1] = v0;
      }
    } else if (m == 3) {  // a three-exchange network
      CT v0 = pc[s], v1 = pc[s + 1], v2 = pc[s + 2];
      CT t;
      if (v1 < v0) { t = v0; v0 = v1; v1 = t; }
      if (v2 < v1) { t = v1; v1 = v2; v2 = t; }
      if (v1 < v0) { t = v0; v0 = v1; v1 = t; }
      pc[s] = v0;
      pc[s + 1] = v1;
      pc[s + 2] = v2;
    } else {
      for (unsigned a = s + 1; a < e; ++a) {
        const CT v = pc[a];
        unsigned b = a;
        while (b > s) {
          const CT u = pc[b - 1];
          if (u <= v) break;
          pc[b] = u;
          --b;
        }
        pc[b] = v;
      }
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += NT) {
    const CT c = pc[p];
    kd[p] = kb + (K)(c >> IB);
    if constexpr (HV) vd[p] = vst[(unsigned)c & ((1u << IB) - 1u)];
  }
  return true;
}

// n elements s -> d by the CTA, CB per thread at a time with all their loads
// issued before the stores.  (16-byte vectors cost the base case's kernel
// spills through the call.)
template <typename K>
__device__ __forceinline__ void copy_elems(const K *s, K *d, int64_t n) {
  constexpr int CB = 8;
  for (int64_t b = threadIdx.x; b < n; b += (int64_t)CB * NT) {
    K r[CB];
#pragma unroll
    for (int q = 0; q < CB; ++q)
      if (b + (int64_t)q * NT < n) r[q] = ld_key<K>(s + b + (int64_t)q * NT);
#pragma unroll
    for (int q = 0; q < CB; ++q)
      if (b + (int64_t)q * NT < n) d[b + (int64_t)q * NT] = r[q];
  }
}

// A plain copy of n records by the CTA (keys, then values).  Not inlined: its
// registers do not add to the base case's.
template <typename K, bool HV>
__device__ __noinline__ void copy_run(const K *ks, K *kd, const K *vs, K *vd, int64_t n) {
  copy_elems<K>(ks, kd, n);
  if constexpr (HV) copy_elems<K>(vs, vd, n);
}

template <typename K, bool HV>
__device__ void phase_finish(const Params &P, int level, unsigned char *smem) {
  using S = Shape<K, HV>;
  Ctl *c = P.ctl;
  const int64_t ntasks = min(ld_cg64(&c->ntasks), (long long)P.tmax);
  Carve cv;
  unsigned char *region = cv.take<unsigned char>(S::FIN_BYTES);
  // LSD passes: two key buffers and (with values) two 16-bit index buffers
  K *lka = (K *)region;
  K *lkb = lka + S::FIN_CAP;
  uint16_t *lia = (uint16_t *)(lkb + S::FIN_CAP);
  uint16_t *lib = lia + S::FIN_CAP;
  uint16_t *wcnt = cv.take<uint16_t>(NWARP * FIN_NB);
  unsigned *dcnt = cv.take<unsigned>(FIN_NB);
  unsigned *doff = cv.take<unsigned>(FIN_NB);
  unsigned *sh = cv.take<unsigned>(NWARP + 1);
  unsigned *wsum = cv.take<unsigned>(NWARP);
  // per-task scalars, two copies: task k uses copy k & 1 while thread 0
  // prepares the other for task k + 1; cmax_sh[2]: the min/max path's own
  long long *task_sh = cv.take<long long>(2);
  Task *tdesc = cv.take<Task>(2);
  K *kmin_sh = cv.take<K>(2);
  K *kmax_sh = cv.take<K>(2);
  unsigned *cmax_sh = cv.take<unsigned>(3);
  int *flag_sh = cv.take<int>(1);
  static_assert(2 * (size_t)S::FIN_LSD_REC * S::FIN_CAP <= (size_t)S::FIN_BYTES,
                "LSD buffers fit");
  static_assert(sizeof(K) * S::FIN_CAP >= 4 * NWARP * FIN_NB, "slots fit in a key buffer");
  static_assert(S::FIN_CAP <= (1 << FIN_IB), "indices fit in FIN_IB bits");
  constexpr int IB = HV ? FIN_IB : 0;
  constexpr bool WIDE = sizeof(K) == 8 || HV;  // 64-bit composites can be needed
  constexpr int FBM32 = FinArea<K, HV, uint32_t>::FBM;
  constexpr int FBM64 = FinArea<K, HV, uint64_t>::FBM;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint16_t *mywc = wcnt + w * FIN_NB;
  long long my_recs = 0, my_tasks = 0, my_copy = 0, my_lsd = 0;
  unsigned bad = 0;  // self-check: a base-case slot out of range, reported once
  // every bin of the widest layout starts at zero for every task (cleared
  // again at the end of each task that used them)
  constexpr int ZFULL = (1 << FBM32) + NT;  // words of the widest bin layout
  auto zero_bins = [&](int words) {
    uint4 *z = (uint4 *)region;
    for (int i = threadIdx.x; i < (words + 3) / 4; i += NT) z[i] = make_uint4(0, 0, 0, 0);
  };
  // Tasks are claimed two ahead by thread 0: q1 = the next task (its id known,
  // its records prefetched into L2 during this one), q2 = the one after (its
  // claim in flight until the end of this task).
  // The descriptors of the current task and the next one are copied into
  // shared memory by thread 0 (asynchronously, no registers), so a task
  // starts without a global load.
  long long q1 = 0, q2 = 0;
  auto fetch_desc = [&](int q, long long t) {
    if (t < ntasks) {
      const char *g = (const char *)&P.tasks[t];
      cp_async16(&tdesc[q], g);
      cp_async16((char *)&tdesc[q] + 16, g + 16);
    }
  };
  auto reset = [&](int q) {
    kmin_sh[q] = (K)~(K)0;
    kmax_sh[q] = (K)0;
    cmax_sh[q] = 0u;
  };
  // thread 0, before the current task's last barrier: publish the next task
  auto advance = [&](int q) {
    task_sh[q] = q1;
    reset(q);
    cp_async_wait_all();  // the next task's descriptor has landed
  };
  auto prefetch_next = [&](int q) {
    const Task &d = tdesc[q];
    if (q1 < ntasks && d.src <= 1 && d.start >= 0 && d.size > 0) {
      const int64_t m = d.size < S::FIN_CAP ? d.size : S::FIN_CAP;
      prefetch_l2<K>((const K *)P.keys[d.src], d.start, m, P.n);
      if constexpr (HV) prefetch_l2<K>((const K *)P.vals[d.src], d.start, m, P.n);
    }
  };
  int par = 0;
  zero_bins(ZFULL);
  if (threadIdx.x == 0) {
    const long long t0 = atomic_add_ll(&c->task_ctr, 1ll);
    task_sh[0] = t0;
    q1 = atomic_add_ll(&c->task_ctr, 1ll);
    reset(0);
    fetch_desc(0, t0);
    cp_async_wait_all();
  }
  __syncthreads();
  while (true) {
    const int64_t ti = task_sh[par];
    if (ti >= ntasks) break;
    if (threadIdx.x == 0) {
      q2 = atomic_add_ll(&c->task_ctr, 1ll);
      fetch_desc(par ^ 1, q1);
    }
    const Task tk = tdesc[par];
    const bool ok = !(tk.src > 1 || tk.dst > 1 || tk.start < 0 || tk.size < 0 ||
                      tk.start + tk.size > P.n ||
                      (tk.kind != TASK_COPY && (tk.size > S::FIN_CAP || tk.hi < 0 || tk.hi > 64)));
    const K *ksrc = (const K *)P.keys[tk.src];
    K *kdst = (K *)P.keys[tk.dst];
    const K *vsrc = HV ? (const K *)P.vals[tk.src] : nullptr;
    K *vdst = HV ? (K *)P.vals[tk.dst] : nullptr;
    if (!ok || tk.kind == TASK_COPY) {
      if (threadIdx.x == 0) {
        advance(par ^ 1);
        if (!ok) check_failed(P, 6, ti, tk.size);
      }
      if (ok) {
        if constexpr (sizeof(K) == 4) {
          copy_run<K, HV>(ksrc + tk.start, kdst + tk.start, HV ? vsrc + tk.start : nullptr,
                          HV ? vdst + tk.start : nullptr, tk.size);
        } else {  // a call here costs the 64-bit base case more spills than it saves
          for (int64_t i = threadIdx.x; i < tk.size; i += NT) {
            kdst[tk.start + i] = ld_key<K>(ksrc + tk.start + i);
            if constexpr (HV) vdst[tk.start + i] = ld_key<K>(vsrc + tk.start + i);
          }
        }
        my_copy += tk.size;
      }
      __syncthreads();
      if (threadIdx.x == 0) q1 = q2;
      par ^= 1;
      continue;
    }
    const int n = (int)tk.size;
    my_recs += n;
    my_tasks += 1;
    const int R = (n + NT - 1) / NT;  // rounds with live items (same for all threads)
    const K *ks = ksrc + tk.start;
    const K *vs = HV ? vsrc + tk.start : nullptr;
    K *kd = kdst + tk.start;
    K *vd = HV ? vdst + tk.start : nullptr;
    // composites over the task's own key range [base, base + 2^hi) when they
    // fit; the bins are counted right after the records are loaded into
    // registers (item j of thread t is record j * NT + t)
    const int hi = tk.hi;
    const int ct = hi + IB <= 32 ? 1 : (WIDE && hi + IB <= 64 ? 2 : 0);
    const int fb0 = min(max(bitlen64((uint64_t)(n - 1)) + 1, 9), ct == 2 ? FBM64 : FBM32);
    const int ksh0 = hi > fb0 ? hi - fb0 : 0;
    const int ish0 = HV && fb0 > hi ? fb0 - hi : 0;
    const int psh0 = fb0 - 9;
    const K kb0 = (K)tk.base;
    unsigned *bins = (unsigned *)region;
    K *vst0 = (K *)(region + (ct == 2 ? FinArea<K, HV, uint64_t>::V_OFF
                                      : FinArea<K, HV, uint32_t>::V_OFF));
    // keys into registers; values copied asynchronously straight into the
    // input-order copy (read from global memory again by the rare paths that
    // need them elsewhere)
    K rk[S::FIN_IT];
#pragma unroll
    for (int j = 0; j < S::FIN_IT; ++j) {
      if (j < R) {
        const int i = j * NT + threadIdx.x;
        if (i < n) {
          rk[j] = ld_key<K>(ks + i);
          if constexpr (HV) {
            if (ct) cp_async_el<K>(vst0 + i, vs + i);
          }
        }
      }
    }
    if (ct) {
#pragma unroll
      for (int j = 0; j < S::FIN_IT; ++j) {
        const int i = j * NT + threadIdx.x;
        if (j < R && i < n) {
          const KOff<K> dk = key_off<K>(rk[j], kb0);
          if (hi < 8 * (int)sizeof(K) && (dk >> hi) != 0) {
            bad = 1u + (unsigned)i;  // a key outside the task's range
          } else {
            const unsigned b = fin_bin<K, HV>(dk, i, ksh0, ish0);
            atomicAdd(&bins[b + (b >> psh0)], 1u);
          }
        }
      }
      if constexpr (HV) cp_async_wait_all();  // the values, before the barrier
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      advance(par ^ 1);
      prefetch_next(par ^ 1);
    }
    bool done = false;
    bool wide = false;  // 64-bit composites: they overlap the widest bin layout
    // words of the bin area this task may leave nonzero (cleared at its end)
    int dirty = ct ? (1 << fb0) + NT : 0;
    if (ct == 1) {
      done = fin_core<K, HV, uint32_t>(rk, n, R, kb0, fb0, ksh0, ish0, region, wsum,
                                       &cmax_sh[par], kd, vd, bad);
    } else if (ct == 2) {
      if constexpr (WIDE)
        done = wide = fin_core<K, HV, uint64_t>(rk, n, R, kb0, fb0, ksh0, ish0, region, wsum,
                                                &cmax_sh[par], kd, vd, bad);
    }
    if (!done) {
      // keys clustered inside the task's range (a bin of more than FIN_CMAX
      // records), or a range too wide: bins over [min, max] of the keys
      K kmn = (K)~(K)0, kmx = (K)0;
#pragma unroll
      for (int j = 0; j < S::FIN_IT; ++j) {
        const int i = j * NT + threadIdx.x;
        if (j < R && i < n) {
          kmn = rk[j] < kmn ? rk[j] : kmn;
          kmx = rk[j] > kmx ? rk[j] : kmx;
        }
      }
      kmn = warp_min(kmn);
      kmx = warp_max(kmx);
      if (lane == 0) {
        if constexpr (sizeof(K) == 4) {
          atomicMin((unsigned *)&kmin_sh[par], (unsigned)kmn);
          atomicMax((unsigned *)&kmax_sh[par], (unsigned)kmx);
        } else {
          atomicMin((unsigned long long *)&kmin_sh[par], (unsigned long long)kmn);
          atomicMax((unsigned long long *)&kmax_sh[par], (unsigned long long)kmx);
        }
      }
      if (threadIdx.x == 0) cmax_sh[2] = 0u;
      zero_bins(ZFULL);
      dirty = ZFULL;
      __syncthreads();
      const K kmin = kmin_sh[par];
      const uint64_t span = (uint64_t)kmax_sh[par] - (uint64_t)kmin;
      if (span == 0) {  // one key: the stable order is the input order
#pragma unroll
        for (int j = 0; j < S::FIN_IT; ++j) {
          const int i = j * NT + threadIdx.x;
          if (j < R && i < n) {
            kd[i] = rk[j];
            if constexpr (HV) vd[i] = ld_key<K>(vs + i);
          }
        }
        done = true;
      } else {
        const int bl = bitlen64(span);
        const int ct1 = bl + IB <= 32 ? 1 : (WIDE && bl + IB <= 64 ? 2 : 0);
        const int fb1 = min(max(bitlen64((uint64_t)(n - 1)) + 1, 9), ct1 == 2 ? FBM64 : FBM32);
        const int ksh1 = bl > fb1 ? bl - fb1 : 0;
        const int ish1 = HV && fb1 > bl ? fb1 - bl : 0;
        if (ct1 == 1) {
          fin_hist<K, HV, uint32_t>(rk, vs, n, R, kmin, ksh1, ish1, fb1 - 9, region);
          __syncthreads();
          done = fin_core<K, HV, uint32_t>(rk, n, R, kmin, fb1, ksh1, ish1, region, wsum,
                                           &cmax_sh[2], kd, vd, bad);
        } else if (ct1 == 2) {
          if constexpr (WIDE) {
            fin_hist<K, HV, uint64_t>(rk, vs, n, R, kmin, ksh1, ish1, fb1 - 9, region);
            __syncthreads();
            done = wide = fin_core<K, HV, uint64_t>(rk, n, R, kmin, fb1, ksh1, ish1, region,
                                                    wsum, &cmax_sh[2], kd, vd, bad);
          }
        }
      }
    }
    if (!done) {
      // a bin with many equal-prefix keys: stable LSD passes over the task's
      // hi bits on (key, original index), the values gathered at the end
      my_lsd += 1;
      dirty = ZFULL;
#pragma unroll
      for (int j = 0; j < S::FIN_IT; ++j) {
        const int i = j * NT + threadIdx.x;
        if (j < R && i < n) {
          lka[i] = rk[j];
          if constexpr (HV) lia[i] = (uint16_t)i;
        }
      }
      __syncthreads();
      K *kin = lka, *kout = lkb;
      uint16_t *iin = lia, *iout = lib;
      const int passes = (tk.hi + FIN_DIG - 1) / FIN_DIG;
      // every warp ranks R consecutive rounds of 32 items (warp w covers
      // [32 R w, 32 R (w+1)) of the current order), R as small as n allows
      for (int q = 0; q < passes; ++q) {
        const int shift = q * FIN_DIG;
        const int bits = tk.hi - shift < FIN_DIG ? tk.hi - shift : FIN_DIG;
        const unsigned dmask = (1u << bits) - 1u;
        unsigned *fslots = (unsigned *)kout;  // kout is free until the scatter
        {
          uint4 *z = (uint4 *)wcnt;
          for (int i = threadIdx.x; i < NWARP * FIN_NB * 2 / 16; i += NT) z[i] = make_uint4(0, 0, 0, 0);
          uint4 *z2 = (uint4 *)fslots;
          for (int i = threadIdx.x; i < NWARP * FIN_NB * 4 / 16; i += NT) z2[i] = make_uint4(0, 0, 0, 0);
        }
        __syncthreads();
        unsigned *myfs = fslots + w * FIN_NB;
        unsigned dr[S::FIN_IT];
#pragma unroll
        for (int j = 0; j < S::FIN_IT; ++j) {
          const int i = w * 32 * R + j * 32 + lane;
          dr[j] = 0xFFFFFFFFu;
          if (j < R && w * 32 * R + j * 32 < n) {  // warp-uniform
            unsigned d = 1u << FIN_DIG;  // dummy digit
            if (i < n) d = (unsigned)(((uint64_t)kin[i] - tk.base) >> shift) & dmask;
            const unsigned r = warp_rank_slots(d, myfs, mywc);
            dr[j] = (d << 16) | r;
          }
        }
        __syncthreads();
        if (threadIdx.x < (1 << FIN_DIG)) {
          const int d = threadIdx.x;
          unsigned run = 0;
#pragma unroll
          for (int qq = 0; qq < NWARP; ++qq) {
            const unsigned x = wcnt[qq * FIN_NB + d];
            wcnt[qq * FIN_NB + d] = (uint16_t)run;
            run += x;
          }
          dcnt[d] = run;
        }
        if (threadIdx.x == 0) *flag_sh = 0;
        __syncthreads();
        {
          const unsigned v = threadIdx.x < (1 << FIN_DIG) ? dcnt[threadIdx.x] : 0u;
          if (v == (unsigned)n) *flag_sh = 1;  // one digit holds everything
          unsigned tot;
          const unsigned o = block_excl_scan<unsigned>(v, sh, tot);
          if (threadIdx.x < (1 << FIN_DIG)) doff[threadIdx.x] = o;
        }
        __syncthreads();
        if (*flag_sh) continue;  // pass would be the identity
#pragma unroll
        for (int j = 0; j < S::FIN_IT; ++j) {
          const int i = w * 32 * R + j * 32 + lane;
          if (j < R && i < n) {
            const unsigned d = dr[j] >> 16;
            const unsigned pp = doff[d] + wcnt[w * FIN_NB + d] + (dr[j] & 0xFFFFu);
            if (d >= (1u << FIN_DIG) || pp >= (unsigned)n) {
              bad = 1u + pp;
              continue;
            }
            kout[pp] = kin[i];
            if constexpr (HV) iout[pp] = iin[i];
          }
        }
        __syncthreads();
        K *tk_ = kin;
        kin = kout;
        kout = tk_;
        uint16_t *ti_ = iin;
        iin = iout;
        iout = ti_;
      }
      // the values by original index, all read before any is written (a
      // task may sort in place: source and destination the same buffer)
      K vg[S::FIN_IT];
      if constexpr (HV) {
#pragma unroll
        for (int j = 0; j < S::FIN_IT; ++j) {
          const int i = j * NT + threadIdx.x;
          vg[j] = (K)0;
          if (j < R && i < n) {
            const unsigned src = iin[i];
            if (src < (unsigned)n) vg[j] = ld_key<K>(vsrc + tk.start + src);
            else bad = 1u + src;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int j = 0; j < S::FIN_IT; ++j) {
        const int i = j * NT + threadIdx.x;
        if (j < R && i < n) {
          kdst[tk.start + i] = kin[i];
          if constexpr (HV) vdst[tk.start + i] = vg[j];
        }
      }
      __syncthreads();
    }
    // clear the bins for the next task once no thread reads this task's
    // composites where they overlap them
    if (wide) __syncthreads();
    zero_bins(wide ? ZFULL : dirty);
    __syncthreads();
    if (threadIdx.x == 0) q1 = q2;
    par ^= 1;
  }
  if (threadIdx.x == 0) {
    if (my_tasks) atomic_add_ll(&c->st_fin_tasks, my_tasks);
    if (my_recs) atomic_add_ll(&c->st_fin_records, my_recs);
    if (my_copy) atomic_add_ll(&c->st_copy_records, my_copy);
    if (my_lsd) atomic_add_ll(&c->st_fin_lsd_tasks, my_lsd);
  }
  if (bad) check_failed(P, 2, bad - 1u, level);
}

// ------------------------------------------------------------------ merge
// Dovetail merging (Alg. 3): in each zone the sorted light bucket B0 and the
// heavy buckets B1..Bm are interleaved.  Heavy bucket i starts at
// zs + lower_bound(B0, k_i) + sum_{i'<i} |B_i'| (the binary searches of
// Alg. 3); every other position takes the next light record.
template <typename K, bool HV>
__device__ void phase_merge_prep(const Params &P, int level, unsigned char *smem) {
  if (P.merge_generic) return;  // the generic merge needs no heavy-run starts
  Ctl *c = P.ctl;
  const int64_t z0 = min(ld_cg64(&c->lvl_zone[level]), (long long)P.mhmax);
  const int64_t z1 = min(ld_cg64(&c->lvl_zone[level + 1]), (long long)P.mhmax);
  long long *sh = (long long *)dts_smem;
  for (int64_t zi = z0 + blockIdx.x; zi < z1; zi += gridDim.x) {
    const MZone Z = ldcg_obj(&P.zones[zi]);
    if (Z.m < 0 || Z.m > HASH_HW / 2 || Z.obuf > 1 || Z.np > Z.m) {
      if (threadIdx.x == 0) check_failed(P, 8, zi, Z.m);
      continue;
    }
    const int q = threadIdx.x;
    long long sz = 0, lb = 0;
    K key = (K)0;
    if (q < Z.m) {
      key = ld_key<K>((const K *)P.mh_keys + Z.mh + q);
      sz = __ldcg((const long long *)&P.mh_sizes[Z.mh + q]);
    }
    long long tot;
    const long long pre = block_excl_scan<long long>(sz, sh, tot);
    // the light bucket follows the np heavy runs stored before it
    if (q == Z.np) sh[NWARP + 2] = pre;
    __syncthreads();
    const long long lof = Z.np < Z.m ? sh[NWARP + 2] : tot;
    const K *B0 = (const K *)P.keys[Z.obuf ^ 1] + Z.zs + lof;
    if (q < Z.m) {
      int64_t a = 0, b = Z.b0;
      while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (ld_key<K>(B0 + mid) < key) a = mid + 1;
        else b = mid;
      }
      lb = a;
      P.mh_start[Z.mh + q] = Z.zs + lb + pre;
    }
    __syncthreads();
  }
}

// Generic merging, the comparison for Alg. 3: in each zone the sorted light
// bucket A (b0 records after the np heavy runs stored before it) and the
// concatenation B of the heavy buckets (sorted: they are numbered by key; the
// light bucket's b0 records sit between B's first lof and the rest) are
// merged stably by merge path, A first on equal keys, with key comparisons
// only.  A work item of
// MERGE_CHUNK outputs is cut into sub-tiles of MERGE_SUB; the split of every
// sub-tile boundary d (how many of the zone's first d outputs come from A) is
// found by one warp with a 32-ary search; each sub-tile's inputs are staged in
// shared memory, every thread merges MERGE_SUB / NT outputs after a merge-path
// search of its own, and the sub-tile is written out in order.

// First i in [max(0, d - nb), min(d, na)] with B[d - 1 - i] < A[i] (the upper
// end when none): a warp probes 32 evenly spaced candidates per round (the
// predicate is monotone in i).  Every lane returns the split.  B[j] is
// Bp[j], or Bp[j + gap] from j = bsplit on.
template <typename K>
__device__ __forceinline__ int64_t merge_split_warp(const K *A, int64_t na, const K *Bp,
                                                    int64_t bsplit, int64_t gap, int64_t nb,
                                                    int64_t d, int lane) {
  int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t p = lo + (int64_t)lane * step;
    bool before = false;  // A[p] is among the first d outputs
    const int64_t jb = d - 1 - p;
    if (p < hi) before = !(ld_key<K>(Bp + jb + (jb < bsplit ? 0 : gap)) < ld_key<K>(A + p));
    const int cnt = __popc(__ballot_sync(0xffffffffu, before));  // lanes 0..cnt-1
    const int64_t nlo = cnt > 0 ? lo + (int64_t)(cnt - 1) * step + 1 : lo;
    const int64_t pc = lo + (int64_t)cnt * step;
    hi = (cnt < 32 && pc < hi) ? pc : hi;
    lo = nlo;
  }
  return lo;
}

template <typename K, bool HV>
__device__ void phase_merge_generic(const Params &P, int level) {
  constexpr int E = MERGE_SUB / NT;
  constexpr int NSUB = MERGE_CHUNK / MERGE_SUB;
  static_assert(E * NT == MERGE_SUB && NSUB * MERGE_SUB == MERGE_CHUNK && NSUB < NWARP,
                "one warp per sub-tile boundary");
  static_assert(MERGE_SUB <= 65536, "16-bit source indices");
  Ctl *c = P.ctl;
  const int64_t z0 = min(ld_cg64(&c->lvl_zone[level]), (long long)P.mhmax);
  const int64_t z1 = min(ld_cg64(&c->lvl_zone[level + 1]), (long long)P.mhmax);
  const int64_t c0 = (int64_t)__ldcg(&c->lvl_chunk[level]);
  const int64_t c1 = (int64_t)__ldcg(&c->lvl_chunk[level + 1]);
  Carve cv;
  K *sk = cv.take<K>(MERGE_SUB);
  K *sv = cv.take<K>(HV ? MERGE_SUB : 1);
  uint16_t *sidx = cv.take<uint16_t>(MERGE_SUB);
  long long *spl = cv.take<long long>(NSUB + 1);
  MZone *Zs = cv.take<MZone>(1);
  long long *lof_sh = cv.take<long long>(1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long my = 0;
  int64_t curz = -1;
  for (int64_t ch = c0 + blockIdx.x; ch < c1; ch += gridDim.x) {
    int64_t a = z0, b = z1 - 1;
    while (a < b) {
      const int64_t mid = (a + b + 1) >> 1;
      if (__ldcg((const long long *)&P.zones[mid].chunk0) <= ch) a = mid;
      else b = mid - 1;
    }
    if (a != curz) {
      __syncthreads();
      if (threadIdx.x == 0) {
        *Zs = ldcg_obj(&P.zones[a]);
        // records of the heavy runs stored before the light bucket
        long long lof = 0;
        for (int q = 0; q < Zs->np && q < Zs->m; ++q)
          lof += __ldcg((const long long *)&P.mh_sizes[Zs->mh + q]);
        *lof_sh = lof;
      }
      __syncthreads();
      curz = a;
    }
    const MZone Z = *Zs;
    const int64_t lof = *lof_sh;
    const int64_t na = Z.b0, nb = Z.ze - Z.zs - Z.b0;
    const int64_t o0 = Z.zs + (ch - Z.chunk0) * MERGE_CHUNK;
    const int64_t o1 = o0 + MERGE_CHUNK < Z.ze ? o0 + MERGE_CHUNK : Z.ze;
    if (Z.obuf > 1 || na < 0 || nb < 0 || ch < Z.chunk0 || o0 >= o1 || Z.np > Z.m ||
        lof < 0 || lof > nb) {
      if (threadIdx.x == 0) latch(P, ERR_INTERNAL);
      __syncthreads();
      continue;
    }
    const int ib = Z.obuf ^ 1;
    const K *kin = (const K *)P.keys[ib];
    K *kout = (K *)P.keys[Z.obuf];
    const K *vin = HV ? (const K *)P.vals[ib] : nullptr;
    K *vout = HV ? (K *)P.vals[Z.obuf] : nullptr;
    const int ns = (int)((o1 - o0 + MERGE_SUB - 1) / MERGE_SUB);
    if (w <= ns) {
      const int64_t e = o0 + (int64_t)w * MERGE_SUB < o1 ? o0 + (int64_t)w * MERGE_SUB : o1;
      const int64_t sp =
          merge_split_warp<K>(kin + Z.zs + lof, na, kin + Z.zs, lof, na, nb, e - Z.zs, lane);
      if (lane == 0) spl[w] = sp;
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      const int64_t sb = o0 + (int64_t)s * MERGE_SUB;
      const int64_t se = sb + MERGE_SUB < o1 ? sb + MERGE_SUB : o1;
      const int64_t i0 = spl[s], i1 = spl[s + 1];
      const int64_t j0 = (sb - Z.zs) - i0, j1 = (se - Z.zs) - i1;
      const int n2 = (int)(se - sb);
      if (i0 < 0 || i1 < i0 || i1 > na || j0 < 0 || j1 < j0 || j1 > nb) {
        if (threadIdx.x == 0) latch(P, ERR_INTERNAL);
        break;  // block-uniform: the splits are in shared memory
      }
      const int la = (int)(i1 - i0), lb = (int)(j1 - j0);  // la + lb = n2
      for (int q = threadIdx.x; q < n2; q += NT) {
        const int64_t jb = j0 + (q - la);
        const int64_t g = q < la ? Z.zs + lof + i0 + q : Z.zs + jb + (jb < lof ? 0 : Z.b0);
        sk[q] = ld_key<K>(kin + g);
        if constexpr (HV) sv[q] = ld_key<K>(vin + g);
      }
      __syncthreads();
      const int d = threadIdx.x * E;
      if (d < n2) {
        int lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (!(sk[la + d - 1 - mid] < sk[mid])) lo = mid + 1;
          else hi = mid;
        }
        int ia = lo, jb = d - lo;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if (d + r < n2) {
            const bool fromA = ia < la && (jb >= lb || !(sk[la + jb] < sk[ia]));
            sidx[d + r] = (uint16_t)(fromA ? ia++ : la + jb++);
          }
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < n2; q += NT) {
        const int x = sidx[q];
        kout[sb + q] = sk[x];
        if constexpr (HV) vout[sb + q] = sv[x];
      }
      __syncthreads();
    }
    my += o1 - o0;
  }
  if (threadIdx.x == 0 && my) atomic_add_ll(&c->st_merge_records, my);
}

template <typename K, bool HV>
__device__ void phase_merge(const Params &P, int level, unsigned char *smem) {
  if (P.merge_generic) {
    phase_merge_generic<K, HV>(P, level);
    return;
  }
  Ctl *c = P.ctl;
  const int64_t z0 = min(ld_cg64(&c->lvl_zone[level]), (long long)P.mhmax);
  const int64_t z1 = min(ld_cg64(&c->lvl_zone[level + 1]), (long long)P.mhmax);
  const int64_t c0 = (int64_t)__ldcg(&c->lvl_chunk[level]);
  const int64_t c1 = (int64_t)__ldcg(&c->lvl_chunk[level + 1]);
  Carve cv;
  long long *hs = cv.take<long long>(HASH_HW / 2 + 1);
  long long *hz = cv.take<long long>(HASH_HW / 2 + 1);
  long long *hp = cv.take<long long>(HASH_HW / 2 + 1);
  long long *sh = cv.take<long long>(NWARP + 1);
  MZone *Zs = cv.take<MZone>(1);
  long long *lof_sh = cv.take<long long>(1);
  long long my = 0;
  int64_t curz = -1;
  for (int64_t ch = c0 + blockIdx.x; ch < c1; ch += gridDim.x) {
    int64_t a = z0, b = z1 - 1;
    while (a < b) {
      const int64_t mid = (a + b + 1) >> 1;
      if (__ldcg((const long long *)&P.zones[mid].chunk0) <= ch) a = mid;
      else b = mid - 1;
    }
    if (a != curz) {
      __syncthreads();
      if (threadIdx.x == 0) *Zs = ldcg_obj(&P.zones[a]);
      __syncthreads();
      const int q = threadIdx.x;
      long long sz = 0;
      if (Zs->m < 0 || Zs->m > HASH_HW / 2 || Zs->np > Zs->m) {
        if (q == 0) check_failed(P, 8, a, Zs->m);
        __syncthreads();
        if (q == 0) Zs->m = 0;
        __syncthreads();
      }
      if (q < Zs->m) {
        sz = __ldcg((const long long *)&P.mh_sizes[Zs->mh + q]);
        hs[q] = __ldcg((const long long *)&P.mh_start[Zs->mh + q]);
        hz[q] = sz;
      }
      long long tot;
      const long long pre = block_excl_scan<long long>(sz, sh, tot);
      if (q < Zs->m) hp[q] = pre;
      // input offset of the light bucket: the heavy runs stored before it
      if (q == Zs->np) *lof_sh = q < Zs->m ? pre : tot;
      __syncthreads();
      curz = a;
    }
    const MZone &Z = *Zs;
    const int64_t lof = *lof_sh;
    const int ib = Z.obuf ^ 1;
    const K *kin = (const K *)P.keys[ib];
    K *kout = (K *)P.keys[Z.obuf];
    const K *vin = HV ? (const K *)P.vals[ib] : nullptr;
    K *vout = HV ? (K *)P.vals[Z.obuf] : nullptr;
    const int64_t o0 = Z.zs + (ch - Z.chunk0) * MERGE_CHUNK;
    const int64_t o1 = o0 + MERGE_CHUNK < Z.ze ? o0 + MERGE_CHUNK : Z.ze;
    // cnt = heavy buckets starting at or before pp: one binary search for a
    // thread's first position, then (positions rise by NT) a forward walk
    int cnt = 0;
    {
      int lo = 0, hi = Z.m;
      const int64_t p0 = o0 + threadIdx.x;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (hs[mid] <= p0) lo = mid + 1;
        else hi = mid;
      }
      cnt = lo;
    }
    // MB positions per thread at a time: their sources first, then all
    // their loads, then the stores (the loads overlap)
    constexpr int MB = 8;
    for (int64_t pb = o0 + threadIdx.x; pb < o1; pb += (int64_t)MB * NT) {
      int64_t from[MB];
#pragma unroll
      for (int r = 0; r < MB; ++r) {
        const int64_t pp = pb + (int64_t)r * NT;
        from[r] = -1;
        if (pp < o1) {
          while (cnt < Z.m && hs[cnt] <= pp) ++cnt;
          const int i = cnt - 1;
          int64_t f;
          if (i >= 0 && pp < hs[i] + hz[i]) {
            f = Z.zs + (i < Z.np ? 0 : Z.b0) + hp[i] + (pp - hs[i]);
          } else {
            const int64_t before = i >= 0 ? hp[i] + hz[i] : 0;
            f = pp - before + lof;
          }
          if (f >= Z.zs && f < Z.ze) from[r] = f;
          else latch(P, ERR_INTERNAL);
        }
      }
      K kk[MB], vv[HV ? MB : 1];
#pragma unroll
      for (int r = 0; r < MB; ++r) {
        if (from[r] >= 0) {
          kk[r] = ld_key<K>(kin + from[r]);
          if constexpr (HV) vv[r] = ld_key<K>(vin + from[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < MB; ++r) {
        if (from[r] >= 0) {
          const int64_t pp = pb + (int64_t)r * NT;
          kout[pp] = kk[r];
          if constexpr (HV) vout[pp] = vv[r];
        }
      }
    }
    my += o1 - o0;
  }
  if (threadIdx.x == 0 && my) atomic_add_ll(&c->st_merge_records, my);
}

// ------------------------------------------------------------------ kernel
__device__ __forceinline__ void tick(const Params &P, int kind) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long now = gtimer();
    P.ctl->t_phase[kind] += now - P.ctl->t_last;
    P.ctl->t_last = now;
  }
}

// After the last level: record the level count and the merge zones' end.
__device__ __forceinline__ void close_levels(const Params &P, int level) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl *c = P.ctl;
    c->nlevels = level;
    const unsigned long long za = __ldcg(&c->zone_alloc);
    c->lvl_zone[level] = (long long)(za >> 40);
    c->lvl_chunk[level] = za & ((1ull << 40) - 1);
  }
}

__device__ __forceinline__ void write_stats(const Params &P, unsigned long long tbeg) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl *c = P.ctl;
    DevStats *d = P.stats;
    d->levels = c->nlevels;
    d->status = *(volatile int *)&c->error;
    for (int l = 0; l < 16; ++l) {
      d->segments[l] = ld_cg64(&c->st_segments[l]);
      d->records[l] = ld_cg64(&c->st_records[l]);
      d->heavy_keys[l] = ld_cg64(&c->st_heavy_keys[l]);
      d->heavy_records[l] = ld_cg64(&c->st_heavy_records[l]);
      d->overflow_records[l] = ld_cg64(&c->st_overflow[l]);
    }
    d->finisher_tasks = ld_cg64(&c->st_fin_tasks);
    d->finisher_records = ld_cg64(&c->st_fin_records);
    d->copy_records = ld_cg64(&c->st_copy_records);
    d->merge_zones = (int64_t)(__ldcg(&c->zone_alloc) >> 40);
    d->merge_records = ld_cg64(&c->st_merge_records);
    d->learned_fixup_records = ld_cg64(&c->st_fix_records);
    d->learned_fixup_steps = ld_cg64(&c->st_fix_steps);
    const long long nzb = ld_cg64(&c->st_bnz);
    const double bsum = __ldcg(&c->st_bsum), bsq = __ldcg(&c->st_bsq);
    const double mean = nzb > 0 ? bsum / (double)nzb : 0.0;
    const double var = nzb > 0 ? bsq / (double)nzb - mean * mean : 0.0;
    d->learned_cv = mean > 0 ? sqrt(var > 0 ? var : 0.0) / mean : 0.0;
    d->learned_mom = mean > 0 ? (double)ld_cg64(&c->st_bmax) / mean : 0.0;
    d->fin_lsd_tasks = ld_cg64(&c->st_fin_lsd_tasks);
    d->learned_used = learned_level(P, 0) ? 1 : 0;
    d->learned_est[0] = P.lrn_est ? P.lrn_est[0] : 0.0;
    d->learned_est[1] = P.lrn_est ? P.lrn_est[1] : 0.0;
    d->free_zones = ld_cg64(&c->st_free_zones);
    d->check_site = ld_cg64(&c->dbg[0]);
    d->check_values[0] = ld_cg64(&c->dbg[1]);
    d->check_values[1] = ld_cg64(&c->dbg[2]);
    for (int k = 0; k < 7; ++k) d->phase_ms[k] = (double)c->t_phase[k] * 1e-6;
    d->phase_ms[7] = tbeg ? (double)(gtimer() - tbeg) * 1e-6 : 0.0;
  }
}

// The same phases as separate launches (one phase per launch, the level loop
// driven by the host).  A profiling aid: every phase shows up as its own
// kernel launch; the persistent kernel below is the product path.
enum {
  KP_SEED = 0, KP_SETUP, KP_SAMPLE, KP_HIST, KP_MSCAN, KP_SCAN, KP_SCATTER, KP_FINISH,
  KP_CLOSE, KP_MERGE_PREP, KP_MERGE, KP_STATS
};
static_assert(KP_SAMPLE == 2 && KP_SCAN == 5 && KP_SCATTER == 6 && KP_STATS == 11,
              "phase_smem_bytes, phase_threads and phase_min_blocks number the phases so");

// One phase (all phases share one body, so that the persistent kernel and
// the per-phase kernel are compiled alike).
template <typename K, bool HV>
__device__ __forceinline__ void run_phase(const Params &P, int phase, int level) {
  unsigned char *smem = dts_smem;
  switch (phase) {
    case KP_SEED: phase_seed<K, HV>(P); break;
    case KP_SETUP: if (blockIdx.x == 0) phase_setup<K, HV>(P, level, smem); break;
    case KP_SAMPLE: phase_sample<K, HV>(P, level, smem); break;
    case KP_HIST: phase_hist<K, HV>(P, level, smem); break;
    case KP_MSCAN: phase_mscan<K, HV>(P, level, smem); break;
    case KP_SCAN: phase_scan<K, HV>(P, level, smem); break;
    case KP_SCATTER: phase_scatter<K, HV>(P, level, smem); break;
    case KP_FINISH: phase_finish<K, HV>(P, level, smem); break;
    case KP_CLOSE: close_levels(P, level); break;
    case KP_MERGE_PREP: phase_merge_prep<K, HV>(P, level, smem); break;
    case KP_MERGE: phase_merge<K, HV>(P, level, smem); break;
    case KP_STATS: write_stats(P, 0); break;
    default: break;
  }
}

// The level loop as a state machine: (phase, level) -> next (phase, level),
// decided alike by every CTA from the control block after a grid barrier.
// Returns KP_DONE after the last merge.
constexpr int KP_DONE = -1;
__device__ __forceinline__ int next_phase(const Params &P, int phase, int &level,
                                          int mfloor) {
  Ctl *c = P.ctl;
  const bool err = *(volatile int *)&c->err_snap != 0;
  switch (phase) {
    case KP_SEED:
      level = 0;
      return KP_SETUP;
    case KP_SETUP: {
      if (err) return KP_CLOSE;
      const long long nseg = ld_cg64(&c->nseg[level & 1]);
      return nseg > 0 ? KP_SAMPLE : KP_FINISH;
    }
    case KP_SAMPLE: return KP_HIST;
    case KP_HIST: return KP_MSCAN;
    case KP_MSCAN: return err ? KP_CLOSE : KP_SCAN;
    case KP_SCAN: return KP_SCATTER;
    case KP_SCATTER: return KP_FINISH;
    case KP_FINISH: {
      ++level;
      if (level >= MAXLEV || err) return KP_CLOSE;
      return ld_cg64(&c->nseg[level & 1]) == 0 ? KP_CLOSE : KP_SETUP;
    }
    case KP_CLOSE:
    case KP_MERGE: {
      // merges run from the deepest level up to mfloor (the levels above it
      // merge in launches of their own after this kernel); levels without
      // zones are skipped
      int l = phase == KP_CLOSE ? *(volatile int *)&c->nlevels - 1 : level - 1;
      while (l >= mfloor && ld_cg64(&c->lvl_zone[l + 1]) == ld_cg64(&c->lvl_zone[l])) --l;
      if (l < mfloor || err) return KP_DONE;
      level = l;
      return KP_MERGE_PREP;
    }
    case KP_MERGE_PREP: return KP_MERGE;
    default: return KP_DONE;
  }
}

// Which phase-time bucket of the stats a phase's time goes to.
__device__ __forceinline__ int phase_kind(int phase) {
  switch (phase) {
    case KP_SAMPLE: return PH_SAMPLE;
    case KP_HIST: return PH_HIST;
    case KP_MSCAN:
    case KP_SCAN: return PH_SCAN;
    case KP_SCATTER: return PH_SCATTER;
    case KP_FINISH: return PH_FINISH;
    case KP_MERGE_PREP:
    case KP_MERGE: return PH_MERGE;
    default: return PH_SETUP;
  }
}

// The persistent kernel.  lev0 = 0: the whole sort from the seed phase.
// lev0 > 0: the first lev0 levels are queued as separate phase launches;
// start at the first level they did not finish (or close if nothing is left)
// and merge only the levels from lev0 down: the queued levels' merges and the
// statistics are launches of their own after this kernel.
template <typename K, bool HV>
__global__ void __launch_bounds__(NT, 2) dtsort_kernel(const __grid_constant__ Params P,
                                                       int lev0) {
  // (phase, level) live in shared memory between phases, so that no register
  // is held across them
  __shared__ int st_phase, st_level;
  Ctl *c = P.ctl;
  if (threadIdx.x == 0) {
    if (lev0 == 0) {
      st_phase = KP_SEED;
      st_level = 0;
      if (blockIdx.x == 0) c->t_last = c->t_begin = gtimer();
    } else {
      const int l = *(volatile int *)&c->levels_done;
      st_level = l;
      st_phase = (*(volatile int *)&c->error || (l > 0 && ld_cg64(&c->nseg[l & 1]) == 0))
                     ? KP_CLOSE : KP_SETUP;
      if (blockIdx.x == 0) tick(P, PH_FINISH);
    }
  }
  __syncthreads();
  while (true) {
    const int phase = *(volatile int *)&st_phase;
    int level = *(volatile int *)&st_level;
    if (phase == KP_DONE) break;
    run_phase<K, HV>(P, phase, level);
    grid_sync(P);
    tick(P, phase_kind(phase));
    const int next = next_phase(P, phase, level, lev0);
    if (threadIdx.x == 0) {
      *(volatile int *)&st_phase = next;
      *(volatile int *)&st_level = level;
    }
    __syncthreads();
  }
  // after queued levels, their merges and the statistics follow as launches
  // of their own
  if (lev0 == 0) write_stats(P, c->t_begin);
}

// One phase per launch.  guard = 1 (launches queued without the host reading
// the control block): a phase of a level that has no subproblems, or any
// phase after an error, returns at once; the base case of a level records
// that the level is done.  prev_kind >= 0: the phase-time bucket the time
// since the previous launch's start goes to.
template <typename K, bool HV>
__global__ void __launch_bounds__(NT, 2) dtsort_phase_kernel(const __grid_constant__ Params P,
                                                             int phase, int level, int guard,
                                                             int prev_kind) {
  Ctl *c = P.ctl;
  if (guard) {
    if (*(volatile int *)&c->error) return;
    if (phase >= KP_SETUP && phase <= KP_FINISH && level > 0 &&
        ld_cg64(&c->nseg[level & 1]) == 0)
      return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (phase == KP_SEED) c->t_last = c->t_begin = gtimer();
    else if (prev_kind >= 0) tick(P, prev_kind);
  }
  run_phase<K, HV>(P, phase, level);
  if (guard && phase == KP_FINISH && blockIdx.x == 0 && threadIdx.x == 0)
    c->levels_done = level + 1;
}

// One phase of a queued level as its own kernel, so that each phase gets a
// register allocation of its own (the same phases inside one kernel share
// one, and a change to one phase moved the others').  Launched without the
// host reading the control block: a phase of a level without subproblems,
// or any phase after an error, returns at once; the base case of a level
// records that the level is done.  prev_kind >= 0: the phase-time bucket the
// time since the previous launch's start goes to.
template <typename K, bool HV, int PH>
__global__ void __launch_bounds__(phase_threads(PH), phase_min_blocks(PH))
    dtsort_phase_one(const __grid_constant__ Params P, int level, int prev_kind) {
  Ctl *c = P.ctl;
  if (PH == KP_STATS) {  // after an error too: the status goes out with them
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (prev_kind >= 0) tick(P, prev_kind);
      write_stats(P, c->t_begin);
    }
    return;
  }
  if (*(volatile int *)&c->error) return;
  if (PH >= KP_SETUP && PH <= KP_FINISH && level > 0 && ld_cg64(&c->nseg[level & 1]) == 0)
    return;
  // a queued merge of a level without zones (or not reached) returns at once
  if ((PH == KP_MERGE_PREP || PH == KP_MERGE) &&
      (level >= *(volatile int *)&c->nlevels ||
       ld_cg64(&c->lvl_zone[level + 1]) == ld_cg64(&c->lvl_zone[level])))
    return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (PH == KP_SEED) c->t_last = c->t_begin = gtimer();
    else if (prev_kind >= 0) tick(P, prev_kind);
  }
  unsigned char *smem = dts_smem;
  if constexpr (PH == KP_SEED) phase_seed<K, HV>(P);
  else if constexpr (PH == KP_SETUP) {
    if (blockIdx.x == 0) phase_setup<K, HV>(P, level, smem);
  } else if constexpr (PH == KP_SAMPLE) phase_sample<K, HV>(P, level, smem);
  else if constexpr (PH == KP_HIST) phase_hist<K, HV>(P, level, smem);
  else if constexpr (PH == KP_MSCAN) phase_mscan<K, HV>(P, level, smem);
  else if constexpr (PH == KP_SCAN) phase_scan<K, HV>(P, level, smem);
  else if constexpr (PH == KP_SCATTER) phase_scatter<K, HV, SCATTER_NT>(P, level, smem);
  else if constexpr (PH == KP_MERGE_PREP) phase_merge_prep<K, HV>(P, level, smem);
  else if constexpr (PH == KP_MERGE) phase_merge<K, HV>(P, level, smem);
  else if constexpr (PH == KP_FINISH) {
    phase_finish<K, HV>(P, level, smem);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->levels_done = level + 1;
      // a level without children ends the recursion: clear its own list too,
      // so that a queued level two further down (same list parity) finds no
      // subproblems instead of this level's (no phase of this level reads
      // the list any more)
      if (ld_cg64(&c->nseg[(level + 1) & 1]) == 0) c->nseg[level & 1] = 0;
    }
  }
}

// ---------------------------------------------------- sampler diagnostic
// Alg. 2 step 1 on one subproblem, exactly as phase_sample draws it.
template <typename K>
__global__ void __launch_bounds__(NT) sample_debug_kernel(const K *keys, int64_t start,
                                                          int64_t size, int hi, uint64_t seed,
                                                          int64_t m, int64_t L, uint64_t *heavy_out,
                                                          int64_t *nheavy_out, uint64_t *max_out) {
  Carve cv;
  K *Ssm = cv.take<K>(SMAX);
  long long *sh = cv.take<long long>(NWARP + 1);
  int M = 1;
  while (M < m) M <<= 1;
  const uint64_t st =
      seed ^ (uint64_t)start ^ ((uint64_t)size * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)hi << 57);
  for (int k = threadIdx.x; k < M; k += NT) {
    if (k < m) {
      const int64_t pos = start + (int64_t)(sm64_at(st, (uint64_t)k) % (uint64_t)size);
      Ssm[k] = ld_key<K>(keys + pos);
    } else {
      Ssm[k] = (K)~(K)0;
    }
  }
  __syncthreads();
  for (int kk = 2; kk <= M; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < M; i += NT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const K a = Ssm[i], b = Ssm[ixj];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) {
            Ssm[i] = b;
            Ssm[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const int64_t nsub = m / L;
  long long carry = 0;
  for (int64_t base = 0; base < nsub; base += NT) {
    const int64_t j = base + threadIdx.x;
    int first = 0;
    K a = 0;
    if (j + 1 < nsub) {
      a = Ssm[(j + 1) * L - 1];
      const K b = Ssm[(j + 2) * L - 1];
      first = (a == b) && (j == 0 || Ssm[j * L - 1] != a);
    }
    long long tot;
    const long long o = block_excl_scan<long long>(first, sh, tot) + carry;
    if (first) heavy_out[o] = (uint64_t)a;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    *nheavy_out = carry;
    *max_out = (uint64_t)Ssm[m - 1];
  }
}

}  // namespace dts
