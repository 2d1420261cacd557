// Device side of dtsort: the stable MSD distribution of DovetailSort (Alg. 2)
// for sm_103a, organised as phases of one persistent cooperative kernel.
//
// One level of the recursion (all subproblems of that level together):
//   setup    (1 CTA)   digit width per subproblem, arena reservations, tiles
//   sample   (CTA/sub) Alg. 2 step 1: sample, sort on chip, heavy keys, the
//                      bucket numbering (light table L, heavy hash table H)
//   hist     (all)     per-block bucket counts (rows of the count matrix)
//   mscan    (all)     column scan of the count matrix, decoupled look-back
//   scan     (CTA/sub) bucket starts; children for the next level, on-chip
//                      base-case tasks, dovetail-merge zones (Alg. 2 step 3)
//   scatter  (all)     Alg. 2 step 2: stable counting sort by bucket id;
//                      per-tile warp ranking, staged bucket-ordered write-out
//   finish   (all)     base case on chip (one counting pass over unique
//                      (key, index) composites; stable LSD passes as the
//                      fallback) and plain copies
// After the last level, the dovetail merges (Alg. 3 semantics) run from the
// deepest level up.  Every spin-wait is bounded by %globaltimer and latches
// DTSORT_ERR_DEVICE_TIMEOUT instead of hanging.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dts {

constexpr int NT = 512;                       // threads per CTA, every phase
constexpr int NWARP = NT / 32;
constexpr int GAMMA_HW = 9;                   // widest digit of one level
constexpr int HEAVY_HW = 128;                 // heavy keys kept per subproblem
constexpr int HEAVY_MIN_SHARE = 250;          // default: 1/4 of the sample
constexpr int NB_HW = (1 << GAMMA_HW) + HEAVY_HW + 1;  // 641
constexpr int NB_PAD = 648;                   // NB_HW + dummy bucket, padded
constexpr int NB_PAIR = NB_PAD / 2;           // 16-bit warp counters, two per word
constexpr int LRN_TAB_N = 512;                // learned prediction table cells
constexpr int SMAX = 8192;                    // largest on-chip sample
constexpr int HASH_HW = 1 << GAMMA_HW;        // hash slots: 4 per heavy key (<= 128)
constexpr int MAXLEV = 136;                   // > 2 * 64 + slack
constexpr int64_t COPY_CHUNK = 1 << 16;       // records per plain-copy task
constexpr int MERGE_CHUNK = 8192;             // output records per merge item
constexpr int MERGE_SUB = 2048;               // generic merge: outputs staged at a time
constexpr int FIN_DIG = 8;                    // base-case digit bits
constexpr int FIN_NB = (1 << FIN_DIG) + 8;    // 256 digits + dummy, padded
constexpr int FIN_IB = 13;                    // index bits of a base-case composite
constexpr uint16_t HEMPTY = 0xFFFF;

enum { ERR_INVALID = 1, ERR_TIMEOUT = 4, ERR_INTERNAL = 6 };
enum { TASK_SORT = 0, TASK_COPY = 1 };
enum { PH_SETUP = 0, PH_SAMPLE, PH_HIST, PH_SCAN, PH_SCATTER, PH_FINISH, PH_MERGE,
       PH_TOTAL };

// A subproblem: records [start, start+size) whose keys all lie in
// [base, base + 2^hi); its digits are taken from key - base.  (Below a digit
// zone base only fixes the shared high bits; below a learned zone it is the
// zone's lower boundary.)
struct Seg {
  int64_t start, size;
  int64_t ntotal;   // length of the array it came from (n of Alg. 2)
  uint64_t base;    // lower bound of the keys
  int32_t hi;       // bits of key - base still unsorted
  uint8_t res;      // buffer (0 = caller's, 1 = workspace) the result goes to
  uint8_t pad[3];
};

// Per subproblem of the current level, filled by setup + sample.  The
// subproblem is cut into blocks of BLK records (rows of its count matrix) and
// the rows into look-back chunks of CH rows.
struct SegInfo {
  int32_t gamma;    // planned digit width
  int32_t lo, t;    // MSD zone digit = key bits [lo, t)
  int32_t nheavy;
  int32_t nb;       // 2^(t-lo) + nheavy + 1 (overflow last)
  int32_t hbits;    // log2 hash capacity (0: no heavy keys)
  int64_t nblk, blk0;  // blocks, first global block index
  int64_t nchk, chk0;  // chunks, first global chunk index
  int64_t boff;     // bucket arrays (totals / starts)
  int64_t hoff;     // heavy keys, sorted
  int64_t zoff;     // light table L: 2^(t-lo)+1 entries
  int64_t hashoff;  // heavy hash table H
  int64_t coff;     // count matrix, u32, nblk x nb (becomes block offsets)
  int64_t soff;     // chunk look-back status words, nchk x nb
  int64_t mhoff;    // persistent heavy store reservation (for merges)
  int32_t learned;  // zones are the learned boundaries (level 0 only)
  int32_t pad_;
};

struct Task {
  int64_t start, size;
  uint64_t base;    // the records' keys lie in [base, base + 2^hi)
  int32_t hi;
  uint8_t src, dst, kind, pad;
};
static_assert(sizeof(Task) == 32, "a task descriptor is two 16-byte copies");

// An MSD zone with heavy buckets, merged after its light bucket is sorted.
struct MZone {
  int64_t zs, b0, ze;   // zone [zs, ze); light bucket of b0 records
  int64_t mh;           // its heavy keys / sizes / final starts in the store
  int64_t chunk0;       // first merge work item
  int32_t m;            // heavy buckets
  uint8_t obuf;         // output buffer; inputs are in the other one
  uint8_t np;           // heavy runs stored before the light bucket (the
                        // rest after it): the input is [np heavy runs]
                        // [light bucket][m - np heavy runs]
  uint8_t pad[2];
};

struct Ctl {
  unsigned bar_count, bar_gen;
  int error, nlevels;
  int err_snap;   // error as of the last grid barrier: every CTA decides alike
  int pad_;
  long long nseg[2];
  long long chunk_ctr, nblocks, nchunks;
  long long ntasks, task_ctr;
  unsigned long long zone_alloc;  // (zones << 40) | chunks
  long long mh_alloc;
  long long merge_ctr;
  long long lvl_zone[MAXLEV + 1];
  unsigned long long lvl_chunk[MAXLEV + 1];
  long long st_segments[16], st_records[16], st_heavy_keys[16],
      st_heavy_records[16], st_overflow[16];
  long long st_fin_lsd_tasks;
  long long st_fin_tasks, st_fin_records, st_copy_records, st_merge_zones,
      st_merge_records, st_fix_records, st_fix_steps, st_free_zones;
  // first failed self-check: site, level, and two values
  long long dbg[4];
  // level-0 light bucket sizes of the first subproblem (imbalance statistics)
  double st_bsum, st_bsq;
  long long st_bmax, st_bnz;
  unsigned long long t_phase[8];
  unsigned long long t_last, t_begin;
  int levels_done;  // levels whose base case ran as a separate launch
  int pad2_;
};

// Statistics as the host reads them (mirrors the public struct's prefix).
struct DevStats {
  int32_t levels, status;
  int64_t segments[16], records[16], heavy_keys[16], heavy_records[16],
      overflow_records[16];
  int64_t finisher_tasks, finisher_records, copy_records, merge_zones,
      merge_records, learned_fixup_records, learned_fixup_steps;
  double learned_cv, learned_mom;
  double phase_ms[8];
  int64_t check_site, check_values[2];
  int64_t fin_lsd_tasks;
  int64_t learned_used;
  double learned_est[2];
  int64_t free_zones;
};

struct Params {
  void *keys[2];          // [0] caller's arrays, [1] workspace ping-pong copy
  void *vals[2];          // NULL for key-only
  int64_t n;
  const int64_t *offsets; // segmented input (NULL: one array [0, n))
  int64_t nsegs_in;
  int32_t key_bits;
  int32_t gamma_max;
  int32_t cap;            // largest base-case bucket
  int32_t heavy_on;
  int32_t heavy_min_share;  // thousandths of a subproblem's sample its heavy
                            // keys must hold to be kept (0: any)
  int32_t merge_generic;  // 1: merge-path merge of each zone instead of Alg. 3
  int64_t target;         // desired bucket size after distribution
  uint64_t seed;
  int32_t sample_factor;  // samples = 2^gamma * L * factor (capped)
  int32_t debug_fault;    // 1: chunk 1 of level 0 never publishes (tests)
  int32_t blk_tiles;      // tiles per count-matrix row (block = blk_tiles * TILE)
  int32_t lrn_B;          // learned zones at level 0 (0: digit zones)
  const void *lrn_spl;    // lrn_B zone lower bounds (key type), spl[0] = 0
  const float *lrn_tab;   // LRN_TAB_N + 1 predicted CDF values on the feature grid
  const int *lrn_on;      // NULL, or the device's decision (1: use the learned zones)
  const double *lrn_est;  // NULL, or the decision's two cost estimates
  unsigned long long wait_ns;  // bound of every spin-wait
  Ctl *ctl;
  Seg *segs[2];
  SegInfo *info;
  int64_t *bcount, *bstart;
  int32_t *lid;
  void *heavy;
  void *hash_keys;
  uint16_t *hash_ids;
  unsigned *cmat;
  unsigned long long *status;
  Task *tasks;
  MZone *zones;
  void *mh_keys;
  int64_t *mh_sizes, *mh_start;
  int64_t maxseg, bmax, hmax, zmax, hashmax, cwords, swords, tmax, mhmax;
  int *dev_status;
  DevStats *stats;
};

// The dynamic shared memory of every kernel here.  Phases take their arrays
// from it by pointer arithmetic only, so the compiler keeps them in the
// shared address space (32-bit addresses, LDS/STS) instead of generic space.
extern __shared__ __align__(16) unsigned char dts_smem[];

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ long long ld_cg64(const long long *p) {
  return (long long)__ldcg((const unsigned long long *)p);
}

// Loads a table entry written in an earlier phase by another SM: through L2
// only, so that no stale L1 line is ever used.
template <typename T>
__device__ __forceinline__ T ldcg_obj(const T *p) {
  static_assert(sizeof(T) % 8 == 0, "8-byte granular");
  T r;
  const unsigned long long *s = (const unsigned long long *)p;
  unsigned long long *d = (unsigned long long *)&r;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 8); ++i) d[i] = __ldcg(s + i);
  return r;
}

__device__ __forceinline__ long long atomic_add_ll(long long *p, long long v) {
  return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

__device__ __forceinline__ void latch(const Params &P, int code) {
  atomicCAS(&P.ctl->error, 0, code);
  atomicCAS(P.dev_status, 0, code);
}

// A failed self-check: latch ERR_INTERNAL and record where (first one wins).
static __device__ __noinline__ void check_failed(const Params &P, int site, long long a, long long b) {
  if (atomicCAS((unsigned long long *)&P.ctl->dbg[0], 0ull, (unsigned long long)site) == 0ull) {
    P.ctl->dbg[1] = a;
    P.ctl->dbg[2] = b;
  }
  latch(P, ERR_INTERNAL);
}

__device__ __forceinline__ uint64_t sm64_fmix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Output i of the SplitMix64 sequence started from state s.
__device__ __forceinline__ uint64_t sm64_at(uint64_t s, uint64_t i) {
  return sm64_fmix(s + (i + 1) * 0x9E3779B97F4A7C15ull);
}

__device__ __forceinline__ uint64_t lowmask(int bits) {
  return bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
}

__device__ __forceinline__ int bitlen64(uint64_t x) { return x ? 64 - __clzll((long long)x) : 0; }

template <typename K>
__device__ __forceinline__ K ld_key(const K *p) {
  if constexpr (sizeof(K) == 4) return (K)__ldcg((const unsigned int *)p);
  else return (K)__ldcg((const unsigned long long *)p);
}

// L2 eviction policy (createpolicy) for stores that carry a cache hint.  The
// scatter writes each bucket's run a little per tile; its stores are kept
// (evict last) so that a 32-byte sector left partly written by one tile is
// more often still in L2 when the next tile completes it (evicted partly
// written, it costs a read-modify-write of the sector in DRAM).  Measured on
// 10^9 32-bit key/value pairs: the two scatters 15.5 -> 14.6 ms.  (Loads
// marked evict-first as well lost: 18.8 ms.)
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// A key-sized store with an L2 eviction policy.
template <typename K>
__device__ __forceinline__ void st_key_hint(K *p, K v, uint64_t pol) {
  if constexpr (sizeof(K) == 4)
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"((uint32_t)v), "l"(pol)
                 : "memory");
  else
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"((uint64_t)v), "l"(pol)
                 : "memory");
}

template <typename K>
__device__ __forceinline__ uint32_t hash_slot(K key, int bits) {
  return (uint32_t)(((uint64_t)key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// Grid-wide barrier for a cooperatively launched grid (all CTAs resident).
static __device__ __forceinline__ void grid_sync(const Params &P) {
  __syncthreads();
  if (threadIdx.x == 0) {
    Ctl *c = P.ctl;
    volatile unsigned *gen = &c->bar_gen;
    unsigned g = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      c->bar_count = 0;
      c->err_snap = *(volatile int *)&c->error;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      unsigned long long t0 = gtimer();
      while (*gen == g) {
        __nanosleep(100);
        if (gtimer() - t0 > P.wait_ns + 3000000000ull) {
          latch(P, ERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Exclusive scan of one value per thread over the CTA; sh needs NWARP+1.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *sh, T &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < NWARP ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NWARP) sh[lane] = s;
  }
  __syncthreads();
  T base = w ? sh[w - 1] : T(0);
  total = sh[NWARP - 1];
  __syncthreads();
  return base + x - v;
}

// Level 0 uses learned zones: a model was fitted and (when an estimate was
// made) the estimate chose it.
__device__ __forceinline__ bool learned_level(const Params &P, int level) {
  return level == 0 && P.lrn_B > 0 && (P.lrn_on == nullptr || *(volatile const int *)P.lrn_on);
}

// Digit of a key on the fast path: bits [lo, lo + log2(gmask+1)) of
// key - base (32-bit arithmetic for 32-bit keys).
template <typename K>
__device__ __forceinline__ unsigned fast_digit(K key, uint64_t base, int lo, unsigned gmask) {
  if constexpr (sizeof(K) == 4) return (((uint32_t)key - (uint32_t)base) >> lo) & gmask;
  else return (unsigned)(((uint64_t)key - base) >> lo) & gmask;
}

// Minimum / maximum over the warp (all lanes active).
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
  if constexpr (sizeof(T) == 4) {
    return (T)__reduce_min_sync(0xffffffffu, (unsigned)v);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u < v ? u : v;
    }
    return v;
  }
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  if constexpr (sizeof(T) == 4) {
    return (T)__reduce_max_sync(0xffffffffu, (unsigned)v);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u > v ? u : v;
    }
    return v;
  }
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Stable rank among this warp's earlier items (in (round, lane) order) with
// the same bucket.  Every lane ORs its bit into its bucket's shared-memory
// slot and reads back the set of peers; the lowest peer advances the
// bucket's running count.  Cost does not grow with the number of distinct
// buckets or the width of the bucket id.  slot: this warp's slots (zero on
// entry, zero again on return); wc: this warp's running counts.
__device__ __forceinline__ unsigned warp_rank_slots(unsigned b, unsigned *slot, uint16_t *wc) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned b0 = __shfl_sync(0xffffffffu, b, 0);
  unsigned peers;
  if (__all_sync(0xffffffffu, b == b0)) {
    peers = 0xffffffffu;  // one bucket for the whole warp
  } else {
    atomicOr(&slot[b], 1u << lane);
    __syncwarp();
    peers = slot[b];
    __syncwarp();
  }
  const unsigned leader = __ffs(peers) - 1;
  unsigned old = 0;
  if (lane == leader) {
    old = wc[b];
    wc[b] = (uint16_t)(old + __popc(peers));
    slot[b] = 0;
  }
  __syncwarp();
  old = __shfl_sync(0xffffffffu, old, leader);
  return old + __popc(peers & lanemask_lt());
}

// Half b & 1 of a word holding two 16-bit counts (bucket b's count).
__device__ __forceinline__ unsigned half16(unsigned word, unsigned b) {
  return (word >> ((b & 1u) << 4)) & 0xFFFFu;
}

// Stable rank among this warp's earlier items (in (round, lane) order) with
// the same bucket b.  Every lane ORs its bit into its bucket's slot and reads
// back the set of peers; the lowest peer advances the bucket's running count
// with one shared atomic (the count before this round is shuffled to the
// peers) and clears the slot.  The next round's atomic is issued after this
// one has returned, so the counts of one bucket advance in round order.  A
// round whose lanes all share one bucket skips the slot.  slot: this warp's
// slots (zero on entry, zero again on return); wc2: this warp's running
// counts, 16 bits each, two per word (bucket b in half b & 1 of word b >> 1).
__device__ __forceinline__ unsigned warp_rank(unsigned b, unsigned *slot, unsigned *wc2) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned b0 = __shfl_sync(0xffffffffu, b, 0);
  unsigned peers;
  const bool one = __all_sync(0xffffffffu, b == b0);
  if (one) {
    peers = 0xffffffffu;
  } else {
    atomicOr(&slot[b], 1u << lane);
    __syncwarp();
    peers = slot[b];
  }
  const unsigned leader = __ffs(peers) - 1;
  unsigned old = 0;
  if (lane == leader) {
    const unsigned sh = (b & 1u) << 4;
    old = atomicAdd(&wc2[b >> 1], (unsigned)__popc(peers) << sh) >> sh;
  }
  old = __shfl_sync(0xffffffffu, old, leader) & 0xFFFFu;
  if (!one) {
    if (lane == leader) slot[b] = 0u;
    __syncwarp();
  }
  return old + __popc(peers & lanemask_lt());
}

// 16 bytes global -> shared without registers (cp.async, L2 only); both
// addresses 16-byte aligned.  cp_async_wait_all() waits for this thread's.
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
// One 4- or 8-byte element, global -> shared (both addresses aligned to the
// element's size), asynchronously: no register holds it.
template <typename T>
__device__ __forceinline__ void cp_async_el(T *sdst, const T *gsrc) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Asks L2 to fetch elements [first, first + count) of array a (clipped to
// [0, n)): one bulk prefetch of the 16-byte aligned part of the range.  A
// hint only: nothing waits for it, and it touches no address outside a.
template <typename K>
__device__ __forceinline__ void prefetch_l2(const K *a, int64_t first, int64_t count, int64_t n) {
  int64_t e = first + count;
  if (first < 0) first = 0;
  if (e > n) e = n;
  if (e <= first) return;
  const uintptr_t lo = ((uintptr_t)(a + first) + 15) & ~(uintptr_t)15;
  const uintptr_t hi = (uintptr_t)(a + e) & ~(uintptr_t)15;
  if (hi <= lo) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo))
               : "memory");
}

// Digit width for a subproblem of size s whose keys have hi unsorted bits:
// the fewest levels (of at most gmax bits each) that bring buckets down to
// about `target` records, bits spread evenly over those levels.  When this is
// the last distribution level (the buckets go to the on-chip base case,
// which sorts fin_dig bits per pass), a wider digit is taken if it saves a
// base-case pass.
__device__ __forceinline__ int plan_gamma(int64_t s, int64_t target, int gmax, int hi,
                                          int fin_dig) {
  int e = 0;
  while (e < 62 && (target << e) < s) ++e;
  if (e < 1) e = 1;
  const int nlev = (e + gmax - 1) / gmax;
  int g = (e + nlev - 1) / nlev;
  g = g < 1 ? 1 : (g > gmax ? gmax : g);
  if (nlev == 1 && hi > g) {
    int best = g, bestp = (hi - g + fin_dig - 1) / fin_dig;
    // at most 2 more bits: 2^g < 8 * s / target keeps the tables bounded
    for (int g2 = g + 1; g2 <= gmax && g2 <= hi && g2 <= g + 2; ++g2) {
      const int p2 = (hi - g2 + fin_dig - 1) / fin_dig;
      if (p2 < bestp) {
        best = g2;
        bestp = p2;
      }
    }
    g = best;
  }
  return g;
}

// ----------------------------------------------------- per-segment tables
template <typename K>
struct SegTables {
  SegInfo info;
  int64_t start, size;
  uint64_t base;
  int32_t hi, seg;
  uint8_t res;
};

// Learned zone of a key: the model's distilled CDF (table on the feature
// grid, linear between cells) predicts a zone, which is then moved to the
// exact zone z with spl[z] <= key < spl[z+1] by integer comparisons.
// *steps receives how far the prediction was off.
template <typename K>
__device__ __forceinline__ unsigned learned_zone(K key, const K *spl, const float *tab, int B,
                                                 unsigned *steps) {
  const float x = log2f((float)key + 1.0f) * (1.0f / (8.0f * sizeof(K)));
  float fc = x * (float)LRN_TAB_N;
  int c = (int)fc;
  c = c < 0 ? 0 : (c > LRN_TAB_N - 1 ? LRN_TAB_N - 1 : c);
  const float fr = fc - (float)c;
  const float pz = fmaf(fr, tab[c + 1] - tab[c], tab[c]) * (float)B;
  int z = (int)pz;
  z = z < 0 ? 0 : (z > B - 1 ? B - 1 : z);
  unsigned st = 0;
  while (z > 0 && key < spl[z]) {
    --z;
    ++st;
  }
  while (z < B - 1 && key >= spl[z + 1]) {
    ++z;
    ++st;
  }
  *steps = st;
  return (unsigned)z;
}

// Exact learned zone by binary search over the boundaries (global memory).
template <typename K>
__device__ __forceinline__ unsigned learned_zone_exact(K key, const K *spl, int B) {
  int lo = 0, hi = B - 1;  // largest z with spl[z] <= key
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ld_key<K>(spl + mid) <= key) lo = mid;
    else hi = mid - 1;
  }
  return (unsigned)lo;
}

// What GetBucketId needs of a subproblem, copied into registers once per
// subproblem (the shared-memory tables are read only for the lookups).
struct BucketCtx {
  uint64_t base, hmask;  // key - base, restricted to the unsorted bits
  int lo, t, nb, hbits, learned, B;
};

template <typename K>
__device__ __forceinline__ BucketCtx bucket_ctx(const SegTables<K> &T) {
  BucketCtx x;
  x.base = T.base;
  x.hmask = lowmask(T.hi);
  x.lo = T.info.lo;
  x.t = T.info.t;
  x.nb = T.info.nb;
  x.hbits = T.info.hbits;
  x.learned = T.info.learned;
  x.B = 1 << T.info.gamma;
  return x;
}

// Entry z of a subproblem's light table L (Alg. 2), one 32-bit word: the
// light bucket id of zone z (bits 0-9), the index in the subproblem's sorted
// heavy list of the zone's first heavy key (bits 10-17), the zone's number of
// heavy keys (bits 18-25), and LE_MERGE (bit 30): the zone's runs need the
// dovetail merge.  A zone's buckets are numbered in key order as
// [heavy keys below its light keys][light bucket][the other heavy keys]: the
// zone's first bucket is z + (first heavy index), its light bucket id minus
// that is the number of heavy buckets placed before the light one.
constexpr int LE_HF = 10, LE_MZ = 18;
constexpr int32_t LE_ID = (1 << LE_HF) - 1, LE_MERGE = 1 << 30;
static_assert(NB_HW <= LE_ID + 1 && HEAVY_HW < 256, "light-table fields fit");
__host__ __device__ constexpr int32_t le_pack(int light, int hfirst, int mz, bool merge) {
  return light | (hfirst << LE_HF) | (mz << LE_MZ) | (merge ? LE_MERGE : 0);
}
__device__ __forceinline__ int le_light(int32_t e) { return e & LE_ID; }
__device__ __forceinline__ int le_hfirst(int32_t e) { return (e >> LE_HF) & 255; }
__device__ __forceinline__ int le_mz(int32_t e) { return (e >> LE_MZ) & 255; }

// Heavy id of key in the hash table H (hk/hid), or HEMPTY.
template <typename K>
__device__ __forceinline__ unsigned probe_heavy(const K *hk, const uint16_t *hid, int hbits,
                                                K key) {
  const uint32_t cap1 = (1u << hbits) - 1u;
  uint32_t s = hash_slot<K>(key, hbits);
  while (true) {
    const uint16_t id = hid[s];
    const K k = hk[s];  // both loads of a probe issued together
    if (id == HEMPTY || k == key) return id;
    s = (s + 1) & cap1;
  }
}

// GetBucketId (Alg. 2): overflow past the sampled key range, heavy keys
// through H, light keys through L by their MSD zone (or learned zone).  A
// key is looked up in H only when its zone holds heavy keys and it lies
// between the zone's smallest and largest heavy key (hl: the subproblem's
// heavy keys, sorted); overflow keys are never heavy (heavy keys are sample
// keys, the overflow bucket starts above the largest one).
// lid/hk/hid/hl/spl/tab: the tables in shared memory.  VERIFY (the
// histogram): a light key of a zone with heavy keys that lies outside the
// interval the zone's layout leaves for light keys marks the zone's entry
// LE_MERGE in lid (the zone needs the dovetail merge).
template <typename K>
__device__ __forceinline__ bool light_out_of_place(int32_t e, unsigned z, const K *hl, K key);
template <typename K, bool VERIFY = false>
__device__ __forceinline__ unsigned bucket_of(const BucketCtx &X, const int32_t *lid,
                                              const K *hk, const uint16_t *hid, const K *hl,
                                              K key, const K *spl = nullptr,
                                              const float *tab = nullptr,
                                              unsigned *steps = nullptr) {
  unsigned z;
  if (X.learned) {
    if (X.hbits) {  // the learned lookup is dearer than a probe: probe first
      const unsigned id = probe_heavy<K>(hk, hid, X.hbits, key);
      if (id != HEMPTY) return id;
    }
    unsigned st;
    z = learned_zone<K>(key, spl, tab, X.B, &st);
    if (steps) *steps = st;
    const int32_t e = lid[z];
    if constexpr (VERIFY) {
      if (le_mz(e) && !(e & LE_MERGE) && light_out_of_place<K>(e, z, hl, key))
        atomicOr(const_cast<int32_t *>(lid) + z, LE_MERGE);
    }
    return (unsigned)le_light(e);
  }
  if constexpr (sizeof(K) == 4) {
    const uint32_t m = ((uint32_t)key - (uint32_t)X.base) & (uint32_t)X.hmask;
    if (X.t < 32 && (m >> X.t) != 0) return (unsigned)(X.nb - 1);
    z = m >> X.lo;
  } else {
    const uint64_t m = ((uint64_t)key - X.base) & X.hmask;
    if (X.t < 64 && (m >> X.t) != 0) return (unsigned)(X.nb - 1);
    z = (unsigned)(m >> X.lo);
  }
  const int32_t e = lid[z];
  if (X.hbits) {
    const int mz = le_mz(e);
    if (mz) {
      // above (below) all of the zone's heavy keys: light, and in place
      // unless heavy buckets are stored after (before) the light one
      const int hf = le_hfirst(e);
      const int mp = le_light(e) - (int)z - hf;
      const K hmin = hl[hf], hmax = hl[hf + mz - 1];
      bool out;
      if (hmax < key) {
        out = mp < mz;
      } else if (key < hmin) {
        out = mp > 0;
      } else if (key == hmin) {  // the zone's first heavy key: no probe
        return z + hf + (mp > 0 ? 0 : 1);
      } else if (key == hmax) {  // and its last
        return z + hf + mz - 1 + (mz - 1 < mp ? 0 : 1);
      } else {
        const unsigned id = probe_heavy<K>(hk, hid, X.hbits, key);
        if (id != HEMPTY) return id;
        out = VERIFY && light_out_of_place<K>(e, z, hl, key);
      }
      if constexpr (VERIFY) {
        if (out && !(e & LE_MERGE)) atomicOr(const_cast<int32_t *>(lid) + z, LE_MERGE);
      }
    }
  }
  return (unsigned)le_light(e);
}

// Zone z's light-table entry e (zone with heavy keys, not yet marked for a
// merge) and a light key of it: true when the key lies outside the interval
// the zone's layout leaves for light keys, i.e. the zone needs the merge.
template <typename K>
__device__ __forceinline__ bool light_out_of_place(int32_t e, unsigned z, const K *hl, K key) {
  const int hf = le_hfirst(e), mz = le_mz(e);
  const int mp = le_light(e) - (int)z - hf;  // heavy buckets before the light one
  return (mp > 0 && key < hl[hf + mp - 1]) || (mp < mz && hl[hf + mp] < key);
}

template <typename K>
__device__ __forceinline__ void load_tables(const Params &P, int seg, int level, SegTables<K> &T,
                                            int32_t *lid_s, K *hk_s, uint16_t *hid_s, K *hl_s,
                                            K *spl_s = nullptr, float *tab_s = nullptr) {
  // all threads call; T lives in shared memory
  if (threadIdx.x == 0) {
    const Seg S = ldcg_obj(&P.segs[level & 1][seg]);
    T.info = ldcg_obj(&P.info[seg]);
    T.start = S.start;
    T.size = S.size;
    T.base = S.base;
    T.hi = S.hi;
    T.res = S.res;
    T.seg = seg;
    // self-check of the subproblem's tables; a bad one is recorded and
    // turned into an empty subproblem so that nothing is indexed with it
    const SegInfo &I = T.info;
    const int zb = I.learned ? I.gamma : I.t - I.lo;
    if (S.start < 0 || S.size < 0 || S.start + S.size > P.n || zb < 0 || zb > GAMMA_HW ||
        I.nb < 1 || I.nb > NB_HW || I.hbits < 0 || I.hbits > GAMMA_HW ||
        (I.learned && P.lrn_B > (1 << GAMMA_HW))) {
      check_failed(P, 5, seg, (long long)I.nb * 65536 + zb * 256 + I.hbits);
      T.size = 0;
      T.info.nb = 0;
      T.info.t = T.info.lo = 0;
      T.info.hbits = 0;
      T.info.learned = 0;
      T.info.zoff = 0;
    }
  }
  __syncthreads();
  const int nz = (T.info.learned ? (1 << T.info.gamma) : (1 << (T.info.t - T.info.lo))) + 1;
  for (int i = threadIdx.x; i < nz; i += (int)blockDim.x) {
    int32_t e = __ldcg(P.lid + T.info.zoff + i);
    // self-check: the entry's bucket and heavy-list range lie in the tables
    if (e < 0 || le_light(e) >= T.info.nb || le_hfirst(e) + le_mz(e) > T.info.nheavy ||
        (le_mz(e) && !T.info.hbits)) {
      check_failed(P, 9, seg, (long long)e);
      e = 0;
    }
    lid_s[i] = e;
  }
  if (T.info.learned && spl_s) {
    const K *spl = (const K *)P.lrn_spl;
    for (int i = threadIdx.x; i < P.lrn_B; i += (int)blockDim.x) spl_s[i] = ld_key<K>(spl + i);
    for (int i = threadIdx.x; i <= LRN_TAB_N; i += (int)blockDim.x) tab_s[i] = __ldcg(P.lrn_tab + i);
  }
  if (T.info.hbits) {
    const int cap = 1 << T.info.hbits;
    const K *hk = (const K *)P.hash_keys + T.info.hashoff;
    for (int i = threadIdx.x; i < cap; i += (int)blockDim.x) {
      hk_s[i] = ld_key<K>(hk + i);
      hid_s[i] = __ldcg(P.hash_ids + T.info.hashoff + i);
    }
    const int nh = T.info.nheavy < HEAVY_HW ? T.info.nheavy : HEAVY_HW;
    for (int i = threadIdx.x; i < nh; i += (int)blockDim.x)
      hl_s[i] = ld_key<K>((const K *)P.heavy + T.info.hoff + i);
  }
  __syncthreads();
}

// index of the subproblem owning global block r (blk0 increasing)
__device__ __forceinline__ int find_blk_seg(const Params &P, int64_t nseg, int64_t r) {
  int64_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldcg((const long long *)&P.info[mid].blk0) <= r) lo = mid;
    else hi = mid - 1;
  }
  return (int)lo;
}

// index of the subproblem owning global look-back chunk c (chk0 increasing)
__device__ __forceinline__ int find_chk_seg(const Params &P, int64_t nseg, int64_t c) {
  int64_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldcg((const long long *)&P.info[mid].chk0) <= c) lo = mid;
    else hi = mid - 1;
  }
  return (int)lo;
}

}  // namespace dts
