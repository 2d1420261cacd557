/*
 * Seeded synthetic inputs for the stable integer sort (shared by the oracle
 * side and the CUDA side; holds none of the sort's arithmetic).
 *
 * Every value is a pure function of (seed, stream, record index), drawn from
 * a counter-based SplitMix64 stream (Steele, Lea, Flood 2014), so the bytes
 * do not depend on the thread count.  Distribution families follow the
 * paper's synthetic inputs (Sec. 6, "Synthetic Distributions") in the shapes
 * the benchmark configurations state:
 *
 *   GEN_UNIFORM      uniform over the full key range
 *   GEN_ZIPF         Zipf(s) ranks over [1, N] (rejection-inversion of
 *                    Hoermann & Derflinger 1996); key = rank - 1
 *   GEN_ZIPF_HASHED  Zipf(s) ranks, key = bijective 64-bit mix of the rank
 *                    (u32: its high half is not a bijection, so u32 uses the
 *                    32-bit mix below)
 *   GEN_EXP          exponential with rate lambda, rounded, clamped to the range
 *   GEN_BITEXP       bit length L uniform in {0..w}, key uniform in [0, 2^L)
 *   GEN_DISTINCT     k distinct random keys, each record picks one uniformly
 *   GEN_HEAVYMIX     with prob. p1 one of k=p2 random heavy keys, else uniform
 *   GEN_SKEWMIX      30% Zipf(1.2, 1e9) hashed >> 1, 70% lognormal(40, 2)
 *                    clamped to [0, 2^63-1]
 *   GEN_BEXP_PAPER   every bit is 0 with probability 1/t (paper's BExp-t)
 *   GEN_UNIF_MU      mu distinct keys: key = mix(rng mod mu)
 *   GEN_EDGES        destination vertex of edge i of a power-law edge list:
 *                    Zipf(s) rank over V vertices (V a power of two), the
 *                    ranks scattered over [0, V) by an odd multiplier mod V;
 *                    the matching sources come from gen_edge_src
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum {
  GEN_UNIFORM = 0,
  GEN_ZIPF = 1,
  GEN_ZIPF_HASHED = 2,
  GEN_EXP = 3,
  GEN_BITEXP = 4,
  GEN_DISTINCT = 5,
  GEN_HEAVYMIX = 6,
  GEN_SKEWMIX = 7,
  GEN_BEXP_PAPER = 8,
  GEN_UNIF_MU = 9,
  GEN_EDGES = 10,
};

#define G_GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t g_fmix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Output i of the SplitMix64 sequence whose start state is output `stream`
 * of the sequence seeded with `seed`. */
uint64_t gen_rng(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t base = g_fmix(seed + (stream + 1) * G_GOLDEN);
  return g_fmix(base + (i + 1) * G_GOLDEN);
}

static double g_unit(uint64_t x) { /* [0, 1) with 53 bits */
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* 32-bit bijective mixer (murmur3 fmix32) for hashing u32 keys. */
static uint32_t g_fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6BU;
  h ^= h >> 13;
  h *= 0xC2B2AE35U;
  h ^= h >> 16;
  return h;
}

/* ---- Zipf by rejection-inversion (Hoermann & Derflinger 1996) ---------- */
typedef struct {
  double s, N;
  double hx1, hN, sq;
} zipf_t;

static double z_helper1(double x) { return fabs(x) > 1e-8 ? log1p(x) / x : 1.0 - x * (0.5 - x / 3.0); }
static double z_helper2(double x) { return fabs(x) > 1e-8 ? expm1(x) / x : 1.0 + x * 0.5 * (1.0 + x / 3.0); }
/* H(x) = integral of x^-s, shifted: ((x^(1-s)) - 1) / (1-s), log x at s = 1 */
static double z_H(const zipf_t *z, double x) {
  double lx = log(x);
  return z_helper2((1.0 - z->s) * lx) * lx;
}
static double z_h(const zipf_t *z, double x) { return exp(-z->s * log(x)); }
static double z_Hinv(const zipf_t *z, double x) {
  double t = x * (1.0 - z->s);
  if (t < -1.0) t = -1.0; /* guard rounding at the left end */
  return exp(z_helper1(t) * x);
}
static void zipf_init(zipf_t *z, double s, double N) {
  z->s = s;
  z->N = N;
  z->hx1 = z_H(z, 1.5) - 1.0;
  z->hN = z_H(z, N + 0.5);
  z->sq = 2.0 - z_Hinv(z, z_H(z, 2.5) - z_h(z, 2.0));
}
/* Rank in [1, N] for record i; retries draw from later streams. */
static uint64_t zipf_draw(const zipf_t *z, uint64_t seed, uint64_t stream, uint64_t i) {
  for (uint64_t attempt = 0;; ++attempt) {
    double U = g_unit(gen_rng(seed, stream + 16 * attempt, i));
    double u = z->hN + U * (z->hx1 - z->hN);
    double x = z_Hinv(z, u);
    double kd = floor(x + 0.5);
    if (kd < 1.0) kd = 1.0;
    if (kd > z->N) kd = z->N;
    if (kd - x <= z->sq || u >= z_H(z, kd + 0.5) - z_h(z, kd)) return (uint64_t)kd;
    if (attempt > 1000) return (uint64_t)kd; /* unreachable in practice */
  }
}

typedef struct {
  int kind, kbytes;
  double p1, p2;
  uint64_t seed;
  int64_t lo, hi;
  void *out;
  zipf_t zipf;
  uint64_t *table; /* distinct / heavy keys */
  int64_t table_n;
} gen_job_t;

static uint64_t draw_one(const gen_job_t *j, uint64_t i) {
  const uint64_t seed = j->seed;
  const int w = j->kbytes * 8;
  switch (j->kind) {
    case GEN_UNIFORM: {
      uint64_t r = gen_rng(seed, 0, i);
      return w == 32 ? (r >> 32) : r;
    }
    case GEN_ZIPF:
      return zipf_draw(&j->zipf, seed, 0, i) - 1;
    case GEN_ZIPF_HASHED: {
      uint64_t rk = zipf_draw(&j->zipf, seed, 0, i);
      return w == 32 ? (uint64_t)g_fmix32((uint32_t)(rk - 1)) : g_fmix(rk);
    }
    case GEN_EXP: {
      double U = g_unit(gen_rng(seed, 0, i));
      double x = floor(-log1p(-U) / j->p1 + 0.5);
      double cap = w == 32 ? 4294967295.0 : 18446744073709549568.0;
      if (x > cap) x = cap;
      return (uint64_t)x;
    }
    case GEN_BITEXP: {
      uint64_t L = gen_rng(seed, 0, i) % (uint64_t)(w + 1);
      uint64_t r = gen_rng(seed, 1, i);
      if (L == 0) return 0;
      uint64_t v = r >> (64 - L);
      return v;
    }
    case GEN_DISTINCT: {
      uint64_t pick = gen_rng(seed, 0, i) % (uint64_t)j->table_n;
      return j->table[pick];
    }
    case GEN_HEAVYMIX: {
      double U = g_unit(gen_rng(seed, 0, i));
      if (U < j->p1) return j->table[gen_rng(seed, 1, i) % (uint64_t)j->table_n];
      uint64_t r = gen_rng(seed, 2, i);
      return w == 32 ? (r >> 32) : r;
    }
    case GEN_SKEWMIX: {
      double U = g_unit(gen_rng(seed, 0, i));
      if (U < 0.3) {
        uint64_t rk = zipf_draw(&j->zipf, seed, 1, i);
        return g_fmix(rk) >> 1;
      }
      double u1 = g_unit(gen_rng(seed, 100, i));
      double u2 = g_unit(gen_rng(seed, 101, i));
      double zz = sqrt(-2.0 * log1p(-u1)) * cos(6.283185307179586 * u2);
      double x = floor(exp(40.0 + 2.0 * zz));
      const double cap = 9223372036854775807.0; /* rounds to 2^63 */
      if (!(x < cap)) return 0x7FFFFFFFFFFFFFFFULL;
      return (uint64_t)x;
    }
    case GEN_BEXP_PAPER: {
      /* bit b is 0 with probability 1/t: one uniform draw per bit */
      uint64_t v = 0;
      for (int b = 0; b < w; ++b) {
        double U = g_unit(gen_rng(seed, (uint64_t)b, i));
        if (U >= 1.0 / j->p1) v |= 1ULL << b;
      }
      return v;
    }
    case GEN_UNIF_MU: {
      uint64_t r = gen_rng(seed, 0, i) % (uint64_t)j->p1;
      return w == 32 ? (uint64_t)g_fmix32((uint32_t)r) : g_fmix(r + 1);
    }
    case GEN_EDGES: {
      uint64_t rk = zipf_draw(&j->zipf, seed, 0, i) - 1;
      return (rk * G_GOLDEN) & ((uint64_t)j->p2 - 1);
    }
    default:
      return 0;
  }
}

static void *gen_main(void *arg) {
  gen_job_t *j = (gen_job_t *)arg;
  if (j->kbytes == 4) {
    uint32_t *o = (uint32_t *)j->out;
    for (int64_t i = j->lo; i < j->hi; ++i) o[i] = (uint32_t)draw_one(j, (uint64_t)i);
  } else {
    uint64_t *o = (uint64_t *)j->out;
    for (int64_t i = j->lo; i < j->hi; ++i) o[i] = draw_one(j, (uint64_t)i);
  }
  return NULL;
}

int gen_default_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

/* Fill out[0..n) (kbytes = 4 or 8) with keys of the given family.
 * Records [first, first+n) of the conceptual stream are produced, so a large
 * input can be generated in pieces.  p1/p2 are the family's parameters:
 *   ZIPF/ZIPF_HASHED: p1 = s, p2 = N;  EXP: p1 = rate;  DISTINCT: p1 = k;
 *   HEAVYMIX: p1 = heavy probability, p2 = number of heavy keys;
 *   BEXP_PAPER: p1 = t;  UNIF_MU: p1 = mu.   Returns 0 on success. */
int gen_keys(int kind, int kbytes, double p1, double p2, uint64_t seed,
             int64_t first, int64_t n, void *out, int nthreads) {
  if (n < 0 || (kbytes != 4 && kbytes != 8)) return -1;
  if (n == 0) return 0;
  if (nthreads <= 0) nthreads = gen_default_threads();
  gen_job_t proto;
  memset(&proto, 0, sizeof(proto));
  proto.kind = kind;
  proto.kbytes = kbytes;
  proto.p1 = p1;
  proto.p2 = p2;
  proto.seed = seed;
  if (kind == GEN_ZIPF || kind == GEN_ZIPF_HASHED || kind == GEN_EDGES)
    zipf_init(&proto.zipf, p1, p2);
  if (kind == GEN_EDGES && (p2 < 2.0 || (((uint64_t)p2) & ((uint64_t)p2 - 1)) != 0)) return -1;
  if (kind == GEN_SKEWMIX) zipf_init(&proto.zipf, 1.2, 1e9);
  if (kind == GEN_DISTINCT || kind == GEN_HEAVYMIX) {
    int64_t k = kind == GEN_DISTINCT ? (int64_t)p1 : (int64_t)p2;
    if (k <= 0) return -1;
    proto.table_n = k;
    proto.table = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)k);
    if (!proto.table) return -1;
    for (int64_t q = 0; q < k; ++q) {
      uint64_t r = gen_rng(seed, 7, (uint64_t)q);
      proto.table[q] = kbytes == 4 ? (r >> 32) : r;
    }
  }
  if (kind == GEN_UNIF_MU && p1 < 1.0) return -1;
  /* shift the output pointer so that draw index == absolute record index */
  char *base = (char *)out - first * kbytes;
  int T = nthreads;
  if ((int64_t)T > n) T = (int)n;
  gen_job_t *jobs = (gen_job_t *)malloc(sizeof(gen_job_t) * (size_t)T);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
  if (!jobs || !th) { free(jobs); free(th); free(proto.table); return -1; }
  for (int t = 0; t < T; ++t) {
    jobs[t] = proto;
    jobs[t].out = base;
    jobs[t].lo = first + n * t / T;
    jobs[t].hi = first + n * (t + 1) / T;
    pthread_create(&th[t], NULL, gen_main, &jobs[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  free(proto.table);
  return 0;
}

/* out[i] = first + i (values that make stability observable). */
int gen_iota(int vbytes, int64_t first, int64_t n, void *out) {
  if (vbytes == 4) {
    uint32_t *o = (uint32_t *)out;
    for (int64_t i = 0; i < n; ++i) o[i] = (uint32_t)(first + i);
  } else {
    uint64_t *o = (uint64_t *)out;
    for (int64_t i = 0; i < n; ++i) o[i] = (uint64_t)(first + i);
  }
  return 0;
}

/* Source vertices of edges [first, first+n) of a list of E edges over V
 * vertices ordered by source: src_i = floor(i V / E), every vertex about E/V
 * out-edges. */
int gen_edge_src(int vbytes, int64_t first, int64_t n, int64_t E, int64_t V, void *out) {
  if (E <= 0 || V <= 0 || V > 0xFFFFFFFFLL || first < 0 || first + n > E) return -1;
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t src = (uint64_t)(((unsigned __int128)(uint64_t)(first + i) * (uint64_t)V) /
                                    (uint64_t)E);
    if (vbytes == 4) ((uint32_t *)out)[i] = (uint32_t)src;
    else ((uint64_t *)out)[i] = src;
  }
  return 0;
}

/* Segment sizes for the batched configuration: size_j = round(lo * (hi/lo)^U_j)
 * (log-uniform in [lo, hi]), and a per-segment family flag (0 uniform,
 * 1 Zipf) drawn with probability 1/2. */
int gen_segment_sizes(uint64_t seed, int64_t nseg, double lo, double hi,
                      int64_t *sizes, int32_t *family) {
  for (int64_t j = 0; j < nseg; ++j) {
    double U = g_unit(gen_rng(seed, 3, (uint64_t)j));
    double v = lo * pow(hi / lo, U);
    sizes[j] = (int64_t)floor(v + 0.5);
    if (family) family[j] = (int32_t)(gen_rng(seed, 4, (uint64_t)j) >> 63);
  }
  return 0;
}
