/*
 * CPU oracle for the stable integer sort of "Parallel Integer Sort: Theory and
 * Practice" (DovetailSort).  TEST INFRASTRUCTURE ONLY: only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Everything here is written for obviousness, not speed:
 *
 *   oracle_sort_*            Sec. 2.3 (problem statement): records with integer
 *                            keys in [r] are reordered into non-decreasing key
 *                            order, stably.  A stable sort's output is unique:
 *                            it is the order of the pairs (key, original index)
 *                            compared lexicographically, which is what a
 *                            textbook merge sort on those pairs computes.
 *   oracle_stable_positions  The same definition for one record j:
 *                            pos(j) = #{i : k_i < k_j} + #{i < j : k_i == k_j}.
 *   oracle_check_stable      The same definition read as a test of a claimed
 *                            output (keys, and for each output slot the
 *                            original index of its record): the pairs (key,
 *                            index) must be strictly increasing, the indices a
 *                            permutation of 0..n-1, and each key the input key
 *                            at its index; exactly one output passes.
 *   oracle_check_sorted_keys The definition for key-only output, where
 *                            stability is unobservable: the input's multiset
 *                            of keys in non-decreasing order (order of
 *                            adjacent slots, and every key value as often as
 *                            in the input, counted per top-16-bit group).
 *   oracle_splitmix64_*      The SplitMix64 generator (Steele, Lea, Flood,
 *                            OOPSLA 2014), used for the sampler's random draws.
 *   oracle_sample_*          Alg. 2 step 1 (Sec. 3.1): draw the sample S, sort
 *                            it, keep every (log n)-th key, keys seen more than
 *                            once in the subsample are heavy.  App. "Overflow
 *                            bucket": the largest sample fixes the key range.
 *   oracle_bucket_ids_*      Alg. 2: arrays h (heavy: zone, key) and l (light:
 *                            zone, dummy), merged and numbered serially;
 *                            GetBucketId (hash lookup H, else light table L).
 *   oracle_dtmerge_*         Alg. 3 (DTMerge), both the heavy-larger case and
 *                            the symmetric light-larger case, in place with a
 *                            temporary array and flip-based rotations.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Stable sort by definition: merge sort on (key, original index) pairs.     */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t key; /* the key, zero-extended to 64 bits (unsigned order kept) */
  uint64_t idx; /* original position in the input */
} pair_t;

static int pair_less(const pair_t *a, const pair_t *b) {
  if (a->key != b->key) return a->key < b->key;
  return a->idx < b->idx;
}

/* Merge sorted a[0..na) and b[0..nb) into out. */
static void merge_pairs(const pair_t *a, int64_t na, const pair_t *b, int64_t nb,
                        pair_t *out) {
  int64_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) {
    if (pair_less(&b[j], &a[i])) out[k++] = b[j++];
    else out[k++] = a[i++];
  }
  while (i < na) out[k++] = a[i++];
  while (j < nb) out[k++] = b[j++];
}

/* Bottom-up merge sort of x[0..n), tmp has room for n pairs. */
static void merge_sort_pairs(pair_t *x, pair_t *tmp, int64_t n) {
  pair_t *src = x, *dst = tmp;
  for (int64_t width = 1; width < n; width *= 2) {
    for (int64_t lo = 0; lo < n; lo += 2 * width) {
      int64_t mid = lo + width < n ? lo + width : n;
      int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
      merge_pairs(src + lo, mid - lo, src + mid, hi - mid, dst + lo);
    }
    pair_t *t = src;
    src = dst;
    dst = t;
  }
  if (src != x) memcpy(x, src, (size_t)n * sizeof(pair_t));
}

typedef struct {
  pair_t *x, *tmp;
  int64_t lo, hi;  /* chunk sort: [lo, hi) */
  int64_t mid;     /* merge step: merge [lo, mid) and [mid, hi) from x into tmp */
} sort_job_t;

static void *chunk_sort_main(void *arg) {
  sort_job_t *j = (sort_job_t *)arg;
  merge_sort_pairs(j->x + j->lo, j->tmp + j->lo, j->hi - j->lo);
  return NULL;
}

static void *chunk_merge_main(void *arg) {
  sort_job_t *j = (sort_job_t *)arg;
  merge_pairs(j->x + j->lo, j->mid - j->lo, j->x + j->mid, j->hi - j->mid,
              j->tmp + j->lo);
  memcpy(j->x + j->lo, j->tmp + j->lo, (size_t)(j->hi - j->lo) * sizeof(pair_t));
  return NULL;
}

int oracle_default_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

/* Sort pairs with T threads: T sorted chunks, then rounds of pairwise merges. */
static int sort_pairs_threaded(pair_t *x, int64_t n, int nthreads) {
  if (n <= 1) return 0;
  if (nthreads <= 0) nthreads = oracle_default_threads();
  if ((int64_t)nthreads > n) nthreads = (int)n;
  pair_t *tmp = (pair_t *)malloc((size_t)n * sizeof(pair_t));
  if (!tmp) return -1;
  int T = nthreads;
  int64_t *bound = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
  sort_job_t *jobs = (sort_job_t *)malloc(sizeof(sort_job_t) * (size_t)T);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
  if (!bound || !jobs || !th) {
    free(tmp); free(bound); free(jobs); free(th);
    return -1;
  }
  for (int t = 0; t <= T; ++t) bound[t] = n * t / T;
  for (int t = 0; t < T; ++t) {
    jobs[t].x = x; jobs[t].tmp = tmp;
    jobs[t].lo = bound[t]; jobs[t].hi = bound[t + 1];
    pthread_create(&th[t], NULL, chunk_sort_main, &jobs[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  /* runs [bound[r], bound[r+1]) are sorted; merge neighbours until one run */
  int runs = T;
  while (runs > 1) {
    int pairs = runs / 2;
    for (int p = 0; p < pairs; ++p) {
      jobs[p].x = x; jobs[p].tmp = tmp;
      jobs[p].lo = bound[2 * p];
      jobs[p].mid = bound[2 * p + 1];
      jobs[p].hi = bound[2 * p + 2];
      pthread_create(&th[p], NULL, chunk_merge_main, &jobs[p]);
    }
    for (int p = 0; p < pairs; ++p) pthread_join(th[p], NULL);
    int nr = 0;
    for (int p = 0; p < pairs; ++p) bound[nr++] = bound[2 * p];
    if (runs % 2) bound[nr++] = bound[runs - 1];
    bound[nr] = n;
    runs = nr;
  }
  free(tmp); free(bound); free(jobs); free(th);
  return 0;
}

/* keys: n keys of kbytes (4 or 8) each; vals: NULL or n values of vbytes.
 * Results go to out_keys / out_vals (may alias the inputs). */
static int sort_generic(const void *keys, const void *vals, int64_t n, int kbytes,
                        int vbytes, void *out_keys, void *out_vals, int nthreads) {
  if (n < 0) return -1;
  if (n == 0) return 0;
  pair_t *x = (pair_t *)malloc((size_t)n * sizeof(pair_t));
  if (!x) return -1;
  for (int64_t i = 0; i < n; ++i) {
    x[i].key = kbytes == 4 ? (uint64_t)((const uint32_t *)keys)[i]
                           : ((const uint64_t *)keys)[i];
    x[i].idx = (uint64_t)i;
  }
  if (sort_pairs_threaded(x, n, nthreads)) { free(x); return -1; }
  void *vcopy = NULL;
  if (vals) {
    /* gather from a copy so that out_vals may alias vals */
    vcopy = malloc((size_t)n * (size_t)vbytes);
    if (!vcopy) { free(x); return -1; }
    memcpy(vcopy, vals, (size_t)n * (size_t)vbytes);
  }
  for (int64_t i = 0; i < n; ++i) {
    if (kbytes == 4) ((uint32_t *)out_keys)[i] = (uint32_t)x[i].key;
    else ((uint64_t *)out_keys)[i] = x[i].key;
    if (vals) {
      if (vbytes == 4) ((uint32_t *)out_vals)[i] = ((const uint32_t *)vcopy)[x[i].idx];
      else ((uint64_t *)out_vals)[i] = ((const uint64_t *)vcopy)[x[i].idx];
    }
  }
  free(vcopy);
  free(x);
  return 0;
}

int oracle_sort_u32(const uint32_t *keys, const uint32_t *vals, int64_t n,
                    uint32_t *out_keys, uint32_t *out_vals, int nthreads) {
  return sort_generic(keys, vals, n, 4, 4, out_keys, out_vals, nthreads);
}

int oracle_sort_u64(const uint64_t *keys, const uint64_t *vals, int64_t n,
                    uint64_t *out_keys, uint64_t *out_vals, int nthreads) {
  return sort_generic(keys, vals, n, 8, 8, out_keys, out_vals, nthreads);
}

/* Segmented: the definition applied to each [off[s], off[s+1]) on its own. */
static int sort_segmented_generic(const void *keys, const void *vals,
                                  const int64_t *off, int64_t nseg, int kbytes,
                                  int vbytes, void *out_keys, void *out_vals,
                                  int nthreads) {
  if (nseg < 0) return -1;
  for (int64_t s = 0; s < nseg; ++s) {
    int64_t a = off[s], b = off[s + 1];
    if (b < a) return -1;
    const char *k = (const char *)keys + a * kbytes;
    const char *v = vals ? (const char *)vals + a * vbytes : NULL;
    char *ok = (char *)out_keys + a * kbytes;
    char *ov = out_vals ? (char *)out_vals + a * vbytes : NULL;
    int t = (b - a) >= (1 << 16) ? nthreads : 1;
    if (sort_generic(k, v, b - a, kbytes, vbytes, ok, ov, t)) return -1;
  }
  return 0;
}

int oracle_sort_segmented_u32(const uint32_t *keys, const uint32_t *vals,
                              const int64_t *off, int64_t nseg, uint32_t *out_keys,
                              uint32_t *out_vals, int nthreads) {
  return sort_segmented_generic(keys, vals, off, nseg, 4, 4, out_keys, out_vals,
                                nthreads);
}

int oracle_sort_segmented_u64(const uint64_t *keys, const uint64_t *vals,
                              const int64_t *off, int64_t nseg, uint64_t *out_keys,
                              uint64_t *out_vals, int nthreads) {
  return sort_segmented_generic(keys, vals, off, nseg, 8, 8, out_keys, out_vals,
                                nthreads);
}

/* ------------------------------------------------------------------------ */
/* Stable output position of chosen records, straight from the definition.   */
/* ------------------------------------------------------------------------ */

typedef struct {
  const void *keys;
  int kbytes;
  int64_t lo, hi;
  const int64_t *js;
  int64_t m;
  int64_t *partial; /* m counts for this thread */
} pos_job_t;

static uint64_t key_at(const void *keys, int kbytes, int64_t i) {
  return kbytes == 4 ? (uint64_t)((const uint32_t *)keys)[i]
                     : ((const uint64_t *)keys)[i];
}

static void *pos_main(void *arg) {
  pos_job_t *p = (pos_job_t *)arg;
  for (int64_t q = 0; q < p->m; ++q) {
    int64_t j = p->js[q];
    uint64_t kj = key_at(p->keys, p->kbytes, j);
    int64_t c = 0;
    for (int64_t i = p->lo; i < p->hi; ++i) {
      uint64_t ki = key_at(p->keys, p->kbytes, i);
      c += (ki < kj) || (ki == kj && i < j);
    }
    p->partial[q] = c;
  }
  return NULL;
}

/* out[q] = stable-sorted position of input record js[q]. */
int oracle_stable_positions(const void *keys, int kbytes, int64_t n,
                            const int64_t *js, int64_t m, int64_t *out,
                            int nthreads) {
  if (nthreads <= 0) nthreads = oracle_default_threads();
  for (int64_t q = 0; q < m; ++q)
    if (js[q] < 0 || js[q] >= n) return -1;
  int T = nthreads;
  pos_job_t *jobs = (pos_job_t *)calloc((size_t)T, sizeof(pos_job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
  int64_t *part = (int64_t *)calloc((size_t)T * (size_t)(m > 0 ? m : 1), sizeof(int64_t));
  if (!jobs || !th || !part) { free(jobs); free(th); free(part); return -1; }
  for (int t = 0; t < T; ++t) {
    jobs[t].keys = keys; jobs[t].kbytes = kbytes;
    jobs[t].lo = n * t / T; jobs[t].hi = n * (t + 1) / T;
    jobs[t].js = js; jobs[t].m = m; jobs[t].partial = part + (int64_t)t * m;
    pthread_create(&th[t], NULL, pos_main, &jobs[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  for (int64_t q = 0; q < m; ++q) {
    int64_t c = 0;
    for (int t = 0; t < T; ++t) c += part[(int64_t)t * m + q];
    out[q] = c;
  }
  free(jobs); free(th); free(part);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Check of a claimed stable-sorted output (Sec. 2.3 definition).            */
/* ------------------------------------------------------------------------ */

typedef struct {
  const void *kin, *kout;
  const void *idx;     /* original index of each output record */
  int kbytes, ibytes;
  int64_t n, lo, hi;
  unsigned char *seen; /* one byte per original index */
  int64_t bad;         /* first failing output slot + 1, or 0 */
} chk_job_t;

static void *chk_main(void *arg) {
  chk_job_t *j = (chk_job_t *)arg;
  for (int64_t i = j->lo; i < j->hi && !j->bad; ++i) {
    const uint64_t ix = key_at(j->idx, j->ibytes, i);
    const uint64_t k = key_at(j->kout, j->kbytes, i);
    int ok = ix < (uint64_t)j->n && key_at(j->kin, j->kbytes, (int64_t)ix) == k;
    if (ok && i + 1 < j->n) {  /* (key, index) strictly increasing */
      const uint64_t k2 = key_at(j->kout, j->kbytes, i + 1);
      ok = k < k2 || (k == k2 && ix < key_at(j->idx, j->ibytes, i + 1));
    }
    /* strictly increasing pairs cannot repeat an index (an index fixes its
       key), so the indices are distinct; `seen` confirms they cover 0..n-1 */
    if (ok) j->seen[ix] = 1;
    else j->bad = i + 1;
  }
  return NULL;
}

/* Returns -1 if the output is the stable sort of kin, else the first failing
 * output slot (or n if some index never appears).  idx: indices of ibytes
 * (4 or 8) bytes. */
int64_t oracle_check_stable(const void *kin, const void *kout, const void *idx, int kbytes,
                            int ibytes, int64_t n, int nthreads) {
  if (n <= 0) return -1;
  if (nthreads <= 0) nthreads = oracle_default_threads();
  unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
  chk_job_t *jobs = (chk_job_t *)calloc((size_t)nthreads, sizeof(chk_job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!seen || !jobs || !th) { free(seen); free(jobs); free(th); return -2; }
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].kin = kin; jobs[t].kout = kout; jobs[t].idx = idx; jobs[t].kbytes = kbytes;
    jobs[t].ibytes = ibytes;
    jobs[t].n = n; jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
    jobs[t].seen = seen;
    pthread_create(&th[t], NULL, chk_main, &jobs[t]);
  }
  int64_t first = -1;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].bad && first < 0) first = jobs[t].bad - 1;
  }
  if (first < 0)
    for (int64_t i = 0; i < n; ++i)
      if (!seen[i]) { first = n; break; }
  free(seen); free(jobs); free(th);
  return first;
}

/* ------------------------------------------------------------------------ */
/* Check of a claimed key-only sorted output (Sec. 2.3 definition).          */
/* ------------------------------------------------------------------------ */
/* Without values stability cannot be observed: the unique answer is the
 * input's multiset of keys in non-decreasing order.  The check reads that
 * definition directly: (1) the output is non-decreasing; (2) it holds every
 * key value exactly as often as the input does.  (2) is counted per group of
 * keys sharing their top 16 bits: the group's input count must equal its
 * output count (the output being sorted, each group is then one contiguous
 * range of it), and inside a group every distinct output key, read as a run
 * of equal keys, must receive from the input exactly as many keys as the run
 * is long, with no input key left without a run. */

#define CSK_BITS 16
#define CSK_G ((int64_t)1 << CSK_BITS)

static uint64_t csk_group(uint64_t k, int kbytes) { return k >> (8 * kbytes - CSK_BITS); }

typedef struct {
  const void *kin, *kout;
  int kbytes;
  int64_t n, lo, hi;
  int64_t *cin, *cout;   /* this thread's group counts */
  int64_t bad;           /* first unsorted output slot + 1, or 0 */
} csk_count_t;

static void *csk_count_main(void *arg) {
  csk_count_t *j = (csk_count_t *)arg;
  for (int64_t i = j->lo; i < j->hi; ++i) {
    const uint64_t a = key_at(j->kout, j->kbytes, i);
    if (!j->bad && i + 1 < j->n && a > key_at(j->kout, j->kbytes, i + 1)) j->bad = i + 1;
    j->cout[csk_group(a, j->kbytes)] += 1;
    j->cin[csk_group(key_at(j->kin, j->kbytes, i), j->kbytes)] += 1;
  }
  return NULL;
}

typedef struct {
  const void *kin;
  int kbytes;
  int64_t lo, hi;
  int64_t *pos;          /* this thread's next slot per group */
  uint64_t *grouped;     /* input keys, grouped */
} csk_scatter_t;

static void *csk_scatter_main(void *arg) {
  csk_scatter_t *j = (csk_scatter_t *)arg;
  for (int64_t i = j->lo; i < j->hi; ++i) {
    const uint64_t k = key_at(j->kin, j->kbytes, i);
    j->grouped[j->pos[csk_group(k, j->kbytes)]++] = k;
  }
  return NULL;
}

typedef struct {
  const void *kout;
  int kbytes;
  const int64_t *start;  /* group g: output and grouped input [start[g], start[g+1]) */
  const uint64_t *grouped;
  int64_t *next;         /* shared group counter */
  int64_t bad;           /* first slot of a mismatching group + 1, or 0; -1 no memory */
} csk_match_t;

/* runs of the sorted output range: distinct keys and their lengths */
static int64_t csk_runs(const void *kout, int kbytes, int64_t a, int64_t b, uint64_t *rk,
                        int64_t *rlen) {
  int64_t r = 0;
  for (int64_t i = a; i < b; ++i) {
    const uint64_t k = key_at(kout, kbytes, i);
    if (r == 0 || rk[r - 1] != k) { rk[r] = k; rlen[r] = 0; ++r; }
    rlen[r - 1] += 1;
  }
  return r;
}

static void *csk_match_main(void *arg) {
  csk_match_t *j = (csk_match_t *)arg;
  while (1) {
    const int64_t g = __atomic_fetch_add(j->next, 1, __ATOMIC_RELAXED);
    if (g >= CSK_G) break;
    const int64_t a = j->start[g], b = j->start[g + 1];
    if (b == a) continue;
    uint64_t *rk = (uint64_t *)malloc((size_t)(b - a) * sizeof(uint64_t));
    int64_t *rlen = (int64_t *)malloc((size_t)(b - a) * sizeof(int64_t));
    if (!rk || !rlen) { free(rk); free(rlen); j->bad = -1; return NULL; }
    const int64_t r = csk_runs(j->kout, j->kbytes, a, b, rk, rlen);
    int ok = 1;
    for (int64_t i = a; i < b && ok; ++i) {
      const uint64_t k = j->grouped[i];
      int64_t lo = 0, hi = r;  /* first run whose key is >= k */
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (rk[mid] < k) lo = mid + 1; else hi = mid;
      }
      if (lo == r || rk[lo] != k || rlen[lo] == 0) ok = 0;  /* no run left for k */
      else rlen[lo] -= 1;
    }
    /* equal totals and no key without a run: every run was used up exactly */
    free(rk); free(rlen);
    if (!ok && (j->bad == 0 || a + 1 < j->bad)) j->bad = a + 1;
  }
  return NULL;
}

/* Returns -1 if kout[0..n) is the input's multiset of keys in non-decreasing
 * order; else the first output slot that is out of order, or the first slot
 * of a group of keys whose multiset differs; -2 if memory ran out. */
int64_t oracle_check_sorted_keys(const void *kin, const void *kout, int kbytes, int64_t n,
                                 int nthreads) {
  if (n <= 0) return -1;
  if (nthreads <= 0) nthreads = oracle_default_threads();
  if ((int64_t)nthreads > n) nthreads = (int)n;
  const int T = nthreads;
  int64_t *cnt = (int64_t *)calloc((size_t)T * 2 * CSK_G, sizeof(int64_t));
  int64_t *start = (int64_t *)malloc((size_t)(CSK_G + 1) * sizeof(int64_t));
  uint64_t *grouped = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  csk_count_t *cj = (csk_count_t *)calloc((size_t)T, sizeof(csk_count_t));
  csk_scatter_t *sj = (csk_scatter_t *)calloc((size_t)T, sizeof(csk_scatter_t));
  csk_match_t *mj = (csk_match_t *)calloc((size_t)T, sizeof(csk_match_t));
  pthread_t *th = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
  int64_t result = -1;
  if (!cnt || !start || !grouped || !cj || !sj || !mj || !th) { result = -2; goto done; }
  /* (1) order, and the group counts of both sides */
  for (int t = 0; t < T; ++t) {
    cj[t].kin = kin; cj[t].kout = kout; cj[t].kbytes = kbytes; cj[t].n = n;
    cj[t].lo = n * t / T; cj[t].hi = n * (t + 1) / T;
    cj[t].cin = cnt + (size_t)t * 2 * CSK_G;
    cj[t].cout = cj[t].cin + CSK_G;
    pthread_create(&th[t], NULL, csk_count_main, &cj[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < T; ++t)
    if (cj[t].bad) { result = cj[t].bad - 1; goto done; }
  /* (2a) equal group counts; group g is output range [start[g], start[g+1]) */
  start[0] = 0;
  for (int64_t g = 0; g < CSK_G; ++g) {
    int64_t ci = 0, co = 0;
    for (int t = 0; t < T; ++t) { ci += cj[t].cin[g]; co += cj[t].cout[g]; }
    if (ci != co) { result = start[g]; goto done; }
    start[g + 1] = start[g] + ci;
  }
  /* (2b) the input keys grouped the same way (each thread its own slots) */
  for (int64_t g = 0; g < CSK_G; ++g) {
    int64_t p = start[g];
    for (int t = 0; t < T; ++t) {
      const int64_t c = cj[t].cin[g];
      cj[t].cin[g] = p;  /* becomes thread t's next slot in group g */
      p += c;
    }
  }
  for (int t = 0; t < T; ++t) {
    sj[t].kin = kin; sj[t].kbytes = kbytes;
    sj[t].lo = n * t / T; sj[t].hi = n * (t + 1) / T;
    sj[t].pos = cj[t].cin; sj[t].grouped = grouped;
    pthread_create(&th[t], NULL, csk_scatter_main, &sj[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  /* (2c) per group: the runs of the output against the input's keys */
  int64_t next = 0;
  for (int t = 0; t < T; ++t) {
    mj[t].kout = kout; mj[t].kbytes = kbytes; mj[t].start = start;
    mj[t].grouped = grouped; mj[t].next = &next;
    pthread_create(&th[t], NULL, csk_match_main, &mj[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < T; ++t) {
    if (mj[t].bad < 0) { result = -2; goto done; }
    if (mj[t].bad > 0 && (result < 0 || mj[t].bad - 1 < result)) result = mj[t].bad - 1;
  }
done:
  free(cnt); free(start); free(grouped); free(cj); free(sj); free(mj); free(th);
  return result;
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden gamma, */
/* each output is the state passed through the 64-bit finaliser.            */
/* ------------------------------------------------------------------------ */

uint64_t oracle_splitmix64_next(uint64_t *state) {
  *state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 sequence whose state starts at s:
 * the state after i+1 steps is s + (i+1)*gamma. */
uint64_t oracle_splitmix64_at(uint64_t s, uint64_t i) {
  uint64_t st = s + i * 0x9E3779B97F4A7C15ULL;
  return oracle_splitmix64_next(&st);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 step 1: sampling and heavy-key detection.                          */
/* ------------------------------------------------------------------------ */

static uint64_t low_mask(int bits) {
  return bits >= 64 ? ~0ULL : ((1ULL << bits) - 1ULL);
}

/* The sampler's random stream for one subproblem.  A subproblem is named by
 * (start, size, hi): hi is the number of low key bits still unsorted.  The
 * stream is the SplitMix64 sequence started from
 *   seed ^ start ^ (size * gamma) ^ (hi << 57),
 * and sample i reads position start + (output_i mod size). */
uint64_t oracle_sample_stream(uint64_t seed, int64_t start, int64_t size, int hi) {
  return seed ^ (uint64_t)start ^ ((uint64_t)size * 0x9E3779B97F4A7C15ULL) ^
         ((uint64_t)hi << 57);
}

int oracle_sample_positions(uint64_t seed, int64_t start, int64_t size, int hi,
                            int64_t count, int64_t *pos_out) {
  if (size <= 0 || count < 0) return -1;
  uint64_t s = oracle_sample_stream(seed, start, size, hi);
  for (int64_t i = 0; i < count; ++i)
    pos_out[i] = start + (int64_t)(oracle_splitmix64_at(s, (uint64_t)i) % (uint64_t)size);
  return 0;
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* The heavy-key rule on a given sample S[0..m):
 *   sort S; the subsample S' holds every L-th key, i.e. S[L-1], S[2L-1], ...;
 *   a key is heavy when it occurs at least twice in S'.
 * Writes the distinct heavy keys in increasing order, returns their number.
 * *max_out receives max(S) (the key-range estimate r'). */
int64_t oracle_heavy_from_sample(const uint64_t *sample, int64_t m, int64_t L,
                                 uint64_t *heavy_out, uint64_t *max_out) {
  if (m <= 0 || L <= 0) { if (max_out) *max_out = 0; return 0; }
  uint64_t *s = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
  if (!s) return -1;
  memcpy(s, sample, (size_t)m * sizeof(uint64_t));
  qsort(s, (size_t)m, sizeof(uint64_t), cmp_u64);
  if (max_out) *max_out = s[m - 1];
  int64_t nsub = m / L;
  int64_t nh = 0;
  for (int64_t j = 0; j + 1 < nsub; ++j) {
    uint64_t a = s[(j + 1) * L - 1], b = s[(j + 2) * L - 1];
    if (a == b && (nh == 0 || heavy_out[nh - 1] != a)) heavy_out[nh++] = a;
  }
  free(s);
  return nh;
}

/* Sampling of one subproblem: draw `count` keys at the positions above, then
 * apply the rule with stride L.  Keys are taken as is; hi only names the
 * stream.  Returns the number of heavy keys. */
int64_t oracle_sample_heavy(const void *keys, int kbytes, uint64_t seed,
                            int64_t start, int64_t size, int hi, int64_t count,
                            int64_t L, uint64_t *heavy_out, uint64_t *max_out) {
  if (count <= 0) { if (max_out) *max_out = 0; return 0; }
  int64_t *pos = (int64_t *)malloc((size_t)count * sizeof(int64_t));
  uint64_t *smp = (uint64_t *)malloc((size_t)count * sizeof(uint64_t));
  if (!pos || !smp) { free(pos); free(smp); return -1; }
  oracle_sample_positions(seed, start, size, hi, count, pos);
  for (int64_t i = 0; i < count; ++i) smp[i] = key_at(keys, kbytes, pos[i]);
  int64_t nh = oracle_heavy_from_sample(smp, count, L, heavy_out, max_out);
  free(pos);
  free(smp);
  return nh;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: bucket ids.                                                       */
/* ------------------------------------------------------------------------ */

/* Zone layout of a subproblem whose keys agree on every bit >= hi:
 *   t  = bit length of (r' & mask(hi)), r' the largest sample;
 *   the MSD zone digit is bits [lo, t) with lo = max(t - gamma, 0);
 *   a key with a 1 anywhere in bits [t, hi) belongs to the overflow bucket. */
void oracle_zone_layout(uint64_t rmax, int hi, int gamma, int *t_out, int *lo_out) {
  uint64_t r = rmax & low_mask(hi);
  int t = 0;
  while (t < 64 && (r >> t) != 0) ++t;
  int lo = t - gamma > 0 ? t - gamma : 0;
  *t_out = t;
  *lo_out = lo;
}

typedef struct {
  uint64_t zone;
  int light;    /* 1 for the light bucket of the zone (dummy key -1) */
  uint64_t key; /* heavy key */
} bucket_entry_t;

/* Order of the merged h/l array: by zone; within a zone the light bucket
 * comes first, then heavy buckets by key. */
static int entry_before(const bucket_entry_t *a, const bucket_entry_t *b) {
  if (a->zone != b->zone) return a->zone < b->zone;
  if (a->light != b->light) return a->light > b->light;
  return a->key < b->key;
}

/* Assigns bucket ids as Alg. 2 does and evaluates GetBucketId for n keys.
 * heavy: nheavy distinct keys (any order).  ids_out[i] receives the bucket id
 * of keys[i]; the overflow bucket is the last id.  If table_out is not NULL
 * it receives, for each id, the zone (or 2^64-1 for overflow) and is sized
 * (2^(t-lo) + nheavy + 1).  Returns the number of buckets. */
int64_t oracle_bucket_ids(const uint64_t *heavy, int64_t nheavy, uint64_t rmax,
                          int hi, int gamma, const void *keys, int kbytes,
                          int64_t n, int32_t *ids_out) {
  int t, lo;
  oracle_zone_layout(rmax, hi, gamma, &t, &lo);
  int64_t nzones = (int64_t)1 << (t - lo);
  uint64_t mhi = low_mask(hi);
  /* h: heavy keys with their zones; l: one light entry per zone */
  int64_t ne = nzones + nheavy;
  bucket_entry_t *h = (bucket_entry_t *)malloc(sizeof(bucket_entry_t) * (size_t)(nheavy + 1));
  bucket_entry_t *l = (bucket_entry_t *)malloc(sizeof(bucket_entry_t) * (size_t)nzones);
  bucket_entry_t *all = (bucket_entry_t *)malloc(sizeof(bucket_entry_t) * (size_t)ne);
  uint64_t *hs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nheavy + 1));
  if (!h || !l || !all || !hs) { free(h); free(l); free(all); free(hs); return -1; }
  memcpy(hs, heavy, sizeof(uint64_t) * (size_t)nheavy);
  qsort(hs, (size_t)nheavy, sizeof(uint64_t), cmp_u64);
  for (int64_t i = 0; i < nheavy; ++i) {
    h[i].zone = (hs[i] & mhi) >> lo;
    h[i].light = 0;
    h[i].key = hs[i];
  }
  for (int64_t z = 0; z < nzones; ++z) {
    l[z].zone = (uint64_t)z;
    l[z].light = 1;
    l[z].key = 0;
  }
  /* merge h and l (both already in entry order) */
  int64_t a = 0, b = 0, k = 0;
  while (a < nheavy && b < nzones) {
    if (entry_before(&l[b], &h[a])) all[k++] = l[b++];
    else all[k++] = h[a++];
  }
  while (a < nheavy) all[k++] = h[a++];
  while (b < nzones) all[k++] = l[b++];
  /* serial ids: L[zone] for light entries, H[key] for heavy entries */
  int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)nzones);
  int64_t *Hid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nheavy + 1));
  if (!L || !Hid) { free(h); free(l); free(all); free(hs); free(L); free(Hid); return -1; }
  int64_t hcount = 0;
  for (int64_t i = 0; i < ne; ++i) {
    if (all[i].light) L[all[i].zone] = i;
    else Hid[hcount++] = i; /* heavy entries appear in increasing key order */
  }
  int64_t overflow_id = ne;
  /* GetBucketId: look the key up among the heavy keys, else overflow test,
   * else the light table by zone. */
  for (int64_t i = 0; i < n; ++i) {
    uint64_t key = key_at(keys, kbytes, i);
    uint64_t *hit = nheavy ? (uint64_t *)bsearch(&key, hs, (size_t)nheavy,
                                                 sizeof(uint64_t), cmp_u64)
                           : NULL;
    if (hit) {
      ids_out[i] = (int32_t)Hid[hit - hs];
    } else if (((key & mhi) >> t) != 0 && t < 64) {
      ids_out[i] = (int32_t)overflow_id;
    } else {
      ids_out[i] = (int32_t)L[(key & mhi) >> lo];
    }
  }
  free(h); free(l); free(all); free(hs); free(L); free(Hid);
  return ne + 1;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3: DTMerge.                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t *k;
  uint64_t *v;
} rec_arr_t;

static void rec_swap(rec_arr_t a, int64_t i, int64_t j) {
  uint64_t t = a.k[i]; a.k[i] = a.k[j]; a.k[j] = t;
  if (a.v) { t = a.v[i]; a.v[i] = a.v[j]; a.v[j] = t; }
}

/* flip (reverse) a[s, e) */
static void rec_flip(rec_arr_t a, int64_t s, int64_t e) {
  for (int64_t i = s, j = e - 1; i < j; ++i, --j) rec_swap(a, i, j);
}

/* # keys in sorted b0[0..n0) that are < x */
static int64_t lower_bound_u64(const uint64_t *b0, int64_t n0, uint64_t x) {
  int64_t lo = 0, hi = n0;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (b0[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

/* One MSD zone, in place: keys/vals[0..n0) is the sorted light bucket B0,
 * followed by m heavy buckets B_1..B_m of sizes hsize[] with keys hkey[]
 * (increasing).  vals may be NULL.  On return the zone is sorted.
 * *copied_out receives the number of records copied out of place to T. */
int oracle_dtmerge_u64(uint64_t *keys, uint64_t *vals, int64_t n0, int64_t m,
                       const uint64_t *hkey, const int64_t *hsize,
                       int64_t *copied_out) {
  rec_arr_t A = {keys, vals};
  int64_t nh = 0;
  for (int64_t i = 0; i < m; ++i) nh += hsize[i];
  int64_t total = n0 + nh;
  /* binary search every heavy key in B0: lb[i] light keys precede B_i, and
   * p[i] = lb[i] + sum_{i' < i} |B_i'| is where B_i starts when sorted */
  int64_t *lb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 2));
  int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
  if (!lb || !p || !cur) { free(lb); free(p); free(cur); return -1; }
  int64_t before = 0;
  for (int64_t i = 0; i < m; ++i) {
    lb[i] = lower_bound_u64(keys, n0, hkey[i]);
    p[i] = lb[i] + before;
    cur[i] = n0 + before;
    before += hsize[i];
  }
  int64_t ncopy = n0 <= nh ? n0 : nh;
  uint64_t *Tk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ncopy + 1));
  uint64_t *Tv = vals ? (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ncopy + 1)) : NULL;
  if (!Tk || (vals && !Tv)) { free(lb); free(p); free(cur); free(Tk); free(Tv); return -1; }
  if (n0 <= nh) {
    /* more heavy records than light: copy B0 to T */
    memcpy(Tk, keys, sizeof(uint64_t) * (size_t)n0);
    if (vals) memcpy(Tv, vals, sizeof(uint64_t) * (size_t)n0);
    for (int64_t i = 0; i < m; ++i) {
      int64_t s = cur[i], sz = hsize[i], d = p[i];
      if (d == s) continue;
      if (d + sz > s) {
        /* destination overlaps the bucket itself: two flips rotate it */
        rec_flip(A, s, s + sz);
        rec_flip(A, d, s + sz);
      } else {
        for (int64_t j = 0; j < sz; ++j) {
          keys[d + j] = keys[s + j];
          if (vals) vals[d + j] = vals[s + j];
        }
      }
    }
    /* light records from T to their final positions */
    int64_t i = 0, add = 0;
    for (int64_t j = 0; j < n0; ++j) {
      while (i < m && hkey[i] < Tk[j]) add += hsize[i++];
      keys[j + add] = Tk[j];
      if (vals) vals[j + add] = Tv[j];
    }
  } else {
    /* symmetric case: copy the heavy buckets out, move the light blocks
     * (B0 cut by the heavy keys) to their places starting from the last
     * block, then copy the heavy buckets back */
    memcpy(Tk, keys + n0, sizeof(uint64_t) * (size_t)nh);
    if (vals) memcpy(Tv, vals + n0, sizeof(uint64_t) * (size_t)nh);
    lb[m] = n0;
    for (int64_t q = m; q >= 0; --q) {
      int64_t bs = q == 0 ? 0 : lb[q - 1];
      int64_t be = lb[q];
      int64_t shift = 0;
      for (int64_t i = 0; i < q; ++i) shift += hsize[i];
      int64_t sz = be - bs;
      if (shift == 0 || sz == 0) continue;
      if (bs + shift < be) {
        /* overlapping move to a later position: flip the block, then the
         * block plus the gap it moves into */
        rec_flip(A, bs, be);
        rec_flip(A, bs, be + shift);
      } else {
        for (int64_t j = sz - 1; j >= 0; --j) {
          keys[bs + shift + j] = keys[bs + j];
          if (vals) vals[bs + shift + j] = vals[bs + j];
        }
      }
    }
    int64_t off = 0;
    for (int64_t i = 0; i < m; ++i) {
      for (int64_t j = 0; j < hsize[i]; ++j) {
        keys[p[i] + j] = Tk[off + j];
        if (vals) vals[p[i] + j] = Tv[off + j];
      }
      off += hsize[i];
    }
  }
  if (copied_out) *copied_out = ncopy;
  (void)total;
  free(lb); free(p); free(cur); free(Tk); free(Tv);
  return 0;
}
