// C-ABI of dtsort (include/dtsort.h): argument checks, workspace layout and
// the one cooperative launch per sort call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include <sys/stat.h>

#include "../../include/dtsort.h"
#include "dtsort_launch.h"

namespace {

using dts::DevStats;
using dts::KernelShape;
using dts::Params;

constexpr int kOps = 4;

struct Layout {
  size_t tkeys, tvals, ctl, segs0, segs1, info, bcount, bstart, lid, heavy, hashk, hashid,
      cmat, status, tasks, zones, mhk, mhs, mhst, total;
  // learned bucketing (lrn_m == 0: digit zones)
  int64_t lrn_m;
  int lrn_B;
  size_t lsample, lws, lws_bytes, lx, lt, lparams, lpart, lspl, ltab, ldec;
  int64_t maxseg, bmax, hmax, zmax, hashmax, cwords, swords, tmax, mhmax;
  int cap;
  int64_t target;
};

struct Opts {
  int gamma_max, cap, heavy_on, heavy_min_share, merge_generic, sample_factor, debug_fault,
      blk_tiles;
  uint64_t seed;
  unsigned long long wait_ns;
};

}  // namespace

struct dtsort_handle_s {
  int device = 0;
  int nsm = 0;
  void *ctl_host = nullptr;  // pinned copy of the control block (phase launches)
  dtsort_options opt{};
  int *d_status = nullptr;
  DevStats *d_stats = nullptr;
  KernelShape shape[kOps]{};
  bool shape_ok[kOps]{};
  int64_t launches = 0;      // kernels launched by the last sort call
};

namespace {

int key_bytes(int op) { return (op == DTSORT_OP_U32 || op == DTSORT_OP_U32_KV) ? 4 : 8; }
bool has_vals(int op) { return op == DTSORT_OP_U32_KV || op == DTSORT_OP_U64_KV; }

cudaError_t get_shape(dtsort_handle h, int op, KernelShape **out) {
  if (!h->shape_ok[op]) {
    cudaError_t e;
    switch (op) {
      case DTSORT_OP_U32: e = dts::shape_u32(&h->shape[op]); break;
      case DTSORT_OP_U32_KV: e = dts::shape_u32kv(&h->shape[op]); break;
      case DTSORT_OP_U64: e = dts::shape_u64(&h->shape[op]); break;
      default: e = dts::shape_u64kv(&h->shape[op]); break;
    }
    if (e != cudaSuccess) return e;
    h->shape_ok[op] = true;
  }
  *out = &h->shape[op];
  return cudaSuccess;
}

// nsegs: arrays in the call (a batch of several gets 4-tile blocks by default:
// its small arrays fill large blocks badly; a single array gets ks.blk).
Opts effective(const dtsort_options &o, const KernelShape &ks, int64_t nsegs = 1) {
  Opts r;
  r.gamma_max = o.gamma_max > 0 ? o.gamma_max : dts::GAMMA_HW;
  r.cap = (o.finisher_capacity > 0 && o.finisher_capacity < ks.fin_cap) ? o.finisher_capacity
                                                                        : ks.fin_cap;
  r.heavy_on = o.heavy_detection >= 0 ? 1 : 0;
  r.heavy_min_share = o.heavy_min_share == 0 ? dts::HEAVY_MIN_SHARE
                                             : (o.heavy_min_share < 0 ? 0 : o.heavy_min_share);
  r.merge_generic = o.merge == DTSORT_MERGE_GENERIC ? 1 : 0;
  r.sample_factor = o.sample_log_factor > 0 ? o.sample_log_factor : 1;
  r.seed = o.seed ? o.seed : 1;
  r.debug_fault = o.debug_fault;
  r.blk_tiles = o.block_tiles > 0 ? o.block_tiles
                                   : (nsegs > 1 ? std::min(4, ks.blk / ks.tile) : ks.blk / ks.tile);
  r.wait_ns = (unsigned long long)(o.wait_limit_ms > 0 ? o.wait_limit_ms : 2000) * 1000000ull;
  return r;
}

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

// Upper bounds of every device table for n records in nsegs arrays.  The
// digit width rule gives 2^gamma < 8*size/target for every subproblem
// (size > cap > target), which bounds the per-level sums below.
Layout make_layout(int kb, int vb, int64_t n, int64_t nsegs, const Opts &o,
                   const KernelShape &ks) {
  Layout L{};
  L.cap = o.cap;
  L.target = std::max<int64_t>(16, (int64_t)o.cap * 85 / 100);  // bucket size the levels aim at
  const int64_t nt = n / L.target + 1;
  L.maxseg = n / (o.cap + 1) + 2;
  // per subproblem 2^gamma < 8 * size / target: buckets <= 1.5 * 2^gamma + 1,
  // heavy keys <= 2^(gamma-1), light-table entries 2^gamma + 1
  L.bmax = 12 * nt + L.maxseg + 1024;
  L.hmax = 4 * nt + L.maxseg + 1024;
  L.zmax = 8 * nt + 2 * L.maxseg + 1024;
  L.hashmax = 16 * nt + 2 * L.maxseg + 1024;  // 2^(gamma+1) slots per subproblem
  // count matrix: one row of <= NB_HW words per block of every subproblem;
  // look-back status: one row per chunk of ks.ch rows
  const int64_t blk = (int64_t)o.blk_tiles * ks.tile;
  L.cwords = (int64_t)dts::NB_HW * (n / blk + 1) + L.bmax;
  L.swords = (int64_t)dts::NB_HW * (n / (blk * ks.ch) + 1) + L.bmax;
  L.tmax = 2 * L.bmax + 2 * (n / dts::COPY_CHUNK + 1) + nsegs + 4096;
  L.mhmax = 4 * L.hmax + 4096;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = up(off + bytes);
    return r;
  };
  L.tkeys = take((size_t)n * kb);
  L.tvals = take((size_t)n * vb);
  L.ctl = take(sizeof(dts::Ctl));
  L.segs0 = take(sizeof(dts::Seg) * (size_t)L.maxseg);
  L.segs1 = take(sizeof(dts::Seg) * (size_t)L.maxseg);
  L.info = take(sizeof(dts::SegInfo) * (size_t)L.maxseg);
  L.bcount = take(8 * (size_t)L.bmax);
  L.bstart = take(8 * (size_t)L.bmax);
  L.lid = take(4 * (size_t)L.zmax);
  L.heavy = take((size_t)kb * L.hmax);
  L.hashk = take((size_t)kb * L.hashmax);
  L.hashid = take(2 * (size_t)L.hashmax);
  L.cmat = take(4 * (size_t)L.cwords);
  L.status = take(8 * (size_t)L.swords);
  L.tasks = take(sizeof(dts::Task) * (size_t)L.tmax);
  L.zones = take(sizeof(dts::MZone) * (size_t)L.mhmax);
  L.mhk = take((size_t)kb * L.mhmax);
  L.mhs = take(8 * (size_t)L.mhmax);
  L.mhst = take(8 * (size_t)L.mhmax);
  L.total = off;
  return L;
}

constexpr int64_t kLrnMinN = (int64_t)1 << 20;   // smaller arrays use digit zones
constexpr int kLrnBatch = 8192;
// extra cost of the learned level 0 over a digit level 0, in distribution
// passes per record: its histogram and scatter locate each key by the model
// and the boundaries (measured on 10^9 u64 key/value pairs of the skewed
// mixture: histograms 9.2 -> 15.3 ms, scatters 29.7 -> 37.7 ms, about one
// pass of those records)
constexpr double kLrnPenalty = 1.0;

// Host copy of the device digit-width rule (plan_gamma), for the number of
// learned zones at level 0.
int plan_gamma_host(int64_t s, int64_t target, int gmax, int hi, int fin_dig) {
  int e = 0;
  while (e < 62 && (target << e) < s) ++e;
  if (e < 1) e = 1;
  const int nlev = (e + gmax - 1) / gmax;
  int g = (e + nlev - 1) / nlev;
  g = g < 1 ? 1 : (g > gmax ? gmax : g);
  if (nlev == 1 && hi > g) {
    int best = g, bestp = (hi - g + fin_dig - 1) / fin_dig;
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

// Distribution levels of a uniformly distributed array of n keys of
// key_bits bits under the device's digit-width rule (an estimate for skewed
// inputs; the persistent kernel takes any further levels).
int predict_levels(int64_t n, int key_bits, const Opts &o, int64_t target) {
  int64_t s = n;
  int hi = key_bits, lv = 0;
  while (s > o.cap && hi > 0 && lv < 6) {
    const int g = plan_gamma_host(s, target, std::min(o.gamma_max, dts::GAMMA_HW), hi,
                                  dts::FIN_DIG);
    s = (s + ((int64_t)1 << g) - 1) >> g;
    hi -= g;
    ++lv;
  }
  return lv;
}

// Appends the learned-bucketing region to a layout: the model sample (about
// 1% of the keys), a workspace to sort it, features/targets, parameters and
// Adam moments, gradient partials, zone boundaries and the prediction table.
void add_learned(Layout &L, int kb, int64_t n, const Opts &o, const KernelShape &ks_u64) {
  int64_t m = n / 100;
  m = std::max<int64_t>(m, (int64_t)1 << 16);
  m = std::min<int64_t>(m, (int64_t)1 << 24);
  m = (m / kLrnBatch) * kLrnBatch;
  L.lrn_m = m;
  L.lrn_B = 1 << plan_gamma_host(n, L.target, std::min(o.gamma_max, dts::GAMMA_HW), 8 * kb,
                                 dts::FIN_DIG);
  Opts od = o;
  od.cap = ks_u64.fin_cap;
  od.blk_tiles = ks_u64.blk / ks_u64.tile;
  const Layout S = make_layout(8, 0, m, 1, od, ks_u64);
  size_t off = L.total;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = up(off + bytes);
    return r;
  };
  L.lsample = take(8 * (size_t)m);
  L.lws_bytes = S.total;
  L.lws = take(S.total);
  L.lx = take(4 * (size_t)m);
  L.lt = take(4 * (size_t)m);
  L.lparams = take(4 * 3 * 352);
  L.lpart = take(4 * (size_t)(kLrnBatch / 256) * 352);
  L.lspl = take((size_t)kb * 1024);
  L.ltab = take(4 * 1024);
  L.ldec = take(64);  // decision flag + two estimates
  L.total = off;
}

dtsort_status from_cuda(cudaError_t e) {
  return e == cudaSuccess ? DTSORT_OK : DTSORT_ERR_CUDA;
}

// ---------------------------------------------------------------- autotune
// Cache of tuned settings, keyed by (GPU name, op, log2 n, log2 arrays).
struct TuneKey {
  std::string gpu;
  int op, ln, ls;
  bool operator<(const TuneKey &o) const {
    if (gpu != o.gpu) return gpu < o.gpu;
    if (op != o.op) return op < o.op;
    if (ln != o.ln) return ln < o.ln;
    return ls < o.ls;
  }
};
struct TuneVal {
  int gamma_max, cap, block_tiles, sample_factor;
  double ms;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
  const char *e = std::getenv("DTSORT_AUTOTUNE_CACHE");
  if (e && *e) return e;
  const char *home = std::getenv("HOME");
  return std::string(home ? home : ".") + "/.cache/dtsort_autotune.tsv";
}

int log2_class(int64_t x) {
  int l = 0;
  while (l < 62 && ((int64_t)1 << (l + 1)) <= x) ++l;
  return l;
}

std::string gpu_name(int device) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "unknown";
  std::string s(p.name);
  for (char &ch : s)
    if (ch == '\t' || ch == '\n') ch = ' ';
  return s;
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE *f = std::fopen(tune_path().c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    char gpu[256];
    int op, ln, ls, g, cap, bt, sf;
    double ms;
    if (std::sscanf(line, "%255[^\t]\t%d\t%d\t%d\t%d\t%d\t%d\t%d\t%lf", gpu, &op, &ln, &ls, &g,
                    &cap, &bt, &sf, &ms) == 9)
      g_tune[TuneKey{gpu, op, ln, ls}] = TuneVal{g, cap, bt, sf, ms};
  }
  std::fclose(f);
}

void tune_store(const TuneKey &k, const TuneVal &v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  g_tune[k] = v;
  const std::string path = tune_path();
  const std::string dir = path.substr(0, path.find_last_of('/'));
  if (!dir.empty() && dir != path) {
    std::string cmd = dir;  // create the directory without a shell
    for (size_t i = 1; i <= cmd.size(); ++i)
      if (i == cmd.size() || cmd[i] == '/') {
        const std::string part = cmd.substr(0, i);
        mkdir(part.c_str(), 0755);
      }
  }
  FILE *f = std::fopen(path.c_str(), "w");
  if (!f) return;
  for (const auto &kv : g_tune)
    std::fprintf(f, "%s\t%d\t%d\t%d\t%d\t%d\t%d\t%d\t%.6f\n", kv.first.gpu.c_str(),
                 kv.first.op, kv.first.ln, kv.first.ls, kv.second.gamma_max, kv.second.cap,
                 kv.second.block_tiles, kv.second.sample_factor, kv.second.ms);
  std::fclose(f);
}

// The handle's options, with the cached tuned setting applied when
// options.autotune is set and the cache holds one for this problem class.
dtsort_options tuned_options(dtsort_handle h, int op, int64_t n, int64_t nsegs) {
  dtsort_options o = h->opt;
  if (o.autotune != 1) return o;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(TuneKey{gpu_name(h->device), op, log2_class(n), log2_class(nsegs)});
  if (it == g_tune.end()) return o;
  o.gamma_max = it->second.gamma_max;
  o.finisher_capacity = it->second.cap;
  o.block_tiles = it->second.block_tiles;
  o.sample_log_factor = it->second.sample_factor;
  return o;
}

dtsort_status run_sort(dtsort_handle h, int op, void *keys, void *vals, const int64_t *offsets,
                       int64_t nsegs, int64_t n, void *ws, size_t ws_bytes, cudaStream_t s,
                       bool allow_learned = true) {
  if (!h) return DTSORT_ERR_INVALID_ARG;
  if (allow_learned) h->launches = 0;  // a top-level call
  if (n < 0 || nsegs < 0) return DTSORT_ERR_INVALID_ARG;
  if (offsets && nsegs == 0) return n == 0 ? DTSORT_OK : DTSORT_ERR_INVALID_ARG;
  if (n == 0) return DTSORT_OK;
  if (n >= ((int64_t)1 << 32)) return DTSORT_ERR_UNSUPPORTED;  // 32-bit block offsets
  if (!keys || (has_vals(op) && !vals) || !ws) return DTSORT_ERR_INVALID_ARG;
  const int kb = key_bytes(op), vb = has_vals(op) ? kb : 0;
  if (((uintptr_t)keys % kb) || (vals && ((uintptr_t)vals % kb)) || ((uintptr_t)ws % 256))
    return DTSORT_ERR_INVALID_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return DTSORT_ERR_CUDA;
  KernelShape *ks = nullptr;
  cudaError_t e = get_shape(h, op, &ks);
  if (e != cudaSuccess) return DTSORT_ERR_CUDA;
  if (ks->blocks_per_sm < 1) return DTSORT_ERR_UNSUPPORTED;
  const Opts o = effective(tuned_options(h, op, n, offsets ? nsegs : 1), *ks, offsets ? nsegs : 1);
  Layout L = make_layout(kb, vb, n, offsets ? nsegs : 1, o, *ks);
  const bool learned = allow_learned &&
                       (h->opt.bucketing == DTSORT_BUCKETING_LEARNED ||
                        h->opt.bucketing == DTSORT_BUCKETING_LEARNED_ALWAYS) &&
                       !offsets && n >= kLrnMinN;
  KernelShape *ks64 = nullptr;
  if (learned) {
    if (get_shape(h, DTSORT_OP_U64, &ks64) != cudaSuccess) return DTSORT_ERR_CUDA;
    add_learned(L, kb, n, o, *ks64);
  }
  if (ws_bytes < L.total) return DTSORT_ERR_WORKSPACE_TOO_SMALL;
  char *w = (char *)ws;
  Params P{};
  P.keys[0] = keys;
  P.keys[1] = w + L.tkeys;
  P.vals[0] = vb ? vals : nullptr;
  P.vals[1] = vb ? (void *)(w + L.tvals) : nullptr;
  P.n = n;
  P.offsets = offsets;
  P.nsegs_in = offsets ? nsegs : 1;
  P.key_bits = 8 * kb;
  P.gamma_max = std::min(o.gamma_max, dts::GAMMA_HW);
  P.cap = L.cap;
  P.heavy_on = o.heavy_on;
  P.heavy_min_share = o.heavy_min_share;
  P.merge_generic = o.merge_generic;
  P.target = L.target;
  P.seed = o.seed;
  P.sample_factor = o.sample_factor;
  P.debug_fault = o.debug_fault;
  P.blk_tiles = o.blk_tiles;
  P.wait_ns = o.wait_ns;
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
  P.dev_status = h->d_status;
  P.stats = h->d_stats;
  P.lrn_B = 0;
  if (learned) {
    // fit the CDF model on ~1% of the keys and derive the level-0 zones:
    // sample, sort the sample (digit zones), features, Adam training,
    // boundaries + prediction table.  All on `s`, no host synchronisation.
    uint64_t *smp = (uint64_t *)(w + L.lsample);
    float *x = (float *)(w + L.lx), *t = (float *)(w + L.lt);
    float *prm = (float *)(w + L.lparams);
    const uint64_t lseed = o.seed ^ 0x4C6561726E6564ull;
    if ((e = dts::lrn_gather(keys, kb, n, lseed, smp, L.lrn_m, s)) != cudaSuccess)
      return DTSORT_ERR_CUDA;
    const dtsort_status st = run_sort(h, DTSORT_OP_U64, smp, nullptr, nullptr, 1, L.lrn_m,
                                      w + L.lws, L.lws_bytes, s, false);
    if (st != DTSORT_OK) return st;
    const int steps = h->opt.learned_train_steps > 0 ? h->opt.learned_train_steps : 200;
    // LEARNED: the device decides, from the sorted sample, whether learned
    // zones pay (level 0 reads its flag) -- first on zones at the sample's
    // quantiles (the best any CDF model can give), before any training: when
    // even those keep the digit zones, the model's features, training and
    // boundaries return at once; otherwise once more on the trained model's
    // zones.  ALWAYS: the model's zones are used.
    const bool decide = h->opt.bucketing == DTSORT_BUCKETING_LEARNED;
    int *on = decide ? (int *)(w + L.ldec) : nullptr;
    double *est = decide ? (double *)(w + L.ldec + 8) : nullptr;
    const int gmx = std::min(o.gamma_max, dts::GAMMA_HW);
    if (decide) {
      if ((e = dts::lrn_quantiles(smp, L.lrn_m, kb, L.lrn_B, w + L.lspl, s)) != cudaSuccess ||
          (e = dts::lrn_decide(smp, L.lrn_m, n, kb, L.lrn_B, w + L.lspl, L.cap, L.target, gmx,
                               kLrnPenalty, on, est, nullptr, s)) != cudaSuccess)
        return DTSORT_ERR_CUDA;
      h->launches += 2;
    }
    if ((e = dts::lrn_features(smp, L.lrn_m, 8 * kb, x, t, on, s)) != cudaSuccess ||
        (e = dts::lrn_init(prm, prm + 352, prm + 704, lseed, on, s)) != cudaSuccess ||
        (e = dts::lrn_train(prm, prm + 352, prm + 704, x, t, L.lrn_m, steps, kLrnBatch, 1e-2f,
                            (float *)(w + L.lpart), on, s)) != cudaSuccess ||
        (e = dts::lrn_splitters(prm, L.lrn_B, kb, w + L.lspl, (float *)(w + L.ltab), on,
                                s)) != cudaSuccess)
      return DTSORT_ERR_CUDA;
    h->launches += 4 + 2 * (int64_t)steps;  // gather, features, init, training, boundaries
    if (decide) {
      if ((e = dts::lrn_decide(smp, L.lrn_m, n, kb, L.lrn_B, w + L.lspl, L.cap, L.target, gmx,
                               kLrnPenalty, on, est, on, s)) != cudaSuccess)
        return DTSORT_ERR_CUDA;
      h->launches += 1;
    }
    P.lrn_B = L.lrn_B;
    P.lrn_spl = w + L.lspl;
    P.lrn_tab = (const float *)(w + L.ltab);
    P.lrn_on = on;
    P.lrn_est = est;
  }
  e = cudaMemsetAsync(P.ctl, 0, sizeof(dts::Ctl), s);
  if (e != cudaSuccess) return DTSORT_ERR_CUDA;
  const int grid = h->nsm * std::min(ks->blocks_per_sm, 2);
  if (h->opt.launch_mode == 1) {
    if (!h->ctl_host && cudaMallocHost(&h->ctl_host, sizeof(dts::Ctl)) != cudaSuccess)
      return DTSORT_ERR_CUDA;
    int cnt = 0;
    switch (op) {
      case DTSORT_OP_U32: e = dts::launch_split_u32(P, grid, s, h->ctl_host, &cnt); break;
      case DTSORT_OP_U32_KV: e = dts::launch_split_u32kv(P, grid, s, h->ctl_host, &cnt); break;
      case DTSORT_OP_U64: e = dts::launch_split_u64(P, grid, s, h->ctl_host, &cnt); break;
      default: e = dts::launch_split_u64kv(P, grid, s, h->ctl_host, &cnt); break;
    }
    h->launches += cnt;
    return from_cuda(e);
  }
  // the levels a uniform input of n keys needs, and for n >= 2^26 two more
  // for skewed inputs, run as separate phase launches, the rest (if any) in
  // the persistent kernel; for a segmented call n (the total) bounds every
  // array's size.  A queued level without work returns at once on the device
  // (two unused levels cost nothing measurable on 10^9 uniform keys; skewed
  // inputs gain 4-9%, their deeper levels then running in the per-phase
  // kernels, which spill less than the persistent one; below 2^26 records the
  // sort is launch-bound and the empty launches would show)
  const int extra = n >= ((int64_t)1 << 26) ? 2 : 0;
  const int head =
      h->opt.launch_mode == 0 ? predict_levels(n, 8 * kb, o, L.target) + extra : 0;
  switch (op) {
    case DTSORT_OP_U32: e = dts::launch_u32(P, grid, head, *ks, h->nsm, s); break;
    case DTSORT_OP_U32_KV: e = dts::launch_u32kv(P, grid, head, *ks, h->nsm, s); break;
    case DTSORT_OP_U64: e = dts::launch_u64(P, grid, head, *ks, h->nsm, s); break;
    default: e = dts::launch_u64kv(P, grid, head, *ks, h->nsm, s); break;
  }
  // the persistent kernel; with queued levels also the seed, 7 phases and 2
  // merge phases per level, and the statistics
  h->launches += 1 + (head > 0 ? 2 + 9 * (int64_t)head : 0);
  return from_cuda(e);
}

}  // namespace

extern "C" {

const char *dtsort_status_string(dtsort_status s) {
  switch (s) {
    case DTSORT_OK: return "DTSORT_OK";
    case DTSORT_ERR_INVALID_ARG: return "DTSORT_ERR_INVALID_ARG: invalid argument";
    case DTSORT_ERR_WORKSPACE_TOO_SMALL: return "DTSORT_ERR_WORKSPACE_TOO_SMALL";
    case DTSORT_ERR_CUDA: return "DTSORT_ERR_CUDA: a CUDA runtime call failed";
    case DTSORT_ERR_DEVICE_TIMEOUT: return "DTSORT_ERR_DEVICE_TIMEOUT: a bounded device wait expired";
    case DTSORT_ERR_UNSUPPORTED: return "DTSORT_ERR_UNSUPPORTED: needs a compute capability 10.3 GPU";
    case DTSORT_ERR_INTERNAL: return "DTSORT_ERR_INTERNAL: an internal device table overflowed";
  }
  return "unknown dtsort status";
}

dtsort_status dtsort_default_options(dtsort_options *opt) {
  if (!opt) return DTSORT_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->gamma_max = dts::GAMMA_HW;
  opt->heavy_detection = 1;
  opt->bucketing = DTSORT_BUCKETING_DIGIT;
  opt->seed = 1;
  opt->sample_log_factor = 1;
  opt->learned_segments = 1024;
  opt->learned_train_steps = 200;
  opt->wait_limit_ms = 2000;
  return DTSORT_OK;
}

dtsort_status dtsort_create(dtsort_handle *out, int device) {
  if (!out) return DTSORT_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return count == 0 ? DTSORT_ERR_UNSUPPORTED : DTSORT_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return DTSORT_ERR_UNSUPPORTED;
  if (!prop.cooperativeLaunch) return DTSORT_ERR_UNSUPPORTED;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return DTSORT_ERR_CUDA;
  dtsort_handle h = new (std::nothrow) dtsort_handle_s();
  if (!h) return DTSORT_ERR_INTERNAL;
  h->device = device;
  h->nsm = prop.multiProcessorCount;
  dtsort_default_options(&h->opt);
  dtsort_status st = DTSORT_OK;
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_stats, sizeof(DevStats)) != cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(h->d_stats, 0, sizeof(DevStats)) != cudaSuccess) {
    st = DTSORT_ERR_CUDA;
  }
  if (cur >= 0) cudaSetDevice(cur);
  if (st != DTSORT_OK) {
    cudaFree(h->d_status);
    cudaFree(h->d_stats);
    delete h;
    return st;
  }
  *out = h;
  return DTSORT_OK;
}

dtsort_status dtsort_destroy(dtsort_handle h) {
  if (!h) return DTSORT_ERR_INVALID_ARG;
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  cudaFree(h->d_status);
  cudaFree(h->d_stats);
  delete h;
  return DTSORT_OK;
}

dtsort_status dtsort_set_options(dtsort_handle h, const dtsort_options *opt) {
  if (!h) return DTSORT_ERR_INVALID_ARG;
  if (!opt) return dtsort_default_options(&h->opt);
  if (opt->gamma_max < 0 || opt->gamma_max > dts::GAMMA_HW || opt->finisher_capacity < 0 ||
      opt->sample_log_factor < 0 || opt->sample_log_factor > 64 ||
      (opt->bucketing != DTSORT_BUCKETING_DIGIT && opt->bucketing != DTSORT_BUCKETING_LEARNED &&
       opt->bucketing != DTSORT_BUCKETING_LEARNED_ALWAYS) ||
      opt->learned_segments < 0 || opt->learned_train_steps < 0 || opt->wait_limit_ms < 0 ||
      opt->debug_fault < 0 || opt->debug_fault > 1 || opt->launch_mode < 0 ||
      opt->launch_mode > 2 || opt->block_tiles < 0 || opt->block_tiles > 8 ||
      (opt->merge != DTSORT_MERGE_DOVETAIL && opt->merge != DTSORT_MERGE_GENERIC) ||
      opt->heavy_min_share < -1 || opt->heavy_min_share > 1000)
    return DTSORT_ERR_INVALID_ARG;
  h->opt = *opt;
  return DTSORT_OK;
}

dtsort_status dtsort_get_options(dtsort_handle h, dtsort_options *opt) {
  if (!h || !opt) return DTSORT_ERR_INVALID_ARG;
  *opt = h->opt;
  return DTSORT_OK;
}

dtsort_status dtsort_workspace_bytes(dtsort_handle h, dtsort_op op, int64_t n,
                                     int64_t num_segments, size_t *bytes) {
  if (!h || !bytes || n < 0 || num_segments < 0 || (int)op < 0 || (int)op >= kOps)
    return DTSORT_ERR_INVALID_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return DTSORT_ERR_CUDA;
  KernelShape *ks = nullptr;
  if (get_shape(h, op, &ks) != cudaSuccess) return DTSORT_ERR_CUDA;
  const int64_t ns = num_segments > 0 ? num_segments : 1;
  const int kb = key_bytes(op), vb = has_vals(op) ? kb : 0;
  // the larger of the single-array and the batch default block sizes, so that
  // a call of either kind fits
  const dtsort_options to = tuned_options(h, op, n, ns);
  Layout L = make_layout(kb, vb, n, ns, effective(to, *ks, 1), *ks);
  {
    const Layout L2 = make_layout(kb, vb, n, ns, effective(to, *ks, 2), *ks);
    if (L2.total > L.total) L = L2;
  }
  const Opts o = effective(to, *ks, ns);
  if ((h->opt.bucketing == DTSORT_BUCKETING_LEARNED ||
       h->opt.bucketing == DTSORT_BUCKETING_LEARNED_ALWAYS) &&
      n >= kLrnMinN) {
    KernelShape *ks64 = nullptr;
    if (get_shape(h, DTSORT_OP_U64, &ks64) != cudaSuccess) return DTSORT_ERR_CUDA;
    add_learned(L, kb, n, o, *ks64);
  }
  *bytes = L.total;
  return DTSORT_OK;
}

dtsort_status dtsort_u32(dtsort_handle h, uint32_t *keys, int64_t n, void *ws, size_t wsb,
                         dtsort_stream s) {
  return run_sort(h, DTSORT_OP_U32, keys, nullptr, nullptr, 1, n, ws, wsb, (cudaStream_t)s);
}
dtsort_status dtsort_u32_kv(dtsort_handle h, uint32_t *keys, uint32_t *values, int64_t n,
                            void *ws, size_t wsb, dtsort_stream s) {
  return run_sort(h, DTSORT_OP_U32_KV, keys, values, nullptr, 1, n, ws, wsb, (cudaStream_t)s);
}
dtsort_status dtsort_u64(dtsort_handle h, uint64_t *keys, int64_t n, void *ws, size_t wsb,
                         dtsort_stream s) {
  return run_sort(h, DTSORT_OP_U64, keys, nullptr, nullptr, 1, n, ws, wsb, (cudaStream_t)s);
}
dtsort_status dtsort_u64_kv(dtsort_handle h, uint64_t *keys, uint64_t *values, int64_t n,
                            void *ws, size_t wsb, dtsort_stream s) {
  return run_sort(h, DTSORT_OP_U64_KV, keys, values, nullptr, 1, n, ws, wsb, (cudaStream_t)s);
}

dtsort_status dtsort_segmented_u32(dtsort_handle h, uint32_t *keys, const int64_t *off,
                                   int64_t ns, int64_t n, void *ws, size_t wsb,
                                   dtsort_stream s) {
  if (!off && n > 0) return DTSORT_ERR_INVALID_ARG;
  return run_sort(h, DTSORT_OP_U32, keys, nullptr, off, ns, n, ws, wsb, (cudaStream_t)s);
}
dtsort_status dtsort_segmented_u32_kv(dtsort_handle h, uint32_t *keys, uint32_t *values,
                                      const int64_t *off, int64_t ns, int64_t n, void *ws,
                                      size_t wsb, dtsort_stream s) {
  if (!off && n > 0) return DTSORT_ERR_INVALID_ARG;
  return run_sort(h, DTSORT_OP_U32_KV, keys, values, off, ns, n, ws, wsb, (cudaStream_t)s);
}
dtsort_status dtsort_segmented_u64(dtsort_handle h, uint64_t *keys, const int64_t *off,
                                   int64_t ns, int64_t n, void *ws, size_t wsb,
                                   dtsort_stream s) {
  if (!off && n > 0) return DTSORT_ERR_INVALID_ARG;
  return run_sort(h, DTSORT_OP_U64, keys, nullptr, off, ns, n, ws, wsb, (cudaStream_t)s);
}
dtsort_status dtsort_segmented_u64_kv(dtsort_handle h, uint64_t *keys, uint64_t *values,
                                      const int64_t *off, int64_t ns, int64_t n, void *ws,
                                      size_t wsb, dtsort_stream s) {
  if (!off && n > 0) return DTSORT_ERR_INVALID_ARG;
  return run_sort(h, DTSORT_OP_U64_KV, keys, values, off, ns, n, ws, wsb, (cudaStream_t)s);
}

dtsort_status dtsort_sort_host(dtsort_handle h, dtsort_op op, void *keys_host, void *values_host,
                               int64_t n, void *dev_keys, void *dev_values, void *ws, size_t wsb,
                               dtsort_stream stream) {
  if (!h || op < 0 || op >= kOps || n < 0) return DTSORT_ERR_INVALID_ARG;
  if (n == 0) return DTSORT_OK;
  const bool hv = has_vals(op);
  if (!keys_host || !dev_keys || (hv && (!values_host || !dev_values)) ||
      (!hv && (values_host || dev_values)))
    return DTSORT_ERR_INVALID_ARG;
  const size_t bytes = (size_t)n * key_bytes(op);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(dev_keys, keys_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (hv && cudaMemcpyAsync(dev_values, values_host, bytes, cudaMemcpyHostToDevice, s) !=
                 cudaSuccess))
    return DTSORT_ERR_CUDA;
  const dtsort_status st =
      run_sort(h, op, dev_keys, hv ? dev_values : nullptr, nullptr, 1, n, ws, wsb, s);
  if (st != DTSORT_OK) return st;
  if (cudaMemcpyAsync(keys_host, dev_keys, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (hv && cudaMemcpyAsync(values_host, dev_values, bytes, cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess))
    return DTSORT_ERR_CUDA;
  return DTSORT_OK;
}

dtsort_status dtsort_last_device_error(dtsort_handle h, dtsort_stream s) {
  if (!h) return DTSORT_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess) return DTSORT_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DTSORT_ERR_CUDA;
  if (v && cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) return DTSORT_ERR_CUDA;
  return (dtsort_status)v;
}

dtsort_status dtsort_get_stats(dtsort_handle h, dtsort_stats *out) {
  if (!h || !out) return DTSORT_ERR_INVALID_ARG;
  DevStats d;
  if (cudaDeviceSynchronize() != cudaSuccess) return DTSORT_ERR_CUDA;
  if (cudaMemcpy(&d, h->d_stats, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DTSORT_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->levels = d.levels;
  out->status = d.status;
  for (int l = 0; l < 16; ++l) {
    out->segments[l] = d.segments[l];
    out->records[l] = d.records[l];
    out->heavy_keys[l] = d.heavy_keys[l];
    out->heavy_records[l] = d.heavy_records[l];
    out->overflow_records[l] = d.overflow_records[l];
  }
  out->finisher_tasks = d.finisher_tasks;
  out->finisher_records = d.finisher_records;
  out->copy_records = d.copy_records;
  out->merge_zones = d.merge_zones;
  out->merge_records = d.merge_records;
  out->learned_fixup_records = d.learned_fixup_records;
  out->learned_fixup_steps = d.learned_fixup_steps;
  out->learned_bucket_cv = d.learned_cv;
  out->learned_bucket_max_over_mean = d.learned_mom;
  for (int k = 0; k < 8; ++k) out->phase_ms[k] = d.phase_ms[k];
  out->finisher_lsd_tasks = d.fin_lsd_tasks;
  out->kernel_launches = h->launches;
  out->learned_zones_used = d.learned_used;
  out->learned_estimate[0] = d.learned_est[0];
  out->learned_estimate[1] = d.learned_est[1];
  out->merge_free_zones = d.free_zones;
  out->check_site = d.check_site;
  out->check_values[0] = d.check_values[0];
  out->check_values[1] = d.check_values[1];
  return DTSORT_OK;
}

// Candidate settings tried by the autotuner.
static const int kTuneGamma[] = {7, 8, 9};
static const int kTuneCapDiv[] = {4, 3, 2};  // capacity = fin_cap * 2 / div
static const int kTuneBlk[] = {4, 8};

dtsort_status dtsort_autotune_scratch_bytes(dtsort_handle h, dtsort_op op, int64_t n,
                                            int64_t num_segments, size_t *bytes) {
  if (!h || !bytes || n < 0 || num_segments < 0 || (int)op < 0 || (int)op >= kOps)
    return DTSORT_ERR_INVALID_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return DTSORT_ERR_CUDA;
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return DTSORT_ERR_CUDA;
  KernelShape *ks = nullptr;
  if (get_shape(h, op, &ks) != cudaSuccess) return DTSORT_ERR_CUDA;
  const int kb = key_bytes(op), vb = has_vals(op) ? kb : 0;
  size_t ws = 0;
  for (int g : kTuneGamma)
    for (int cd : kTuneCapDiv)
      for (int bt : kTuneBlk) {
        dtsort_options o = h->opt;
        o.gamma_max = g;
        o.finisher_capacity = ks->fin_cap * 2 / cd;
        o.block_tiles = bt;
        const Opts e = effective(o, *ks);
        ws = std::max(ws, make_layout(kb, vb, n, num_segments > 0 ? num_segments : 1, e, *ks).total);
      }
  *bytes = up((size_t)n * kb) + up((size_t)n * vb) + ws;
  return DTSORT_OK;
}

dtsort_status dtsort_autotune(dtsort_handle h, dtsort_op op, const void *keys, const void *values,
                              const int64_t *offsets, int64_t num_segments, int64_t n,
                              void *scratch, size_t scratch_bytes, dtsort_stream stream,
                              dtsort_options *best_out) {
  if (!h || (int)op < 0 || (int)op >= kOps || n <= 0 || !keys || !scratch ||
      (has_vals(op) && !values) || (offsets && num_segments <= 0) || ((uintptr_t)scratch % 256))
    return DTSORT_ERR_INVALID_ARG;
  size_t need = 0;
  dtsort_status st = dtsort_autotune_scratch_bytes(h, op, n, offsets ? num_segments : 1, &need);
  if (st != DTSORT_OK) return st;
  if (scratch_bytes < need) return DTSORT_ERR_WORKSPACE_TOO_SMALL;
  KernelShape *ks = nullptr;
  if (get_shape(h, op, &ks) != cudaSuccess) return DTSORT_ERR_CUDA;
  const int kb = key_bytes(op), vb = has_vals(op) ? kb : 0;
  char *w = (char *)scratch;
  void *ck = w;
  void *cv = vb ? (void *)(w + up((size_t)n * kb)) : nullptr;
  void *ws = w + up((size_t)n * kb) + up((size_t)n * vb);
  const size_t wsb = scratch_bytes - up((size_t)n * kb) - up((size_t)n * vb);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return DTSORT_ERR_CUDA;
  const dtsort_options saved = h->opt;
  dtsort_options best = saved;
  double best_ms = 1e30;
  for (int g : kTuneGamma)
    for (int cd : kTuneCapDiv)
      for (int bt : kTuneBlk) {
        dtsort_options o = saved;
        o.autotune = 0;
        o.gamma_max = g;
        o.finisher_capacity = ks->fin_cap * 2 / cd;
        o.block_tiles = bt;
        h->opt = o;
        double tmin = 1e30;
        for (int rep = 0; rep < 2 && st == DTSORT_OK; ++rep) {
          if (cudaMemcpyAsync(ck, keys, (size_t)n * kb, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
              (vb && cudaMemcpyAsync(cv, values, (size_t)n * vb, cudaMemcpyDeviceToDevice, s) !=
                         cudaSuccess)) {
            st = DTSORT_ERR_CUDA;
            break;
          }
          cudaEventRecord(e0, s);
          st = run_sort(h, op, ck, cv, offsets, offsets ? num_segments : 1, n, ws, wsb, s);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) st = DTSORT_ERR_CUDA;
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          tmin = std::min(tmin, (double)ms);
        }
        if (st != DTSORT_OK) break;
        if (tmin < best_ms) {
          best_ms = tmin;
          best = o;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->opt = saved;
  if (st != DTSORT_OK) return st;
  // a device-side failure during the trials voids the result
  int dev_st = 0;
  if (cudaMemcpy(&dev_st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DTSORT_ERR_CUDA;
  if (dev_st) return (dtsort_status)dev_st;
  h->opt.gamma_max = best.gamma_max;
  h->opt.finisher_capacity = best.finisher_capacity;
  h->opt.block_tiles = best.block_tiles;
  tune_store(TuneKey{gpu_name(h->device), (int)op, log2_class(n),
                     log2_class(offsets ? num_segments : 1)},
             TuneVal{best.gamma_max, best.finisher_capacity, best.block_tiles,
                     best.sample_log_factor > 0 ? best.sample_log_factor : 1, best_ms});
  if (best_out) *best_out = h->opt;
  return DTSORT_OK;
}

dtsort_status dtsort_debug_sample(dtsort_handle h, const void *keys, int key_bytes_,
                                  int64_t start, int64_t size, int hi, uint64_t seed,
                                  int64_t count, int64_t L, uint64_t *heavy_out,
                                  int64_t *nheavy_out, uint64_t *max_out, dtsort_stream s) {
  if (!h || !keys || !heavy_out || !nheavy_out || !max_out) return DTSORT_ERR_INVALID_ARG;
  if ((key_bytes_ != 4 && key_bytes_ != 8) || start < 0 || size <= 0 || count <= 0 ||
      count > dts::SMAX || L <= 0 || hi < 0 || hi > 8 * key_bytes_)
    return DTSORT_ERR_INVALID_ARG;
  cudaError_t e = key_bytes_ == 4
                      ? dts::launch_sample_u32(keys, start, size, hi, seed, count, L, heavy_out,
                                               nheavy_out, max_out, (cudaStream_t)s)
                      : dts::launch_sample_u64(keys, start, size, hi, seed, count, L, heavy_out,
                                               nheavy_out, max_out, (cudaStream_t)s);
  return from_cuda(e);
}

}  // extern "C"
