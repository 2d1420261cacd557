// Learned CDF bucketing: a 1 -> 16 -> 16 -> 1 tanh MLP, fit on a sample of
// the keys, proposes the level-0 zone boundaries; membership is then decided
// exactly by integer comparison with those boundaries, so the sort's output
// does not depend on the model.
//
// Parameters (321 floats, the layout of the fp64 reference model):
//   W1[16] b1[16] W2[16][16] (W2[j][k] multiplies h1[k]) b2[16] W3[16] b3
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 . h2 + b3
// Feature of a key: x = log2(1 + key) / w (w = key bits).  Loss of a batch of
// B pairs (x, t): (1/B) sum (y - t)^2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dts {

constexpr int MLP_H = 16;
constexpr int MLP_NP = MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;  // 321
constexpr int MLP_OW1 = 0, MLP_OB1 = 16, MLP_OW2 = 32, MLP_OB2 = 288, MLP_OW3 = 304,
              MLP_OB3 = 320;
constexpr int MLP_BLK = 256;       // points per gradient block
constexpr int LRN_TAB = 512;       // cells of the per-key prediction table

__device__ __forceinline__ float mlp_feature(uint64_t key, int w) {
  return log2f((float)key + 1.0f) * (1.0f / (float)w);
}

// y = F(x) with parameters p (shared or global)
__device__ __forceinline__ float mlp_eval(const float *p, float x) {
  float h1[MLP_H];
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) h1[k] = tanhf(fmaf(p[MLP_OW1 + k], x, p[MLP_OB1 + k]));
  float y = p[MLP_OB3];
#pragma unroll 4
  for (int j = 0; j < MLP_H; ++j) {
    float z = p[MLP_OB2 + j];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) z = fmaf(p[MLP_OW2 + j * MLP_H + k], h1[k], z);
    y = fmaf(p[MLP_OW3 + j], tanhf(z), y);
  }
  return y;
}

// Forward for n points.
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float *__restrict__ params,
                                                          const float *__restrict__ x,
                                                          int64_t n, float *__restrict__ y) {
  __shared__ float p[MLP_NP];
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = mlp_eval(p, x[i]);
}

// Gradient of the batch loss.  Point i of the batch is x[idx(i)] with
// idx(i) = first + i * stride (mod m).  Block b handles points
// [b*256, (b+1)*256) of the batch and writes its partial gradient (sums in a
// fixed order, so the result is deterministic) to part[b][0..321); the loss
// contribution goes to part[b][321].
// en: NULL, or a device flag; 0 makes the kernel return at once (the model
// is not wanted).  The same holds for the other training kernels below.
__global__ void __launch_bounds__(MLP_BLK) mlp_grad_kernel(
    const float *__restrict__ params, const float *__restrict__ x, const float *__restrict__ t,
    int64_t m, int64_t first, int64_t stride, int64_t batch, float *__restrict__ part,
    const int *en) {
  if (en && !*en) return;
  __shared__ float p[MLP_NP];
  __shared__ float xs[MLP_BLK], dys[MLP_BLK], es[MLP_BLK];
  __shared__ float h1s[MLP_BLK][MLP_H + 1], h2s[MLP_BLK][MLP_H + 1];
  __shared__ float dz2s[MLP_BLK][MLP_H + 1], dz1s[MLP_BLK][MLP_H + 1];
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  const int tid = threadIdx.x;
  const int64_t bi = (int64_t)blockIdx.x * MLP_BLK + tid;
  const bool valid = bi < batch;
  float xv = 0.f, tv = 0.f;
  if (valid) {
    const int64_t idx = (first + bi * stride) % m;
    xv = x[idx];
    tv = t[idx];
  }
  float h1[MLP_H], h2[MLP_H];
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) h1[k] = tanhf(fmaf(p[MLP_OW1 + k], xv, p[MLP_OB1 + k]));
  float y = p[MLP_OB3];
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) {
    float z = p[MLP_OB2 + j];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) z = fmaf(p[MLP_OW2 + j * MLP_H + k], h1[k], z);
    h2[j] = tanhf(z);
    y = fmaf(p[MLP_OW3 + j], h2[j], y);
  }
  const float err = y - tv;
  const float dy = valid ? 2.0f * err / (float)batch : 0.0f;
  float dz2[MLP_H];
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) dz2[j] = dy * p[MLP_OW3 + j] * (1.0f - h2[j] * h2[j]);
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) {
    float dh1 = 0.f;
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) dh1 = fmaf(dz2[j], p[MLP_OW2 + j * MLP_H + k], dh1);
    dz1s[tid][k] = dh1 * (1.0f - h1[k] * h1[k]);
    h1s[tid][k] = h1[k];
    h2s[tid][k] = h2[k];
    dz2s[tid][k] = dz2[k];
  }
  xs[tid] = xv;
  dys[tid] = dy;
  es[tid] = valid ? err * err : 0.0f;
  __syncthreads();
  float *out = part + (int64_t)blockIdx.x * (MLP_NP + 1);
  // dW2[j][k] = sum_p dz2[p][j] h1[p][k]   (thread = one (j, k))
  {
    const int j = tid / MLP_H, k = tid % MLP_H;
    float s = 0.f;
    for (int q = 0; q < MLP_BLK; ++q) s = fmaf(dz2s[q][j], h1s[q][k], s);
    out[MLP_OW2 + tid] = s;
  }
  if (tid < MLP_H) {
    float w1 = 0.f, b1 = 0.f, b2 = 0.f, w3 = 0.f;
    for (int q = 0; q < MLP_BLK; ++q) {
      w1 = fmaf(dz1s[q][tid], xs[q], w1);
      b1 += dz1s[q][tid];
      b2 += dz2s[q][tid];
      w3 = fmaf(dys[q], h2s[q][tid], w3);
    }
    out[MLP_OW1 + tid] = w1;
    out[MLP_OB1 + tid] = b1;
    out[MLP_OB2 + tid] = b2;
    out[MLP_OW3 + tid] = w3;
  } else if (tid == MLP_H) {
    float b3 = 0.f, l = 0.f;
    for (int q = 0; q < MLP_BLK; ++q) {
      b3 += dys[q];
      l += es[q];
    }
    out[MLP_OB3] = b3;
    out[MLP_NP] = l;
  }
}

// Sums the nb partial gradients in block order into grad[0..321] (and the
// batch loss into grad[321]), then, when step > 0, applies Adam (Kingma & Ba):
// m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// p <- p - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
__global__ void __launch_bounds__(352) mlp_adam_kernel(float *__restrict__ params,
                                                       float *__restrict__ mom,
                                                       float *__restrict__ vel,
                                                       const float *__restrict__ part, int nb,
                                                       int64_t batch, float *__restrict__ grad,
                                                       int step, float lr, const int *en) {
  if (en && !*en) return;
  const int i = threadIdx.x;
  if (i > MLP_NP) return;
  float g = 0.f;
  for (int b = 0; b < nb; ++b) g += part[(int64_t)b * (MLP_NP + 1) + i];
  if (i == MLP_NP) {
    if (grad) grad[MLP_NP] = g / (float)batch;  // mean squared error
    return;
  }
  if (grad) grad[i] = g;
  if (step <= 0) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float m = b1 * mom[i] + (1.f - b1) * g;
  const float v = b2 * vel[i] + (1.f - b2) * g * g;
  mom[i] = m;
  vel[i] = v;
  const float mh = m / (1.f - powf(b1, (float)step));
  const float vh = v / (1.f - powf(b2, (float)step));
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Zone boundaries from the model: spl[j] (j = 0..B-1) = smallest key whose
// model value reaches j/B (spl[0] = 0), made non-decreasing; and the
// prediction table tab[c] = F(c / LRN_TAB), c = 0..LRN_TAB, made
// non-decreasing and clamped to [0, 1].
template <typename K>
__global__ void __launch_bounds__(512) lrn_splitters_kernel(const float *__restrict__ params,
                                                            int B, int w, K *__restrict__ spl,
                                                            float *__restrict__ tab,
                                                            const int *en) {
  if (en && !*en) return;
  __shared__ float p[MLP_NP];
  __shared__ float ts[LRN_TAB + 1];
  __shared__ K ss[1024];
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    K r = 0;
    if (j > 0) {
      const float target = (float)j / (float)B;
      // binary search on the key: smallest r with F(feature(r)) >= target
      K lo = 0, hi = (K)~(K)0;
      if (mlp_eval(p, mlp_feature((uint64_t)hi, w)) < target) {
        r = hi;
      } else {
        while (lo < hi) {
          const K mid = lo + (K)((hi - lo) >> 1);
          if (mlp_eval(p, mlp_feature((uint64_t)mid, w)) >= target) hi = mid;
          else lo = mid + 1;
        }
        r = lo;
      }
    }
    ss[j] = r;
  }
  for (int c = threadIdx.x; c <= LRN_TAB; c += blockDim.x)
    ts[c] = mlp_eval(p, (float)c / (float)LRN_TAB);
  __syncthreads();
  if (threadIdx.x == 0) {
    K run = 0;
    for (int j = 0; j < B; ++j) {
      run = ss[j] > run ? ss[j] : run;
      spl[j] = run;
    }
    float f = 0.f;
    for (int c = 0; c <= LRN_TAB; ++c) {
      float v = ts[c];
      v = v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
      f = v > f ? v : f;
      tab[c] = f;
    }
  }
}

// Deterministic parameter initialisation from a seed: uniform in
// [-a, a] per layer (a = sqrt(6 / (fan_in + fan_out))), biases 0.
__global__ void mlp_init_kernel(float *__restrict__ params, float *__restrict__ mom,
                                float *__restrict__ vel, uint64_t seed, const int *en) {
  if (en && !*en) return;
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= MLP_NP) return;
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)(z >> 40) * (1.0f / 16777216.0f);  // [0, 1)
  float a = 0.f;
  if (i < MLP_OB1) a = sqrtf(6.f / 17.f);
  else if (i >= MLP_OW2 && i < MLP_OB2) a = sqrtf(6.f / 32.f);
  else if (i >= MLP_OW3 && i < MLP_OB3) a = sqrtf(6.f / 17.f);
  params[i] = (2.f * u - 1.f) * a;
  mom[i] = 0.f;
  vel[i] = 0.f;
}

// Distribution levels below a subproblem of s records under the digit-width
// rule (the fewest levels of at most gmax bits that bring buckets to target),
// none when it fits the base case.
__device__ __forceinline__ int levels_below(double s, double cap, double target, int gmax) {
  if (s <= cap) return 0;
  int e = 0;
  while (e < 62 && target * (double)(1ull << e) < s) ++e;
  return (e + gmax - 1) / gmax;
}

// Whether learned level-0 zones pay, from the sorted model sample (m keys of
// the n): the record-passes below level 0 with the digit zones against those
// with the model's zones [spl[z], spl[z+1]) plus the learned level's extra
// cost of `penalty` record-passes per record.  Each zone's cost follows the
// digit levels below it along the child that holds the median of its sample
// keys (a skewed zone splits off only its top key bits per level, so its bulk
// passes through many levels): every subproblem on that path above the
// base-case capacity is distributed once, and the other children of each
// step cost the levels the digit-width rule gives their mean size.  One CTA,
// a thread per zone; writes the decision and both estimates (per record).
// en (optional): a decision already taken; when it kept the digit zones
// (*en == 0) this one is skipped and both stay.
template <typename K>
__global__ void __launch_bounds__(512) lrn_decide_kernel(
    const uint64_t *__restrict__ sorted, int64_t m, int64_t n, int key_bits, int B,
    const K *__restrict__ spl, int cap, int64_t target, int gmax, double penalty, int *on,
    double *est, const int *en) {
  if (en && !*en) return;
  __shared__ double red[2][32];
  const uint64_t mask = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1ull);
  const uint64_t rmax = sorted[m - 1] & mask;
  const int t = rmax ? 64 - __clzll((long long)rmax) : 0;
  const int g = 31 - __clz(B);
  const int lo = t - g > 0 ? t - g : 0;
  const int nz = 1 << (t - lo);
  // first index in [a, b) with sorted[i] >= v (b when none)
  auto lower_bound_in = [&](int64_t a, int64_t b, uint64_t v) -> int64_t {
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if (sorted[mid] < v) a = mid + 1;
      else b = mid;
    }
    return a;
  };
  auto lower_bound = [&](uint64_t v) -> int64_t { return lower_bound_in(0, m, v); };
  const double per = (double)n / (double)m;  // records per sample key
  auto cost = [&](int64_t c0, int64_t c1) {
    double total = 0.0;
    int64_t a = c0, b = c1;
    for (int step = 0; step < 64 && b > a; ++step) {
      const double s = (double)(b - a) * per;
      if (s <= (double)cap) break;
      const uint64_t kmin = sorted[a] & mask, kmax = sorted[b - 1] & mask;
      if (kmin == kmax) break;  // one key value: moved, not distributed
      total += s;               // this subproblem is distributed once
      // its digit: the width rule's bits at the top of its key range
      int e = 0;
      while (e < 62 && (double)target * (double)(1ull << e) < s) ++e;
      if (e < 1) e = 1;
      const int nlev = (e + gmax - 1) / gmax;
      int gw = (e + nlev - 1) / nlev;
      gw = gw > gmax ? gmax : gw;
      const int t = 64 - __clzll((long long)(kmax - kmin));
      gw = gw > t ? t : gw;
      const int sh = t - gw;
      const uint64_t d = ((sorted[a + (b - a) / 2] & mask) - kmin) >> sh;
      const uint64_t lo_v = kmin + (d << sh);
      const uint64_t hi_v = sh < 64 ? lo_v + (1ull << sh) : lo_v;
      const int64_t na = lower_bound_in(a, b, lo_v);
      const int64_t nb = hi_v > lo_v ? lower_bound_in(na, b, hi_v) : b;
      // the other children at their mean size
      const double so = (double)((b - a) - (nb - na)) * per;
      const double mean = so / (double)((1ull << gw) - 1ull);
      total += so * (double)levels_below(mean, (double)cap, (double)target, gmax);
      if (nb - na >= b - a) break;  // no progress (cannot happen: kmin < kmax)
      a = na;
      b = nb;
    }
    return total;
  };
  double ad = 0.0, al = 0.0;
  for (int z = threadIdx.x; z < nz; z += blockDim.x)
    ad += cost(lower_bound((uint64_t)z << lo),
               z + 1 < nz ? lower_bound((uint64_t)(z + 1) << lo) : m);
  for (int z = threadIdx.x; z < B; z += blockDim.x)
    al += cost(z ? lower_bound((uint64_t)spl[z]) : 0,
               z + 1 < B ? lower_bound((uint64_t)spl[z + 1]) : m);
  for (int o = 16; o > 0; o >>= 1) {
    ad += __shfl_xor_sync(0xffffffffu, ad, o);
    al += __shfl_xor_sync(0xffffffffu, al, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ad;
    red[1][threadIdx.x >> 5] = al;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double cd = 0.0, cl = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      cd += red[0][i];
      cl += red[1][i];
    }
    cl += penalty * (double)n;
    *on = cd > cl ? 1 : 0;
    est[0] = cd / (double)n;
    est[1] = cl / (double)n;
  }
}

// Zone lower bounds at the sample's quantiles: spl[z] = the sorted sample's
// key of rank z m / B (spl[0] = 0).  These are the zones a perfect CDF model
// would give; the decision taken on them before any training bounds what the
// trained model can gain.
template <typename K>
__global__ void __launch_bounds__(256) lrn_quantile_kernel(const uint64_t *__restrict__ sorted,
                                                           int64_t m, int B, K *spl) {
  for (int z = blockIdx.x * 256 + threadIdx.x; z < B; z += gridDim.x * 256)
    spl[z] = z ? (K)sorted[(int64_t)z * m / B] : (K)0;
}

}  // namespace dts
