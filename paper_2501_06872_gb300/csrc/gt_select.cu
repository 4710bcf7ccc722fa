// Configuration search for the transposition: graph features, the search
// grid, the analytic cost model (Eqs. 2-3 of Sec. IV-B with GB300 constants),
// the exhaustive autotuner, and the learned selector (a 2x64 ReLU MLP whose
// forward pass, backward pass and Adam update run in the kernels below).
// None of this touches the transposition's integer arithmetic: a configuration
// only changes speed, never the output bytes.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "gt.h"
#include "gt_device.cuh"

namespace gt {
namespace {

constexpr uint32_t kNF = GT_N_FEATURES;
constexpr uint32_t kK = GT_TUNE_GRID;
constexpr uint32_t kH = GT_SEL_HIDDEN;
constexpr uint32_t kDegBins = 32;
constexpr uint32_t kLocRows = 4096;     // rows sampled for the locality features
constexpr uint32_t kLocPairs = 32;      // neighbour pairs read per sampled row (at most)
constexpr uint32_t kTopK = 512;         // coverage feature: top-512 sampled destinations
constexpr uint32_t kFreqCap = 1u << 16; // sample frequencies >= this are listed exactly
constexpr uint32_t kBigCap = 64;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// Parameter vector layout of the selector (floats).
constexpr uint32_t kOffMu = 0;
constexpr uint32_t kOffSd = kOffMu + kNF;
constexpr uint32_t kOffLo = kOffSd + kNF;  // trained feature range (not used by the network)
constexpr uint32_t kOffHi = kOffLo + kNF;
constexpr uint32_t kOffW1 = kOffHi + kNF;
constexpr uint32_t kOffB1 = kOffW1 + kH * kNF;
constexpr uint32_t kOffW2 = kOffB1 + kH;
constexpr uint32_t kOffB2 = kOffW2 + kH * kH;
constexpr uint32_t kOffW3 = kOffB2 + kH;
constexpr uint32_t kOffB3 = kOffW3 + kK * kH;
constexpr uint32_t kParams = kOffB3 + kK;

// Feature workspace (one device block).
struct FeatWs {
  unsigned long long vcnt[kDegBins];
  unsigned long long esum[kDegBins];
  unsigned long long maxdeg;
  unsigned long long loc_pairs;
  unsigned long long loc_same;
  double loc_sum;
  uint32_t maxfreq;
  uint32_t nbig;
  uint32_t big[kBigCap];
  uint32_t fh[kFreqCap];  // fh[c] = sampled destinations seen exactly c times (1 <= c < kFreqCap)
};

__device__ __forceinline__ uint32_t deg_bin(uint64_t d) {
  if (d == 0) return 0;
  uint32_t b = 64u - (uint32_t)__clzll((long long)d);  // 1 + floor(log2 d)
  return b > kDegBins - 1 ? kDegBins - 1 : b;
}

// Out-degree histogram (vertex counts and edge sums per log2 bin) and the
// maximum out-degree, from row_ptr alone.
__global__ void k_feat_deg(const uint64_t *__restrict__ row_ptr, uint32_t n, FeatWs *ws) {
  __shared__ unsigned long long s_cnt[kDegBins], s_sum[kDegBins];
  __shared__ unsigned long long s_max;
  if (threadIdx.x < kDegBins) {
    s_cnt[threadIdx.x] = 0;
    s_sum[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  unsigned long long mx = 0;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t d = row_ptr[u + 1] - row_ptr[u];
    const uint32_t b = deg_bin(d);
    atomicAdd(&s_cnt[b], 1ull);
    atomicAdd(&s_sum[b], (unsigned long long)d);
    mx = d > mx ? d : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(kFull, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(&s_max, mx);
  __syncthreads();
  if (threadIdx.x < kDegBins) {
    if (s_cnt[threadIdx.x]) atomicAdd(&ws->vcnt[threadIdx.x], s_cnt[threadIdx.x]);
    if (s_sum[threadIdx.x]) atomicAdd(&ws->esum[threadIdx.x], s_sum[threadIdx.x]);
  }
  if (threadIdx.x == 0) atomicMax(&ws->maxdeg, s_max);
}

// Sample j reads col_idx at floor(r_j * m / 2^64), r_j the j-th SplitMix64
// output of `seed`, and counts the destination in an open-addressing table.
__global__ void k_feat_sample(const uint32_t *__restrict__ col_idx, uint64_t m, uint32_t ns, uint64_t seed,
                              uint32_t *keys, uint32_t *cnt, uint32_t tlog2) {
  const uint32_t mask = (1u << tlog2) - 1u;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
    const uint64_t r = mix64(seed + (uint64_t)(j + 1) * kGamma);
    const uint32_t v = col_idx[__umul64hi(r, m)];
    uint32_t slot = (v * 0x9E3779B1u) >> (32u - tlog2);
#pragma unroll 1
    for (uint32_t i = 0; i <= mask; ++i) {
      const uint32_t old = atomicCAS(&keys[slot], kEmptyKey, v);
      if (old == kEmptyKey || old == v) {
        atomicAdd(&cnt[slot], 1u);
        break;
      }
      slot = (slot + 1u) & mask;
    }
  }
}

__global__ void k_feat_freq(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ cnt, uint32_t ts,
                            FeatWs *ws) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ts; s += gridDim.x * blockDim.x) {
    if (keys[s] == kEmptyKey) continue;
    const uint32_t c = cnt[s];
    atomicMax(&ws->maxfreq, c);
    if (c < kFreqCap) {
      atomicAdd(&ws->fh[c], 1u);
    } else {
      const uint32_t i = atomicAdd(&ws->nbig, 1u);
      if (i < kBigCap) ws->big[i] = c;  // at most ns / 2^16 <= 16 such destinations
    }
  }
}

// Locality: for kLocRows rows u_j = floor(r_j * n / 2^64) (SplitMix64 of
// seed ^ 0x4C4F43 ("LOC")), the first kLocPairs consecutive neighbour pairs
// (a, b): sum of log2(|a - b| + 1) and the count of pairs with a / 32 == b / 32
// (same 128-byte line of a per-vertex u32 array).  Rows whose row_ptr entries
// are out of order or beyond m are skipped.
__global__ void k_feat_loc(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col_idx, uint32_t n,
                           uint64_t m, uint32_t rows, uint64_t seed, FeatWs *ws) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  double sum = 0.0;
  unsigned long long pairs = 0, same = 0;
  for (uint32_t j = warp; j < rows; j += nwarps) {
    const uint64_t r = mix64((seed ^ 0x4C4F43ull) + (uint64_t)(j + 1) * kGamma);
    const uint64_t u = __umul64hi(r, (uint64_t)n);
    const uint64_t beg = row_ptr[u], end = row_ptr[u + 1];
    if (end > m || beg > end || end - beg < 2) continue;
    const uint64_t np = min64(end - beg - 1, kLocPairs);
    if (lane < np) {
      const uint32_t a = col_idx[beg + lane], b = col_idx[beg + lane + 1];
      const uint32_t dlt = a > b ? a - b : b - a;
      sum += log2((double)dlt + 1.0);
      pairs += 1;
      same += ((a >> 5) == (b >> 5)) ? 1 : 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(kFull, sum, o);
    pairs += __shfl_xor_sync(kFull, pairs, o);
    same += __shfl_xor_sync(kFull, same, o);
  }
  if (lane == 0 && pairs) {
    atomicAdd(&ws->loc_sum, sum);
    atomicAdd(&ws->loc_pairs, pairs);
    atomicAdd(&ws->loc_same, same);
  }
}

// Turns the integer summaries into the GT_N_FEATURES floats (one CTA of
// 1024 threads).  The coverage of the kTopK most frequent sampled
// destinations takes the exactly listed large frequencies first, then walks
// the frequency histogram downwards: thread t sums the 64 bins of its chunk,
// a suffix scan over the chunks finds the chunk where kTopK is reached, and
// that chunk's thread walks its bins.
constexpr uint32_t kFinThreads = 1024;
constexpr uint32_t kFinChunk = kFreqCap / kFinThreads;

__global__ void __launch_bounds__(kFinThreads) k_feat_final(FeatWs *ws, uint32_t n, uint32_t n_cols, uint64_t m,
                                                            uint32_t ns, int has_vals, float *out) {
  __shared__ unsigned long long s_cnt[kFinThreads], s_sum[kFinThreads];
  __shared__ unsigned long long s_left, s_cov;
  const uint32_t t = threadIdx.x;
  unsigned long long cnt = 0, sum = 0;
  for (uint32_t c = max(t * kFinChunk, 1u); c < (t + 1) * kFinChunk; ++c) {
    cnt += ws->fh[c];
    sum += (unsigned long long)c * ws->fh[c];
  }
  s_cnt[t] = cnt;
  s_sum[t] = sum;
  if (t == 0) {
    const uint32_t nb = ws->nbig < kBigCap ? ws->nbig : kBigCap;
    for (uint32_t i = 1; i < nb; ++i) {  // insertion sort, descending (at most ns / 2^16 <= 16 entries)
      const uint32_t x = ws->big[i];
      uint32_t j = i;
      while (j > 0 && ws->big[j - 1] < x) {
        ws->big[j] = ws->big[j - 1];
        --j;
      }
      ws->big[j] = x;
    }
    uint64_t left = kTopK, cov = 0;
    for (uint32_t i = 0; i < nb && left; ++i, --left) cov += ws->big[i];
    s_left = left;
    s_cov = cov;
  }
  __syncthreads();
  // inclusive suffix sums over chunks (Hillis-Steele)
  for (uint32_t off = 1; off < kFinThreads; off <<= 1) {
    const unsigned long long ac = t + off < kFinThreads ? s_cnt[t + off] : 0;
    const unsigned long long as = t + off < kFinThreads ? s_sum[t + off] : 0;
    __syncthreads();
    s_cnt[t] += ac;
    s_sum[t] += as;
    __syncthreads();
  }
  const unsigned long long left = s_left;
  const unsigned long long above_c = t + 1 < kFinThreads ? s_cnt[t + 1] : 0;
  const unsigned long long above_s = t + 1 < kFinThreads ? s_sum[t + 1] : 0;
  __syncthreads();
  if (left > 0) {
    if (t == 0 && s_cnt[0] < left) {
      s_cov += s_sum[0];  // fewer than kTopK distinct destinations left: all of them
    } else if (above_c < left && s_cnt[t] >= left) {
      unsigned long long need = left - above_c, cov = above_s;
      for (uint32_t c = (t + 1) * kFinChunk - 1; c >= max(t * kFinChunk, 1u) && need; --c) {
        const unsigned long long k = min((unsigned long long)ws->fh[c], need);
        cov += k * c;
        need -= k;
      }
      s_cov += cov;  // exactly one thread gets here
    }
  }
  __syncthreads();
  if (t != 0) return;
  const double dn = (double)n;  // rows
  for (uint32_t b = 0; b < kDegBins; ++b) out[b] = (float)((double)ws->vcnt[b] / dn);
  out[32] = (float)(log2((double)n_cols) / 32.0);
  out[33] = (float)(log2((double)m + 1.0) / 32.0);
  out[34] = (float)(log2((double)ws->maxdeg + 1.0) / 32.0);
  // edges out of the ceil(n/100) vertices of highest out-degree, walking the
  // log2 bins downwards and taking a proportional share of the boundary bin
  double take = (double)(((uint64_t)n + 99u) / 100u), got = 0.0;
  for (int b = (int)kDegBins - 1; b >= 0 && take > 0.0; --b) {
    const double c = (double)ws->vcnt[b];
    if (c == 0.0) continue;
    if (c <= take) {
      got += (double)ws->esum[b];
      take -= c;
    } else {
      got += (double)ws->esum[b] * (take / c);
      take = 0.0;
    }
  }
  out[35] = m ? (float)(got / (double)m) : 0.f;
  out[36] = ns ? (float)((double)s_cov / (double)ns) : 0.f;
  out[37] = ns ? (float)(log2((double)ws->maxfreq * (double)m / (double)ns + 1.0) / 32.0) : 0.f;
  const double lp = (double)ws->loc_pairs;
  out[38] = lp > 0 ? (float)(ws->loc_sum / lp / 32.0) : 0.f;
  out[39] = lp > 0 ? (float)((double)ws->loc_same / lp) : 0.f;
  out[40] = has_vals ? 1.f : 0.f;
}

uint32_t ceil_log2(uint64_t x) {
  uint32_t b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

// ---- MLP kernels (f32; all reductions in a fixed order) ---------------------

__global__ void k_norm(const float *__restrict__ X, const float *__restrict__ p, uint32_t B, float *Xn) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kNF) return;
  const uint32_t f = i % kNF;
  Xn[i] = (X[i] - p[kOffMu + f]) / p[kOffSd + f];
}

// Y[b][o] = act(b_o + sum_i W[o][i] X[b][i]).
__global__ void k_dense(const float *__restrict__ W, const float *__restrict__ bias, const float *__restrict__ X,
                        uint32_t B, uint32_t in, uint32_t out, int relu, float *Y) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * out) return;
  const uint32_t b = t / out, o = t % out;
  const float *w = W + (size_t)o * in;
  const float *x = X + (size_t)b * in;
  float acc = bias[o];
  for (uint32_t i = 0; i < in; ++i) acc = fmaf(w[i], x[i], acc);
  Y[t] = (relu && acc < 0.f) ? 0.f : acc;
}

// Masked mean squared error: loss = sum M (Yh - Y)^2 / max(1, sum M),
// dY = 2 M (Yh - Y) / max(1, sum M).  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ Yh, const float *__restrict__ Y,
                                             const float *__restrict__ M, uint32_t cnt, float *loss, float *dY) {
  __shared__ float s_a[256], s_m[256];
  float a = 0.f, mm = 0.f;
  for (uint32_t i = threadIdx.x; i < cnt; i += 256) {
    const float d = Yh[i] - Y[i];
    a = fmaf(M[i] * d, d, a);
    mm += M[i];
  }
  s_a[threadIdx.x] = a;
  s_m[threadIdx.x] = mm;
  __syncthreads();
  for (uint32_t o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_a[threadIdx.x] += s_a[threadIdx.x + o];
      s_m[threadIdx.x] += s_m[threadIdx.x + o];
    }
    __syncthreads();
  }
  const float den = fmaxf(1.f, s_m[0]);
  if (threadIdx.x == 0) *loss = s_a[0] / den;
  for (uint32_t i = threadIdx.x; i < cnt; i += 256) dY[i] = 2.f * M[i] * (Yh[i] - Y[i]) / den;
}

// dW[o][i] = sum_b dY[b][o] X[b][i]; db[o] = sum_b dY[b][o] (thread i == in).
__global__ void k_dense_bwd_w(const float *__restrict__ dY, const float *__restrict__ X, uint32_t B, uint32_t in,
                              uint32_t out, float *dW, float *db) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= out * (in + 1)) return;
  const uint32_t o = t / (in + 1), i = t % (in + 1);
  float acc = 0.f;
  if (i == in) {
    for (uint32_t b = 0; b < B; ++b) acc += dY[(size_t)b * out + o];
    db[o] = acc;
  } else {
    for (uint32_t b = 0; b < B; ++b) acc = fmaf(dY[(size_t)b * out + o], X[(size_t)b * in + i], acc);
    dW[(size_t)o * in + i] = acc;
  }
}

// dX[b][i] = [H[b][i] > 0] * sum_o dY[b][o] W[o][i]  (H: the ReLU output feeding the layer).
__global__ void k_dense_bwd_x(const float *__restrict__ dY, const float *__restrict__ W, const float *__restrict__ H,
                              uint32_t B, uint32_t in, uint32_t out, float *dX) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * in) return;
  const uint32_t b = t / in, i = t % in;
  float acc = 0.f;
  for (uint32_t o = 0; o < out; ++o) acc = fmaf(dY[(size_t)b * out + o], W[(size_t)o * in + i], acc);
  dX[t] = H[t] > 0.f ? acc : 0.f;
}

// Adam (Kingma & Ba 2015) on params[lo, hi): bias-corrected moments.
// Adam with an L2 penalty wd/2 |W|^2 on the trained entries: the gradient
// seen by the moments is g + wd * p.
__global__ void k_adam(float *p, const float *__restrict__ g, float *m1, float *m2, uint32_t lo, uint32_t hi,
                       float lr, float b1, float b2, float eps, float bc1, float bc2, float wd) {
  const uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  const float gi = g[i] + wd * p[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  p[i] -= lr * (a / bc1) / (sqrtf(v / bc2) + eps);
}

inline uint32_t blocks(uint64_t n, uint32_t t) { return (uint32_t)((n + t - 1) / t); }

}  // namespace
}  // namespace gt

using namespace gt;

struct gt_selector_s {
  int device = 0;
  float lo[GT_N_FEATURES], hi[GT_N_FEATURES];  // host copy of the trained feature range
  float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
  uint32_t steps = 0;
  uint32_t cap = 0;  // batch capacity of the activation buffers
  float *xn = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *d2 = nullptr, *d1 = nullptr;
  float *loss = nullptr;
};

namespace {

thread_local const char *g_sel_err = "no error";

gt_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GT_OK;
  g_sel_err = cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? GT_ERR_NO_MEMORY : GT_ERR_CUDA;
}

gt_status sel_reserve(gt_selector s, uint32_t B) {
  if (B <= s->cap) return GT_OK;
  float *bufs[7] = {s->xn, s->h1, s->h2, s->y, s->dy, s->d2, s->d1};
  for (float *b : bufs) cudaFree(b);
  s->xn = s->h1 = s->h2 = s->y = s->dy = s->d2 = s->d1 = nullptr;
  s->cap = 0;
  const size_t sizes[7] = {(size_t)B * kNF, (size_t)B * kH, (size_t)B * kH, (size_t)B * kK,
                           (size_t)B * kK,  (size_t)B * kH, (size_t)B * kH};
  float **dst[7] = {&s->xn, &s->h1, &s->h2, &s->y, &s->dy, &s->d2, &s->d1};
  for (int i = 0; i < 7; ++i) {
    gt_status st = cuda_status(cudaMalloc(dst[i], sizes[i] * 4));
    if (st != GT_OK) return st;
  }
  s->cap = B;
  return GT_OK;
}

// Forward pass into the selector's activation buffers; output in s->y.
cudaError_t sel_forward(gt_selector s, const float *X, uint32_t B, cudaStream_t st) {
  const float *p = s->params;
  k_norm<<<blocks((uint64_t)B * kNF, 256), 256, 0, st>>>(X, p, B, s->xn);
  k_dense<<<blocks((uint64_t)B * kH, 128), 128, 0, st>>>(p + kOffW1, p + kOffB1, s->xn, B, kNF, kH, 1, s->h1);
  k_dense<<<blocks((uint64_t)B * kH, 128), 128, 0, st>>>(p + kOffW2, p + kOffB2, s->h1, B, kH, kH, 1, s->h2);
  k_dense<<<blocks((uint64_t)B * kK, 128), 128, 0, st>>>(p + kOffW3, p + kOffB3, s->h2, B, kH, kK, 0, s->y);
  return cudaGetLastError();
}

// SplitMix64 stream on the host (initialisation only).
uint64_t host_mix(uint64_t x) {
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x;
}

}  // namespace

extern "C" {

uint64_t gt_selector_param_count(void) { return kParams; }

gt_status gt_graph_features_rect(uint32_t n, uint32_t n_cols, uint64_t m, int has_vals, const uint64_t *row_ptr,
                                 const uint32_t *col_idx, uint64_t seed, float *features, void *stream) {
  if (n == 0 || n_cols == 0 || !row_ptr || !features || (m > 0 && !col_idx)) return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t ns64 = ((uint64_t)n_cols + 99) / 100;
  ns64 = std::max<uint64_t>(ns64, 1024);
  ns64 = std::min<uint64_t>(ns64, 1u << 20);
  const uint32_t ns = m ? (uint32_t)ns64 : 0u;
  const uint32_t tlog2 = ceil_log2(std::max<uint64_t>(2ull * ns, 1024));
  const size_t ts = (size_t)1 << tlog2;
  void *blk = nullptr;
  const size_t bytes = sizeof(FeatWs) + ts * 8;
  gt_status st = cuda_status(cudaMallocAsync(&blk, bytes, s));
  if (st != GT_OK) return st;
  FeatWs *ws = (FeatWs *)blk;
  uint32_t *keys = (uint32_t *)((char *)blk + sizeof(FeatWs));
  uint32_t *cnt = keys + ts;
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(FeatWs), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xFF, ts * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, ts * 4, s);
  if (e == cudaSuccess) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t g = (uint32_t)std::min<uint64_t>(blocks(n, 256), (uint64_t)sms * 8);
    k_feat_deg<<<g, 256, 0, s>>>(row_ptr, n, ws);
    if (ns) {
      k_feat_sample<<<std::min<uint32_t>(blocks(ns, 256), sms * 8), 256, 0, s>>>(col_idx, m, ns, seed, keys, cnt,
                                                                                  tlog2);
      k_feat_freq<<<std::min<uint32_t>(blocks(ts, 256), sms * 8), 256, 0, s>>>(keys, cnt, (uint32_t)ts, ws);
      k_feat_loc<<<blocks((uint64_t)kLocRows * 32, 256), 256, 0, s>>>(row_ptr, col_idx, n, m, kLocRows, seed, ws);
    }
    k_feat_final<<<1, kFinThreads, 0, s>>>(ws, n, n_cols, m, ns, has_vals, features);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(blk, s);
  return cuda_status(e != cudaSuccess ? e : e2);
}

gt_status gt_graph_features(uint32_t n, uint64_t m, int has_vals, const uint64_t *row_ptr, const uint32_t *col_idx,
                            uint64_t seed, float *features, void *stream) {
  return gt_graph_features_rect(n, n, m, has_vals, row_ptr, col_idx, seed, features, stream);
}

gt_status gt_selector_create(gt_selector *sel, const float *host_params, uint64_t seed) {
  if (!sel) return GT_ERR_INVALID_ARG;
  *sel = nullptr;
  gt_selector s = new (std::nothrow) gt_selector_s();
  if (!s) return GT_ERR_NO_MEMORY;
  cudaGetDevice(&s->device);
  float **dst[5] = {&s->params, &s->grads, &s->m1, &s->m2, &s->loss};
  const size_t sizes[5] = {kParams, kParams, kParams, kParams, 1};
  for (int i = 0; i < 5; ++i) {
    gt_status st = cuda_status(cudaMalloc(dst[i], sizes[i] * 4));
    if (st != GT_OK) {
      gt_selector_destroy(s);
      return st;
    }
  }
  std::vector<float> p(kParams, 0.f);
  if (host_params) {
    memcpy(p.data(), host_params, kParams * 4);
  } else {
    // mu = 0, sd = 1, unbounded range; weights uniform in +-sqrt(6 / fan_in) (He), biases 0
    for (uint32_t f = 0; f < kNF; ++f) {
      p[kOffSd + f] = 1.f;
      p[kOffLo + f] = -FLT_MAX;
      p[kOffHi + f] = FLT_MAX;
    }
    uint64_t ctr = 0;
    auto fill = [&](uint32_t off, uint32_t count, uint32_t fan_in) {
      const double lim = sqrt(6.0 / fan_in);
      for (uint32_t i = 0; i < count; ++i) {
        const double u = (double)(host_mix(seed + (++ctr) * kGamma) >> 11) * (1.0 / 9007199254740992.0);
        p[off + i] = (float)((2.0 * u - 1.0) * lim);
      }
    };
    fill(kOffW1, kH * kNF, kNF);
    fill(kOffW2, kH * kH, kH);
    fill(kOffW3, kK * kH, kH);
  }
  memcpy(s->lo, p.data() + kOffLo, sizeof(s->lo));
  memcpy(s->hi, p.data() + kOffHi, sizeof(s->hi));
  cudaError_t e = cudaMemcpy(s->params, p.data(), kParams * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->grads, 0, kParams * 4);
  if (e == cudaSuccess) e = cudaMemset(s->m1, 0, kParams * 4);
  if (e == cudaSuccess) e = cudaMemset(s->m2, 0, kParams * 4);
  if (e != cudaSuccess) {
    gt_selector_destroy(s);
    return cuda_status(e);
  }
  *sel = s;
  return GT_OK;
}

gt_status gt_selector_get_params(gt_selector sel, float *host_params) {
  if (!sel || !host_params) return GT_ERR_INVALID_ARG;
  return cuda_status(cudaMemcpy(host_params, sel->params, kParams * 4, cudaMemcpyDeviceToHost));
}

gt_status gt_selector_set_params(gt_selector sel, const float *host_params) {
  if (!sel || !host_params) return GT_ERR_INVALID_ARG;
  for (uint32_t f = 0; f < kNF; ++f)
    if (!(host_params[kOffSd + f] > 0.f) || !(host_params[kOffLo + f] <= host_params[kOffHi + f]))
      return GT_ERR_INVALID_ARG;
  gt_status st = cuda_status(cudaMemcpy(sel->params, host_params, kParams * 4, cudaMemcpyHostToDevice));
  if (st != GT_OK) return st;
  memcpy(sel->lo, host_params + kOffLo, sizeof(sel->lo));
  memcpy(sel->hi, host_params + kOffHi, sizeof(sel->hi));
  sel->steps = 0;
  cudaMemset(sel->m1, 0, kParams * 4);
  cudaMemset(sel->m2, 0, kParams * 4);
  return GT_OK;
}

gt_status gt_selector_forward(gt_selector sel, const float *features, uint32_t batch, float *scores,
                              void *stream) {
  if (!sel || !features || !scores || batch == 0) return GT_ERR_INVALID_ARG;
  gt_status st = sel_reserve(sel, batch);
  if (st != GT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = sel_forward(sel, features, batch, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scores, sel->y, (size_t)batch * kK * 4, cudaMemcpyDeviceToDevice, s);
  return cuda_status(e);
}

gt_status gt_selector_backward(gt_selector sel, const float *features, const float *target, const float *mask,
                               uint32_t batch, float *loss, float *grads, void *stream) {
  if (!sel || !features || !target || !mask || batch == 0) return GT_ERR_INVALID_ARG;
  gt_status st = sel_reserve(sel, batch);
  if (st != GT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = sel_forward(sel, features, batch, s);
  if (e != cudaSuccess) return cuda_status(e);
  const float *p = sel->params;
  float *g = sel->grads;
  const uint32_t B = batch;
  k_mse<<<1, 256, 0, s>>>(sel->y, target, mask, B * kK, sel->loss, sel->dy);
  // layer 3: h2 -> y
  k_dense_bwd_w<<<blocks((uint64_t)kK * (kH + 1), 128), 128, 0, s>>>(sel->dy, sel->h2, B, kH, kK, g + kOffW3,
                                                                       g + kOffB3);
  k_dense_bwd_x<<<blocks((uint64_t)B * kH, 128), 128, 0, s>>>(sel->dy, p + kOffW3, sel->h2, B, kH, kK, sel->d2);
  // layer 2: h1 -> h2
  k_dense_bwd_w<<<blocks((uint64_t)kH * (kH + 1), 128), 128, 0, s>>>(sel->d2, sel->h1, B, kH, kH, g + kOffW2,
                                                                       g + kOffB2);
  k_dense_bwd_x<<<blocks((uint64_t)B * kH, 128), 128, 0, s>>>(sel->d2, p + kOffW2, sel->h1, B, kH, kH, sel->d1);
  // layer 1: xn -> h1
  k_dense_bwd_w<<<blocks((uint64_t)kH * (kNF + 1), 128), 128, 0, s>>>(sel->d1, sel->xn, B, kNF, kH, g + kOffW1,
                                                                        g + kOffB1);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(g, 0, (size_t)kOffW1 * 4, s);  // mu, sd, lo, hi are not trained
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, sel->loss, 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && grads) e = cudaMemcpyAsync(grads, g, (size_t)kParams * 4, cudaMemcpyDeviceToDevice, s);
  return cuda_status(e);
}

gt_status gt_selector_adam_step(gt_selector sel, float lr, float beta1, float beta2, float eps, float weight_decay,
                                void *stream) {
  if (!sel || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
      !(weight_decay >= 0.f))
    return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  sel->steps += 1;
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)sel->steps));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)sel->steps));
  k_adam<<<blocks(kParams - kOffW1, 256), 256, 0, s>>>(sel->params, sel->grads, sel->m1, sel->m2, kOffW1, kParams, lr,
                                                       beta1, beta2, eps, bc1, bc2, weight_decay);
  return cuda_status(cudaGetLastError());
}

gt_status gt_selector_in_range(gt_selector sel, const float *host_features, int *in_range) {
  if (!sel || !host_features || !in_range) return GT_ERR_INVALID_ARG;
  // the trained range widened by 5 % of its width on each side
  int ok = 1;
  for (uint32_t f = 0; f < kNF; ++f) {
    const double lo = sel->lo[f], hi = sel->hi[f];
    const double pad = 0.05 * (hi - lo) + 1e-6;
    if (host_features[f] < lo - pad || host_features[f] > hi + pad) ok = 0;
  }
  *in_range = ok;
  return GT_OK;
}

void gt_selector_destroy(gt_selector sel) {
  if (!sel) return;
  float *bufs[12] = {sel->params, sel->grads, sel->m1, sel->m2, sel->loss, sel->xn,
                     sel->h1,     sel->h2,    sel->y,  sel->dy, sel->d2,   sel->d1};
  for (float *b : bufs) cudaFree(b);
  delete sel;
}

// ---- search grid, analytic model, autotuner ---------------------------------

gt_status gt_tune_grid_config(uint32_t index, uint32_t n_vertices, uint64_t n_edges, gt_config *cfg) {
  if (!cfg || index >= kK) return GT_ERR_INVALID_ARG;
  gt_status st = gt_default_config(cfg, n_vertices, n_edges);
  if (st != GT_OK) return st;
  cfg->method = GT_METHOD_HLH;
  cfg->flags = GT_FLAG_AGGREGATE;
  cfg->stage_edges = 0;
  cfg->radix_tile = 0;
  cfg->radix_digit_bits = 0;
  uint32_t k = 0;
  auto radix = [&](uint32_t tile, uint32_t ctas, uint32_t digit) {
    cfg->method = GT_METHOD_RADIX;
    cfg->radix_tile = tile;
    cfg->ctas_per_sm = ctas;
    cfg->radix_digit_bits = digit;
  };
  switch (index) {
    case 0: k = 0; break;               // Atomic GT (Algorithm 1)
    case 1: k = 512; break;             // HLH, Eq. 1 sizing
    case 2: radix(0, 4, 8); break;      // bulk-staged tiles (two CTAs per SM whatever ctas_per_sm says)
    case 3: radix(0, 4, 7); break;
    case 4: radix(0, 4, 6); break;
    case 5: radix(4096, 2, 8); break;   // register tiles
    case 6: radix(4096, 2, 7); break;
    case 7: radix(4096, 3, 6); break;
    case 8: radix(2048, 4, 8); break;
    case 9: radix(2048, 4, 7); break;
    case 10: radix(2048, 6, 8); break;
    default: radix(2048, 6, 6); break;
  }
  if (cfg->method == GT_METHOD_RADIX || k > n_vertices / 2) k = 0;
  cfg->hdv_k = k;
  cfg->table_log2 = k ? ceil_log2(2ull * k) : 0;
  return GT_OK;
}

// Sec. IV-B cost model per edge, instantiated with GB300 rates:
//   Atomic (Eq. 2): 2 random accesses (count, scatter), each h*t_hit + (1-h)*t_miss,
//                   plus the sort of every list and the streaming of Steps 1-3
//   HLH    (Eq. 3): HDV edges (coverage c) update shared memory; LDV edges as
//                   Atomic, and only they are sorted
//   Radix:          ceil(log2(n) / 8) digit passes of t_pass each, plus the
//                   row expansion, degree runs and scan
// h = fraction of the random-access working set (12 B per vertex, 4-8 B per
// edge of output) that fits in L2, raised to the sampled same-line locality.
// The rates are GB300 measurements: random 4-byte DRAM accesses cap near
// 24 G/s, L2-resident atomics run at 127-195 G/s; per-edge costs of the list
// sort, of the streaming steps and of one digit pass come from the per-step
// timings of the library (one digit pass: 8.6 ps/edge at 2^32 edges, 12-16
// ps/edge at 2^22-2^24 edges).
gt_status gt_tune_analytic(const float *features, uint32_t n_vertices, uint64_t n_edges, uint32_t *index) {
  if (!features || !index) return GT_ERR_INVALID_ARG;
  const double ps = 1e-12;
  const double t_miss = 1.0 / 24e9;
  const double t_hit = 1.0 / 150e9;
  const double t_smem = 1.0 / 600e9;
  const double t_sort = 40 * ps;     // LDV list sort (scratch round trip + shared-memory sort)
  const double t_fixed = 12 * ps;    // streaming of col_idx/row_ptr/vals in Steps 1 and 3, scan
  const double t_sample = 2 * ps;    // Step 0 and the HDV insertion points
  const double t_pass = 12 * ps;     // one digit pass (upsweep + downsweep)
  const double t_runs = 4 * ps;      // row expansion, degree runs, scan
  const double l2 = 126.0 * 1024 * 1024;
  const int has_vals = features[40] > 0.5f;
  const double vscale = has_vals ? 1.25 : 1.0;
  const double wset = 12.0 * n_vertices + (has_vals ? 8.0 : 4.0) * (double)n_edges;
  double h = std::min(1.0, l2 / std::max(1.0, wset));
  h = std::max(h, (double)features[39]);
  const double c = std::min(1.0, std::max(0.0, (double)features[36]));
  const double t_rand = h * t_hit + (1.0 - h) * t_miss;
  const double atomic = 2.0 * t_rand + vscale * (t_sort + t_fixed);
  const double hlh = 2.0 * (c * t_smem + (1.0 - c) * t_rand) + vscale * ((1.0 - c) * t_sort + t_fixed) + t_sample;
  const double passes = std::max(1u, (ceil_log2((uint64_t)n_vertices) + 7) / 8);
  const double radix = vscale * passes * t_pass + t_runs;
  uint32_t best = 0;
  double t = atomic;
  if (hlh < t) {
    best = 1;
    t = hlh;
  }
  if (radix < t) best = 2;
  (void)n_edges;
  *index = best;
  return GT_OK;
}

}  // extern "C"

// gt_plan_tune lives here too: it only drives the public entry points.
namespace {

gt_status run_timed(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                    uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, uint32_t reps, cudaStream_t s,
                    float *median_ms) {
  gt_status st = gt_transpose(plan, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, s);  // warm-up
  if (st != GT_OK) return st;
  std::vector<float> t(reps);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return cuda_status(cudaGetLastError());
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_status(cudaGetLastError());
  }
  for (uint32_t r = 0; r < reps && st == GT_OK; ++r) {
    cudaEventRecord(a, s);
    st = gt_transpose(plan, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, s);
    cudaEventRecord(b, s);
    if (st == GT_OK) {
      cudaError_t e = cudaEventSynchronize(b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], a, b);
      st = cuda_status(e);
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != GT_OK) return st;
  st = gt_plan_status(plan);
  if (st != GT_OK) return st;
  std::sort(t.begin(), t.end());
  *median_ms = t[reps / 2];
  return GT_OK;
}

// Grid points that run the same kernel sequence on an n-column matrix: radix
// points whose digit caps give the same pass count (hence the same digits)
// differ in nothing else, and the bulk-staged tile ignores ctas_per_sm.
uint32_t radix_passes(const gt_config &c, uint32_t n) {
  uint32_t bits = 0;
  while (bits < 32 && ((n ? n - 1 : 0) >> bits)) ++bits;
  if (bits == 0) bits = 1;
  const uint32_t cap = c.radix_digit_bits ? c.radix_digit_bits : 8u;
  return (bits + cap - 1) / cap;
}

bool same_config(const gt_config &a, const gt_config &b, uint32_t n) {
  if (a.method != b.method) return false;
  if (a.method == GT_METHOD_RADIX)
    return a.radix_tile == b.radix_tile && (a.radix_tile == 0 || a.ctas_per_sm == b.ctas_per_sm) &&
           radix_passes(a, n) == radix_passes(b, n);
  return a.hdv_k == b.hdv_k && a.table_log2 == b.table_log2 && a.block_threads == b.block_threads &&
         a.ctas_per_sm == b.ctas_per_sm && a.warp_edges == b.warp_edges && a.stage_edges == b.stage_edges &&
         a.flags == b.flags;
}

}  // namespace

extern "C" gt_status gt_plan_tune(gt_plan plan, int mode, gt_selector sel, const uint64_t *row_ptr,
                                  const uint32_t *col_idx, const float *vals, uint64_t *col_ptr, uint32_t *row_idx,
                                  float *vals_out, uint32_t reps, gt_tune_entry *table, uint32_t *chosen,
                                  void *stream) {
  if (!plan || !row_ptr || !col_ptr) return GT_ERR_INVALID_ARG;
  if (mode != GT_TUNE_ANALYTIC && mode != GT_TUNE_EXHAUSTIVE && mode != GT_TUNE_LEARNED) return GT_ERR_INVALID_ARG;
  if (mode == GT_TUNE_LEARNED && !sel) return GT_ERR_INVALID_ARG;
  gt_config cur;
  gt_plan_get_config(plan, &cur);
  uint32_t n_rows = 0, n = 0;  // n: columns (the grid and the analytic model size by destinations)
  uint64_t m = 0;
  gt_plan_shape(plan, &n_rows, &n, &m);
  cudaStream_t s = (cudaStream_t)stream;
  gt_config grid[kK];
  for (uint32_t i = 0; i < kK; ++i) gt_tune_grid_config(i, n, m, &grid[i]);
  if (table)
    for (uint32_t i = 0; i < kK; ++i) {
      table[i].cfg = grid[i];
      table[i].ms = -1.f;
      table[i].score = 0.f;
      table[i].status = GT_OK;
    }
  uint32_t pick = 0;
  gt_status st = GT_OK;
  if (mode == GT_TUNE_EXHAUSTIVE) {
    if (reps == 0) reps = 3;
    float best = 0.f;
    bool have = false;
    for (uint32_t i = 0; i < kK; ++i) {
      float ms = -1.f;
      gt_status ei = GT_OK;
      uint32_t dup = i;
      for (uint32_t j = 0; j < i; ++j)
        if (same_config(grid[i], grid[j], n)) {
          dup = j;
          break;
        }
      if (dup != i && table) {
        ms = table[dup].ms;
        ei = (gt_status)table[dup].status;
      } else if (dup == i) {
        ei = gt_plan_set_config(plan, &grid[i]);
        if (ei == GT_OK) ei = run_timed(plan, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, reps, s, &ms);
      }
      if (table) {
        table[i].ms = ei == GT_OK ? ms : -1.f;
        table[i].status = ei;
      }
      if (ei == GT_ERR_OUT_OF_RANGE || ei == GT_ERR_BAD_ROW_PTR) {
        st = ei;  // the input is invalid: no configuration can succeed
        break;
      }
      if (ei == GT_OK && dup == i && (!have || ms < best)) {
        best = ms;
        pick = i;
        have = true;
      }
    }
    if (st == GT_OK && !have) st = GT_ERR_CUDA;
  } else {
    float *feat = nullptr;
    st = cuda_status(cudaMallocAsync(&feat, (kNF + kK) * 4, s));
    if (st != GT_OK) return st;
    st = gt_graph_features_rect(n_rows, n, m, vals != nullptr, row_ptr, col_idx, cur.seed, feat, s);
    float hf[kNF + kK];
    if (st == GT_OK && mode == GT_TUNE_LEARNED) st = gt_selector_forward(sel, feat, 1, feat + kNF, s);
    if (st == GT_OK) st = cuda_status(cudaMemcpyAsync(hf, feat, sizeof(hf), cudaMemcpyDeviceToHost, s));
    if (st == GT_OK) st = cuda_status(cudaStreamSynchronize(s));
    cudaFreeAsync(feat, s);
    if (st != GT_OK) return st;
    int in_range = 1;
    if (mode == GT_TUNE_LEARNED) gt_selector_in_range(sel, hf, &in_range);
    if (mode == GT_TUNE_ANALYTIC || !in_range) {
      st = gt_tune_analytic(hf, n, m, &pick);  // outside the trained range the analytic model decides
    } else {
      pick = 0;
      for (uint32_t i = 1; i < kK; ++i)
        if (hf[kNF + i] < hf[kNF + pick]) pick = i;
    }
    if (table)
      for (uint32_t i = 0; i < kK && mode == GT_TUNE_LEARNED; ++i) table[i].score = hf[kNF + i];
  }
  if (st != GT_OK) {
    gt_plan_set_config(plan, &cur);
    return st;
  }
  if (chosen) *chosen = pick;
  return gt_plan_set_config(plan, &grid[pick]);
}
