// Seeded synthetic graph generators on the GPU (libgtgen.so).  Test and
// benchmark inputs only: nothing here transposes anything.
//
// R-MAT (Chakrabarti, Zhan, Faloutsos 2004) picks, for every edge and every
// level, one quadrant with probabilities (a, b, c, d).  The source bit of a
// level is 0 with probability a+b independently of the other levels, so the
// out-degree vector is multinomial; it is drawn exactly by splitting the edge
// count level by level with binomial draws (BTRS, Hormann 1993, for large
// means; inversion for small ones).  Each edge slot j of source u then draws
// its destination bits conditionally on u's bits: P(dst bit 0 | src bit 0) =
// a/(a+b), P(dst bit 0 | src bit 1) = c/(c+d).  This gives R-MAT graphs
// directly in CSR order, with rows in generation order.  The uniform graph
// (G(n, m) with replacement) uses p = 1/2 splits and uniform destinations.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ inline uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x;
}

// Same stream naming as the numpy generators: key = fold(seed, ids...).
__host__ __device__ inline uint64_t fold(uint64_t k, uint64_t id) { return mix64(k ^ (id + kGolden)); }
__host__ __device__ inline uint64_t draw(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * kGolden); }

struct Stream {
  uint64_t key, ctr;
  __device__ double uniform() {  // (0, 1)
    uint64_t r = draw(key, ctr++);
    return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  }
};

// Binomial(n, p) variate.
__device__ uint64_t binomial(uint64_t n, double p, Stream &rs) {
  if (n == 0 || p <= 0.0) return 0;
  if (p >= 1.0) return n;
  bool flip = p > 0.5;
  if (flip) p = 1.0 - p;
  const double q = 1.0 - p;
  const double dn = (double)n;
  uint64_t x;
  if (dn * p < 10.0) {
    // inversion by sequential search
    const double s = p / q, a = (dn + 1.0) * s;
    double r = pow(q, dn);
    double u = rs.uniform();
    x = 0;
    while (u > r && x < n) {
      u -= r;
      ++x;
      r *= (a / (double)x - s);
      if (r <= 0.0) break;
    }
  } else {
    // BTRS: transformed rejection with squeeze
    const double spq = sqrt(dn * p * q);
    const double b = 1.15 + 2.53 * spq;
    const double a = -0.0873 + 0.0248 * b + 0.01 * p;
    const double c = dn * p + 0.5;
    const double vr = 0.92 - 4.2 / b;
    const double alpha = (2.83 + 5.1 / b) * spq;
    const double lpq = log(p / q);
    const double mo = floor((dn + 1.0) * p);
    const double h = lgamma(mo + 1.0) + lgamma(dn - mo + 1.0);
    while (true) {
      double u = rs.uniform() - 0.5;
      double v = rs.uniform();
      double us = 0.5 - fabs(u);
      double k = floor((2.0 * a / us + b) * u + c);
      if (k < 0.0 || k > dn) continue;
      if (us >= 0.07 && v <= vr) {
        x = (uint64_t)k;
        break;
      }
      v = log(v * alpha / (a / (us * us) + b));
      if (v <= h - lgamma(k + 1.0) - lgamma(dn - k + 1.0) + (k - mo) * lpq) {
        x = (uint64_t)k;
        break;
      }
    }
  }
  return flip ? n - x : x;
}

// One level of the splitting tree: child 2i gets Binomial(cur[i], p0).
__global__ void k_split(const unsigned long long *cur, unsigned long long *next, uint64_t nodes, uint32_t level,
                        double p0, uint64_t key) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nodes; i += (uint64_t)gridDim.x * blockDim.x) {
    Stream rs{fold(fold(key, level), i), 0};
    uint64_t n = cur[i];
    uint64_t left = binomial(n, p0, rs);
    next[2 * i] = left;
    next[2 * i + 1] = n - left;
  }
}

__device__ inline uint32_t rmat_dst(uint64_t key_u, uint32_t u, uint64_t j, uint32_t scale, uint32_t t0, uint32_t t1) {
  uint32_t v = 0;
  uint64_t r = 0;
  for (uint32_t l = 0; l < scale; ++l) {
    if ((l & 1u) == 0) r = draw(key_u, j * 16 + (l >> 1));
    uint32_t x = (l & 1u) ? (uint32_t)r : (uint32_t)(r >> 32);
    uint32_t sbit = (u >> (scale - 1 - l)) & 1u;
    uint32_t dbit = x >= (sbit ? t1 : t0) ? 1u : 0u;
    v |= dbit << (scale - 1 - l);
  }
  return v;
}

// Warp per output row u' (= perm[u]); row u's j-th destination is drawn from
// stream (seed, "dst", u) and relabelled through perm.
__global__ void k_fill_rmat(uint32_t n, uint32_t scale, const uint32_t *inv_perm, const uint32_t *perm,
                            const uint64_t *row_ptr, uint32_t *col_idx, uint64_t key, uint32_t t0, uint32_t t1,
                            int uniform) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t r = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
    const uint32_t up = (uint32_t)r;
    const uint32_t u = inv_perm ? inv_perm[up] : up;
    const uint64_t b = row_ptr[up], e = row_ptr[up + 1];
    const uint64_t ku = fold(key, u);
    for (uint64_t j = lane; j < e - b; j += 32) {
      uint32_t v;
      if (uniform) v = (uint32_t)(((draw(ku, j) >> 32) * (uint64_t)n) >> 32);
      else v = rmat_dst(ku, u, j, scale, t0, t1);
      col_idx[b + j] = perm ? perm[v] : v;
    }
  }
}

__global__ void k_permute_degrees(uint32_t n, const unsigned long long *deg, const uint32_t *perm,
                                  unsigned long long *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[perm ? perm[i] : i] = deg[i];
}

// Feistel bijection on [0, n): 4 rounds over the next even power of two,
// cycle walking back into range.
__device__ inline uint64_t feistel(uint64_t x, uint32_t half, const uint64_t *keys, uint64_t n) {
  const uint64_t hmask = (1ull << half) - 1;
  do {
    uint64_t l = x >> half, r = x & hmask;
    for (int k = 0; k < 4; ++k) {
      uint64_t f = mix64(r ^ keys[k]) & hmask;
      uint64_t nl = r;
      r = l ^ f;
      l = nl;
    }
    x = (l << half) | r;
  } while (x >= n);
  return x;
}

__global__ void k_feistel(uint32_t n, uint32_t half, uint64_t k0, uint64_t k1, uint64_t k2, uint64_t k3,
                          uint32_t *perm, uint32_t *inv) {
  const uint64_t keys[4] = {k0, k1, k2, k3};
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t p = (uint32_t)feistel(i, half, keys, n);
    perm[i] = p;
    if (inv) inv[p] = (uint32_t)i;
  }
}

__global__ void k_invert(uint32_t n, const uint32_t *perm, uint32_t *inv) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    inv[perm[i]] = (uint32_t)i;
}

__global__ void k_histogram(const uint32_t *col_idx, uint64_t m, uint32_t *counts) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[col_idx[i]], 1u);
}

__global__ void k_vals(uint64_t m, uint64_t key, float lo, float hi, float *vals) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t r = draw(key, i) >> 40;
    double u = (double)r * (1.0 / 16777216.0);
    vals[i] = (float)(lo + (hi - lo) * u);
  }
}

// ---- batched Zipf-degree matrices -------------------------------------------

// Zipf(s) on {1..N} by rejection-inversion (Hormann, Derflinger 1996) with
// H(x) = (x^(1-s) - 1) / (1-s), the integral of x^-s (s != 1).
struct ZipfRI {
  double s, N, hx1, hN, sp;
  __device__ double H(double x) const { return (pow(x, 1.0 - s) - 1.0) / (1.0 - s); }
  __device__ double Hinv(double y) const { return pow(1.0 + y * (1.0 - s), 1.0 / (1.0 - s)); }
  __device__ double h(double x) const { return pow(x, -s); }
  __device__ void init(double s_, double N_) {
    s = s_;
    N = N_;
    hx1 = H(1.5) - 1.0;
    hN = H(N + 0.5);
    sp = 2.0 - Hinv(H(2.5) - h(2.0));
  }
  __device__ uint32_t sample(Stream &rs) const {
    for (int it = 0; it < 1000; ++it) {
      const double u = hN + rs.uniform() * (hx1 - hN);
      const double x = Hinv(u);
      double k = floor(x + 0.5);
      if (k < 1.0) k = 1.0;
      if (k > N) k = N;
      if (k - x <= sp || u >= H(k + 0.5) - h(k)) return (uint32_t)k;
    }
    return 1u;
  }
};

__device__ inline uint32_t find_graph(const unsigned long long *off, uint32_t ng, uint64_t x) {
  uint32_t lo = 0, hi = ng;  // largest g with off[g] <= x
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) / 2;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Out-degree of every row of every matrix: round(Z * mean / mu), clamped to [1, n].
__global__ void k_zipf_degrees(uint32_t ng, const unsigned long long *voff, const uint32_t *nv, const double *scale,
                               double s_out, uint64_t key, unsigned long long *deg) {
  const uint64_t total = voff[ng];
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = find_graph(voff, ng, x);
    const uint64_t r = x - voff[g];
    ZipfRI z;
    z.init(s_out, (double)nv[g]);
    Stream rs{fold(fold(key, g), r), 0};
    double d = floor((double)z.sample(rs) * scale[g] + 0.5);
    if (d < 1.0) d = 1.0;
    if (d > (double)nv[g]) d = (double)nv[g];
    deg[x] = (unsigned long long)d;
  }
}

// Row pointers of every matrix inside one buffer: matrix g's n_g + 1 entries
// start at voff[g] + g; ex is the exclusive prefix of the union degrees.
__global__ void k_batch_rowptr(uint32_t ng, const unsigned long long *voff, const unsigned long long *ex,
                               unsigned long long *rp) {
  const uint64_t total = voff[ng];
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total + ng;
       x += (uint64_t)gridDim.x * blockDim.x) {
    // x indexes the row-pointer buffer: graph g owns [voff[g] + g, voff[g+1] + g + 1)
    uint32_t lo = 0, hi = ng;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) / 2;
      if (voff[mid] + mid <= x) lo = mid;
      else hi = mid;
    }
    const uint32_t g = lo;
    const uint64_t i = x - (voff[g] + g);  // 0..n_g
    rp[x] = ex[voff[g] + i] - ex[voff[g]];
  }
}

// Destinations: Zipf(s_in) rank over a seeded Feistel permutation of [0, n_g).
__global__ void k_zipf_dst(uint32_t ng, const unsigned long long *eoff, const uint32_t *nv, double s_in, uint64_t key,
                           uint64_t pkey, uint32_t *col) {
  const uint64_t total = eoff[ng];
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = find_graph(eoff, ng, e);
    const uint64_t le = e - eoff[g];
    const uint32_t n = nv[g];
    ZipfRI z;
    z.init(s_in, (double)n);
    Stream rs{fold(fold(key, g), le), 0};
    const uint32_t rank = z.sample(rs) - 1u;
    uint32_t bits = 2;
    while (bits < 32 && (1u << bits) < n) ++bits;
    if (bits % 2) ++bits;
    const uint64_t gk = fold(pkey, g);
    const uint64_t keys[4] = {fold(gk, 0), fold(gk, 1), fold(gk, 2), fold(gk, 3)};
    col[e] = (uint32_t)feistel(rank, bits / 2, keys, n);
  }
}

inline uint32_t grid_for(uint64_t n, uint32_t threads) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > 65535ull * 8) g = 65535ull * 8;
  if (g < 1) g = 1;
  return (uint32_t)g;
}

}  // namespace

extern "C" {

uint64_t gtgen_stream_key(uint64_t seed, uint64_t id) { return fold(mix64(seed), id); }

// Out-degrees of a 2^scale-vertex R-MAT (or uniform when p0 = 0.5) graph with
// m edges: deg[u] for natural IDs.  tmp and deg hold 2^scale u64 each.
int gtgen_split_degrees(uint32_t scale, uint64_t m, double p0, uint64_t key, unsigned long long *deg,
                        unsigned long long *tmp, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *bufs[2] = {tmp, deg};
  // start so that the last level writes into deg
  int cur = (scale % 2 == 0) ? 1 : 0;  // after `scale` swaps we end in deg
  cudaMemcpyAsync(bufs[cur], &m, 8, cudaMemcpyHostToDevice, s);
  for (uint32_t l = 0; l < scale; ++l) {
    uint64_t nodes = 1ull << l;
    k_split<<<grid_for(nodes, 256), 256, 0, s>>>(bufs[cur], bufs[cur ^ 1], nodes, l, p0, key);
    cur ^= 1;
  }
  if (scale == 0) cudaMemcpyAsync(deg, &m, 8, cudaMemcpyHostToDevice, s);
  cudaError_t e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? 0 : (int)e;
}

int gtgen_permute_degrees(uint32_t n, const unsigned long long *deg, const uint32_t *perm, unsigned long long *out,
                          void *stream) {
  k_permute_degrees<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, deg, perm, out);
  return (int)cudaGetLastError();
}

int gtgen_fill(uint32_t n, uint32_t scale, const uint32_t *inv_perm, const uint32_t *perm, const uint64_t *row_ptr,
               uint32_t *col_idx, uint64_t key, double a, double b, double c, int uniform, void *stream) {
  const double d = 1.0 - a - b - c;
  double p0 = a / (a + b), p1 = c / (c + d);
  uint32_t t0 = (uint32_t)fmin(floor(p0 * 4294967296.0), 4294967295.0);
  uint32_t t1 = (uint32_t)fmin(floor(p1 * 4294967296.0), 4294967295.0);
  uint64_t warps = n;
  uint64_t g = (warps + 7) / 8;
  if (g > 152ull * 64) g = 152ull * 64;
  if (g < 1) g = 1;
  k_fill_rmat<<<(uint32_t)g, 256, 0, (cudaStream_t)stream>>>(n, scale, inv_perm, perm, row_ptr, col_idx, key, t0, t1,
                                                             uniform);
  return (int)cudaGetLastError();
}

int gtgen_feistel(uint32_t n, uint64_t seed, uint32_t *perm, uint32_t *inv, void *stream) {
  uint32_t bits = 2;
  while (bits < 64 && (1ull << bits) < n) ++bits;
  if (bits % 2) ++bits;
  uint32_t half = bits / 2;
  // round keys: fold(fold(mix64(seed), S_PERM=2), r), as in the numpy generator
  uint64_t base = fold(mix64(seed), 2);
  uint64_t k[4];
  for (int r = 0; r < 4; ++r) k[r] = fold(base, (uint64_t)r);
  k_feistel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, half, k[0], k[1], k[2], k[3], perm, inv);
  return (int)cudaGetLastError();
}

int gtgen_invert(uint32_t n, const uint32_t *perm, uint32_t *inv, void *stream) {
  k_invert<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, perm, inv);
  return (int)cudaGetLastError();
}

int gtgen_histogram(const uint32_t *col_idx, uint64_t m, uint32_t *counts, void *stream) {
  k_histogram<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(col_idx, m, counts);
  return (int)cudaGetLastError();
}

int gtgen_vals(uint64_t m, uint64_t key, float lo, float hi, float *vals, void *stream) {
  k_vals<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(m, key, lo, hi, vals);
  return (int)cudaGetLastError();
}

// Batched Zipf matrices (see k_zipf_degrees / k_zipf_dst): voff/eoff are the
// union vertex / edge offsets (ng + 1 entries), nv the sizes, scale[g] =
// mean_g / mu_g.  deg: [voff[ng]] out-degrees (u64).
int gtgen_zipf_degrees(uint32_t ng, const unsigned long long *voff, const uint32_t *nv, const double *scale,
                       double s_out, uint64_t key, unsigned long long *deg, void *stream) {
  k_zipf_degrees<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(ng, voff, nv, scale, s_out, key, deg);
  return (int)cudaGetLastError();
}

int gtgen_batch_rowptr(uint32_t ng, const unsigned long long *voff, const unsigned long long *ex,
                       unsigned long long *rp, void *stream) {
  k_batch_rowptr<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(ng, voff, ex, rp);
  return (int)cudaGetLastError();
}

int gtgen_zipf_dst(uint32_t ng, const unsigned long long *eoff, const uint32_t *nv, double s_in, uint64_t key,
                   uint64_t pkey, uint32_t *col, void *stream) {
  k_zipf_dst<<<152 * 32, 256, 0, (cudaStream_t)stream>>>(ng, eoff, nv, s_in, key, pkey, col);
  return (int)cudaGetLastError();
}

}  // extern "C"
