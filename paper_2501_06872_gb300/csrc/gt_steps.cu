// Steps 0-3 of the transposition on sm_103a: HDV sampling and hash table,
// partition boundaries, in-degree count, HDV insertion points, decoupled
// look-back scan, and the scatter.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {

// ---------------------------------------------------------------------------
// Shared-memory layouts (computed identically on host and device).
// ---------------------------------------------------------------------------
struct SmemLayout {
  uint32_t keys, hvals, hstart, cnt, stage, bars, total;
};

__host__ __device__ inline uint32_t align_up_u32(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// count: keys | hvals | cnt[W][kmax] | stage[W][2][S] | bars[W][2]
// scatter: keys | hvals | hstart[kmax] | cnt[W][kmax] | stage[W][2][S*(1+vals)] | bars[W][2]
__host__ __device__ inline SmemLayout make_layout(bool scatter, uint32_t W, uint32_t kmax, uint32_t tlog2,
                                                   bool staged, uint32_t S, bool vals) {
  SmemLayout L;
  uint32_t T = kmax ? (1u << tlog2) : 0u;
  uint32_t off = 0;
  L.keys = off;
  off += T * 4u;
  L.hvals = off;
  off = align_up_u32(off + T * 2u, 16);
  L.hstart = off;
  if (scatter) off += kmax * 8u;
  L.cnt = off;
  off = align_up_u32(off + W * kmax * 4u, 16);
  L.stage = off;
  if (staged) off += W * 2u * S * 4u * ((scatter && vals) ? 2u : 1u);
  off = align_up_u32(off, 8);
  L.bars = off;
  if (staged) off += W * 2u * 8u;
  L.total = align_up_u32(off, 16);
  return L;
}

uint32_t smem_count_bytes(uint32_t W, uint32_t kmax, uint32_t tlog2, int staged, uint32_t S, int has_vals) {
  return make_layout(false, W, kmax, tlog2, staged != 0, S, has_vals != 0).total;
}
uint32_t smem_scatter_bytes(uint32_t W, uint32_t kmax, uint32_t tlog2, int staged, uint32_t S, int has_vals) {
  return make_layout(true, W, kmax, tlog2, staged != 0, S, has_vals != 0).total;
}

// ---------------------------------------------------------------------------
// Step 0: sampling (Sec. IV-C, Step 0) -> HDV list and hash table.
// ---------------------------------------------------------------------------

// Draws ns random edge positions and counts destination frequencies in a
// global open-addressing table of 2^ts_log2 slots (ns <= 2^(ts_log2-1)).
__global__ void k_sample(const uint32_t *__restrict__ col_idx, uint32_t n, uint64_t m, uint32_t ns,
                         uint64_t seed, uint32_t *skeys, uint32_t *scnt, uint32_t ts_log2) {
  const uint32_t mask = (1u << ts_log2) - 1u;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    uint64_t r = mix64(seed + (uint64_t)(s + 1) * 0x9E3779B97F4A7C15ull);
    uint64_t pos = __umul64hi(r, m);
    uint32_t v = col_idx[pos];
    if (v >= n) continue;  // reported by the count pass
    uint32_t slot = hash_slot(v, ts_log2);
#pragma unroll 1
    for (uint32_t i = 0; i <= mask; ++i) {
      uint32_t old = atomicCAS(&skeys[slot], kEmptyKey, v);
      if (old == kEmptyKey || old == v) {
        atomicAdd(&scnt[slot], 1u);
        break;
      }
      slot = (slot + 1u) & mask;
    }
  }
}

__global__ void k_freq_hist(const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ scnt, uint32_t ts,
                            uint32_t *fhist) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ts; s += gridDim.x * blockDim.x) {
    if (skeys[s] != kEmptyKey) atomicAdd(&fhist[min(scnt[s], kFreqBins - 1u)], 1u);
  }
}

// One CTA of 1024 threads.  A(f) = #keys with (clamped) frequency >= f.
// thr = smallest f >= fmin with A(f) <= kmax; need = kmax - A(thr) ties are
// taken at frequency thr-1 (if thr-1 >= fmin).
__global__ void __launch_bounds__(1024) k_select(const uint32_t *__restrict__ fhist, uint32_t kmax, uint32_t fmin,
                                                 uint32_t *meta) {
  constexpr uint32_t C = kFreqBins / 1024;
  __shared__ uint64_t s_sum[1024];
  __shared__ uint32_t s_f0;
  const uint32_t t = threadIdx.x;
  uint64_t local = 0;
  for (uint32_t i = 0; i < C; ++i) local += fhist[t * C + i];
  s_sum[t] = local;
  if (t == 0) s_f0 = kFreqBins;
  __syncthreads();
  // suffix sums over chunks (Hillis-Steele, 10 steps)
  for (uint32_t off = 1; off < 1024; off <<= 1) {
    uint64_t add = (t + off < 1024) ? s_sum[t + off] : 0;
    __syncthreads();
    s_sum[t] += add;
    __syncthreads();
  }
  // A at the start of my chunk = s_sum[t]; walk my chunk from the top.
  uint64_t above = (t + 1 < 1024) ? s_sum[t + 1] : 0;  // A(t*C + C)
  uint32_t best = kFreqBins;
  uint64_t a = above;
  for (int i = (int)C - 1; i >= 0; --i) {
    a += fhist[t * C + i];  // A(t*C + i)
    if (a <= kmax) best = t * C + (uint32_t)i;
  }
  if (above <= kmax && best == kFreqBins) best = (t + 1) * C;  // boundary case
  atomicMin(&s_f0, best);
  __shared__ unsigned long long s_athr;
  if (t == 0) s_athr = 0;
  __syncthreads();
  const uint32_t thr = s_f0 > fmin ? s_f0 : fmin;
  // A(thr), summed by every thread over its own chunk
  uint64_t part = 0;
  for (uint32_t i = 0; i < C; ++i)
    if (t * C + i >= thr) part += fhist[t * C + i];
  if (part) atomicAdd(&s_athr, (unsigned long long)part);
  __syncthreads();
  if (t == 0) {
    const uint64_t athr = s_athr;
    uint32_t need = 0;
    if (thr >= 1 && thr - 1 >= fmin && athr < kmax) need = (uint32_t)(kmax - athr);
    meta[kMetaThr] = thr;
    meta[kMetaNeed] = need;
  }
}

__global__ void k_collect(const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ scnt, uint32_t ts,
                          uint32_t *meta, uint32_t *cand, uint32_t kmax, uint32_t *ties) {
  const uint32_t thr = meta[kMetaThr];
  const uint32_t need = meta[kMetaNeed];
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ts; s += gridDim.x * blockDim.x) {
    uint32_t key = skeys[s];
    if (key == kEmptyKey) continue;
    uint32_t c = min(scnt[s], kFreqBins - 1u);
    if (c >= thr) {
      uint32_t i = atomicAdd(&meta[kMetaNCand], 1u);
      if (i < kmax) cand[i] = key;
    } else if (need > 0 && c + 1u == thr) {
      uint32_t i = atomicAdd(&meta[kMetaNTie], 1u);
      if (i < kTieCap) ties[i] = key;
    }
  }
}

// Bitonic sort of buf[0..len) (len a power of two) ascending, whole CTA.
__device__ void cta_bitonic_u32(uint32_t *buf, uint32_t len) {
  for (uint32_t k = 2; k <= len; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        uint32_t p = i ^ j;
        if (p > i) {
          bool up = (i & k) == 0;
          uint32_t a = buf[i], b = buf[p];
          if ((a > b) == up) {
            buf[i] = b;
            buf[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

// One CTA: picks the `need` smallest-ID ties, sorts the HDV list by ID (the
// compact index of an HDV is its rank), and builds the hash-table image.
__global__ void __launch_bounds__(1024) k_finalize(uint32_t *meta, const uint32_t *__restrict__ cand,
                                                   const uint32_t *__restrict__ ties, uint32_t kmax,
                                                   uint32_t *hdv_ids, uint32_t *hkeys, uint16_t *hvals,
                                                   uint32_t tlog2) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t *tbuf = sm;               // kTieCap
  uint32_t *cbuf = sm + kTieCap;     // kMaxHdv
  uint32_t *tk = cbuf + kMaxHdv;     // 2^tlog2 keys
  uint16_t *tv = (uint16_t *)(tk + (1u << tlog2));
  const uint32_t nc = min(meta[kMetaNCand], kmax);
  const uint32_t nt = min(meta[kMetaNTie], kTieCap);
  const uint32_t need = meta[kMetaNeed];
  uint32_t tl = 1;
  while (tl < nt) tl <<= 1;
  for (uint32_t i = threadIdx.x; i < tl; i += blockDim.x) tbuf[i] = (i < nt) ? ties[i] : kEmptyKey;
  __syncthreads();
  if (nt > 1) cta_bitonic_u32(tbuf, tl);
  const uint32_t take = min(min(need, nt), kmax - nc);
  const uint32_t K = nc + take;
  uint32_t cl = 1;
  while (cl < K) cl <<= 1;
  for (uint32_t i = threadIdx.x; i < cl; i += blockDim.x) {
    uint32_t x = kEmptyKey;
    if (i < nc) x = cand[i];
    else if (i < K) x = tbuf[i - nc];
    cbuf[i] = x;
  }
  __syncthreads();
  if (K > 1) cta_bitonic_u32(cbuf, cl);
  const uint32_t T = 1u << tlog2, mask = T - 1u;
  for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) tk[i] = kEmptyKey;
  __syncthreads();
  for (uint32_t h = threadIdx.x; h < K; h += blockDim.x) {
    uint32_t v = cbuf[h];
    hdv_ids[h] = v;
    uint32_t s = hash_slot(v, tlog2);
    for (uint32_t i = 0; i <= mask; ++i) {
      uint32_t old = atomicCAS(&tk[s], kEmptyKey, v);
      if (old == kEmptyKey) {
        tv[s] = (uint16_t)h;
        break;
      }
      s = (s + 1u) & mask;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) {
    hkeys[i] = tk[i];
    hvals[i] = tv[i];
  }
  if (threadIdx.x == 0) meta[kMetaK] = K;
}

// ---------------------------------------------------------------------------
// Partition boundaries (part2tid of Algorithm 2).  Partitions are equal in
// cost, where an edge costs 8 units and a row 1 unit (a warp walks rows 256
// at a time but edges 32 at a time), so long runs of empty rows do not make
// stragglers.  A boundary falls at the start of its row unless the row is
// longer than half a partition (then the row is split and its parts are
// processed by neighbouring warps).  Warp p owns edges [part[p], part[p+1])
// in Steps 1 and 3.
// ---------------------------------------------------------------------------
__global__ void k_partition(const uint64_t *__restrict__ row_ptr, uint32_t n_rows, uint64_t m, uint32_t P,
                            uint64_t psize, int allow_split, unsigned long long *part, uint32_t *status) {
  const uint32_t n = n_rows;
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  if (p == 0) {
    part[0] = 0;
    if (row_ptr[0] != 0 || row_ptr[n] != m) set_status(status, GT_ERR_BAD_ROW_PTR);
    return;
  }
  if (p == P) {
    part[P] = m;
    return;
  }
  // cost(r) = 8 * row_ptr[r] + r is non-decreasing in r for a valid row_ptr
  const uint64_t total = 8ull * m + n;
  const uint64_t d = (uint64_t)(((unsigned __int128)total * p) / P);
  uint32_t lo = 0, hi = n;  // largest r in [0, n) with cost(r) <= d
  while (hi - lo > 1) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (8ull * row_ptr[mid] + mid <= d) lo = mid;
    else hi = mid;
  }
  const uint64_t rs = row_ptr[lo], re = row_ptr[lo + 1];
  uint64_t b = rs;
  if (allow_split && re - rs > psize / 2) {
    const uint64_t c0 = 8ull * rs + lo;
    uint64_t inside = d > c0 ? (d - c0) / 8 : 0;
    b = rs + inside;
    if (b > re) b = re;
  }
  if (b > m) b = m;
  part[p] = b;
}

// Partitioned form: the bucketed edge list has no rows to respect, so warp p
// owns the equal range [p * psize, (p + 1) * psize) (clipped to m); rows cut
// by a boundary are handled as split rows.
__global__ void k_partition_even(uint32_t P, uint64_t m, uint64_t psize, unsigned long long *part) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p <= P) part[p] = min64((uint64_t)p * psize, m);
}

// Two-phase Step 3 (Sec. V-F): warp p's partition [part[p], part[p+1]) is
// split into a head of 80 % of its edges and a tail, part2[2p], part2[2p+1],
// part2[2p+2].  Where rows may not be split, the split moves to a row start
// inside the partition.
__global__ void k_split_tails(const uint64_t *__restrict__ row_ptr, uint32_t n_rows,
                              const unsigned long long *__restrict__ part, uint32_t P, int allow_split,
                              unsigned long long *part2) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  if (p == P) {
    part2[2 * (size_t)P] = part[P];
    return;
  }
  const uint64_t e0 = part[p], e1 = part[p + 1];
  uint64_t b = e1 > e0 ? e0 + ((e1 - e0) * 4) / 5 : e0;
  if (!allow_split && b > e0 && b < e1) {
    uint32_t lo = 0, hi = n_rows;  // the row holding edge b
    while (hi - lo > 1) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (row_ptr[mid] <= b) lo = mid;
      else hi = mid;
    }
    const uint64_t rs = row_ptr[lo];
    b = rs >= e0 ? rs : min64(row_ptr[lo + 1], e1);
  }
  part2[2 * (size_t)p] = e0;
  part2[2 * (size_t)p + 1] = b;
}

// ---------------------------------------------------------------------------
// Step 1: in-degree count (Algorithm 2, Step 1).
// ---------------------------------------------------------------------------
struct CountArgs {
  const uint32_t *col_idx;
  uint32_t n;
  uint64_t m;
  const unsigned long long *part;
  const uint32_t *hkeys;
  const uint16_t *hvals;
  uint32_t tlog2, kmax;
  const uint32_t *meta;
  uint32_t *deg;
  uint32_t *hdv_cnt;
  unsigned long long *meta64;
  uint32_t *status;
  uint32_t stage_edges;
  int vec_ok;  // col_idx is 16-byte aligned
  int steal;   // part holds 2P + 1 bounds: warp p counts ranges 2p and 2p + 1 separately
};

template <bool HDV, bool AGG>
__device__ __forceinline__ void count_one(const CountArgs &a, const uint32_t *keys, const uint16_t *hv,
                                          uint32_t *mycnt, uint32_t K, uint32_t v, bool act, uint32_t &hdv_local) {
  bool valid = act && v < a.n;
  if (act && v >= a.n) set_status(a.status, GT_ERR_OUT_OF_RANGE);
  int h = -1;
  if (HDV && valid && K) h = hdv_lookup(keys, hv, a.tlog2, v);
  if (h >= 0) {
    atomicAdd(&mycnt[h], 1u);
    ++hdv_local;
  }
  bool ldv = valid && h < 0;
  if (AGG) {
    uint32_t key = ldv ? v : kEmptyKey;
    uint32_t mm = __match_any_sync(kFull, key);
    if (ldv && (mm & lanemask_lt()) == 0) red_add_u32(&a.deg[v], __popc(mm));
  } else if (ldv) {
    red_add_u32(&a.deg[v], 1u);
  }
}

template <bool HDV, bool AGG, bool STAGED>
__global__ void __launch_bounds__(1024) k_count(CountArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t W = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const SmemLayout L = make_layout(false, W, HDV ? a.kmax : 0, a.tlog2, STAGED, a.stage_edges, false);
  uint32_t *keys = (uint32_t *)(smem + L.keys);
  uint16_t *hv = (uint16_t *)(smem + L.hvals);
  uint32_t *cnt = (uint32_t *)(smem + L.cnt);
  const uint32_t K = HDV ? a.meta[kMetaK] : 0u;
  if (HDV) {
    const uint32_t T = 1u << a.tlog2;
    for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) {
      keys[i] = a.hkeys[i];
      hv[i] = a.hvals[i];
    }
    for (uint32_t i = threadIdx.x; i < W * a.kmax; i += blockDim.x) cnt[i] = 0u;
  }
  __syncthreads();
  const uint32_t p = blockIdx.x * W + w;
  uint32_t *mycnt = cnt + w * a.kmax;
  uint32_t hdv_local = 0;
  // the warp's partition, or with the two-phase Step 3 its head (80 %) and
  // tail (20 %) as two ranges with separate HDV counts
  const uint32_t nsub = a.steal ? 2u : 1u;
  for (uint32_t sub = 0; sub < nsub; ++sub) {
  const uint32_t sp = a.steal ? 2u * p + sub : p;
  const uint64_t e0 = a.part[sp], e1 = a.part[sp + 1];

  if (!STAGED && !a.vec_ok) {
    for (uint64_t c = e0; c < e1; c += 32) {
      uint64_t e = c + lane;
      bool act = e < e1;
      uint32_t v = act ? a.col_idx[e] : kEmptyKey;
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, v, act, hdv_local);
    }
  } else if (!STAGED) {
    // head up to a 16-byte boundary, uint4 body, tail
    uint64_t a4 = min64((e0 + 3) & ~3ull, e1);
    uint64_t b4 = max64(a4, e1 & ~3ull);
    {
      uint64_t e = e0 + lane;
      bool act = e < a4;
      uint32_t v = act ? a.col_idx[e] : kEmptyKey;
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, v, act, hdv_local);
    }
    const uint4 *vec = reinterpret_cast<const uint4 *>(a.col_idx);
    for (uint64_t q0 = a4 >> 2; q0 < (b4 >> 2); q0 += 32) {
      uint64_t q = q0 + lane;
      bool act = q < (b4 >> 2);
      uint4 x = act ? __ldcs(vec + q) : make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, x.x, act, hdv_local);
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, x.y, act, hdv_local);
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, x.z, act, hdv_local);
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, x.w, act, hdv_local);
    }
    {
      uint64_t e = b4 + lane;
      bool act = e < e1 && e >= a4;
      uint32_t v = act ? a.col_idx[e] : kEmptyKey;
      count_one<HDV, AGG>(a, keys, hv, mycnt, K, v, act, hdv_local);
    }
  } else if (e0 < e1) {
    // Bulk-copy staging: two buffers of S edges per warp, filled by the TMA
    // engine (cp.async.bulk) while the warp consumes the other one.
    const uint32_t S = a.stage_edges;
    uint32_t *sbuf = (uint32_t *)(smem + L.stage) + (size_t)w * 2u * S;
    uint64_t *bars = (uint64_t *)(smem + L.bars) + w * 2u;
    if (lane == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      fence_barrier_init();
    }
    __syncwarp();
    const uint64_t ts0 = e0 & ~3ull;
    const uint64_t mfloor = a.m & ~3ull;  // bulk copies never read past this
    const uint64_t ntile = (e1 - ts0 + S - 1) / S;
    auto issue = [&](uint64_t i) {
      if (lane == 0 && i < ntile) {
        uint64_t ts = ts0 + i * S;
        uint64_t te = min64(ts + S, e1);
        uint64_t ce = min64((te + 3) & ~3ull, mfloor);
        uint32_t bytes = ce > ts ? (uint32_t)((ce - ts) * 4u) : 0u;
        uint32_t b = (uint32_t)(i & 1u);
        fence_proxy_async();
        mbar_arrive_expect_tx(&bars[b], bytes);
        if (bytes) bulk_g2s(sbuf + b * S, a.col_idx + ts, bytes, &bars[b]);
      }
    };
    issue(0);
    issue(1);
    uint64_t waited = 0;
    bool ok = true;
    for (uint64_t i = 0; i < ntile; ++i) {
      const uint32_t b = (uint32_t)(i & 1u);
      if (!mbar_wait(&bars[b], (uint32_t)((i >> 1) & 1u))) {
        ok = false;
        break;
      }
      waited = i + 1;
      const uint64_t ts = ts0 + i * S;
      const uint64_t te = min64(ts + S, e1);
      const uint64_t ce = min64((te + 3) & ~3ull, mfloor);
      for (uint32_t j = lane; j < S; j += 32) {
        uint64_t e = ts + j;
        bool act = e >= e0 && e < te;
        uint32_t v = kEmptyKey;
        if (act) v = (e < ce) ? sbuf[b * S + j] : a.col_idx[e];
        count_one<HDV, AGG>(a, keys, hv, mycnt, K, v, act, hdv_local);
      }
      __syncwarp();
      issue(i + 2);
    }
    if (!ok) {
      set_status(a.status, GT_ERR_TIMEOUT);
      // let copies already issued land before the CTA's shared memory goes away
      for (uint64_t i = waited; i < min64(waited + 2, ntile); ++i) mbar_wait(&bars[i & 1u], (uint32_t)((i >> 1) & 1u));
    }
  }
  __syncwarp();
  if (HDV) {
    for (uint32_t h = lane; h < K; h += 32) {
      a.hdv_cnt[(size_t)sp * a.kmax + h] = mycnt[h];
      mycnt[h] = 0u;
    }
    __syncwarp();
  }
  }  // ranges of the warp
  if (HDV) {
    for (int o = 16; o > 0; o >>= 1) hdv_local += __shfl_xor_sync(kFull, hdv_local, o);
    if (lane == 0 && hdv_local) atomicAdd(&a.meta64[0], (unsigned long long)hdv_local);
  }
}

// ---------------------------------------------------------------------------
// Step 2a: HDV insertion points.  hdv_cnt[p][h] becomes the number of edges
// into HDV h in partitions before p; the total is written to deg[hdv_ids[h]].
// Block (32, 32): x = HDV within a group of 32, y = slice of partitions.
// ---------------------------------------------------------------------------
__global__ void k_hdv_colscan(uint32_t *hdv_cnt, uint32_t P, uint32_t kmax, const uint32_t *__restrict__ meta,
                              const uint32_t *__restrict__ hdv_ids, uint32_t *deg, uint32_t *status) {
  __shared__ uint64_t s[32][33];
  const uint32_t x = threadIdx.x, y = threadIdx.y;
  const uint32_t h = blockIdx.x * 32 + x;
  const uint32_t K = meta[kMetaK];
  const bool act = h < K;
  const uint32_t chunk = (P + 31) / 32;
  const uint32_t p0 = min(y * chunk, P), p1 = min(p0 + chunk, P);
  uint64_t sum = 0;
  if (act)
    for (uint32_t p = p0; p < p1; ++p) sum += hdv_cnt[(size_t)p * kmax + h];
  s[y][x] = sum;
  __syncthreads();
  if (y == 0) {
    uint64_t run = 0;
    for (uint32_t i = 0; i < 32; ++i) {
      uint64_t t = s[i][x];
      s[i][x] = run;
      run += t;
    }
    if (act) {
      if (run > 0xFFFFFFFFull) set_status(status, GT_ERR_UNSUPPORTED);
      deg[hdv_ids[h]] = (uint32_t)run;
    }
  }
  __syncthreads();
  if (act) {
    uint64_t run = s[y][x];
    for (uint32_t p = p0; p < p1; ++p) {
      size_t idx = (size_t)p * kmax + h;
      uint32_t c = hdv_cnt[idx];
      hdv_cnt[idx] = (uint32_t)run;
      run += c;
    }
  }
}

// The same scan for many partitions (the partitioned form has one per range
// of warp_edges edges): grid (HDV groups of 32, Q slices of partitions).
// k_hdv_slicesum writes each slice's total per HDV to psum[q][h];
// k_hdv_slicescan turns them into slice starting points (one thread per HDV)
// and writes the totals; k_hdv_sliceapply rewrites each slice's counts as
// insertion points from its starting point.
__device__ __forceinline__ void hdv_slice(uint32_t P, uint32_t Q, uint32_t &p0, uint32_t &p1) {
  const uint32_t cq = (P + Q - 1) / Q;
  const uint32_t q0 = min(blockIdx.y * cq, P), q1 = min(q0 + cq, P);
  const uint32_t chunk = (q1 - q0 + 31) / 32;
  p0 = min(q0 + threadIdx.y * chunk, q1);
  p1 = min(p0 + chunk, q1);
}

__global__ void k_hdv_slicesum(const uint32_t *__restrict__ hdv_cnt, uint32_t P, uint32_t Q, uint32_t kmax,
                               const uint32_t *__restrict__ meta, unsigned long long *psum) {
  __shared__ uint64_t s[32][33];
  const uint32_t x = threadIdx.x, y = threadIdx.y, h = blockIdx.x * 32 + x;
  const bool act = h < meta[kMetaK];
  uint32_t p0, p1;
  hdv_slice(P, Q, p0, p1);
  uint64_t sum = 0;
  if (act)
    for (uint32_t p = p0; p < p1; ++p) sum += hdv_cnt[(size_t)p * kmax + h];
  s[y][x] = sum;
  __syncthreads();
  if (y == 0 && act) {
    uint64_t t = 0;
    for (uint32_t i = 0; i < 32; ++i) t += s[i][x];
    psum[(size_t)blockIdx.y * kmax + h] = t;
  }
}

__global__ void k_hdv_slicescan(unsigned long long *psum, uint32_t Q, uint32_t kmax, const uint32_t *__restrict__ meta,
                                const uint32_t *__restrict__ hdv_ids, uint32_t *deg, uint32_t *status) {
  const uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= meta[kMetaK]) return;
  uint64_t run = 0;
  for (uint32_t q = 0; q < Q; ++q) {
    const size_t i = (size_t)q * kmax + h;
    const uint64_t t = psum[i];
    psum[i] = run;
    run += t;
  }
  if (run > 0xFFFFFFFFull) set_status(status, GT_ERR_UNSUPPORTED);
  deg[hdv_ids[h]] = (uint32_t)run;
}

__global__ void k_hdv_sliceapply(uint32_t *hdv_cnt, uint32_t P, uint32_t Q, uint32_t kmax,
                                 const uint32_t *__restrict__ meta, const unsigned long long *__restrict__ psum) {
  __shared__ uint64_t s[32][33];
  const uint32_t x = threadIdx.x, y = threadIdx.y, h = blockIdx.x * 32 + x;
  const bool act = h < meta[kMetaK];
  uint32_t p0, p1;
  hdv_slice(P, Q, p0, p1);
  uint64_t sum = 0;
  if (act)
    for (uint32_t p = p0; p < p1; ++p) sum += hdv_cnt[(size_t)p * kmax + h];
  s[y][x] = sum;
  __syncthreads();
  if (y == 0) {
    uint64_t run = act ? psum[(size_t)blockIdx.y * kmax + h] : 0;
    for (uint32_t i = 0; i < 32; ++i) {
      const uint64_t t = s[i][x];
      s[i][x] = run;
      run += t;
    }
  }
  __syncthreads();
  if (act) {
    uint64_t run = s[y][x];
    for (uint32_t p = p0; p < p1; ++p) {
      const size_t idx = (size_t)p * kmax + h;
      const uint32_t c = hdv_cnt[idx];
      hdv_cnt[idx] = (uint32_t)run;
      run += c;
    }
  }
}

// ---------------------------------------------------------------------------
// Step 2b: single-pass decoupled look-back exclusive scan deg -> col_ptr
// (Merrill & Garland 2016).  Tile status words pack a 2-bit flag (1 =
// aggregate, 2 = inclusive prefix) over a 62-bit value.  Also writes the LDV
// insertion points (cursor = col_ptr) and validates row_ptr.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = kScanTile / kScanThreads;  // 16
static_assert(kScanItems == 16, "scan layout");
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kValMask = (1ull << 62) - 1;

__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t *__restrict__ deg, uint32_t n, uint32_t n_rows,
                                                       uint64_t m, const uint64_t *__restrict__ row_ptr, uint64_t *col_ptr,
                                                       unsigned long long *cursor, unsigned long long *state,
                                                       uint32_t *meta, uint32_t *status) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_prefix;
  const uint32_t t = threadIdx.x, lane = t & 31u, wid = t >> 5;
  if (t == 0) s_tile = atomicAdd(&meta[kMetaScanTicket], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * kScanTile + (uint64_t)t * kScanItems;
  uint32_t d[kScanItems];
  if (base + kScanItems <= n) {
    const uint4 *p4 = reinterpret_cast<const uint4 *>(deg + base);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint4 q = p4[i];
      d[4 * i] = q.x;
      d[4 * i + 1] = q.y;
      d[4 * i + 2] = q.z;
      d[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) d[i] = (base + i < n) ? deg[base + i] : 0u;
  }
  // row_ptr validation on the same index range (the grid covers max(n, n_rows))
  if (row_ptr) {
    bool bad = false;
    for (int i = 0; i < kScanItems; ++i) {
      uint64_t r = base + i;
      if (r < n_rows && row_ptr[r] > row_ptr[r + 1]) bad = true;
    }
    if (bad) set_status(status, GT_ERR_BAD_ROW_PTR);
  }
  uint64_t tsum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) tsum += d[i];
  // block exclusive scan of thread sums
  uint64_t inc = tsum;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (t == 0) {
    uint64_t run = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) {
      uint64_t x = s_warp[i];
      s_warp[i] = run;
      run += x;
    }
    // publish this tile's aggregate (tile 0 publishes its inclusive prefix)
    const uint64_t agg = run;
    st_volatile_u64((uint64_t *)&state[tile], (tile == 0 ? kFlagInc : kFlagAgg) | (agg & kValMask));
    s_prefix = (tile == 0) ? 0ull : agg;  // the look-back warp reads the aggregate from here
  }
  __syncthreads();
  if (tile != 0 && wid == 0) {
    const uint64_t agg = s_prefix;
    uint64_t excl = 0;
    int64_t look = (int64_t)tile - 1;
    bool timed_out = false;
    while (true) {
      int64_t idx = look - (int64_t)lane;
      uint64_t st = kFlagInc;  // before tile 0: inclusive prefix 0
      if (idx >= 0) {
        uint32_t spins = 0;
        st = ld_volatile_u64((const uint64_t *)&state[idx]);
        while ((st >> 62) == 0) {
          if (++spins > kSpinLimit) {
            timed_out = true;
            st = kFlagInc;
            break;
          }
          __nanosleep(64);
          st = ld_volatile_u64((const uint64_t *)&state[idx]);
        }
      }
      uint32_t incmask = __ballot_sync(kFull, (st >> 62) == 2);
      uint64_t val = st & kValMask;
      if (incmask) {
        uint32_t first = __ffs(incmask) - 1;
        uint64_t v = (lane <= first) ? val : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        excl += v;
        break;
      }
      for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
      excl += val;
      look -= 32;
    }
    if (lane == 0) {
      if (timed_out) set_status(status, GT_ERR_TIMEOUT);
      st_volatile_u64((uint64_t *)&state[tile], kFlagInc | ((excl + agg) & kValMask));
      s_prefix = excl;
    }
  }
  __syncthreads();
  uint64_t run = s_prefix + s_warp[wid] + (inc - tsum);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t idx = base + i;
    if (idx < n) {
      col_ptr[idx] = run;
      if (cursor) cursor[idx] = run;
    }
    run += d[i];
    if (idx + 1 == n) {
      col_ptr[n] = run;
      if (run != m) set_status(status, GT_ERR_OUT_OF_RANGE);
    }
  }
}

cudaError_t launch_scan(const uint32_t *deg, uint32_t n, uint64_t m, const uint64_t *row_ptr, uint64_t *col_ptr,
                        unsigned long long *cursor, unsigned long long *state, uint32_t ntiles, uint32_t *meta,
                        uint32_t *status, cudaStream_t s) {
  k_scan<<<ntiles, kScanThreads, 0, s>>>(deg, n, n, m, row_ptr, col_ptr, cursor, state, meta, status);
  return cudaGetLastError();
}

__global__ void k_hdv_start(const uint32_t *__restrict__ meta, const uint32_t *__restrict__ hdv_ids,
                            const uint64_t *__restrict__ col_ptr, unsigned long long *hdv_start) {
  uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < meta[kMetaK]) hdv_start[h] = col_ptr[hdv_ids[h]];
}

// ---------------------------------------------------------------------------
// Step 3: scatter (Algorithm 2, Step 3).  Warp p revisits edges
// [part[p], part[p+1]) in CSR order, 32 per step.  HDV edges take slot
// col_ptr[h] + (edges into h in earlier partitions) + (earlier edges into h
// in this partition); LDV edges take slots from atomic cursors, one
// aggregated atomic per distinct destination per step.  Because a warp waits
// for each step's atomics before issuing the next step's, the slots a warp
// takes in one LDV list increase along its edges.
// ---------------------------------------------------------------------------
struct ScatterArgs {
  const uint64_t *row_ptr;
  const uint32_t *col_idx;
  const float *vals;
  uint32_t n;       // columns: destinations lie in [0, n)
  uint32_t n_rows;  // rows: row_ptr has n_rows + 1 entries
  uint64_t m;
  const unsigned long long *part;
  const uint32_t *hkeys;
  const uint16_t *hvals;
  uint32_t tlog2, kmax;
  const uint32_t *meta;
  const uint32_t *hdv_off;
  const unsigned long long *hdv_start;
  unsigned long long *cursor;
  const uint64_t *col_ptr;
  uint32_t *row_idx;
  float *vals_out;
  unsigned long long *ldv64;  // weighted, sorted output: LDV entries go here (one 8-byte store); null = outputs
  uint32_t *status;
  int flag_mode;
  uint32_t stage_edges;
  unsigned long long *ptime;  // optional [2 * P]: global-timer ns at the start and end of each warp's work
  // two-phase Step 3 (Sec. V-F): part holds the 2P + 1 head / tail bounds,
  // hdv_off their insertion points; each warp does its head, then claims
  // tails from *steal_next until all P are taken
  int steal;
  uint32_t P;
  uint32_t *steal_next;
  // partitioned form: the source of edge e is src[e] (the edge list is
  // bucketed by destination, so there are no rows to search); split-row tags
  // carry the edge's position e in the bucketed list
  const uint32_t *src = nullptr;
  // unsorted weighted output: every entry (HDV ones too) goes to ldv64 as one
  // 8-byte store; k_unpack then streams them to row_idx / vals_out
  int pack_all = 0;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <bool HDV, bool VALS, bool STAGED>
__global__ void __launch_bounds__(1024) k_scatter(ScatterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (cta_status_set(a.status)) return;  // invalid input: write nothing
  const uint32_t W = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const SmemLayout L = make_layout(true, W, HDV ? a.kmax : 0, a.tlog2, STAGED, a.stage_edges, VALS);
  uint32_t *keys = (uint32_t *)(smem + L.keys);
  uint16_t *hv = (uint16_t *)(smem + L.hvals);
  unsigned long long *hstart = (unsigned long long *)(smem + L.hstart);
  uint32_t *cur = (uint32_t *)(smem + L.cnt);
  const uint32_t K = HDV ? a.meta[kMetaK] : 0u;
  const uint32_t p = blockIdx.x * W + w;
  if (HDV) {
    const uint32_t T = 1u << a.tlog2;
    for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) {
      keys[i] = a.hkeys[i];
      hv[i] = a.hvals[i];
    }
    for (uint32_t i = threadIdx.x; i < K; i += blockDim.x) hstart[i] = a.hdv_start[i];
  }
  __syncthreads();
  if (a.ptime && lane == 0) a.ptime[2 * (size_t)p] = global_ns();
  uint32_t *mycur = cur + w * a.kmax;

  // Range sp of the edge sequence, [part[sp], part[sp + 1]), with its own HDV
  // insertion points: the warp's partition, or a head or tail of one.
  auto process = [&](uint32_t sp) {
  const uint64_t e0 = a.part[sp], e1 = a.part[sp + 1];
  if (HDV) {
    for (uint32_t h = lane; h < K; h += 32) mycur[h] = a.hdv_off[(size_t)sp * a.kmax + h];
    __syncwarp();
  }
  if (e0 >= e1) return;

  // rows at both ends of the partition (they may be shared with neighbours)
  uint32_t row_first, row_last;
  if (a.src) {
    row_first = a.src[e0];
    row_last = a.src[e1 - 1];
  } else {
    uint32_t lo = 0, hi = a.n_rows;
    while (hi - lo > 1) {
      uint32_t mid = lo + (hi - lo) / 2;
      if (a.row_ptr[mid] <= e0) lo = mid;
      else hi = mid;
    }
    row_first = lo;
    lo = row_first;
    hi = a.n_rows;
    while (hi - lo > 1) {
      uint32_t mid = lo + (hi - lo) / 2;
      if (a.row_ptr[mid] <= e1 - 1) lo = mid;
      else hi = mid;
    }
    row_last = lo;
  }
  // a row run continues past an end of the range: in the bucketed list, the
  // row's edges into one destination range are consecutive
  const uint64_t rs_first = a.src ? 0 : a.row_ptr[row_first], rs_last = a.src ? 0 : a.row_ptr[row_last];
  const bool split_first =
      VALS && a.flag_mode && (a.src ? (e0 > 0 && a.src[e0 - 1] == row_first) : rs_first < e0);
  const bool split_last =
      VALS && a.flag_mode && (a.src ? (e1 < a.m && a.src[e1] == row_last) : a.row_ptr[row_last + 1] > e1);
  uint32_t u_lo = row_first;

  auto step = [&](uint64_t e, bool act, uint32_t v, float wv) {
    uint32_t my_u;
    if (a.src) {
      my_u = act ? __ldcs(a.src + e) : 0u;
    } else {
      my_u = find_row(a.row_ptr, a.n_rows, u_lo, e, act, lane, a.status);
      uint32_t last_lane = 31u - __clz(__ballot_sync(kFull, act) | 1u);
      u_lo = __shfl_sync(kFull, my_u, last_lane);
    }
    bool valid = act && v < a.n;
    int h = -1;
    if (HDV && valid && K) h = hdv_lookup(keys, hv, a.tlog2, v);
    unsigned long long slot = 0;
    if (HDV) {
      uint32_t hk = (h >= 0) ? (uint32_t)h : kEmptyKey;
      uint32_t mm = __match_any_sync(kFull, hk);
      uint32_t base = 0;
      if (h >= 0) {
        base = mycur[h];
        slot = hstart[h] + base + __popc(mm & lanemask_lt());
      }
      __syncwarp();
      if (h >= 0 && (mm & lanemask_lt()) == 0) mycur[h] = base + __popc(mm);
      __syncwarp();
    }
    bool ldv = valid && h < 0;
    uint32_t key = ldv ? v : kEmptyKey;
    uint32_t mm2 = __match_any_sync(kFull, key);
    uint32_t leader = __ffs(mm2) - 1;
    unsigned long long b = 0;
    if (ldv && lane == leader) b = atomicAdd(&a.cursor[v], (unsigned long long)__popc(mm2));
    b = __shfl_sync(kFull, b, leader);
    if (ldv) slot = b + __popc(mm2 & lanemask_lt());
    if (valid) {
      uint32_t uu = my_u;
      uint32_t wbits = VALS ? __float_as_uint(wv) : 0u;
      if (VALS && ldv && ((split_first && my_u == row_first) || (split_last && my_u == row_last))) {
        // split row: tag the entry and carry its position in the row; the
        // LDV sort orders tagged duplicates by it and re-reads the value.
        if (a.col_ptr[v + 1] - a.col_ptr[v] >= 2) {
          uu |= kSplitFlag;
          wbits = a.src ? (uint32_t)e : (uint32_t)(e - (my_u == row_first ? rs_first : rs_last));
        }
      }
      if (VALS && a.ldv64 && (ldv || a.pack_all)) {  // LDV entries wait in the scratch for the list sort
        a.ldv64[slot] = ((unsigned long long)wbits << 32) | uu;
      } else {
        a.row_idx[slot] = uu;
        if (VALS) a.vals_out[slot] = __uint_as_float(wbits);
      }
    }
    asm volatile("" ::: "memory");
  };

  if (!STAGED) {
    // the next chunk's loads are in flight while this chunk waits on its atomics
    uint64_t e = e0 + lane;
    bool act = e < e1;
    uint32_t v = act ? __ldcs(a.col_idx + e) : kEmptyKey;
    float wv = (VALS && act) ? __ldcs(a.vals + e) : 0.f;
#pragma unroll 1
    for (uint64_t c = e0; c < e1; c += 32) {
      const uint64_t en = c + 32 + lane;
      const bool actn = en < e1;
      uint32_t vn = kEmptyKey;
      float wn = 0.f;
      if (actn) {
        vn = __ldcs(a.col_idx + en);
        if (VALS) wn = __ldcs(a.vals + en);
      }
      step(e, act, v, wv);
      e = en;
      act = actn;
      v = vn;
      wv = wn;
    }
  } else {
    const uint32_t S = a.stage_edges;
    uint32_t *sbuf = (uint32_t *)(smem + L.stage) + (size_t)w * 2u * S * (VALS ? 2u : 1u);
    uint32_t *svals = sbuf + 2u * S;  // used only when VALS
    uint64_t *bars = (uint64_t *)(smem + L.bars) + w * 2u;
    if (lane == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      fence_barrier_init();
    }
    __syncwarp();
    const uint64_t ts0 = e0 & ~3ull;
    const uint64_t mfloor = a.m & ~3ull;
    const uint64_t ntile = (e1 - ts0 + S - 1) / S;
    auto issue = [&](uint64_t i) {
      if (lane == 0 && i < ntile) {
        uint64_t ts = ts0 + i * S;
        uint64_t te = min64(ts + S, e1);
        uint64_t ce = min64((te + 3) & ~3ull, mfloor);
        uint32_t bytes = ce > ts ? (uint32_t)((ce - ts) * 4u) : 0u;
        uint32_t b = (uint32_t)(i & 1u);
        fence_proxy_async();
        mbar_arrive_expect_tx(&bars[b], VALS ? 2u * bytes : bytes);
        if (bytes) {
          bulk_g2s(sbuf + b * S, a.col_idx + ts, bytes, &bars[b]);
          if (VALS) bulk_g2s(svals + b * S, a.vals + ts, bytes, &bars[b]);
        }
      }
    };
    issue(0);
    issue(1);
    uint64_t waited = 0;
    bool ok = true;
#pragma unroll 1
    for (uint64_t i = 0; i < ntile; ++i) {
      const uint32_t b = (uint32_t)(i & 1u);
      if (!mbar_wait(&bars[b], (uint32_t)((i >> 1) & 1u))) {
        ok = false;
        break;
      }
      waited = i + 1;
      const uint64_t ts = ts0 + i * S;
      const uint64_t te = min64(ts + S, e1);
      const uint64_t ce = min64((te + 3) & ~3ull, mfloor);
      const uint64_t cstart = max64(ts, e0);
#pragma unroll 1
      for (uint64_t c = cstart; c < te; c += 32) {
        uint64_t e = c + lane;
        bool act = e < te;
        uint32_t v = kEmptyKey;
        float wv = 0.f;
        if (act) {
          if (e < ce) {
            v = sbuf[b * S + (uint32_t)(e - ts)];
            if (VALS) wv = __uint_as_float(svals[b * S + (uint32_t)(e - ts)]);
          } else {
            v = a.col_idx[e];
            if (VALS) wv = a.vals[e];
          }
        }
        step(e, act, v, wv);
      }
      __syncwarp();
      issue(i + 2);
    }
    if (!ok) {
      set_status(a.status, GT_ERR_TIMEOUT);
      for (uint64_t i = waited; i < min64(waited + 2, ntile); ++i) mbar_wait(&bars[i & 1u], (uint32_t)((i >> 1) & 1u));
    }
  }
  };  // process

  if (!a.steal) {
    process(p);
  } else {
    process(2 * p);  // phase 1: the head of the warp's own partition
    for (;;) {       // phase 2: tails, claimed one at a time by whichever warp is free
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(a.steal_next, 1u);
      t = __shfl_sync(kFull, t, 0);
      if (t >= a.P) break;
      process(2 * t + 1);
    }
  }
  if (a.ptime) {
    __syncwarp();
    if (lane == 0) a.ptime[2 * (size_t)p + 1] = global_ns();
  }
}

// Unsorted weighted output: the packed entries (value bits << 32 | source)
// the scatter left at their final slots, streamed to row_idx and vals_out.
__global__ void k_unpack(const unsigned long long *__restrict__ packed, uint64_t m, uint32_t *row_idx,
                         float *vals_out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const unsigned long long e = __ldcs(packed + i);
    __stcs(row_idx + i, (uint32_t)e);
    __stcs(vals_out + i, __uint_as_float((uint32_t)(e >> 32)));
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <bool HDV, bool AGG, bool ST>
static cudaError_t set_count_attr() {
  return allow_max_dynamic_smem(k_count<HDV, AGG, ST>);
}
template <bool HDV, bool V, bool ST>
static cudaError_t set_scatter_attr() {
  return allow_max_dynamic_smem(k_scatter<HDV, V, ST>);
}

cudaError_t configure_steps() {
  cudaError_t e = cudaSuccess;
#define GT_TRY(x)                  \
  do {                             \
    cudaError_t r_ = (x);          \
    if (r_ != cudaSuccess) e = r_; \
  } while (0)
  GT_TRY((set_count_attr<true, true, false>()));
  GT_TRY((set_count_attr<true, false, false>()));
  GT_TRY((set_count_attr<false, true, false>()));
  GT_TRY((set_count_attr<false, false, false>()));
  GT_TRY((set_count_attr<true, true, true>()));
  GT_TRY((set_count_attr<true, false, true>()));
  GT_TRY((set_count_attr<false, true, true>()));
  GT_TRY((set_count_attr<false, false, true>()));
  GT_TRY((set_scatter_attr<true, true, false>()));
  GT_TRY((set_scatter_attr<true, false, false>()));
  GT_TRY((set_scatter_attr<false, true, false>()));
  GT_TRY((set_scatter_attr<false, false, false>()));
  GT_TRY((set_scatter_attr<true, true, true>()));
  GT_TRY((set_scatter_attr<true, false, true>()));
  GT_TRY((set_scatter_attr<false, true, true>()));
  GT_TRY((set_scatter_attr<false, false, true>()));
  GT_TRY(allow_max_dynamic_smem(k_finalize));
#undef GT_TRY
  return e;
}

cudaError_t launch_sort(const DevWork &w, const gt_config &cfg, const Problem &pb, cudaStream_t s);

cudaError_t run_transpose(const DevWork &w, const gt_config &cfg, const Problem &pb, cudaStream_t s,
                          StepEvents *ev, uint32_t *launches) {
  cudaError_t err;
  uint32_t nl = 0;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev->ev[i], s);
  };
  mark(0);
  const bool hdv = w.kmax > 0;
  const bool agg = (cfg.flags & GT_FLAG_AGGREGATE) != 0 || w.has_vals;  // weighted graphs need ordered ranks
  // per-call resets
  if ((err = cudaMemsetAsync(w.status, 0, sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(w.meta, 0, kMetaCount * sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(w.meta64, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess) return err;
  if (w.method == GT_METHOD_RADIX) {
    // timing slots: count = row expansion, digit passes and col_ptr; the rest are 0
    mark(1);
    nl = 0;
    if ((err = cudaMemsetAsync(w.r_nlong, 0, 4, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(w.r_gaps, 0, 8, s)) != cudaSuccess) return err;
    if (w.m == 0 && (err = cudaMemsetAsync(pb.col_ptr, 0, ((size_t)w.n + 1) * 8, s)) != cudaSuccess) return err;
    if ((err = run_radix(w, pb, s, &nl, ev)) != cudaSuccess) return err;
    mark(2);
    mark(3);
    mark(4);
    mark(5);
    if (launches) *launches = nl;
    return cudaGetLastError();
  }

  if ((err = cudaMemsetAsync(w.deg, 0, (size_t)w.n * sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(w.scan_state, 0, (size_t)w.ntiles * sizeof(unsigned long long), s)) != cudaSuccess)
    return err;

  // Partitioned form: bucket the edges by destination range first; the steps
  // below then read the bucketed (destination, source, value) list.
  const uint32_t *e_dst = pb.col_idx;
  const float *e_val = pb.vals;
  const uint32_t *e_src = nullptr;
  if (w.part_bits) {
    if (ev) {
      cudaEventRecord(ev->part[0], s);
      ev->has_part = 1;
    }
    if ((err = cudaMemsetAsync(w.r_nlong, 0, 4, s)) != cudaSuccess) return err;
    if ((err = run_partition(w, pb, s, &nl)) != cudaSuccess) return err;
    if (ev) {
      cudaEventRecord(ev->part[1], s);
      cudaEventRecord(ev->ev[0], s);  // Step 0 starts here: sample_ms leaves the bucketing out
    }
    e_dst = w.q_key;
    e_val = (const float *)w.q_w;
    e_src = w.q_u;
  }

  // Step 0
  if (hdv) {
    const uint32_t ts = 1u << w.ts_log2;
    if ((err = cudaMemsetAsync(w.skeys, 0xFF, (size_t)ts * 4, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(w.scnt, 0, (size_t)ts * 4, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(w.fhist, 0, (size_t)kFreqBins * 4, s)) != cudaSuccess) return err;
    if (w.ns > 0) {
      uint32_t g = (w.ns + 255) / 256;
      if (g > 4096) g = 4096;
      k_sample<<<g, 256, 0, s>>>(e_dst, w.n, w.m, w.ns, cfg.seed, w.skeys, w.scnt, w.ts_log2);
    }
    uint32_t g2 = (ts + 255) / 256;
    if (g2 > 4096) g2 = 4096;
    k_freq_hist<<<g2, 256, 0, s>>>(w.skeys, w.scnt, ts, w.fhist);
    k_select<<<1, 1024, 0, s>>>(w.fhist, w.kmax, 2u, w.meta);
    k_collect<<<g2, 256, 0, s>>>(w.skeys, w.scnt, ts, w.meta, w.cand, w.kmax, w.ties);
    size_t fsm = (size_t)(kTieCap + kMaxHdv) * 4 + (size_t)(1u << w.tlog2) * 6 + 16;
    k_finalize<<<1, 1024, fsm, s>>>(w.meta, w.cand, w.ties, w.kmax, w.hdv_ids, w.hkeys, w.hvals, w.tlog2);
    nl += (w.ns > 0) + 4;
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  mark(1);

  // partitions
  // unsorted output (GT_FLAG_UNSORTED): no LDV sort, no split-row tags
  const bool unsorted = (cfg.flags & GT_FLAG_UNSORTED) != 0;
  const int flag_mode = unsorted ? 0 : w.flag_mode;
  const int allow_split = unsorted || w.flag_mode || !w.has_vals;
  if (w.part_bits)
    k_partition_even<<<(w.P + 1 + 255) / 256, 256, 0, s>>>(w.P, w.m, w.psize, w.part);
  else
    k_partition<<<(w.P + 1 + 255) / 256, 256, 0, s>>>(pb.row_ptr, w.n_rows, w.m, w.P, w.psize, allow_split, w.part,
                                                      w.status);
  nl += 2;  // partition + count
  // two-phase Step 3: every partition split into a head and a tail, counted apart
  const unsigned long long *ranges = w.part;
  if (w.steal) {
    k_split_tails<<<(w.P + 1 + 255) / 256, 256, 0, s>>>(pb.row_ptr, w.n_rows, w.part, w.P, allow_split, w.part2);
    ranges = w.part2;
    ++nl;
  }

  // Step 1
  CountArgs ca{e_dst, w.n, w.m, ranges, w.hkeys, w.hvals, w.tlog2, w.kmax, w.meta, w.deg, w.hdv_cnt,
               w.meta64, w.status, w.stage_edges, (((uintptr_t)e_dst) & 15u) == 0, w.steal};
  const uint32_t threads = w.W * 32;
  if (hdv) {
    if (w.staged) {
      if (agg) k_count<true, true, true><<<w.G, threads, w.smem_count, s>>>(ca);
      else k_count<true, false, true><<<w.G, threads, w.smem_count, s>>>(ca);
    } else {
      if (agg) k_count<true, true, false><<<w.G, threads, w.smem_count, s>>>(ca);
      else k_count<true, false, false><<<w.G, threads, w.smem_count, s>>>(ca);
    }
  } else {
    if (w.staged) {
      if (agg) k_count<false, true, true><<<w.G, threads, w.smem_count, s>>>(ca);
      else k_count<false, false, true><<<w.G, threads, w.smem_count, s>>>(ca);
    } else {
      if (agg) k_count<false, true, false><<<w.G, threads, w.smem_count, s>>>(ca);
      else k_count<false, false, false><<<w.G, threads, w.smem_count, s>>>(ca);
    }
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  mark(2);

  // Step 2
  if (hdv) {
    dim3 b(32, 32);
    const uint32_t nranges = w.steal ? 2 * w.P : w.P;
    if (w.hdv_q > 1) {  // many partitions: slice totals, their scan, then the slices
      dim3 g((w.kmax + 31) / 32, w.hdv_q);
      k_hdv_slicesum<<<g, b, 0, s>>>(w.hdv_cnt, nranges, w.hdv_q, w.kmax, w.meta, w.hdv_psum);
      k_hdv_slicescan<<<(w.kmax + 255) / 256, 256, 0, s>>>(w.hdv_psum, w.hdv_q, w.kmax, w.meta, w.hdv_ids, w.deg,
                                                          w.status);
      k_hdv_sliceapply<<<g, b, 0, s>>>(w.hdv_cnt, nranges, w.hdv_q, w.kmax, w.meta, w.hdv_psum);
      nl += 2;
    } else {
      k_hdv_colscan<<<(w.kmax + 31) / 32, b, 0, s>>>(w.hdv_cnt, nranges, w.kmax, w.meta, w.hdv_ids, w.deg, w.status);
    }
  }
  k_scan<<<w.ntiles, kScanThreads, 0, s>>>(w.deg, w.n, w.n_rows, w.m, pb.row_ptr, pb.col_ptr, w.cursor,
                                           w.scan_state, w.meta, w.status);
  if (hdv) k_hdv_start<<<(w.kmax + 255) / 256, 256, 0, s>>>(w.meta, w.hdv_ids, pb.col_ptr, w.hdv_start);
  nl += hdv ? 3 : 1;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  mark(3);

  // Step 3
  if (w.ptime && (err = cudaMemsetAsync(w.ptime, 0, (size_t)w.P * 16, s)) != cudaSuccess) return err;
  if (w.steal && (err = cudaMemsetAsync(w.steal_next, 0, 4, s)) != cudaSuccess) return err;
  ScatterArgs sa{pb.row_ptr, e_dst, e_val,  w.n, w.n_rows, w.m,       ranges,   w.hkeys,
                 w.hvals,    w.tlog2,    w.kmax,   w.meta,      w.hdv_cnt, w.hdv_start, w.cursor,
                 pb.col_ptr, pb.row_idx, pb.vals_out,
                 (unsorted && !pb.vals) ? nullptr : (unsigned long long *)w.scratch,
                 w.status, flag_mode, w.stage_edges, w.ptime, w.steal, w.P, w.steal_next, e_src,
                 (unsorted && pb.vals) ? 1 : 0};
  const bool vals = pb.vals != nullptr;
#define GT_SC(H, V, ST) k_scatter<H, V, ST><<<w.G, threads, w.smem_scatter, s>>>(sa)
  if (hdv) {
    if (vals) {
      if (w.staged) GT_SC(true, true, true);
      else GT_SC(true, true, false);
    } else {
      if (w.staged) GT_SC(true, false, true);
      else GT_SC(true, false, false);
    }
  } else {
    if (vals) {
      if (w.staged) GT_SC(false, true, true);
      else GT_SC(false, true, false);
    } else {
      if (w.staged) GT_SC(false, false, true);
      else GT_SC(false, false, false);
    }
  }
#undef GT_SC
  nl += 1;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  mark(4);

  // LDV sort (it re-reads row_ptr, col_idx and vals for split rows); unsorted
  // weighted output: the packed entries to the outputs
  if (!unsorted) {
    err = launch_sort(w, cfg, pb, s);
    nl += 4;
  } else if (pb.vals && w.m) {
    const uint32_t gu = (uint32_t)min64((w.m + 255) / 256, (uint64_t)w.num_sms * 16);
    k_unpack<<<gu, 256, 0, s>>>((const unsigned long long *)w.scratch, w.m, pb.row_idx, pb.vals_out);
    err = cudaGetLastError();
    nl += 1;
  }
  if (err == cudaSuccess && pb.inputs_read) err = cudaEventRecord(pb.inputs_read, s);
  mark(5);
  if (launches) *launches = nl;
  return err;
}

}  // namespace gt
