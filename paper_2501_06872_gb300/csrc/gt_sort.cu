// LDV list sort (the optional neighbour sort of Sec. II-B, made mandatory):
// every LDV list of the CSC is ordered by source.  HDV lists are skipped:
// their slots were assigned in edge order, which is already source order.
//
// Ties (parallel edges u->v) keep CSR order.  LDV slots of one warp were
// assigned in edge order, so a sort that is stable with respect to the
// current slot order is enough, except for rows shared by two partitions
// ("split rows"), whose entries carry a tag (bit 31 of row_idx) and their
// position inside the row (in the value slot); those are ordered by that
// position and their values are re-read from the input.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {

struct SortArgs {
  uint32_t n;
  const uint64_t *col_ptr;
  const uint64_t *row_ptr;
  const float *vals;  // input values (for tagged entries)
  uint32_t *row_idx;
  float *vals_out;
  const uint32_t *hkeys;
  const uint16_t *hvals;
  uint32_t tlog2, kmax;
  uint32_t *meta;
  uint32_t *biglist;
  uint32_t big_cap;
  uint32_t *status;
  int flag_mode;
  uint32_t *scr_u;
  float *scr_w;
  uint32_t key_bits;  // bits of a vertex ID (ceil(log2 n))
};

// ---------------------------------------------------------------------------
// Element encoding for the comparison sorts.
//   weighted:   key = (u << 32) | (tagged ? pos_in_row : index_in_list), payload = value bits or pos
//   unweighted: key = u  (equal keys are indistinguishable)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finish_entry(const SortArgs &a, uint64_t key, uint32_t pay, uint32_t tag,
                                             uint64_t slot) {
  uint32_t u = (uint32_t)(key >> 32);
  a.row_idx[slot] = u;
  uint32_t wb = pay;
  if (tag) wb = __float_as_uint(a.vals[a.row_ptr[u] + pay]);
  a.vals_out[slot] = __uint_as_float(wb);
}

// Warp bitonic sort of 32 (key, pay, tag) triples held one per lane, ascending.
__device__ __forceinline__ void warp_bitonic(uint64_t &key, uint32_t &pay, uint32_t &tag, uint32_t lane) {
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      uint64_t ok = __shfl_xor_sync(kFull, key, j);
      uint32_t op = __shfl_xor_sync(kFull, pay, j);
      uint32_t ot = __shfl_xor_sync(kFull, tag, j);
      bool up = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      bool take = (lower == up) ? (ok < key) : (ok > key);
      if (take) {
        key = ok;
        pay = op;
        tag = ot;
      }
    }
  }
}

__device__ __forceinline__ void warp_bitonic_u32(uint32_t &key, uint32_t lane) {
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      uint32_t ok = __shfl_xor_sync(kFull, key, j);
      bool up = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      if ((lower == up) ? (ok < key) : (ok > key)) key = ok;
    }
  }
}

// Small lists: one warp per group of 32 consecutive destinations.  Lists of
// length 2..32 are sorted in registers; longer LDV lists go to the big list.
template <bool VALS>
__global__ void __launch_bounds__(256) k_sort_small(SortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (cta_status_set(a.status)) return;
  uint32_t *keys = (uint32_t *)smem;
  uint16_t *hv = (uint16_t *)(keys + (a.kmax ? (1u << a.tlog2) : 0u));
  const uint32_t K = a.kmax ? a.meta[kMetaK] : 0u;
  if (K) {
    const uint32_t T = 1u << a.tlog2;
    for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) {
      keys[i] = a.hkeys[i];
      hv[i] = a.hvals[i];
    }
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps_total = gridDim.x * (blockDim.x >> 5);
  const uint32_t ngroups = (a.n + 31) / 32;
  uint32_t sorted_local = 0;
  for (uint32_t g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < ngroups; g += warps_total) {
    const uint32_t v = g * 32 + lane;
    uint64_t c0 = 0, c1 = 0;
    bool need = false;
    if (v < a.n) {
      c0 = a.col_ptr[v];
      c1 = a.col_ptr[v + 1];
      need = c1 - c0 >= 2;
      if (need && K && hdv_lookup(keys, hv, a.tlog2, v) >= 0) need = false;
    }
    const uint64_t len = c1 - c0;
    const bool big = need && len > kWarpSortCap;
    if (big) {
      uint32_t i = atomicAdd(&a.meta[kMetaBig], 1u);
      if (i < a.big_cap) a.biglist[i] = v;
      else set_status(a.status, GT_ERR_UNSUPPORTED);
    }
    uint32_t todo = __ballot_sync(kFull, need && !big);
    sorted_local += __popc(__ballot_sync(kFull, need));
    while (todo) {
      const uint32_t j = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint64_t s0 = __shfl_sync(kFull, c0, j);
      const uint32_t L = (uint32_t)__shfl_sync(kFull, len, j);
      const bool act = lane < L;
      if (VALS) {
        uint64_t key = ~0ull;
        uint32_t pay = 0, tag = 0;
        if (act) {
          uint32_t u = a.row_idx[s0 + lane];
          pay = __float_as_uint(a.vals_out[s0 + lane]);
          tag = (a.flag_mode && (u & kSplitFlag)) ? 1u : 0u;
          if (tag) u &= ~kSplitFlag;
          key = ((uint64_t)u << 32) | (tag ? pay : lane);
        }
        warp_bitonic(key, pay, tag, lane);
        if (act) finish_entry(a, key, pay, tag, s0 + lane);
      } else {
        uint32_t key = act ? a.row_idx[s0 + lane] : 0xFFFFFFFFu;
        warp_bitonic_u32(key, lane);
        if (act) a.row_idx[s0 + lane] = key;
      }
    }
  }
  // every lane holds the same warp-wide count
  if (lane == 0 && sorted_local) atomicAdd(&a.meta[kMetaSorted], sorted_local);
}

// ---------------------------------------------------------------------------
// Big lists: one CTA per list.  Up to kSortSmemCap entries are sorted in
// shared memory (bitonic on the composite key); longer lists use a stable
// LSD radix sort on the source ID through the plan's scratch arrays.
// ---------------------------------------------------------------------------
constexpr int kBigThreads = 1024;

template <bool VALS>
__device__ void smem_sort_list(const SortArgs &a, uint64_t s0, uint32_t L, unsigned char *smem) {
  uint32_t cap = 1;
  while (cap < L) cap <<= 1;
  if (VALS) {
    uint64_t *k = (uint64_t *)smem;
    uint32_t *p = (uint32_t *)(k + kSortSmemCap);
    uint8_t *t = (uint8_t *)(p + kSortSmemCap);
    for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
      uint64_t key = ~0ull;
      uint32_t pay = 0, tag = 0;
      if (i < L) {
        uint32_t u = a.row_idx[s0 + i];
        pay = __float_as_uint(a.vals_out[s0 + i]);
        tag = (a.flag_mode && (u & kSplitFlag)) ? 1u : 0u;
        if (tag) u &= ~kSplitFlag;
        key = ((uint64_t)u << 32) | (tag ? pay : i);
      }
      k[i] = key;
      p[i] = pay;
      t[i] = (uint8_t)tag;
    }
    __syncthreads();
    for (uint32_t kk = 2; kk <= cap; kk <<= 1) {
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
          uint32_t q = i ^ j;
          if (q > i) {
            bool up = (i & kk) == 0;
            uint64_t x = k[i], y = k[q];
            if ((x > y) == up) {
              k[i] = y;
              k[q] = x;
              uint32_t tp = p[i];
              p[i] = p[q];
              p[q] = tp;
              uint8_t tt = t[i];
              t[i] = t[q];
              t[q] = tt;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) finish_entry(a, k[i], p[i], t[i], s0 + i);
  } else {
    uint32_t *k = (uint32_t *)smem;
    for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) k[i] = (i < L) ? a.row_idx[s0 + i] : 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t kk = 2; kk <= cap; kk <<= 1) {
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
          uint32_t q = i ^ j;
          if (q > i) {
            bool up = (i & kk) == 0;
            uint32_t x = k[i], y = k[q];
            if ((x > y) == up) {
              k[i] = y;
              k[q] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) a.row_idx[s0 + i] = k[i];
  }
  __syncthreads();
}

// One stable counting pass on digit (key >> shift) & (2^dbits - 1) of the
// (tag-masked) source ID, src -> dst, by the whole CTA in input order.
template <bool VALS>
__device__ void radix_pass(const uint32_t *su, const float *sw, uint32_t *du, float *dw, uint32_t L, uint32_t shift,
                           uint32_t dbits, uint32_t kmask, unsigned char *smem) {
  const uint32_t nb = 1u << dbits;
  uint32_t *base = (uint32_t *)smem;   // [nb]
  uint32_t *wc = base + 256;            // [nb][32]
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) base[i] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) atomicAdd(&base[((su[i] & kmask) >> shift) & (nb - 1)], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t d = 0; d < nb; ++d) {
      uint32_t c = base[d];
      base[d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (uint32_t c = 0; c < L; c += blockDim.x) {
    const uint32_t i = c + threadIdx.x;
    const bool act = i < L;
    uint32_t u = act ? su[i] : 0u;
    float wv = (VALS && act) ? sw[i] : 0.f;
    uint32_t d = act ? (((u & kmask) >> shift) & (nb - 1)) : nb;
    for (uint32_t dd = lane; dd < nb; dd += 32) wc[dd * 32 + w] = 0;
    __syncthreads();
    uint32_t mm = __match_any_sync(kFull, d);
    uint32_t rank = __popc(mm & lanemask_lt());
    if (act && rank == 0) wc[d * 32 + w] = __popc(mm);
    __syncthreads();
    // exclusive scan over warps for every digit: warp w handles digits w, w+32, ...
    for (uint32_t dd = w; dd < nb; dd += 32) {
      uint32_t x = wc[dd * 32 + lane];
      uint32_t inc = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += y;
      }
      const uint32_t b0 = base[dd];
      wc[dd * 32 + lane] = b0 + inc - x;
      __syncwarp();
      if (lane == 31) base[dd] = b0 + inc;
    }
    __syncthreads();
    if (act) {
      uint32_t pos = wc[d * 32 + w] + rank;
      du[pos] = u;
      if (VALS) dw[pos] = wv;
    }
    __syncthreads();
  }
}

template <bool VALS>
__device__ void radix_sort_list(const SortArgs &a, uint64_t s0, uint32_t L, unsigned char *smem) {
  const uint32_t bits = a.key_bits;
  const uint32_t passes = bits <= 16 ? 2u : 4u;
  const uint32_t dbits = (bits + passes - 1) / passes;
  const uint32_t kmask = a.flag_mode ? ~kSplitFlag : 0xFFFFFFFFu;
  uint32_t *ou = a.row_idx + s0;
  float *ow = VALS ? a.vals_out + s0 : nullptr;
  uint32_t *xu = a.scr_u + s0;
  float *xw = VALS ? a.scr_w + s0 : nullptr;
  for (uint32_t ps = 0; ps < passes; ++ps) {
    const uint32_t shift = ps * dbits;
    if ((ps & 1u) == 0) radix_pass<VALS>(ou, ow, xu, xw, L, shift, dbits, kmask, smem);
    else radix_pass<VALS>(xu, xw, ou, ow, L, shift, dbits, kmask, smem);
  }
  if (VALS && a.flag_mode) {
    // tagged runs: order by position in row, then re-read the values
    for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) {
      uint32_t u = ou[i];
      if (!(u & kSplitFlag)) continue;
      if (i > 0 && ou[i - 1] == u) continue;  // not the first of its run
      uint32_t j = i + 1;
      while (j < L && ou[j] == u) ++j;
      // insertion sort of positions in [i, j)
      for (uint32_t x = i + 1; x < j; ++x) {
        uint32_t t = __float_as_uint(ow[x]);
        uint32_t y = x;
        while (y > i && __float_as_uint(ow[y - 1]) > t) {
          ow[y] = ow[y - 1];
          --y;
        }
        ow[y] = __uint_as_float(t);
      }
      const uint32_t uu = u & ~kSplitFlag;
      const uint64_t rs = a.row_ptr[uu];
      for (uint32_t x = i; x < j; ++x) ow[x] = a.vals[rs + __float_as_uint(ow[x])];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) ou[i] &= ~kSplitFlag;
  }
  __syncthreads();
}

template <bool VALS>
__global__ void __launch_bounds__(kBigThreads) k_sort_big(SortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (cta_status_set(a.status)) return;
  __shared__ uint32_t s_item;
  const uint32_t nbig = min(a.meta[kMetaBig], a.big_cap);
  uint32_t large_local = 0;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(&a.meta[kMetaTicket], 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= nbig) break;
    const uint32_t v = a.biglist[it];
    const uint64_t s0 = a.col_ptr[v];
    const uint32_t L = (uint32_t)(a.col_ptr[v + 1] - s0);
    if (L <= kSortSmemCap) {
      smem_sort_list<VALS>(a, s0, L, smem);
    } else {
      radix_sort_list<VALS>(a, s0, L, smem);
      ++large_local;
    }
  }
  if (threadIdx.x == 0 && large_local) atomicAdd(&a.meta[kMetaLarge], large_local);
}

static size_t big_smem_bytes() {
  size_t bitonic = (size_t)kSortSmemCap * (8 + 4 + 1);
  size_t radix = (256 + 256 * 32) * 4;
  return bitonic > radix ? bitonic : radix;
}

cudaError_t configure_sort() {
  cudaError_t e[4] = {allow_max_dynamic_smem(k_sort_big<true>), allow_max_dynamic_smem(k_sort_big<false>),
                      allow_max_dynamic_smem(k_sort_small<true>), allow_max_dynamic_smem(k_sort_small<false>)};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

cudaError_t launch_sort(const DevWork &w, const gt_config &cfg, const Problem &pb, cudaStream_t s) {
  (void)cfg;
  uint32_t bits = 0;
  while (bits < 32 && (w.n - 1) >> bits) ++bits;
  SortArgs sa{w.n,     pb.col_ptr, pb.row_ptr, pb.vals,      pb.row_idx, pb.vals_out, w.hkeys, w.hvals, w.tlog2,
              w.kmax,  w.meta,     w.biglist,  w.big_cap,    w.status,   w.flag_mode, w.scr_u, w.scr_w, bits};
  const bool vals = pb.vals != nullptr;
  const size_t ssm = w.kmax ? (size_t)(1u << w.tlog2) * 6 + 16 : 0;
  const uint32_t groups = (w.n + 31) / 32;
  uint32_t g = (groups + 7) / 8;
  const uint32_t gmax = (uint32_t)w.num_sms * 8u;
  if (g > gmax) g = gmax;
  if (g == 0) g = 1;
  if (vals) k_sort_small<true><<<g, 256, ssm, s>>>(sa);
  else k_sort_small<false><<<g, 256, ssm, s>>>(sa);
  const uint32_t gb = (uint32_t)w.num_sms * 2u;
  if (vals) k_sort_big<true><<<gb, kBigThreads, big_smem_bytes(), s>>>(sa);
  else k_sort_big<false><<<gb, kBigThreads, big_smem_bytes(), s>>>(sa);
  return cudaGetLastError();
}

}  // namespace gt
