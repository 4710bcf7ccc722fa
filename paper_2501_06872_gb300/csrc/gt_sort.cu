// LDV list sort (the optional neighbour sort of Sec. II-B, made mandatory):
// every LDV list of the CSC is ordered by source.  HDV lists are skipped:
// their slots were assigned in edge order, which is already source order.
//
// Ties (parallel edges u->v) keep CSR order.  The LDV slots one warp takes in
// a list increase along its edges, so a sort that is stable with respect to
// the slot order is enough -- except for rows shared by two partitions
// ("split rows"), whose entries carry a tag (bit 31 of the source) and their
// position inside the row in place of the value; those are ordered by that
// position and their values are re-read from the input.
//
// Data flow.  Weighted graphs: the scatter left every LDV entry in the packed
// scratch array (u64: value bits << 32 | source); this pass sorts each list
// and writes row_idx / vals_out.  Unweighted graphs: the scatter wrote
// row_idx directly and lists are sorted in place.
//
// List classes (by length L): 1 copy; 2..32 one warp, registers; 33..256
// one warp, its own shared-memory slice; 257..2048 one CTA, shared memory
// (all bitonic on a unique key); > 2048 stable LSD radix through scratch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {

struct SortArgs {
  uint32_t n;  // columns: the lists to sort
  const uint64_t *col_ptr;
  const uint64_t *row_ptr;
  const float *vals;  // input values (tagged entries re-read theirs)
  uint32_t *row_idx;
  float *vals_out;
  unsigned long long *ldv64;  // weighted: packed LDV entries [m]
  uint32_t *scr32;            // unweighted: radix second buffer [m]
  const uint32_t *hkeys;
  const uint16_t *hvals;
  uint32_t tlog2, kmax;
  uint32_t *meta;
  uint32_t *midlist, *biglist, *largelist;
  uint32_t mid_cap, big_cap, large_cap;
  uint32_t *status;
  int flag_mode;
  uint32_t key_bits;  // bits of a row ID, the sort key (ceil(log2 n_rows))
  // partitioned form: tagged entries carry their position in the bucketed
  // edge list, whose values are qvals (null: a position inside the CSR row)
  const float *qvals = nullptr;
};

struct WarpSync {
  __device__ void operator()() const { __syncwarp(); }
};
struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};

__device__ __forceinline__ uint32_t umask_of(const SortArgs &a) { return a.flag_mode ? ~kSplitFlag : 0xFFFFFFFFu; }

// Value bits of a tagged entry of source u whose value slot holds pos.
__device__ __forceinline__ uint32_t tagged_value(const SortArgs &a, uint32_t u, uint32_t pos) {
  return __float_as_uint(a.qvals ? a.qvals[pos] : a.vals[a.row_ptr[u] + pos]);
}

// Writes one finished weighted entry (packed) to the outputs.
__device__ __forceinline__ void emit_packed(const SortArgs &a, uint64_t slot, unsigned long long ent) {
  uint32_t u = (uint32_t)ent;
  uint32_t wb = (uint32_t)(ent >> 32);
  if (a.flag_mode && (u & kSplitFlag)) {
    u &= ~kSplitFlag;
    wb = tagged_value(a, u, wb);
  }
  a.row_idx[slot] = u;
  a.vals_out[slot] = __uint_as_float(wb);
}

// Unique ordering key of a weighted entry at list index i.
__device__ __forceinline__ unsigned long long packed_key(const SortArgs &a, unsigned long long ent, uint32_t i) {
  const uint32_t u = (uint32_t)ent;
  const bool tag = a.flag_mode && (u & kSplitFlag);
  return ((unsigned long long)(u & umask_of(a)) << 32) | (tag ? (uint32_t)(ent >> 32) : i);
}

// Sort key of an untagged weighted entry at list index i (< 2048): the
// source above the index.  Sorting these keys alone leaves the entries in
// place, to be picked up by index: half the shared-memory traffic of
// moving (key, entry) pairs.
constexpr uint32_t kIndexBits = 11;
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
__device__ __forceinline__ unsigned long long index_key(const SortArgs &a, unsigned long long ent, uint32_t i) {
  return ((unsigned long long)((uint32_t)ent & umask_of(a)) << kIndexBits) | i;
}

// Bitonic sort of S (a power of two, <= 32) keys in each aligned group of S
// lanes: the groups sort independently (every exchange distance is < S), and
// the last merge runs ascending in every group.
template <uint32_t S, bool PAY, typename K, typename P>
__device__ __forceinline__ void warp_bitonic_groups(K &key, P &pay, uint32_t lane) {
#pragma unroll
  for (uint32_t k = 2; k <= S; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const K ok = __shfl_xor_sync(kFull, key, j);
      P op = pay;
      if (PAY) op = __shfl_xor_sync(kFull, pay, j);
      const bool keep_min = ((lane & j) == 0) == ((k == S) || (lane & k) == 0);
      const bool take = (ok < key) == keep_min;  // keys are distinct (padding aside)
      key = take ? ok : key;
      if (PAY) pay = take ? op : pay;
    }
  }
}

// Sorts the lists of this warp's 32 destinations whose length L satisfies
// lo < L <= S (2 <= L), 32 / S lists per step, one group of S lanes each.
// todo: the lanes (destinations) whose list qualifies.
template <bool VALS, uint32_t S>
__device__ __forceinline__ void sort_short_lists(const SortArgs &a, uint32_t todo, uint64_t c0, uint64_t len,
                                                 uint32_t lane) {
  constexpr uint32_t G = 32 / S;
  const uint32_t grp = lane / S, e = lane % S;
  while (todo) {
    uint32_t myj = 32;  // the destination lane whose list this group sorts (32: none)
#pragma unroll
    for (uint32_t q = 0; q < G; ++q) {
      if (todo) {
        const uint32_t j = __ffs(todo) - 1;
        todo &= todo - 1;
        if (grp == q) myj = j;
      }
    }
    const uint64_t s0 = __shfl_sync(kFull, c0, myj & 31u);
    uint32_t L = (uint32_t)__shfl_sync(kFull, len, myj & 31u);
    if (myj == 32) L = 0;
    const bool act = e < L;
    if (VALS) {
      unsigned long long ent = act ? a.ldv64[s0 + e] : 0ull;
      const bool tagged = act && a.flag_mode && ((uint32_t)ent & kSplitFlag);
      if (!__any_sync(kFull, tagged)) {
        // sort (source, index) keys; each lane then fetches its entry from
        // the lane that loaded it
        unsigned long long key = act ? index_key(a, ent, e) : ~0ull;
        uint32_t dummy = 0;
        warp_bitonic_groups<S, false>(key, dummy, lane);
        const unsigned long long got = __shfl_sync(kFull, ent, grp * S + ((uint32_t)key & (S - 1u)));
        if (act) emit_packed(a, s0 + e, got);
      } else {
        unsigned long long key = act ? packed_key(a, ent, e) : ~0ull;
        warp_bitonic_groups<S, true>(key, ent, lane);
        if (act) emit_packed(a, s0 + e, ent);
      }
    } else {
      uint32_t key = act ? a.row_idx[s0 + e] : 0xFFFFFFFFu;
      uint32_t dummy = 0;
      warp_bitonic_groups<S, false>(key, dummy, lane);
      if (act) a.row_idx[s0 + e] = key;
    }
  }
}

// ---------------------------------------------------------------------------
// Lists of length <= 32 (and length-1 copies); longer lists go to worklists.
// One warp per group of 32 consecutive destinations.
// ---------------------------------------------------------------------------
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
    bool ldv = false;
    if (v < a.n) {
      c0 = a.col_ptr[v];
      c1 = a.col_ptr[v + 1];
      ldv = c1 > c0 && !(K && hdv_lookup(keys, hv, a.tlog2, v) >= 0);
    }
    const uint64_t len = c1 - c0;
    if (VALS && ldv && len == 1) emit_packed(a, c0, a.ldv64[c0]);
    const bool need = ldv && len >= 2;
    if (need && len > kWarpSortCap) {
      if (len <= kMidCap) {
        uint32_t i = atomicAdd(&a.meta[kMetaMid], 1u);
        if (i < a.mid_cap) a.midlist[i] = v;
        else set_status(a.status, GT_ERR_UNSUPPORTED);
      } else if (len <= kSortSmemCap) {
        uint32_t i = atomicAdd(&a.meta[kMetaBig], 1u);
        if (i < a.big_cap) a.biglist[i] = v;
        else set_status(a.status, GT_ERR_UNSUPPORTED);
      } else {
        uint32_t i = atomicAdd(&a.meta[kMetaLargeN], 1u);
        if (i < a.large_cap) a.largelist[i] = v;
        else set_status(a.status, GT_ERR_UNSUPPORTED);
      }
    }
    sorted_local += __popc(__ballot_sync(kFull, need));
    // short lists several to a warp: groups of 4, 8, 16 or 32 lanes
    sort_short_lists<VALS, 4>(a, __ballot_sync(kFull, need && len <= 4), c0, len, lane);
    sort_short_lists<VALS, 8>(a, __ballot_sync(kFull, need && len > 4 && len <= 8), c0, len, lane);
    sort_short_lists<VALS, 16>(a, __ballot_sync(kFull, need && len > 8 && len <= 16), c0, len, lane);
    sort_short_lists<VALS, 32>(a, __ballot_sync(kFull, need && len > 16 && len <= kWarpSortCap), c0, len, lane);
  }
  if (lane == 0 && sorted_local) atomicAdd(&a.meta[kMetaSorted], sorted_local);
}

// ---------------------------------------------------------------------------
// Bitonic network in shared memory over cap (power of two) elements.
// ---------------------------------------------------------------------------
template <typename K, bool PAY, typename Sync>
__device__ __forceinline__ void smem_bitonic(K *key, unsigned long long *pay, uint32_t cap, uint32_t tid,
                                             uint32_t nthreads, Sync sync) {
  for (uint32_t k = 2; k <= cap; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < cap / 2; i += nthreads) {
        // j is a power of two: the pair's lower index inserts a 0 bit at j
        const uint32_t lo = ((i & ~(j - 1u)) << 1) | (i & (j - 1u));
        const uint32_t hi = lo + j;
        const bool up = (lo & k) == 0;
        const K ka = key[lo], kb = key[hi];
        if ((ka > kb) == up) {
          key[lo] = kb;
          key[hi] = ka;
          if (PAY) {
            const unsigned long long t = pay[lo];
            pay[lo] = pay[hi];
            pay[hi] = t;
          }
        }
      }
      sync();
    }
  }
}


// Compare-exchange of two elements, a at the lower index.
template <typename K>
__device__ __forceinline__ void ce_pair(K &a, K &b, bool up) {
  const bool sw = (b < a) == up;  // keys are distinct (padding aside, where either order is right)
  const K t = a;
  a = sw ? b : a;
  b = sw ? t : b;
}

// The steps of bitonic merge k whose exchange distance stays inside one
// warp's chunk of 32R consecutive elements, held as x[r] = element
// ebase + 32r (ebase = chunk start + lane): distances >= 32 swap registers
// of the lane, shorter ones shuffle between lanes.
template <typename K, uint32_t R>
__device__ __forceinline__ void reg_merge(K (&x)[R], uint32_t k, uint32_t ebase, uint32_t lane) {
#pragma unroll
  for (uint32_t j = 16 * R; j >= 1; j >>= 1) {
    if (j >= k) continue;  // merge k has the steps k/2 ... 1
    if (j >= 32) {
#pragma unroll
      for (uint32_t r = 0; r < R; ++r)
        if ((r & (j >> 5)) == 0) ce_pair(x[r], x[r | (j >> 5)], ((ebase + 32 * r) & k) == 0);
    } else {
      const bool lower = (lane & j) == 0;
#pragma unroll
      for (uint32_t r = 0; r < R; ++r) {
        const K o = __shfl_xor_sync(kFull, x[r], j);
        const bool keep_min = lower == (((ebase + 32 * r) & k) == 0);
        x[r] = ((o < x[r]) == keep_min) ? o : x[r];
      }
    }
  }
}

// Bitonic sort of NW * 32R keys held by NW warps in registers (warp w holds
// elements w * 32R ...).  Merge steps with distances of a whole chunk or
// more (NW > 1 only) go through sk[] in shared memory, one barrier each; the
// rest stay in registers.  On return x[r] holds sorted element w * 32R +
// 32r + lane.
template <typename K, uint32_t NW, uint32_t R, typename Sync>
__device__ __forceinline__ void reg_bitonic(K (&x)[R], K *sk, uint32_t w, uint32_t lane, Sync sync) {
  constexpr uint32_t C = 32 * R, N = NW * C;
  const uint32_t ebase = w * C + lane;
#pragma unroll 1
  for (uint32_t k = 2; k <= N; k <<= 1) {
    if (NW > 1 && k > C) {
#pragma unroll
      for (uint32_t r = 0; r < R; ++r) sk[ebase + 32 * r] = x[r];
      sync();
      for (uint32_t j = k >> 1; j >= C; j >>= 1) {
        for (uint32_t i = w * 32 + lane; i < N / 2; i += NW * 32) {
          const uint32_t lo = ((i & ~(j - 1u)) << 1) | (i & (j - 1u)), hi = lo + j;
          const K ka = sk[lo], kb = sk[hi];
          if ((ka > kb) == ((lo & k) == 0)) {
            sk[lo] = kb;
            sk[hi] = ka;
          }
        }
        sync();
      }
#pragma unroll
      for (uint32_t r = 0; r < R; ++r) x[r] = sk[ebase + 32 * r];
    }
    reg_merge<K, R>(x, k, ebase, lane);
  }
}

// Sorts one list of L <= NW * 32R entries with the calling NW warps (warp w,
// lane) and writes it to the outputs.  Weighted lists without split-row
// tags sort (source, index) keys in registers and pick their entries from
// pay[] by index; lists with tags order (key, entry) pairs in shared memory
// (the tag's position breaks ties).  key / pay: NW * 32R u64 slots each.
template <bool VALS, uint32_t NW, uint32_t R, typename Sync, typename AnyTag>
__device__ __forceinline__ void reg_sort_list(const SortArgs &a, uint64_t s0, uint32_t L, unsigned long long *key,
                                              unsigned long long *pay, uint32_t w, uint32_t lane, Sync sync,
                                              AnyTag any_tag) {
  constexpr uint32_t C = 32 * R, N = NW * C;
  const uint32_t ebase = w * C + lane;
  if (!VALS) {
    uint32_t x[R];
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t e = ebase + 32 * r;
      x[r] = e < L ? a.row_idx[s0 + e] : 0xFFFFFFFFu;
    }
    reg_bitonic<uint32_t, NW, R>(x, (uint32_t *)key, w, lane, sync);
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t e = ebase + 32 * r;
      if (e < L) a.row_idx[s0 + e] = x[r];
    }
    sync();
    return;
  }
  unsigned long long x[R];
  bool tag = false;
#pragma unroll
  for (uint32_t r = 0; r < R; ++r) {
    const uint32_t e = ebase + 32 * r;
    x[r] = ~0ull;
    if (e < L) {
      const unsigned long long ent = a.ldv64[s0 + e];
      pay[e] = ent;
      tag |= a.flag_mode && ((uint32_t)ent & kSplitFlag);
      x[r] = index_key(a, ent, e);
    }
  }
  const bool any = any_tag(tag);
  sync();
  reg_bitonic<unsigned long long, NW, R>(x, key, w, lane, sync);
  if (!any) {
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t e = ebase + 32 * r;
      if (e < L) emit_packed(a, s0 + e, pay[(uint32_t)x[r] & kIndexMask]);
    }
    sync();
    return;
  }
  // Split rows: the entries of one tagged source are parallel edges whose
  // order is their position (value slot), not their slot index.  Each run of
  // them in the sorted keys is put in position order by the thread at its
  // start; a list with a run longer than 64 takes (key, entry) pairs through
  // a shared-memory network instead.
#pragma unroll
  for (uint32_t r = 0; r < R; ++r) key[ebase + 32 * r] = x[r];
  sync();
  const uint32_t t = w * 32 + lane;
  bool longrun = false;
  for (uint32_t e = t; e < L; e += NW * 32) {
    const uint64_t src_e = key[e] >> kIndexBits;
    const unsigned long long ent = pay[(uint32_t)key[e] & kIndexMask];
    if (!((uint32_t)ent & kSplitFlag) || (e > 0 && (key[e - 1] >> kIndexBits) == src_e)) continue;
    uint32_t f = e + 1;
    while (f < L && f - e <= 64 && (key[f] >> kIndexBits) == src_e) ++f;
    if (f - e > 64) {
      longrun = true;
      continue;
    }
    for (uint32_t q = e + 1; q < f; ++q) {  // insertion sort by position
      const unsigned long long kq = key[q];
      const uint32_t pq = (uint32_t)(pay[(uint32_t)kq & kIndexMask] >> 32);
      uint32_t z = q;
      while (z > e && (uint32_t)(pay[(uint32_t)key[z - 1] & kIndexMask] >> 32) > pq) {
        key[z] = key[z - 1];
        --z;
      }
      key[z] = kq;
    }
  }
  if (!any_tag(longrun)) {
    sync();
    for (uint32_t e = t; e < L; e += NW * 32) emit_packed(a, s0 + e, pay[(uint32_t)key[e] & kIndexMask]);
  } else {
    sync();
    for (uint32_t i = t; i < N; i += NW * 32) {
      key[i] = i < L ? packed_key(a, pay[i], i) : ~0ull;
      if (i >= L) pay[i] = 0ull;
    }
    sync();
    smem_bitonic<unsigned long long, true>(key, pay, N, t, NW * 32, sync);
    for (uint32_t i = t; i < L; i += NW * 32) emit_packed(a, s0 + i, pay[i]);
  }
  sync();
}

constexpr int kWarpThreads = 256;
constexpr int kRadixThreads = 1024;

// 33..kMidCap: one warp per list in its own shared-memory slice.
template <bool VALS>
__global__ void __launch_bounds__(kWarpThreads) k_sort_warp(SortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (cta_status_set(a.status)) return;
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const size_t per = VALS ? 16u : 4u;
  unsigned char *mine = smem + (size_t)w * kMidCap * per;
  unsigned long long *key = (unsigned long long *)mine;
  unsigned long long *pay = key + kMidCap;
  const uint32_t nmid = min(a.meta[kMetaMid], a.mid_cap);
  while (true) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(&a.meta[kMetaMidTicket], 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= nmid) break;
    const uint32_t v = a.midlist[it];
    const uint64_t s0 = a.col_ptr[v];
    const uint32_t L = (uint32_t)(a.col_ptr[v + 1] - s0);
    auto any = [](bool x) { return __any_sync(kFull, x) != 0; };
    if (L <= 64) reg_sort_list<VALS, 1, 2>(a, s0, L, key, pay, 0, lane, WarpSync{}, any);
    else if (L <= 128) reg_sort_list<VALS, 1, 4>(a, s0, L, key, pay, 0, lane, WarpSync{}, any);
    else reg_sort_list<VALS, 1, 8>(a, s0, L, key, pay, 0, lane, WarpSync{}, any);
  }
}

// kMidCap+1..kSortSmemCap: one CTA of 16 warps per list, the bitonic
// network in registers (2 or 4 keys per lane) with the cross-warp steps in
// shared memory.
constexpr int kCtaThreads = 512;

template <bool VALS>
__global__ void __launch_bounds__(kCtaThreads) k_sort_cta(SortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (cta_status_set(a.status)) return;
  __shared__ uint32_t s_item;
  unsigned long long *key = (unsigned long long *)smem;
  unsigned long long *pay = key + kSortSmemCap;
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t nbig = min(a.meta[kMetaBig], a.big_cap);
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(&a.meta[kMetaTicket], 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= nbig) break;
    const uint32_t v = a.biglist[it];
    const uint64_t s0 = a.col_ptr[v];
    const uint32_t L = (uint32_t)(a.col_ptr[v + 1] - s0);
    auto any = [](bool x) { return __syncthreads_or(x) != 0; };
    if (L <= 512) reg_sort_list<VALS, 16, 1>(a, s0, L, key, pay, w, lane, CtaSync{}, any);
    else if (L <= 1024) reg_sort_list<VALS, 16, 2>(a, s0, L, key, pay, w, lane, CtaSync{}, any);
    else reg_sort_list<VALS, 16, 4>(a, s0, L, key, pay, w, lane, CtaSync{}, any);
  }
}

// ---------------------------------------------------------------------------
// > kSortSmemCap: stable LSD radix sort on the (tag-masked) source ID, one
// CTA per list.  The list is cut into 32 contiguous warp ranges; per pass
// every warp scatters its range in order from per-(digit, warp) offsets and
// counts the next pass's digits per destination warp range as it writes.
// Buffers are SoA views (u[], w[]); weighted lists start in the packed
// scratch (AoS) and alternate between the outputs and the same scratch
// region viewed as SoA.
// ---------------------------------------------------------------------------
struct Buf {
  uint32_t *u;
  uint32_t *w;                 // null for unweighted
  unsigned long long *packed;  // non-null: AoS entries (value bits << 32 | source)
  __device__ uint32_t getu(uint32_t i) const { return packed ? (uint32_t)packed[i] : u[i]; }
  __device__ uint32_t getw(uint32_t i) const { return packed ? (uint32_t)(packed[i] >> 32) : (w ? w[i] : 0u); }
  __device__ void put(uint32_t i, uint32_t uu, uint32_t ww) const {
    if (packed) {
      packed[i] = ((unsigned long long)ww << 32) | uu;
    } else {
      u[i] = uu;
      if (w) w[i] = ww;
    }
  }
};

// Sorts a[0, len) (u32 positions of one split-row run; all distinct) with the
// whole CTA: bitonic in shared memory up to kRunSmem values, else a stable
// LSD radix sort (8-bit digits over the bits of the largest value) through
// tmp[0, len), the result back in a.  smem: at least 2 * 256 * 32 words.
constexpr uint32_t kRunSmem = 4096;

__device__ void cta_sort_run(uint32_t *a, uint32_t *tmp, uint32_t len, uint32_t *smem) {
  __shared__ uint32_t s_max;
  const uint32_t tid = threadIdx.x, nt = blockDim.x, w = tid >> 5, lane = tid & 31u;
  if (len <= kRunSmem) {
    uint32_t cap = 2;
    while (cap < len) cap <<= 1;
    for (uint32_t i = tid; i < cap; i += nt) smem[i] = i < len ? a[i] : 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t k = 2; k <= cap; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = tid; i < cap; i += nt) {
          const uint32_t l = i ^ j;
          if (l > i) {
            const uint32_t x = smem[i], y = smem[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              smem[i] = y;
              smem[l] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = tid; i < len; i += nt) a[i] = smem[i];
    __syncthreads();
    return;
  }
  if (tid == 0) s_max = 0;
  __syncthreads();
  uint32_t mx = 0;
  for (uint32_t i = tid; i < len; i += nt) mx = max(mx, a[i]);
  atomicMax(&s_max, mx);
  __syncthreads();
  const uint32_t bits = 32u - (uint32_t)__clz((int)(s_max | 1u));
  const uint32_t passes = (bits + 7) / 8;
  uint32_t *hist = smem, *tot = smem + 256 * 32;  // hist[digit][warp], tot[digit]
  const uint32_t nwarps = nt >> 5;
  const uint32_t chunk = (len + nwarps - 1) / nwarps;
  uint32_t *src = a, *dst = tmp;
  for (uint32_t ps = 0; ps < passes; ++ps) {
    const uint32_t shift = ps * 8;
    for (uint32_t i = tid; i < 256 * 32; i += nt) hist[i] = 0;
    __syncthreads();
    const uint32_t r0 = min(w * chunk, len), r1 = min(r0 + chunk, len);
    for (uint32_t i = r0 + lane; i < r1; i += 32) atomicAdd(&hist[((src[i] >> shift) & 255u) * 32 + w], 1u);
    __syncthreads();
    for (uint32_t d = w; d < 256; d += nwarps) {  // per digit: prefix over warps
      const uint32_t x = hist[d * 32 + lane];
      uint32_t inc = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += y;
      }
      hist[d * 32 + lane] = inc - x;
      if (lane == 31) tot[d] = inc;
    }
    __syncthreads();
    if (w == 0) {  // prefix over digits
      uint32_t run = 0;
      for (uint32_t d0 = 0; d0 < 256; d0 += 32) {
        const uint32_t t = tot[d0 + lane];
        uint32_t inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, inc, o);
          if (lane >= (uint32_t)o) inc += y;
        }
        tot[d0 + lane] = run + inc - t;
        run += __shfl_sync(kFull, inc, 31);
      }
    }
    __syncthreads();
    for (uint32_t i = tid; i < 256 * 32; i += nt) hist[i] += tot[i >> 5];
    __syncthreads();
    for (uint32_t c = r0; c < r1; c += 32) {  // stable scatter, each warp in order
      const uint32_t i = c + lane;
      const bool act = i < r1;
      const uint32_t x = act ? src[i] : 0u;
      const uint32_t d = act ? ((x >> shift) & 255u) : 256u;
      const uint32_t mm = __match_any_sync(kFull, d);
      const uint32_t rank = __popc(mm & lanemask_lt());
      uint32_t base = 0;
      if (act) base = hist[d * 32 + w];
      __syncwarp();
      if (act && rank == 0) hist[d * 32 + w] = base + __popc(mm);
      __syncwarp();
      if (act) dst[base + rank] = x;
    }
    __syncthreads();
    uint32_t *t = src;
    src = dst;
    dst = t;
  }
  if (src != a)
    for (uint32_t i = tid; i < len; i += nt) a[i] = src[i];
  __syncthreads();
}

// Sorts one LDV list [s0, s0 + L) stably by its (tag-masked) source ID and
// writes row_idx / vals_out: an LSD radix sort over the bits of a vertex ID
// with per-(digit, warp) offsets, the list cut into 32 contiguous warp ranges
// (1024 threads); every warp scatters its range in order and counts the next
// pass's digits per destination warp range as it writes.  The first pass
// reads `src`; the passes then alternate between the views x and y.  Tagged
// runs (split rows) are then ordered by their position in the row: a run of
// <= 64 entries by the thread at its start, longer ones by the whole CTA.
// words: the hist / next tables, [256][kHistStride] words each.
struct SortShared {
  uint32_t tagged, nlong;
  uint32_t long_i[kRadixThreads], long_n[kRadixThreads];
};

constexpr uint32_t kHistStride = 33;

template <bool VALS>
__device__ void sort_list(const SortArgs &a, uint64_t s0, uint32_t L, Buf src, const Buf x, const Buf y,
                          uint32_t *words, SortShared &sh) {
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t umask = umask_of(a);
  const uint32_t bits = a.key_bits ? a.key_bits : 1u;
  const uint32_t passes = (bits + 7) / 8;
  const uint32_t dbits = (bits + passes - 1) / passes;
  const uint32_t nb = 1u << dbits;
  const uint32_t chunk = (L + 31) / 32;
  // per-(digit, warp) counters at d * kHistStride + w: lanes of one warp
  // with different digits, and lanes of one digit row, fall in different banks
  uint32_t *hist = words;                       // [256][kHistStride]
  uint32_t *next = words + 256 * kHistStride;  // [256][kHistStride]
  // first pass's per-warp counts; notes whether any entry is tagged
  for (uint32_t i = threadIdx.x; i < 256 * kHistStride; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) sh.tagged = 0;
  __syncthreads();
  {
    const uint32_t r0 = min(w * chunk, L), r1 = min(r0 + chunk, L);
    uint32_t anytag = 0;
    for (uint32_t i = r0 + lane; i < r1; i += 32) {
      const uint32_t u = src.getu(i);
      anytag |= u & ~umask;
      atomicAdd(&hist[(u & umask & (nb - 1)) * kHistStride + w], 1u);
    }
    if (anytag) sh.tagged = 1;
  }
  __syncthreads();
  Buf dst = x;
  for (uint32_t ps = 0; ps < passes; ++ps) {
    const uint32_t shift = ps * dbits;
    // exclusive scan over (digit, warp), digit-major: per-digit prefix over
    // warps, per-digit totals, prefix over digits, then combine
    for (uint32_t d = w; d < nb; d += 32) {
      uint32_t xv = hist[d * kHistStride + lane];
      uint32_t inc = xv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t yv = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += yv;
      }
      hist[d * kHistStride + lane] = inc - xv;
      if (lane == 31) next[d] = inc;  // digit total (next[] is cleared below)
    }
    __syncthreads();
    if (w == 0) {
      uint32_t run = 0;
      for (uint32_t d0 = 0; d0 < nb; d0 += 32) {
        uint32_t t = (d0 + lane < nb) ? next[d0 + lane] : 0u;
        uint32_t inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t yv = __shfl_up_sync(kFull, inc, o);
          if (lane >= (uint32_t)o) inc += yv;
        }
        if (d0 + lane < nb) next[d0 + lane] = run + inc - t;
        run += __shfl_sync(kFull, inc, 31);
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nb * 32; i += blockDim.x) hist[(i >> 5) * kHistStride + (i & 31u)] += next[i >> 5];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 256 * kHistStride; i += blockDim.x) next[i] = 0;
    __syncthreads();
    const uint32_t r0 = min(w * chunk, L), r1 = min(r0 + chunk, L);
    const uint32_t nshift = shift + dbits;
    const bool more = ps + 1 < passes;
    // pos / chunk by a multiply-high with a reciprocal rounded up (at most one
    // too large, corrected below)
    const uint32_t cmag = chunk > 1u ? 0xFFFFFFFFu / chunk + 1u : 0u;
    // the next 32 entries are loaded while this step ranks and scatters
    uint32_t u_n = 0u, w_n = 0u;
    if (r0 + lane < r1) {
      u_n = src.getu(r0 + lane);
      if (VALS) w_n = src.getw(r0 + lane);
    }
    for (uint32_t c = r0; c < r1; c += 32) {
      const uint32_t i = c + lane;
      const bool act = i < r1;
      const uint32_t u = u_n;
      const uint32_t wv = w_n;
      if (i + 32 < r1) {
        u_n = src.getu(i + 32);
        if (VALS) w_n = src.getw(i + 32);
      }
      const uint32_t d = act ? (((u & umask) >> shift) & (nb - 1)) : nb;
      const uint32_t mm = __match_any_sync(kFull, d);
      const uint32_t rank = __popc(mm & lanemask_lt());
      uint32_t base = 0;
      if (act) base = hist[d * kHistStride + w];
      __syncwarp();
      if (act && rank == 0) hist[d * kHistStride + w] = base + __popc(mm);
      __syncwarp();
      if (act) {
        const uint32_t pos = base + rank;
        dst.put(pos, u, VALS ? wv : 0u);
        if (more) {
          uint32_t q = chunk > 1u ? __umulhi(pos, cmag) : pos;
          if (q * chunk > pos) --q;
          atomicAdd(&next[(((u & umask) >> nshift) & (nb - 1)) * kHistStride + min(q, 31u)], 1u);
        }
      }
    }
    __syncthreads();
    uint32_t *t = hist;
    hist = next;
    next = t;
    src = dst;
    dst = (dst.u == x.u) ? y : x;
  }
  // src holds the sorted list (SoA, or AoS in the scratch)
  if (VALS && a.flag_mode && sh.tagged) {
    const Buf other = (src.u == x.u) ? y : x;
    for (uint32_t base = 0; base < L; base += blockDim.x) {
      if (threadIdx.x == 0) sh.nlong = 0;
      __syncthreads();
      const uint32_t i = base + threadIdx.x;
      if (i < L) {
        const uint32_t u = src.getu(i);
        if ((u & kSplitFlag) && (i == 0 || src.getu(i - 1) != u)) {
          uint32_t lo = i, hi = L;  // end of the run: first index past i with another source
          while (hi - lo > 1) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if (src.getu(mid) == u) lo = mid;
            else hi = mid;
          }
          const uint32_t j = hi;
          if (j - i <= 64) {  // by position (the entries of the run share their source)
            for (uint32_t xi = i + 1; xi < j; ++xi) {
              const uint32_t tpos = src.getw(xi);
              uint32_t yi = xi;
              while (yi > i && src.getw(yi - 1) > tpos) {
                src.put(yi, u, src.getw(yi - 1));
                --yi;
              }
              src.put(yi, u, tpos);
            }
          } else {
            const uint32_t q = atomicAdd(&sh.nlong, 1u);
            sh.long_i[q] = i;
            sh.long_n[q] = j - i;
          }
        }
      }
      __syncthreads();
      const uint32_t nl = sh.nlong;
      for (uint32_t q = 0; q < nl; ++q) {
        const uint32_t i0 = sh.long_i[q], n0 = sh.long_n[q];
        if (src.packed) {  // AoS: the run's positions through the other buffer's SoA view, then back
          const uint32_t ur = src.getu(i0);
          for (uint32_t k = threadIdx.x; k < n0; k += blockDim.x) other.w[i0 + k] = src.getw(i0 + k);
          __syncthreads();
          cta_sort_run(other.w + i0, other.u + i0, n0, words);
          for (uint32_t k = threadIdx.x; k < n0; k += blockDim.x) src.put(i0 + k, ur, other.w[i0 + k]);
          __syncthreads();
        } else {  // SoA; the other buffer (SoA or the AoS scratch) is free as temporary space
          cta_sort_run(src.w + i0, other.w ? other.w + i0 : (uint32_t *)other.packed + i0, n0, words);
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) {
    uint32_t u = src.getu(i);
    if (VALS) {
      uint32_t wb = src.getw(i);
      if (a.flag_mode && (u & kSplitFlag)) {
        u &= ~kSplitFlag;
        wb = tagged_value(a, u, wb);
      }
      a.row_idx[s0 + i] = u;
      a.vals_out[s0 + i] = __uint_as_float(wb);
    } else if (src.u != a.row_idx + s0) {
      a.row_idx[s0 + i] = u;
    }
  }
  __syncthreads();
}

// > kSortSmemCap: one CTA per list, through global memory: the outputs and
// the list's scratch alternate (weighted lists start in the packed scratch).
template <bool VALS>
__global__ void __launch_bounds__(kRadixThreads) k_sort_radix(SortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (cta_status_set(a.status)) return;
  __shared__ uint32_t s_item;
  __shared__ SortShared sh;
  const uint32_t nlarge = min(a.meta[kMetaLargeN], a.large_cap);
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(&a.meta[kMetaLargeTicket], 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= nlarge) break;
    const uint32_t v = a.largelist[it];
    const uint64_t s0 = a.col_ptr[v];
    const uint32_t L = (uint32_t)(a.col_ptr[v + 1] - s0);
    const Buf out{a.row_idx + s0, VALS ? (uint32_t *)(a.vals_out + s0) : nullptr, nullptr};
    if (VALS) {  // the list's 8L scratch bytes hold its entries packed, as the scatter left them
      sort_list<VALS>(a, s0, L, Buf{nullptr, nullptr, a.ldv64 + s0}, out, Buf{nullptr, nullptr, a.ldv64 + s0},
                      (uint32_t *)smem, sh);
    } else {
      sort_list<VALS>(a, s0, L, out, Buf{a.scr32 + s0, nullptr, nullptr}, out, (uint32_t *)smem, sh);
    }
  }
}

static size_t warp_smem_bytes(bool vals) { return (size_t)(kWarpThreads / 32) * kMidCap * (vals ? 16 : 4); }
static size_t cta_smem_bytes(bool vals) { return (size_t)kSortSmemCap * (vals ? 16 : 4); }
static size_t radix_smem_bytes() { return (size_t)2 * 256 * kHistStride * 4; }

cudaError_t configure_sort() {
  cudaError_t e[8] = {allow_max_dynamic_smem(k_sort_warp<true>),  allow_max_dynamic_smem(k_sort_warp<false>),
                      allow_max_dynamic_smem(k_sort_cta<true>),   allow_max_dynamic_smem(k_sort_cta<false>),
                      allow_max_dynamic_smem(k_sort_radix<true>), allow_max_dynamic_smem(k_sort_radix<false>),
                      allow_max_dynamic_smem(k_sort_small<true>), allow_max_dynamic_smem(k_sort_small<false>)};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

cudaError_t launch_sort(const DevWork &w, const gt_config &cfg, const Problem &pb, cudaStream_t s) {
  (void)cfg;
  uint32_t bits = 0;
  while (bits < 32 && (w.n_rows - 1) >> bits) ++bits;
  SortArgs sa;
  sa.n = w.n;
  sa.col_ptr = pb.col_ptr;
  sa.row_ptr = pb.row_ptr;
  sa.vals = pb.vals;
  sa.row_idx = pb.row_idx;
  sa.vals_out = pb.vals_out;
  sa.ldv64 = (unsigned long long *)w.scratch;
  sa.scr32 = (uint32_t *)w.scratch;
  sa.hkeys = w.hkeys;
  sa.hvals = w.hvals;
  sa.tlog2 = w.tlog2;
  sa.kmax = w.kmax;
  sa.meta = w.meta;
  sa.status = w.status;
  sa.flag_mode = w.flag_mode;
  sa.key_bits = bits;
  sa.qvals = w.part_bits ? (const float *)w.q_w : nullptr;
  // worklist regions inside biglist: mid | big | large
  sa.mid_cap = (uint32_t)(w.m / (kWarpSortCap + 1) + 1);
  sa.big_cap = (uint32_t)(w.m / (kMidCap + 1) + 1);
  sa.large_cap = (uint32_t)(w.m / (kSortSmemCap + 1) + 1);
  sa.midlist = w.biglist;
  sa.biglist = w.biglist + sa.mid_cap;
  sa.largelist = sa.biglist + sa.big_cap;
  const bool vals = pb.vals != nullptr;
  const size_t ssm = w.kmax ? (size_t)(1u << w.tlog2) * 6 + 16 : 0;
  const uint32_t groups = (w.n + 31) / 32;
  uint32_t g = (groups + 7) / 8;
  const uint32_t gmax = (uint32_t)w.num_sms * 8u;
  if (g > gmax) g = gmax;
  if (g == 0) g = 1;
  if (vals) k_sort_small<true><<<g, 256, ssm, s>>>(sa);
  else k_sort_small<false><<<g, 256, ssm, s>>>(sa);
  const uint32_t gw = (uint32_t)w.num_sms * 4u;
  if (vals) k_sort_warp<true><<<gw, kWarpThreads, warp_smem_bytes(true), s>>>(sa);
  else k_sort_warp<false><<<gw, kWarpThreads, warp_smem_bytes(false), s>>>(sa);
  const uint32_t gc = (uint32_t)w.num_sms * 4u;
  if (vals) k_sort_cta<true><<<gc, kCtaThreads, cta_smem_bytes(true), s>>>(sa);
  else k_sort_cta<false><<<gc, kCtaThreads, cta_smem_bytes(false), s>>>(sa);
  const uint32_t gr = (uint32_t)w.num_sms * 2u;
  if (vals) k_sort_radix<true><<<gr, kRadixThreads, radix_smem_bytes(), s>>>(sa);
  else k_sort_radix<false><<<gr, kRadixThreads, radix_smem_bytes(), s>>>(sa);
  return cudaGetLastError();
}

}  // namespace gt
