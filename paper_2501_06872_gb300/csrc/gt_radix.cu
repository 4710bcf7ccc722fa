// Radix method: the CSC as a stable LSD radix sort of the CSR edge sequence
// by destination.  Sec. II-A defines the transpose; sorting the (source,
// destination, value) triples stably by destination from CSR order gives
// every in-list in ascending source order with parallel edges in CSR order
// (Gustavson's sort-based transposition, Sec. VI, done as a counting sort
// per digit).  Every pass streams the data once, so the method is bound by
// HBM bandwidth whatever the vertex order; it is the method chosen for
// graphs whose working set is far larger than L2.
//
// Per call: the row expansion writes the source of every edge; then per
// digit pass (passes = ceil(bits(n-1) / the digit cap, 8 by default) for n
// columns, digits split evenly):
//   upsweep    per-CTA digit counts of the CTA's contiguous tile range
//              (with the bulk downsweep, two upsweep CTAs per range)
//   offsets    exclusive scan of the table in (digit, CTA) order
//   downsweep  each persistent CTA walks its tiles in order, ranks every tile
//              stably in shared memory and writes coalesced digit runs from
//              running per-digit offsets (k_radix_down_bulk: bulk-copy staged
//              4096-edge tiles, 2 CTAs per SM; k_radix_down: register tiles)
// The last pass writes row_idx / vals_out and the sorted keys; col_ptr then
// comes straight from the sorted keys (k_radix_colptr).  Batches run the
// same passes over the union of their graphs (key = graph, destination).
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {

constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr int kRBins = 256;

// Lanes holding the same dbits-bit digit (and active): AND of one ballot per
// bit -- cheaper than __match_any_sync for digits of a few bits.
__device__ __forceinline__ uint32_t match_digit(uint32_t d, uint32_t dbits, bool act) {
  // digits have at most 8 bits; the bits above dbits are 0 in every lane, so
  // their ballots change nothing and the loop unrolls at compile time
  (void)dbits;
  uint32_t mm = __ballot_sync(kFull, act);
#pragma unroll
  for (uint32_t b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t bb = __ballot_sync(kFull, bit);
    mm &= bit ? bb : ~bb;
  }
  return mm;
}

// Batch view: the sub-batch (graphs g0 .. g0+ng-1 of a call) whose layout
// k_b_layout wrote on the device for this call.  Its graphs lie one after
// another in a union edge space, column space and row-window space; a union
// key is (local graph << vbits) | column.  slot == nullptr: a single graph
// (the sizes are the kernel arguments).
struct BatchView {
  const BatchSlot *slot;
  uint32_t vbits;
};

__device__ __forceinline__ uint32_t upper_graph(const unsigned long long *off, uint32_t ng, uint64_t x) {
  uint32_t lo = 0, hi = ng;  // largest g with off[g] <= x
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) / 2;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The graph's status word of the call (if the caller passed one) and the
// batch's status word both receive the first error.
__device__ __forceinline__ void graph_error(const BatchSlot &sl, uint32_t g, uint32_t *status, gt_status code) {
  if (sl.gstatus) atomicCAS((unsigned int *)(sl.gstatus + g), 0u, (unsigned int)code);
  set_status(status, code);
}

struct RadixArgs {
  // CSR (first pass)
  const uint64_t *row_ptr;
  const uint32_t *col_idx;
  const float *vals;
  uint32_t n;
  uint64_t m;
  // this pass
  const uint32_t *in_key, *in_u, *in_w;
  uint32_t *out_key, *out_u, *out_w;
  uint32_t shift, dbits;
  uint32_t ntiles, tiles_per_cta;
  uint32_t tile;  // elements per tile (threads * items)
  uint32_t *table;                    // [G][256] counts
  const unsigned long long *offsets;  // [G][256] starting positions
  uint32_t *status;
  BatchView batch;
  uint32_t sub = 1;  // upsweep CTAs per downsweep CTA (table rows = G * sub)
  uint32_t *g_key = nullptr, *g_w = nullptr;  // batch first upsweep: gathered union keys / values
};

// Sizes of a pass: the kernel arguments, or for a sub-batch the union edge
// count of this call (tiles of `tile` edges over `ctas` persistent CTAs).
struct PassSizes {
  uint64_t m, ntiles;
  uint32_t tpc;
};
__device__ __forceinline__ PassSizes pass_sizes(const RadixArgs &a, uint32_t ctas) {
  if (!a.batch.slot) return PassSizes{a.m, a.ntiles, a.tiles_per_cta};
  const uint64_t m = a.batch.slot->m, nt = (m + a.tile - 1) / a.tile;
  return PassSizes{m, nt, (uint32_t)((nt + ctas - 1) / ctas)};
}

// Pass modes: plain arrays; a batch's first upsweep, which reads through the
// descriptors (and gathers the union keys); a batch's last downsweep, which
// stores through them.
enum RadixMode : int { kPlain = 0, kBatchFirst = 1, kBatchLast = 2 };
__host__ __device__ constexpr bool loads_batch(int mode) { return mode == kBatchFirst; }
__host__ __device__ constexpr bool stores_batch(int mode) { return mode == kBatchLast; }

// Writes the source row of every edge (src[e] = u for e in row u).  Rows of
// at most kLongRow edges: 32 rows per warp step, whose edges form one
// contiguous range; each lane finds the row of its position among the 32 row
// ends held in registers.  Longer rows are listed for k_expand_long.
constexpr uint32_t kLongRow = 2048;

__global__ void k_expand_rows(const uint64_t *__restrict__ row_ptr, uint32_t n_rows, uint64_t m, uint32_t *src,
                              uint32_t *long_rows, uint32_t *n_long, uint32_t long_cap, uint32_t *status) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0 && (row_ptr[0] != 0 || row_ptr[n_rows] != m))
    set_status(status, GT_ERR_BAD_ROW_PTR);
  for (uint64_t r0 = (blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < n_rows; r0 += warps * 32) {
    const uint64_t r = r0 + lane;
    uint64_t ri = r + 1;
    if (ri > n_rows) ri = n_rows;
    uint64_t rend = row_ptr[ri];  // end of row r (clamped)
    uint64_t rbeg = r < n_rows ? row_ptr[r] : rend;
    if (rend > m || rbeg > rend) {  // invalid row pointers: report, write nothing out of range
      set_status(status, GT_ERR_BAD_ROW_PTR);
      rend = rbeg = 0;
    }
    const bool is_long = r < n_rows && rend - rbeg > kLongRow;
    if (is_long) {
      uint32_t i = atomicAdd(n_long, 1u);
      if (i < long_cap) long_rows[i] = (uint32_t)r;
      else set_status(status, GT_ERR_UNSUPPORTED);
    }
    const uint32_t longmask = __ballot_sync(kFull, is_long);
    const uint64_t b = __shfl_sync(kFull, rbeg, 0);
    const uint64_t e = __shfl_sync(kFull, rend, 31);
    if (longmask == 0) {  // at most 32 x kLongRow edges: offsets from b fit 32 bits
      const uint32_t rrel = (uint32_t)(rend - b);
      for (uint64_t p0 = b; p0 < e; p0 += 32) {
        const uint64_t p = p0 + lane;
        const uint32_t pos = count_le32(rrel, (uint32_t)(p - b));  // warp-collective
        if (p < e) src[p] = (uint32_t)(r0 + pos);
      }
    } else {
      // short rows of this window one by one (the long ones are skipped)
      uint32_t todo = __ballot_sync(kFull, r < n_rows && !is_long && rend > rbeg);
      while (todo) {
        const uint32_t j = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint64_t qb = __shfl_sync(kFull, rbeg, j), qe = __shfl_sync(kFull, rend, j);
        for (uint64_t p = qb + lane; p < qe; p += 32) src[p] = (uint32_t)(r0 + j);
      }
    }
  }
}

// One CTA per long row.
__global__ void k_expand_long(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ long_rows,
                              const uint32_t *__restrict__ n_long, uint32_t long_cap, uint32_t *src) {
  const uint32_t cnt = min(*n_long, long_cap);
  for (uint32_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const uint32_t r = long_rows[i];
    const uint64_t b = row_ptr[r], e = row_ptr[r + 1];  // checked by k_expand_rows
    for (uint64_t p = b + threadIdx.x; p < e; p += blockDim.x) src[p] = r;
  }
}

// Counts the digits of this CTA's tiles: per-warp shared-memory histograms,
// 8 loads in flight per thread.
template <bool FIRST, int MODE>
__global__ void __launch_bounds__(kRThreads) k_radix_up(RadixArgs a) {
  __shared__ uint32_t cnt[kRWarps][kRBins];
  for (uint32_t i = threadIdx.x; i < kRWarps * kRBins; i += blockDim.x) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t mask = (1u << a.dbits) - 1u;
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const PassSizes ps = pass_sizes(a, gridDim.x / a.sub);
  const uint64_t t0 = (uint64_t)(blockIdx.x / a.sub) * ps.tpc;
  uint64_t e0 = min64(t0 * a.tile, ps.m), e1 = min64((t0 + ps.tpc) * a.tile, ps.m);
  if (a.sub > 1) {  // this CTA counts part (blockIdx.x % sub) of the downsweep CTA's range
    const uint64_t part = (e1 - e0 + a.sub - 1) / a.sub, s0 = e0 + (blockIdx.x % a.sub) * part;
    e1 = min64(s0 + part, e1);
    e0 = min64(s0, e1);
  }
  const uint32_t *src = a.in_key;
  constexpr int U = 8;
  uint32_t bad = 0;
  for (uint64_t c = e0 + (uint64_t)w * 32 * U; c < e1; c += (uint64_t)kRWarps * 32 * U) {
    uint32_t key[U];
    if (loads_batch(MODE)) {
      const BatchSlot &sl = *a.batch.slot;
      // union edge e of the sub-batch is edge sl.e0 + e of the call
      uint32_t g = upper_graph(sl.eoff, sl.ng, sl.e0 + (c < e1 ? c : e1 - 1));
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const uint64_t e = c + (uint64_t)i * 32 + lane;
        key[i] = 0xFFFFFFFFu;
        if (e < e1) {
          while (sl.e0 + e >= sl.eoff[g + 1]) ++g;
          const gt_graph_desc &d = sl.descs[g];
          const uint64_t le = sl.e0 + e - sl.eoff[g];
          uint32_t v = __ldcs(d.col_idx + le);
          if (v >= desc_cols(d)) {  // reported; kept inside the graph's own key range
            bad = 1;
            graph_error(sl, g, a.status, GT_ERR_OUT_OF_RANGE);
            v = desc_cols(d) - 1u;
          }
          key[i] = (g << a.batch.vbits) | (v & ((1u << a.batch.vbits) - 1u));
          if (a.g_key) {  // gather the union key (and value) for a plain first pass
            a.g_key[e] = key[i];
            if (a.g_w) a.g_w[e] = __float_as_uint(__ldcs(d.vals + le));
          }
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const uint64_t e = c + (uint64_t)i * 32 + lane;
        key[i] = e < e1 ? __ldcs(src + e) : 0xFFFFFFFFu;
      }
    }
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint64_t e = c + (uint64_t)i * 32 + lane;
      if (e < e1) {
        if (FIRST && !loads_batch(MODE) && key[i] >= a.n) bad = 1;
        atomicAdd(&cnt[w][(key[i] >> a.shift) & mask], 1u);
      }
    }
  }
  if (bad) set_status(a.status, GT_ERR_OUT_OF_RANGE);
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < kRBins; d += blockDim.x) {
    uint32_t t = 0;
#pragma unroll
    for (int x = 0; x < kRWarps; ++x) t += cnt[x][d];
    a.table[(size_t)blockIdx.x * kRBins + d] = t;
  }
}

// Exclusive scan of table[G][256] in (digit, cta) order -> offsets[G][256].
// One CTA of 1024 threads: 4 segments of CTAs x 256 digits, 8 loads in flight.
__global__ void __launch_bounds__(1024) k_radix_offsets(const uint32_t *__restrict__ table, uint32_t G,
                                                        unsigned long long *offsets) {
  __shared__ unsigned long long part[4][kRBins];
  const uint32_t d = threadIdx.x & (kRBins - 1), seg = threadIdx.x >> 8;
  const uint32_t per = (G + 3) / 4;
  const uint32_t c0 = min(seg * per, G), c1 = min(c0 + per, G);
  unsigned long long s = 0;
  uint32_t c = c0;
  for (; c + 8 <= c1; c += 8) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = table[(size_t)(c + i) * kRBins + d];
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
  }
  for (; c < c1; ++c) s += table[(size_t)c * kRBins + d];
  part[seg][d] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    // digit totals -> exclusive prefix over digits (one warp, 8 digits per lane)
    unsigned long long tot[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t dd = threadIdx.x * 8 + i;
      tot[i] = part[0][dd] + part[1][dd] + part[2][dd] + part[3][dd];
      sum += tot[i];
    }
    unsigned long long inc = sum;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(kFull, inc, o);
      if (threadIdx.x >= (uint32_t)o) inc += y;
    }
    unsigned long long run = inc - sum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t dd = threadIdx.x * 8 + i;
      // turn the four segment sums of digit dd into their starting positions
      unsigned long long r = run;
      for (int q = 0; q < 4; ++q) {
        unsigned long long x = part[q][dd];
        part[q][dd] = r;
        r += x;
      }
      run += tot[i];
    }
  }
  __syncthreads();
  unsigned long long run = part[seg][d];
  c = c0;
  for (; c + 8 <= c1; c += 8) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = table[(size_t)(c + i) * kRBins + d];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      offsets[(size_t)(c + i) * kRBins + d] = run;
      run += x[i];
    }
  }
  for (; c < c1; ++c) {
    offsets[(size_t)c * kRBins + d] = run;
    run += table[(size_t)c * kRBins + d];
  }
}

template <bool VALS, int ITEMS>
__global__ void __launch_bounds__(kRThreads) k_radix_down(RadixArgs a) {
  constexpr uint32_t TILE = kRThreads * ITEMS;
  extern __shared__ __align__(16) uint32_t stage[];  // [TILE] keys | [TILE] sources | [TILE] values
  __shared__ uint32_t wcnt[kRWarps][kRBins];
  __shared__ unsigned long long run_off[kRBins];
  __shared__ uint32_t tile_tot[kRBins];
  __shared__ uint32_t tile_start[kRBins];
  __shared__ uint32_t wsum[kRWarps];
  uint32_t *skey = stage, *su = stage + TILE, *sw = stage + 2 * TILE;
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t mask = (1u << a.dbits) - 1u;
  for (uint32_t d = threadIdx.x; d < kRBins; d += blockDim.x)
    run_off[d] = a.offsets[(size_t)blockIdx.x * kRBins + d];
  const uint64_t t0 = (uint64_t)blockIdx.x * a.tiles_per_cta;
  const uint64_t t1 = min64(t0 + a.tiles_per_cta, a.ntiles);
  for (uint64_t tile = t0; tile < t1; ++tile) {
    for (uint32_t i = threadIdx.x; i < kRWarps * kRBins; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    const uint64_t tbase = tile * TILE;
    const uint64_t base = tbase + (uint64_t)w * (ITEMS * 32);
    const uint32_t tcount = (uint32_t)min64(TILE, a.m - tbase);
    uint32_t key[ITEMS], uu[ITEMS], ww[ITEMS], rk[ITEMS];
    // all of this warp's loads are in flight before any ranking
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint64_t e = base + (uint64_t)i * 32 + lane;
      if (e < a.m) {
        key[i] = __ldcs(a.in_key + e);
        uu[i] = __ldcs(a.in_u + e);
        ww[i] = VALS ? __ldcs(a.in_w + e) : 0u;
      } else {
        key[i] = 0u;
        uu[i] = 0u;
        ww[i] = 0u;
      }
    }
    __syncthreads();
    // stable rank within the warp: items in order, lanes in order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool act = base + (uint64_t)i * 32 + lane < a.m;
      const uint32_t d = (key[i] >> a.shift) & mask;
      const uint32_t mm = match_digit(d, a.dbits, act);
      const uint32_t r = __popc(mm & lanemask_lt());
      uint32_t b = 0;
      if (act) b = wcnt[w][d];
      __syncwarp();
      if (act && r == 0) wcnt[w][d] = b + __popc(mm);
      __syncwarp();
      rk[i] = act ? (b + r) : 0xFFFFFFFFu;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps and the tile total; then the
    // tile-local start of every digit (exclusive scan over digits)
    uint32_t tot = 0;
    {
      const uint32_t d = threadIdx.x;  // kRThreads == kRBins
      uint32_t run = 0;
#pragma unroll
      for (int x = 0; x < kRWarps; ++x) {
        uint32_t c = wcnt[x][d];
        wcnt[x][d] = run;
        run += c;
      }
      tot = run;
      tile_tot[d] = run;
      uint32_t inc = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += y;
      }
      if (lane == 31) wsum[w] = inc;
      __syncthreads();
      uint32_t before = 0;
      for (uint32_t x = 0; x < w; ++x) before += wsum[x];
      tile_start[d] = before + inc - run;
    }
    __syncthreads();
    // place the tile in shared memory in (digit, rank) order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (rk[i] != 0xFFFFFFFFu) {
        const uint32_t d = (key[i] >> a.shift) & mask;
        const uint32_t lp = tile_start[d] + wcnt[w][d] + rk[i];
        skey[lp] = key[i];
        su[lp] = uu[i];
        if (VALS) sw[lp] = ww[i];
      }
    }
    __syncthreads();
    // consecutive threads write consecutive positions of each digit's run
    for (uint32_t j = threadIdx.x; j < tcount; j += blockDim.x) {
      const uint32_t k = skey[j];
      const uint32_t d = (k >> a.shift) & mask;
      const uint64_t pos = run_off[d] + (j - tile_start[d]);
      a.out_key[pos] = k;
      a.out_u[pos] = su[j];
      if (VALS) a.out_w[pos] = sw[j];
    }
    __syncthreads();
    run_off[threadIdx.x] += tot;
    __syncthreads();
  }
}

// Downsweep with bulk-copy staging (plain arrays, 16-byte aligned): two
// persistent CTAs of 256 threads per SM, each walking its contiguous tiles of
// 4096 edges.  The next tile's keys, sources and values arrive in shared
// memory through cp.async.bulk (the TMA engine), double-buffered behind
// mbarriers, while the current tile is ranked (ballot digit matching,
// stable).  The tile is then pulled into registers and written back to the
// same buffer in (digit, rank) order, and leaves as coalesced digit runs;
// the freed buffer receives the tile after next.  A ragged final tile is
// loaded with plain loads.  Every mbarrier wait is bounded; on expiry the CTA
// reports GT_ERR_TIMEOUT, waits (bounded) for its copies in flight and
// returns.
constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kBItems = 16;
constexpr uint32_t kBTile = kBThreads * kBItems;
constexpr uint32_t kBCtasPerSm = 2;  // registers (~120 x 256 threads) and 2 x ~109 KB of shared memory

__host__ __device__ constexpr uint32_t bulk_arrays(bool vals) { return vals ? 3u : 2u; }
__host__ constexpr size_t bulk_dyn_smem(bool vals) { return (size_t)2 * bulk_arrays(vals) * kBTile * 4; }

// SVI / SVO (weighted plain passes only): the pass reads / writes (source,
// value) as one interleaved u64 array at in_u / out_u instead of two u32
// arrays: one bulk copy and one 8-byte store per edge for the pair.
template <bool VALS, int MODE, bool SVI = false, bool SVO = false>
__global__ void __launch_bounds__(kBThreads, kBCtasPerSm) k_radix_down_bulk(RadixArgs a) {
  static_assert(!loads_batch(MODE), "the bulk downsweep reads plain arrays");
  static_assert(VALS || (!SVI && !SVO), "interleaved pairs carry values");
  static_assert(MODE == kPlain || !SVO, "batches store through their descriptors");
  constexpr uint32_t NA = bulk_arrays(VALS);
  extern __shared__ __align__(128) uint32_t dsm[];  // buf[2][NA][TILE]
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t wcnt[kBWarps][kRBins];
  __shared__ unsigned long long run_off[kRBins];
  __shared__ unsigned long long dst_base[kRBins];  // run_off[d] - (tile-local start of d) for the current tile
  __shared__ uint32_t wsum[kBWarps];
  __shared__ uint32_t s_abort;
  const uint32_t tid = threadIdx.x, w = tid >> 5, lane = tid & 31u;
  const uint32_t mask = (1u << a.dbits) - 1u;
  const PassSizes ps = pass_sizes(a, gridDim.x);
  const uint64_t t0 = (uint64_t)blockIdx.x * ps.tpc;
  const uint64_t t1 = min64(t0 + ps.tpc, ps.ntiles);
  if (t0 >= t1) return;
  run_off[tid] = a.offsets[(size_t)blockIdx.x * a.sub * kRBins + tid];  // kBThreads == kRBins
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  auto full = [&](uint64_t t) { return (t + 1) * kBTile <= ps.m; };
  auto issue = [&](uint64_t t, uint32_t b) {  // one thread
    uint32_t *dst = dsm + b * NA * kBTile;
    const uint64_t e = t * kBTile;
    mbar_arrive_expect_tx(&bar[b], NA * kBTile * 4u);
    bulk_g2s(dst, a.in_key + e, kBTile * 4u, &bar[b]);
    if (SVI) {
      bulk_g2s(dst + kBTile, a.in_u + 2 * e, kBTile * 8u, &bar[b]);  // pairs land interleaved
    } else {
      bulk_g2s(dst + kBTile, a.in_u + e, kBTile * 4u, &bar[b]);
      if (VALS) bulk_g2s(dst + 2 * kBTile, a.in_w + e, kBTile * 4u, &bar[b]);
    }
  };
  if (tid == 0 && full(t0)) issue(t0, 0);
  // bit b: parity of buffer b's next phase
  uint32_t par = 0u;
  // Per tile: every warp ranks its items as soon as it has written its part
  // of the previous tile (the digit counters are per-warp rows); barriers
  // separate only the steps that read other warps' data.
  for (uint64_t t = t0; t < t1; ++t) {
    const uint32_t b = (uint32_t)((t - t0) & 1u);
    uint32_t *bk = dsm + b * NA * kBTile, *bu = bk + kBTile, *bw = bk + 2 * kBTile;
    const uint64_t tbase = t * kBTile;
    const uint32_t tcount = (uint32_t)min64(kBTile, ps.m - tbase);
    const uint32_t wpar = (par >> b) & 1u;  // parity of this tile's copy
    if (tcount == kBTile) {
      if (!mbar_wait(&bar[b], wpar)) s_abort = 1;
      par ^= 1u << b;
    } else {  // the ragged last tile: plain loads (its buffer held tile t - 2, written out long ago)
      for (uint32_t j = tid; j < tcount; j += kBThreads) {
        bk[j] = __ldcs(a.in_key + tbase + j);
        if (SVI) {
          reinterpret_cast<uint2 *>(bu)[j] = __ldcs(reinterpret_cast<const uint2 *>(a.in_u) + tbase + j);
        } else {
          bu[j] = __ldcs(a.in_u + tbase + j);
          if (VALS) bw[j] = __ldcs(a.in_w + tbase + j);
        }
      }
      __syncthreads();
    }
    // this warp's counter row (no other warp touches it until the barrier below)
#pragma unroll
    for (int x = 0; x < kRBins / 32; ++x) wcnt[w][x * 32 + lane] = 0;
    __syncwarp();
    // stable rank within the warp (items in order, lanes in order); the
    // tile moves into registers
    uint32_t key[kBItems], uu[kBItems], ww[kBItems], rk[kBItems];
#pragma unroll
    for (int i = 0; i < kBItems; ++i) {
      const uint32_t j = w * (kBItems * 32) + i * 32 + lane;
      const bool act = j < tcount;
      key[i] = act ? bk[j] : 0u;
      if (SVI) {
        const uint2 p = act ? reinterpret_cast<const uint2 *>(bu)[j] : make_uint2(0u, 0u);
        uu[i] = p.x;
        ww[i] = p.y;
      } else {
        uu[i] = act ? bu[j] : 0u;
        ww[i] = (VALS && act) ? bw[j] : 0u;
      }
    }
#pragma unroll
    for (int i = 0; i < kBItems; ++i) {
      const bool act = w * (kBItems * 32) + i * 32 + lane < tcount;
      const uint32_t d = (key[i] >> a.shift) & mask;
      const uint32_t mm = match_digit(d, a.dbits, act);
      const uint32_t r = __popc(mm & lanemask_lt());
      uint32_t c = 0;
      if (act) c = wcnt[w][d];
      __syncwarp();
      if (act && r == 0) wcnt[w][d] = c + __popc(mm);
      __syncwarp();
      rk[i] = act ? (c + r) : 0xFFFFFFFFu;
    }
    __syncthreads();  // (A) every warp ranked this tile and wrote out the previous one
    if (s_abort) {
      if (tid == 0) {
        set_status(a.status, GT_ERR_TIMEOUT);
        if (tcount == kBTile) mbar_wait(&bar[b], wpar);  // the only copy that can be in flight
      }
      return;
    }
    // the other buffer (the previous tile) is free: copy the next tile into it
    if (t + 1 < t1 && full(t + 1) && tid == 0) {
      fence_proxy_async();
      issue(t + 1, b ^ 1u);
    }
    // per digit (one thread each): exclusive prefix over warps, tile total,
    // then the tile-local start of every digit
    uint32_t run = 0;
#pragma unroll
    for (int x = 0; x < kBWarps; ++x) {
      const uint32_t c = wcnt[x][tid];
      wcnt[x][tid] = run;
      run += c;
    }
    const uint32_t tot = run;
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, inc, o);
      if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();  // (B)
    {
      uint32_t before = 0;
#pragma unroll
      for (int x = 0; x < kBWarps; ++x) before += (x < (int)w) ? wsum[x] : 0u;
      const uint32_t ts = before + inc - tot;  // tile-local start of digit tid
      dst_base[tid] = run_off[tid] - ts;
      run_off[tid] += tot;
#pragma unroll
      for (int x = 0; x < kBWarps; ++x) wcnt[x][tid] += ts;  // per-warp bases, tile-local
    }
    __syncthreads();  // (C)
    // back into the same buffer in (digit, rank) order; weighted tiles keep
    // (source, value) pairs interleaved in the source and value arrays' space
#pragma unroll
    for (int i = 0; i < kBItems; ++i) {
      if (rk[i] != 0xFFFFFFFFu) {
        const uint32_t d = (key[i] >> a.shift) & mask;
        const uint32_t lp = wcnt[w][d] + rk[i];
        bk[lp] = key[i];
        if (VALS) reinterpret_cast<uint2 *>(bu)[lp] = make_uint2(uu[i], ww[i]);
        else bu[lp] = uu[i];
      }
    }
    __syncthreads();  // (D)
    auto put = [&](uint32_t j) {
      const uint32_t k = bk[j];
      const uint32_t d = (k >> a.shift) & mask;
      const uint64_t pos = dst_base[d] + j;
      uint32_t u, wv = 0;
      if (VALS) {
        const uint2 uw = reinterpret_cast<const uint2 *>(bu)[j];
        u = uw.x;
        wv = uw.y;
      } else {
        u = bu[j];
      }
      a.out_key[pos] = k;
      if (stores_batch(MODE)) {  // the last pass of a batch stores through the graph's descriptor
        const BatchSlot &sl = *a.batch.slot;
        const uint32_t g = k >> a.batch.vbits;
        const gt_graph_desc &gd = sl.descs[g];
        const uint64_t lp = sl.e0 + pos - sl.eoff[g];
        gd.row_idx[lp] = u;
        if (VALS) gd.vals_out[lp] = __uint_as_float(wv);
      } else if (SVO) {
        reinterpret_cast<uint2 *>(a.out_u)[pos] = make_uint2(u, wv);
      } else {
        a.out_u[pos] = u;
        if (VALS) a.out_w[pos] = wv;
      }
    };
    if (tcount == kBTile) {
#pragma unroll 4
      for (int q = 0; q < kBItems; ++q) put(q * kBThreads + tid);
    } else {
      for (uint32_t j = tid; j < tcount; j += kBThreads) put(j);
    }
    // no barrier: the next tile's ranking overlaps this write phase
  }
}

// col_ptr straight from the sorted keys: col_ptr[v] = #edges with key < v.
// Each warp takes chunks of 256 positions [c, c + 256).  The entries the
// chunk determines form one vertex range [key[c-1] + 1, key of the chunk's
// last position] (up to n for the last chunk), and for v in it col_ptr[v] =
// c + (chunk keys < v), a binary search over the chunk's keys in shared
// memory: the warp stores the range with coalesced writes, no atomics.  A
// chunk whose range is longer than kChunkRange (a long run of empty
// vertices) stores per run start instead: short ranges by their lane, medium
// ones by the warp together, long ones listed for k_radix_gaps.  Keys >= n
// (an out-of-range input, already reported) are treated as n.
constexpr uint32_t kGapLong = 1024;
constexpr uint32_t kCpChunk = 256;
constexpr uint32_t kChunkRange = 4096;

__device__ __forceinline__ void colptr_range(uint64_t a, uint64_t b, uint64_t val, uint64_t *col_ptr,
                                             unsigned long long *gaps, uint32_t gap_cap, uint32_t *status,
                                             uint32_t lane) {
  const uint64_t len = b >= a ? b - a + 1 : 0;
  if (len > 0 && len <= 32)
    for (uint64_t v = a; v <= b; ++v) col_ptr[v] = val;
  if (len > kGapLong) {
    const uint32_t i = atomicAdd((uint32_t *)gaps, 1u);
    if (i < gap_cap) {
      gaps[1 + 2 * (uint64_t)i] = (a << 32) | b;
      gaps[2 + 2 * (uint64_t)i] = val;
    } else {
      set_status(status, GT_ERR_UNSUPPORTED);
    }
  }
  uint32_t mid = __ballot_sync(kFull, len > 32 && len <= kGapLong);
  while (mid) {  // the warp stores each medium range together
    const int j = __ffs(mid) - 1;
    mid &= mid - 1;
    const uint64_t ja = __shfl_sync(kFull, a, j), jb = __shfl_sync(kFull, b, j);
    const uint64_t jv = __shfl_sync(kFull, val, j);
    for (uint64_t v = ja + lane; v <= jb; v += 32) col_ptr[v] = jv;
  }
}

// Key -> position in the col_ptr space: the key itself (clamped to n), or,
// for a batch, the compact union index voff[graph] + column (clamped to the
// graph's column count), which is monotone in the key.
template <bool BATCH>
__device__ __forceinline__ uint32_t cp_index(uint32_t k, uint32_t n, const BatchView &bv) {
  if (!BATCH) return min(k, n);
  const BatchSlot &sl = *bv.slot;
  const uint32_t g = k >> bv.vbits;
  if (g >= sl.ng) return n;
  const uint32_t v = k & ((1u << bv.vbits) - 1u);
  return (uint32_t)(sl.voff[g] - sl.v0 + min(v, desc_cols(sl.descs[g])));
}

template <bool BATCH>
__global__ void __launch_bounds__(256) k_radix_colptr(const uint32_t *__restrict__ key, uint64_t m, uint32_t n,
                                                      uint64_t *col_ptr, unsigned long long *gaps, uint32_t gap_cap,
                                                      uint32_t *status, BatchView bv) {
  __shared__ uint32_t sk[8][kCpChunk];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  uint32_t *ck = sk[w];
  if (BATCH) {  // this call's sub-batch: its union edges and columns
    m = bv.slot->m;
    n = (uint32_t)bv.slot->nv;
  }
  const uint64_t nwarps = (uint64_t)gridDim.x * 8;
  for (uint64_t c = ((uint64_t)blockIdx.x * 8 + w) * kCpChunk; c < m; c += nwarps * kCpChunk) {
    const uint32_t cnt = (uint32_t)min64(kCpChunk, m - c);
#pragma unroll
    for (int i = 0; i < (int)(kCpChunk / 32); ++i) {
      const uint32_t j = i * 32 + lane;
      ck[j] = j < cnt ? cp_index<BATCH>(__ldcs(key + c + j), n, bv) : 0xFFFFFFFFu;
    }
    __syncwarp();
    const uint64_t lo = c == 0 ? 0 : (uint64_t)cp_index<BATCH>(key[c - 1], n, bv) + 1;
    const uint64_t hi = (c + cnt == m) ? (uint64_t)n : (uint64_t)ck[cnt - 1];
    if (hi + 1 <= lo + kChunkRange) {
      for (uint64_t v = lo + lane; v <= hi; v += 32) {
        uint32_t l = 0, r = cnt;  // first chunk index with key >= v
        while (l < r) {
          const uint32_t mid = (l + r) >> 1;
          if ((uint64_t)ck[mid] < v) l = mid + 1;
          else r = mid;
        }
        col_ptr[v] = c + l;
      }
    } else {
      // per run start: (key[p-1], key[p]] gets p; the last position also
      // (key[m-1], n] gets m
#pragma unroll 1
      for (uint32_t i = 0; i < kCpChunk / 32; ++i) {
        const uint32_t j = i * 32 + lane;
        const uint64_t p = c + j;
        uint64_t a = 1, b = 0, a2 = 1, b2 = 0;
        if (j < cnt) {
          const uint32_t k = ck[j];
          const uint64_t kp = j ? (uint64_t)ck[j - 1] : (c == 0 ? ~0ull : lo - 1);
          if (p == 0 || kp != k) {
            a = p == 0 ? 0 : kp + 1;
            b = k;
          }
          if (p + 1 == m) {
            a2 = (uint64_t)k + 1;
            b2 = n;
          }
        }
        colptr_range(a, b, p, col_ptr, gaps, gap_cap, status, lane);
        colptr_range(a2, b2, m, col_ptr, gaps, gap_cap, status, lane);
      }
    }
    __syncwarp();
  }
}

// The listed long ranges, each by the whole grid.
__global__ void k_radix_gaps(const unsigned long long *__restrict__ gaps, uint32_t gap_cap, uint64_t *col_ptr) {
  const uint32_t cnt = min(*(const uint32_t *)gaps, gap_cap);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t i = 0; i < cnt; ++i) {
    const uint64_t r = gaps[1 + 2 * (uint64_t)i], val = gaps[2 + 2 * (uint64_t)i];
    const uint64_t a = r >> 32, b = r & 0xFFFFFFFFull;
    for (uint64_t v = a + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= b; v += stride) col_ptr[v] = val;
  }
}

// ---------------------------------------------------------------------------

static uint32_t key_bits_of(uint32_t n) {
  uint32_t bits = 0;
  while (bits < 32 && (n - 1) >> bits) ++bits;
  return bits ? bits : 1u;
}

template <int ITEMS>
static cudaError_t allow_down() {
  cudaError_t e1 = allow_max_dynamic_smem(k_radix_down<true, ITEMS>);
  cudaError_t e2 = allow_max_dynamic_smem(k_radix_down<false, ITEMS>);
  return e1 != cudaSuccess ? e1 : e2;
}

cudaError_t configure_radix() {
  cudaError_t e[2] = {allow_down<8>(), allow_down<16>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  cudaError_t b[8] = {allow_max_dynamic_smem(k_radix_down_bulk<true, kPlain>),
                      allow_max_dynamic_smem(k_radix_down_bulk<false, kPlain>),
                      allow_max_dynamic_smem(k_radix_down_bulk<true, kBatchLast>),
                      allow_max_dynamic_smem(k_radix_down_bulk<false, kBatchLast>),
                      allow_max_dynamic_smem(k_radix_down_bulk<true, kPlain, false, true>),
                      allow_max_dynamic_smem(k_radix_down_bulk<true, kPlain, true, false>),
                      allow_max_dynamic_smem(k_radix_down_bulk<true, kPlain, true, true>),
                      allow_max_dynamic_smem(k_radix_down_bulk<true, kBatchLast, true, false>)};
  for (cudaError_t x : b)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

static void launch_down(bool vals, uint32_t items, uint32_t G, size_t dsm, cudaStream_t s, const RadixArgs &ra) {
  if (items == 8) {
    if (vals) k_radix_down<true, 8><<<G, kRThreads, dsm, s>>>(ra);
    else k_radix_down<false, 8><<<G, kRThreads, dsm, s>>>(ra);
  } else {
    if (vals) k_radix_down<true, 16><<<G, kRThreads, dsm, s>>>(ra);
    else k_radix_down<false, 16><<<G, kRThreads, dsm, s>>>(ra);
  }
}

cudaError_t run_radix(const DevWork &w, const Problem &pb, cudaStream_t s, uint32_t *launches, StepEvents *ev) {
  const uint64_t m = w.m;
  const uint32_t n = w.n;  // columns: the keys
  const bool vals = pb.vals != nullptr;
  uint32_t nl = 0;
  cudaError_t err;
  const uint32_t bits = key_bits_of(n);
  const uint32_t passes = (bits + w.r_dcap - 1) / w.r_dcap;
  const uint32_t dbits = (bits + passes - 1) / passes;
  const uint32_t items = w.r_items;
  // buffers: A = (a_key, a_u, a_w); B = (b_key, row_idx, vals_out).  Pass p
  // writes B when (passes - p) is even, so the last pass writes the outputs.
  // Weighted bulk passes keep (source, value) pairs interleaved, in the a_u
  // block (2 round_up(m, 4) words) and in r_b_sv, except in the last pass's
  // outputs: one 8-byte store per edge instead of two 4-byte ones, and one
  // bulk copy per tile for the pair.
  uint32_t *b_u = pb.row_idx, *b_w = (uint32_t *)pb.vals_out;
  // bulk-staged downsweep: every array a pass reads must be 16-byte aligned
  auto al16 = [](const void *p) { return p == nullptr || (((uintptr_t)p) & 15u) == 0; };
  const bool bulk = w.r_bulk && al16(pb.col_idx) && al16(pb.vals) && al16(b_u) && al16(b_w) && al16(w.r_a_key) &&
                    al16(w.r_a_u) && al16(w.r_a_w) && al16(w.r_b_key) && al16(w.r_b_sv);
  const uint32_t tile = bulk ? kBTile : kRThreads * items;
  const uint32_t ntiles = (uint32_t)((m + tile - 1) / tile);
  const uint32_t G = bulk ? (uint32_t)w.num_sms * kBCtasPerSm : w.rG;
  const uint32_t sub = bulk ? 2u : 1u;
  const uint32_t tpc = (ntiles + G - 1) / G;
  const bool first_to_b = ((passes - 1) % 2) == 0;
  // source rows of the first pass go to the buffer the first pass does not write
  uint32_t *src_rows = first_to_b ? w.r_a_u : b_u;
  {  // source of every edge: rows [0, n_rows)
    uint64_t warps = ((uint64_t)w.n_rows + 31) / 32;
    uint32_t g = (uint32_t)min64((warps + 7) / 8, (uint64_t)w.num_sms * 16);
    if (g == 0) g = 1;
    const uint32_t long_cap = (uint32_t)(m / (kLongRow + 1) + 1);
    k_expand_rows<<<g, 256, 0, s>>>(pb.row_ptr, w.n_rows, m, src_rows, w.r_long, w.r_nlong, long_cap, w.status);
    k_expand_long<<<w.num_sms * 4, 256, 0, s>>>(pb.row_ptr, w.r_long, w.r_nlong, long_cap, src_rows);
    nl += 2;
  }
  if (m == 0) {  // the expansion only validated row_ptr
    if (pb.inputs_read && (err = cudaEventRecord(pb.inputs_read, s)) != cudaSuccess) return err;
    if (launches) *launches += nl;
    return cudaGetLastError();
  }
  const uint32_t *in_key = pb.col_idx, *in_u = src_rows, *in_w = (const uint32_t *)pb.vals;
  const bool sv = bulk && vals;
  bool in_sv = false;
  for (uint32_t p = 1; p <= passes; ++p) {
    const bool toB = ((passes - p) % 2) == 0;
    // interleaved pairs everywhere but the last pass's outputs (B's middle
    // passes use their own pair buffer)
    const bool out_sv = sv && p < passes && (!toB || w.r_b_sv);
    uint32_t *ok = toB ? w.r_b_key : w.r_a_key, *ou = toB ? b_u : w.r_a_u, *ow = toB ? b_w : w.r_a_w;
    if (out_sv && toB) {
      ou = w.r_b_sv;
      ow = nullptr;
    }
    RadixArgs ra{pb.row_ptr, pb.col_idx, pb.vals, n, m, in_key, in_u, in_w, ok, ou, ow,
                 (p - 1) * dbits, dbits, ntiles, tpc, tile, w.r_table, w.r_offsets, w.status, BatchView{}, sub};
    if (p == 1) k_radix_up<true, kPlain><<<G * sub, kRThreads, 0, s>>>(ra);
    else k_radix_up<false, kPlain><<<G * sub, kRThreads, 0, s>>>(ra);
    k_radix_offsets<<<1, 1024, 0, s>>>(w.r_table, G * sub, w.r_offsets);
    if (ev && ev->ndown + 2 <= 8) cudaEventRecord(ev->down[ev->ndown], s);
    if (bulk) {
      const size_t dsm = bulk_dyn_smem(vals);
      if (!vals) k_radix_down_bulk<false, kPlain><<<G, kBThreads, dsm, s>>>(ra);
      else if (in_sv && out_sv) k_radix_down_bulk<true, kPlain, true, true><<<G, kBThreads, dsm, s>>>(ra);
      else if (in_sv) k_radix_down_bulk<true, kPlain, true, false><<<G, kBThreads, dsm, s>>>(ra);
      else if (out_sv) k_radix_down_bulk<true, kPlain, false, true><<<G, kBThreads, dsm, s>>>(ra);
      else k_radix_down_bulk<true, kPlain><<<G, kBThreads, dsm, s>>>(ra);
    } else {
      const size_t dsm = (size_t)tile * 4 * (vals ? 3 : 2);
      launch_down(vals, items, G, dsm, s, ra);
    }
    if (ev && ev->ndown + 2 <= 8) {
      cudaEventRecord(ev->down[ev->ndown + 1], s);
      ev->ndown += 2;
    }
    nl += 3;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // the first pass was the last to read col_idx and vals (row_ptr: the expansion)
    if (p == 1 && pb.inputs_read && (err = cudaEventRecord(pb.inputs_read, s)) != cudaSuccess) return err;
    in_key = ok;
    in_u = ou;
    in_w = ow;
    in_sv = out_sv;
  }
  uint32_t g = (uint32_t)min64((m + 255) / 256, (uint64_t)w.num_sms * 16);
  k_radix_colptr<false><<<g, 256, 0, s>>>(w.r_b_key, m, n, pb.col_ptr, w.r_gaps, w.r_gap_cap, w.status, BatchView{});
  k_radix_gaps<<<w.num_sms * 4, 256, 0, s>>>(w.r_gaps, w.r_gap_cap, pb.col_ptr);
  nl += 2;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// Partitioned HLH: the destination-range bucketing of the two-level form.
// One digit pass of the radix method on the top part_bits bits of the
// destination, from the CSR (destinations, expanded sources, values) into
// the bucketed arrays; being a stable counting sort on those bits, it keeps
// every bucket in CSR order.
cudaError_t run_partition(const DevWork &w, const Problem &pb, cudaStream_t s, uint32_t *launches) {
  const uint64_t m = w.m;
  const bool vals = pb.vals != nullptr;
  uint32_t nl = 0;
  const uint32_t bits = key_bits_of(w.n);
  const uint32_t dbits = w.part_bits < bits ? w.part_bits : bits;
  {  // source of every edge: rows [0, n_rows)
    uint64_t warps = ((uint64_t)w.n_rows + 31) / 32;
    uint32_t g = (uint32_t)min64((warps + 7) / 8, (uint64_t)w.num_sms * 16);
    if (g == 0) g = 1;
    const uint32_t long_cap = (uint32_t)(m / (kLongRow + 1) + 1);
    k_expand_rows<<<g, 256, 0, s>>>(pb.row_ptr, w.n_rows, m, w.r_a_u, w.r_long, w.r_nlong, long_cap, w.status);
    k_expand_long<<<w.num_sms * 4, 256, 0, s>>>(pb.row_ptr, w.r_long, w.r_nlong, long_cap, w.r_a_u);
    nl += 2;
  }
  auto al16 = [](const void *p) { return p == nullptr || (((uintptr_t)p) & 15u) == 0; };
  const bool bulk = al16(pb.col_idx) && al16(pb.vals);  // the plan's own arrays come from cudaMalloc
  const uint32_t tile = bulk ? kBTile : kRThreads * 16u;
  const uint32_t ntiles = (uint32_t)((m + tile - 1) / tile);
  const uint32_t G = (uint32_t)w.num_sms * 2u;  // the digit tables hold num_sms * 8 rows
  const uint32_t sub = bulk ? 2u : 1u;
  const uint32_t tpc = (ntiles + G - 1) / G;
  RadixArgs ra{pb.row_ptr, pb.col_idx, pb.vals, w.n, m, pb.col_idx, w.r_a_u, (const uint32_t *)pb.vals,
               w.q_key, w.q_u, w.q_w, bits - dbits, dbits, ntiles, tpc, tile, w.r_table, w.r_offsets, w.status,
               BatchView{}, sub};
  k_radix_up<true, kPlain><<<G * sub, kRThreads, 0, s>>>(ra);
  k_radix_offsets<<<1, 1024, 0, s>>>(w.r_table, G * sub, w.r_offsets);
  if (bulk) {
    if (vals) k_radix_down_bulk<true, kPlain><<<G, kBThreads, bulk_dyn_smem(true), s>>>(ra);
    else k_radix_down_bulk<false, kPlain><<<G, kBThreads, bulk_dyn_smem(false), s>>>(ra);
  } else {
    launch_down(vals, 16u, G, (size_t)tile * 4 * (vals ? 3 : 2), s, ra);
  }
  nl += 3;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batches (sub-batch of graphs laid out in union edge / vertex spaces)
// ---------------------------------------------------------------------------

// ---- 64-bit vertex IDs -------------------------------------------------------
// The same stable sort of the CSR edge sequence by destination, for matrices
// with more than 2^32 - 1 rows or columns: the 64-bit keys are sorted as two
// 32-bit halves by the digit passes above (low half first, carrying the high
// half and the edge index; then the high half, carrying the index), and the
// sorted edge indices gather the source rows (a search of row_ptr) and the
// values.  col_ptr comes from the sorted keys over the 64-bit column space.

// row_ptr: row_ptr[0] = 0, non-decreasing, row_ptr[n_rows] = m.
__global__ void k64_check_rows(const uint64_t *__restrict__ row_ptr, uint64_t n_rows, uint64_t m, uint32_t *status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (u == 0 && (row_ptr[0] != 0 || row_ptr[n_rows] != m)) set_status(status, GT_ERR_BAD_ROW_PTR);
  bool bad = false;
  for (; u < n_rows; u += stride) bad |= row_ptr[u] > row_ptr[u + 1];
  if (bad) set_status(status, GT_ERR_BAD_ROW_PTR);
}

// Key halves and the identity index; destinations >= n_cols are reported.
__global__ void k64_prepare(const uint64_t *__restrict__ col_idx, uint64_t m, uint64_t n_cols, uint32_t *key_lo,
                            uint32_t *key_hi, uint32_t *idx, uint32_t *status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint64_t v = __ldcs(col_idx + e);
    bad |= v >= n_cols;
    key_lo[e] = (uint32_t)v;
    key_hi[e] = (uint32_t)(v >> 32);
    idx[e] = (uint32_t)e;
  }
  if (bad) set_status(status, GT_ERR_OUT_OF_RANGE);
}

// Slot i of the output takes edge perm[i]: its row (the last row whose
// offset is <= the edge), its value and its destination.
__global__ void k64_gather(const uint64_t *__restrict__ row_ptr, uint64_t n_rows, const uint64_t *__restrict__ col_idx,
                           const float *__restrict__ vals, const uint32_t *__restrict__ perm, uint64_t m,
                           uint64_t *row_idx, float *vals_out, uint64_t *keys) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
    const uint64_t e = perm[i];
    uint64_t lo = 0, hi = n_rows;  // largest u < n_rows with row_ptr[u] <= e
    while (hi - lo > 1) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (row_ptr[mid] <= e) lo = mid;
      else hi = mid;
    }
    row_idx[i] = lo;
    if (vals) vals_out[i] = vals[e];
    keys[i] = col_idx[e];
  }
}

// col_ptr[v] = number of sorted keys < v, for v in [0, n_cols].  One warp per
// chunk of 2048 consecutive entries: the keys that fall in the chunk are found
// by two searches; a chunk without keys is one constant, else every entry
// searches the chunk's keys.
constexpr uint64_t k64Chunk = 2048;

__device__ __forceinline__ uint64_t lower_bound64(const uint64_t *a, uint64_t lo, uint64_t hi, uint64_t x) {
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k64_colptr(const uint64_t *__restrict__ keys, uint64_t m, uint64_t n_cols, uint64_t *col_ptr) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t chunks = (n_cols + 1 + k64Chunk - 1) / k64Chunk;
  for (uint64_t c = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < chunks; c += warps) {
    const uint64_t v0 = c * k64Chunk;
    const uint64_t v1 = v0 + k64Chunk < n_cols + 1 ? v0 + k64Chunk : n_cols + 1;
    uint64_t lo = 0, hi = 0;
    if (lane == 0) {
      lo = lower_bound64(keys, 0, m, v0);
      hi = lower_bound64(keys, lo, m, v1);
    }
    lo = __shfl_sync(kFull, lo, 0);
    hi = __shfl_sync(kFull, hi, 0);
    for (uint64_t v = v0 + lane; v < v1; v += 32) col_ptr[v] = lo == hi ? lo : lower_bound64(keys, lo, hi, v);
  }
}

cudaError_t run_radix_u64(const U64Work &w, cudaStream_t s) {
  cudaError_t err;
  const uint64_t m = w.m;
  const uint32_t g = (uint32_t)w.num_sms * 16;
  k64_check_rows<<<g, 256, 0, s>>>(w.row_ptr, w.n_rows, m, w.status);
  if (m > 0) {
    k64_prepare<<<g, 256, 0, s>>>(w.col_idx, m, w.n_cols, w.a_key, w.a_u, w.a_w, w.status);
    uint32_t bits = 0;
    while (bits < 64 && ((w.n_cols - 1) >> bits)) ++bits;
    if (bits == 0) bits = 1;
    const uint32_t lo_bits = bits < 32 ? bits : 32, hi_bits = bits > 32 ? bits - 32 : 0;
    const uint32_t Gb = (uint32_t)w.num_sms * kBCtasPerSm, sub = 2;
    const uint32_t ntiles = (uint32_t)((m + kBTile - 1) / kBTile), tpc = (ntiles + Gb - 1) / Gb;
    // current arrays: (key half, payload 1, payload 2)
    uint32_t *ck = w.a_key, *cu = w.a_u, *cw = w.a_w, *nk = w.b_key, *nu = w.b_u, *nw = w.b_w;
    auto pass = [&](uint32_t shift, uint32_t dbits, bool three) -> cudaError_t {
      RadixArgs ra{nullptr, nullptr, nullptr, 0, m, ck, cu, three ? cw : nullptr, nk, nu, three ? nw : nullptr,
                   shift, dbits, ntiles, tpc, kBTile, w.table, w.offsets, w.status, BatchView{nullptr, 0}, sub};
      k_radix_up<false, kPlain><<<Gb * sub, kRThreads, 0, s>>>(ra);
      k_radix_offsets<<<1, 1024, 0, s>>>(w.table, Gb * sub, w.offsets);
      if (three) k_radix_down_bulk<true, kPlain><<<Gb, kBThreads, bulk_dyn_smem(true), s>>>(ra);
      else k_radix_down_bulk<false, kPlain><<<Gb, kBThreads, bulk_dyn_smem(false), s>>>(ra);
      std::swap(ck, nk);
      std::swap(cu, nu);
      std::swap(cw, nw);
      return cudaGetLastError();
    };
    // low half: key = low 32 bits, carrying (high half, index)
    const uint32_t pa = (lo_bits + 7) / 8, da = (lo_bits + pa - 1) / pa;
    for (uint32_t p = 0; p < pa; ++p)
      if ((err = pass(p * da, da, true)) != cudaSuccess) return err;
    // high half: key = the carried high half, carrying the index
    const uint32_t *perm = cw;
    if (hi_bits) {
      ck = cu;   // the high halves become the keys
      cu = cw;   // the indices the payload
      nk = nu;   // free arrays of the other set
      nu = nw;
      const uint32_t pb = (hi_bits + 7) / 8, db = (hi_bits + pb - 1) / pb;
      for (uint32_t p = 0; p < pb; ++p)
        if ((err = pass(p * db, db, false)) != cudaSuccess) return err;
      perm = cu;
    }
    k64_gather<<<g, 256, 0, s>>>(w.row_ptr, w.n_rows, w.col_idx, w.vals, perm, m, w.row_idx, w.vals_out, w.keys);
  }
  k64_colptr<<<g, 256, 0, s>>>(w.keys, m, w.n_cols, w.col_ptr);
  return cudaGetLastError();
}

// ---- layout of one batch call (device-side, read by every later kernel) ----

// The call's arguments, stored where the captured kernels read them.
__global__ void k_b_set_call(BatchCall *call, const gt_graph_desc *descs, int32_t *status, uint32_t n_graphs) {
  call->descs = descs;
  call->status = status;
  call->n_graphs = n_graphs;
}

// One CTA of kLayoutThreads threads.  Per graph: the descriptor's checks
// (an excluded graph gets its status code and no edges, columns or rows),
// then exclusive prefix sums of the edges, columns and 32-row windows over
// the graphs in order, the exclusion of every graph from the first one whose
// prefix end passes a limit of the plan, and the sub-batch of every graph:
// slot(g) = floor(eoff[g] / cap_e) + floor(voff[g] / cap_v) + floor(g / cap_g),
// non-decreasing in g, so each sub-batch is a run of graphs with at most
// cap_e + max graph edges edges, cap_v + max columns columns and cap_g graphs.
constexpr uint32_t kLayoutThreads = 1024;

__global__ void __launch_bounds__(kLayoutThreads) k_b_layout(const BatchCall *__restrict__ call, BatchLimitsDev lim,
                                                             unsigned long long *eoff, unsigned long long *voff,
                                                             unsigned long long *woff, uint32_t *gx, BatchSlot *slots,
                                                             BatchTotals *totals, uint32_t *status) {
  __shared__ unsigned long long s_e[kLayoutThreads], s_v[kLayoutThreads], s_w[kLayoutThreads];
  __shared__ uint32_t s_cut;
  const uint32_t tid = threadIdx.x;
  const uint32_t n = min(call->n_graphs, lim.max_graphs);
  const gt_graph_desc *descs = call->descs;
  int32_t *gst = call->status;
  if (tid == 0) s_cut = n;
  const uint32_t per = (n + kLayoutThreads - 1) / kLayoutThreads;
  const uint32_t g0 = min(tid * per, n), g1 = min(g0 + per, n);
  // checks and chunk sums
  unsigned long long se = 0, sv = 0, sw = 0;
  for (uint32_t g = g0; g < g1; ++g) {
    const gt_graph_desc d = descs[g];
    gt_status code = GT_OK;
    const uint32_t cols = desc_cols(d);
    if (d.n_vertices == 0 || !d.row_ptr || !d.col_ptr || (d.n_edges > 0 && (!d.col_idx || !d.row_idx)))
      code = GT_ERR_INVALID_ARG;
    else if (lim.has_vals && d.n_edges > 0 && (!d.vals || !d.vals_out))
      code = GT_ERR_INVALID_ARG;
    else if (!lim.has_vals && (d.vals || d.vals_out))
      code = GT_ERR_INVALID_ARG;
    else if (cols > lim.max_cols || d.n_edges > lim.max_graph_edges)
      code = GT_ERR_UNSUPPORTED;
    if (gst) gst[g] = (int32_t)code;
    gx[g] = code != GT_OK;
    if (code != GT_OK) {
      set_status(status, code);
      continue;
    }
    se += d.n_edges;
    sv += cols;
    sw += (d.n_vertices + 31u) / 32u;
  }
  s_e[tid] = se, s_v[tid] = sv, s_w[tid] = sw;
  __syncthreads();
  for (uint32_t o = 1; o < kLayoutThreads; o <<= 1) {  // inclusive scans over the chunks
    unsigned long long ye = 0, yv = 0, yw = 0;
    if (tid >= o) ye = s_e[tid - o], yv = s_v[tid - o], yw = s_w[tid - o];
    __syncthreads();
    s_e[tid] += ye, s_v[tid] += yv, s_w[tid] += yw;
    __syncthreads();
  }
  unsigned long long re = tid ? s_e[tid - 1] : 0, rv = tid ? s_v[tid - 1] : 0, rw = tid ? s_w[tid - 1] : 0;
  for (uint32_t g = g0; g < g1; ++g) {
    eoff[g] = re, voff[g] = rv, woff[g] = rw;
    if (!gx[g]) {
      const gt_graph_desc &d = descs[g];
      re += d.n_edges;
      rv += desc_cols(d);
      rw += (d.n_vertices + 31u) / 32u;
      if (re > lim.max_edges || rv > lim.max_cols_total) atomicMin(&s_cut, g);
    }
  }
  __syncthreads();
  // graphs from the first one past a limit on are excluded (their prefix ends only grow)
  const uint32_t cut = s_cut;
  for (uint32_t g = max(g0, cut); g < g1; ++g) {
    if (!gx[g]) {
      if (gst) gst[g] = GT_ERR_UNSUPPORTED;
      set_status(status, GT_ERR_UNSUPPORTED);
    }
    gx[g] = 1;
    eoff[g] = eoff[cut], voff[g] = voff[cut], woff[g] = woff[cut];  // eoff[cut] is never rewritten
  }
  if (tid == kLayoutThreads - 1) {
    const uint32_t last = n;
    if (cut < n) {
      eoff[last] = eoff[cut], voff[last] = voff[cut], woff[last] = woff[cut];
    } else {
      eoff[last] = s_e[tid], voff[last] = s_v[tid], woff[last] = s_w[tid];
    }
  }
  __syncthreads();
  // sub-batches: slot s holds graphs [first(s), first(s + 1)) with
  // first(s) = the first graph whose slot is >= s (n if none)
  auto slot_of = [&](uint32_t g) -> unsigned long long {
    return eoff[g] / lim.cap_e + voff[g] / lim.cap_v + g / lim.cap_g;
  };
  auto first = [&](uint32_t sidx) -> uint32_t {
    uint32_t lo = 0, hi = n;  // first g in [0, n) with slot_of(g) >= sidx, else n
    while (lo < hi) {
      const uint32_t mid = (lo + hi) / 2;
      if (slot_of(mid) >= sidx) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  };
  for (uint32_t sidx = tid; sidx < lim.slots; sidx += kLayoutThreads) {
    const uint32_t a = first(sidx), b = first(sidx + 1);
    BatchSlot sl;
    sl.descs = descs + a;
    sl.gstatus = gst ? gst + a : nullptr;
    sl.gx = gx + a;
    sl.eoff = eoff + a, sl.voff = voff + a, sl.woff = woff + a;
    sl.e0 = eoff[a], sl.v0 = voff[a], sl.w0 = woff[a];
    sl.m = eoff[b] - eoff[a], sl.nv = voff[b] - voff[a], sl.windows = woff[b] - woff[a];
    sl.g0 = a, sl.ng = b - a;
    slots[sidx] = sl;
  }
  // graphs past the last sub-batch (not reachable within the plan's limits)
  const uint32_t tail = first(lim.slots);
  for (uint32_t g = max(tail, g0); g < g1; ++g)
    if (!gx[g]) {
      gx[g] = 1;
      if (gst) gst[g] = GT_ERR_UNSUPPORTED;
      set_status(status, GT_ERR_UNSUPPORTED);
    }
  if (tid == 0) {
    totals->n_graphs = n;
    totals->n_edges = eoff[min(tail, n)];
    uint32_t used = 0;
    for (uint32_t sidx = 0; sidx < lim.slots; ++sidx) used += first(sidx + 1) > first(sidx);
    totals->slots_used = used;
  }
}

// Per graph: row_ptr[0] == 0 and row_ptr[n_rows] == m (n_vertices is the row count).
__global__ void k_b_check(BatchView bv, uint32_t *status) {
  const BatchSlot &sl = *bv.slot;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < sl.ng; g += gridDim.x * blockDim.x) {
    if (sl.gx[g]) continue;
    const gt_graph_desc &d = sl.descs[g];
    if (d.row_ptr[0] != 0 || d.row_ptr[d.n_vertices] != d.n_edges) graph_error(sl, g, status, GT_ERR_BAD_ROW_PTR);
  }
}

// Source rows of every union edge: windows of 32 rows of one graph per warp step.
__global__ void k_b_expand(BatchView bv, uint32_t *src, uint32_t *long_g, uint32_t *long_r, uint32_t *n_long,
                           uint32_t long_cap, uint32_t *status) {
  const BatchSlot &sl = *bv.slot;
  const uint64_t windows = sl.windows;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t wi = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); wi < windows; wi += warps) {
    const uint32_t g = upper_graph(sl.woff, sl.ng, sl.w0 + wi);
    const gt_graph_desc &d = sl.descs[g];
    const uint32_t n = d.n_vertices;  // rows
    const uint64_t m = d.n_edges, base = sl.eoff[g] - sl.e0;
    const uint64_t r0 = (sl.w0 + wi - sl.woff[g]) * 32;
    const uint64_t r = r0 + lane;
    uint64_t ri = r + 1;
    if (ri > n) ri = n;
    uint64_t rend = d.row_ptr[ri];
    uint64_t rbeg = r < n ? d.row_ptr[r] : rend;
    if (rend > m || rbeg > rend) {
      graph_error(sl, g, status, GT_ERR_BAD_ROW_PTR);
      rend = rbeg = 0;
    }
    const bool is_long = r < n && rend - rbeg > kLongRow;
    if (is_long) {
      uint32_t i = atomicAdd(n_long, 1u);
      if (i < long_cap) {
        long_g[i] = g;
        long_r[i] = (uint32_t)r;
      } else {
        set_status(status, GT_ERR_UNSUPPORTED);
      }
    }
    const uint32_t longmask = __ballot_sync(kFull, is_long);
    const uint64_t b = __shfl_sync(kFull, rbeg, 0);
    const uint64_t e = __shfl_sync(kFull, rend, 31);
    const bool sane = __all_sync(kFull, !(rend > m || rbeg > rend)) && e >= b;
    if (longmask == 0 && sane) {  // at most 32 x kLongRow edges: offsets from b fit 32 bits
      const uint32_t rrel = (uint32_t)(rend - b);
      for (uint64_t p0 = b; p0 < e; p0 += 32) {
        const uint64_t p = p0 + lane;
        const uint32_t pos = count_le32(rrel, (uint32_t)(p - b));  // warp-collective
        if (p < e) src[base + p] = (uint32_t)(r0 + pos);
      }
    } else {
      uint32_t todo = __ballot_sync(kFull, r < n && !is_long && rend > rbeg);
      while (todo) {
        const uint32_t j = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint64_t qb = __shfl_sync(kFull, rbeg, j), qe = __shfl_sync(kFull, rend, j);
        for (uint64_t p = qb + lane; p < qe; p += 32) src[base + p] = (uint32_t)(r0 + j);
      }
    }
  }
}

__global__ void k_b_expand_long(BatchView bv, const uint32_t *__restrict__ long_g, const uint32_t *__restrict__ long_r,
                                const uint32_t *__restrict__ n_long, uint32_t long_cap, uint32_t *src) {
  const BatchSlot &sl = *bv.slot;
  const uint32_t cnt = min(*n_long, long_cap);
  for (uint32_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const uint32_t g = long_g[i], r = long_r[i];
    const gt_graph_desc &d = sl.descs[g];
    const uint64_t b = d.row_ptr[r], e = d.row_ptr[r + 1], base = sl.eoff[g] - sl.e0;
    for (uint64_t p = b + threadIdx.x; p < e; p += blockDim.x) src[base + p] = r;
  }
}

// A sub-batch without edges: its union col_ptr is all zero.
__global__ void k_b_zero_ucp(BatchView bv, unsigned long long *ucp) {
  const BatchSlot &sl = *bv.slot;
  if (sl.m != 0) return;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x <= sl.nv; x += (uint64_t)gridDim.x * blockDim.x)
    ucp[x] = 0;
}

// col_ptr of every graph from the union col_ptr (and the last entry).
__global__ void k_b_colptr(BatchView bv, const unsigned long long *__restrict__ ucp) {
  const BatchSlot &sl = *bv.slot;
  const uint64_t nv = sl.nv;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < nv + sl.ng;
       x += (uint64_t)gridDim.x * blockDim.x) {
    if (x < nv) {
      const uint32_t g = upper_graph(sl.voff, sl.ng, sl.v0 + x);
      sl.descs[g].col_ptr[sl.v0 + x - sl.voff[g]] = ucp[x] - (sl.eoff[g] - sl.e0);
    } else {
      const uint32_t g = (uint32_t)(x - nv);
      if (sl.gx[g]) continue;
      const gt_graph_desc &d = sl.descs[g];
      d.col_ptr[desc_cols(d)] = d.n_edges;
    }
  }
}

cudaError_t launch_batch_layout(const BatchWork &bw, cudaStream_t s) {
  k_b_layout<<<1, kLayoutThreads, 0, s>>>(bw.call, bw.lim, bw.eoff, bw.voff, bw.woff, bw.gx, bw.slots, bw.totals,
                                          bw.status);
  return cudaGetLastError();
}

cudaError_t launch_batch_call(BatchCall *call, const gt_graph_desc *descs, int32_t *status, uint32_t n_graphs,
                              cudaStream_t s) {
  k_b_set_call<<<1, 1, 0, s>>>(call, descs, status, n_graphs);
  return cudaGetLastError();
}

// The kernels of sub-batch `slot` (its sizes are read on the device).
cudaError_t run_radix_batch(const BatchWork &bw, uint32_t slot, cudaStream_t s, uint32_t *launches) {
  uint32_t nl = 0;
  cudaError_t err;
  BatchView bv{bw.slots + slot, bw.vbits};
  const bool vals = bw.has_vals != 0;
  const uint64_t M = bw.cap_edges;  // sizes the grids; the kernels read this call's sizes
  const uint32_t passes = bw.passes, dbits = bw.dbits;
  if ((err = cudaMemsetAsync(bw.n_long, 0, 4, s)) != cudaSuccess) return err;
  const uint32_t gchk = (bw.lim.cap_g + 255) / 256;
  k_b_check<<<gchk < 1024 ? gchk : 1024, 256, 0, s>>>(bv, bw.status);
  ++nl;
  const bool first_to_b = ((passes - 1) % 2) == 0;
  uint32_t *src_rows = first_to_b ? bw.a_u : bw.b_u;
  k_b_expand<<<(uint32_t)bw.num_sms * 16, 256, 0, s>>>(bv, src_rows, bw.long_g, bw.long_r, bw.n_long, bw.long_cap,
                                                       bw.status);
  k_b_expand_long<<<bw.num_sms * 4, 256, 0, s>>>(bv, bw.long_g, bw.long_r, bw.n_long, bw.long_cap, src_rows);
  nl += 2;
  // The first upsweep reads through the descriptors and gathers the union
  // keys and values into the buffers the first pass does not write; every
  // pass then runs the bulk-staged downsweep on plain arrays, the last one
  // storing through the descriptors.
  const uint32_t Gb = (uint32_t)bw.num_sms * kBCtasPerSm, subb = 2;
  const uint32_t ntb = (uint32_t)((M + kBTile - 1) / kBTile), tpcb = (ntb + Gb - 1) / Gb;
  uint32_t *gk = first_to_b ? bw.a_key : bw.b_key, *gw = vals ? (first_to_b ? bw.a_w : bw.b_w) : nullptr;
  const uint32_t *in_key = gk, *in_u = src_rows, *in_w = gw;
  // weighted: the passes between the first and the last keep (source,
  // value) pairs interleaved on both sides
  bool in_sv = false;
  for (uint32_t p = 1; p <= passes; ++p) {
    const bool toB = ((passes - p) % 2) == 0;
    const bool out_sv = vals && p < passes;
    uint32_t *ok = toB ? bw.b_key : bw.a_key, *ou = toB ? bw.b_u : bw.a_u, *ow = toB ? bw.b_w : bw.a_w;
    RadixArgs ra{nullptr, nullptr, nullptr, 0, M, in_key, in_u, in_w, ok, ou, ow,
                 (p - 1) * dbits, dbits, ntb, tpcb, kBTile, bw.table, bw.offsets, bw.status, bv, subb,
                 p == 1 ? gk : nullptr, p == 1 ? gw : nullptr};
    const uint32_t rows = Gb * subb;
    if (p == 1) k_radix_up<true, kBatchFirst><<<rows, kRThreads, 0, s>>>(ra);
    else k_radix_up<false, kPlain><<<rows, kRThreads, 0, s>>>(ra);
    k_radix_offsets<<<1, 1024, 0, s>>>(bw.table, rows, bw.offsets);
    const size_t dsm = bulk_dyn_smem(vals);
    if (p == passes && vals && in_sv) k_radix_down_bulk<true, kBatchLast, true, false><<<Gb, kBThreads, dsm, s>>>(ra);
    else if (p == passes && vals) k_radix_down_bulk<true, kBatchLast><<<Gb, kBThreads, dsm, s>>>(ra);
    else if (p == passes) k_radix_down_bulk<false, kBatchLast><<<Gb, kBThreads, dsm, s>>>(ra);
    else if (vals && in_sv) k_radix_down_bulk<true, kPlain, true, true><<<Gb, kBThreads, dsm, s>>>(ra);
    else if (vals) k_radix_down_bulk<true, kPlain, false, true><<<Gb, kBThreads, dsm, s>>>(ra);
    else k_radix_down_bulk<false, kPlain><<<Gb, kBThreads, dsm, s>>>(ra);
    nl += 3;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    in_key = ok;
    in_u = ou;
    in_w = ow;
    in_sv = out_sv;
  }
  // union col_ptr straight from the sorted keys (compact column space)
  const uint32_t gr = (uint32_t)min64((M + 255) / 256, (uint64_t)bw.num_sms * 16);
  if ((err = cudaMemsetAsync(bw.gaps, 0, 8, s)) != cudaSuccess) return err;
  k_b_zero_ucp<<<bw.num_sms * 4, 256, 0, s>>>(bv, bw.ucp);
  k_radix_colptr<true><<<gr ? gr : 1, 256, 0, s>>>(bw.b_key, M, 0, (uint64_t *)bw.ucp, bw.gaps, bw.gap_cap, bw.status,
                                                   bv);
  k_radix_gaps<<<bw.num_sms * 4, 256, 0, s>>>(bw.gaps, bw.gap_cap, (uint64_t *)bw.ucp);
  k_b_colptr<<<(uint32_t)bw.num_sms * 16, 256, 0, s>>>(bv, bw.ucp);
  nl += 4;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

}  // namespace gt
