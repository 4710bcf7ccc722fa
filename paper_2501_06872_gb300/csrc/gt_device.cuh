// Device-side helpers shared by the graph-transposition kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gt.h"

namespace gt {

constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;  // never a vertex ID (n <= 2^32 - 1)
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kMaxHdv = 4096;                // compact HDV index fits 12 bits
constexpr int kMaxTableLog2 = 13;            // hash table of at most 8192 slots
constexpr uint32_t kSplitFlag = 0x80000000u; // marks split-row LDV entries in row_idx (n <= 2^31 only)

// Indices into the per-plan u32 "meta" block.
enum MetaIdx : int {
  kMetaK = 0,        // HDV selected by Step 0
  kMetaThr = 1,      // sample-frequency threshold
  kMetaNeed = 2,     // ties to take at threshold-1
  kMetaNCand = 3,    // candidates with frequency >= threshold
  kMetaNTie = 4,     // tie candidates collected
  kMetaBig = 5,      // LDV lists longer than one warp (sort worklist length)
  kMetaTicket = 6,   // work ticket of the big-list sort
  kMetaSorted = 7,   // LDV lists of length >= 2 that were sorted
  kMetaLarge = 8,    // of those, handled by the radix path
  kMetaScanTicket = 9,
  kMetaMid = 10,         // lists for the warp sort
  kMetaMidTicket = 11,
  kMetaLargeN = 12,      // lists for the radix sort
  kMetaLargeTicket = 13,
  kMetaCount = 16
};

// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum
// minus the kernel's own static shared memory.
template <typename F>
inline cudaError_t allow_max_dynamic_smem(F *func) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, (const void *)func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute((const void *)func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

// Bounded spin: iterations before a device-side wait gives up (GT_ERR_TIMEOUT).
constexpr uint32_t kSpinLimit = 1u << 24;

__host__ __device__ __forceinline__ uint64_t min64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint64_t max64(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ void set_status(uint32_t *status, gt_status code) {
  atomicCAS(status, 0u, (uint32_t)code);
}

// CTA-uniform read of the status word: true if an earlier step reported an
// error (all threads of the CTA get the same answer).
__device__ __forceinline__ bool cta_status_set(const uint32_t *status) {
  __shared__ uint32_t s_status;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_status = *(const volatile uint32_t *)status;
  __syncthreads();
  return s_status != 0u;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

// SplitMix64 output function (Steele, Lea, Flood 2014) -- used only to pick
// sampling positions, which never influence the output bytes.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x;
}

// Multiplicative (Fibonacci) hash of a vertex ID onto 2^log2 slots.
__device__ __forceinline__ uint32_t hash_slot(uint32_t v, uint32_t log2) {
  return (v * 0x9E3779B1u) >> (32u - log2);
}

// Open-addressing lookup (linear probing) in a shared-memory table image:
// returns the compact HDV index, or -1 for an LDV.  The table always keeps at
// least half of its slots empty, so the probe ends.
__device__ __forceinline__ int hdv_lookup(const uint32_t *keys, const uint16_t *vals, uint32_t log2,
                                          uint32_t v) {
  const uint32_t mask = (1u << log2) - 1u;
  uint32_t s = hash_slot(v, log2);
#pragma unroll 1
  for (uint32_t i = 0; i <= mask; ++i) {
    uint32_t k = keys[s];
    if (k == v) return (int)vals[s];
    if (k == kEmptyKey) return -1;
    s = (s + 1u) & mask;
  }
  return -1;
}

// Fire-and-forget global add (no return value needed).
__device__ __forceinline__ void red_add_u32(uint32_t *p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_volatile_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- bulk-copy (TMA engine) staging: mbarrier + cp.async.bulk ------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Waits for the phase with the given parity; gives up after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  uint32_t addr = smem_u32(bar);
#pragma unroll 1
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 1-D bulk copy global -> shared, completion signalled on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---- row search over CSR offsets (shared by the scatter and the radix method) ----

// Number of window entries (row ends, non-decreasing across lanes) <= e.
__device__ __forceinline__ uint32_t count_le(uint64_t rend, uint64_t e) {
  uint32_t pos = 0;
#pragma unroll
  for (uint32_t s = 16; s > 0; s >>= 1) {
    uint64_t x = __shfl_sync(kFull, rend, pos + s - 1);
    if (x <= e) pos += s;
  }
  uint64_t x = __shfl_sync(kFull, rend, pos);
  if (x <= e) pos += 1;
  return pos;  // 0..32
}

// count_le on 32-bit offsets from the window start (windows of short rows
// hold at most 32 x 2048 edges): half the shuffles.
__device__ __forceinline__ uint32_t count_le32(uint32_t rend, uint32_t e) {
  uint32_t pos = 0;
#pragma unroll
  for (uint32_t s = 16; s > 0; s >>= 1) {
    const uint32_t x = __shfl_sync(kFull, rend, pos + s - 1);
    if (x <= e) pos += s;
  }
  const uint32_t x = __shfl_sync(kFull, rend, pos);
  if (x <= e) pos += 1;
  return pos;  // 0..32
}

// Index of the row containing edge e: largest u with row_ptr[u] <= e, searched
// from row base_u on (warp-collective).  One 32-row window covers the dense
// case; sparse stretches are walked 256 rows per round with independent loads.
__device__ __forceinline__ uint32_t find_row(const uint64_t *__restrict__ row_ptr, uint32_t n, uint32_t base_u,
                                             uint64_t e, bool act, uint32_t lane, uint32_t *status) {
  bool found = !act;
  uint32_t my_u = 0;
  uint64_t bu = base_u;
  {
    uint64_t ri = bu + 1 + lane;
    if (ri > n) ri = n;
    uint32_t pos = count_le(row_ptr[ri], e);
    if (!found && pos < 32) {
      my_u = (uint32_t)(bu + pos);
      found = true;
    }
  }
  if (__all_sync(kFull, found)) return my_u;
  bu += 32;
#pragma unroll 1
  while (bu < n) {
    uint64_t r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint64_t ri = bu + 1 + lane + 32u * i;
      if (ri > n) ri = n;
      r[i] = row_ptr[ri];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint32_t pos = count_le(r[i], e);
      if (!found && pos < 32) {
        my_u = (uint32_t)(bu + 32u * i + pos);
        found = true;
      }
    }
    if (__all_sync(kFull, found)) return my_u;
    bu += 256;
  }
  if (!found) {
    set_status(status, GT_ERR_BAD_ROW_PTR);
    my_u = n - 1;
  }
  return my_u;
}

}  // namespace gt
