// gt_transpose_noalloc: the transposition with its workspace carved from a
// fixed array that is part of the library image, so the call itself never
// allocates device memory.
//
// Who needs this: programs that must not allocate on the call path -- for
// example a host application whose memory pool has reserved all of the
// device memory up front, or a latency-critical loop that cannot accept the
// device-wide synchronisation cudaMalloc/cudaFree may cause.  They pass their
// own input and output arrays; everything else comes from the array below.
//
// Limits and sharing: the array holds kNoAllocBytes (64 MiB) on every GPU
// that loads the library, for the life of the process.  Graphs whose
// workspace does not fit are rejected with GT_ERR_UNSUPPORTED.  All calls on
// a device share the array and it keeps the previous call's contents (the
// counters that must start at zero are cleared by every call); calls that
// overlap on the GPU, from any stream or thread, race on it and give
// undefined results.  The call runs the pure-atomic configuration (no HDV
// table), synchronises `stream` and returns the device status.
//
// Set-up: every call looks up the array's device address on the current
// device (cudaGetSymbolAddress, a host-side lookup that allocates nothing),
// so a new context after cudaDeviceReset, whose module image may sit at
// another address, is never handed a stale pointer.  The first call in each
// CUDA context also sets the kernels' shared-memory limits (kept per context
// by its unique ID); make that first call before any stream capture on the
// device.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include "gt.h"
#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {
cudaError_t configure_steps();
cudaError_t configure_sort();
}  // namespace gt

namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Unique ID of the CUDA context in which the kernels' limits were last set,
// per device ordinal (0 = never).
std::atomic<unsigned long long> g_configured_ctx[kMaxDevices];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Unique ID of the current context through the driver's cuCtxGetCurrent and
// cuCtxGetId (looked up once, without linking the driver library); 0 when
// either is unavailable, which makes every call set the limits again.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::atomic<int> looked_up{0};
  if (!looked_up.load()) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = (CtxGetCurrentFn)f1;
      get_id = (CtxGetIdFn)f2;
    }
    cudaGetLastError();
    looked_up.store(1);
  }
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Enqueued work may still use the shared array: wait for it before an error
// return, so that the caller's next call cannot overlap it unknowingly.
gt_status fail_after_enqueue(cudaStream_t s, cudaError_t e) {
  gt_status st = gt::from_cuda(e);
  cudaGetLastError();
  cudaStreamSynchronize(s);
  cudaGetLastError();
  return st;
}

}  // namespace

extern "C" gt_status gt_transpose_noalloc(uint32_t n_vertices, uint64_t n_edges, const uint64_t *row_ptr,
                                          const uint32_t *col_idx, const float *vals, uint64_t *col_ptr,
                                          uint32_t *row_idx, float *vals_out, void *stream) {
  if (!row_ptr || !col_ptr) return GT_ERR_INVALID_ARG;
  if (n_edges > 0 && (!col_idx || !row_idx)) return GT_ERR_INVALID_ARG;
  if ((vals == nullptr) != (vals_out == nullptr)) return GT_ERR_INVALID_ARG;
  if (n_vertices == 0 && n_edges != 0) return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    gt_status st = ce != cudaSuccess ? gt::from_cuda(ce) : GT_ERR_UNSUPPORTED;
    cudaGetLastError();
    return st;
  }
  // the device address of the static array in the current context
  void *base = nullptr;
  if ((ce = cudaGetSymbolAddress(&base, g_noalloc_scratch)) != cudaSuccess || !base) {
    gt_status st = gt::from_cuda(ce != cudaSuccess ? ce : cudaErrorInvalidSymbol);
    cudaGetLastError();
    return st;
  }
  // the kernels' shared-memory limits, once per context
  const unsigned long long ctx = current_context_id();
  if (ctx == 0 || g_configured_ctx[dev].load() != ctx) {
    if ((ce = gt::configure_steps()) != cudaSuccess || (ce = gt::configure_sort()) != cudaSuccess) {
      gt_status st = gt::from_cuda(ce);
      cudaGetLastError();
      return st;
    }
    g_configured_ctx[dev].store(ctx);
  }
  if (n_vertices == 0) {
    if ((ce = cudaMemsetAsync(col_ptr, 0, 8, s)) != cudaSuccess) return fail_after_enqueue(s, ce);
    return gt::from_cuda(cudaStreamSynchronize(s));
  }

  // launch shape: 256-thread CTAs, 4 per SM, partitions of >= 4096 edges per warp
  int sms = 0;
  if ((ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
    gt_status st = gt::from_cuda(ce);
    cudaGetLastError();
    return st;
  }
  gt_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.block_threads = 256;
  cfg.ctas_per_sm = 4;
  cfg.warp_edges = 4096;
  cfg.sample_permille = 10;
  cfg.flags = GT_FLAG_AGGREGATE;
  gt::DevWork w;
  w.n = n_vertices;
  w.n_rows = n_vertices;
  w.m = n_edges;
  w.has_vals = vals ? 1 : 0;
  w.num_sms = sms;
  w.kmax = 0;
  w.tlog2 = 0;
  w.W = cfg.block_threads / 32;
  uint64_t want = (n_edges + (uint64_t)w.W * cfg.warp_edges - 1) / ((uint64_t)w.W * cfg.warp_edges);
  uint64_t cap = (uint64_t)sms * cfg.ctas_per_sm;
  if (want < 1) want = 1;
  if (want > cap) want = cap;
  w.G = (uint32_t)want;
  w.P = w.G * w.W;
  w.psize = n_edges ? (n_edges + w.P - 1) / w.P : 1;
  w.staged = 0;
  w.stage_edges = 0;
  w.smem_count = gt::smem_count_bytes(w.W, 0, 0, 0, 0, w.has_vals);
  w.smem_scatter = gt::smem_scatter_bytes(w.W, 0, 0, 0, 0, w.has_vals);
  w.ns = 0;
  w.ts_log2 = 10;
  w.ntiles = (uint32_t)((n_vertices + gt::kScanTile - 1) / gt::kScanTile);
  w.big_cap = (uint32_t)gt::worklist_entries(n_edges);
  w.flag_mode = (w.has_vals && n_vertices <= 0x80000000u) ? 1 : 0;

  // carve the workspace out of the static array
  const size_t n = n_vertices, m = n_edges;
  size_t off = 0;
  unsigned char *b = (unsigned char *)base;
  auto take = [&](size_t bytes) -> void * {
    void *p = b + off;
    off += align256(bytes ? bytes : 16);
    return p;
  };
  w.deg = (uint32_t *)take(n * 4);
  w.cursor = (unsigned long long *)take(n * 8);
  w.hdv_cnt = (uint32_t *)take(16);
  w.hdv_ids = (uint32_t *)take(16);
  w.hdv_start = (unsigned long long *)take(16);
  w.hkeys = (uint32_t *)take(16);
  w.hvals = (uint16_t *)take(16);
  w.part = (unsigned long long *)take(((size_t)w.P + 1) * 8);
  w.scan_state = (unsigned long long *)take((size_t)w.ntiles * 8);
  w.status = (uint32_t *)take(4);
  w.meta = (uint32_t *)take(gt::kMetaCount * 4);
  w.meta64 = (unsigned long long *)take(32);
  w.skeys = (uint32_t *)take(16);
  w.scnt = (uint32_t *)take(16);
  w.fhist = (uint32_t *)take(16);
  w.cand = (uint32_t *)take(16);
  w.ties = (uint32_t *)take(16);
  w.biglist = (uint32_t *)take((size_t)w.big_cap * 4);
  w.scratch = take(m * (vals ? 8 : 4));
  if (off > kNoAllocBytes) return GT_ERR_UNSUPPORTED;  // graph too large for the fixed scratch

  gt::Problem pb{row_ptr, col_idx, vals, col_ptr, row_idx, vals_out};
  uint32_t launches = 0;
  if ((ce = gt::run_transpose(w, cfg, pb, s, nullptr, &launches)) != cudaSuccess) return fail_after_enqueue(s, ce);
  // the device status word, read on the same stream: one host wait
  uint32_t st = 0;
  if ((ce = cudaMemcpyAsync(&st, w.status, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail_after_enqueue(s, ce);
  if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) {
    gt_status e = gt::from_cuda(ce);
    cudaGetLastError();
    return e;
  }
  return (gt_status)st;
}
