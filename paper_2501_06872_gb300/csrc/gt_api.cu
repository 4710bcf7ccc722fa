// C ABI of libgt.so: plan management, workspace, argument checks.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "gt.h"
#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {
cudaError_t configure_steps();
cudaError_t configure_sort();
cudaError_t configure_radix();

// Raises the kernels' shared-memory limits, once per device (thread-safe).
cudaError_t configure_kernels(int device) {
  static std::mutex mu;
  static std::vector<char> done;
  std::lock_guard<std::mutex> lock(mu);
  if ((size_t)device >= done.size()) done.resize((size_t)device + 1, 0);
  if (done[(size_t)device]) return cudaSuccess;
  cudaError_t e = configure_steps();
  if (e == cudaSuccess) e = configure_sort();
  if (e == cudaSuccess) e = configure_radix();
  if (e == cudaSuccess) done[(size_t)device] = 1;
  return e;
}
}  // namespace gt

struct gt_plan_s {
  gt::DevWork w;
  gt_config cfg;
  int device = 0;
  cudaStream_t last = nullptr;
  uint64_t ws_bytes = 0;
  void *allocs[32] = {};
  int nalloc = 0;
  // device copies for gt_transpose_host (allocated on first use); the
  // asynchronous path adds a second output set (h_col_ptr[1] ...)
  uint64_t *h_row_ptr[2] = {}, *h_col_ptr[2] = {};
  uint32_t *h_col_idx[2] = {}, *h_row_idx[2] = {};
  float *h_vals[2] = {}, *h_vals_out[2] = {};
  void *host_allocs[12] = {};
  int nhost = 0;
  // gt_transpose_host_async: input copies on in_stream once the last
  // transposition that read that input set is past its inputs
  // (ev_inputs_read[set]); output copies on copy_stream; input and output
  // sets used in turn (ev_copied[set] guards an output set's reuse)
  cudaStream_t copy_stream = nullptr, in_stream = nullptr;
  cudaEvent_t ev_computed = nullptr, ev_copied[2] = {}, ev_inputs_read[2] = {}, ev_inputs_in = nullptr;
  int slot = 0, slots = 1;
  bool second_tried = false;  // the second input and output sets are attempted once
  cudaEvent_t pending_inputs_read = nullptr;  // handed to the next transposition's Problem
  // per-step timing
  bool timing = false;
  std::vector<gt::StepEvents> events;
  // gt_transpose_host_async while timing: events around each call's input
  // copies (on in_stream) and output copies (on copy_stream)
  struct HostEvents {
    cudaEvent_t in0, in1, out0, out1;
  };
  std::vector<HostEvents> host_events;
  uint32_t launches = 0;
};

namespace {
constexpr size_t kMaxHostEvents = 64;  // calls whose copies are timed per enable

void drop_events(gt_plan p) {
  for (auto &e : p->events) {
    for (int i = 0; i < 6; ++i) cudaEventDestroy(e.ev[i]);
    for (int i = 0; i < 8; ++i) cudaEventDestroy(e.down[i]);
    for (int i = 0; i < 2; ++i) cudaEventDestroy(e.part[i]);
  }
  p->events.clear();
  for (auto &h : p->host_events)
    for (cudaEvent_t x : {h.in0, h.in1, h.out0, h.out1}) cudaEventDestroy(x);
  p->host_events.clear();
}
}  // namespace

namespace {

uint32_t ceil_log2_u64(uint64_t x) {
  uint32_t b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

bool config_valid(const gt_config &c) {
  if (c.hdv_k > (uint32_t)gt::kMaxHdv) return false;
  if (c.hdv_k > 0) {
    if (c.table_log2 < 1 || c.table_log2 > (uint32_t)gt::kMaxTableLog2) return false;
    if ((1ull << c.table_log2) < 2ull * c.hdv_k) return false;
  }
  if (c.block_threads < 64 || c.block_threads > 1024 || c.block_threads % 32) return false;
  if (c.ctas_per_sm < 1 || c.ctas_per_sm > 32) return false;
  if (c.warp_edges < 32) return false;
  if (c.stage_edges != 0 && (c.stage_edges < 128 || c.stage_edges > 4096 || c.stage_edges % 128)) return false;
  if (c.sample_permille > 1000) return false;
  if (c.method > GT_METHOD_RADIX) return false;
  if (c.radix_tile != 0 && c.radix_tile != 2048 && c.radix_tile != 4096) return false;
  if (c.radix_digit_bits != 0 && (c.radix_digit_bits < 4 || c.radix_digit_bits > 8)) return false;
  if ((c.flags & GT_FLAG_STEAL_TAILS) && c.stage_edges != 0) return false;  // the two phases use direct loads
  if (c.partition_bits > 8) return false;
  // the partitioned form reads the bucketed arrays with direct loads, in ranges taken in order
  if (c.partition_bits && c.method == GT_METHOD_HLH && (c.stage_edges != 0 || (c.flags & GT_FLAG_STEAL_TAILS)))
    return false;
  return true;
}

// Derives the launch shape of Steps 1-3 from the configuration and sizes.
gt_status derive_shape(gt::DevWork &w, const gt_config &c, int num_sms) {
  w.num_sms = num_sms;
  w.kmax = (w.m > 0) ? c.hdv_k : 0;
  w.tlog2 = w.kmax ? c.table_log2 : 0;
  w.W = c.block_threads / 32;
  // partitioned form: the top bits of the destination, at most all of them
  w.part_bits = 0;
  // (weighted matrices with more than 2^31 rows cannot tag split rows: they run unpartitioned)
  if (c.method == GT_METHOD_HLH && c.partition_bits && w.m > 0 && !(w.has_vals && w.n_rows > 0x80000000u)) {
    uint32_t kb = 0;
    while (kb < 32 && (w.n - 1) >> kb) ++kb;
    w.part_bits = c.partition_bits < kb ? c.partition_bits : kb;
  }
  uint64_t want = (w.m + (uint64_t)w.W * c.warp_edges - 1) / ((uint64_t)w.W * c.warp_edges);
  // one wave of warp partitions, except in the partitioned form: there every
  // range of warp_edges edges is a partition of its own, and CTAs launched in
  // order walk the bucketed edges front to back
  uint64_t cap = w.part_bits ? ((1ull << 31) - 1) / w.W : (uint64_t)num_sms * c.ctas_per_sm;
  if (want < 1) want = 1;
  if (want > cap) want = cap;
  w.G = (uint32_t)want;
  w.P = w.G * w.W;
  // more than 32 K partitions: the HDV insertion points are scanned in slices
  // of at least 1024 partitions (at most 1024 slices)
  w.hdv_q = 1;
  if (w.P > 32768u) {
    const uint32_t q = (w.P + 1023) / 1024;
    w.hdv_q = q < 1024 ? q : 1024;
  }
  w.psize = w.m ? (w.m + w.P - 1) / w.P : 1;
  if (w.psize == 0) w.psize = 1;
  w.staged = c.stage_edges ? 1 : 0;
  w.stage_edges = c.stage_edges;
  w.smem_count = gt::smem_count_bytes(w.W, w.kmax, w.tlog2, w.staged, w.stage_edges, w.has_vals);
  w.smem_scatter = gt::smem_scatter_bytes(w.W, w.kmax, w.tlog2, w.staged, w.stage_edges, w.has_vals);
  if (w.smem_count > 227u * 1024u || w.smem_scatter > 227u * 1024u) return GT_ERR_INVALID_ARG;
  uint64_t ns = w.kmax ? ((uint64_t)w.n * c.sample_permille + 999) / 1000 : 0;
  if (ns > (1u << 22)) ns = 1u << 22;
  if (w.m == 0) ns = 0;
  w.ns = (uint32_t)ns;
  w.ts_log2 = ceil_log2_u64(ns * 2 < 1024 ? 1024 : ns * 2);
  // the look-back scan covers the columns and, in the same grid, validates the rows
  const uint64_t span = w.n > w.n_rows ? w.n : w.n_rows;
  w.ntiles = (uint32_t)((span + gt::kScanTile - 1) / gt::kScanTile);
  if (w.ntiles == 0) w.ntiles = 1;
  w.big_cap = (uint32_t)gt::worklist_entries(w.m);
  w.flag_mode = (w.has_vals && w.n_rows <= 0x80000000u) ? 1 : 0;
  w.method = (int)c.method;
  // radix method: radix_tile selects the tile (256 threads x 8 or 16 items),
  // ctas_per_sm the persistent grid
  w.r_items = c.radix_tile == 2048 ? 8u : 16u;
  w.r_bulk = c.radix_tile == 0 ? 1 : 0;
  w.rG = (uint32_t)num_sms * c.ctas_per_sm;
  w.r_dcap = c.radix_digit_bits ? c.radix_digit_bits : 8u;
  w.ptimes = (c.flags & GT_FLAG_PARTITION_TIMES) ? 1 : 0;
  w.steal = (c.flags & GT_FLAG_STEAL_TAILS) ? 1 : 0;
  if (w.method == GT_METHOD_RADIX) {
    w.kmax = 0;
    w.tlog2 = 0;
    w.ns = 0;
  }
  return GT_OK;
}

gt_status plan_alloc(gt_plan p, void **ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (p->nalloc >= 32) return GT_ERR_NO_MEMORY;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return GT_ERR_NO_MEMORY;
  }
  p->allocs[p->nalloc++] = *ptr;
  p->ws_bytes += bytes;
  return GT_OK;
}

void plan_free_ws(gt_plan p) {
  for (int i = 0; i < p->nalloc; ++i) cudaFree(p->allocs[i]);
  p->nalloc = 0;
  p->ws_bytes = 0;
  gt::DevWork keep = p->w;
  p->w = gt::DevWork();
  p->w.n = keep.n;
  p->w.n_rows = keep.n_rows;
  p->w.m = keep.m;
  p->w.has_vals = keep.has_vals;
}

gt_status plan_alloc_ws(gt_plan p) {
  gt::DevWork &w = p->w;
  const size_t n = w.n, m = w.m;
  const size_t T = w.kmax ? ((size_t)1 << w.tlog2) : 1;
  const size_t ts = (size_t)1 << w.ts_log2;
  gt_status st;
#define GT_AL(field, bytes)                                                    \
  do {                                                                         \
    if ((st = plan_alloc(p, (void **)&w.field, (bytes))) != GT_OK) return st; \
  } while (0)
  GT_AL(status, 4);
  GT_AL(meta, gt::kMetaCount * 4);
  GT_AL(meta64, 4 * 8);
  if (w.method == GT_METHOD_RADIX) {  // col_ptr comes from the sorted keys: no degree array, no scan state
    GT_AL(r_a_key, m * 4);
    // weighted: one block, either (sources | values) as two u32 arrays or the
    // interleaved (source, value) pairs of the bulk-staged passes; the values
    // start on a 16-byte boundary (bulk copies read them)
    const size_t m4 = (m + 3) & ~(size_t)3;
    GT_AL(r_a_u, w.has_vals ? m4 * 8 : m * 4);
    if (w.has_vals) w.r_a_w = w.r_a_u + m4;
    GT_AL(r_b_key, m * 4);
    if (w.has_vals) GT_AL(r_b_sv, m4 * 8);
    GT_AL(r_long, (m / 2049 + 1) * 4);
    w.r_gap_cap = (uint32_t)(n / 1024 + 2);
    GT_AL(r_gaps, (1 + 2 * (size_t)w.r_gap_cap) * 8);
    GT_AL(r_nlong, 4);
    // bulk-staged passes: up to 4 CTAs per SM x 2 sub-CTAs of the upsweep
    const size_t rows = w.rG > (uint32_t)w.num_sms * 8u ? w.rG : (size_t)w.num_sms * 8u;
    GT_AL(r_table, rows * 256 * 4);
    GT_AL(r_offsets, rows * 256 * 8);
    if (cudaMemset(w.status, 0, 4) != cudaSuccess) return GT_ERR_CUDA;
    if (cudaMemset(w.meta, 0, gt::kMetaCount * 4) != cudaSuccess) return GT_ERR_CUDA;
    if (cudaMemset(w.meta64, 0, 32) != cudaSuccess) return GT_ERR_CUDA;
    return GT_OK;
  }
  GT_AL(deg, n * 4);
  GT_AL(scan_state, (size_t)w.ntiles * 8);
  GT_AL(cursor, n * 8);
  GT_AL(hdv_cnt, (size_t)w.P * (w.steal ? 2 : 1) * (w.kmax ? w.kmax : 1) * 4);
  GT_AL(hdv_ids, (w.kmax ? w.kmax : 1) * 4);
  if (w.hdv_q > 1 && w.kmax) GT_AL(hdv_psum, (size_t)w.hdv_q * w.kmax * 8);
  GT_AL(hdv_start, (w.kmax ? w.kmax : 1) * 8);
  GT_AL(hkeys, T * 4);
  GT_AL(hvals, T * 2);
  GT_AL(part, ((size_t)w.P + 1) * 8);
  GT_AL(skeys, (w.kmax ? ts : 1) * 4);
  GT_AL(scnt, (w.kmax ? ts : 1) * 4);
  GT_AL(fhist, (w.kmax ? gt::kFreqBins : 1) * 4);
  GT_AL(cand, (w.kmax ? w.kmax : 1) * 4);
  GT_AL(ties, (w.kmax ? gt::kTieCap : 1) * 4);
  GT_AL(biglist, (size_t)w.big_cap * 4);
  GT_AL(scratch, m * (w.has_vals ? 8 : 4));
  if (w.ptimes) GT_AL(ptime, (size_t)w.P * 2 * 8);
  if (w.steal) {
    GT_AL(part2, ((size_t)w.P * 2 + 1) * 8);
    GT_AL(steal_next, 4);
  }
  if (w.part_bits) {  // bucketing pass: row sources, bucketed triples, digit tables
    GT_AL(r_a_u, m * 4);
    GT_AL(q_key, m * 4);
    GT_AL(q_u, m * 4);
    if (w.has_vals) GT_AL(q_w, m * 4);
    GT_AL(r_long, (m / 2049 + 1) * 4);
    GT_AL(r_nlong, 4);
    const size_t rows = (size_t)w.num_sms * 8u;
    GT_AL(r_table, rows * 256 * 4);
    GT_AL(r_offsets, rows * 256 * 8);
  }
#undef GT_AL
  if (cudaMemset(w.status, 0, 4) != cudaSuccess) return GT_ERR_CUDA;
  if (cudaMemset(w.meta, 0, gt::kMetaCount * 4) != cudaSuccess) return GT_ERR_CUDA;
  if (cudaMemset(w.meta64, 0, 32) != cudaSuccess) return GT_ERR_CUDA;
  return GT_OK;
}

gt_status apply_config(gt_plan p, const gt_config &c) {
  if (!config_valid(c)) return GT_ERR_INVALID_ARG;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return GT_ERR_CUDA;
  gt::DevWork w;
  w.n = p->w.n;
  w.n_rows = p->w.n_rows;
  w.m = p->w.m;
  w.has_vals = p->w.has_vals;
  gt_status st = derive_shape(w, c, sms);
  if (st != GT_OK) return st;
  plan_free_ws(p);
  p->w = w;
  p->cfg = c;
  st = plan_alloc_ws(p);
  if (st != GT_OK) plan_free_ws(p);
  return st;
}

}  // namespace

namespace gt {
thread_local const char *g_last_cuda = "no error";

gt_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return GT_OK;
  g_last_cuda = cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return GT_ERR_NO_MEMORY;
  return GT_ERR_CUDA;
}
}  // namespace gt

using gt::from_cuda;
using gt::g_last_cuda;

extern "C" {

uint32_t gt_version(void) { return 100; }

const char *gt_last_cuda_error(void) { return g_last_cuda; }

const char *gt_status_string(gt_status s) {
  switch (s) {
    case GT_OK: return "ok";
    case GT_ERR_INVALID_ARG: return "invalid argument";
    case GT_ERR_OUT_OF_RANGE: return "col_idx entry out of range";
    case GT_ERR_BAD_ROW_PTR: return "invalid row_ptr";
    case GT_ERR_NO_MEMORY: return "out of device memory";
    case GT_ERR_CUDA: return "CUDA runtime error";
    case GT_ERR_TIMEOUT: return "bounded device wait expired";
    case GT_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}

gt_status gt_default_config(gt_config *cfg, uint32_t n_vertices, uint64_t n_edges) {
  if (!cfg) return GT_ERR_INVALID_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->block_threads = 256;
  cfg->ctas_per_sm = 4;
  cfg->warp_edges = 4096;
  cfg->stage_edges = 0;
  cfg->sample_permille = 10;
  cfg->flags = GT_FLAG_AGGREGATE;
  cfg->seed = 0x5EED0001ull;
  // Eq. 1 with the per-CTA shared memory of 4 CTAs/SM as |cache|, a 6-byte
  // record at load factor 1/2, 8 bytes of per-CTA HDV data and one 4-byte
  // counter per warp: k = 48 KB / (12 + 8 + 4*8) ~ 945 -> 512 (power of two).
  uint32_t k = 512;
  if (n_edges < (1ull << 18)) k = 0;
  if (k > n_vertices / 2) {
    k = 0;
  }
  cfg->hdv_k = k;
  cfg->table_log2 = k ? ceil_log2_u64(2ull * k) : 0;
  // Graphs whose per-vertex arrays and output far exceed L2 make every random
  // access of the HLH method a DRAM access; the radix method streams instead.
  cfg->method = n_edges >= (1ull << 22) ? GT_METHOD_RADIX : GT_METHOD_HLH;
  return GT_OK;
}

gt_status gt_plan_create_rect(gt_plan *plan, uint32_t n_rows, uint32_t n_cols, uint64_t n_edges, int has_vals,
                              const gt_config *cfg, void *stream) {
  (void)stream;
  if (!plan) return GT_ERR_INVALID_ARG;
  *plan = nullptr;
  if (has_vals && n_edges > (1ull << 32)) return GT_ERR_UNSUPPORTED;
  if (n_edges >= (1ull << 62)) return GT_ERR_UNSUPPORTED;
  if ((n_rows == 0 || n_cols == 0) && n_edges != 0) return GT_ERR_INVALID_ARG;
  gt_plan p = new (std::nothrow) gt_plan_s();
  if (!p) return GT_ERR_NO_MEMORY;
  cudaError_t ge = cudaGetDevice(&p->device);
  if (ge != cudaSuccess) {
    from_cuda(ge);
    cudaGetLastError();
    delete p;
    return GT_ERR_CUDA;
  }
  {
    cudaError_t ce = gt::configure_kernels(p->device);
    if (ce != cudaSuccess) {
      from_cuda(ce);
      cudaGetLastError();
      delete p;
      return GT_ERR_CUDA;
    }
  }
  p->w.n = n_cols;
  p->w.n_rows = n_rows;
  p->w.m = n_edges;
  p->w.has_vals = has_vals ? 1 : 0;
  gt_config c;
  if (cfg) c = *cfg;
  else gt_default_config(&c, n_cols, n_edges);
  gt_status st = apply_config(p, c);
  if (st != GT_OK) {
    plan_free_ws(p);
    delete p;
    return st;
  }
  *plan = p;
  return GT_OK;
}

gt_status gt_plan_create(gt_plan *plan, uint32_t n_vertices, uint64_t n_edges, int has_vals, const gt_config *cfg,
                         void *stream) {
  return gt_plan_create_rect(plan, n_vertices, n_vertices, n_edges, has_vals, cfg, stream);
}

gt_status gt_plan_set_config(gt_plan plan, const gt_config *cfg) {
  if (!plan || !cfg) return GT_ERR_INVALID_ARG;
  if (!config_valid(*cfg)) return GT_ERR_INVALID_ARG;
  if (plan->last) cudaStreamSynchronize(plan->last);
  return apply_config(plan, *cfg);
}

gt_status gt_plan_get_config(gt_plan plan, gt_config *cfg) {
  if (!plan || !cfg) return GT_ERR_INVALID_ARG;
  *cfg = plan->cfg;
  return GT_OK;
}

// Launch shape of a smaller matrix on a plan's buffers (every buffer size is
// monotone in the column count and m for a fixed configuration; none depends
// on the row count).
static gt_status shape_for(gt_plan plan, uint32_t n_rows, uint32_t n, uint64_t m, gt::DevWork &w) {
  w = plan->w;
  if (n == w.n && n_rows == w.n_rows && m == w.m) return GT_OK;
  gt::DevWork t;
  t.n = n;
  t.n_rows = n_rows;
  t.m = m;
  t.has_vals = w.has_vals;
  gt_status st = derive_shape(t, plan->cfg, w.num_sms);
  if (st != GT_OK) return st;
  w.n = t.n;
  w.n_rows = t.n_rows;
  w.m = t.m;
  w.kmax = t.kmax;
  w.tlog2 = t.tlog2;
  w.W = t.W;
  w.G = t.G;
  w.P = t.P;
  w.psize = t.psize;
  w.ns = t.ns;
  w.ts_log2 = t.ts_log2;
  w.ntiles = t.ntiles;
  w.big_cap = t.big_cap;
  w.flag_mode = t.flag_mode;
  w.staged = t.staged;
  w.stage_edges = t.stage_edges;
  w.smem_count = t.smem_count;
  w.smem_scatter = t.smem_scatter;
  w.method = t.method;
  w.rG = t.rG;
  w.r_items = t.r_items;
  w.r_bulk = t.r_bulk;
  w.r_dcap = t.r_dcap;
  w.ptimes = t.ptimes;
  w.steal = t.steal;
  w.part_bits = t.part_bits;
  w.hdv_q = t.hdv_q < w.hdv_q ? t.hdv_q : w.hdv_q;
  w.r_gap_cap = (uint32_t)(t.n / 1024 + 2) < w.r_gap_cap ? (uint32_t)(t.n / 1024 + 2) : w.r_gap_cap;
  return GT_OK;
}

static gt_status transpose_impl(gt_plan plan, uint32_t n_rows, uint32_t n, uint64_t m, const uint64_t *row_ptr,
                                const uint32_t *col_idx, const float *vals, uint64_t *col_ptr, uint32_t *row_idx,
                                float *vals_out, void *stream) {
  if (!plan || !row_ptr || !col_ptr) return GT_ERR_INVALID_ARG;
  if (m > 0 && (!col_idx || !row_idx)) return GT_ERR_INVALID_ARG;
  if ((vals == nullptr) != (vals_out == nullptr)) return GT_ERR_INVALID_ARG;
  if (vals && !plan->w.has_vals) return GT_ERR_INVALID_ARG;
  if ((n == 0 || n_rows == 0) && m != 0) return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  plan->last = s;
  // no rows or no columns (and no entries): every offset is 0; row_ptr is not read
  if (n == 0 || n_rows == 0) return from_cuda(cudaMemsetAsync(col_ptr, 0, ((size_t)n + 1) * 8, s));
  gt::DevWork w;
  gt_status sst = shape_for(plan, n_rows, n, m, w);
  if (sst != GT_OK) return sst;
  // bulk copies need 16-byte aligned sources; fall back to direct loads otherwise
  if (w.staged && ((((uintptr_t)col_idx) & 15u) || (vals && (((uintptr_t)vals) & 15u)))) {
    w.staged = 0;
    w.smem_count = gt::smem_count_bytes(w.W, w.kmax, w.tlog2, 0, 0, w.has_vals);
    w.smem_scatter = gt::smem_scatter_bytes(w.W, w.kmax, w.tlog2, 0, 0, w.has_vals);
  }
  gt::Problem pb{row_ptr, col_idx, vals, col_ptr, row_idx, vals_out};
  pb.inputs_read = plan->pending_inputs_read;
  gt::StepEvents *ev = nullptr;
  if (plan->timing) {
    gt::StepEvents e;
    for (int i = 0; i < 6; ++i)
      if (cudaEventCreate(&e.ev[i]) != cudaSuccess) return GT_ERR_CUDA;
    for (int i = 0; i < 8; ++i)
      if (cudaEventCreate(&e.down[i]) != cudaSuccess) return GT_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreate(&e.part[i]) != cudaSuccess) return GT_ERR_CUDA;
    e.ndown = 0;
    e.has_part = 0;
    plan->events.push_back(e);
    ev = &plan->events.back();
  }
  return from_cuda(gt::run_transpose(w, plan->cfg, pb, s, ev, &plan->launches));
}

gt_status gt_transpose(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                       uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, void *stream) {
  if (!plan) return GT_ERR_INVALID_ARG;
  return transpose_impl(plan, plan->w.n_rows, plan->w.n, plan->w.m, row_ptr, col_idx, vals, col_ptr, row_idx,
                        vals_out, stream);
}

gt_status gt_transpose_sub_rect(gt_plan plan, uint32_t n_rows, uint32_t n_cols, uint64_t n_edges,
                                const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                                uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, void *stream) {
  if (!plan) return GT_ERR_INVALID_ARG;
  if (n_rows > plan->w.n_rows || n_cols > plan->w.n || n_edges > plan->w.m) return GT_ERR_INVALID_ARG;
  return transpose_impl(plan, n_rows, n_cols, n_edges, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream);
}

gt_status gt_transpose_sub(gt_plan plan, uint32_t n_vertices, uint64_t n_edges, const uint64_t *row_ptr,
                           const uint32_t *col_idx, const float *vals, uint64_t *col_ptr, uint32_t *row_idx,
                           float *vals_out, void *stream) {
  return gt_transpose_sub_rect(plan, n_vertices, n_vertices, n_edges, row_ptr, col_idx, vals, col_ptr, row_idx,
                               vals_out, stream);
}

gt_status gt_plan_enable_timing(gt_plan plan, int enable) {
  if (!plan) return GT_ERR_INVALID_ARG;
  if (plan->last) cudaStreamSynchronize(plan->last);
  drop_events(plan);
  plan->timing = enable != 0;
  return GT_OK;
}

gt_status gt_plan_timing(gt_plan plan, gt_timing *t) {
  if (!plan || !t) return GT_ERR_INVALID_ARG;
  memset(t, 0, sizeof(*t));
  if (plan->events.empty()) return GT_OK;
  if (cudaEventSynchronize(plan->events.back().ev[5]) != cudaSuccess) return GT_ERR_CUDA;
  double acc[5] = {0, 0, 0, 0, 0};
  double part = 0;
  double dom = 0;
  uint32_t ndom = 0;
  for (auto &e : plan->events) {
    for (int i = 0; i < 5; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.ev[i], e.ev[i + 1]) != cudaSuccess) return GT_ERR_CUDA;
      acc[i] += ms;
    }
    if (e.has_part) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.part[0], e.part[1]) != cudaSuccess) return GT_ERR_CUDA;
      part += ms;
    }
    if (e.ndown) {
      for (uint32_t i = 0; i + 1 < e.ndown; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.down[i], e.down[i + 1]) != cudaSuccess) return GT_ERR_CUDA;
        dom += ms;
        ++ndom;
      }
    } else {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.ev[3], e.ev[4]) != cudaSuccess) return GT_ERR_CUDA;
      dom += ms;
      ++ndom;
    }
  }
  const double c = (double)plan->events.size();
  t->calls = (uint32_t)plan->events.size();
  t->sample_ms = (float)(acc[0] / c);
  t->count_ms = (float)(acc[1] / c);
  t->scan_ms = (float)(acc[2] / c);
  t->scatter_ms = (float)(acc[3] / c);
  t->sort_ms = (float)(acc[4] / c);
  t->dominant_ms = ndom ? (float)(dom / ndom) : 0.f;
  t->dominant_launches = ndom;
  t->partition_ms = (float)(part / c);
  t->total_ms = (float)((acc[0] + acc[1] + acc[2] + acc[3] + acc[4] + part) / c);
  return GT_OK;
}

gt_status gt_plan_status(gt_plan plan) {
  if (!plan) return GT_ERR_INVALID_ARG;
  {
    cudaError_t se = cudaStreamSynchronize(plan->last);
    if (se != cudaSuccess) return from_cuda(se);
  }
  uint32_t st = 0;
  {
    cudaError_t ce = cudaMemcpy(&st, plan->w.status, 4, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return from_cuda(ce);
  }
  if (st) cudaMemset(plan->w.status, 0, 4);
  return (gt_status)st;
}

gt_status gt_plan_stats(gt_plan plan, gt_stats *stats) {
  if (!plan || !stats) return GT_ERR_INVALID_ARG;
  {
    cudaError_t se = cudaStreamSynchronize(plan->last);
    if (se != cudaSuccess) return from_cuda(se);
  }
  uint32_t meta[gt::kMetaCount];
  unsigned long long m64[4];
  if (cudaMemcpy(meta, plan->w.meta, sizeof(meta), cudaMemcpyDeviceToHost) != cudaSuccess) return GT_ERR_CUDA;
  if (cudaMemcpy(m64, plan->w.meta64, sizeof(m64), cudaMemcpyDeviceToHost) != cudaSuccess) return GT_ERR_CUDA;
  memset(stats, 0, sizeof(*stats));
  stats->hdv_selected = plan->w.kmax ? meta[gt::kMetaK] : 0;
  stats->partitions = plan->w.P;
  stats->hdv_edges = m64[0];
  stats->n_edges = plan->w.m;
  stats->ldv_sorted_cols = meta[gt::kMetaSorted];
  stats->large_cols = meta[gt::kMetaLargeN];
  stats->kernel_launches = plan->launches;
  return GT_OK;
}

uint64_t gt_plan_workspace_bytes(gt_plan plan) { return plan ? plan->ws_bytes : 0; }

uint32_t gt_plan_vertices(gt_plan plan) { return plan ? plan->w.n_rows : 0; }

gt_status gt_plan_shape(gt_plan plan, uint32_t *n_rows, uint32_t *n_cols, uint64_t *n_edges) {
  if (!plan) return GT_ERR_INVALID_ARG;
  if (n_rows) *n_rows = plan->w.n_rows;
  if (n_cols) *n_cols = plan->w.n;
  if (n_edges) *n_edges = plan->w.m;
  return GT_OK;
}

uint64_t gt_plan_edges(gt_plan plan) { return plan ? plan->w.m : 0; }

static gt_status host_alloc(gt_plan plan, void **field, size_t bytes) {
  void *q = nullptr;
  if (plan->nhost >= 12 || cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return GT_ERR_NO_MEMORY;
  }
  plan->host_allocs[plan->nhost++] = q;
  *field = q;
  return GT_OK;
}

// Device staging of the host paths: input and output set 0 (and, with
// second_set, set 1 if it can be allocated).
static gt_status host_staging(gt_plan plan, bool second_set) {
  const size_t n = plan->w.n, nr = plan->w.n_rows, m = plan->w.m;
  const bool v = plan->w.has_vals != 0;
  auto alloc_set = [&](int k) {
    return host_alloc(plan, (void **)&plan->h_row_ptr[k], (nr + 1) * 8) == GT_OK &&
           host_alloc(plan, (void **)&plan->h_col_ptr[k], (n + 1) * 8) == GT_OK &&
           host_alloc(plan, (void **)&plan->h_col_idx[k], m * 4) == GT_OK &&
           host_alloc(plan, (void **)&plan->h_row_idx[k], m * 4) == GT_OK &&
           (!v || host_alloc(plan, (void **)&plan->h_vals[k], m * 4) == GT_OK) &&
           (!v || host_alloc(plan, (void **)&plan->h_vals_out[k], m * 4) == GT_OK);
  };
  auto drop_set = [&](int k, int keep) {  // frees what a failed alloc_set(k) got
    while (plan->nhost > keep) cudaFree(plan->host_allocs[--plan->nhost]);
    plan->h_row_ptr[k] = plan->h_col_ptr[k] = nullptr;
    plan->h_col_idx[k] = plan->h_row_idx[k] = nullptr;
    plan->h_vals[k] = plan->h_vals_out[k] = nullptr;
  };
  if (!plan->h_row_ptr[0]) {
    const int keep = plan->nhost;
    if (!alloc_set(0)) {
      drop_set(0, keep);
      return GT_ERR_NO_MEMORY;
    }
  }
  if (second_set && !plan->second_tried) {  // optional: without it the calls share one set
    plan->second_tried = true;
    if (const char *env = getenv("GT_HOST_SETS")) {  // "1": one set only (testing)
      if (strtoul(env, nullptr, 10) == 1) return GT_OK;
    }
    const int keep = plan->nhost;
    if (alloc_set(1)) plan->slots = 2;
    else drop_set(1, keep);
  }
  return GT_OK;
}

static gt_status host_args(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                           uint64_t *col_ptr, uint32_t *row_idx, float *vals_out) {
  if (!plan || !row_ptr || !col_ptr) return GT_ERR_INVALID_ARG;
  if (plan->w.m > 0 && (!col_idx || !row_idx)) return GT_ERR_INVALID_ARG;
  if ((vals == nullptr) != (vals_out == nullptr)) return GT_ERR_INVALID_ARG;
  if (vals && !plan->w.has_vals) return GT_ERR_INVALID_ARG;
  return GT_OK;
}

gt_status gt_transpose_host(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                            uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, void *stream) {
  gt_status ast = host_args(plan, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out);
  if (ast != GT_OK) return ast;
  const size_t n = plan->w.n, nr = plan->w.n_rows, m = plan->w.m;
  cudaStream_t s = (cudaStream_t)stream;
  if ((ast = host_staging(plan, false)) != GT_OK) return ast;
  // asynchronous calls still copying use the same device buffers
  if (plan->in_stream && cudaStreamSynchronize(plan->in_stream) != cudaSuccess) return GT_ERR_CUDA;
  if (plan->copy_stream && cudaStreamSynchronize(plan->copy_stream) != cudaSuccess) return GT_ERR_CUDA;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(plan->h_row_ptr[0], row_ptr, (nr + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return from_cuda(e);
  if (m && (e = cudaMemcpyAsync(plan->h_col_idx[0], col_idx, m * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return from_cuda(e);
  if (vals && m && (e = cudaMemcpyAsync(plan->h_vals[0], vals, m * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return from_cuda(e);
  gt_status st = gt_transpose(plan, plan->h_row_ptr[0], plan->h_col_idx[0], vals ? plan->h_vals[0] : nullptr,
                              plan->h_col_ptr[0], plan->h_row_idx[0], vals ? plan->h_vals_out[0] : nullptr, stream);
  if (st != GT_OK) return st;
  if ((e = cudaMemcpyAsync(col_ptr, plan->h_col_ptr[0], (n + 1) * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return from_cuda(e);
  if (m && (e = cudaMemcpyAsync(row_idx, plan->h_row_idx[0], m * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return from_cuda(e);
  if (vals && m &&
      (e = cudaMemcpyAsync(vals_out, plan->h_vals_out[0], m * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return from_cuda(e);
  return gt_plan_status(plan);
}

gt_status gt_transpose_host_async(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                                  uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, void *stream) {
  gt_status ast = host_args(plan, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out);
  if (ast != GT_OK) return ast;
  const size_t n = plan->w.n, nr = plan->w.n_rows, m = plan->w.m;
  cudaStream_t s = (cudaStream_t)stream;
  if ((ast = host_staging(plan, true)) != GT_OK) return ast;
  if (!plan->copy_stream) {
    if (cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&plan->in_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_computed, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_copied[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_copied[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_inputs_read[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_inputs_read[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_inputs_in, cudaEventDisableTiming) != cudaSuccess)
      return from_cuda(cudaGetLastError());
    // the device inputs are free once everything enqueued on s so far is done
    if (cudaEventRecord(plan->ev_inputs_read[0], s) != cudaSuccess ||
        cudaEventRecord(plan->ev_inputs_read[1], s) != cudaSuccess)
      return GT_ERR_CUDA;
  }
  const int k = plan->slot;
  plan->slot = (plan->slot + 1) % plan->slots;
  cudaError_t e;
  // inputs: on in_stream, once the last transposition that read set k is past its inputs
  cudaStream_t in = plan->in_stream;
  if ((e = cudaStreamWaitEvent(in, plan->ev_inputs_read[k], 0)) != cudaSuccess) return from_cuda(e);
  gt_plan_s::HostEvents *hev = nullptr;
  if (plan->timing && plan->host_events.size() < kMaxHostEvents) {
    gt_plan_s::HostEvents h{};
    if (cudaEventCreate(&h.in0) != cudaSuccess || cudaEventCreate(&h.in1) != cudaSuccess ||
        cudaEventCreate(&h.out0) != cudaSuccess || cudaEventCreate(&h.out1) != cudaSuccess) {
      for (cudaEvent_t x : {h.in0, h.in1, h.out0, h.out1})
        if (x) cudaEventDestroy(x);
      return from_cuda(cudaGetLastError());
    }
    plan->host_events.push_back(h);
    hev = &plan->host_events.back();
    if ((e = cudaEventRecord(hev->in0, in)) != cudaSuccess) return from_cuda(e);
  }
  if ((e = cudaMemcpyAsync(plan->h_row_ptr[k], row_ptr, (nr + 1) * 8, cudaMemcpyHostToDevice, in)) != cudaSuccess)
    return from_cuda(e);
  if (m && (e = cudaMemcpyAsync(plan->h_col_idx[k], col_idx, m * 4, cudaMemcpyHostToDevice, in)) != cudaSuccess)
    return from_cuda(e);
  if (vals && m && (e = cudaMemcpyAsync(plan->h_vals[k], vals, m * 4, cudaMemcpyHostToDevice, in)) != cudaSuccess)
    return from_cuda(e);
  if (hev && (e = cudaEventRecord(hev->in1, in)) != cudaSuccess) return from_cuda(e);
  if ((e = cudaEventRecord(plan->ev_inputs_in, in)) != cudaSuccess) return from_cuda(e);
  // the transposition: after its inputs arrived and output set k's last copy-out
  if ((e = cudaStreamWaitEvent(s, plan->ev_inputs_in, 0)) != cudaSuccess) return from_cuda(e);
  if ((e = cudaStreamWaitEvent(s, plan->ev_copied[k], 0)) != cudaSuccess) return from_cuda(e);
  plan->pending_inputs_read = plan->ev_inputs_read[k];
  gt_status st = gt_transpose(plan, plan->h_row_ptr[k], plan->h_col_idx[k], vals ? plan->h_vals[k] : nullptr,
                              plan->h_col_ptr[k], plan->h_row_idx[k], vals ? plan->h_vals_out[k] : nullptr, stream);
  plan->pending_inputs_read = nullptr;
  if (st != GT_OK) return st;
  // outputs: on copy_stream, after the transposition
  cudaStream_t c = plan->copy_stream;
  if ((e = cudaEventRecord(plan->ev_computed, s)) != cudaSuccess) return from_cuda(e);
  if ((e = cudaStreamWaitEvent(c, plan->ev_computed, 0)) != cudaSuccess) return from_cuda(e);
  if (hev && (e = cudaEventRecord(hev->out0, c)) != cudaSuccess) return from_cuda(e);
  if ((e = cudaMemcpyAsync(col_ptr, plan->h_col_ptr[k], (n + 1) * 8, cudaMemcpyDeviceToHost, c)) != cudaSuccess)
    return from_cuda(e);
  if (m && (e = cudaMemcpyAsync(row_idx, plan->h_row_idx[k], m * 4, cudaMemcpyDeviceToHost, c)) != cudaSuccess)
    return from_cuda(e);
  if (vals && m &&
      (e = cudaMemcpyAsync(vals_out, plan->h_vals_out[k], m * 4, cudaMemcpyDeviceToHost, c)) != cudaSuccess)
    return from_cuda(e);
  if (hev && (e = cudaEventRecord(hev->out1, c)) != cudaSuccess) return from_cuda(e);
  if ((e = cudaEventRecord(plan->ev_copied[k], c)) != cudaSuccess) return from_cuda(e);
  return GT_OK;
}

gt_status gt_plan_partition_times(gt_plan plan, float *busy_ms, uint32_t cap, uint32_t *count) {
  if (!plan || (cap > 0 && !busy_ms)) return GT_ERR_INVALID_ARG;
  if (count) *count = 0;
  if (!plan->w.ptime) return GT_ERR_INVALID_ARG;  // the plan's configuration does not record them
  cudaError_t e;
  if (plan->last && (e = cudaStreamSynchronize(plan->last)) != cudaSuccess) return from_cuda(e);
  const uint32_t P = plan->w.P;
  std::vector<unsigned long long> t((size_t)P * 2);
  if ((e = cudaMemcpy(t.data(), plan->w.ptime, t.size() * 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return from_cuda(e);
  for (uint32_t p = 0; p < P && p < cap; ++p)
    busy_ms[p] = t[2 * (size_t)p + 1] >= t[2 * (size_t)p] ? (float)((t[2 * (size_t)p + 1] - t[2 * (size_t)p]) * 1e-6)
                                                          : 0.f;
  if (count) *count = P;
  return GT_OK;
}

gt_status gt_transpose_u64(uint64_t n_rows, uint64_t n_cols, uint64_t n_edges, const uint64_t *row_ptr,
                           const uint64_t *col_idx, const float *vals, uint64_t *col_ptr, uint64_t *row_idx,
                           float *vals_out, void *stream) {
  if (!row_ptr || !col_ptr) return GT_ERR_INVALID_ARG;
  if (n_edges > 0 && (!col_idx || !row_idx)) return GT_ERR_INVALID_ARG;
  if ((vals == nullptr) != (vals_out == nullptr)) return GT_ERR_INVALID_ARG;
  if ((n_rows == 0 || n_cols == 0) && n_edges != 0) return GT_ERR_INVALID_ARG;
  if (n_edges > 0xFFFFFFFFull || n_cols == ~0ull) return GT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (n_rows == 0 || n_cols == 0) {
    if ((e = cudaMemsetAsync(col_ptr, 0, (size_t)(n_cols + 1) * 8, s)) != cudaSuccess) return from_cuda(e);
    return from_cuda(cudaStreamSynchronize(s));
  }
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || (e = gt::configure_kernels(dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
    gt_status st = from_cuda(e);
    cudaGetLastError();
    return st;
  }
  gt::U64Work w;
  w.n_rows = n_rows;
  w.n_cols = n_cols;
  w.m = n_edges;
  w.num_sms = sms;
  w.row_ptr = row_ptr;
  w.col_idx = col_idx;
  w.vals = vals;
  w.col_ptr = col_ptr;
  w.row_idx = row_idx;
  w.vals_out = vals_out;
  // stream-ordered workspace, freed on the same stream
  const size_t m = n_edges ? (size_t)n_edges : 1, rows = (size_t)sms * 8;
  void *bufs[10] = {};
  const size_t sizes[10] = {m * 4, m * 4, m * 4, m * 4, m * 4, m * 4, m * 8, rows * 256 * 4, rows * 256 * 8, 16};
  gt_status st = GT_OK;
  for (int i = 0; i < 10 && st == GT_OK; ++i)
    if ((e = cudaMallocAsync(&bufs[i], sizes[i], s)) != cudaSuccess) st = from_cuda(e);
  if (st == GT_OK) {
    w.a_key = (uint32_t *)bufs[0], w.a_u = (uint32_t *)bufs[1], w.a_w = (uint32_t *)bufs[2];
    w.b_key = (uint32_t *)bufs[3], w.b_u = (uint32_t *)bufs[4], w.b_w = (uint32_t *)bufs[5];
    w.keys = (uint64_t *)bufs[6];
    w.table = (uint32_t *)bufs[7];
    w.offsets = (unsigned long long *)bufs[8];
    w.status = (uint32_t *)bufs[9];
    if ((e = cudaMemsetAsync(w.status, 0, 4, s)) != cudaSuccess || (e = gt::run_radix_u64(w, s)) != cudaSuccess)
      st = from_cuda(e);
  }
  uint32_t dstat = 0;
  if (st == GT_OK && (e = cudaMemcpyAsync(&dstat, w.status, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    st = from_cuda(e);
  for (void *b : bufs)
    if (b) cudaFreeAsync(b, s);
  e = cudaStreamSynchronize(s);
  if (st == GT_OK && e != cudaSuccess) st = from_cuda(e);
  cudaGetLastError();
  return st != GT_OK ? st : (gt_status)dstat;
}

gt_status gt_plan_host_timing(gt_plan plan, gt_host_timing *t) {
  if (!plan || !t) return GT_ERR_INVALID_ARG;
  memset(t, 0, sizeof(*t));
  const size_t c = plan->host_events.size();
  if (c == 0) return GT_OK;
  cudaError_t e;
  for (const auto &h : plan->host_events)
    if ((e = cudaEventSynchronize(h.out1)) != cudaSuccess) return from_cuda(e);
  // intervals relative to the first call's input start
  std::vector<double> a(c), b(c), d0(c), d1(c);
  cudaEvent_t base = plan->host_events[0].in0;
  for (size_t i = 0; i < c; ++i) {
    const auto &h = plan->host_events[i];
    float x[4];
    cudaEvent_t ev[4] = {h.in0, h.in1, h.out0, h.out1};
    for (int j = 0; j < 4; ++j)
      if ((e = cudaEventElapsedTime(&x[j], base, ev[j])) != cudaSuccess) return from_cuda(e);
    a[i] = x[0], b[i] = x[1], d0[i] = x[2], d1[i] = x[3];
  }
  // each direction's copies run one call after another on their own stream,
  // so the overlap is the sum of the pairwise interval intersections
  double h2d = 0, d2h = 0, ov = 0, end = 0;
  for (size_t i = 0; i < c; ++i) {
    h2d += b[i] - a[i];
    d2h += d1[i] - d0[i];
    if (d1[i] > end) end = d1[i];
    for (size_t j = 0; j < c; ++j) {
      const double lo = a[i] > d0[j] ? a[i] : d0[j], hi = b[i] < d1[j] ? b[i] : d1[j];
      if (hi > lo) ov += hi - lo;
    }
  }
  t->calls = (uint32_t)c;
  t->h2d_ms = (float)(h2d / (double)c);
  t->d2h_ms = (float)(d2h / (double)c);
  t->overlap_ms = (float)(ov / (double)c);
  t->span_ms = (float)end;
  return GT_OK;
}

gt_status gt_plan_host_wait(gt_plan plan) {
  if (!plan) return GT_ERR_INVALID_ARG;
  for (cudaStream_t q : {plan->in_stream, plan->copy_stream}) {
    if (!q) continue;
    cudaError_t e = cudaStreamSynchronize(q);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return gt_plan_status(plan);
}

void gt_plan_destroy(gt_plan plan) {
  if (!plan) return;
  if (plan->last) cudaStreamSynchronize(plan->last);
  if (plan->copy_stream) {
    cudaStreamSynchronize(plan->in_stream);
    cudaStreamSynchronize(plan->copy_stream);
    for (cudaEvent_t x : {plan->ev_computed, plan->ev_copied[0], plan->ev_copied[1], plan->ev_inputs_read[0],
                          plan->ev_inputs_read[1], plan->ev_inputs_in})
      if (x) cudaEventDestroy(x);
    cudaStreamDestroy(plan->in_stream);
    cudaStreamDestroy(plan->copy_stream);
  }
  drop_events(plan);
  plan_free_ws(plan);
  for (int i = 0; i < plan->nhost; ++i) cudaFree(plan->host_allocs[i]);
  delete plan;
}

}  // extern "C"
