// Host-side view of a plan's device workspace and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gt.h"

namespace gt {

// Columns of a batch descriptor's matrix (n_cols == 0: a graph, n_vertices x n_vertices).
__host__ __device__ inline uint32_t desc_cols(const gt_graph_desc &d) { return d.n_cols ? d.n_cols : d.n_vertices; }

constexpr uint32_t kFreqBins = 1u << 16;   // sample-frequency histogram bins
constexpr uint32_t kTieCap = 8192;         // tie candidates kept at the threshold
constexpr uint32_t kScanTile = 4096;       // elements per decoupled-look-back tile
constexpr uint32_t kSortSmemCap = 2048;    // longest list sorted in one CTA's shared memory
constexpr uint32_t kMidCap = 256;          // longest list sorted in one warp's shared-memory slice
constexpr uint32_t kWarpSortCap = 32;      // longest list sorted in one warp's registers

// Entries of the sort worklists (mid | big | large regions) for m edges.
inline uint64_t worklist_entries(uint64_t m) {
  return m / (kWarpSortCap + 1) + m / (kMidCap + 1) + m / (kSortSmemCap + 1) + 3;
}

struct DevWork {
  // sizes and derived launch shape: n columns (destinations: col_ptr has n + 1
  // entries, keys and degree arrays span [0, n)), n_rows rows (row_ptr has
  // n_rows + 1 entries, row_idx values span [0, n_rows)); a graph has n_rows == n
  uint32_t n = 0;
  uint32_t n_rows = 0;
  uint64_t m = 0;
  int has_vals = 0;
  uint32_t kmax = 0, tlog2 = 0, W = 0, G = 0, P = 0;
  uint64_t psize = 0;
  uint32_t ns = 0, ts_log2 = 0;
  uint32_t ntiles = 0;
  uint32_t big_cap = 0;
  int flag_mode = 0;  // split-row duplicate ordering via row_idx bit 31 (weighted, n_rows <= 2^31)
  int staged = 0;     // bulk-copy staging of col_idx/vals tiles
  uint32_t stage_edges = 0;
  uint32_t smem_count = 0, smem_scatter = 0;
  int num_sms = 0;
  // buffers (device)
  uint32_t *deg = nullptr;                   // [n]
  unsigned long long *cursor = nullptr;      // [n]
  uint32_t *hdv_cnt = nullptr;               // [P * kmax]
  uint32_t *hdv_ids = nullptr;               // [kmax]
  unsigned long long *hdv_start = nullptr;   // [kmax]
  uint32_t *hkeys = nullptr;                 // [2^tlog2]
  uint16_t *hvals = nullptr;                 // [2^tlog2]
  unsigned long long *part = nullptr;        // [P + 1]
  unsigned long long *scan_state = nullptr;  // [ntiles]
  uint32_t *status = nullptr;                // [1]
  uint32_t *meta = nullptr;                  // [kMetaCount]
  unsigned long long *meta64 = nullptr;      // [4]
  uint32_t *skeys = nullptr, *scnt = nullptr;  // [2^ts_log2]
  uint32_t *fhist = nullptr;                   // [kFreqBins]
  uint32_t *cand = nullptr;                    // [kmax]
  uint32_t *ties = nullptr;                    // [kTieCap]
  uint32_t *biglist = nullptr;                 // [big_cap]
  int steal = 0;                               // two-phase Step 3: heads, then tails claimed by free warps
  unsigned long long *part2 = nullptr;         // [2P + 1] head / tail bounds (steal only)
  uint32_t *steal_next = nullptr;              // [1] next tail to claim (steal only)
  int ptimes = 0;                              // record Step 3's per-partition start/end times
  unsigned long long *ptime = nullptr;         // [2 * P] global-timer ns (ptimes only)
  // HLH, [m] entries: weighted graphs keep LDV entries here as u64 (value bits
  // << 32 | source, bit 31 of the source tagging split rows) until the LDV sort
  // moves them to the outputs; the long-list radix sort uses it as its second buffer.
  void *scratch = nullptr;
  // radix method
  int method = 0;
  uint32_t rG = 0;                            // persistent CTAs of the digit passes
  uint32_t r_items = 16;                      // elements per thread of a downsweep tile (8 or 16)
  int r_bulk = 0;                             // bulk-copy staged downsweep (two 256-thread CTAs per SM)
  uint32_t r_dcap = 8;                        // widest digit of a pass (4..8)
  uint32_t *r_a_key = nullptr, *r_a_u = nullptr, *r_a_w = nullptr;  // [m] ping buffer
  uint32_t *r_b_key = nullptr;                // [m] keys of the pong buffer (u/w live in the outputs)
  uint32_t *r_b_sv = nullptr;                 // weighted: [2m] interleaved (source, value) pairs of the pong
                                              // buffer's middle passes (the last pass writes the outputs)
  uint32_t *r_long = nullptr;                 // rows longer than the window expansion handles
  unsigned long long *r_gaps = nullptr;       // [1 + 2 * r_gap_cap]: count, then (lo << 32 | hi, value) ranges
  uint32_t r_gap_cap = 0;                     // long col_ptr ranges listed per call
  uint32_t *r_nlong = nullptr;                // [1] (zeroed per call)
  uint32_t *r_table = nullptr;                // [rG][256]
  unsigned long long *r_offsets = nullptr;    // [rG][256]
  // partitioned HLH (part_bits > 0): the edges bucketed stably by the top
  // part_bits bits of the destination, as (destination, source, value) arrays
  // [m]; Steps 0-3 and the LDV sort read them in place of the CSR.  The row
  // expansion writes its sources to r_a_u; r_long / r_nlong / r_table /
  // r_offsets serve the bucketing pass.
  uint32_t part_bits = 0;
  uint32_t *q_key = nullptr, *q_u = nullptr, *q_w = nullptr;
  // HDV insertion points over many partitions: hdv_q > 1 slices of
  // partitions, each slice's per-HDV total and then starting point in
  // hdv_psum [hdv_q][kmax]
  uint32_t hdv_q = 1;
  unsigned long long *hdv_psum = nullptr;
};

struct Problem {
  const uint64_t *row_ptr;
  const uint32_t *col_idx;
  const float *vals;
  uint64_t *col_ptr;
  uint32_t *row_idx;
  float *vals_out;
  // if set: recorded on the stream once no later kernel of the call reads
  // row_ptr, col_idx or vals (the next call's inputs may then be copied in)
  cudaEvent_t inputs_read = nullptr;
};

// Events recorded between the steps of one call (null = not timed).
struct StepEvents {
  cudaEvent_t ev[6];
  cudaEvent_t down[8];  // radix: around each downsweep launch (up to 4 passes)
  uint32_t ndown = 0;
  cudaEvent_t part[2];  // partitioned HLH: around the expansion and bucketing pass
  int has_part = 0;
};

// Enqueues the whole transposition on `stream`.  Returns cudaSuccess or the
// first launch error; *launches receives the number of kernels enqueued.
cudaError_t run_transpose(const DevWork &w, const gt_config &cfg, const Problem &pb, cudaStream_t stream,
                          StepEvents *events, uint32_t *launches);

// Radix method: enqueues the row expansion, the digit passes and col_ptr
// from the sorted keys (w.r_nlong and the gap count must be zeroed).
// Partitioned HLH: expands the rows into w.r_a_u and buckets the edges stably
// by the top w.part_bits bits of the destination (one digit pass of the radix
// method) into w.q_key / w.q_u / w.q_w.  Reports bad row pointers and
// out-of-range destinations in w.status.
cudaError_t run_partition(const DevWork &w, const Problem &pb, cudaStream_t stream, uint32_t *launches);
cudaError_t run_radix(const DevWork &w, const Problem &pb, cudaStream_t stream, uint32_t *launches,
                      StepEvents *events);

// 64-bit vertex IDs: sizes, the caller's arrays and a stream-ordered
// workspace (two sets of key-half / payload arrays, the sorted keys, the
// digit tables and a status word).
struct U64Work {
  uint64_t n_rows = 0, n_cols = 0, m = 0;
  int num_sms = 0;
  const uint64_t *row_ptr = nullptr, *col_idx = nullptr;
  const float *vals = nullptr;
  uint64_t *col_ptr = nullptr, *row_idx = nullptr;
  float *vals_out = nullptr;
  uint32_t *a_key = nullptr, *a_u = nullptr, *a_w = nullptr, *b_key = nullptr, *b_u = nullptr, *b_w = nullptr;
  uint64_t *keys = nullptr;
  uint32_t *table = nullptr;
  unsigned long long *offsets = nullptr;
  uint32_t *status = nullptr;
};

cudaError_t run_radix_u64(const U64Work &w, cudaStream_t s);

// The arguments of one batch call, in device memory (written by a small
// kernel before the captured sequence, which reads them).
struct BatchCall {
  const gt_graph_desc *descs;  // device, n_graphs entries
  int32_t *status;             // device, n_graphs per-graph gt_status codes, or null
  uint32_t n_graphs;
};

// A batch plan's limits and sub-batch rule, passed to the layout kernel.
struct BatchLimitsDev {
  uint32_t max_graphs, max_cols;
  uint64_t max_graph_edges, max_edges, max_cols_total;
  uint64_t cap_e, cap_v;  // sub-batch slot = eoff / cap_e + voff / cap_v + g / cap_g
  uint32_t cap_g, slots;
  int has_vals;
};

// One sub-batch of a call: graphs [g0, g0 + ng), laid out by k_b_layout.
struct BatchSlot {
  const gt_graph_desc *descs;                    // the call's descriptors + g0
  int32_t *gstatus;                              // the call's status array + g0, or null
  const uint32_t *gx;                            // excluded graphs (nonzero) + g0
  const unsigned long long *eoff, *voff, *woff;  // the call's prefix sums + g0 (entries g0 .. g0 + ng)
  unsigned long long e0, v0, w0;                 // eoff[g0], voff[g0], woff[g0]
  unsigned long long m, nv, windows;             // union edges, columns, 32-row windows
  uint32_t g0, ng;
};

struct BatchTotals {
  uint64_t n_edges;
  uint32_t n_graphs, slots_used;
};

struct BatchWork {
  int has_vals = 0;
  int num_sms = 0;
  uint32_t vbits = 1, passes = 1, dbits = 1;
  uint64_t cap_edges = 0;                                       // union edges one sub-batch may hold
  BatchLimitsDev lim{};
  uint32_t *a_key = nullptr, *a_u = nullptr, *a_w = nullptr;  // [cap_edges]
  uint32_t *b_key = nullptr, *b_u = nullptr, *b_w = nullptr;  // [cap_edges]
  unsigned long long *ucp = nullptr;                            // [columns of one sub-batch + 1]
  uint32_t *table = nullptr;                                    // [rows][256]
  unsigned long long *offsets = nullptr;                        // [rows][256]
  uint32_t *long_g = nullptr, *long_r = nullptr, *n_long = nullptr;
  uint32_t long_cap = 0;
  unsigned long long *gaps = nullptr;  // [1 + 2 * gap_cap] long col_ptr ranges
  uint32_t gap_cap = 0;
  uint32_t *status = nullptr;
  BatchCall *call = nullptr;
  unsigned long long *eoff = nullptr, *voff = nullptr, *woff = nullptr;  // [max_graphs + 1]
  uint32_t *gx = nullptr;                                                 // [max_graphs]
  BatchSlot *slots = nullptr;                                             // [lim.slots]
  BatchTotals *totals = nullptr;
};

// Stores a call's arguments for the captured sequence; lays the call out.
cudaError_t launch_batch_call(BatchCall *call, const gt_graph_desc *descs, int32_t *status, uint32_t n_graphs,
                              cudaStream_t s);
cudaError_t launch_batch_layout(const BatchWork &bw, cudaStream_t s);
// The kernels of one sub-batch slot (sizes read on the device).
cudaError_t run_radix_batch(const BatchWork &bw, uint32_t slot, cudaStream_t s, uint32_t *launches);

// Exclusive look-back scan (Step 2) as a separate launch; row_ptr may be null
// (no row-pointer validation); cursor may be null.
cudaError_t launch_scan(const uint32_t *deg, uint32_t n, uint64_t m, const uint64_t *row_ptr, uint64_t *col_ptr,
                        unsigned long long *cursor, unsigned long long *state, uint32_t ntiles, uint32_t *meta,
                        uint32_t *status, cudaStream_t s);

// Shared-memory bytes needed by the count / scatter kernels for a shape.
uint32_t smem_count_bytes(uint32_t W, uint32_t kmax, uint32_t tlog2, int staged, uint32_t stage_edges,
                          int has_vals);
uint32_t smem_scatter_bytes(uint32_t W, uint32_t kmax, uint32_t tlog2, int staged, uint32_t stage_edges,
                            int has_vals);

// Maps a CUDA error to a gt_status and records its text for
// gt_last_cuda_error() (cudaSuccess -> GT_OK).
gt_status from_cuda(cudaError_t e);

// Raises the dynamic shared-memory limits of the kernels, once per device
// (the current device must be `device`; thread-safe).
cudaError_t configure_kernels(int device);

}  // namespace gt
