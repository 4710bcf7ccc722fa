// C ABI of batch plans: many independent graphs transposed by the radix
// method over their union.  A plan is sized by limits; every call passes its
// own device descriptor array, graph count and per-graph status array, which
// kernels read at run time: a layout kernel splits the call into sub-batches
// (runs of graphs of bounded size), and each sub-batch slot runs the same
// kernel sequence on the sizes the layout wrote.  The whole sequence is
// captured once into a CUDA graph and replayed by every later call.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "gt.h"
#include "gt_device.cuh"
#include "gt_internal.h"

struct gt_batch_plan_s {
  gt::BatchWork bw;
  gt_batch_limits lim;
  gt_config cfg;
  int device = 0;
  cudaStream_t last = nullptr;
  bool use_graph = true;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  std::vector<void *> allocs;
  uint64_t ws_bytes = 0;
  uint32_t launches = 0;
};

namespace {

constexpr uint64_t kSubBatchEdges = 1ull << 31;    // union edges of one sub-batch
constexpr uint64_t kSubBatchCols = 1ull << 31;     // union columns of one sub-batch

uint32_t bits_of(uint64_t x) {  // bits needed for values 0..x
  uint32_t b = 0;
  while (b < 64 && (x >> b)) ++b;
  return b;
}

gt_status balloc(gt_batch_plan p, void **ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return GT_ERR_NO_MEMORY;
  }
  p->allocs.push_back(*ptr);
  p->ws_bytes += bytes;
  return GT_OK;
}

void bfree(gt_batch_plan p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
  p->exec_stream = nullptr;
  for (void *q : p->allocs) cudaFree(q);
  p->allocs.clear();
  p->ws_bytes = 0;
}

// The kernel sequence of one call (after its arguments were stored).
cudaError_t enqueue_all(gt_batch_plan p, cudaStream_t s, uint32_t *launches) {
  cudaError_t e = cudaMemsetAsync(p->bw.status, 0, 4, s);
  if (e != cudaSuccess) return e;
  if ((e = gt::launch_batch_layout(p->bw, s)) != cudaSuccess) return e;
  uint32_t nl = 1;
  for (uint32_t slot = 0; slot < p->bw.lim.slots; ++slot) {
    e = gt::run_radix_batch(p->bw, slot, s, &nl);
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches = nl;
  return cudaSuccess;
}

gt_status check_config(const gt_config *cfg, gt_config *out) {
  gt_config c;
  if (cfg) {
    c = *cfg;
    if (c.method != GT_METHOD_RADIX) return GT_ERR_INVALID_ARG;
    if (c.radix_tile != 0) return GT_ERR_INVALID_ARG;  // batches run the bulk-staged digit passes
  } else {
    memset(&c, 0, sizeof(c));
    c.method = GT_METHOD_RADIX;
    c.ctas_per_sm = 2;
    c.block_threads = 256;
    c.warp_edges = 4096;
    c.sample_permille = 10;
    c.flags = GT_FLAG_AGGREGATE;
  }
  if (c.batch_key_bits != 0 && (c.batch_key_bits < 16 || c.batch_key_bits > 32)) return GT_ERR_INVALID_ARG;
  if (c.batch_edges_log2 != 0 && (c.batch_edges_log2 < 16 || c.batch_edges_log2 > 31)) return GT_ERR_INVALID_ARG;
  *out = c;
  return GT_OK;
}

// Sub-batch rule, key width and workspace for the plan's limits and config.
gt_status plan_build(gt_batch_plan p, int has_vals) {
  const gt_batch_limits &L = p->lim;
  gt::BatchWork &bw = p->bw;
  const gt_config &c = p->cfg;
  bw.has_vals = has_vals ? 1 : 0;
  const uint32_t vbits = L.max_cols > 1 ? bits_of((uint64_t)L.max_cols - 1) : 1;
  // keys of at most 28 bits (four passes of 7-bit digits, whose runs fill
  // sectors better than 8-bit ones) unless the columns alone need more, or
  // the width the configuration asks for
  uint32_t cap_bits = vbits + 1 > 28 ? 32 : 28;
  if (c.batch_key_bits) cap_bits = c.batch_key_bits > vbits ? c.batch_key_bits : vbits;
  if (cap_bits > 32) cap_bits = 32;
  const uint32_t gfull = L.max_graphs > 1 ? bits_of((uint64_t)L.max_graphs - 1) : 0;
  const uint32_t gbits = gfull < cap_bits - vbits ? gfull : cap_bits - vbits;
  const uint32_t kbits = vbits + gbits;
  bw.vbits = vbits;
  bw.passes = (kbits + 7) / 8;
  bw.dbits = (kbits + bw.passes - 1) / bw.passes;
  // edges of one sub-batch: the whole batch plus one graph, within the cap
  uint64_t edge_cap = kSubBatchEdges;
  if (c.batch_edges_log2) edge_cap = 1ull << c.batch_edges_log2;
  if (const char *env = getenv("GT_BATCH_MAX_EDGES")) {  // smaller sub-batches (testing)
    unsigned long long v = strtoull(env, nullptr, 10);
    if (v > 0 && v < edge_cap) edge_cap = v;
  }
  // a sub-batch holds at least two of the largest graphs
  if (edge_cap < 2 * L.max_graph_edges) edge_cap = 2 * L.max_graph_edges;
  if (edge_cap > (1ull << 32)) return GT_ERR_UNSUPPORTED;
  uint64_t ws_edges = L.max_edges + L.max_graph_edges;
  if (ws_edges > edge_cap) ws_edges = edge_cap;
  if (ws_edges < 1) ws_edges = 1;
  const uint64_t cap_e = ws_edges > L.max_graph_edges ? ws_edges - L.max_graph_edges : 1;
  uint64_t ws_cols = L.max_cols_total + L.max_cols;
  if (ws_cols > kSubBatchCols) ws_cols = kSubBatchCols;
  const uint64_t cap_v = ws_cols > L.max_cols ? ws_cols - L.max_cols : 1;
  const uint32_t cap_g = 1u << gbits;
  const uint64_t slots = (L.max_edges + cap_e - 1) / cap_e + (L.max_cols_total + cap_v - 1) / cap_v +
                         ((uint64_t)L.max_graphs + cap_g - 1) / cap_g + 1;
  if (slots > 4096) return GT_ERR_UNSUPPORTED;
  bw.cap_edges = ws_edges;
  bw.lim.max_graphs = L.max_graphs;
  bw.lim.max_cols = L.max_cols;
  bw.lim.max_graph_edges = L.max_graph_edges;
  bw.lim.max_edges = L.max_edges;
  bw.lim.max_cols_total = L.max_cols_total;
  bw.lim.cap_e = cap_e;
  bw.lim.cap_v = cap_v;
  bw.lim.cap_g = cap_g;
  bw.lim.slots = (uint32_t)slots;
  bw.lim.has_vals = bw.has_vals;

  gt_status st;
  const size_t M = ws_edges, NV = ws_cols;
  bw.long_cap = (uint32_t)(M / 2049 + 1);
#define GT_BA(field, bytes)                                                  \
  do {                                                                       \
    if ((st = balloc(p, (void **)&bw.field, (bytes))) != GT_OK) return st; \
  } while (0)
  // weighted: each side is one block, (sources | values) as two u32 arrays
  // or the interleaved (source, value) pairs of the middle passes
  // (the value halves start on a 16-byte boundary: bulk copies read them)
  const size_t M4 = (M + 3) & ~(size_t)3;
  GT_BA(a_key, M * 4);
  GT_BA(a_u, has_vals ? M4 * 8 : M * 4);
  GT_BA(b_key, M * 4);
  GT_BA(b_u, has_vals ? M4 * 8 : M * 4);
  if (has_vals) {
    bw.a_w = bw.a_u + M4;
    bw.b_w = bw.b_u + M4;
  }
  GT_BA(ucp, (NV + 1) * 8);
  const size_t rows = (size_t)bw.num_sms * 8u;  // bulk passes: 2 CTAs per SM x 2 upsweep CTAs (up to 4 x 2)
  GT_BA(table, rows * 256 * 4);
  GT_BA(offsets, rows * 256 * 8);
  bw.gap_cap = (uint32_t)(NV / 1024 + 2);
  GT_BA(gaps, (1 + 2 * (size_t)bw.gap_cap) * 8);
  GT_BA(long_g, (size_t)bw.long_cap * 4);
  GT_BA(long_r, (size_t)bw.long_cap * 4);
  GT_BA(n_long, 4);
  GT_BA(status, 4);
  GT_BA(call, sizeof(gt::BatchCall));
  GT_BA(eoff, ((size_t)L.max_graphs + 1) * 8);
  GT_BA(voff, ((size_t)L.max_graphs + 1) * 8);
  GT_BA(woff, ((size_t)L.max_graphs + 1) * 8);
  GT_BA(gx, (size_t)L.max_graphs * 4);
  GT_BA(slots, (size_t)bw.lim.slots * sizeof(gt::BatchSlot));
  GT_BA(totals, sizeof(gt::BatchTotals));
#undef GT_BA
  if (cudaMemset(bw.status, 0, 4) != cudaSuccess || cudaMemset(bw.totals, 0, sizeof(gt::BatchTotals)) != cudaSuccess)
    return GT_ERR_CUDA;
  return GT_OK;
}

}  // namespace

extern "C" {

gt_status gt_batch_limits_from_descs(uint32_t n_graphs, const gt_graph_desc *descs, gt_batch_limits *limits) {
  if (!limits || (n_graphs > 0 && !descs)) return GT_ERR_INVALID_ARG;
  memset(limits, 0, sizeof(*limits));
  limits->max_graphs = n_graphs ? n_graphs : 1;
  limits->max_cols = 1;
  for (uint32_t g = 0; g < n_graphs; ++g) {
    const gt_graph_desc &d = descs[g];
    const uint32_t cols = gt::desc_cols(d);
    if (cols > limits->max_cols) limits->max_cols = cols;
    if (d.n_edges > limits->max_graph_edges) limits->max_graph_edges = d.n_edges;
    limits->max_edges += d.n_edges;
    limits->max_cols_total += cols;
  }
  if (limits->max_cols_total == 0) limits->max_cols_total = 1;
  return GT_OK;
}

gt_status gt_batch_plan_create(gt_batch_plan *plan, const gt_batch_limits *limits, int has_vals, const gt_config *cfg,
                               void *stream) {
  (void)stream;
  if (!plan || !limits) return GT_ERR_INVALID_ARG;
  *plan = nullptr;
  if (limits->max_graphs == 0 || limits->max_cols == 0) return GT_ERR_INVALID_ARG;
  if (limits->max_graph_edges > limits->max_edges) return GT_ERR_INVALID_ARG;
  if (has_vals && limits->max_graph_edges > (1ull << 32)) return GT_ERR_UNSUPPORTED;
  gt_config c;
  gt_status st = check_config(cfg, &c);
  if (st != GT_OK) return st;
  gt_batch_plan p = new (std::nothrow) gt_batch_plan_s();
  if (!p) return GT_ERR_NO_MEMORY;
  p->cfg = c;
  p->lim = *limits;
  p->use_graph = (c.flags & GT_FLAG_NO_GRAPH) == 0;
  cudaError_t ce;
  if ((ce = cudaGetDevice(&p->device)) != cudaSuccess || (ce = gt::configure_kernels(p->device)) != cudaSuccess) {
    st = gt::from_cuda(ce);
    cudaGetLastError();
    delete p;
    return st;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  p->bw.num_sms = sms;
  if ((st = plan_build(p, has_vals)) != GT_OK) {
    bfree(p);
    delete p;
    return st;
  }
  *plan = p;
  return GT_OK;
}

gt_status gt_batch_plan_set_config(gt_batch_plan plan, const gt_config *cfg) {
  if (!plan || !cfg) return GT_ERR_INVALID_ARG;
  gt_config c;
  gt_status st = check_config(cfg, &c);
  if (st != GT_OK) return st;
  if (plan->last) cudaStreamSynchronize(plan->last);
  const int has_vals = plan->bw.has_vals;
  const int sms = plan->bw.num_sms;
  bfree(plan);
  plan->bw = gt::BatchWork();
  plan->bw.num_sms = sms;
  plan->cfg = c;
  plan->use_graph = (c.flags & GT_FLAG_NO_GRAPH) == 0;
  return plan_build(plan, has_vals);
}

gt_status gt_batch_plan_get_config(gt_batch_plan plan, gt_config *cfg) {
  if (!plan || !cfg) return GT_ERR_INVALID_ARG;
  *cfg = plan->cfg;
  return GT_OK;
}

gt_status gt_transpose_batched(gt_batch_plan plan, uint32_t n_graphs, const gt_graph_desc *d_descs,
                               gt_status *d_status, void *stream) {
  if (!plan) return GT_ERR_INVALID_ARG;
  if (n_graphs > plan->lim.max_graphs) return GT_ERR_UNSUPPORTED;
  if (n_graphs > 0 && !d_descs) return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  plan->last = s;
  cudaError_t e;
  // this call's arguments, where the captured kernels read them
  if ((e = gt::launch_batch_call(plan->bw.call, d_descs, (int32_t *)d_status, n_graphs, s)) != cudaSuccess)
    return gt::from_cuda(e);
  if (!plan->use_graph || s == nullptr) return gt::from_cuda(enqueue_all(plan, s, &plan->launches));
  if (!plan->exec || plan->exec_stream != s) {
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    plan->exec = nullptr;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      gt_status st = gt::from_cuda(e);
      cudaGetLastError();
      return st;
    }
    cudaError_t qe = enqueue_all(plan, s, &plan->launches);
    e = cudaStreamEndCapture(s, &graph);
    if (qe != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      gt_status st = gt::from_cuda(qe != cudaSuccess ? qe : e);
      cudaGetLastError();
      return st;
    }
    e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      plan->exec = nullptr;
      gt_status st = gt::from_cuda(e);
      cudaGetLastError();
      return st;
    }
    plan->exec_stream = s;
  }
  return gt::from_cuda(cudaGraphLaunch(plan->exec, s));
}

gt_status gt_batch_plan_status(gt_batch_plan plan) {
  if (!plan) return GT_ERR_INVALID_ARG;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(plan->last)) != cudaSuccess) return gt::from_cuda(e);
  uint32_t st = 0;
  if ((e = cudaMemcpy(&st, plan->bw.status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return gt::from_cuda(e);
  return (gt_status)st;
}

gt_status gt_batch_plan_info(gt_batch_plan plan, gt_batch_info *info) {
  if (!plan || !info) return GT_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  cudaError_t e;
  if (plan->last && (e = cudaStreamSynchronize(plan->last)) != cudaSuccess) return gt::from_cuda(e);
  gt::BatchTotals t;
  if ((e = cudaMemcpy(&t, plan->bw.totals, sizeof(t), cudaMemcpyDeviceToHost)) != cudaSuccess) return gt::from_cuda(e);
  info->n_graphs = t.n_graphs;
  info->sub_batches = t.slots_used;
  info->passes_max = plan->bw.passes;
  info->kernel_launches = plan->launches;
  info->n_edges = t.n_edges;
  info->workspace_bytes = plan->ws_bytes;
  info->slots = plan->bw.lim.slots;
  info->key_bits = plan->bw.vbits + (uint32_t)__builtin_ctz(plan->bw.lim.cap_g);
  info->sub_batch_edges = plan->bw.cap_edges;
  return GT_OK;
}

gt_status gt_batch_tune_grid_config(uint32_t index, gt_config *cfg) {
  // (union key bits, log2 of sub-batch edges): the key width sets the digit
  // width and pass count and the graphs per sub-batch; the edge cap sets the
  // sub-batch size (workspace) and count
  static const uint32_t kGrid[GT_BATCH_TUNE_GRID][2] = {{28, 31}, {32, 31}, {24, 31}, {28, 30}, {32, 30}, {28, 29}};
  if (!cfg || index >= GT_BATCH_TUNE_GRID) return GT_ERR_INVALID_ARG;
  gt_config c;
  check_config(nullptr, &c);
  c.batch_key_bits = kGrid[index][0];
  c.batch_edges_log2 = kGrid[index][1];
  *cfg = c;
  return GT_OK;
}

gt_status gt_batch_plan_tune(gt_batch_plan plan, uint32_t n_graphs, const gt_graph_desc *d_descs,
                             gt_status *d_status, uint32_t reps, float *table_ms, uint32_t *chosen, void *stream) {
  if (!plan || reps == 0) return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t keep_flags = plan->cfg.flags;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce;
  if ((ce = cudaEventCreate(&e0)) != cudaSuccess || (ce = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return gt::from_cuda(ce);
  }
  float best = -1.f;
  uint32_t best_i = 0;
  gt_status st = GT_OK;
  for (uint32_t i = 0; i < GT_BATCH_TUNE_GRID; ++i) {
    float ms_i = -1.f;
    gt_config c;
    gt_batch_tune_grid_config(i, &c);
    c.flags = keep_flags;
    if (gt_batch_plan_set_config(plan, &c) == GT_OK &&
        gt_transpose_batched(plan, n_graphs, d_descs, d_status, stream) == GT_OK &&
        gt_batch_plan_status(plan) == GT_OK) {
      std::vector<float> t;
      for (uint32_t r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        if (gt_transpose_batched(plan, n_graphs, d_descs, d_status, stream) != GT_OK) break;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
      }
      if (t.size() == reps) {
        std::sort(t.begin(), t.end());
        ms_i = t[t.size() / 2];
      }
    }
    cudaGetLastError();
    if (table_ms) table_ms[i] = ms_i;
    if (ms_i >= 0.f && (best < 0.f || ms_i < best)) {
      best = ms_i;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.f) return GT_ERR_UNSUPPORTED;
  gt_config c;
  gt_batch_tune_grid_config(best_i, &c);
  c.flags = keep_flags;
  if ((st = gt_batch_plan_set_config(plan, &c)) != GT_OK) return st;
  // the outputs hold the batch's transposition under the chosen configuration
  if ((st = gt_transpose_batched(plan, n_graphs, d_descs, d_status, stream)) != GT_OK) return st;
  if (chosen) *chosen = best_i;
  return gt_batch_plan_status(plan);
}

void gt_batch_plan_destroy(gt_batch_plan plan) {
  if (!plan) return;
  if (plan->last) cudaStreamSynchronize(plan->last);
  bfree(plan);
  delete plan;
}

}  // extern "C"
