// C ABI of batch plans: many independent graphs transposed by the radix
// method over their union, split into sub-batches, the whole kernel sequence
// captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <stdlib.h>

#include <new>
#include <vector>

#include "gt.h"
#include "gt_device.cuh"
#include "gt_internal.h"

namespace gt {
}  // namespace gt

struct gt_batch_plan_s {
  gt::BatchWork bw;
  std::vector<gt::SubBatch> subs;
  gt_config cfg;
  int device = 0;
  cudaStream_t last = nullptr;
  bool use_graph = true;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  std::vector<void *> allocs;
  uint64_t ws_bytes = 0;
  uint32_t launches = 0;
  uint32_t n_graphs = 0;
  uint64_t total_m = 0;
  uint32_t passes_max = 0;
};

namespace {

constexpr uint64_t kSubBatchEdges = 1ull << 31;

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
  for (void *q : p->allocs) cudaFree(q);
  p->allocs.clear();
}

cudaError_t enqueue_all(gt_batch_plan p, cudaStream_t s, uint32_t *launches) {
  cudaError_t e = cudaMemsetAsync(p->bw.status, 0, 4, s);
  if (e != cudaSuccess) return e;
  uint32_t nl = 0;
  for (const gt::SubBatch &sb : p->subs) {
    e = gt::run_radix_batch(p->bw, sb, s, &nl);
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches = nl;
  return cudaSuccess;
}

}  // namespace

extern "C" {

gt_status gt_batch_plan_create(gt_batch_plan *plan, uint32_t n_graphs, const gt_graph_desc *descs, int has_vals,
                               const gt_config *cfg, void *stream) {
  (void)stream;
  if (!plan) return GT_ERR_INVALID_ARG;
  *plan = nullptr;
  if (n_graphs == 0 || !descs) return GT_ERR_INVALID_ARG;
  for (uint32_t g = 0; g < n_graphs; ++g) {
    const gt_graph_desc &d = descs[g];
    if (d.n_vertices == 0 || !d.row_ptr || !d.col_ptr) return GT_ERR_INVALID_ARG;
    if (d.n_edges > 0 && (!d.col_idx || !d.row_idx)) return GT_ERR_INVALID_ARG;
    if (has_vals && (!d.vals || !d.vals_out)) return GT_ERR_INVALID_ARG;
    if (!has_vals && (d.vals || d.vals_out)) return GT_ERR_INVALID_ARG;
    if (has_vals && d.n_edges > (1ull << 32)) return GT_ERR_UNSUPPORTED;
  }
  gt_config c;
  if (cfg) {
    c = *cfg;
    if (c.method != GT_METHOD_RADIX) return GT_ERR_INVALID_ARG;
    if (c.radix_tile != 0 && c.radix_tile != 2048 && c.radix_tile != 4096) return GT_ERR_INVALID_ARG;
    if (c.ctas_per_sm < 1 || c.ctas_per_sm > 32) return GT_ERR_INVALID_ARG;
  } else {
    memset(&c, 0, sizeof(c));
    c.method = GT_METHOD_RADIX;
    c.ctas_per_sm = 4;
    c.block_threads = 256;
    c.warp_edges = 4096;
    c.sample_permille = 10;
    c.flags = GT_FLAG_AGGREGATE;
  }
  gt_batch_plan p = new (std::nothrow) gt_batch_plan_s();
  if (!p) return GT_ERR_NO_MEMORY;
  p->cfg = c;
  p->n_graphs = n_graphs;
  p->use_graph = (c.flags & GT_FLAG_NO_GRAPH) == 0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return GT_ERR_CUDA;
  }
  if (gt::configure_kernels(p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return GT_ERR_CUDA;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  p->bw.has_vals = has_vals ? 1 : 0;
  p->bw.num_sms = sms;
  p->bw.rG = (uint32_t)sms * c.ctas_per_sm;
  p->bw.r_items = c.radix_tile == 2048 ? 8u : 16u;

  // split into sub-batches: bounded union size and key width
  uint64_t sub_cap = kSubBatchEdges;
  if (const char *env = getenv("GT_BATCH_MAX_EDGES")) {  // smaller sub-batches (testing)
    unsigned long long v = strtoull(env, nullptr, 10);
    if (v > 0 && v < sub_cap) sub_cap = v;
  }
  std::vector<uint32_t> starts;
  {
    uint32_t g = 0;
    while (g < n_graphs) {
      uint32_t g1 = g;
      uint64_t sm = 0, sn = 0;
      uint32_t maxn = 1;
      while (g1 < n_graphs) {
        const gt_graph_desc &d = descs[g1];
        const uint32_t nc = gt::desc_cols(d);  // keys and the union col_ptr span the columns
        const uint32_t nmax = nc > maxn ? nc : maxn;
        const uint32_t vb = bits_of(nmax - 1 ? nmax - 1 : 1);
        // keys of at most 28 bits (four passes of 7-bit digits, whose runs fill
        // sectors better than 8-bit ones) unless the columns alone need more
        const uint32_t cap = vb + 1 > 28 ? 32 : 28;
        const uint32_t keyw = vb + bits_of(g1 - g);
        const bool fits = sm + d.n_edges <= sub_cap && sn + nc < (1ull << 31) && keyw <= cap;
        if (g1 > g && !fits) break;
        sm += d.n_edges;
        sn += nc;
        maxn = nmax;
        ++g1;
      }
      starts.push_back(g);
      g = g1;
    }
    starts.push_back(n_graphs);
  }
  // device descriptors and offsets
  gt_status st;
  gt_graph_desc *d_descs = nullptr;
  if ((st = balloc(p, (void **)&d_descs, sizeof(gt_graph_desc) * n_graphs)) != GT_OK) goto fail;
  if (cudaMemcpy(d_descs, descs, sizeof(gt_graph_desc) * n_graphs, cudaMemcpyHostToDevice) != cudaSuccess) {
    st = GT_ERR_CUDA;
    goto fail;
  }
  {
    uint64_t max_m = 0, max_nv = 0;
    for (size_t i = 0; i + 1 < starts.size(); ++i) {
      gt::SubBatch sb;
      sb.g0 = starts[i];
      sb.ng = starts[i + 1] - starts[i];
      std::vector<unsigned long long> eoff(sb.ng + 1), voff(sb.ng + 1), woff(sb.ng + 1);
      uint32_t maxn = 1;
      eoff[0] = voff[0] = woff[0] = 0;
      for (uint32_t j = 0; j < sb.ng; ++j) {
        const gt_graph_desc &d = descs[sb.g0 + j];
        const uint32_t nc = gt::desc_cols(d);
        eoff[j + 1] = eoff[j] + d.n_edges;
        voff[j + 1] = voff[j] + nc;                        // union column space
        woff[j + 1] = woff[j] + (d.n_vertices + 31) / 32;  // 32-row windows of the expansion
        if (nc > maxn) maxn = nc;
      }
      sb.m = eoff[sb.ng];
      sb.nv = (uint32_t)voff[sb.ng];
      sb.windows = woff[sb.ng];
      sb.vbits = bits_of(maxn - 1);
      if (sb.vbits == 0) sb.vbits = 1;
      const uint32_t kbits = sb.vbits + bits_of(sb.ng - 1);
      sb.passes = (kbits + 7) / 8;
      sb.dbits = (kbits + sb.passes - 1) / sb.passes;
      if (sb.passes > p->passes_max) p->passes_max = sb.passes;
      sb.descs = d_descs + sb.g0;
      unsigned long long *offs = nullptr;
      if ((st = balloc(p, (void **)&offs, sizeof(unsigned long long) * 3 * (sb.ng + 1))) != GT_OK) goto fail;
      sb.eoff = offs;
      sb.voff = offs + (sb.ng + 1);
      sb.woff = offs + 2 * (sb.ng + 1);
      if (cudaMemcpy(sb.eoff, eoff.data(), 8 * (sb.ng + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(sb.voff, voff.data(), 8 * (sb.ng + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(sb.woff, woff.data(), 8 * (sb.ng + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        st = GT_ERR_CUDA;
        goto fail;
      }
      p->subs.push_back(sb);
      p->total_m += sb.m;
      if (sb.m > max_m) max_m = sb.m;
      if (sb.nv > max_nv) max_nv = sb.nv;
    }
    gt::BatchWork &bw = p->bw;
    const size_t M = max_m ? max_m : 1, NV = max_nv ? max_nv : 1;
    bw.long_cap = (uint32_t)(M / 2049 + 1);
#define GT_BA(field, bytes)                                                  \
  do {                                                                       \
    if ((st = balloc(p, (void **)&bw.field, (bytes))) != GT_OK) goto fail; \
  } while (0)
    GT_BA(a_key, M * 4);
    GT_BA(a_u, M * 4);
    GT_BA(b_key, M * 4);
    GT_BA(b_u, M * 4);
    if (has_vals) {
      GT_BA(a_w, M * 4);
      GT_BA(b_w, M * 4);
    }
    GT_BA(ucp, (NV + 1) * 8);
    // rows: the register passes' CTAs, or the bulk passes' CTAs (up to 4 per SM) x 2 sub-CTAs
    const size_t rows = bw.rG > (uint32_t)bw.num_sms * 8u ? bw.rG : (size_t)bw.num_sms * 8u;
    GT_BA(table, rows * 256 * 4);
    GT_BA(offsets, rows * 256 * 8);
    bw.gap_cap = (uint32_t)(NV / 1024 + 2);
    GT_BA(gaps, (1 + 2 * (size_t)bw.gap_cap) * 8);
    GT_BA(long_g, (size_t)bw.long_cap * 4);
    GT_BA(long_r, (size_t)bw.long_cap * 4);
    GT_BA(n_long, 4);
    GT_BA(status, 4);
    GT_BA(meta, gt::kMetaCount * 4);
#undef GT_BA
    if (cudaMemset(bw.status, 0, 4) != cudaSuccess) {
      st = GT_ERR_CUDA;
      goto fail;
    }
  }
  *plan = p;
  return GT_OK;
fail:
  bfree(p);
  delete p;
  return st;
}

gt_status gt_transpose_batched(gt_batch_plan plan, void *stream) {
  if (!plan) return GT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  plan->last = s;
  cudaError_t e;
  if (!plan->use_graph || s == nullptr) {
    e = enqueue_all(plan, s, &plan->launches);
    return e == cudaSuccess ? GT_OK : GT_ERR_CUDA;
  }
  if (!plan->exec || plan->exec_stream != s) {
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    plan->exec = nullptr;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      cudaGetLastError();
      return GT_ERR_CUDA;
    }
    cudaError_t qe = enqueue_all(plan, s, &plan->launches);
    e = cudaStreamEndCapture(s, &graph);
    if (qe != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return GT_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      plan->exec = nullptr;
      cudaGetLastError();
      return GT_ERR_CUDA;
    }
    plan->exec_stream = s;
  }
  e = cudaGraphLaunch(plan->exec, s);
  return e == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}

gt_status gt_batch_plan_status(gt_batch_plan plan) {
  if (!plan) return GT_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(plan->last) != cudaSuccess) return GT_ERR_CUDA;
  uint32_t st = 0;
  if (cudaMemcpy(&st, plan->bw.status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GT_ERR_CUDA;
  return (gt_status)st;
}

gt_status gt_batch_plan_info(gt_batch_plan plan, gt_batch_info *info) {
  if (!plan || !info) return GT_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->n_graphs = plan->n_graphs;
  info->sub_batches = (uint32_t)plan->subs.size();
  info->passes_max = plan->passes_max;
  info->kernel_launches = plan->launches;
  info->n_edges = plan->total_m;
  info->workspace_bytes = plan->ws_bytes;
  return GT_OK;
}

void gt_batch_plan_destroy(gt_batch_plan plan) {
  if (!plan) return;
  if (plan->last) cudaStreamSynchronize(plan->last);
  bfree(plan);
  delete plan;
}

}  // extern "C"
