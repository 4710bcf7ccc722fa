/*
 * gt.h -- C ABI of the GB300 graph-transposition library (libgt.so).
 *
 * Graph transposition (Sec. II-A of "On Optimizing Locality of Graph
 * Transposition on Modern Architectures", PoTra) turns the CSR of a directed
 * graph with n vertices and m edges (out-edge offsets row_ptr[n+1] and
 * destination IDs col_idx[m], optionally one f32 value per edge) into its CSC
 * (in-edge offsets col_ptr[n+1], source IDs row_idx[m], values carried
 * bit-for-bit).  Every CSC list comes out in ascending source order, and
 * parallel edges with the same (source, destination) keep their CSR order:
 * the result is the stable sort of the CSR edge sequence by destination.
 * The result never depends on the gt_config used (except with
 * GT_FLAG_UNSORTED, which drops the order within lists).
 *
 * Method (all steps run in CUDA kernels for sm_103a; there is no CPU path):
 *   Step 0  (Sec. IV-C, Step 0)  sample ceil(n * sample_permille / 1000)
 *           random positions of col_idx, take the most frequent destinations
 *           as high-degree vertices (HDV), build an open-addressing hash table
 *           mapping HDV IDs to a compact index (Sec. IV-A).
 *   Step 1  (Algorithm 2, Step 1)  in-degree count; HDV edges go to counters
 *           private to a warp in shared memory, low-degree (LDV) edges to
 *           global atomics aggregated per warp.
 *   Step 2  (Algorithm 2, Step 2)  per-warp HDV counts are scanned into
 *           per-warp insertion points, and one single-pass decoupled
 *           look-back scan turns the degrees into col_ptr.
 *   Step 3  (Algorithm 2, Step 3)  each warp revisits the same edges (the
 *           part2tid rule); HDV edges take deterministic slots from its
 *           private insertion points, LDV edges take slots from atomic
 *           cursors (Algorithm 1, Step 3).
 *   Sort    (Sec. II-B, optional sort)  LDV lists are sorted by source.
 * A second method (GT_METHOD_RADIX) computes the same bytes as a stable LSD
 * radix sort by destination; gt_config.method selects it.
 *
 * Conventions
 *   - Every array argument of gt_transpose* is a DEVICE pointer owned by the
 *     caller (inputs are read only; outputs are written completely).  The
 *     plan owns only its workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that enqueue work return once it is enqueued; errors
 *     the host can see are returned at once, errors only the device can see
 *     (out-of-range ID, bad row_ptr, timed-out wait) are latched in the plan's
 *     status word and read with gt_plan_status() after the work completes.
 *     Outputs are unspecified when any error is reported.
 *   - Vertex IDs are u32 (n <= 2^32 - 1); edge offsets are u64
 *     (m <= 2^32 for weighted graphs, see gt_plan_create).
 *   - Rectangular sparse matrices (n_rows x n_cols, gt_plan_create_rect)
 *     follow the same definition: row_ptr has n_rows + 1 entries, col_idx
 *     values lie in [0, n_cols), col_ptr has n_cols + 1 entries and row_idx
 *     holds row IDs.  A graph is the square case n_rows = n_cols = n.
 *   - A plan may be used by one stream at a time.
 */
#ifndef GT_H_
#define GT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gt_status {
    GT_OK = 0,
    GT_ERR_INVALID_ARG = 1,   /* null pointer, size mismatch, bad config field   */
    GT_ERR_OUT_OF_RANGE = 2,  /* some col_idx[e] >= n_cols (device-detected)      */
    GT_ERR_BAD_ROW_PTR = 3,   /* row_ptr[0] != 0, decreasing, row_ptr[n_rows] != m */
    GT_ERR_NO_MEMORY = 4,     /* workspace allocation failed                       */
    GT_ERR_CUDA = 5,          /* a CUDA runtime call failed                        */
    GT_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired                */
    GT_ERR_UNSUPPORTED = 7    /* size outside what the library handles             */
} gt_status;

/* Launch/method configuration.  Any valid configuration yields the same bytes. */
typedef struct gt_config {
    uint32_t hdv_k;           /* max number of HDV (0 = pure atomic, Algorithm 1)         */
    uint32_t table_log2;      /* log2 of hash-table slots; 2^table_log2 >= 2*hdv_k       */
    uint32_t block_threads;   /* threads per CTA for the count/scatter passes (64..1024, multiple of 32) */
    uint32_t ctas_per_sm;     /* CTAs per SM for the count/scatter (HLH) or digit (radix) passes (1..32) */
    uint32_t warp_edges;      /* target edges per warp partition (>= 32)                   */
    uint32_t stage_edges;     /* edges per bulk-copy stage per warp (0 = direct loads; else 128..4096, multiple of 128) */
    uint32_t sample_permille; /* sample size in 1/1000 of n (Sec. IV-C uses 10 = 1 %)     */
    uint32_t flags;           /* GT_FLAG_* bits                                            */
    uint32_t method;          /* GT_METHOD_*                                               */
    uint32_t radix_tile;      /* GT_METHOD_RADIX: 0 = bulk-copy staged 4096-edge tiles, two 256-thread
                                 CTAs per SM whatever ctas_per_sm says (needs 16-byte aligned arrays,
                                 else as 4096); 2048 or 4096 = register tiles of 256 threads,
                                 ctas_per_sm CTAs per SM */
    uint64_t seed;            /* seed of the sampling positions                            */
    uint32_t batch_key_bits;  /* batch plans: widest union key (graph, column) in bits, 16..32;
                                 0 = 28 (or 32 when the columns need more than 27 bits)       */
    uint32_t batch_edges_log2;/* batch plans: log2 of the union edges of one sub-batch, 16..31;
                                 0 = 31                                                          */
    uint32_t radix_digit_bits;/* GT_METHOD_RADIX: widest digit of a pass, 4..8 (0 = 8): the
                                 passes are ceil(key bits / radix_digit_bits) equal digits   */
    uint32_t partition_bits;  /* GT_METHOD_HLH: 0 = Steps 0-3 on the CSR as given; 1..8 = the
                                 partitioned (two-level) form: the edges are first bucketed,
                                 stably, by the top partition_bits bits of the destination
                                 (2^partition_bits destination ranges, capped at the column
                                 bits), then Steps 0-3 and the LDV sort run over the bucketed
                                 edge list in ranges of warp_edges edges taken in order, so the
                                 counters, cursors and partly written lists the GPU touches at
                                 any time belong to a few destination ranges and stay in L2.
                                 Needs stage_edges == 0 and no GT_FLAG_STEAL_TAILS; uses 12-16
                                 more bytes per edge of workspace.  Same output bytes.
                                 Weighted matrices with more than 2^31 rows run unpartitioned. */
} gt_config;

#define GT_FLAG_AGGREGATE 1u  /* aggregate LDV atomics across a warp (__match_any_sync) */
#define GT_FLAG_NO_GRAPH 2u   /* batches: launch kernels directly, no CUDA graph        */
/* GT_METHOD_HLH only: skip the LDV list sort; the lists of low-degree
 * destinations come out in arbitrary order (each holds the right multiset of
 * (source, value) pairs; HDV lists stay in edge order).  Unweighted entries
 * are written straight to row_idx; weighted ones go to the plan's scratch as
 * one 8-byte store each and a streaming pass copies them to row_idx and
 * vals_out.  This is the output of PoTra and Atomic GT as the paper times
 * them (Sec. V excludes the sort).  The radix method ignores it: its lists are
 * always sorted. */
#define GT_FLAG_UNSORTED 4u
/* GT_METHOD_HLH: record the start and end (global timer) of every warp
 * partition in Step 3, read with gt_plan_partition_times (Sec. V-F measures
 * Step 3's load imbalance between the threads' partitions). */
#define GT_FLAG_PARTITION_TIMES 8u
/* GT_METHOD_HLH: two-phase Step 3 (Sec. V-F).  Every warp partition is split
 * into a head (80 % of its edges) and a tail whose HDV counts and insertion
 * points Steps 1-2 keep apart; in Step 3 each warp scatters its own head, then
 * warps claim the tails one at a time from an atomic counter, so warps that
 * finish early take over the work of slow ones.  HDV slots stay deterministic
 * (each range keeps its own insertion points); the output bytes do not change.
 * Needs stage_edges == 0. */
#define GT_FLAG_STEAL_TAILS 16u

/* GT_METHOD_HLH: PoTra's hash-based LDV-HDV method (Algorithm 2; hdv_k = 0 is
 *   Atomic GT, Algorithm 1) with the LDV list sort.
 * GT_METHOD_RADIX: stable LSD radix sort of the CSR edge sequence by
 *   destination (ceil(bits / radix_digit_bits) passes of equal digits);
 *   streams the data once per digit, independent of vertex order.  Uses
 *   12-16 bytes per edge of extra workspace. */
#define GT_METHOD_HLH 0u
#define GT_METHOD_RADIX 1u

typedef struct gt_stats {
    uint32_t hdv_selected;    /* HDV actually selected by Step 0 (<= hdv_k)  */
    uint32_t partitions;      /* warp partitions of Steps 1 and 3            */
    uint64_t hdv_edges;       /* edges whose destination is an HDV (coverage numerator, Sec. IV-B) */
    uint64_t n_edges;         /* m                                           */
    uint32_t ldv_sorted_cols; /* LDV lists of length >= 2 that were sorted    */
    uint32_t large_cols;      /* of those, lists longer than one CTA's shared-memory sort */
    uint32_t kernel_launches; /* kernels the last gt_transpose enqueued       */
} gt_stats;

/* Average device time per gt_transpose call, per step, over the calls made
 * since timing was (re)enabled.  Measured with CUDA events recorded on the
 * caller's stream between the steps. */
typedef struct gt_timing {
    uint32_t calls;
    float sample_ms;   /* Step 0: sampling, HDV selection, hash table       */
    float count_ms;    /* Step 1: partition bounds + in-degree count         */
    float scan_ms;     /* Step 2: HDV insertion points + look-back scan      */
    float scatter_ms;  /* Step 3: scatter                                    */
    float sort_ms;     /* LDV list sort                                      */
    float total_ms;    /* GT_METHOD_RADIX: count_ms holds the row expansion, the
                          digit passes and col_ptr; the rest are 0           */
    float dominant_ms; /* average duration of one launch of the dominant
                          kernel: the scatter (HLH) or a digit downsweep (radix) */
    uint32_t dominant_launches; /* launches averaged                        */
    float partition_ms; /* partitioned HLH (gt_config.partition_bits > 0): the row
                           expansion and the destination bucketing pass, which run
                           before Step 0 (included in total_ms); else 0        */
} gt_timing;

typedef struct gt_plan_s *gt_plan;

/* Fills *cfg with the analytic default for a graph of this size (Eq. 1 sizing). */
gt_status gt_default_config(gt_config *cfg, uint32_t n_vertices, uint64_t n_edges);

/* Creates a plan for graphs with exactly n_vertices and n_edges.  has_vals != 0
 * reserves the extra workspace of weighted graphs.  cfg == NULL takes
 * gt_default_config.  The stream is used for workspace initialisation.
 * Weighted graphs need n_edges <= 2^32; unweighted need n_edges < 2^63. */
gt_status gt_plan_create(gt_plan *plan, uint32_t n_vertices, uint64_t n_edges, int has_vals,
                         const gt_config *cfg, void *stream);

/* Plan for an n_rows x n_cols sparse matrix with n_edges entries (CSR in,
 * CSC out; gt_plan_create(n) is gt_plan_create_rect(n, n)).  cfg == NULL
 * takes gt_default_config(cfg, n_cols, n_edges).  When n_rows or n_cols is
 * 0, n_edges must be 0; gt_transpose then zero-fills col_ptr and does not
 * read row_ptr.  Weighted matrices with the HLH method order split rows by a
 * tag bit in row_idx, which needs n_rows <= 2^31 (larger matrices fall back
 * to the untagged order, which is still stable). */
gt_status gt_plan_create_rect(gt_plan *plan, uint32_t n_rows, uint32_t n_cols, uint64_t n_edges, int has_vals,
                              const gt_config *cfg, void *stream);

/* Replaces the configuration (reallocating workspace if needed). Synchronous. */
gt_status gt_plan_set_config(gt_plan plan, const gt_config *cfg);
gt_status gt_plan_get_config(gt_plan plan, gt_config *cfg);

/* Enqueues the transposition (Steps 0-3 and the LDV sort) on `stream`.
 * row_ptr: u64[n_rows+1]; col_idx: u32[m]; vals: f32[m] or NULL;
 * col_ptr: u64[n_cols+1]; row_idx: u32[m]; vals_out: f32[m], NULL iff vals is NULL.
 * (n_rows = n_cols = n for a plan made by gt_plan_create.)
 * Output arrays must not overlap inputs.  Row pointers are validated on the
 * device (GT_ERR_BAD_ROW_PTR) and destinations range-checked (GT_ERR_OUT_OF_RANGE). */
gt_status gt_transpose(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx,
                       const float *vals, uint64_t *col_ptr, uint32_t *row_idx, float *vals_out,
                       void *stream);

/* gt_transpose for a graph no larger than the plan's (n_vertices <= the
 * plan's n, n_edges <= the plan's m), on the plan's workspace: one plan can
 * serve a stream of graphs of varying size. */
gt_status gt_transpose_sub(gt_plan plan, uint32_t n_vertices, uint64_t n_edges, const uint64_t *row_ptr,
                           const uint32_t *col_idx, const float *vals, uint64_t *col_ptr, uint32_t *row_idx,
                           float *vals_out, void *stream);

/* gt_transpose_sub for an n_rows x n_cols matrix no larger than the plan's
 * in each of the three sizes. */
gt_status gt_transpose_sub_rect(gt_plan plan, uint32_t n_rows, uint32_t n_cols, uint64_t n_edges,
                                const uint64_t *row_ptr, const uint32_t *col_idx, const float *vals,
                                uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, void *stream);

/* Same as gt_transpose on HOST arrays (pinned memory recommended): copies the
 * inputs to plan-owned device buffers, transposes, copies the outputs back and
 * synchronises the stream.  Returns the device status as well. */
gt_status gt_transpose_host(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx,
                            const float *vals, uint64_t *col_ptr, uint32_t *row_idx,
                            float *vals_out, void *stream);

/* Asynchronous gt_transpose_host: enqueues the transposition on `stream`,
 * its input copies on a stream the plan owns and its output copies on a
 * second one, and returns without waiting.  A call's input copies start as
 * soon as the previous call's transposition has stopped reading its device
 * inputs (after the first digit pass of the radix method; at the end of the
 * HLH method).  The plan keeps two device output sets when memory allows
 * (allocated on the first call) and uses them in turn, so a transposition
 * need not wait for the previous call's output copies: a loop of calls keeps
 * both copy directions and the SMs busy together.  Host buffers must stay
 * untouched (inputs) and unread (outputs) until gt_plan_host_wait returns;
 * calls that overwrite one set of host output buffers leave the last call's
 * CSC there.  gt_plan_host_wait waits for all outstanding calls and returns
 * the device status.  Calls on one plan use one stream. */
gt_status gt_transpose_host_async(gt_plan plan, const uint64_t *row_ptr, const uint32_t *col_idx,
                                  const float *vals, uint64_t *col_ptr, uint32_t *row_idx, float *vals_out,
                                  void *stream);
gt_status gt_plan_host_wait(gt_plan plan);

/* Copy timing of gt_transpose_host_async calls made while per-step timing is
 * enabled (gt_plan_enable_timing; up to 64 calls per enable), from CUDA
 * events recorded around each call's input copies (on the plan's input
 * stream) and output copies (on its output stream).  Synchronises those
 * events.  All fields are 0 when no call was recorded. */
typedef struct gt_host_timing {
    uint32_t calls;     /* calls recorded                                          */
    float h2d_ms;       /* average duration of one call's input copies              */
    float d2h_ms;       /* average duration of one call's output copies             */
    float overlap_ms;   /* average time per call with copies in both directions in
                           progress at once                                          */
    float span_ms;      /* first recorded input copy start to last output copy end  */
} gt_host_timing;
gt_status gt_plan_host_timing(gt_plan plan, gt_host_timing *timing);

/* The transposition (Sec. II-A) of a matrix with 64-bit vertex IDs, for more
 * than 2^32 - 1 rows or columns.  row_ptr: u64[n_rows+1]; col_idx: u64[m]
 * (< n_cols); vals: f32[m] or NULL; col_ptr: u64[n_cols+1]; row_idx: u64[m];
 * vals_out: f32[m], NULL iff vals is NULL -- all DEVICE arrays owned by the
 * caller.  Same output order as gt_transpose (the stable sort of the CSR edge
 * sequence by destination).  Method: the radix method's digit passes over
 * the two 32-bit halves of the keys, carrying the edge index, then a gather
 * of the sources (a search of row_ptr) and values, and col_ptr over the
 * 64-bit column space.  n_edges < 2^32.  The workspace (32 bytes per edge
 * plus a few MB) is allocated and freed stream-ordered on `stream`
 * (cudaMallocAsync).  Synchronises `stream` and returns the device status
 * (GT_ERR_BAD_ROW_PTR, GT_ERR_OUT_OF_RANGE). */
gt_status gt_transpose_u64(uint64_t n_rows, uint64_t n_cols, uint64_t n_edges, const uint64_t *row_ptr,
                           const uint64_t *col_idx, const float *vals, uint64_t *col_ptr, uint64_t *row_idx,
                           float *vals_out, void *stream);

/* Allocation-free variant of gt_transpose (no counterpart in the paper).
 * For callers that must not allocate device memory on the call path, e.g. a
 * host program whose pool already owns all device memory, or a latency-
 * critical loop that cannot take the synchronisation cudaMalloc/cudaFree may
 * cause.  The caller passes device inputs/outputs exactly as for
 * gt_transpose; the workspace comes from a fixed 64 MiB array that every GPU
 * loading this library holds until the process exits.  Graphs whose
 * workspace does not fit (roughly 12 bytes per vertex plus 4 bytes per edge,
 * 8 with values) return GT_ERR_UNSUPPORTED before anything is enqueued.
 * Runs the pure-atomic configuration, synchronises `stream`, and returns the
 * device status (CUDA failures: GT_ERR_CUDA with the text in
 * gt_last_cuda_error(); a call that fails after enqueueing work waits for it
 * before returning).  All calls share the array and it keeps the previous
 * call's contents: calls that overlap on the GPU race.  Every call looks up
 * the array's address in the current context; the first call in each CUDA
 * context also sets kernel limits and should come before any stream capture
 * on that device. */
gt_status gt_transpose_noalloc(uint32_t n_vertices, uint64_t n_edges, const uint64_t *row_ptr,
                               const uint32_t *col_idx, const float *vals, uint64_t *col_ptr,
                               uint32_t *row_idx, float *vals_out, void *stream);

/* ---- Batches: many independent graphs in one launch sequence ------------
 * (north-star addition "batching"; each graph's output is the transposition
 * of Sec. II-A, equal to gt_transpose's.)  A batch plan is sized by limits;
 * every gt_transpose_batched call passes its own DEVICE descriptor array,
 * graph count and DEVICE per-graph status array.  Kernels read them at run
 * time: a layout kernel checks every descriptor, lays the graphs out one after
 * another in a union edge / column space, and splits them into sub-batches
 * (runs of graphs with at most 2^batch_edges_log2 edges, 2^31 columns and
 * 2^(key bits - column bits) graphs); each sub-batch is transposed by the
 * radix method over the union key (local graph, column).  The kernel sequence
 * is captured once into a CUDA graph per stream and replayed by later calls,
 * so batches of any shape within the limits reuse one plan.  The output of
 * every graph equals gt_transpose's. */
typedef struct gt_graph_desc {
    uint32_t n_vertices;      /* rows (the vertices of a graph), >= 1                */
    uint32_t n_cols;          /* columns of a rectangular matrix; 0 = n_vertices    */
    uint64_t n_edges;
    const uint64_t *row_ptr;  /* device, n_vertices + 1 */
    const uint32_t *col_idx;  /* device, n_edges, values < columns */
    const float *vals;        /* device, n_edges, or NULL (all graphs alike) */
    uint64_t *col_ptr;        /* device, columns + 1 (output) */
    uint32_t *row_idx;        /* device, n_edges (output) */
    float *vals_out;          /* device, n_edges, NULL iff vals is NULL */
} gt_graph_desc;

/* The largest batch one call of a plan may pass. */
typedef struct gt_batch_limits {
    uint32_t max_graphs;      /* descriptors per call, >= 1                          */
    uint32_t max_cols;        /* columns (n_cols, else n_vertices) of any graph, >= 1 */
    uint64_t max_graph_edges; /* edges of any one graph                              */
    uint64_t max_edges;       /* edges of all graphs of a call together              */
    uint64_t max_cols_total;  /* columns of all graphs of a call together            */
} gt_batch_limits;

typedef struct gt_batch_info {
    uint32_t n_graphs;        /* graphs of the last call                      */
    uint32_t sub_batches;     /* sub-batches the last call used               */
    uint32_t passes_max;      /* digit passes of every sub-batch              */
    uint32_t kernel_launches; /* kernels in one batch call (all slots)        */
    uint64_t n_edges;         /* edges of the last call's transposed graphs   */
    uint64_t workspace_bytes;
    uint32_t slots;           /* sub-batch slots of the captured sequence     */
    uint32_t key_bits;        /* union key width                              */
    uint64_t sub_batch_edges; /* edges one sub-batch may hold                 */
} gt_batch_info;

typedef struct gt_batch_plan_s *gt_batch_plan;

/* Limits that fit exactly the given HOST descriptor list. */
gt_status gt_batch_limits_from_descs(uint32_t n_graphs, const gt_graph_desc *descs, gt_batch_limits *limits);

/* Creates a plan for batches within `limits` (workspace allocated here).
 * has_vals: every graph carries values (or none does).  cfg: NULL or
 * method GT_METHOD_RADIX with radix_tile 0 (the bulk-staged digit passes);
 * batch_key_bits / batch_edges_log2 shape the sub-batches; flags bit
 * GT_FLAG_NO_GRAPH launches the kernels directly instead of replaying a CUDA
 * graph.  Fails with GT_ERR_UNSUPPORTED when the limits need more than 4096
 * sub-batch slots or a graph larger than a sub-batch. */
gt_status gt_batch_plan_create(gt_batch_plan *plan, const gt_batch_limits *limits, int has_vals,
                               const gt_config *cfg, void *stream);

/* Replaces the configuration (reallocates the workspace; synchronous). */
gt_status gt_batch_plan_set_config(gt_batch_plan plan, const gt_config *cfg);
gt_status gt_batch_plan_get_config(gt_batch_plan plan, gt_config *cfg);

/* Enqueues the transposition of graphs d_descs[0 .. n_graphs) on `stream`.
 * d_descs: DEVICE array of descriptors (read by the kernels when they run);
 * d_status: DEVICE array of n_graphs gt_status codes (32-bit), or NULL: each
 * gets GT_OK, or the first error of that graph -- GT_ERR_INVALID_ARG (n_vertices
 * 0, a null array, values present or absent against the plan),
 * GT_ERR_UNSUPPORTED (beyond the plan's limits), GT_ERR_BAD_ROW_PTR,
 * GT_ERR_OUT_OF_RANGE.  Graphs with an error are skipped (their outputs are
 * unspecified); the others are transposed.  The first call on a stream
 * captures the CUDA graph: make it before any outside capture of that stream.
 * Host errors: n_graphs above the limit -> GT_ERR_UNSUPPORTED.  Any device
 * error is also latched in the plan's status word (gt_batch_plan_status). */
gt_status gt_transpose_batched(gt_batch_plan plan, uint32_t n_graphs, const gt_graph_desc *d_descs,
                               gt_status *d_status, void *stream);

/* Synchronises the last stream; returns the first device error of the last call. */
gt_status gt_batch_plan_status(gt_batch_plan plan);
/* Synchronises the last stream; shape of the plan and of its last call. */
gt_status gt_batch_plan_info(gt_batch_plan plan, gt_batch_info *info);

/* Batch autotuner: times the batch configurations of gt_batch_tune_grid_config
 * on this batch (1 warm-up + reps calls each, median of CUDA-event times) and
 * installs the fastest.  The batch's outputs then hold its transposition.
 * table: optional host array of GT_BATCH_TUNE_GRID entries (ms = -1 where a
 * point could not run); chosen: optional grid index.  Synchronous. */
#define GT_BATCH_TUNE_GRID 6
gt_status gt_batch_tune_grid_config(uint32_t index, gt_config *cfg);
gt_status gt_batch_plan_tune(gt_batch_plan plan, uint32_t n_graphs, const gt_graph_desc *d_descs,
                             gt_status *d_status, uint32_t reps, float *table_ms, uint32_t *chosen, void *stream);
void gt_batch_plan_destroy(gt_batch_plan plan);

/* ---- Configuration search: features, grid, analytic model, autotuner, -----
 * ---- learned selector.  None of it changes the output bytes. ------------- */

#define GT_N_FEATURES 41  /* graph features of gt_graph_features            */
#define GT_TUNE_GRID 12   /* configurations of the search grid              */
#define GT_SEL_HIDDEN 64  /* width of the selector's two hidden layers      */

/* Graph features (device f32[GT_N_FEATURES] written on `stream`), computed by
 * kernels from row_ptr and a seeded sample of col_idx:
 *   [0..31]  fraction of vertices per out-degree bin: bin 0 = degree 0, bin b
 *            (1..31) = degree in [2^(b-1), 2^b), bin 31 also holds larger
 *   [32]     log2(n)/32    [33] log2(m+1)/32    [34] log2(max out-degree+1)/32
 *   [35]     fraction of edges leaving the ceil(n/100) vertices of highest
 *            out-degree, estimated from the log2 bins (per-bin vertex counts
 *            and edge sums, proportional share of the boundary bin)
 *   [36]     coverage (Sec. IV-B): share of ns samples of col_idx that fall on
 *            the 512 most frequent sampled destinations; ns = clamp(ceil(n/100),
 *            1024, 2^20), sample j at floor(r_j m / 2^64), r_j = SplitMix64
 *            output j (j = 1..ns: mix(seed + j*0x9E3779B97F4A7C15))
 *   [37]     log2(max sample frequency * m / ns + 1)/32 (estimated max in-degree)
 *   [38],[39] locality over 4096 sampled rows u_j = floor(r'_j n / 2^64)
 *            (r' from seed ^ 0x4C4F43), first 32 neighbour pairs (a, b) of each
 *            row with >= 2 edges: mean log2(|a-b|+1)/32, and the fraction of
 *            pairs with a/32 == b/32 (same 128-byte line of a u32 array)
 *   [40]     has_vals
 * Allocates its small workspace stream-ordered (cudaMallocAsync). */
gt_status gt_graph_features(uint32_t n_vertices, uint64_t n_edges, int has_vals, const uint64_t *row_ptr,
                            const uint32_t *col_idx, uint64_t seed, float *features, void *stream);

/* The same features for an n_rows x n_cols matrix: "vertices" in [0..31],
 * [35], [38] and [39] are rows (out-degrees, sampled rows u_j over n_rows);
 * [32] is log2(n_cols)/32 and ns = clamp(ceil(n_cols/100), 1024, 2^20).
 * gt_graph_features(n) is gt_graph_features_rect(n, n). */
gt_status gt_graph_features_rect(uint32_t n_rows, uint32_t n_cols, uint64_t n_edges, int has_vals,
                                 const uint64_t *row_ptr, const uint32_t *col_idx, uint64_t seed, float *features,
                                 void *stream);

/* Grid point `index` (0..GT_TUNE_GRID-1) for a graph of this size
 * (n_vertices: the column count of a rectangular matrix).  The two choices
 * of the paper's probe (Sec. IV-B) and ten radix configurations whose digit
 * width (pass count), tile kind and CTAs per SM change the time:
 *   0 Atomic GT (hdv_k = 0, Algorithm 1)   1 HLH, k = 512 (Eq. 1 sizing)
 *   2 radix, bulk-staged 4096-edge tiles, digits <= 8 bits (the default)
 *   3 same, digits <= 7   4 same, digits <= 6
 *   5 radix, register tiles of 4096 edges, 2 CTAs/SM, digits <= 8   6 same, digits <= 7
 *   7 register 4096, 3 CTAs/SM, digits <= 6
 *   8 register tiles of 2048 edges, 4 CTAs/SM, digits <= 8   9 same, digits <= 7
 *   10 register 2048, 6 CTAs/SM, digits <= 8   11 register 2048, 6 CTAs/SM, digits <= 6
 * An HDV count above n/2 becomes 0 (the point then equals Atomic GT). */
gt_status gt_tune_grid_config(uint32_t index, uint32_t n_vertices, uint64_t n_edges, gt_config *cfg);

/* Analytic choice (the Sec. IV-B cost model, Eqs. 2-3, with GB300 rates and a
 * streaming term for the radix method) from host copies of the features:
 * writes the grid index (0, 1 or 2).  n_vertices: the column count of a
 * rectangular matrix. */
gt_status gt_tune_analytic(const float *features, uint32_t n_vertices, uint64_t n_edges, uint32_t *index);

typedef struct gt_selector_s *gt_selector;

/* Learned selector: an MLP GT_N_FEATURES -> 64 -> 64 -> GT_TUNE_GRID (ReLU),
 * f32, on the device.  Parameter vector (gt_selector_param_count floats):
 * mu[F], sd[F] (input standardisation, x' = (x - mu) / sd, not trained),
 * lo[F], hi[F] (the feature range of the training graphs, not trained and
 * not used by the network), W1[64][F], b1[64], W2[64][64], b2[64],
 * W3[K][64], b3[K].  Output i is a score for grid point i; the learned mode
 * takes the smallest, except for a graph whose features leave [lo, hi]
 * (widened by 5 % of its width), where it takes the analytic choice.
 * host_params == NULL: mu = 0, sd = 1, unbounded range, weights uniform in
 * +-sqrt(6/fan_in) from SplitMix64(seed), biases 0. */
uint64_t gt_selector_param_count(void);
gt_status gt_selector_create(gt_selector *sel, const float *host_params, uint64_t seed);
gt_status gt_selector_get_params(gt_selector sel, float *host_params);
/* Replaces all parameters (every sd must be > 0) and resets Adam's state. */
gt_status gt_selector_set_params(gt_selector sel, const float *host_params);
/* scores (device f32[batch][GT_TUNE_GRID]) for features (device f32[batch][F]). */
gt_status gt_selector_forward(gt_selector sel, const float *features, uint32_t batch, float *scores,
                              void *stream);
/* Forward + backward of the masked mean squared error
 *   L = sum_{b,i} M[b][i] (y[b][i] - T[b][i])^2 / max(1, sum M)
 * into the selector's gradient buffer; loss (device f32[1]) and grads (device
 * f32[param_count], mu/sd entries 0) are optional copies. */
gt_status gt_selector_backward(gt_selector sel, const float *features, const float *target, const float *mask,
                               uint32_t batch, float *loss, float *grads, void *stream);
/* *in_range = 1 if host features (F floats) lie in the selector's trained
 * range (widened by 5 % of its width), else 0. */
gt_status gt_selector_in_range(gt_selector sel, const float *host_features, int *in_range);
/* One Adam step (bias-corrected) with the last gradients on W and b; the
 * moments see g + weight_decay * p (an L2 penalty weight_decay/2 |W, b|^2;
 * 0 = plain Adam). */
gt_status gt_selector_adam_step(gt_selector sel, float lr, float beta1, float beta2, float eps, float weight_decay,
                                void *stream);
void gt_selector_destroy(gt_selector sel);

typedef struct gt_tune_entry {
    gt_config cfg;    /* grid point                                           */
    float ms;         /* exhaustive: median device time of the timed calls; -1 if not run */
    float score;      /* learned: the selector's score (computed even when the
                         graph is outside the trained range)                */
    int32_t status;   /* gt_status of this point's run                        */
} gt_tune_entry;

#define GT_TUNE_ANALYTIC 0    /* features + gt_tune_analytic                  */
#define GT_TUNE_EXHAUSTIVE 1  /* time every grid point (1 warm-up + reps calls) */
#define GT_TUNE_LEARNED 2     /* features + selector, smallest score (analytic outside its range) */

/* Chooses a configuration for the plan's graph and installs it
 * (gt_plan_set_config).  The exhaustive mode runs real transpositions into
 * the given outputs (which then hold the CSC).  table: optional host array of
 * GT_TUNE_GRID entries; chosen: optional grid index.  Synchronous. */
gt_status gt_plan_tune(gt_plan plan, int mode, gt_selector sel, const uint64_t *row_ptr, const uint32_t *col_idx,
                       const float *vals, uint64_t *col_ptr, uint32_t *row_idx, float *vals_out, uint32_t reps,
                       gt_tune_entry *table, uint32_t *chosen, void *stream);

/* Sizes the plan was created for (gt_plan_vertices: the row count, which is
 * the vertex count of a graph).  gt_plan_shape: any pointer may be NULL. */
uint32_t gt_plan_vertices(gt_plan plan);
uint64_t gt_plan_edges(gt_plan plan);
gt_status gt_plan_shape(gt_plan plan, uint32_t *n_rows, uint32_t *n_cols, uint64_t *n_edges);

/* Synchronises the plan's last stream and returns (then clears) the latched
 * device status. */
gt_status gt_plan_status(gt_plan plan);

/* Statistics of the last completed gt_transpose (synchronises). */
gt_status gt_plan_stats(gt_plan plan, gt_stats *stats);

/* Starts (enable != 0, clearing earlier records) or stops per-step timing. */
gt_status gt_plan_enable_timing(gt_plan plan, int enable);

/* Averages of the recorded calls (synchronises the plan's stream). */
gt_status gt_plan_timing(gt_plan plan, gt_timing *timing);

/* Step 3's per-partition busy times (ms, end - start of each warp
 * partition) of the last gt_transpose of a plan configured with
 * GT_FLAG_PARTITION_TIMES (HLH method): writes min(P, cap) entries and
 * *count = P (the warp partitions).  Synchronises.  GT_ERR_INVALID_ARG if the
 * plan does not record them. */
gt_status gt_plan_partition_times(gt_plan plan, float *busy_ms, uint32_t cap, uint32_t *count);

/* Device bytes held by the plan's workspace. */
uint64_t gt_plan_workspace_bytes(gt_plan plan);

void gt_plan_destroy(gt_plan plan);

const char *gt_status_string(gt_status status);

/* Text of the last CUDA runtime error seen by this thread (GT_ERR_CUDA detail). */
const char *gt_last_cuda_error(void);

/* Library version (major*10000 + minor*100 + patch). */
uint32_t gt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GT_H_ */
