/*
 * Oracle for graph transposition (CSR -> CSC).  TEST INFRASTRUCTURE ONLY:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Sec. II-A, "Terminology"): a CSR graph lists, for every
 * vertex u, its out-neighbours col_idx[row_ptr[u] .. row_ptr[u+1]).  Its CSC
 * lists, for every vertex v, the sources of its in-edges.  Graph
 * transposition (Sec. II-A) turns one into the other; per-edge weights ride
 * along unchanged (Sec. II-A, edge-weighted graphs).
 *
 * Ordering contract (the paper leaves the order inside a CSC list to an
 * optional sort, Sec. II-B; ScanTrans/MergeTrans produce sorted lists,
 * Sec. II-C): every CSC list is in ascending source order, and edges with the
 * same (source, destination) keep their CSR order.  That is exactly a stable
 * sort of the CSR edge sequence by destination.
 *
 * Rectangular matrices (a sparse n_rows x n_cols matrix in CSR: row_ptr has
 * n_rows + 1 entries, col_idx values lie in [0, n_cols)) follow the same
 * definition: the CSC has n_cols + 1 offsets and lists row IDs.  A graph is
 * the square case n_rows = n_cols = n.
 *
 * Algorithm: the three steps of Atomic GT (Algorithm 1) run by ONE thread, so
 * every fetch_and_add becomes a plain increment and the edge visit order is
 * the CSR order -- a sequential counting sort, stable by construction:
 *   Step 1  counters[v] = in-degree of v
 *   Step 2  t_offsets = exclusive prefix sum of counters; IP = copy
 *   Step 3  for u ascending, for e in row u ascending: t_edges[IP[v]++] = u
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_RANGE 2   /* some col_idx[e] >= n_cols */
#define OR_ERR_ROWPTR 3  /* row_ptr[0] != 0, not monotone, or row_ptr[n_rows] != m */
#define OR_ERR_NOMEM 4
#define OR_ERR_DEGREE 5  /* an in-degree does not fit 32 bits (not reachable for m <= 2^32 - 1) */

static int check_csr(uint32_t n_rows, uint32_t n_cols, uint64_t m, const uint64_t *row_ptr,
                     const uint32_t *col_idx) {
    if (!row_ptr) return OR_ERR_ARG;
    if (m > 0 && !col_idx) return OR_ERR_ARG;
    if (row_ptr[0] != 0 || row_ptr[n_rows] != m) return OR_ERR_ROWPTR;
    for (uint64_t u = 0; u < n_rows; ++u)
        if (row_ptr[u] > row_ptr[u + 1]) return OR_ERR_ROWPTR;
    for (uint64_t e = 0; e < m; ++e)
        if (col_idx[e] >= n_cols) return OR_ERR_RANGE;
    return OR_OK;
}

/*
 * Full transposition of an n_rows x n_cols matrix, Algorithm 1 run serially.
 * col_ptr has n_cols + 1 entries, row_idx m entries, vals_out m entries when
 * vals != NULL.
 */
int oracle_transpose_rect(uint32_t n_rows, uint32_t n_cols, uint64_t m, const uint64_t *row_ptr,
                          const uint32_t *col_idx, const float *vals, uint64_t *col_ptr, uint32_t *row_idx,
                          float *vals_out) {
    int st = check_csr(n_rows, n_cols, m, row_ptr, col_idx);
    if (st) return st;
    if (!col_ptr || (m > 0 && !row_idx) || (vals && m > 0 && !vals_out)) return OR_ERR_ARG;

    /* Step 1: in-degrees (counters), one per column. */
    uint64_t *ip = (uint64_t *)calloc((size_t)n_cols + 1, sizeof(uint64_t));
    if (!ip) return OR_ERR_NOMEM;
    for (uint64_t e = 0; e < m; ++e) ip[col_idx[e]] += 1;

    /* Step 2: t_offsets = exclusive prefix sum; IP starts as a copy. */
    uint64_t run = 0;
    for (uint64_t v = 0; v < n_cols; ++v) {
        uint64_t d = ip[v];
        col_ptr[v] = run;
        ip[v] = run;
        run += d;
    }
    col_ptr[n_cols] = run;

    /* Step 3: visit edges in CSR order (rows ascending) and append u to the list of v. */
    for (uint64_t u = 0; u < n_rows; ++u) {
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint64_t slot = ip[col_idx[e]]++;
            row_idx[slot] = (uint32_t)u;
            if (vals) vals_out[slot] = vals[e];
        }
    }
    free(ip);
    return OR_OK;
}

/* The square case: a graph with n vertices. */
int oracle_transpose(uint32_t n, uint64_t m, const uint64_t *row_ptr, const uint32_t *col_idx,
                     const float *vals, uint64_t *col_ptr, uint32_t *row_idx, float *vals_out) {
    return oracle_transpose_rect(n, n, m, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out);
}

/*
 * The same definition restricted to destinations v in [v_lo, v_hi): for hosts
 * whose memory cannot hold a whole output.  col_ptr_part has v_hi - v_lo + 1
 * entries holding the GLOBAL offsets col_ptr[v_lo .. v_hi]; row_idx_part and
 * vals_out_part hold entries col_ptr[v_lo] .. col_ptr[v_hi]-1 of the full
 * output.  Running it over consecutive ranges reproduces oracle_transpose.
 * With row_idx_part == NULL only col_ptr_part is produced (the sizes the
 * caller needs to hold the range's lists).
 */
int oracle_transpose_range(uint32_t n, uint64_t m, const uint64_t *row_ptr, const uint32_t *col_idx,
                           const float *vals, uint32_t v_lo, uint32_t v_hi, uint64_t *col_ptr_part,
                           uint32_t *row_idx_part, float *vals_out_part) {
    int st = check_csr(n, n, m, row_ptr, col_idx);
    if (st) return st;
    if (v_lo > v_hi || v_hi > n || !col_ptr_part) return OR_ERR_ARG;
    uint32_t w = v_hi - v_lo;
    uint64_t *ip = (uint64_t *)calloc((size_t)w + 1, sizeof(uint64_t));
    if (!ip) return OR_ERR_NOMEM;
    uint64_t below = 0; /* edges whose destination is < v_lo */
    for (uint64_t e = 0; e < m; ++e) {
        uint32_t v = col_idx[e];
        if (v < v_lo) below++;
        else if (v < v_hi) ip[v - v_lo] += 1;
    }
    uint64_t run = below;
    for (uint32_t i = 0; i < w; ++i) {
        uint64_t d = ip[i];
        col_ptr_part[i] = run;
        ip[i] = run - below; /* local slot */
        run += d;
    }
    col_ptr_part[w] = run;
    if (!row_idx_part) { free(ip); return OR_OK; } /* sizes only */
    for (uint64_t u = 0; u < n; ++u) {
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = col_idx[e];
            if (v < v_lo || v >= v_hi) continue;
            uint64_t slot = ip[v - v_lo]++;
            row_idx_part[slot] = (uint32_t)u;
            if (vals) vals_out_part[slot] = vals[e];
        }
    }
    free(ip);
    return OR_OK;
}

static size_t lower_bound_u32(const uint32_t *a, size_t len, uint32_t x) {
    size_t lo = 0, hi = len;
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/*
 * Sampled columns of the same definition, for graphs whose full output does
 * not fit host memory.  cols: strictly increasing vertex IDs (ncols of them).
 * Outputs: col_start[i] = col_ptr[cols[i]] (number of edges with destination
 * < cols[i]); col_deg[i] = in-degree of cols[i]; the lists themselves are
 * concatenated in cols order into out_rows/out_vals (capacity out_cap; the
 * call fails with OR_ERR_ARG if the lists do not fit).  With out_rows == NULL
 * only col_start and col_deg are produced.
 */
int oracle_columns_rect(uint32_t n_rows, uint32_t n_cols, uint64_t m, const uint64_t *row_ptr,
                        const uint32_t *col_idx, const float *vals, const uint32_t *cols, uint64_t ncols,
                        uint64_t *col_start, uint64_t *col_deg, uint32_t *out_rows, float *out_vals,
                        uint64_t out_cap) {
    int st = check_csr(n_rows, n_cols, m, row_ptr, col_idx);
    if (st) return st;
    for (uint64_t i = 0; i < ncols; ++i) {
        if (cols[i] >= n_cols || (i > 0 && cols[i] <= cols[i - 1])) return OR_ERR_ARG;
    }
    /* below[i] = number of edges whose destination lies in [cols[i-1], cols[i]) ... counted
       by bucketing every destination at its lower-bound position among cols. */
    uint64_t *bucket = (uint64_t *)calloc((size_t)ncols + 1, sizeof(uint64_t));
    uint64_t *deg = (uint64_t *)calloc((size_t)ncols + 1, sizeof(uint64_t));
    if (!bucket || !deg) { free(bucket); free(deg); return OR_ERR_NOMEM; }
    for (uint64_t e = 0; e < m; ++e) {
        uint32_t v = col_idx[e];
        size_t pos = lower_bound_u32(cols, (size_t)ncols, v);
        if (pos < ncols && cols[pos] == v) deg[pos] += 1;
        else bucket[pos] += 1; /* strictly below cols[pos] (or above all) */
    }
    /* col_ptr[cols[i]] = sum over j <= i of bucket[j] + sum over j < i of deg[j]. */
    uint64_t run = 0, total = 0;
    for (uint64_t i = 0; i < ncols; ++i) {
        run += bucket[i];
        col_start[i] = run;
        col_deg[i] = deg[i];
        run += deg[i];
        total += deg[i];
    }
    if (!out_rows) { free(bucket); free(deg); return OR_OK; } /* sizes only */
    if (total > out_cap) { free(bucket); free(deg); return OR_ERR_ARG; }
    /* Write cursor for each sampled column inside the concatenated output. */
    uint64_t acc = 0;
    for (uint64_t i = 0; i < ncols; ++i) { uint64_t d = deg[i]; deg[i] = acc; acc += d; }
    for (uint64_t u = 0; u < n_rows; ++u) {
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = col_idx[e];
            size_t pos = lower_bound_u32(cols, (size_t)ncols, v);
            if (pos < ncols && cols[pos] == v) {
                uint64_t slot = deg[pos]++;
                out_rows[slot] = (uint32_t)u;
                if (vals && out_vals) out_vals[slot] = vals[e];
            }
        }
    }
    free(bucket);
    free(deg);
    return OR_OK;
}

int oracle_columns(uint32_t n, uint64_t m, const uint64_t *row_ptr, const uint32_t *col_idx,
                   const float *vals, const uint32_t *cols, uint64_t ncols, uint64_t *col_start,
                   uint64_t *col_deg, uint32_t *out_rows, float *out_vals, uint64_t out_cap) {
    return oracle_columns_rect(n, n, m, row_ptr, col_idx, vals, cols, ncols, col_start, col_deg, out_rows,
                               out_vals, out_cap);
}

/*
 * 64-bit vertex IDs (matrices with more than 2^32 - 1 rows or columns): the
 * same definition and the same three steps of Algorithm 1 run by one thread,
 * with u64 column indices in and u64 row IDs out.  col_ptr has n_cols + 1
 * entries; the counters take 8 (n_cols + 1) bytes of host memory.
 */
int oracle_transpose64(uint64_t n_rows, uint64_t n_cols, uint64_t m, const uint64_t *row_ptr,
                       const uint64_t *col_idx, const float *vals, uint64_t *col_ptr, uint64_t *row_idx,
                       float *vals_out) {
    if (!row_ptr || !col_ptr || (m > 0 && (!col_idx || !row_idx)) || (vals && m > 0 && !vals_out)) return OR_ERR_ARG;
    if (row_ptr[0] != 0 || row_ptr[n_rows] != m) return OR_ERR_ROWPTR;
    for (uint64_t u = 0; u < n_rows; ++u)
        if (row_ptr[u] > row_ptr[u + 1]) return OR_ERR_ROWPTR;
    for (uint64_t e = 0; e < m; ++e)
        if (col_idx[e] >= n_cols) return OR_ERR_RANGE;

    /* Step 1: in-degrees. */
    uint64_t *ip = (uint64_t *)calloc((size_t)n_cols + 1, sizeof(uint64_t));
    if (!ip) return OR_ERR_NOMEM;
    for (uint64_t e = 0; e < m; ++e) ip[col_idx[e]] += 1;

    /* Step 2: exclusive prefix sum; IP starts as a copy. */
    uint64_t run = 0;
    for (uint64_t v = 0; v < n_cols; ++v) {
        uint64_t d = ip[v];
        col_ptr[v] = run;
        ip[v] = run;
        run += d;
    }
    col_ptr[n_cols] = run;

    /* Step 3: edges in CSR order append their source to their destination's list. */
    for (uint64_t u = 0; u < n_rows; ++u) {
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint64_t slot = ip[col_idx[e]]++;
            row_idx[slot] = u;
            if (vals) vals_out[slot] = vals[e];
        }
    }
    free(ip);
    return OR_OK;
}
