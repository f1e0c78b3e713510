/*
 * wrs.h - C ABI of the GB300 alias-table library (weighted random sampling,
 * "Weighted Random Sampling on GPUs", Lehmann, Huebschle-Schneider, Sanders,
 * arXiv 2106.12270).
 *
 * Problem (Sec. 1): items 0..N-1 with weights w_i >= 0 and total W; draw
 * item i with probability w_i / W, with replacement.
 *
 * Alias table (Sec. 2.2): N rows, each one bucket of W/N.  Row b keeps the
 * share prob_b (in [0,1], in units of one bucket) for item b and gives the
 * rest to item alias_b.  A row is 8 bytes: {float prob; uint32 alias}.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers (GPU global memory), h_* are
 *    host pointers.  The caller owns every buffer it passes; the library
 *    never frees, resizes or keeps a caller buffer beyond the call (except
 *    where a table object is documented to own memory).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls named *_rows / wrs_step_* / wrs_sample* only enqueue
 *    work on that stream and return without synchronising; their device
 *    results are valid once the stream reaches that point.
 *  - Every call returns an int status (enum wrs_status).  Argument errors
 *    are detected on the host before anything is enqueued, and output
 *    buffers are then left untouched.  Errors that depend on the data (a
 *    negative or non-finite weight, a zero total) are found on the device
 *    and reported through wrs_build_info.status.
 *  - N is limited to [1, 2^31 - 1] (indices are 32-bit).
 *  - No call here uses more than one GPU; every call runs on the current
 *    CUDA device of the calling thread.
 */
#ifndef WRS_H
#define WRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------- */
/* Status codes                                                            */
/* ---------------------------------------------------------------------- */
enum wrs_status {
    WRS_OK = 0,
    WRS_EINVAL = 1,      /* bad argument or negative weight */
    WRS_EZEROSUM = 2,    /* all weights are zero: no distribution (Sec. 1) */
    WRS_ENONFINITE = 3,  /* a weight is NaN or infinite */
    WRS_ENOMEM = 4,      /* device allocation failed or budget exceeded */
    WRS_ETIMEOUT = 5,    /* reserved: no kernel waits on another, none times out */
    WRS_ECUDA = 6,       /* a CUDA runtime call failed */
    WRS_EBUSY = 7,       /* request loop: no room right now */
    WRS_ENOTFOUND = 8    /* request loop: unknown ticket */
};

/* Text for a status code (static storage, never NULL). */
const char *wrs_strerror(int status);
/* CUDA error of the last call that returned WRS_ECUDA on this thread. */
int wrs_last_cuda_error(void);
/* ABI version: increases when a signature or struct layout changes. */
int wrs_abi_version(void);

/* ---------------------------------------------------------------------- */
/* Data layout                                                             */
/* ---------------------------------------------------------------------- */

/* One alias-table row (Sec. 2.2): row b keeps `prob` of its bucket for item
 * b and gives 1 - prob to item `alias`.  prob is the paper's T^w_b / (W/N). */
typedef struct wrs_row {
    float prob;
    uint32_t alias;
} wrs_row;

/* Tuning knobs of the build. */
typedef struct wrs_config {
    /* Buckets per pack section ("N/s items per section", Sec. 2.2); one CTA
     * packs one section.  Multiple of 256 in [256, 8192]; default 1024. */
    uint32_t section_size;
    /* Split search (Sec. 4.1): WRS_SPLIT_PARY (partial p-ary search,
     * Algorithm 1; default) or WRS_SPLIT_BINARY (one binary search per
     * split, the PSA baseline). */
    uint32_t split_method;
    uint32_t reserved[6];
} wrs_config;

enum wrs_split_method { WRS_SPLIT_PARY = 0, WRS_SPLIT_BINARY = 1 };

/* Fill *cfg with the defaults. */
void wrs_config_default(wrs_config *cfg);

/* Summary of one build, written by the device at the end of the build.
 * Layout is fixed (ABI); all fields little-endian. */
typedef struct wrs_build_info {
    int32_t status;   /* WRS_OK or a data error (EINVAL/ENONFINITE/EZEROSUM/ETIMEOUT) */
    int32_t scale;    /* fixed-point scale S: q_i = round(w_i * 2^S) */
    double W;         /* sum of the weights, exact, rounded once to FP64 */
    double avg;       /* W / N in FP64: the bucket size (Sec. 2.2) */
    uint64_t nl;      /* number of light items, w_i <= avg */
    uint64_t nh;      /* number of heavy items, w_i > avg */
    uint32_t Q[4];    /* bucket in fixed point: sum of all q_i (Q[0] low word, Q[2..3] = 0) */
    float light_max;  /* largest FP32 value <= avg: light iff w_i <= light_max */
    uint32_t sections;/* number of pack sections s */
    uint64_t reserved[4];
} wrs_build_info;

/* ---------------------------------------------------------------------- */
/* Construction (PSA on the GPU, Sec. 2.2 and Sec. 4)                      */
/* ---------------------------------------------------------------------- */

/* Bytes of device workspace a build of n items needs. */
int wrs_build_workspace_bytes(uint64_t n, const wrs_config *cfg,
                              uint64_t *bytes);

/* Offsets (bytes from the workspace start) of the build's intermediate
 * arrays, for inspection after a build:
 *   lh:     n entries {uint32 item, float weight}; light items in index order
 *           from the front (entry a = l[a]), heavy items in index order from
 *           the back (entry n-1-b = h[b])  (Sec. 4.2 "weight in l and h").
 *   ckl:    checkpoints of the light prefix sums, one per 32 entries: record c
 *           (16 bytes) = {uint32 seg, uint32 pad, uint64 s} where s is the sum
 *           of the fixed-point weights q of l[0..32c) that lie in partition
 *           segment `seg`; the sum over the earlier segments is seg_pre[seg].
 *   ckh:    the same for the heavy list h.
 *   seg_pre: segment prefixes, 48 bytes each: {uint32 sl[4], uint32 sh[4],
 *           uint64 nl, uint64 pad}: q sums (128-bit fields, values < 2^64)
 *           of the light and heavy items before the segment and the number
 *           of light items before it.
 *   splits: s+1 records {uint32 i, uint32 j, uint32 pad[2], uint32 D[4],
 *           uint32 E[4]}: the Vose state after t*section_size buckets
 *           (Sec. 2.2 split).
 * Fixed point: q_i = round(w_i * 2^S) (S = wrs_build_info.scale, so that
 * W*2^S lies in [2^61, 2^62)); the bucket Q = wrs_build_info.Q is the exact
 * sum of all q_i.  With sigma the q sums (light items clamped to at most
 * floor(Q/N), heavy items to at least floor(Q/N)+1):
 *   D'(i) = i*Q - N*sigma_l(i)  (N times the light deficit before l[i]) and
 *   E'(j) = N*sigma_h(j) - j*Q  (N times the heavy excess before h[j]);
 *   split record t holds D = D'(i_t), E = E'(j_t). */
typedef struct wrs_layout {
    uint64_t lh, ckl, ckh, seg_pre, splits;
    uint64_t sections;       /* s */
    uint64_t total_bytes;
} wrs_layout;
int wrs_build_layout(uint64_t n, const wrs_config *cfg, wrs_layout *out);

/* Full build: d_w (n FP32 weights, device) -> d_rows (n rows, device).
 * Steps: total weight, classify + stable partition + prefix sums, split
 * search, sweep-pack (Sec. 2.2, Sec. 4).  No allocation, no host sync.
 * d_ws: >= wrs_build_workspace_bytes(n) bytes, 256-byte aligned, device.
 * d_info: device wrs_build_info, written at the end of the build.
 * cfg may be NULL (defaults).  The weights are not modified. */
int wrs_build_rows(const float *d_w, uint64_t n, wrs_row *d_rows,
                   void *d_ws, uint64_t ws_bytes, const wrs_config *cfg,
                   wrs_build_info *d_info, void *stream);

/* PSA+ construction (Sec. 4 "PSA+"): greedy packing inside every tile of
 * 1024 consecutive items that holds at least min_items light and heavy
 * items (the tile's lights and heavies, each in index order, swept as in
 * PSA until the current heavy is above the average with no light left, or
 * at most the average with no next heavy in the tile), then the PSA
 * construction on the items left over, in index order; the heavy current at
 * the stop carries its remaining weight.  The table is a valid alias table
 * for w (tested by reconstructed mass) but not the same table as
 * wrs_build_rows'.
 * d_ws: at least wrs_build_plus_workspace_bytes(n, cfg) bytes, 256-byte
 * aligned.  *greedy_items (host, may be NULL) receives how many items the
 * greedy step finished (0 when a whole-table step failed).  Unlike
 * wrs_build_rows this call synchronises `stream` once (the size of the rest
 * decides its launches).  Errors as wrs_build_rows; with min_items larger
 * than 1024 it builds wrs_build_rows' table. */
int wrs_build_plus_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes);
int wrs_build_rows_plus(const float *d_w, uint64_t n, wrs_row *d_rows, void *d_ws,
                        uint64_t ws_bytes, const wrs_config *cfg, uint32_t min_items,
                        wrs_build_info *d_info, uint64_t *greedy_items, void *stream);

/* Full build from host memory: h_w (n FP32 weights, host) -> h_rows (n rows,
 * host), with the copies on `stream`: weights in, the build of
 * wrs_build_rows, rows and the summary (h_info, host) out.  With pinned host
 * buffers the call only enqueues; the caller syncs the stream before reading
 * h_rows.  Two workspaces on two streams let one call's copy out overlap the
 * next call's copy in and build.  d_ws: >= wrs_build_host_workspace_bytes(n)
 * bytes, 256-byte aligned, device (the build workspace plus a device copy of
 * the weights and the rows). */
int wrs_build_host_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes);
int wrs_build_rows_host(const float *h_w, uint64_t n, wrs_row *h_rows, void *d_ws,
                        uint64_t ws_bytes, const wrs_config *cfg, wrs_build_info *h_info,
                        void *stream);

/* The same build without allocating anything (the paper has no counterpart;
 * it serves callers that cannot allocate device memory when they build: a
 * service whose device memory is all reserved at start-up, or code inside a
 * framework that owns the allocator, where a cudaMalloc would break the
 * memory plan or bring an implicit device synchronisation).  The caller
 * still passes the weights, the rows and d_info; the workspace is a 32 MiB
 * device array inside this library, which every GPU that loads the library
 * holds until the process exits.
 *  - n must be at most 3,500,000; larger n returns WRS_EINVAL and enqueues
 *    nothing (use wrs_build_rows with a caller workspace instead).
 *  - Every call looks up the array's device address on the current device
 *    (this allocates nothing); the first call on a device also loads the
 *    library's device code there, so make that first call before any
 *    stream capture.
 *  - Every call on a device shares the one array: calls whose work overlaps
 *    on the GPU (different streams, or different host threads) race and give
 *    wrong tables.  Serialise them, e.g. on one stream.  The array keeps the
 *    last call's contents; a build never relies on it being cleared.
 * Results are identical to wrs_build_rows. */
int wrs_build_rows_noalloc(const float *d_w, uint64_t n, wrs_row *d_rows,
                           const wrs_config *cfg, wrs_build_info *d_info, void *stream);

/* The same build, one step per call (each enqueues its kernels; run them in
 * this order on one stream with the same workspace).  They exist so each
 * step can be checked on its own. */
/* a1: W = sum w_i exactly, avg = W/N, fixed-point scale (Sec. 1, Sec. 2.2). */
int wrs_step_total(const float *d_w, uint64_t n, void *d_ws, uint64_t ws_bytes,
                   const wrs_config *cfg, void *stream);
/* a2+a3: classify light/heavy, stable partition into lh, prefix sums of the
 * light deficits and heavy excesses (Sec. 2.2, Sec. 4.2). */
int wrs_step_partition(const float *d_w, uint64_t n, void *d_ws,
                       uint64_t ws_bytes, const wrs_config *cfg, void *stream);
/* a4: split search for every section boundary (Sec. 2.2, Sec. 4.1). */
int wrs_step_split(uint64_t n, void *d_ws, uint64_t ws_bytes,
                   const wrs_config *cfg, void *stream);
/* a5: sweep-pack every section into rows (Sec. 2.2, Sec. 4.2). */
int wrs_step_pack(uint64_t n, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                  const wrs_config *cfg, void *stream);
/* Copy the build summary out of the workspace into d_info (device). */
int wrs_step_info(uint64_t n, void *d_ws, uint64_t ws_bytes,
                  const wrs_config *cfg, wrs_build_info *d_info, void *stream);

/* ---------------------------------------------------------------------- */
/* Sampling (Sec. 2.2 Walker's rule, Sec. 5)                               */
/* ---------------------------------------------------------------------- */

/* Philox-4x32-10 counter layout (Salmon et al., SC'11): key = (seed_lo,
 * seed_hi); counter = (c_lo, c_hi, stream_lo, stream_hi).  Call c yields two
 * samples: 2c uses output words (x0,x1), 2c+1 uses (x2,x3) as u = x_hi<<32 |
 * x_lo.  With P = u * rows (128-bit): row = P >> 64 (integer part of U*N),
 * coin = bits 32..63 of P (fraction of U*N); the sample is the row if
 * coin < ceil(prob_row * 2^32), else alias_row. */
enum wrs_stream_tag {
    WRS_TAG_NAIVE = 0,     /* plain sampling: stream_hi of wrs_sample_rows */
    WRS_TAG_SECTION = 1,   /* sectioned sampling: (section, WRS_TAG_SECTION) */
    WRS_TAG_COUNTS = 2,    /* sectioned counts tree nodes */
    WRS_TAG_BATCH = 3,     /* batched sampling: (table, WRS_TAG_BATCH) */
    WRS_TAG_DIAG = 4       /* the Philox-rate probe (wrs_diag_philox) */
};

/* a6: naive sampling (Sec. 5 "baseline"): samples first .. first+count-1 of
 * the stream (seed, stream_lo, stream_hi) from n rows; d_out[t] receives
 * sample first+t as an item index in [0, n).  Deterministic: the same
 * arguments give the same samples on any launch configuration. */
int wrs_sample_rows(const wrs_row *d_rows, uint64_t n, uint64_t first,
                    uint64_t count, uint64_t seed, uint32_t stream_lo,
                    uint32_t stream_hi, uint32_t *d_out, void *stream);

/* Sampling modes (Sec. 5): NAIVE draws each sample from the whole table;
 * the sectioned modes first split the count over sections of the table and
 * draw every section's samples inside it, so that its rows stay in cache:
 * CACHED gathers rows through L1/L2, LIMITED additionally reserves shared
 * memory so only one CTA runs per SM (fewer sections evict each other),
 * SMEM copies each section's rows into shared memory first, each row as
 * its integer keep threshold ceil(prob 2^32) and its alias.  The three
 * sectioned modes produce identical samples; they differ only in speed. */
enum wrs_sample_mode {
    WRS_SAMPLE_NAIVE = 0,
    WRS_SAMPLE_CACHED = 1,
    WRS_SAMPLE_LIMITED = 2,
    WRS_SAMPLE_SMEM = 3,
    WRS_SAMPLE_AUTO = 4   /* wrs_sample_auto: pick one of the above */
};

/* Number of sections for n rows with at most section_rows rows each:
 * nsec = ceil(n / section_rows); section s covers rows
 * [floor(s*n/nsec), floor((s+1)*n/nsec)). */
int wrs_sample_sections(uint64_t n, uint32_t section_rows, uint64_t *nsec);

/* a7: sectioned sampling (Sec. 5 "cached sectioned", "cached limited
 * sectioned", "shared memory sectioned" sampling).  Draws `count` samples:
 * d_counts[s] (device, nsec uint64) receives how many fall into section s
 * (recursive binomial split keyed by (seed, tree node), normal
 * approximation above 96 samples per node), d_offsets[s] the start of its
 * samples in d_out; d_out[d_offsets[s] + q] is the q-th sample of section s
 * (Walker's rule inside the section, counter (q/2, 0, s, WRS_TAG_SECTION)).
 * The output is grouped by section, not in the order of naive sampling.
 * section_rows: 1..2^31; SMEM mode needs section_rows <= 24576 (its rows
 * live in shared memory). */
int wrs_sample_sectioned_rows(const wrs_row *d_rows, uint64_t n, uint64_t count,
                              uint64_t seed, uint32_t mode, uint32_t section_rows,
                              uint64_t *d_counts, uint64_t *d_offsets, uint32_t *d_out,
                              void *stream);

/* Sampling method selection (the paper compares its samplers over table
 * size and sample count, Sec. 6): the mode and section size wrs_sample_auto
 * uses for n rows and count samples.  The rule comes from the measured
 * heat map of all modes on GB300 (bench --sampler-heatmap):
 *   - shared-memory sectioned sampling, 4096 rows per section, for tables of
 *     at least 2^23 rows with at least 2^23 draws and 8 draws per row, and
 *     for tables of at least 2^20 rows with at least 128 draws per row;
 *   - cached sectioned sampling, 8192 rows per section, for the other tables
 *     of at least 2^23 rows with at least 2^23 draws;
 *   - naive sampling otherwise. */
int wrs_sample_auto_choice(uint64_t n, uint64_t count, uint32_t *mode, uint32_t *section_rows);

/* Device workspace of wrs_sample_auto: the per-section counts and offsets of
 * the chosen sectioned mode (0 bytes when it picks naive sampling). */
int wrs_sample_auto_workspace_bytes(uint64_t n, uint64_t count, uint64_t *bytes);

/* Draws `count` samples into d_out with the mode wrs_sample_auto_choice
 * picks: naive (samples 0..count-1 of stream (seed, 0, WRS_TAG_NAIVE), as
 * wrs_sample_rows) or sectioned (as wrs_sample_sectioned_rows, grouped by
 * section; counts and offsets in d_ws).  *mode_used (may be NULL) receives
 * the mode.  Every mode draws from the same distribution; the output depends
 * on (n, count, seed) only. */
int wrs_sample_auto(const wrs_row *d_rows, uint64_t n, uint64_t count, uint64_t seed,
                    uint32_t *d_out, void *d_ws, uint64_t ws_bytes, uint32_t *mode_used,
                    void *stream);

/* ---------------------------------------------------------------------- */
/* Batches of independent tables (one launch for many tables)              */
/* ---------------------------------------------------------------------- */

/* Summary of one table of a batch (device-written, 32 bytes). */
typedef struct wrs_table_summary {
    int32_t status;   /* WRS_OK; WRS_EINVAL for an empty segment, a segment of
                         more than 2^24 items or a negative weight;
                         WRS_ENONFINITE; WRS_EZEROSUM */
    uint32_t n;       /* items of the table */
    double W;         /* exact total weight rounded to FP64 */
    uint64_t nl, nh;  /* light and heavy counts */
} wrs_table_summary;

/* Device workspace bytes for a batch of `total` items (all tables) in ntab
 * tables: about 9 bytes per item and 150 per table. */
int wrs_build_batched_workspace_bytes(uint64_t total, uint32_t ntab, uint64_t *bytes);

/* Host-side plan: h_order receives the table ids largest first, the order in
 * which the batched build hands tables to its persistent CTAs (longest job
 * first keeps the CTAs evenly loaded).  h_off: ntab+1 host offsets. */
int wrs_batch_order(const uint64_t *h_off, uint32_t ntab, uint32_t *h_order);

/* a8: build ntab tables with one launch sequence.  Table t has the weights
 * d_w[d_off[t] .. d_off[t+1]) and gets the rows d_rows[d_off[t] ..
 * d_off[t+1]) with table-local alias indices (PSA per table, Sec. 2.2 and
 * Sec. 4).  The default (segmented) build: a warp per table (a whole CTA
 * for a table of more than half a warp's share of the batch's items and
 * more than 8192 items) computes its exact total, Q and stable partition
 * with the prefix-sum checkpoints; then the single-table split and pack
 * run over the sections (1024 buckets) of every table at once.  d_off: ntab+1 device uint64
 * offsets, non-decreasing, d_off[0] = 0; d_order: ntab device table ids (a
 * permutation, e.g. from wrs_batch_order) or NULL for 0..ntab-1; d_info:
 * ntab device summaries.  A table with an error gets a status in its
 * summary and its rows are left untouched; the others are still built.  A
 * workspace smaller than wrs_build_batched_workspace_bytes of the batch
 * leaves the tables that do not fit with WRS_EINVAL.  No host sync. */
int wrs_build_batched_rows(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                           const uint32_t *d_order, wrs_row *d_rows, void *d_ws,
                           uint64_t ws_bytes, wrs_table_summary *d_info, void *stream);

/* How the batched build runs.  threads = 0 (and chunk = 0): the segmented
 * build above.  Otherwise the chunked kernel: one persistent CTA per table
 * runs the whole pipeline and sweeps in chunks (Sec. 4.2 "chunked loading"),
 * carrying the exact Vose state from chunk to chunk instead of a split
 * search.  The tables do not depend on the choice (chunk ends and sections
 * are splits of the same sweep), only the time does. */
typedef struct wrs_batch_tuning {
    uint32_t threads;      /* 0 (segmented) or threads of a chunked CTA: 256 or 512 */
    uint32_t chunk;        /* 0 (segmented) or buckets per chunk: 512, 1024, 2048, 4096 */
    uint32_t ctas_per_sm;  /* resident CTAs per SM; 0 = as many as fit */
    float ms;              /* measured time of one build (wrs_batch_autotune) */
    uint32_t reserved[4];
} wrs_batch_tuning;

/* The default: the segmented build (threads = chunk = 0). */
int wrs_batch_tuning_default(wrs_batch_tuning *t);

/* wrs_build_batched_rows with an explicit tiling (NULL = the default).
 * WRS_EINVAL for a tiling outside the listed values. */
int wrs_build_batched_rows_tuned(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                                 const uint32_t *d_order, wrs_row *d_rows, void *d_ws,
                                 uint64_t ws_bytes, wrs_table_summary *d_info,
                                 const wrs_batch_tuning *tuning, void *stream);

/* Autotuner for the batched build: builds this batch once with every
 * candidate (the segmented build and every threads x chunk tiling of the
 * chunked kernel), times each with CUDA events on
 * `stream` (best of two runs after a warm-up), and returns the fastest in
 * *best; `all` (room for up to *nall entries, may be NULL) receives every
 * candidate with its time and *nall their number.  The buffers hold a valid
 * build afterwards.  The choice is cached per batch shape (number of tables
 * and total items); a later call with the same shape returns the cached
 * choice without timing unless `force` is nonzero.  Synchronises `stream`. */
int wrs_batch_autotune(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                       const uint32_t *d_order, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                       wrs_table_summary *d_info, void *stream, int force,
                       wrs_batch_tuning *best, wrs_batch_tuning *all, uint32_t *nall);

/* a9: sample many tables in one launch.  Samples d_cnt_off[t] ..
 * d_cnt_off[t+1]-1 of d_out come from table t (rows at d_off[t]..) as
 * table-local item indices; sample q of table t uses Philox counter
 * (q/2, 0, t, WRS_TAG_BATCH) under key (seed_lo, seed_hi), as in
 * wrs_sample_rows with stream (t, WRS_TAG_BATCH). */
int wrs_sample_batched_rows(const wrs_row *d_rows, const uint64_t *d_off, uint32_t ntab,
                            const uint64_t *d_cnt_off, uint64_t seed, uint32_t *d_out,
                            void *stream);

/* ---------------------------------------------------------------------- */
/* Tables and batches as objects (the problem statement's interface)       */
/* ---------------------------------------------------------------------- */
/* Sec. 1 states the problem as: build a structure from weights w_1..w_N,
 * then draw samples i with probability w_i / W.  These calls give exactly
 * that interface over the buffer calls above: a wrs_table owns the device
 * rows of one alias table (Sec. 2.2), a wrs_batch those of many.  Objects
 * belong to the device that was current when they were built; sampling
 * from another device returns WRS_EINVAL.  Scratch memory of a call is
 * taken with cudaMallocAsync on the call's stream and freed on it. */
typedef struct wrs_table wrs_table;
typedef struct wrs_batch wrs_batch;

/* Process-wide build settings used by wrs_build (section size, split
 * method); the buffer calls take theirs per call.  wrs_set_config checks
 * the values as wrs_build_rows does (WRS_EINVAL, nothing changed);
 * wrs_get_config returns the current ones (wrs_config_default until set). */
int wrs_set_config(const wrs_config *cfg);
int wrs_get_config(wrs_config *cfg);

/* Build the alias table of n FP32 weights (PSA, Sec. 2.2 and Sec. 4):
 * w is a device pointer (w_on_device != 0, 4-byte aligned) or a host
 * pointer (copied in on `stream`).  The call synchronises `stream` and
 * returns the build's status: WRS_OK with *out set, or an argument, memory
 * or data error (WRS_EINVAL for a negative weight, WRS_ENONFINITE,
 * WRS_EZEROSUM) with *out untouched and nothing left allocated.  The table
 * equals wrs_build_rows of the same weights under wrs_get_config's settings
 * bit for bit.  Free it with wrs_table_destroy. */
int wrs_build(const float *w, uint64_t n, int w_on_device, void *stream, wrs_table **out);

/* Draw `count` samples from a table into d_out (device, count uint32 item
 * indices) with a sampling mode of Sec. 5 (enum wrs_sample_mode):
 *  - WRS_SAMPLE_NAIVE: samples 0..count-1 of stream (seed, 0, WRS_TAG_NAIVE),
 *    as wrs_sample_rows;
 *  - WRS_SAMPLE_CACHED / WRS_SAMPLE_LIMITED (8192 rows per section) and
 *    WRS_SAMPLE_SMEM (4096 rows per section): as wrs_sample_sectioned_rows,
 *    output grouped by section;
 *  - WRS_SAMPLE_AUTO: as wrs_sample_auto.
 * Deterministic for (table, count, seed, mode).  Only enqueues work. */
int wrs_sample(const wrs_table *t, uint64_t count, uint64_t seed, uint32_t *d_out, int mode,
               void *stream);

/* Size, exact total weight W and light/heavy counts of a built table
 * (any out pointer may be NULL).  An imported table reports the W it was
 * given and UINT64_MAX for nl and nh (unknown). */
int wrs_table_info(const wrs_table *t, uint64_t *n, double *W, uint64_t *nl, uint64_t *nh);
/* Device pointer to the table's n rows (valid until wrs_table_destroy), for
 * the buffer calls. */
int wrs_table_rows(const wrs_table *t, const wrs_row **d_rows);
/* Copy the n rows into dst (host or device); blocks until done.  This is
 * the checkpoint path: wrs_table_import restores the same table. */
int wrs_table_export(const wrs_table *t, wrs_row *dst, int dst_on_device);
/* A table from n rows (host or device, e.g. written by wrs_table_export)
 * and its total weight W (NaN if unknown).  The rows are checked on the
 * device: every prob in [0, 1] and every alias < n, else WRS_EINVAL. */
int wrs_table_import(const wrs_row *src, uint64_t n, int src_on_device, double W,
                     wrs_table **out);
int wrs_table_destroy(wrs_table *t);

/* Build ntab tables of a batch in one launch (as wrs_build_batched_rows,
 * with the tables handed out largest first and the tiling that
 * wrs_batch_autotune chose for this batch shape, if it has timed one, else
 * the default).  d_w, d_off as for wrs_build_batched_rows (device).  The
 * call synchronises `stream`.  Tables with a data error keep a status
 * (wrs_batch_status); the others are built.  Returns WRS_EINVAL for
 * offsets that do not start at 0 or decrease. */
int wrs_build_batched(const float *d_w, const uint64_t *d_off, uint32_t ntab, void *stream,
                      wrs_batch **out);
/* Per-table status (host int32[ntab]) / summaries (host wrs_table_summary[ntab]). */
int wrs_batch_status(const wrs_batch *b, int32_t *h_status);
int wrs_batch_summaries(const wrs_batch *b, wrs_table_summary *h_out);
/* Device rows, device offsets (ntab+1) and table count of a batch (any out
 * pointer may be NULL). */
int wrs_batch_rows(const wrs_batch *b, const wrs_row **d_rows, const uint64_t **d_off,
                   uint32_t *ntab);
/* Copy the rows of every table (d_off[ntab] rows, table-local aliases) into
 * dst (host or device); blocks until done. */
int wrs_batch_export(const wrs_batch *b, wrs_row *dst, int dst_on_device);
/* Sample every table of a batch in one launch, as wrs_sample_batched_rows:
 * d_cnt_off (device, ntab+1) delimits each table's samples in d_out. */
int wrs_sample_batched(const wrs_batch *b, const uint64_t *d_cnt_off, uint64_t seed,
                       uint32_t *d_out, void *stream);
int wrs_batch_destroy(wrs_batch *b);

/* ---------------------------------------------------------------------- */
/* Request loop: resident tables, continuous batching                      */
/* ---------------------------------------------------------------------- */
/* A server owns one worker thread on the calling thread's current device.
 * Requests are queued from any thread and served in steps: all admissible
 * requests that have arrived are built -- tables below 2^17 items with one
 * batched-build launch, larger ones each with the multi-CTA pipeline of
 * wrs_build_rows (section size 1024, p-ary splits) -- and sampled with one
 * sampling launch; up to max_inflight steps run on the GPU at once while new
 * arrivals form the next step.  Builds are admitted while resident tables
 * plus in-flight scratch stay within hbm_budget bytes (a table costs 8 bytes
 * per item while resident and about 12-14 bytes per item while it is
 * built); they are admitted in arrival order, and a build that can never fit
 * fails with WRS_ENOMEM.  The paper has no counterpart: it is how a serving
 * system uses the method.
 *
 * Results do not depend on batching: a table equals wrs_build_rows of the
 * same weights, and the samples of a request equal wrs_sample_rows(rows, n,
 * 0, count, seed, stream_lo, WRS_TAG_NAIVE) on that table.
 *
 * Buffers passed to a request must stay valid until the request is done:
 * weights w (host or device, 1..2^31-1 items) and the sample output out
 * (host or device, count uint32).  Tickets name requests; the ticket of a
 * build also names its table. */
typedef struct wrs_server wrs_server;

typedef struct wrs_server_statistics {
    uint64_t completed, builds, samples, releases, errors;
    uint64_t items_built, samples_drawn, steps;
    double mean_step_requests;
    uint64_t resident_bytes, peak_bytes;
    double p50_ms, p99_ms, mean_ms;   /* latency: submit to completion */
    double wall_s;                    /* first submit to last completion */
} wrs_server_statistics;

int wrs_server_create(uint64_t hbm_budget, uint32_t max_inflight, wrs_server **out);
int wrs_server_submit_build(wrs_server *s, const float *w, uint64_t n, int w_on_device,
                            uint64_t *ticket);
int wrs_server_submit_sample(wrs_server *s, uint64_t table, uint64_t count, uint64_t seed,
                             uint32_t stream_lo, uint32_t *out, int out_on_device,
                             uint64_t *ticket);
int wrs_server_submit_release(wrs_server *s, uint64_t table, uint64_t *ticket);
/* done = 1 once the request finished; status is its result (WRS_OK,
 * WRS_ENOMEM, WRS_ENOTFOUND for an unknown or released table, a data error
 * of the build, WRS_ECUDA). */
int wrs_server_poll(wrs_server *s, uint64_t ticket, int *done, int *status);
int wrs_server_wait(wrs_server *s, uint64_t ticket, int *status);
/* Device rows of a built, resident table (valid until it is released). */
int wrs_server_table(wrs_server *s, uint64_t table, const wrs_row **d_rows, uint64_t *n,
                     double *W);
/* Copy the rows of a built, resident table into dst (n rows, host or device);
 * blocks until the copy is done.  This is the checkpoint/export path. */
int wrs_server_export(wrs_server *s, uint64_t table, wrs_row *dst, int dst_on_device);
int wrs_server_stats(wrs_server *s, wrs_server_statistics *out);
/* Finish every queued request, free every table, stop the worker. */
int wrs_server_destroy(wrs_server *s);

/* ---------------------------------------------------------------------- */
/* Measurement support                                                     */
/* ---------------------------------------------------------------------- */

/* Random-gather probe (the paper has no counterpart; it measures the
 * hardware): `count` uniformly random 8-byte reads from d_rows[0..nrows),
 * one 4-byte store each into d_out[0..count).  The bench uses the best rate
 * over load paths and launch shapes as the roofline of the naive sampler,
 * whose cost is the same gather.  flavor: 0 = read-only path
 * (ld.global.nc), 1 = L2-only (ld.global.cg), 2 = streaming (ld.global.cs);
 * ctas_per_sm: 1..64 CTAs of 256 threads per SM (grid-stride loop);
 * loads_in_flight: 4, 8 or 16 independent loads per thread.  Contents of
 * d_out (4-byte aligned) are meaningless. */
int wrs_diag_random_gather(const wrs_row *d_rows, uint64_t nrows, uint64_t count,
                           uint64_t seed, int flavor, uint32_t ctas_per_sm,
                           uint32_t loads_in_flight, uint32_t *d_out, void *stream);

/* Per-table baseline of the batched build (measurement support; the paper
 * has no batched build): builds the tables of a batch laid out as for
 * wrs_build_batched_rows one after another with wrs_build_rows, one launch
 * sequence per table, from a loop on the host.  h_off: ntab+1 HOST offsets
 * (empty tables are skipped); d_ws: a build workspace for the largest table
 * (wrs_build_workspace_bytes); d_info: ntab device wrs_build_info records.
 * Rows and summaries equal wrs_build_rows of each segment (so, bit for bit,
 * the rows of wrs_build_batched_rows).  Returns the first argument or CUDA
 * error; data errors land in d_info[t].status. */
int wrs_diag_build_each(const float *d_w, const uint64_t *h_off, uint32_t ntab,
                        wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                        const wrs_config *cfg, wrs_build_info *d_info, void *stream);

/* Pack variants of Sec. 4.2 (Fig. 3), for measurement: the sweep-pack step
 * (wrs_step_pack) done by a sequential sweep per section instead of the
 * merge-path pack.  Same contract as wrs_step_pack: d_ws holds a build's
 * state after wrs_step_split with the same n and cfg; every variant writes
 * the rows wrs_step_pack writes, bit for bit.
 *   variant 0: one thread per section, list entries read from global
 *              memory, each weight gathered from d_w by the item index
 *              (d_w: the build's weights, device, 4-byte aligned);
 *   variant 1: the same with the weight read from the list entry (d_w may
 *              be NULL);
 *   variant 2: one warp per section stages its entries in shared memory,
 *              one lane sweeps them (d_w may be NULL).
 * Errors: WRS_EINVAL for another variant or misaligned pointers, otherwise
 * as wrs_step_pack. */
int wrs_diag_pack_variant(const float *d_w, uint64_t n, wrs_row *d_rows, void *d_ws,
                          uint64_t ws_bytes, const wrs_config *cfg, uint32_t variant,
                          void *stream);

/* Precision study (Sec. 2.2 keeps the prefix sums of the light and heavy
 * weights, the split comparisons and the sweep's residual in FP64; the
 * build does them in exact fixed point): the split and pack steps redone on
 * a build's lists with floating-point prefix arithmetic, for measurement.
 *   prec 0: FP64;  prec 1: pairs of FP32 values (hi + lo, about 48 bits)
 *   with compensated additions (TwoSum / Fast2Sum).
 * Checkpoint sums every 32 list entries (scanned), splits by a 32-ary search
 * over them and a warp search inside one interval, then the merge-path pack
 * of every section on keys A(i) = i avg - sl(i) and B(j) = sh(j+1) - (j+1) avg
 * (heavy h[j] closes before light l[i] iff B(j) <= A(i)); rows by item index.
 * d_ws: a build's workspace after wrs_step_partition (same n and cfg);
 * d_pws: wrs_diag_prec_workspace_bytes(n, cfg) bytes, 256-byte aligned.
 * section_size at most 1024.  The table is valid (tested by reconstructed
 * mass); it is not the exact build's table.  Errors: WRS_EINVAL for another
 * prec, a larger section or short/misaligned buffers. */
int wrs_diag_prec_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes);
int wrs_diag_prec_split_pack(uint64_t n, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                             void *d_pws, uint64_t pws_bytes, const wrs_config *cfg,
                             uint32_t prec, void *stream);

/* Philox-rate probe (measures the hardware; no counterpart in the paper):
 * ceil(count/2) Philox-4x32-10 calls, call c on counter
 * (c_lo, c_hi, 0, WRS_TAG_DIAG) under key (seed_lo, seed_hi), writing
 * d_out[2c] = x0 ^ x1 and d_out[2c+1] = x2 ^ x3 (d_out holds count
 * uint32; an 8-byte aligned device pointer).  The same calls and output bytes
 * as a sectioned sampler without the rows: the bench uses its rate as the
 * arithmetic roofline of the cached sectioned sampler.  Errors: WRS_EINVAL
 * for a null or not 8-byte aligned d_out with count > 0, WRS_ECUDA for a
 * failed launch. */
int wrs_diag_philox(uint64_t count, uint64_t seed, uint32_t *d_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* WRS_H */
