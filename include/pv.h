/*
 * libpv — query-pipeline code variants on one GB300 GPU (sm_103a).
 *
 * C ABI for the data-parallel hot path of Breß et al., "Generating Custom
 * Code for Efficient Query Execution on Heterogeneous Processors":
 *   register the columns of in-memory, column-major tables that already live
 *   in device memory (Section 7.6: column store, data cached on the device
 *   before execution, Section 9.1), build a hash table on a dimension in a
 *   build pipeline (Table 2; HASH_PUT of Table 1), run a probe/scan pipeline
 *   program (Table 1, Section 3.1) under one variant configuration
 *   (Section 3.3: execution strategy, data structure, code transformations),
 *   and fetch its result.
 *
 * Conventions for every call:
 *   - Return value: PV_OK (0) or a negative pv_status; pv_last_error() then
 *     holds a one-line message (ctx-owned, valid until the next call on ctx).
 *   - Device pointers are plain CUDA device addresses on the ctx's device.
 *     Columns are BORROWED: the caller keeps them alive and unmodified while
 *     any pipeline that reads them may run; the library never frees them.
 *   - Hash tables, results and graphs are OWNED by the ctx and released by
 *     pv_free() or pv_destroy().  Handles are ctx-local int32 > 0.
 *   - All GPU work is enqueued asynchronously on the ctx stream.  Errors that
 *     kernels detect (table full, cuckoo cycle, key out of range, duplicate
 *     build key, output overflow) are recorded in a device error word and
 *     returned by the next pv_sync(), pv_result_shape() or pv_fetch_result().
 *   - No call falls back to the CPU.  A pipeline whose shape has no compiled
 *     kernel runs on the generic GPU kernels; a variant axis that the chosen
 *     kernels do not implement returns PV_ERR_UNSUPPORTED.
 *   - A ctx is not thread-safe; use one ctx per host thread.
 */
#ifndef PV_H
#define PV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pv_status;
enum {
  PV_OK = 0,
  PV_ERR_INVALID_ARG = -1,      /* bad handle, size, alignment or spec */
  PV_ERR_UNSUPPORTED = -2,      /* beyond a documented limit, or a variant axis the kernels lack */
  PV_ERR_HT_FULL = -3,          /* linear-probing table or local table chain exhausted */
  PV_ERR_CUCKOO_CYCLE = -4,     /* cuckoo eviction chain exceeded its bound */
  PV_ERR_KEY_OUT_OF_RANGE = -5, /* perfect-array key outside the declared domain */
  PV_ERR_DUP_BUILD_KEY = -6,    /* two surviving build rows with one key */
  PV_ERR_OUTPUT_OVERFLOW = -7,  /* more projected rows than the output capacity */
  PV_ERR_TIMEOUT = -8,          /* pv_sync watchdog expired; work may still run */
  PV_ERR_CUDA = -9,             /* a CUDA runtime call failed */
  PV_ERR_OOM = -10              /* the allocator returned NULL */
};

typedef enum { PV_I32 = 0, PV_I64 = 1, PV_U8 = 2 } pv_type;

typedef struct pv_ctx pv_ctx;
typedef int32_t pv_col;   /* column handle */
typedef int32_t pv_ht;    /* hash-table handle */
typedef int32_t pv_res;   /* result handle */
typedef int32_t pv_graph; /* captured-graph handle */

#define PV_MAX_PREDS 4
#define PV_MAX_PROBES 4
#define PV_MAX_KEYS 3
#define PV_MAX_AGGS 8
#define PV_MAX_TERMS 3
#define PV_MAX_PROJ 4
#define PV_MAX_PAYLOAD 4

/* FILTER comparison (Table 1): column op constant, or lo <= column <= hi.
 * PV_PREFIX (string starts with a constant) is for pv_dict_range only; a
 * pv_pred never carries it. */
typedef enum { PV_LT = 0, PV_LE = 1, PV_GT = 2, PV_GE = 3, PV_EQ = 4, PV_BETWEEN = 5, PV_PREFIX = 6 } pv_cmp;
/* Distributive aggregate functions (Section 7.6). */
typedef enum { PV_SUM = 0, PV_COUNT = 1, PV_MIN = 2, PV_MAX = 3 } pv_func;
/* ARITHMETIC term (Table 1): x, x + c or c - x; an aggregate's value is the
 * product of its terms (e.g. price * (100 - disc) * (100 + tax)). */
typedef enum { PV_TERM_X = 0, PV_TERM_X_PLUS_C = 1, PV_TERM_C_MINUS_X = 2 } pv_term_kind;
/* Value reference: a column of the probe pipeline's table, or payload b of
 * the build row matched by probe a (HASH_PROBE binds the payload). */
typedef enum { PV_REF_COL = 0, PV_REF_PAYLOAD = 1 } pv_ref_kind;

typedef struct { int32_t kind; int32_t a; int32_t b; } pv_ref;
typedef struct { pv_col col; int32_t op; int64_t c0; int64_t c1; } pv_pred;
typedef struct { int32_t kind; pv_ref x; int64_t c; } pv_term;
typedef struct { int32_t func; int32_t n_terms; pv_term terms[PV_MAX_TERMS]; } pv_agg;
typedef struct { pv_ht ht; pv_col fk; } pv_probe;

/* Build pipeline (Table 2): LOOP over the key column's table, FILTER by the
 * conjunction of preds, HASH_PUT key -> payload columns.  Key and payload
 * columns are int32 (PV_I32) or uint8 (PV_U8) and have the same row count.
 * A table slot is 64 bits (32-bit key, 32 bits of payload): with one payload
 * column the slot holds its value; with two to four, the slot holds the build
 * row and a probe gathers the payload values from the payload columns (which
 * must then stay alive and unchanged while pipelines probe the table; such
 * tables are probed by the generic kernels). */
typedef struct {
  pv_col key;
  int32_t n_preds;
  pv_pred preds[PV_MAX_PREDS];
  int32_t n_payload;
  pv_col payload[PV_MAX_PAYLOAD];
} pv_build_spec;

/* Hash-table implementations (Section 5.1; perfect array added for dense
 * key domains) and hash functions (Section 9.2.2: Murmur or multiply-shift). */
typedef enum { PV_HT_LINEAR = 0, PV_HT_CUCKOO = 1, PV_HT_PERFECT = 2 } pv_ht_kind;
typedef enum { PV_HASH_MURMUR = 0, PV_HASH_MULTSHIFT = 1 } pv_hash_fn;

typedef struct {
  int32_t kind;           /* pv_ht_kind */
  int32_t hash;           /* pv_hash_fn (ignored by PV_HT_PERFECT) */
  int32_t cuckoo_k;       /* cuckoo hash functions, 2..4 (0 = 3) */
  int32_t max_evictions;  /* cuckoo eviction-chain bound (0 = 32 * log2(capacity)) */
  double load_factor;     /* slots >= rows / load_factor, power of two (<= 0: 0.5) */
  uint64_t seed;          /* hash-function seeds are derived from it */
} pv_ht_variant;

/* Probe/scan pipeline program (Table 1, Table 2): LOOP over the fact table,
 * FILTER (conjunction of preds), HASH_PROBE each probe in order (a miss drops
 * the row), then ARITHMETIC and one sink:
 *   n_proj > 0              PROJECT proj (n_aggs must be 0)
 *   n_keys > 0              HASH_AGGREGATE(keys, aggs)
 *   otherwise               AGGREGATE(aggs)
 * All fact columns referenced must have the same row count.
 * Group keys (the attribute set G of HASH_AGGREGATE, Table 1): one part of any
 * column type; two 32-bit parts (packed into one 64-bit key); or three parts,
 * or two of which one is 64 bits wide (a composite key: each part minus its
 * minimum, in mixed radix over the parts' value spans taken from column or
 * build-payload statistics; the product of the spans must be at most 2^40,
 * else PV_ERR_UNSUPPORTED). */
typedef struct {
  int32_t n_preds;
  pv_pred preds[PV_MAX_PREDS];
  int32_t n_probes;
  pv_probe probes[PV_MAX_PROBES];
  int32_t n_keys;
  pv_ref keys[PV_MAX_KEYS];
  int32_t n_aggs;
  pv_agg aggs[PV_MAX_AGGS];
  int32_t n_proj;
  pv_ref proj[PV_MAX_PROJ];
  int64_t capacity_hint;  /* PROJECT: output row capacity (0 = fact rows);
                             HASH_AGGREGATE: expected groups (0 = from column stats) */
} pv_pipeline_spec;

/* Variant configuration (Section 3.3, 4, 6; Table 5's dimensions). */
typedef enum { PV_EXEC_SINGLE_PASS = 0, PV_EXEC_MULTI_PASS = 1 } pv_exec;
/* PV_AGG_CLUSTER (perfect tables): the table is partitioned over the shared memory of the CTAs of a
 * thread-block cluster (the smallest power of two, 2..16, whose part fits) and updated with
 * cluster-scope atomics, then merged into the global table. */
typedef enum { PV_AGG_LOCAL = 0, PV_AGG_GLOBAL = 1, PV_AGG_CLUSTER = 2 } pv_agg_strategy;
/* PV_COMPACTED (grouped pipelines): branched first operation (the filters, else the
 * first probe); its surviving rows are queued per warp and run one per lane through
 * the rest of the pipeline, so later operations see full warps. */
typedef enum { PV_BRANCH = 0, PV_PREDICATED = 1, PV_COMPACTED = 2 } pv_pred_mode;
/* PV_STAGED (grouped predicated pipelines of compiled shapes, thread-private
 * tables, items_per_thread 1, no prefetch; else PV_ERR_UNSUPPORTED): grid-stride
 * chunks of 128 rows per warp; while a warp computes one chunk, the TMA engine
 * copies its next chunk of every column it reads into the warp's shared-memory
 * stage (bulk copies completing on an mbarrier).  A wait that gives up (a copy
 * that never completes) reports PV_ERR_TIMEOUT at the next pv_sync. */
typedef enum { PV_GRID_STRIDE = 0, PV_CHUNKED = 1, PV_STAGED = 2 } pv_access;

typedef struct {
  int32_t exec;              /* pv_exec: projection single pass (warp-aggregated atomics) or
                                count -> prefix sum -> scatter; aggregation: fused, or keys first */
  int32_t agg;               /* pv_agg_strategy for HASH_AGGREGATE */
  int32_t pred;              /* pv_pred_mode (all operations of the pipeline share it) */
  int32_t access;            /* pv_access: coalesced grid-stride, per-thread chunks, or TMA-staged chunks */
  int32_t ht;                /* pv_ht_kind of the aggregation table */
  int32_t hash;              /* pv_hash_fn of the aggregation table */
  int32_t block;             /* threads per CTA: 64..1024, multiple of 32 (0 = 256) */
  int32_t grid_mult;         /* CTAs = grid_mult * SMs (0 = as many as fit at once) */
  int32_t items_per_thread;  /* unroll: 4-row items per thread per trip, 1, 2 or 4 (0 = 2) */
  int32_t threads_per_table; /* PV_AGG_LOCAL: 1 = thread-private tables, 0 = one per CTA */
  int32_t cuckoo_k;          /* aggregation cuckoo hash functions (0 = 3) */
  int32_t prefetch;          /* grid-stride pipelines: bulk-prefetch each warp's column chunks this
                                many loop trips ahead into L2 (0 = off) */
  int32_t warp_agg;          /* HASH_AGGREGATE into global or cluster tables: 1 = lanes of a warp holding
                                the same group key first combine their aggregates (match_any), one lane
                                updates the table (Section 4's local pre-aggregation applied within a
                                warp); 0 = every row updates.  Shared-memory (local) tables ignore it. */
  int32_t interp;            /* 0: the kernel compiled for the pipeline's shape when one exists, else the
                                generic kernels; 1: always the generic kernels, which read the pipeline
                                program (predicates, probes, key parts, aggregate terms, projected values)
                                at run time, one row per thread.  The generic kernels implement the
                                branched and predicated modes, grid-stride access, single and multi pass,
                                and global or CTA-local tables; the other axes (chunked access, compacted
                                mode, thread-private and cluster tables, warp pre-aggregation) return
                                PV_ERR_UNSUPPORTED there. */
  int32_t compact_probes;    /* PV_COMPACTED, grouped pipelines without filters: probes the first stage
                                runs over whole items before queueing the survivors, 1 (0 = 1) or 2.
                                With 2, the second probe's key column is read in full instead of being
                                gathered for the queued rows; ungrouped pipelines and pipelines with
                                filters or one probe return PV_ERR_UNSUPPORTED for 2. */
  int32_t first_items;       /* PV_COMPACTED: 4-row items a lane takes through the first stage per loop trip,
                                1 (0 = 1) or 2; with 2 the loads of both items are in flight together before
                                either is filtered and queued.  Compiled for pipelines whose first operation
                                is a filter; probe-first pipelines return PV_ERR_UNSUPPORTED for 2, and 2
                                without PV_COMPACTED is PV_ERR_INVALID_ARG. */
  uint64_t seed;             /* aggregation hash seeds */
} pv_variant;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on `device` that enqueues on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  If alloc is non-NULL,
 * every device allocation goes through alloc(bytes, user) and free_(ptr,
 * user) (e.g. a framework's caching allocator); otherwise cudaMallocAsync /
 * cudaFreeAsync on the ctx stream.  *out is set to NULL on error. */
pv_status pv_create(pv_ctx** out, int device, void* cuda_stream,
                    void* (*alloc)(size_t bytes, void* user),
                    void (*free_)(void* ptr, void* user), void* user);
/* Waits for the ctx stream, then frees every owned table, result and graph. */
pv_status pv_destroy(pv_ctx* ctx);
/* Message of the last failing call on ctx; "" if none.  Never NULL. */
const char* pv_last_error(const pv_ctx* ctx);
/* Multiprocessor count and L2 bytes of the ctx device. */
pv_status pv_device_info(pv_ctx* ctx, int32_t* sm_count, int64_t* l2_bytes);
/* L2 fetch granularity of the process's CUDA context on the ctx device (the context limit
 * cudaLimitMaxL2FetchGranularity): the bytes an L2 miss fetches from DRAM at most, 32, 64 or 128.  Not in the
 * paper: a memory-system setting for the lazily loaded columns of branched and compacted execution (Section
 * 6), whose rows are read sparsely.  At 32 bytes DRAM moves the sector-exact bytes; a context never given a
 * value fetched whole 128-byte lines for these kernels on GB300 (although the runtime reports 64 for it).
 * The limit belongs to the CUDA context, so it applies to every kernel the process launches on that device
 * afterwards (this library's and others'), and it ends with the process: no GPU setting changes.  *previous
 * (optional) receives the value the runtime reports before the call.  Other values are PV_ERR_INVALID_ARG;
 * the runtime refusing the limit is PV_ERR_CUDA.  Blocks; not capturable. */
pv_status pv_set_l2_fetch_bytes(pv_ctx* ctx, int32_t bytes, int32_t* previous);

/* Registers a borrowed device column (column-major table storage, Section
 * 7.5).  dev_ptr must be 16-byte aligned (vector loads); n_rows >= 0.
 * table/name are copied and only used in messages. */
pv_status pv_register_column(pv_ctx* ctx, const char* table, const char* name, int32_t type,
                             const void* dev_ptr, int64_t n_rows, pv_col* out);
/* Min and max of a column, computed on the GPU and cached (column
 * statistics for perfect-array domains and the cost model).  Blocks. */
pv_status pv_column_stats(pv_ctx* ctx, pv_col col, int64_t* min_out, int64_t* max_out);

/* ---- build pipelines ---------------------------------------------------- */

/* Runs one build pipeline (Table 2: LOOP, FILTER, HASH_PUT) into a new
 * ctx-owned table of the requested implementation (Section 5.1).  Build and
 * probe use the same table and parameters: the handle carries them.
 * Duplicate surviving keys raise PV_ERR_DUP_BUILD_KEY at the next sync. */
pv_status pv_build_hash_table(pv_ctx* ctx, const pv_build_spec* spec, const pv_ht_variant* var,
                              pv_ht* out);

/* Enqueues the build pipeline of an existing table again into the same slots
 * (clear, insert, duplicate check) after its input columns changed in place.
 * Allocates nothing and does not synchronise, so it may be recorded by
 * pv_graph_capture_begin/end together with the pipelines that probe the table;
 * the payload statistics of the first build (perfect-array domains) are kept. */
pv_status pv_rebuild_hash_table(pv_ctx* ctx, pv_ht ht);

/* ---- probe / scan pipelines --------------------------------------------- */

/* Enqueues the pipeline program under the variant and returns a ctx-owned
 * result handle.  Allocates the result (and scratch) before enqueueing.
 * Every spec within the limits above runs: on the kernel compiled for its
 * shape, or else on the generic kernels (see pv_variant.interp).  Limits that
 * return PV_ERR_UNSUPPORTED: more than 8 distinct fact columns; a group key of
 * three parts (or of two, one 64 bits wide) whose parts' value spans multiply
 * to more than 2^40; a variant axis the chosen kernels do not implement. */
pv_status pv_run_pipeline(pv_ctx* ctx, const pv_pipeline_spec* spec, const pv_variant* var,
                          pv_res* out);
/* Enqueues the same pipeline again into the same result buffers (clearing
 * them first).  Allocates nothing, so it may be recorded by
 * pv_graph_capture_begin/end. */
pv_status pv_rerun(pv_ctx* ctx, pv_res res);
/* Waits for the ctx stream (bounded by the watchdog, default 60 s) and
 * returns the first kernel-detected error since the last sync, clearing it. */
pv_status pv_sync(pv_ctx* ctx);
/* Watchdog limit of pv_sync in milliseconds (> 0). */
pv_status pv_set_timeout_ms(pv_ctx* ctx, int64_t ms);

/* Result layout: grouped results are n_keys key columns then n_aggs
 * aggregate columns (int64; key columns keep their source type widened to
 * int64), one row per non-empty group, in unspecified order.  Ungrouped
 * results are one row of n_aggs int64 columns (SUM/COUNT of no rows are 0;
 * MIN/MAX of no rows read 0).  Projection results keep each column's source
 * type and, for PV_EXEC_MULTI_PASS, input row order.  These calls sync. */
pv_status pv_result_shape(pv_ctx* ctx, pv_res res, int64_t* n_rows, int32_t* n_cols);
pv_status pv_result_col_type(pv_ctx* ctx, pv_res res, int32_t col, int32_t* type);
/* Copies column col (n_rows values of its type) into dst, which holds
 * dst_rows values, on the device if dst_on_device else in host memory.
 * Memory of the other kind (as the CUDA pointer attributes tell; managed
 * memory is either) is PV_ERR_INVALID_ARG, before anything is copied. */
pv_status pv_fetch_result(pv_ctx* ctx, pv_res res, int32_t col, void* dst, int64_t dst_rows,
                          int32_t dst_on_device);
/* All n_cols result columns at once: column col goes to dst[col], which holds
 * dst_rows[col] values (device or host memory as for pv_fetch_result).  The
 * copies are enqueued together and the call synchronises once. */
pv_status pv_fetch_results(pv_ctx* ctx, pv_res res, int32_t n_cols, void* const* dst, const int64_t* dst_rows,
                           int32_t dst_on_device);
/* Registers result column `col` of pipeline result `res` as a column of
 * table `table` (a pipeline's output feeding a later pipeline: a build over a
 * probe pipeline's result, or an aggregation over an earlier aggregation).
 * The column is the result's own device buffer, BORROWED from the result, so
 * it reflects every rerun of the result (also inside a captured graph), and
 * its row count is read on the device by each kernel that reads it, when
 * that kernel runs: a later pipeline or build enqueued behind the producing
 * pipeline on the ctx stream sees the rows it produced.  Column statistics
 * (perfect-array domains) are those of the column's source: the projected
 * fact column, the probed table's payload, or the group-key part; an
 * aggregate column's are computed from the rows present when first needed.
 * Pipelines over such columns run on the generic kernels; all their fact
 * columns must come from the same result.  pv_free(res) also forgets the
 * columns registered from it.  Errors: PV_ERR_INVALID_ARG for a bad handle or
 * column index; PV_ERR_CUDA. */
pv_status pv_register_result_column(pv_ctx* ctx, pv_res res, int32_t col, const char* table, const char* name,
                                    pv_col* out);

/* Which kernels a result runs on: *generic = 1 for the generic kernels, 0 for
 * the kernel compiled for its shape; the shape's canonical signature (the
 * fact column types by slot, predicate slots, probe key slots, key parts,
 * aggregate terms and projected values) is copied NUL-terminated into
 * buf[0..cap) when buf is non-NULL and cap > 0 (truncated to fit). */
pv_status pv_result_kernel(pv_ctx* ctx, pv_res res, int32_t* generic, char* buf, int64_t cap);

/* Enqueues, without synchronising, the copies of a result into caller memory:
 * column col (its full capacity: every row the result can hold, of the
 * column's type) to dst[col], which holds dst_rows[col] >= that capacity
 * values, and the result's row count (int64) to *rows_dst.  dst and rows_dst
 * are host memory (page-locked for the copies to be asynchronous) or device
 * memory when dst_on_device (memory of the other kind is PV_ERR_INVALID_ARG,
 * as for pv_fetch_result).  The values are defined once the ctx stream has
 * passed this point (pv_sync, or an event recorded after the call); rows
 * beyond *rows_dst are undefined.  Kernel-detected errors are reported by the
 * next pv_sync.  Lets a caller overlap the next step's input copies and
 * kernels with this step's result copies. */
pv_status pv_enqueue_fetch(pv_ctx* ctx, pv_res res, int32_t n_cols, void* const* dst, const int64_t* dst_rows,
                           int64_t* rows_dst, int32_t dst_on_device);
/* As pv_enqueue_fetch, but one kernel copies only the result's live rows:
 * the first min(row count, capacity) rows of column col to dst[col] (which
 * must still hold dst_rows[col] >= the capacity values: the count is not
 * known on the host when the call is enqueued), and that number of rows
 * (int64) to *rows_dst.  dst and rows_dst must be memory the device can
 * write: device (or managed) memory, or page-locked host memory (written
 * through its device address); pageable host memory is PV_ERR_INVALID_ARG.
 * The bytes crossing to the host are those of the live rows, not of the
 * capacity.  Defined once the ctx stream has passed this point; safe to
 * capture in a graph.  Kernel-detected errors (an overflowing result: its
 * first capacity rows are copied) are reported by the next pv_sync. */
pv_status pv_enqueue_fetch_rows(pv_ctx* ctx, pv_res res, int32_t n_cols, void* const* dst, const int64_t* dst_rows,
                                int64_t* rows_dst);
/* Rows a result can hold (the capacity pv_enqueue_fetch copies). */
pv_status pv_result_capacity(pv_ctx* ctx, pv_res res, int64_t* rows);

/* Releases a table, result or graph handle (columns: forgets the handle). */
pv_status pv_free(pv_ctx* ctx, int32_t handle);

/* ---- CUDA graphs -------------------------------------------------------- */

/* Records every pv_rerun, pv_rebuild_hash_table (and pv_l2_flush) enqueued between begin and end
 * into one CUDA graph, replayed by pv_graph_launch on the ctx stream (many
 * small pipelines without per-launch overhead).  No other pv call may run
 * in between. */
pv_status pv_graph_capture_begin(pv_ctx* ctx);
pv_status pv_graph_capture_end(pv_ctx* ctx, pv_graph* out);
pv_status pv_graph_launch(pv_ctx* ctx, pv_graph g);

/* ---- measurement support ------------------------------------------------ */

/* Cold-cache timing: overwrites a ctx-owned buffer of twice the L2 size (evicting
 * every other line), then discards that buffer's lines from L2 without write-back,
 * leaving L2 cold and clean. */
pv_status pv_l2_flush(pv_ctx* ctx);
/* Kernels enqueued by the last pv_run_pipeline / pv_rerun / pv_build_hash_table. */
pv_status pv_last_launch_count(pv_ctx* ctx, int32_t* n);
/* Per-kernel GPU timing: when enabled, every kernel the library enqueues is
 * bracketed by two CUDA events on the ctx stream.  pv_kernel_times syncs and
 * writes the durations (ms) of the kernels enqueued by the last
 * pv_run_pipeline / pv_rerun / pv_build_hash_table, in launch order, into
 * ms[0..max), and their count into *n.  Not recorded inside graph capture. */
pv_status pv_set_kernel_timing(pv_ctx* ctx, int32_t enable);
pv_status pv_kernel_times(pv_ctx* ctx, float* ms, int32_t max, int32_t* n);
/* Measured random-atomic throughput, the roofline of global aggregation
 * tables that outgrow L2 (Section 9.2.2 aggregation with many groups): a
 * ctx-allocated table of `slots` x `words` zeroed 64-bit words receives
 * n_updates updates, each adding 1 with atomicAdd to every word of one
 * uniformly hashed slot.  One warm-up pass, an L2 flush, then one timed pass;
 * *ms = its duration from CUDA events.  Synchronises; allocates and frees the
 * table; not capturable.  words in 1..16; the table is at most 64 GB. */
pv_status pv_atomic_peak(pv_ctx* ctx, int64_t slots, int32_t words, int64_t n_updates, float* ms);
/* Enqueues one kernel that busy-waits for `ns` nanoseconds of GPU clock
 * (bounded; for exercising the pv_sync watchdog). */
pv_status pv_debug_spin(pv_ctx* ctx, int64_t ns);

/* ---- dictionary-coded strings ------------------------------------------- */

/* String predicates of FILTER (Table 1; Section 9.2.1 names the missing LIKE
 * operator as the reason some SSB and TPC-H queries were left out).  A string
 * column is an int32 column of codes into a dictionary: dict[0..n_entries)
 * are distinct NUL-terminated strings in strictly ascending byte order
 * (strcmp), and a row's code is the rank of its string.  Codes order like the
 * strings, so these host-only calls (no ctx, no device work) turn a string
 * predicate into a predicate on the codes.  The caller owns every buffer.
 * Errors: PV_ERR_INVALID_ARG for null pointers, n_entries outside 0..2^31-1,
 * a dictionary that is not strictly ascending, or a bad op. */

/* Inclusive code range [*lo, *hi] of the rows whose string s satisfies
 * s op s0 (PV_LT, PV_LE, PV_GT, PV_GE, PV_EQ), s0 <= s <= s1 (PV_BETWEEN), or
 * s starts with s0 (PV_PREFIX).  The constants need not be in the dictionary.
 * An empty range is returned as *lo = 1, *hi = 0.  s1 is read for
 * PV_BETWEEN only. */
pv_status pv_dict_range(const char* const* dict, int64_t n_entries, int32_t op, const char* s0, const char* s1,
                        int64_t* lo, int64_t* hi);
/* Codes of the dictionary strings that match the SQL LIKE pattern ('%' any
 * run of bytes, '_' one byte, no escape character), ascending: the first
 * min(count, capacity) go to codes[], the count to *n_match.  A set that is
 * not one range is applied as a semi-join: a build pipeline over these codes
 * and a HASH_PROBE of the code column. */
pv_status pv_dict_match(const char* const* dict, int64_t n_entries, const char* pattern, int32_t* codes,
                        int64_t capacity, int64_t* n_match);

/* ---- cost model --------------------------------------------------------- */

/* A small fp32 network that predicts a variant's log run time from plan
 * features, column statistics and variant features, so that the variant of
 * each query can be chosen per query (the run-time optimizer Section 9.4
 * leaves to future work) instead of one heuristic per workload (Section
 * 8.3).  With F features (1..PV_MLP_MAX_FEATURES) and H = PV_MLP_HIDDEN:
 *     xh = (x - mu) / sigma;  z1 = xh W1 + b1;  h1 = relu(z1)
 *     z2 = h1 W2 + b2;        h2 = relu(z2);    y = h2 w3 + b3
 * params is one float vector of F*H + H + H*H + H + H + 1 values in the order
 * W1 (F x H row-major), b1, W2 (H x H row-major), b2, w3, b3.  All pointers
 * are device memory owned by the caller; every call enqueues on the ctx
 * stream and allocates nothing.  Errors: PV_ERR_INVALID_ARG for null
 * pointers or sizes out of range, PV_ERR_CUDA. */
#define PV_MLP_HIDDEN 64
#define PV_MLP_MAX_FEATURES 64

/* Forward pass of `batch` rows of x (batch x F, row-major) into y (batch).
 * act (batch x 2H: z1 then z2 per row) is written when non-NULL and is what
 * pv_mlp_backward needs. */
pv_status pv_mlp_forward(pv_ctx* ctx, const float* params, const float* x, const float* mu, const float* sigma,
                         int32_t batch, int32_t n_features, float* y, float* act);
/* Gradient of the mean squared error L = mean((y - target)^2) with respect to
 * params into grad (overwritten), and L into *loss (device float).  y and act
 * come from pv_mlp_forward on the same x; dz is caller scratch of
 * batch x (2H + 1) floats. */
pv_status pv_mlp_backward(pv_ctx* ctx, const float* params, const float* x, const float* mu, const float* sigma,
                          const float* act, const float* y, const float* target, int32_t batch,
                          int32_t n_features, float* dz, float* grad, float* loss);
/* One Adam step (Kingma and Ba, Algorithm 1) on n parameters in place, with
 * moment vectors m, v (zero before step 1) and step number step >= 1. */
pv_status pv_mlp_adam(pv_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t n, float lr,
                      float beta1, float beta2, float eps, int32_t step);

/* ---- allocation-free entry point ----------------------------------------- */

/* Largest row count pv_filter_project_noalloc accepts. */
#define PV_NOALLOC_MAX_ROWS (1LL << 28)

/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory: code whose device memory is owned by another
 * allocator (a database buffer pool or a framework's caching allocator that
 * has reserved the device), and latency-critical code that cannot pay for
 * cudaMalloc's device-wide synchronisation.  It needs no pv_ctx.
 *
 * Computes the multi-pass projection (count -> prefix sum -> scatter, as
 * pv_run_pipeline with PV_EXEC_MULTI_PASS) of
 *     SELECT a, price FROM t WHERE a_lo <= a <= a_hi AND b_lo <= b <= b_hi
 * over n_rows rows of the int32 columns a, b and the int64 column price
 * (device pointers, 16-byte aligned), writing the matching rows in input order
 * to out_a / out_price (device, out_capacity rows each).  On the stream it
 * writes *out_count (device int64) = rows written = min(matches,
 * out_capacity) and *out_status (device int32) = PV_OK, or
 * PV_ERR_OUTPUT_OVERFLOW when more rows matched than fit.
 *
 * It allocates nothing: its scratch (an error word plus per-tile counts and
 * offsets, about 1 MB) is one statically sized array in device memory that
 * every GPU loading this library holds until the process exits.  The first
 * call on a device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress) and caches it; make that first call before
 * any stream capture.  Every call shares the one array and each clears what
 * must start at zero, so calls that overlap on the GPU (other streams, other
 * host threads) race: order them on one stream.
 *
 * Returns PV_ERR_INVALID_ARG for n_rows outside [0, PV_NOALLOC_MAX_ROWS], a
 * negative capacity, null or misaligned pointers; PV_ERR_CUDA if a CUDA call
 * fails; otherwise PV_OK once the work is enqueued (asynchronous). */
pv_status pv_filter_project_noalloc(const int32_t* a, const int32_t* b, const int64_t* price, int64_t n_rows,
                                    int64_t a_lo, int64_t a_hi, int64_t b_lo, int64_t b_hi, int32_t* out_a,
                                    int64_t* out_price, int64_t out_capacity, int64_t* out_count,
                                    int32_t* out_status, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PV_H */
