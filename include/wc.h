/*
 * wc.h -- exact word-frequency counting on one GB300 GPU (sm_103a).
 *
 * The library implements the map and reduce of the MapReduce word counter of
 * arXiv 2206.05269 entirely on the GPU:
 *
 *   map    (Sec. 2 and Sec. 3.1: strip punctuation, lowercase, split into
 *           words): a word is a maximal run of ASCII letters [A-Za-z], each
 *           letter lowercased; every other byte separates words; a document
 *           edge separates words.
 *   reduce (Sec. 3.1-3.3: one dictionary per document, then the counts of
 *           each key summed across documents): exact integer counts per
 *           document, per document class and overall.
 *   order  count descending, then word bytes ascending (a proper prefix
 *           sorts first).
 *
 * The paper lists a GPU dictionary as future work (Sec. 5.2); here it is a
 * two-level open-addressing table (per-block shared memory, then global
 * memory) keyed by the full word bytes, so two different words never merge.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers, h_* are host pointers.
 *  - Calls that take a cudaStream_t are stream-ordered and asynchronous: the
 *    caller's device inputs must stay alive and unmodified until the stream
 *    reaches the call; results are valid once the stream has reached it.
 *    wc_table_size, wc_table_status and wc_table_export wait for the table.
 *  - Every call returns a wc_status; the library never aborts, prints or
 *    traps.  wc_last_error(ctx) gives a message for the last failure.
 *  - The library owns wc_table and wc_batch objects until *_free.
 *  - A context may be used from one host thread at a time.
 *  - Device-side capacity overflows (table, long-word table, long-word byte
 *    arena, probe limits) are reported as WC_ERR_CAPACITY by wc_table_status,
 *    wc_table_size and wc_table_export; such a table holds no partial result.
 *    Count again with larger capacities (wc_count_opts).
 */
#ifndef WC_H_
#define WC_H_

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WC_OK = 0,
    WC_ERR_INVALID_ARG = 1,  /* bad pointer, size, index or option */
    WC_ERR_OOM = 2,          /* device allocation failed */
    WC_ERR_BUDGET = 3,       /* the context's device-memory budget would be exceeded */
    WC_ERR_CAPACITY = 4,     /* a device table or arena overflowed; retry larger */
    WC_ERR_CUDA = 5,         /* a CUDA runtime call failed (message in wc_last_error) */
    WC_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    WC_ERR_INTERNAL = 7,
    WC_ERR_UNSUPPORTED = 8   /* input outside the documented limits */
} wc_status;

typedef struct {
    int device;                 /* CUDA device ordinal */
    uint64_t mem_budget_bytes;  /* 0 = no budget; device memory the context may hold at once: its
                                   tables, scratch and wc_buffer_alloc buffers, each charged from
                                   its allocation until its stream-ordered free has executed */
    int count_bits;             /* width of global/class counts: 32 or 64 (per-document counts are 32) */
    int autotune;               /* 1 = pick batched-kernel shapes by timing, cached per size class */
    const char *tune_cache_path;/* JSON cache for the autotuner; NULL = in-memory only */
} wc_config;

typedef struct wc_ctx wc_ctx;
typedef struct wc_table wc_table;
typedef struct wc_batch wc_batch;

/* Optional capacity hints for one count; zero fields pick automatic sizes. */
typedef struct {
    uint64_t table_slots;   /* short-word table slots (rounded up to a power of two) */
    uint64_t long_slots;    /* long-word (> 16 letters) table slots */
    uint64_t arena_bytes;   /* bytes for the distinct long words' text */
    int no_level1;          /* 1 = no shared-memory level-1 table (every word goes to the global
                               tables): the same result, for measuring what the level-1 table
                               saves; 0 = default */
} wc_count_opts;

enum { WC_TABLE_DOC = 0, WC_TABLE_CLASS = 1, WC_TABLE_GLOBAL = 2 };

/* Creates a context on cfg->device (NULL cfg = defaults: device 0, no
 * budget, 64-bit counts, no autotune).  *out is set on WC_OK only.  The
 * context is the resident state of the paper's GPU reduce (Sec. 3.3: the
 * device that sums the per-document counts), extended to the map (Sec. 5.2's
 * GPU dictionary): a stream-ordered memory pool charged against the budget,
 * capacity history, pinned metadata slots.  Errors: WC_ERR_INVALID_ARG (bad
 * device or count width), WC_ERR_CUDA. */
wc_status wc_create(const wc_config *cfg, wc_ctx **out);
/* Destroys the context and its memory pool.  Free every table, batch and plan
 * made with it first: they hold the context, and freeing one after its
 * context is gone is undefined. */
void wc_destroy(wc_ctx *ctx);

/* Counts the words of one document d_text[0, nbytes) into a new table with
 * ctx count width.  Implements Sec. 3 map + reduce for a single document
 * (the paper's per-document dictionary, built on the GPU).  nbytes may be 0.
 * d_text may have any alignment. */
wc_status wc_count(wc_ctx *ctx, const uint8_t *d_text, uint64_t nbytes, cudaStream_t stream,
                   wc_table **out);
wc_status wc_count_ex(wc_ctx *ctx, const uint8_t *d_text, uint64_t nbytes,
                      const wc_count_opts *opts, cudaStream_t stream, wc_table **out);

/* Counts one document held in host memory h_text[0, nbytes): the same table
 * as copying the text to the device and calling wc_count (the paper's map +
 * reduce with its host -> device copy, Sec. 3.3 and Sec. 4.1, made to overlap).
 * The text is copied into d_buf (device memory of at least nbytes bytes
 * owned by the caller, or NULL: the library takes it from the context's
 * pool and releases it after the count) in pieces of about piece_bytes (0:
 * automatic) cut after a non-letter byte, on a copy stream of the context,
 * and each piece is counted on `stream` as soon as it has landed, so copying
 * overlaps counting.  h_text must stay valid until the stream reaches the
 * end of the call; pinned memory lets the copies run asynchronously, other
 * memory is copied synchronously.  opts (may be NULL) sets capacities as for
 * wc_count_ex.  Errors as wc_count_ex. */
wc_status wc_count_host(wc_ctx *ctx, const uint8_t *h_text, uint64_t nbytes, uint8_t *d_buf, uint64_t piece_bytes,
                        const wc_count_opts *opts, cudaStream_t stream, wc_table **out);

/* Counts one document held in host memory that need not fit on the device
 * (Sec. 3.3's reduce applied across chunks): h_text[0, nbytes) is cut into
 * chunks of about chunk_bytes (0: 512 MB; at least 1 MB) after a non-letter
 * byte, each chunk is counted with wc_count_host through one reused device
 * buffer of the chunk size (its long words are copied into its table, so the
 * buffer can take the next chunk), a chunk whose table overflows is counted
 * again with four times the capacities (at most four times), and each
 * chunk's table is merged into the running total (wc_merge).  Device memory:
 * the buffer, one chunk's tables and two totals.  Waits for each chunk's
 * status; *out is the total.  Errors as wc_count_host and wc_merge. */
wc_status wc_count_stream(wc_ctx *ctx, const uint8_t *h_text, uint64_t nbytes, uint64_t chunk_bytes,
                          cudaStream_t stream, wc_table **out);

/* Counts ndocs documents in one pass: document i is d_text[d_offsets[i],
 * d_offsets[i+1]) (device uint64, non-decreasing, d_offsets[0] may be > 0).
 * d_class (device uint32, may be NULL) assigns each document a class below
 * nclasses.  Produces per-document tables (32-bit counts), per-class tables
 * and the global table (ctx count width): Sec. 3.1's per-document
 * dictionaries and Sec. 3.3's sum across documents.  ndocs and the offsets
 * on the host (h_offsets, same layout) are needed to plan the launch. */
wc_status wc_count_batched(wc_ctx *ctx, const uint8_t *d_text, const uint64_t *d_offsets,
                           const uint64_t *h_offsets, uint32_t ndocs, const uint32_t *d_class,
                           uint32_t nclasses, cudaStream_t stream, wc_batch **out);

/* wc_count_batched with flags.  WC_BATCH_EXACT_BOUNDS sizes the output and
 * the spill tables from bounds no input can exceed (a document of s bytes
 * has at most s/2 + 1 distinct words, s/18 + 1 of them 17 letters or
 * longer) instead of from estimates: far more memory, but it cannot fail
 * with WC_ERR_CAPACITY, so it is the recount after one.  Other flags:
 * WC_ERR_INVALID_ARG. */
enum { WC_BATCH_EXACT_BOUNDS = 1 };
wc_status wc_count_batched_ex(wc_ctx *ctx, const uint8_t *d_text, const uint64_t *d_offsets,
                              const uint64_t *h_offsets, uint32_t ndocs, const uint32_t *d_class,
                              uint32_t nclasses, uint32_t flags, cudaStream_t stream, wc_batch **out);

/* Waits for the batch; device-side overflow of its tables or output is
 * reported as WC_ERR_CAPACITY (count again with WC_BATCH_EXACT_BOUNDS;
 * nothing partial is kept). */
wc_status wc_batch_status(const wc_batch *batch);

/* Borrows one table of a batch (owned by the batch, freed with it; calling
 * wc_table_free on it does nothing).  kind = WC_TABLE_DOC (idx < ndocs, 32-bit
 * counts), WC_TABLE_CLASS (idx < nclasses, 32-bit counts) or
 * WC_TABLE_GLOBAL (ctx count width).  Waits for the batch; class and global
 * tables are built on the first request (Sec. 3.3's sum across documents). */
wc_status wc_batch_table(const wc_batch *batch, int kind, uint32_t idx, const wc_table **out);

/* Per-document top-k (Sec. 4.3 reports each speech's most frequent words):
 * borrows a table (owned by the batch, freed with it or when its plan runs
 * again; wc_table_free on it does nothing) whose rows are, document after
 * document, the first min(k, n_i) rows of document i's table, i.e. its top k
 * in (count desc, word asc) order.  Document i owns rows [h_first[i],
 * h_first[i] + h_n[i]); h_first and h_n (host, ndocs entries each, either may
 * be NULL) are filled before the call returns.  Read the rows with
 * wc_table_size / wc_table_export (32-bit counts).  Waits for the batch. */
wc_status wc_batch_topk(const wc_batch *batch, uint32_t k, uint64_t *h_first, uint32_t *h_n, const wc_table **out);

/* Waits for the batch; total per-document entries and their word bytes. */
wc_status wc_batch_size(const wc_batch *batch, uint64_t *nentries, uint64_t *word_bytes);

/* Copies every per-document table at once.  Entries are stored per document
 * (each document's entries are contiguous and in (count desc, word asc)
 * order); document i owns entries [h_doc_start[i], h_doc_start[i] +
 * h_doc_n[i]).  h_words / h_word_offsets (nentries+1) / h_counts (nentries)
 * are laid out as in wc_table_export over all entries.  Any pointer may be
 * NULL.  Waits until the copies are complete. */
wc_status wc_batch_export(const wc_batch *batch, uint64_t *h_doc_start, uint32_t *h_doc_n, uint8_t *h_words,
                          uint64_t *h_word_offsets, uint32_t *h_counts, cudaStream_t stream);

/* Vocabulary-id form of a batch (Sec. 3.3 sums every document's counts per
 * key; here the batch's global table, ordered by word, is that one shared
 * dictionary).  wc_batch_vocab borrows a table (owned by the batch, freed
 * with it or when its plan runs again; wc_table_free on it does nothing)
 * holding the batch's distinct words in word order, each with its global
 * count (64-bit, wc_table_export); a word's id is its row, so ids order as
 * their words.  wc_batch_export_ids copies every per-document entry as
 * (id, count): h_ids and h_counts (uint32, wc_batch_size entries, in the
 * order of wc_batch_export's rows: each document's entries contiguous, count
 * desc then word asc) and h_doc_start / h_doc_n as in wc_batch_export; any
 * pointer may be NULL.  An id decoded through the vocabulary is the word
 * wc_batch_export gives for that row.  Both wait for the batch and build the
 * class/global tables and the vocabulary on first use (device memory from
 * the context's pool).  Export size: 8 bytes a row plus the vocabulary once,
 * where wc_batch_export needs the word bytes plus 12 bytes a row. */
wc_status wc_batch_vocab(const wc_batch *batch, const wc_table **vocab);
wc_status wc_batch_export_ids(const wc_batch *batch, uint64_t *h_doc_start, uint32_t *h_doc_n, uint32_t *h_ids,
                              uint32_t *h_counts, cudaStream_t stream);

/* Plans: resident state for counting the same layout of documents again and
 * again (serving, repeated batches).  wc_plan_create plans ndocs documents
 * with the given host offsets (size classes, work items, capacities) and
 * allocates the output and scratch once.  wc_plan_run counts text laid out
 * with those offsets: the first run (after autotuning when the context
 * asks for it and knows no shapes yet: every per-document kernel shape of
 * each size class is timed on this input and the fastest kept, saved per
 * GPU in tune_cache_path; a context whose cache holds an entry for its GPU,
 * or one of whose plans was tuned already, uses those shapes untimed)
 * captures all device work into a CUDA graph; later runs with the same
 * pointers and stream replay it.  *out belongs to the plan and is rewritten
 * by the next run; wait for it (wc_batch_status) before reading it.  Run
 * the first call outside any stream capture. */
typedef struct wc_plan wc_plan;
wc_status wc_plan_create(wc_ctx *ctx, const uint64_t *h_offsets, uint32_t ndocs, uint32_t nclasses,
                         cudaStream_t stream, wc_plan **out);
wc_status wc_plan_run(wc_plan *plan, const uint8_t *d_text, const uint64_t *d_offsets, const uint32_t *d_class,
                      cudaStream_t stream, const wc_batch **out);
void wc_plan_free(wc_plan *plan);

/* Top-k of class `cls` by the ratio of in-class to out-of-class count
 * (Sec. 4.3's search for words one class uses more than the others, made
 * exact): cin/cout descending with cout = global - cin (cout = 0 ranks
 * first), then cin descending, then word ascending.  Writes up to k rows:
 * h_idx = index into the class table's sorted order, h_cin, h_cout.
 * *nout = rows written.  Waits for the batch. */
wc_status wc_class_ratio_topk(wc_ctx *ctx, const wc_batch *batch, uint32_t cls, uint32_t k,
                              cudaStream_t stream, uint64_t *h_idx, uint64_t *h_cin,
                              uint64_t *h_cout, uint32_t *nout);

/* Sums n tables word by word into a new table (Sec. 3.3: counts 10, 4 and 3
 * of one word reduce to 17).  Count width = ctx count width. */
wc_status wc_merge(wc_ctx *ctx, const wc_table *const *in, uint32_t n, cudaStream_t stream,
                   wc_table **out);

/* The first k rows of a table in its sorted order (k >= size: all rows):
 * the most frequent words, as Sec. 4.3 reports per speech.  Asynchronous;
 * *out is a new table owned by the caller (wc_table_free).  Errors:
 * WC_ERR_INVALID_ARG, WC_ERR_OOM / WC_ERR_BUDGET. */
wc_status wc_topk(wc_ctx *ctx, const wc_table *in, uint32_t k, cudaStream_t stream,
                  wc_table **out);

/* Waits for the table; reports WC_ERR_CAPACITY / WC_ERR_TIMEOUT from the device. */
wc_status wc_table_status(const wc_table *t);

/* Waits for the table, then gives its distinct words (the keys of the
 * paper's dictionary, Sec. 3.1), total count (tokens) and the bytes needed
 * for wc_table_export's h_words.  Any output pointer may be NULL.  A table
 * whose device work overflowed reports WC_ERR_CAPACITY and sizes 0. */
wc_status wc_table_size(const wc_table *t, uint64_t *nwords, uint64_t *ntokens,
                        uint64_t *word_bytes);

/* Copies the sorted table to the host (the word -> count dictionary of
 * Sec. 3.1, in count-descending, word-ascending order): h_words (word_bytes
 * bytes, words back to back), h_word_offsets (nwords+1 entries), h_counts
 * (nwords entries of uint32 or uint64 per wc_table_count_bits).  Buffers are
 * caller-owned, sized from wc_table_size.  Any pointer may be NULL to skip
 * that array.  Waits until the copy is complete. */
wc_status wc_table_export(const wc_table *t, uint8_t *h_words, uint64_t *h_word_offsets,
                          void *h_counts, cudaStream_t stream);
int wc_table_count_bits(const wc_table *t);

void wc_table_free(wc_table *t);
void wc_batch_free(wc_batch *b);

/* Counting for callers that cannot allocate device memory (the paper has no
 * counterpart: this is a deployment variant of wc_count).  Such callers
 * include code running while another component owns all device memory
 * through its own allocator, and services that forbid allocation after
 * start-up because an allocation can stall or fail at the wrong moment.
 * No context is needed and nothing is allocated: the hash tables and sort
 * scratch live in one fixed __device__ array of about 15.5 MB that every GPU
 * which loads the library holds until the process exits.
 *   d_text[0, nbytes): one document, nbytes <= 1 MiB (larger: returns
 *     WC_ERR_UNSUPPORTED; use wc_count).
 *   Outputs (device, caller-owned), the sorted table in wc_count's layout:
 *     d_khi, d_klo: big-endian first 16 letters of each word; d_cnt: counts;
 *     d_lref: 0, or 1 + index into d_loff/d_llen of a word of 17+ letters
 *     whose lowercased bytes are at d_arena + d_loff[i] (each followed by a
 *     0 byte).  out_cap >= 204800 entries, long_cap >= 8192, arena_cap >=
 *     nbytes + nbytes/16 + 16, else WC_ERR_INVALID_ARG.
 *     d_meta (8 x uint64): [0] distinct words, [1] words of 17+ letters,
 *     [3] total count, [4] bytes of all words; the low 32 bits of [7] are
 *     status bits, nonzero when the fixed tables overflowed (then the table
 *     is not valid).
 * Stream-ordered and asynchronous like wc_count: results are valid once the
 * stream has reached the call.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept per
 * device ordinal for the life of the process: calling after cudaDeviceReset,
 * or with a non-primary context current, is not supported.  All calls on a
 * device share the array and each clears it; calls whose work overlaps on the
 * GPU race, so keep them on one stream, in order. */
wc_status wc_count_noalloc(const uint8_t *d_text, uint64_t nbytes, uint64_t *d_khi, uint64_t *d_klo,
                           uint64_t *d_cnt, uint32_t *d_lref, uint64_t out_cap, uint64_t *d_loff,
                           uint64_t *d_llen, uint64_t long_cap, uint8_t *d_arena, uint64_t arena_cap,
                           uint64_t *d_meta, cudaStream_t stream);

/* The paper's numeric MapReduce (Sec. 4.2): *d_out (one device double) =
 * sum_{i=1}^{n} term(i) with term(i) = sqrt(i) (WC_SERIES_SQRT) or
 * (-1)^(i+1) / i (WC_SERIES_ALT_HARMONIC, whose limit is ln 2).  Each term is
 * an IEEE double (correctly rounded sqrt and division); the terms are summed
 * with Neumaier-compensated additions, per thread over a strided share of one
 * block's contiguous range, then over warps and blocks in a fixed order, so a
 * given GPU always returns the same value (no atomics).  n = 0 gives 0.
 * Asynchronous on `stream`; scratch (16 bytes a block) comes from the
 * context's pool.  Errors: WC_ERR_INVALID_ARG (unknown series, null
 * pointer), WC_ERR_UNSUPPORTED (n >= 2^53: indices no longer exact in
 * double), WC_ERR_BUDGET / WC_ERR_OOM. */
enum { WC_SERIES_SQRT = 0, WC_SERIES_ALT_HARMONIC = 1 };
wc_status wc_series_sum(wc_ctx *ctx, int series, uint64_t n, double *d_out, cudaStream_t stream);

/* The reduce of the paper's hybrid pipeline (Sec. 3.3 "Reduce on GPU",
 * measured in Sec. 4.1): the host maps every document to a dictionary and
 * lays the per-document counts of each word out as one row of a zero-padded
 * row-major matrix d_matrix[rows][cols] (device, uint32, caller-owned); this
 * call writes each row's sum to d_sums[rows] (device, uint64, caller-owned).
 * Kept to measure that design beside wc_count on the same GPU.  Asynchronous
 * on `stream`; rows = 0 does nothing.  Null pointers with rows > 0, or a
 * matrix of 2^64 bytes or more: WC_ERR_INVALID_ARG; launch failure:
 * WC_ERR_CUDA. */
wc_status wc_row_sums(const uint32_t *d_matrix, uint64_t rows, uint64_t cols, uint64_t *d_sums, cudaStream_t stream);

/* Device buffers charged against the context's budget.  The library's own
 * tables and scratch come from the context's stream-ordered pool and count
 * against mem_budget_bytes; these calls let a caller hold its input there
 * too (a serving loop's request text), so that one budget covers everything
 * resident for the context.  The paper's GPU reduce copies its count matrix
 * to the device for each call (Sec. 3.3); nothing there is budgeted.
 *   wc_buffer_alloc: `bytes` of device memory (256-byte aligned), allocated
 *     in stream order on `stream`; *out is set on WC_OK only.  WC_ERR_BUDGET
 *     when the budget cannot hold `bytes` more (nothing is allocated: wait
 *     for the context's other work to be freed and try again); WC_ERR_OOM.
 *   wc_buffer_free: returns a buffer (same context, pointer and byte count)
 *     in stream order on `stream`: work enqueued on `stream` before the call
 *     may still read it, so its bytes stay charged to the budget until the
 *     stream has passed the free; a NULL pointer is a no-op.
 *   wc_mem_usage: the bytes the context holds now (tables, scratch and these
 *     buffers not yet freed) and the largest such figure since creation or
 *     the last reset; reset != 0 restarts the peak from the current use.
 *     Any output pointer may be NULL. */
wc_status wc_buffer_alloc(wc_ctx *ctx, uint64_t bytes, cudaStream_t stream, void **out);
wc_status wc_buffer_free(wc_ctx *ctx, void *p, uint64_t bytes, cudaStream_t stream);
wc_status wc_mem_usage(wc_ctx *ctx, uint64_t *used, uint64_t *peak, int reset);

/* Stage tracing.  While enabled, the context records CUDA events on the
 * launching stream around three stages of wc_count / wc_count_ex (head
 * selection: the sampling pass and the head kernels; the main counting
 * kernel alone; compaction + sort) and around the compaction + sort of
 * wc_merge, and counts the kernels it launches.  wc_profile_read waits for
 * the recorded events and returns the summed stage times in milliseconds
 * (any output pointer may be null), how many main counting kernels were
 * timed, and how many kernels the library launched since enabling.
 * Enabling (or disabling) discards what was recorded. */
wc_status wc_profile_enable(wc_ctx *ctx, int enable);
wc_status wc_profile_read(wc_ctx *ctx, double *ms_head, double *ms_count, double *ms_finish,
                          uint64_t *count_launches, uint64_t *kernel_launches);

/* Read ceiling (measurement, not the paper's method): reads d_text[0,
 * nbytes) once with 16-byte streaming loads (any alignment; byte loads for
 * the ragged ends) and folds every byte into d_sink (device, sink_words
 * uint64 words, overwritten; at least one).  A pass that reads the text
 * once cannot beat this kernel's time, so it is the practical HBM limit for
 * the counting kernel.  Asynchronous on `stream`; null pointers or
 * sink_words == 0: WC_ERR_INVALID_ARG. */
wc_status wc_read_ceiling(const uint8_t *d_text, uint64_t nbytes, uint64_t *d_sink, uint32_t sink_words,
                          cudaStream_t stream);

/* Self-test of the device-side failure path (no part of the paper's method:
 * every device wait of the library is bounded and reports WC_ERR_TIMEOUT
 * instead of hanging).  Runs the counting kernel's bounded barrier wait in
 * one block on `stream`, on a barrier that expects one arrival: with
 * arrive != 0 the block makes that arrival first and the call returns
 * WC_OK; with arrive == 0 nothing arrives, the wait gives up after `polls`
 * polls (1 .. 2^22) and the call returns WC_ERR_TIMEOUT, the context staying
 * usable.  Waits for the stream.  polls outside that range:
 * WC_ERR_INVALID_ARG. */
wc_status wc_selftest_wait(wc_ctx *ctx, uint32_t polls, int arrive, cudaStream_t stream);

const char *wc_status_str(wc_status s);
const char *wc_last_error(const wc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* WC_H_ */
