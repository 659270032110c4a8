// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "wc_device.cuh"

namespace wc {

// Raises kernel `func`'s dynamic shared-memory limit to `bytes` on the
// calling thread's current device.  The attribute belongs to that device's
// context, so it is set once per (kernel, device, size): a process that
// counts on several devices sets it on each.  Safe to call from several host
// threads at once.
cudaError_t ensure_smem_limit(const void *func, int bytes);

// ---------------------------------------------------------------- counting
struct CountLaunch {
    const uint8_t *text;     // document bytes are text[lo, hi); long words may
                             // match representatives anywhere in text[0, hi)
    uint64_t lo, hi;
    GTable g;
    int grid;                // 0 = one persistent block per SM
    void *head_scratch;      // head_scratch_bytes() or null (no shared-memory head)
    cudaEvent_t main_ev[2];  // recorded (when non-null) right before the main counting kernel
    int head_mode;           // 0: build a head (texts >= count_global_head_min()); 1: reuse the
                             // head an earlier launch built in head_scratch; 2: no head
    int no_level1;           // 1: no shared-memory level-1 table at all (measurement)
};
// Tokenises and counts text[lo, hi) into g (8-byte, 16-byte and long tables).
cudaError_t launch_count_global(const CountLaunch &c, cudaStream_t s);
int count_global_chunk_bytes();
uint64_t count_global_head_min();
// One block runs the counting kernel's bounded barrier wait (see wc_selftest_wait).
cudaError_t launch_wait_selftest(uint32_t *d_status, uint32_t polls, int arrive, cudaStream_t s);
// Kernel launches of one launch_count_global: head selection when `head` and
// the text is long enough, the counting kernel, and the deferred long-word
// inserts when head scratch is given (`scratch`).
int count_global_launches(uint64_t nbytes, bool head, bool scratch);
size_t head_scratch_bytes();

// ---------------------------------------------------------------- dependent launches
// A kernel launched with launch_dependent may have its blocks scheduled
// before the previous kernel in the stream has finished; it must call
// grid_dependency_wait() before touching anything that kernel (or earlier
// work) reads or writes.  grid_dependency_trigger() lets the next dependent
// launch start once every block of the calling kernel has called it.  Both
// are no-ops for ordinary launches.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- numeric MapReduce
// Blocks of the series sum for n terms, and its two launches (per-block
// compensated partial sums into part[nb], then their fixed-order sum).
int series_blocks(unsigned long long n);
cudaError_t launch_series(int series, unsigned long long n, double2 *part, int nb, double *d_out, cudaStream_t s);

// Row sums of a row-major uint32 matrix (the hybrid pipeline's reduce).
cudaError_t launch_row_sums(const uint32_t *m, unsigned long long rows, unsigned long long cols,
                            unsigned long long *out, cudaStream_t s);

// ---------------------------------------------------------------- tables
// A compacted, sorted table in device memory.  Entry i: big-endian key
// halves (first 16 letters), count, and lref (0 = word fits the key, else
// 1 + index into loff/llen of a long word whose bytes are in arena).
struct DevTable {
    uint64_t cap;            // entry capacity of the arrays below
    uint64_t lcap;           // long-word entry capacity
    uint64_t arena_cap;
    int count_bits;          // 32 or 64
    unsigned long long *d_meta;   // [0] n entries, [1] n long, [2] arena bytes used, [3] tokens
    uint32_t *d_status;
    unsigned long long *khi, *klo;
    void *cnt;               // uint32_t or unsigned long long [cap]
    uint32_t *lref;
    unsigned long long *loff, *llen;
    uint8_t *arena;
};

// Scratch for compaction + sort of up to `cap` entries.
// Radix passes of the entry sort: 10 byte digits of the packed 16-letter
// prefix (5 bits a letter, 80 bits), 8 digits of the complemented count, and
// 4 document digits when a batch is sorted per document.
constexpr int kSortKeyPasses = 10;
constexpr int kSortPasses = kSortKeyPasses + 8;
constexpr int kSortPassesSeg = kSortPasses + 4;

// A radix pass sorts tiles of kSortTileElems entries.  A small sort (at most
// kSortFusedMaxTiles tiles by capacity) needs no scan pass: each tile finds
// its digit offsets from the counts of the tile groups before its own group
// and of the tiles before it in its group, in groups of sort_group_tiles(t)
// tiles for t tiles (a power of two of at least sqrt(t)), so at most
// sort_group_stride(capacity tiles) groups.  Larger sorts scan the tile
// counts in a pass of their own.
constexpr uint64_t kSortTileElems = 4096;
constexpr uint64_t kSortFusedMaxTiles = 1024;
__host__ __device__ constexpr uint64_t sort_group_tiles(uint64_t ntiles) {
    uint64_t g = 1;
    while (g * g < ntiles) g <<= 1;
    return g;
}
constexpr uint64_t sort_group_stride(uint64_t ntiles_cap) {
    uint64_t r = 1;
    while (r * r < ntiles_cap) r++;
    return r + 1;
}

struct SortScratch {
    uint64_t cap;
    unsigned long long *khi, *klo, *cnt;
    unsigned long long *pk;  // packed prefix, low 64 bits (written by the sort)
    uint32_t *pk2;           // packed prefix, high 16 bits
    uint32_t *lref;
    uint32_t *perm[2];
    uint32_t *doc;           // document of each entry (segmented sorts)
    uint32_t *hist_all;      // 24 x 256
    uint32_t *tile_hist;     // 256 x ntiles
    uint32_t *cur;           // 25
    uint32_t *group_hist[2]; // 256 x group_stride each: digit counts per tile group, by pass parity
    uint32_t group_stride;
    uint32_t *look[2];       // 256 x ntiles each: per-tile digit counts published for the look-back, by pass parity
    uint32_t *tile_ctr;      // [2]: tiles taken in launch order, by pass parity
    // merge sort of a single table (null when the scratch was carved without
    // it): 128-bit keys, the high and low words of buffer 0, then of buffer 1
    // (the indices travel in perm[0] and perm[1])
    unsigned long long *mk[4];
    // permutation buffer c (0 or 1), selected without indexing the parameter array
    __device__ __forceinline__ uint32_t *perm_buf(uint32_t c) const { return c ? perm[1] : perm[0]; }
    __device__ __forceinline__ uint32_t *group_buf(uint32_t c) const { return c ? group_hist[1] : group_hist[0]; }
    __device__ __forceinline__ uint32_t *look_buf(uint32_t c) const { return c ? look[1] : look[0]; }
};
// Slot of SortScratch::cur where a radix pass records a look-back that gave
// up waiting (the finish then reports WC_ERR_TIMEOUT).
constexpr int kCurSortError = 30;
// with_msort: also the merge sort's key buffers (32 bytes an entry), which a
// single table's finish then uses (see finish_table).
size_t sort_scratch_bytes(uint64_t cap, bool with_msort = false);
void sort_scratch_carve(SortScratch &s, void *base, uint64_t cap, bool with_msort = false);
// Zeroes what a sort accumulates into (digit histograms, pass cursors, group
// counts, the first pass's look-back buffer and the tile counters): every
// sort of a scratch starts with this (stream-ordered memsets).
void sort_state_reset(SortScratch &ss, cudaStream_t st);

// Word bytes of table entries for ordering long words that share a prefix.
struct LongView {
    const uint32_t *lref;
    const unsigned long long *loff, *llen;
    const uint8_t *arena;
};
// Slot of SortScratch::cur naming the permutation buffer that holds a
// finished sort's order.
constexpr int kCurFinal = 31;
// Radix passes the host knows to be constant, not launched at all: the count
// digits above the bytes of `max_count` (a bound on every count) and the
// document digits above those of `ndocs - 1` (bit p: pass p skipped).
uint32_t sort_skip_mask(uint64_t max_count, uint64_t ndocs);
// Stable LSD radix sort of ss's n = meta[0] entries by (count desc, word asc);
// with passes == kSortPassesSeg the document is the most significant key.
// The result is the permutation ss.perm_buf(ss.cur[kCurFinal]) (device value).
cudaError_t sort_entries(SortScratch &ss, const unsigned long long *meta, const LongView &v, int passes,
                         cudaStream_t st, uint32_t skip = 0);
int sort_entries_launches(int passes, uint64_t cap, uint32_t skip = 0);

// Compacts the global hash tables into unsorted scratch arrays and copies
// the long words into out.arena; then sorts and writes `out`.  The sort is a
// merge sort when ss has its key buffers and `skip` shows every count below
// 2^32 (the radix sort's count digits 4..7 skipped), else the radix sort.
// finish_table_launches(ss, skip) kernels are launched.
int finish_table_launches(const SortScratch &ss, uint32_t skip = 0);
cudaError_t finish_table(const GTable &g, uint64_t gcap8, uint64_t gcap, uint64_t glcap, SortScratch &ss,
                         DevTable &out, cudaStream_t s, uint32_t skip = 0);

// Compaction scans read kScanUnroll slots a thread per step (independent
// loads in flight) and reserve output positions with one atomic per block
// and step: block_take returns the first of `mine` positions reserved for
// the calling thread and adds the block's `tok` to *tokens and its count of
// positions to *kind (either may be null).
// Every thread of the block must call it (the loops step block-uniformly).
constexpr int kScanUnroll = 4;
struct BlockTake {
    uint32_t wsum[32];
    unsigned long long tok[32];
    unsigned long long base;
};
__device__ __forceinline__ unsigned long long block_take(BlockTake &sh, uint32_t mine, unsigned long long tok,
                                                         unsigned long long *counter, unsigned long long *tokens,
                                                         unsigned long long *kind = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    uint32_t incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) tok += __shfl_xor_sync(0xFFFFFFFFu, tok, d);
    if (lane == 31) sh.wsum[warp] = incl;
    if (lane == 0) sh.tok[warp] = tok;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        unsigned long long tt = 0;
        for (int w = 0; w < nw; w++) {
            const uint32_t v = sh.wsum[w];
            sh.wsum[w] = run;
            run += v;
            tt += sh.tok[w];
        }
        sh.base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
        if (tokens && tt) atomicAdd(tokens, tt);
        if (kind && run) atomicAdd(kind, (unsigned long long)run);
    }
    __syncthreads();
    const unsigned long long pos = sh.base + sh.wsum[warp] + incl - mine;
    __syncthreads();
    return pos;
}

// One table's sort arguments (device copies of them for finish_tables).
struct SortJob {
    SortScratch s;
    const unsigned long long *meta;
    LongView v;
    DevTable out;
};
// finish_table for n tables at once: each table's compaction, then every
// sort pass and the final gather as one launch over all n tables (grid.y).
// d_jobs: device memory of finish_tables_job_bytes(n), alive until the
// stream has run the launches.  finish_tables_launches(n, largest cap) kernels.
struct FinishSpec {
    GTable g;
    uint64_t gcap8, gcap, glcap;
    SortScratch *ss;
    DevTable *out;
};
size_t finish_tables_job_bytes(int n);
int finish_tables_launches(int n, uint64_t cap, uint32_t skip = 0);
cudaError_t finish_tables(const FinishSpec *spec, int n, void *d_jobs, cudaStream_t s, uint32_t skip = 0);

// Entries of finished tables re-inserted into a global hash table (merge).
struct MergeSrc {
    const unsigned long long *meta;
    const unsigned long long *khi, *klo;
    const void *cnt;
    const uint32_t *lref;
    const unsigned long long *loff, *llen;
    const uint8_t *arena;
    int count_bits;
    uint64_t cap;
    uint64_t arena_cap;
};
cudaError_t launch_merge_insert(const MergeSrc *d_src, const uint64_t *h_chunk_start, uint32_t nsrc,
                                uint64_t total_chunks, const GTable &g, cudaStream_t s);
constexpr int kMergeChunk = 1024;

cudaError_t launch_topk_copy(const DevTable &in, uint64_t k, DevTable &out, cudaStream_t s);

// Export: word lengths -> offsets -> bytes, on the device.
size_t export_scratch_bytes(uint64_t cap);
cudaError_t launch_export(const DevTable &t, void *scratch, uint8_t *d_words, unsigned long long *d_offs,
                          cudaStream_t s);

}  // namespace wc
