// Batched counting entry points: planning, capacities, launches, per-document
// views, class and global tables, the class-ratio ranking and bulk export.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wc.h"
#include "wc_batch.h"
#include "wc_host.h"

using namespace wc;

namespace {

constexpr uint64_t kSmallMax = 8 << 10;     // whole documents up to 8 KB: small shape
constexpr uint64_t kMediumMax = 32 << 10;   // whole documents up to 32 KB: medium shape; larger: large shape
constexpr uint64_t kSplitMin = 64 << 10;    // documents above 64 KB are split into ranges
constexpr uint64_t kRange = 32 << 10;       // byte range per item of a split document
constexpr uint32_t kMaxDocs = 1u << 24;     // (document, word) keys carry 24 document bits

uint64_t pow2_ge(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Distinct-word estimate of one document of s bytes: the larger of a Heaps'-law
// term 16 * T^0.6 (T = s/5 tokens) and s/16 (a large vocabulary seen in a
// mid-sized document), never above the exact bound ceil(s/2).
uint64_t est_distinct(uint64_t s) {
    if (!s) return 0;
    double t = (double)s / 5.0 + 1.0;
    double e = std::max(16.0 * std::pow(t, 0.6), (double)s / 16.0);
    return std::min<uint64_t>((uint64_t)std::min(e, t) + 16, s / 2 + 1);
}
// Output entries reserved for one document: the CSR output is never cleared,
// so reserve generously (s/8 entries is about two thirds of its tokens).
uint64_t out_reserve(uint64_t s) { return std::min<uint64_t>(s / 2 + 1, std::max(est_distinct(s), s / 8)) + 4; }

}  // namespace

struct BatchScratch {
    DocItem *items = nullptr;
    size_t ibytes = 0;
    uint32_t *next = nullptr;  // [2] queue cursors
    unsigned long long *smeta = nullptr;
    CountScratch cs;           // (document, word) tables + sort scratch
};

struct wc_batch {
    wc_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t ndocs = 0, nclasses = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    BatchArgs args{};
    uint32_t *d_class = nullptr;  // copy of the classes
    // planning
    std::vector<DocItem> items;
    uint32_t nsmall = 0, nmedium = 0;  // items: small, then medium, then large
    int shape_small = 1, shape_medium = 3, shape_large = 4;
    uint64_t cap8 = 0, cap16 = 0, caplong = 0;
    BatchScratch scr;
    // after sync
    bool synced = false;
    wc_status sync_status = WC_OK;
    uint64_t entries = 0, word_bytes = 0;
    // lazily built
    bool tables_built = false;
    bool exact = false;  // capacities at the exact bounds
    uint64_t max_doc_bytes = 0, total_bytes = 0;  // bounds on counts: no count exceeds half of these
    std::vector<wc_table *> class_tables;
    wc_table *global = nullptr;
    CountScratch gscratch;        // global hash tables kept for ratio lookups
    std::vector<wc_table *> views;
    // vocabulary ids (built on request, dropped when a plan runs again)
    wc_table *vocab = nullptr;    // the distinct words in word order, global counts
    uint32_t *d_ids = nullptr;    // per-document entry -> row of vocab
    size_t ids_bytes = 0;
};

static void drop_vocab(wc_batch *b, cudaStream_t s);

static wc_status batch_sync(const wc_batch *cb) {
    wc_batch *b = const_cast<wc_batch *>(cb);
    if (b->synced) return b->sync_status;
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return b->ctx->cuda_fail(e, "batch sync");
    unsigned long long meta[4];
    uint32_t st = 0;
    e = cudaMemcpy(meta, b->args.meta, sizeof(meta), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&st, b->args.status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return b->ctx->cuda_fail(e, "batch metadata");
    b->entries = meta[0];
    b->sync_status = WC_OK;
    if (st & (ST_TABLE_FULL | ST_LONG_FULL | ST_ARENA_FULL | ST_OUT_FULL)) b->sync_status = WC_ERR_CAPACITY;
    else if (st & ST_TIMEOUT) b->sync_status = WC_ERR_TIMEOUT;
    if (b->sync_status != WC_OK) {
        b->entries = 0;
        b->ctx->fail(b->sync_status, ("batched count overflowed a device table or output (status bits " +
                                      std::to_string(st) + "); count again").c_str());
    }
    b->synced = true;
    return b->sync_status;
}

// Words bytes and token totals of a view (meta[3], meta[4] zeroed before;
// any grid).
__global__ void k_view_meta(DevTable t, unsigned long long n) {
    __shared__ unsigned long long sb[32], st[32];
    unsigned long long bytes = 0, tok = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t r = t.lref[i];
        unsigned long long hi = t.khi[i], lo = t.klo[i];
        unsigned long long len;
        if (r) len = t.llen[r - 1];
        else if (lo) len = 16 - (__ffsll((long long)lo) - 1) / 8;
        else len = 8 - (__ffsll((long long)hi) - 1) / 8;
        bytes += len;
        tok += static_cast<const uint32_t *>(t.cnt)[i];
    }
    for (int d = 16; d; d >>= 1) {
        bytes += __shfl_xor_sync(0xFFFFFFFFu, bytes, d);
        tok += __shfl_xor_sync(0xFFFFFFFFu, tok, d);
    }
    if ((threadIdx.x & 31) == 0) { sb[threadIdx.x >> 5] = bytes; st[threadIdx.x >> 5] = tok; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long B = 0, T = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { B += sb[w]; T += st[w]; }
        if (T) atomicAdd(&t.d_meta[3], T);
        if (B) atomicAdd(&t.d_meta[4], B);
        if (blockIdx.x == 0) {
            t.d_meta[0] = n;
            *t.d_status = 0;
        }
    }
}
static int view_meta_grid(unsigned long long n) {
    const unsigned long long g = (n + 2047) / 2048;
    return (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
}

// A wc_table that reads entries [start, start+n) of the batch output.
static wc_status make_view(wc_batch *b, uint64_t start, uint64_t n, wc_table **out) {
    wc_ctx *ctx = b->ctx;
    wc_table *t = new wc_table();
    t->ctx = ctx;
    t->owner = b;
    t->bytes = 512;
    wc_status s = ctx->alloc(&t->mem, t->bytes, b->stream);
    if (s != WC_OK) { delete t; return s; }
    cudaMemsetAsync(t->mem, 0, t->bytes, b->stream);
    DevTable &d = t->dt;
    d.cap = std::max<uint64_t>(n, 1);
    d.lcap = b->args.lcap;
    d.arena_cap = b->args.arena_cap;
    d.count_bits = 32;
    d.d_meta = static_cast<unsigned long long *>(t->mem);
    d.d_status = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(t->mem) + 256);
    d.khi = b->args.out_khi + start;
    d.klo = b->args.out_klo + start;
    d.cnt = b->args.out_cnt + start;
    d.lref = b->args.out_lref + start;
    d.loff = b->args.loff;
    d.llen = b->args.llen;
    d.arena = b->args.arena;
    k_view_meta<<<view_meta_grid(n), 256, 0, b->stream>>>(d, n);
    t->stream = b->stream;
    cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming);
    table_mark_done(t, b->stream);
    *out = t;
    return WC_OK;
}

static void free_owned_table(wc_table *t) {
    if (!t) return;
    cudaEventSynchronize(t->done);
    t->ctx->release(t->mem, t->bytes, t->stream);
    t->ctx->meta_give(t->meta_slot);
    cudaEventDestroy(t->done);
    delete t;
}

// ---------------------------------------------------------------- batched count
// Host planning: items per size class (largest first) and capacities.
// Capacities from estimates, or (exact) from the bounds no input can exceed:
// a document of s bytes has at most s/2 + 1 distinct words and s/18 + 1
// words of 17 or more letters, whose bytes (each followed by a 0) fit in
// s + its long-word count.
static wc_status batch_plan(wc_ctx *ctx, const uint64_t *h_offsets, uint32_t ndocs, uint32_t nclasses, bool exact,
                            wc_batch **out) {
    if (ndocs >= kMaxDocs) return ctx->fail(WC_ERR_UNSUPPORTED, "2^24 documents or more in one batch");
    for (uint32_t i = 0; i < ndocs; i++)
        if (h_offsets[i + 1] < h_offsets[i]) return ctx->fail(WC_ERR_INVALID_ARG, "offsets decrease");
    if (ndocs && h_offsets[ndocs] >= (1ull << 40)) return ctx->fail(WC_ERR_UNSUPPORTED, "offsets of 2^40 or more");
    wc_batch *b = new wc_batch();
    b->ctx = ctx;
    b->ndocs = ndocs;
    b->nclasses = nclasses;
    std::vector<DocItem> small, medium, large;
    uint64_t out_est = 0, glob_est = 0, long_est = 0, total = 0;
    for (uint32_t d = 0; d < ndocs; d++) {
        const uint64_t lo = h_offsets[d], hi = h_offsets[d + 1], s = hi - lo;
        if (!s) continue;
        const uint64_t e = exact ? s / 2 + 1 : est_distinct(s);
        out_est += exact ? s / 2 + 5 : out_reserve(s);
        long_est += exact ? s / 18 + 1 : std::min<uint64_t>(s / 18 + 1, e / 8 + 2);
        total += s;
        b->max_doc_bytes = std::max(b->max_doc_bytes, s);
        if (s <= kSmallMax) small.push_back({lo, hi, d, 0});
        else if (s <= kMediumMax) medium.push_back({lo, hi, d, 0});
        else if (s <= kSplitMin) large.push_back({lo, hi, d, 0});
        else {
            glob_est += e;
            for (uint64_t r = lo; r < hi; r += kRange) large.push_back({r, std::min(hi, r + kRange), d, 1});
        }
    }
    auto by_size = [](const DocItem &x, const DocItem &y) { return x.hi - x.lo > y.hi - y.lo; };
    std::stable_sort(small.begin(), small.end(), by_size);
    std::stable_sort(medium.begin(), medium.end(), by_size);
    std::stable_sort(large.begin(), large.end(), by_size);
    b->nsmall = (uint32_t)small.size();
    b->nmedium = (uint32_t)medium.size();
    b->items = small;
    b->items.insert(b->items.end(), medium.begin(), medium.end());
    b->items.insert(b->items.end(), large.begin(), large.end());
    b->total_bytes = total;
    b->args.out_cap = out_est + 1024;
    b->args.lcap = long_est + 1024;
    b->args.arena_cap = exact ? total + b->args.lcap + 65536 : b->args.lcap * 24 + 65536;
    // planned: split documents; reserve: documents whose shared table fills
    // up (exact: every (document, word) pair may spill)
    b->exact = exact;
    b->cap8 = pow2_ge(exact ? 2 * out_est + (1u << 18) : 2 * glob_est + out_est / 32 + (1u << 18));
    b->cap16 = pow2_ge(exact ? out_est + out_est / 4 + (1u << 17) : glob_est + out_est / 64 + (1u << 17));
    b->caplong = pow2_ge(exact ? 2 * long_est + (1u << 14) : glob_est / 8 + (1u << 14));
    b->shape_small = ctx->tuned_small;
    b->shape_medium = ctx->tuned_medium;
    b->shape_large = ctx->tuned_large;
    *out = b;
    return WC_OK;
}

// Output block (owned by the batch) and, if keep_scratch, the scratch too.
static wc_status batch_alloc(wc_batch *b, cudaStream_t stream) {
    wc_ctx *ctx = b->ctx;
    auto r = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t nd = std::max<uint32_t>(b->ndocs, 1);
    const uint64_t out_cap = b->args.out_cap, lcap = b->args.lcap, arena_cap = b->args.arena_cap;
    b->bytes = r(64) + r(16) + r(out_cap * 8) * 2 + r(out_cap * 4) * 2 + r(nd * 8) + r(nd * 4) * 2 + r(lcap * 8) * 2 +
               r(arena_cap) + r(nd * 4);
    wc_status st = ctx->alloc(&b->mem, b->bytes, stream);
    if (st != WC_OK) return st;
    uint8_t *p = static_cast<uint8_t *>(b->mem);
    auto take = [&](size_t n) { uint8_t *q = p; p += r(n); return q; };
    BatchArgs &a = b->args;
    a.meta = reinterpret_cast<unsigned long long *>(take(64));
    a.status = reinterpret_cast<uint32_t *>(take(16));
    a.out_khi = reinterpret_cast<unsigned long long *>(take(out_cap * 8));
    a.out_klo = reinterpret_cast<unsigned long long *>(take(out_cap * 8));
    a.out_cnt = reinterpret_cast<uint32_t *>(take(out_cap * 4));
    a.out_lref = reinterpret_cast<uint32_t *>(take(out_cap * 4));
    a.doc_start = reinterpret_cast<unsigned long long *>(take(nd * 8));
    a.doc_n = reinterpret_cast<uint32_t *>(take(nd * 4));
    a.doc_flags = reinterpret_cast<uint32_t *>(take(nd * 4));
    a.loff = reinterpret_cast<unsigned long long *>(take(lcap * 8));
    a.llen = reinterpret_cast<unsigned long long *>(take(lcap * 8));
    a.arena = take(arena_cap);
    b->d_class = reinterpret_cast<uint32_t *>(take(nd * 4));
    a.ndocs = b->ndocs;
    // scratch: items + queue cursors, (document, word) tables, sort scratch
    CapPlan plan{b->cap8, b->cap16, b->caplong, 0};
    st = scratch_create(ctx, plan, false, stream, b->scr.cs);
    b->scr.ibytes = sizeof(DocItem) * std::max<size_t>(b->items.size(), 1) + 256 + 16 * 8;
    void *ib = nullptr;
    if (st == WC_OK) st = ctx->alloc(&ib, b->scr.ibytes, stream);
    if (st != WC_OK) return st;
    b->scr.items = static_cast<DocItem *>(ib);
    b->scr.next = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(ib) + sizeof(DocItem) * std::max<size_t>(b->items.size(), 1));
    b->scr.smeta = reinterpret_cast<unsigned long long *>(b->scr.next + 64);
    cudaError_t e = cudaSuccess;
    if (!b->items.empty())
        e = cudaMemcpyAsync(b->scr.items, b->items.data(), sizeof(DocItem) * b->items.size(), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "batch items");
    return WC_OK;
}

static void batch_release_scratch(wc_batch *b, cudaStream_t stream) {
    wc_ctx *ctx = b->ctx;
    if (b->scr.items) ctx->release(b->scr.items, b->scr.ibytes, stream);
    if (b->scr.cs.mem) ctx->release(b->scr.cs.mem, b->scr.cs.bytes, stream);
    b->scr.items = nullptr;
    b->scr.cs.mem = nullptr;
}

// All device work of one batched count, in stream order (capturable: no
// allocations, no host copies).
static cudaError_t batch_enqueue(wc_batch *b, const uint8_t *d_text, const uint64_t *d_offsets,
                                 const uint32_t *d_class, cudaStream_t stream, int shape_small, int shape_medium,
                                 int shape_large,
                                 uint64_t *launches) {
    BatchArgs &a = b->args;
    const size_t nd = std::max<uint32_t>(b->ndocs, 1);
    a.text = d_text;
    a.doc_off = reinterpret_cast<const unsigned long long *>(d_offsets);
    cudaMemsetAsync(a.meta, 0, 64 + 256, stream);
    cudaMemsetAsync(a.doc_start, 0, nd * 8, stream);
    cudaMemsetAsync(a.doc_n, 0, nd * 4, stream);
    cudaMemsetAsync(a.doc_flags, 0, nd * 4, stream);
    if (b->nclasses && d_class) cudaMemcpyAsync(b->d_class, d_class, 4ull * b->ndocs, cudaMemcpyDeviceToDevice, stream);
    cudaMemsetAsync(b->scr.next, 0, 256, stream);
    CountScratch &cs = b->scr.cs;
    const size_t hb = ((cs.gcap8 * sizeof(G8Slot) + 255) & ~(size_t)255) + ((cs.gcap * sizeof(GSlot) + 255) & ~(size_t)255) +
                      ((cs.glcap * sizeof(LSlot) + 255) & ~(size_t)255);
    cudaMemsetAsync(cs.mem, 0, hb, stream);
    a.g = cs.gtable(a.status);
    cudaError_t e = cudaSuccess;
    uint64_t n = 0;
    if (b->nsmall) {
        BatchArgs s1 = a;
        s1.items = b->scr.items;
        s1.nitems = b->nsmall;
        s1.next_item = b->scr.next;
        e = launch_docs(s1, shape_small, stream);
        n++;
    }
    if (e == cudaSuccess && b->nmedium) {
        BatchArgs s2 = a;
        s2.items = b->scr.items + b->nsmall;
        s2.nitems = b->nmedium;
        s2.next_item = b->scr.next + 1;
        e = launch_docs(s2, shape_medium, stream, n > 0);
        n++;
    }
    const size_t nbig = b->items.size() - b->nsmall - b->nmedium;
    if (e == cudaSuccess && nbig) {
        BatchArgs s3 = a;
        s3.items = b->scr.items + b->nsmall + b->nmedium;
        s3.nitems = (uint32_t)nbig;
        s3.next_item = b->scr.next + 2;
        e = launch_docs(s3, shape_large, stream, n > 0);
        n++;
    }
    if (e == cudaSuccess) {
        const uint32_t skip = sort_skip_mask(b->max_doc_bytes / 2 + 1, b->ndocs);
        e = launch_segmented_finish(a, a.g, cs.gcap8, cs.gcap, cs.glcap, cs.ss, b->scr.smeta, stream, skip);
        n += segmented_finish_launches(cs.ss.cap, skip);
    }
    if (launches) *launches = n;
    return e;
}

wc_status wc_count_batched(wc_ctx *ctx, const uint8_t *d_text, const uint64_t *d_offsets, const uint64_t *h_offsets,
                           uint32_t ndocs, const uint32_t *d_class, uint32_t nclasses, cudaStream_t stream,
                           wc_batch **out) {
    return wc_count_batched_ex(ctx, d_text, d_offsets, h_offsets, ndocs, d_class, nclasses, 0u, stream, out);
}

wc_status wc_count_batched_ex(wc_ctx *ctx, const uint8_t *d_text, const uint64_t *d_offsets, const uint64_t *h_offsets,
                              uint32_t ndocs, const uint32_t *d_class, uint32_t nclasses, uint32_t flags,
                              cudaStream_t stream, wc_batch **out) {
    if (!ctx || !out) return WC_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)WC_BATCH_EXACT_BOUNDS) return ctx->fail(WC_ERR_INVALID_ARG, "unknown batch flags");
    *out = nullptr;
    if (ndocs && (!h_offsets || !d_offsets)) return ctx->fail(WC_ERR_INVALID_ARG, "null offsets");
    if (nclasses && !d_class) return ctx->fail(WC_ERR_INVALID_ARG, "classes without a class array");
    if (ndocs && h_offsets[ndocs] > h_offsets[0] && !d_text) return ctx->fail(WC_ERR_INVALID_ARG, "null text");
    cudaSetDevice(ctx->device);
    wc_batch *b = nullptr;
    wc_status st = batch_plan(ctx, h_offsets, ndocs, nclasses, (flags & WC_BATCH_EXACT_BOUNDS) != 0, &b);
    if (st != WC_OK) return st;
    b->stream = stream;
    if ((st = batch_alloc(b, stream)) != WC_OK) {
        batch_release_scratch(b, stream);
        if (b->mem) ctx->release(b->mem, b->bytes, stream);
        delete b;
        return st;
    }
    uint64_t n = 0;
    cudaError_t e = batch_enqueue(b, d_text, d_offsets, d_class, stream, b->shape_small, b->shape_medium,
                                  b->shape_large, &n);
    ctx->launches += n;
    batch_release_scratch(b, stream);
    cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    cudaEventRecord(b->done, stream);
    if (e != cudaSuccess) {
        wc_batch_free(b);
        return ctx->cuda_fail(e, "batched count launch");
    }
    *out = b;
    return WC_OK;
}

// ---------------------------------------------------------------- plans: resident state + CUDA graph
struct wc_plan {
    wc_batch *b = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint8_t *g_text = nullptr;
    const uint64_t *g_off = nullptr;
    const uint32_t *g_cls = nullptr;
    cudaStream_t own = nullptr;   // graphs are captured and replayed here
    cudaEvent_t in_ev = nullptr;
    uint64_t graph_launches = 0;
    bool tuned = false;
};

// Times the per-document kernel shapes on the plan's own input (three runs
// each, median) and keeps the fastest per size class.
static wc_status plan_autotune(wc_plan *pl, const uint8_t *d_text, const uint64_t *d_offsets, const uint32_t *d_class,
                               cudaStream_t stream) {
    wc_batch *b = pl->b;
    wc_ctx *ctx = b->ctx;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_shapes = [&](int ss, int sm, int sl) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, stream);
            batch_enqueue(b, d_text, d_offsets, d_class, stream, ss, sm, sl, nullptr);
            cudaEventRecord(e1, stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    int bs = b->shape_small, bm = b->shape_medium, bl = b->shape_large;
    if (b->nsmall) {
        float t = 1e30f;
        for (int s : {0, 1, 2, 6, 7}) {
            float ms = time_shapes(s, bm, bl);
            if (ms < t) { t = ms; bs = s; }
        }
    }
    if (b->nmedium) {
        float t = 1e30f;
        for (int m = 2; m <= 4; m++) {
            float ms = time_shapes(bs, m, bl);
            if (ms < t) { t = ms; bm = m; }
        }
    }
    if (b->items.size() > b->nsmall + b->nmedium) {
        float t = 1e30f;
        for (int l = 3; l <= 5; l++) {
            float ms = time_shapes(bs, bm, l);
            if (ms < t) { t = ms; bl = l; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->shape_small = ctx->tuned_small = bs;
    b->shape_medium = ctx->tuned_medium = bm;
    b->shape_large = ctx->tuned_large = bl;
    ctx->tuned = true;
    ctx->tune_save();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WC_OK : ctx->cuda_fail(e, "autotune");
}

wc_status wc_plan_create(wc_ctx *ctx, const uint64_t *h_offsets, uint32_t ndocs, uint32_t nclasses, cudaStream_t stream,
                         wc_plan **out) {
    if (!ctx || !out || (ndocs && !h_offsets)) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    wc_plan *pl = new wc_plan();
    wc_status st = batch_plan(ctx, h_offsets, ndocs, nclasses, false, &pl->b);
    if (st == WC_OK) {
        pl->b->stream = stream;
        st = batch_alloc(pl->b, stream);
    }
    if (st != WC_OK) {
        wc_plan_free(pl);
        return st;
    }
    cudaEventCreateWithFlags(&pl->b->done, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&pl->in_ev, cudaEventDisableTiming);
    if (cudaStreamCreateWithFlags(&pl->own, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        wc_plan_free(pl);
        return ctx->fail(WC_ERR_CUDA, "cudaStreamCreate");
    }
    // items and scratch were staged on the caller's stream
    cudaEventRecord(pl->in_ev, stream);
    cudaStreamWaitEvent(pl->own, pl->in_ev, 0);
    *out = pl;
    return WC_OK;
}

wc_status wc_plan_run(wc_plan *pl, const uint8_t *d_text, const uint64_t *d_offsets, const uint32_t *d_class,
                      cudaStream_t stream, const wc_batch **out) {
    if (!pl || !out) return WC_ERR_INVALID_ARG;
    wc_batch *b = pl->b;
    wc_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    if (ctx->autotune && !ctx->tuned && !pl->tuned) {
        wc_status st = plan_autotune(pl, d_text, d_offsets, d_class, stream);
        if (st != WC_OK) return st;
    }
    pl->tuned = true;
    // the graph lives on the plan's own stream, ordered after the caller's
    cudaEventRecord(pl->in_ev, stream);
    cudaStreamWaitEvent(pl->own, pl->in_ev, 0);
    if (!pl->exec || pl->g_text != d_text || pl->g_off != d_offsets || pl->g_cls != d_class) {
        if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(pl->own, cudaStreamCaptureModeThreadLocal);
        uint64_t n = 0;
        if (e == cudaSuccess) {
            cudaError_t e2 = batch_enqueue(b, d_text, d_offsets, d_class, pl->own, b->shape_small, b->shape_medium,
                                           b->shape_large, &n);
            e = cudaStreamEndCapture(pl->own, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return ctx->cuda_fail(e, "capturing the batched count");
        pl->g_text = d_text;
        pl->g_off = d_offsets;
        pl->g_cls = d_class;
        pl->graph_launches = n;
    }
    // the plan's batch is rewritten: drop tables built from the previous run
    for (auto *v : b->views) free_owned_table(v);
    b->views.clear();
    for (auto *t : b->class_tables) free_owned_table(t);
    b->class_tables.clear();
    free_owned_table(b->global);
    b->global = nullptr;
    if (b->gscratch.mem) { ctx->release(b->gscratch.mem, b->gscratch.bytes, stream); b->gscratch.mem = nullptr; }
    drop_vocab(b, stream);
    b->tables_built = false;
    b->synced = false;
    b->word_bytes = 0;
    b->stream = stream;
    cudaError_t e = cudaGraphLaunch(pl->exec, pl->own);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGraphLaunch");
    ctx->launches += pl->graph_launches;
    cudaEventRecord(b->done, pl->own);
    cudaStreamWaitEvent(stream, b->done, 0);
    *out = b;
    return WC_OK;
}

void wc_plan_free(wc_plan *pl) {
    if (!pl) return;
    if (pl->own) cudaStreamSynchronize(pl->own);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->in_ev) cudaEventDestroy(pl->in_ev);
    if (pl->own) cudaStreamDestroy(pl->own);
    if (pl->b) {
        batch_release_scratch(pl->b, pl->b->stream);
        wc_batch_free(pl->b);
    }
    delete pl;
}

wc_status wc_batch_status(const wc_batch *b) {
    if (!b) return WC_ERR_INVALID_ARG;
    return batch_sync(b);
}

// ---------------------------------------------------------------- class / global tables
// One block per document: its entries are added to its class table and to
// the global table (Sec. 3.3: the counts of a key summed across documents).
__global__ void k_batch_tables(BatchArgs a, const uint32_t *cls, const GTable *gt, uint32_t nclasses, GTable gg) {
    const uint32_t d = blockIdx.x;
    const unsigned long long s = a.doc_start[d];
    const uint32_t n = a.doc_n[d];
    const uint32_t c = nclasses ? cls[d] : 0u;
    const GTable *gc = nclasses && c < nclasses ? &gt[c] : nullptr;
    if (nclasses && c >= nclasses) {  // reported through the global table's status
        if (threadIdx.x == 0) atomicOr(gg.status, ST_BAD_CLASS);
        return;
    }
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long j = s + i;
        const unsigned long long c = a.out_cnt[j];
        const uint32_t r = a.out_lref[j];
        if (r == 0) {
            const unsigned long long hi8 = a.out_khi[j], lo8 = a.out_klo[j];
            uint4 k;
            k.x = __byte_perm((uint32_t)(hi8 >> 32), 0, 0x0123);
            k.y = __byte_perm((uint32_t)hi8, 0, 0x0123);
            k.z = __byte_perm((uint32_t)(lo8 >> 32), 0, 0x0123);
            k.w = __byte_perm((uint32_t)lo8, 0, 0x0123);
            table_insert_key(gg, k, c);
            if (gc) table_insert_key(*gc, k, c);
        } else {
            const uint8_t *w = a.arena + a.loff[r - 1];
            long_insert(gg, w, a.llen[r - 1], c, nullptr, nullptr);
            if (gc) long_insert(*gc, w, a.llen[r - 1], c, nullptr, nullptr);
        }
    }
}

// Class and global tables: every document's rows are added (k_batch_tables)
// into one hash table per class and one for all documents, each then
// compacted and sorted.  A table's distinct words lie between the largest
// of its documents' table sizes and their sum (the exact bound); tables are
// first sized for max(2 x the largest, a quarter of the sum) and, if one
// overflows, all are built again at the bound.
static wc_status build_tables_at(wc_batch *b, const std::vector<uint64_t> &est, std::vector<wc_table *> &tabs,
                                 bool *overflow) {
    wc_ctx *ctx = b->ctx;
    cudaStream_t s = b->stream;
    const uint32_t nt = b->nclasses + 1;  // class tables, then the global table
    wc_status st = WC_OK;
    std::vector<CountScratch> scr(nt);
    tabs.assign(nt, nullptr);
    auto cleanup = [&](uint32_t upto) {
        for (uint32_t c = 0; c < upto; c++)
            if (c < b->nclasses && scr[c].mem) ctx->release(scr[c].mem, scr[c].bytes, s);
    };
    for (uint32_t c = 0; c < nt && st == WC_OK; c++) {
        const uint64_t d = std::max<uint64_t>(est[c], 256);
        CapPlan plan;
        plan.cap8 = pow2_ge(std::max<uint64_t>(1024, 2 * d));
        plan.cap16 = pow2_ge(std::max<uint64_t>(1024, d + d / 4));
        plan.caplong = pow2_ge(std::max<uint64_t>(256, 2 * std::min<uint64_t>(d, b->args.lcap)));
        plan.arena = std::max<uint64_t>(4096, b->args.arena_cap);
        CountScratch &cs = c < b->nclasses ? scr[c] : b->gscratch;
        if ((st = scratch_create(ctx, plan, false, s, cs)) != WC_OK) break;
        if ((st = table_create(ctx, cs.entries(), plan.caplong, plan.arena, c < b->nclasses ? 32 : ctx->count_bits,
                               s, &tabs[c])) != WC_OK)
            break;
        tabs[c]->owner = b;
    }
    if (st != WC_OK) {
        cleanup(nt);
        for (auto *t : tabs) free_owned_table(t);
        tabs.clear();
        return st;
    }
    std::vector<GTable> g(std::max<uint32_t>(b->nclasses, 1));
    for (uint32_t c = 0; c < b->nclasses; c++) g[c] = scr[c].gtable(tabs[c]->dt.d_status);
    // device copies: the class hash tables, then the sort jobs of all tables
    const size_t gbytes = (sizeof(GTable) * g.size() + 255) & ~(size_t)255;
    const size_t dbytes = gbytes + finish_tables_job_bytes((int)nt);
    void *dg = nullptr;
    if ((st = ctx->alloc(&dg, dbytes, s)) != WC_OK) {
        cleanup(nt);
        for (auto *t : tabs) free_owned_table(t);
        tabs.clear();
        return st;
    }
    cudaMemcpyAsync(dg, g.data(), sizeof(GTable) * g.size(), cudaMemcpyHostToDevice, s);
    const GTable gg = b->gscratch.gtable(tabs[b->nclasses]->dt.d_status);
    if (b->ndocs) k_batch_tables<<<b->ndocs, 128, 0, s>>>(b->args, b->d_class, static_cast<GTable *>(dg), b->nclasses, gg);
    cudaError_t e = cudaGetLastError();
    std::vector<FinishSpec> spec(nt);
    for (uint32_t c = 0; c < nt; c++) {
        CountScratch &cs = c < b->nclasses ? scr[c] : b->gscratch;
        spec[c] = FinishSpec{c < b->nclasses ? g[c] : gg, cs.gcap8, cs.gcap, cs.glcap, &cs.ss, &tabs[c]->dt};
    }
    const uint32_t skip = sort_skip_mask(b->total_bytes / 2 + 1, 0);
    if (e == cudaSuccess) e = finish_tables(spec.data(), (int)nt, static_cast<uint8_t *>(dg) + gbytes, s, skip);
    uint64_t capmax = 0;
    for (uint32_t c = 0; c < nt; c++) capmax = std::max<uint64_t>(capmax, spec[c].ss->cap);
    ctx->launches += 1 + (uint64_t)finish_tables_launches((int)nt, capmax, skip);
    cleanup(nt);
    ctx->release(dg, dbytes, s);
    for (auto *t : tabs) table_mark_done(t, s);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "class/global tables");
    *overflow = false;
    for (auto *t : tabs)
        if (table_sync(t) == WC_ERR_CAPACITY) *overflow = true;
    return WC_OK;
}

static wc_status build_tables(wc_batch *b) {
    if (b->tables_built) return WC_OK;
    wc_status st = batch_sync(b);
    if (st != WC_OK) return st;
    wc_ctx *ctx = b->ctx;
    const uint32_t nd = b->ndocs, nt = b->nclasses + 1;
    // the documents' table sizes (and classes), for the capacities
    std::vector<uint32_t> dn(nd), dc(nd, 0u);
    cudaError_t e = cudaSuccess;
    if (nd) e = cudaMemcpy(dn.data(), b->args.doc_n, 4ull * nd, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nd && b->nclasses) e = cudaMemcpy(dc.data(), b->d_class, 4ull * nd, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "class/global table sizes");
    std::vector<uint64_t> sum(nt, 0), mx(nt, 0), est(nt);
    for (uint32_t d = 0; d < nd; d++) {
        const uint32_t c = b->nclasses ? dc[d] : 0u;
        if (b->nclasses && c >= b->nclasses) return ctx->fail(WC_ERR_INVALID_ARG, "a class id is not below nclasses");
        if (b->nclasses) {
            sum[c] += dn[d];
            mx[c] = std::max<uint64_t>(mx[c], dn[d]);
        }
        sum[b->nclasses] += dn[d];
        mx[b->nclasses] = std::max<uint64_t>(mx[b->nclasses], dn[d]);
    }
    for (uint32_t t = 0; t < nt; t++) est[t] = std::min(sum[t], std::max(2 * mx[t], sum[t] / 4));
    std::vector<wc_table *> tabs;
    bool overflow = false;
    if ((st = build_tables_at(b, est, tabs, &overflow)) != WC_OK) return st;
    if (overflow) {  // again at the exact bound: the sum of the documents' sizes
        for (auto *t : tabs) free_owned_table(t);
        if (b->gscratch.mem) { ctx->release(b->gscratch.mem, b->gscratch.bytes, b->stream); b->gscratch.mem = nullptr; }
        if ((st = build_tables_at(b, sum, tabs, &overflow)) != WC_OK) return st;
        if (overflow) return ctx->fail(WC_ERR_INTERNAL, "class/global tables overflowed at their exact bound");
    }
    b->class_tables.assign(tabs.begin(), tabs.begin() + b->nclasses);
    b->global = tabs[b->nclasses];
    b->tables_built = true;
    return WC_OK;
}

// Rows [first[d], first[d] + min(k, n_d)) of the output are document d's
// first rows (its top k): one warp per document.
__global__ void k_batch_topk(BatchArgs a, const unsigned long long *first, uint32_t k, DevTable out) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long d = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < a.ndocs;
         d += nw) {
        const unsigned long long src = a.doc_start[d], dst = first[d];
        const uint32_t n = a.doc_n[d], m = n < k ? n : k;
        for (uint32_t j = lane; j < m; j += 32) {
            out.khi[dst + j] = a.out_khi[src + j];
            out.klo[dst + j] = a.out_klo[src + j];
            static_cast<uint32_t *>(out.cnt)[dst + j] = a.out_cnt[src + j];
            out.lref[dst + j] = a.out_lref[src + j];
        }
    }
}

wc_status wc_batch_topk(const wc_batch *cb, uint32_t k, uint64_t *h_first, uint32_t *h_n, const wc_table **out) {
    if (!cb || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    wc_batch *b = const_cast<wc_batch *>(cb);
    wc_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    wc_status st = batch_sync(b);
    if (st != WC_OK) return st;
    const uint32_t nd = b->ndocs;
    std::vector<uint32_t> n(nd);
    std::vector<unsigned long long> first(nd + 1, 0);
    cudaError_t e = cudaSuccess;
    if (nd) e = cudaMemcpy(n.data(), b->args.doc_n, 4ull * nd, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "batch top-k");
    for (uint32_t d = 0; d < nd; d++) first[d + 1] = first[d] + std::min(k, n[d]);
    const uint64_t rows = first[nd];
    for (uint32_t d = 0; d < nd; d++) {
        if (h_first) h_first[d] = first[d];
        if (h_n) h_n[d] = std::min(k, n[d]);
    }
    // one block: metadata, the rows' keys, counts and long references, the offsets
    auto r = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const uint64_t cap = std::max<uint64_t>(rows, 1);
    wc_table *t = new wc_table();
    t->ctx = ctx;
    t->owner = b;
    t->bytes = r(512) + r(cap * 8) * 2 + r(cap * 4) * 2 + r(8ull * (nd + 1));
    st = ctx->alloc(&t->mem, t->bytes, b->stream);
    if (st != WC_OK) { delete t; return st; }
    uint8_t *p = static_cast<uint8_t *>(t->mem);
    e = cudaMemsetAsync(p, 0, 512, b->stream);
    DevTable &d = t->dt;
    d.cap = cap;
    d.lcap = b->args.lcap;
    d.arena_cap = b->args.arena_cap;
    d.count_bits = 32;
    d.d_meta = reinterpret_cast<unsigned long long *>(p);
    d.d_status = reinterpret_cast<uint32_t *>(p + 256);
    p += r(512);
    d.khi = reinterpret_cast<unsigned long long *>(p);
    p += r(cap * 8);
    d.klo = reinterpret_cast<unsigned long long *>(p);
    p += r(cap * 8);
    d.cnt = p;
    p += r(cap * 4);
    d.lref = reinterpret_cast<uint32_t *>(p);
    p += r(cap * 4);
    unsigned long long *d_first = reinterpret_cast<unsigned long long *>(p);
    d.loff = b->args.loff;  // long words stay in the batch's arena
    d.llen = b->args.llen;
    d.arena = b->args.arena;
    // pageable source: the call returns once the bytes are staged
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_first, first.data(), 8ull * (nd + 1), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nd && rows) {
        const unsigned long long g = std::min<unsigned long long>((nd + 7) / 8, 4096);
        k_batch_topk<<<(int)g, 256, 0, b->stream>>>(b->args, d_first, k, d);
        ctx->launches++;
    }
    if (e == cudaSuccess) {
        k_view_meta<<<view_meta_grid(rows), 256, 0, b->stream>>>(d, rows);
        ctx->launches++;
        e = cudaGetLastError();
    }
    cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming);
    table_mark_done(t, b->stream);
    b->views.push_back(t);  // freed with the batch
    if (e != cudaSuccess) return ctx->cuda_fail(e, "batch top-k");
    *out = t;
    return WC_OK;
}

wc_status wc_batch_table(const wc_batch *cb, int kind, uint32_t idx, const wc_table **out) {
    if (!cb || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    wc_batch *b = const_cast<wc_batch *>(cb);
    cudaSetDevice(b->ctx->device);
    wc_status st = batch_sync(b);
    if (st != WC_OK) return st;
    if (kind == WC_TABLE_DOC) {
        if (idx >= b->ndocs) return WC_ERR_INVALID_ARG;
        if (b->views.empty()) b->views.assign(b->ndocs, nullptr);
        if (!b->views[idx]) {
            unsigned long long start = 0;
            uint32_t n = 0;
            cudaMemcpy(&start, b->args.doc_start + idx, 8, cudaMemcpyDeviceToHost);
            cudaMemcpy(&n, b->args.doc_n + idx, 4, cudaMemcpyDeviceToHost);
            if ((st = make_view(b, start, n, &b->views[idx])) != WC_OK) return st;
        }
        *out = b->views[idx];
        return WC_OK;
    }
    if ((st = build_tables(b)) != WC_OK) return st;
    if (kind == WC_TABLE_CLASS) {
        if (idx >= b->nclasses) return WC_ERR_INVALID_ARG;
        *out = b->class_tables[idx];
        return WC_OK;
    }
    if (kind == WC_TABLE_GLOBAL) {
        *out = b->global;
        return WC_OK;
    }
    return WC_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------- class ratio ranking
// cout of each class entry = global count - cin (global counts looked up in
// the global hash tables, read only).
__device__ unsigned long long lookup_count(const GTable &g, uint4 k, const uint8_t *lw, unsigned long long llen) {
    if (lw) {
        const unsigned long long h = long_hash(lw, llen);
        unsigned long long s = h & g.lmask;
        for (int probe = 0; probe < kGlobalProbeLimit; probe++) {
            const LSlot &sl = g.lslots[s];
            if (sl.h == 0 && sl.addr == 0) return 0;
            if (sl.h == h) {
                const uint8_t *rep = reinterpret_cast<const uint8_t *>(sl.addr);
                bool eq = true;
                for (unsigned long long i = 0; i < llen && eq; i++) eq = (rep[i] | 0x20u) == (lw[i] | 0x20u);
                if (eq && !is_letter(rep[llen])) return sl.cnt;
            }
            s = (s + 1) & g.lmask;
        }
        return 0;
    }
    if ((k.z | k.w) == 0u) {
        const unsigned long long key = ((unsigned long long)k.y << 32) | k.x;
        unsigned long long s = hash8(key) >> __clzll((long long)g.mask8);
        for (int probe = 0; probe < kGlobalProbeLimit; probe++) {
            if (g.slots8[s].key == key) return g.slots8[s].cnt;
            if (g.slots8[s].key == 0) return 0;
            s = (s + 1) & g.mask8;
        }
        return 0;
    }
    unsigned long long s = home16(k, g.mask);
    for (int probe = 0; probe < kGlobalProbeLimit; probe++) {
        const uint4 c = g.slots[s].key;
        if (key_eq(c, k)) return g.slots[s].cnt;
        if (key_zero(c)) return 0;
        s = (s + 1) & g.mask;
    }
    return 0;
}

struct RatioArgs {
    DevTable cls;
    GTable g;
    unsigned long long *cin, *cout;
    uint32_t k;
    unsigned long long *out_idx;
    unsigned long long *out_n;
};

__global__ void k_ratio_prepare(RatioArgs r) {
    const unsigned long long n = r.cls.d_meta[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long c = static_cast<const uint32_t *>(r.cls.cnt)[i];
        const uint32_t lr = r.cls.lref[i];
        const unsigned long long hi8 = r.cls.khi[i], lo8 = r.cls.klo[i];
        uint4 k;
        k.x = __byte_perm((uint32_t)(hi8 >> 32), 0, 0x0123);
        k.y = __byte_perm((uint32_t)hi8, 0, 0x0123);
        k.z = __byte_perm((uint32_t)(lo8 >> 32), 0, 0x0123);
        k.w = __byte_perm((uint32_t)lo8, 0, 0x0123);
        const uint8_t *lw = lr ? r.cls.arena + r.cls.loff[lr - 1] : nullptr;
        const unsigned long long g = lookup_count(r.g, k, lw, lr ? r.cls.llen[lr - 1] : 0);
        r.cin[i] = c;
        r.cout[i] = g >= c ? g - c : 0;  // g < c cannot happen for consistent tables
    }
}

// true when entry a ranks above entry b: cin/cout descending (cout = 0 is
// infinite), then cin descending, then word ascending (the table's own
// order: equal-count entries appear in word order, so a lower index wins).
__device__ __forceinline__ bool ratio_better(unsigned long long ia, unsigned long long ca, unsigned long long oa,
                                             unsigned long long ib, unsigned long long cb, unsigned long long ob) {
    const bool infa = oa == 0, infb = ob == 0;
    if (infa != infb) return infa;
    if (!infa) {
        // ca/oa vs cb/ob by 128-bit cross products
        const unsigned long long l_lo = ca * ob, l_hi = __umul64hi(ca, ob);
        const unsigned long long r_lo = cb * oa, r_hi = __umul64hi(cb, oa);
        if (l_hi != r_hi) return l_hi > r_hi;
        if (l_lo != r_lo) return l_lo > r_lo;
    }
    if (ca != cb) return ca > cb;
    return ia < ib;
}

// The top k of a list of entries (src[0, n) holds entry indices, or is the
// identity when src is null) by k rounds of a block-wide arg-best; the winners
// go to dst[0, min(k, n)) and *dst_n.  taken[] (n flags, zeroed) marks them.
__device__ void ratio_topk_block(const RatioArgs &r, const unsigned long long *src, unsigned long long n,
                                 unsigned char *taken, unsigned long long *dst, unsigned long long *dst_n) {
    __shared__ unsigned long long bi[32], bc[32], bo[32];
    const uint32_t k = (uint32_t)(n < r.k ? n : r.k);
    for (uint32_t round = 0; round < k; round++) {
        unsigned long long mi = ~0ull, mc = 0, mo = 0, mj = 0;
        for (unsigned long long j = threadIdx.x; j < n; j += blockDim.x) {
            if (taken[j]) continue;
            const unsigned long long i = src ? src[j] : j;
            if (mi == ~0ull || ratio_better(i, r.cin[i], r.cout[i], mi, mc, mo)) {
                mi = i; mc = r.cin[i]; mo = r.cout[i]; mj = j;
            }
        }
        for (int d = 16; d; d >>= 1) {
            const unsigned long long oi = __shfl_xor_sync(0xFFFFFFFFu, mi, d), oc = __shfl_xor_sync(0xFFFFFFFFu, mc, d),
                                     oo = __shfl_xor_sync(0xFFFFFFFFu, mo, d), oj = __shfl_xor_sync(0xFFFFFFFFu, mj, d);
            if (oi != ~0ull && (mi == ~0ull || ratio_better(oi, oc, oo, mi, mc, mo))) { mi = oi; mc = oc; mo = oo; mj = oj; }
        }
        __shared__ unsigned long long bj[32];
        if ((threadIdx.x & 31) == 0) {
            bi[threadIdx.x >> 5] = mi; bc[threadIdx.x >> 5] = mc; bo[threadIdx.x >> 5] = mo; bj[threadIdx.x >> 5] = mj;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long xi = ~0ull, xc = 0, xo = 0, xj = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++)
                if (bi[w] != ~0ull && (xi == ~0ull || ratio_better(bi[w], bc[w], bo[w], xi, xc, xo))) {
                    xi = bi[w]; xc = bc[w]; xo = bo[w]; xj = bj[w];
                }
            dst[round] = xi;
            taken[xj] = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *dst_n = k;
}

// Large k (above kRatioKeepMax): stage 1, block b keeps the top k of its
// slice of the class entries by k rounds of arg-best (the overall top k is
// among the blocks' winners); stage 2 (one block), the top k of the winners.
constexpr unsigned long long kRatioSlice = 1024;
__global__ void __launch_bounds__(256) k_ratio_select_slices(RatioArgs r, unsigned char *taken, unsigned long long *cand,
                                                            unsigned long long *cand_n) {
    const unsigned long long n = r.cls.d_meta[0];
    const unsigned long long lo = (unsigned long long)blockIdx.x * kRatioSlice;
    if (lo >= n) {
        if (threadIdx.x == 0) cand_n[blockIdx.x] = 0;
        return;
    }
    const unsigned long long m = n - lo < kRatioSlice ? n - lo : kRatioSlice;
    __shared__ unsigned long long ids[kRatioSlice];
    for (unsigned long long j = threadIdx.x; j < m; j += blockDim.x) ids[j] = lo + j;
    __syncthreads();
    ratio_topk_block(r, ids, m, taken + lo, cand + (unsigned long long)blockIdx.x * r.k, cand_n + blockIdx.x);
}
__global__ void __launch_bounds__(1024) k_ratio_select(RatioArgs r, unsigned char *taken, const unsigned long long *cand,
                                                       const unsigned long long *cand_n, unsigned int nblocks) {
    // gather the winners densely at the front of cand's slots (in order)
    __shared__ unsigned long long off[1];
    unsigned long long *list = const_cast<unsigned long long *>(cand);
    if (threadIdx.x == 0) {
        unsigned long long o = 0;
        for (unsigned int b = 0; b < nblocks; b++) {
            for (unsigned long long j = 0; j < cand_n[b]; j++) list[o + j] = cand[(unsigned long long)b * r.k + j];
            o += cand_n[b];
        }
        off[0] = o;
    }
    __syncthreads();
    ratio_topk_block(r, list, off[0], taken, r.out_idx, r.out_n);
}

// k up to kRatioKeepMax: block b sorts the 1024 list entries
// src[b * 1024, (b + 1) * 1024) by rank (a bitonic network in shared memory;
// entries past len and the pad index kNoEntry rank last) and keeps its first
// `keep` in dst[b * keep, (b + 1) * keep).  The list's top k is among the
// kept entries, and each round shrinks the list by 1024 / keep >= 2 until one
// block holds it.  src null: the identity list of the class entries.
constexpr int kRatioSort = 1024;
constexpr uint32_t kRatioKeepMax = kRatioSort / 2;
constexpr unsigned long long kNoEntry = ~0ull;
__device__ __forceinline__ bool ranks_before(unsigned long long ia, unsigned long long ca, unsigned long long oa,
                                             unsigned long long ib, unsigned long long cb, unsigned long long ob) {
    if (ib == kNoEntry) return ia != kNoEntry;
    if (ia == kNoEntry) return false;
    return ratio_better(ia, ca, oa, ib, cb, ob);
}
__global__ void __launch_bounds__(kRatioSort / 2) k_ratio_round(RatioArgs r, const unsigned long long *src,
                                                                unsigned long long len, unsigned long long *dst,
                                                                uint32_t keep) {
    __shared__ unsigned long long si[kRatioSort], sc[kRatioSort], so[kRatioSort];
    const unsigned long long base = (unsigned long long)blockIdx.x * kRatioSort;
    for (int j = threadIdx.x; j < kRatioSort; j += blockDim.x) {
        const unsigned long long p = base + j;
        const unsigned long long i = p < len ? (src ? src[p] : p) : kNoEntry;
        si[j] = i;
        sc[j] = i != kNoEntry ? r.cin[i] : 0ull;
        so[j] = i != kNoEntry ? r.cout[i] : 0ull;
    }
    __syncthreads();
    // ascending merges whose first stage compares mirrored positions: pairs
    // reaching past the block's valid entries meet padding (ranked last)
    // and never swap; stages within 64 positions stay inside one warp's
    // positions and need only a warp barrier (as in the per-document sort)
    const unsigned long long nv = len > base ? (len - base < (unsigned long long)kRatioSort ? len - base : kRatioSort) : 0ull;
    const int t = threadIdx.x;  // one compare-exchange pair per thread
    for (int size = 2; size <= kRatioSort; size <<= 1)
        for (int stride = size >> 1; stride; stride >>= 1) {
            const int a = 2 * t - (t & (stride - 1));
            const int b = stride == (size >> 1) ? (a ^ (size - 1)) : a + stride;
            if ((unsigned long long)b < nv && ranks_before(si[b], sc[b], so[b], si[a], sc[a], so[a])) {
                unsigned long long x = si[a]; si[a] = si[b]; si[b] = x;
                x = sc[a]; sc[a] = sc[b]; sc[b] = x;
                x = so[a]; so[a] = so[b]; so[b] = x;
            }
            const int span = 2 * stride, span_next = stride > 1 ? stride : 2 * size;
            if (span <= 64 && span_next <= 64) __syncwarp();
            else __syncthreads();
        }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < keep; j += blockDim.x) dst[(unsigned long long)blockIdx.x * keep + j] = si[j];
}

// Rows j < m of the ranking: (entry index, cin, cout).
__global__ void k_ratio_rows(RatioArgs r, const unsigned long long *list, unsigned long long m, unsigned long long *rows) {
    for (unsigned long long j = threadIdx.x; j < m; j += blockDim.x) {
        const unsigned long long i = list[j];
        rows[3 * j] = i;
        rows[3 * j + 1] = r.cin[i];
        rows[3 * j + 2] = r.cout[i];
    }
}

wc_status wc_class_ratio_topk(wc_ctx *ctx, const wc_batch *cb, uint32_t cls, uint32_t k, cudaStream_t stream,
                              uint64_t *h_idx, uint64_t *h_cin, uint64_t *h_cout, uint32_t *nout) {
    if (!ctx || !cb || !nout) return WC_ERR_INVALID_ARG;
    *nout = 0;
    wc_batch *b = const_cast<wc_batch *>(cb);
    if (cls >= b->nclasses) return ctx->fail(WC_ERR_INVALID_ARG, "class index out of range");
    cudaSetDevice(ctx->device);
    wc_status st = build_tables(b);
    if (st != WC_OK) return st;
    const wc_table *ct = b->class_tables[cls];
    if ((st = table_sync(ct)) != WC_OK) return st;
    if ((st = table_sync(b->global)) != WC_OK) return st;
    const uint64_t n = ct->n;
    const uint64_t m = std::min<uint64_t>(k, n);  // rows of the answer
    if (m == 0) return WC_OK;
    const bool rounds = k <= kRatioKeepMax;
    const uint64_t nblk = (n + kRatioSlice - 1) / kRatioSlice;  // first-round blocks (kRatioSort == kRatioSlice)
    // cin, cout, the answer rows; then two round lists (bitonic rounds) or
    // the top k + its length, the slices' winners + lengths and taken flags
    const size_t list_bytes = nblk * (size_t)m * 8;
    const size_t bytes = n * 16 + m * 24 +
                         (rounds ? 2 * list_bytes : ((size_t)k + 1) * 8 + nblk * ((size_t)k + 1) * 8 + n + nblk * k) + 256;
    void *mem = nullptr;
    if ((st = ctx->alloc(&mem, bytes, stream)) != WC_OK) return st;
    uint8_t *p = static_cast<uint8_t *>(mem);
    RatioArgs r;
    r.cls = ct->dt;
    r.g = b->gscratch.gtable(b->global->dt.d_status);
    r.cin = reinterpret_cast<unsigned long long *>(p);
    r.cout = r.cin + n;
    unsigned long long *rows = r.cout + n;
    r.k = k;
    r.out_idx = r.out_n = nullptr;
    const int sms = ctx->sms;
    uint64_t launches = 2;  // prepare, rows
    k_ratio_prepare<<<std::max<int>(1, std::min<int>(sms * 4, (int)((n + 255) / 256))), 256, 0, stream>>>(r);
    const unsigned long long *top = nullptr;
    if (rounds) {
        unsigned long long *list[2] = {rows + 3 * m, rows + 3 * m + nblk * m};
        const unsigned long long *src = nullptr;
        uint64_t len = n;
        int w = 0;
        for (;;) {
            const uint64_t nb = (len + kRatioSort - 1) / kRatioSort;
            k_ratio_round<<<(unsigned int)nb, kRatioSort / 2, 0, stream>>>(r, src, len, list[w], (uint32_t)m);
            launches++;
            if (nb == 1) break;
            src = list[w];
            len = nb * m;
            w ^= 1;
        }
        top = list[w];
    } else {
        r.out_idx = rows + 3 * m;
        r.out_n = r.out_idx + k;
        unsigned long long *cand = r.out_n + 1, *cand_n = cand + nblk * k;
        unsigned char *taken = reinterpret_cast<unsigned char *>(cand_n + nblk);
        cudaMemsetAsync(taken, 0, n + nblk * k, stream);
        k_ratio_select_slices<<<(unsigned int)nblk, 256, 0, stream>>>(r, taken, cand, cand_n);
        k_ratio_select<<<1, 1024, 0, stream>>>(r, taken + n, cand, cand_n, (unsigned int)nblk);
        top = r.out_idx;
        launches += 2;
    }
    ctx->launches += launches;
    k_ratio_rows<<<1, 256, 0, stream>>>(r, top, m, rows);
    std::vector<unsigned long long> h(3 * m);
    cudaError_t e = cudaMemcpyAsync(h.data(), rows, m * 24, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    ctx->release(mem, bytes, stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "class ratio ranking");
    for (uint64_t j = 0; j < m; j++) {
        if (h_idx) h_idx[j] = h[3 * j];
        if (h_cin) h_cin[j] = h[3 * j + 1];
        if (h_cout) h_cout[j] = h[3 * j + 2];
    }
    *nout = (uint32_t)m;
    return WC_OK;
}

// ---------------------------------------------------------------- bulk export
wc_status wc_batch_size(const wc_batch *b, uint64_t *nentries, uint64_t *word_bytes) {
    if (!b) return WC_ERR_INVALID_ARG;
    wc_status st = batch_sync(b);
    if (st != WC_OK) return st;
    wc_batch *mb = const_cast<wc_batch *>(b);
    if (!mb->word_bytes && mb->entries) {
        wc_table *v = nullptr;
        if ((st = make_view(mb, 0, mb->entries, &v)) != WC_OK) return st;
        st = table_sync(v);
        mb->word_bytes = v->word_bytes;
        free_owned_table(v);
        if (st != WC_OK) return st;
    }
    if (nentries) *nentries = mb->entries;
    if (word_bytes) *word_bytes = mb->word_bytes;
    return WC_OK;
}

wc_status wc_batch_export(const wc_batch *cb, uint64_t *h_doc_start, uint32_t *h_doc_n, uint8_t *h_words,
                          uint64_t *h_word_offsets, uint32_t *h_counts, cudaStream_t stream) {
    if (!cb) return WC_ERR_INVALID_ARG;
    wc_batch *b = const_cast<wc_batch *>(cb);
    cudaSetDevice(b->ctx->device);
    uint64_t n = 0, wb = 0;
    wc_status st = wc_batch_size(b, &n, &wb);
    if (st != WC_OK) return st;
    cudaError_t e = cudaSuccess;
    if (h_doc_start && b->ndocs)
        e = cudaMemcpyAsync(h_doc_start, b->args.doc_start, 8ull * b->ndocs, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && h_doc_n && b->ndocs)
        e = cudaMemcpyAsync(h_doc_n, b->args.doc_n, 4ull * b->ndocs, cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return b->ctx->cuda_fail(e, "batch export");
    if (!n) {
        if (h_word_offsets) h_word_offsets[0] = 0;
        e = cudaStreamSynchronize(stream);
        return e == cudaSuccess ? WC_OK : b->ctx->cuda_fail(e, "batch export");
    }
    wc_table *v = nullptr;
    if ((st = make_view(b, 0, n, &v)) != WC_OK) return st;
    st = wc_table_export(v, h_words, h_word_offsets, h_counts, stream);
    free_owned_table(v);
    return st;
}

void wc_batch_free(wc_batch *b) {
    if (!b) return;
    wc_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    if (b->done) cudaEventSynchronize(b->done);
    for (auto *v : b->views) free_owned_table(v);
    for (auto *t : b->class_tables) free_owned_table(t);
    free_owned_table(b->global);
    if (b->gscratch.mem) ctx->release(b->gscratch.mem, b->gscratch.bytes, b->stream);
    drop_vocab(b, b->stream);
    ctx->release(b->mem, b->bytes, b->stream);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

// ---------------------------------------------------------------- vocabulary ids
// The reduce of Sec. 3.3 keys every count by a word; here the batch's global
// table, ordered by word, is the one dictionary, and each per-document entry
// is stored as (row of that dictionary, count): words sort the same way as
// their ids, and a document's table needs 8 bytes a row.
static void drop_vocab(wc_batch *b, cudaStream_t s) {
    if (b->vocab) free_owned_table(b->vocab);
    b->vocab = nullptr;
    if (b->d_ids) b->ctx->release(b->d_ids, b->ids_bytes, s);
    b->d_ids = nullptr;
    b->ids_bytes = 0;
}

// The 16-byte table key of entry (khi, klo) (big-endian halves of the first
// 16 letters), as the count kernels build it.
__device__ __forceinline__ uint4 entry_key(unsigned long long hi8, unsigned long long lo8) {
    uint4 k;
    k.x = __byte_perm((uint32_t)(hi8 >> 32), 0, 0x0123);
    k.y = __byte_perm((uint32_t)hi8, 0, 0x0123);
    k.z = __byte_perm((uint32_t)(lo8 >> 32), 0, 0x0123);
    k.w = __byte_perm((uint32_t)lo8, 0, 0x0123);
    return k;
}

// Sort input: the global table's entries with every count zero, so that the
// stable (count desc, word asc) sort orders them by word alone.
__global__ void k_vocab_prep(DevTable G, SortScratch ss, unsigned long long *meta) {
    const unsigned long long n = G.d_meta[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) meta[0] = n;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        ss.khi[i] = G.khi[i];
        ss.klo[i] = G.klo[i];
        ss.cnt[i] = 0ull;
        ss.lref[i] = G.lref[i];
    }
}

// Row i of the vocabulary = the i-th word in word order (with its global
// count and the global table's long-word bytes); the id table maps each
// word to i + 1.
__global__ void k_vocab_place(DevTable G, SortScratch ss, DevTable V, GTable vg) {
    const unsigned long long n = G.d_meta[0];
    const uint32_t *perm = ss.perm_buf(ss.cur[kCurFinal]);
    if (blockIdx.x == 0 && threadIdx.x < 8) V.d_meta[threadIdx.x] = G.d_meta[threadIdx.x];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t src = perm[i];
        const unsigned long long hi8 = G.khi[src], lo8 = G.klo[src];
        const uint32_t r = G.lref[src];
        V.khi[i] = hi8;
        V.klo[i] = lo8;
        V.lref[i] = r;
        static_cast<unsigned long long *>(V.cnt)[i] = G.count_bits == 64
                                                          ? static_cast<const unsigned long long *>(G.cnt)[src]
                                                          : static_cast<const uint32_t *>(G.cnt)[src];
        if (r == 0) table_insert_key(vg, entry_key(hi8, lo8), i + 1);
        else long_insert(vg, G.arena + G.loff[r - 1], G.llen[r - 1], i + 1, nullptr, nullptr);
    }
}

// The vocabulary row of every per-document entry.
__global__ void k_vocab_ids(BatchArgs a, GTable vg, uint32_t *ids, unsigned long long n) {
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t r = a.out_lref[j];
        const unsigned long long v =
            r ? lookup_count(vg, make_uint4(0u, 0u, 0u, 0u), a.arena + a.loff[r - 1], a.llen[r - 1])
              : lookup_count(vg, entry_key(a.out_khi[j], a.out_klo[j]), nullptr, 0ull);
        ids[j] = (uint32_t)(v - 1ull);  // every document word is in the vocabulary
    }
}

static wc_status build_vocab(wc_batch *b) {
    if (b->vocab) return WC_OK;
    wc_status st = build_tables(b);
    if (st != WC_OK) return st;
    wc_ctx *ctx = b->ctx;
    cudaStream_t s = b->stream;
    wc_table *G = b->global;
    if ((st = table_sync(G)) != WC_OK) return st;
    const uint64_t n = G->n, nlong = G->nlong;
    // sort scratch + the id hash tables (sized from the known word counts)
    CapPlan plan;
    plan.cap8 = pow2_ge(std::max<uint64_t>(1024, 2 * n));
    plan.cap16 = pow2_ge(std::max<uint64_t>(1024, n + n / 4));
    plan.caplong = pow2_ge(std::max<uint64_t>(256, 2 * nlong));
    plan.arena = 4096;
    CountScratch cs;
    if ((st = scratch_create(ctx, plan, false, s, cs)) != WC_OK) return st;
    wc_table *V = nullptr;
    if ((st = table_create(ctx, std::max<uint64_t>(1, n), 1, 16, 64, s, &V)) != WC_OK) {
        ctx->release(cs.mem, cs.bytes, s);
        return st;
    }
    V->owner = b;
    V->dt.loff = G->dt.loff;  // long words: the global table's bytes
    V->dt.llen = G->dt.llen;
    V->dt.arena = G->dt.arena;
    V->dt.lcap = G->dt.lcap;
    V->dt.arena_cap = G->dt.arena_cap;
    void *ids = nullptr;
    const size_t ib = 4 * std::max<uint64_t>(1, b->entries);
    if ((st = ctx->alloc(&ids, ib, s)) != WC_OK) {
        free_owned_table(V);
        ctx->release(cs.mem, cs.bytes, s);
        return st;
    }
    void *dmeta = nullptr;
    if ((st = ctx->alloc(&dmeta, 64, s)) != WC_OK) {
        ctx->release(ids, ib, s);
        free_owned_table(V);
        ctx->release(cs.mem, cs.bytes, s);
        return st;
    }
    unsigned long long *smeta = static_cast<unsigned long long *>(dmeta);
    cudaMemsetAsync(smeta, 0, 64, s);
    const GTable vg = cs.gtable(V->dt.d_status);
    const int grid = std::max(1, std::min(ctx->sms * 8, (int)((std::max<uint64_t>(n, b->entries) + 255) / 256)));
    cudaStreamWaitEvent(s, G->done, 0);
    sort_state_reset(cs.ss, s);
    k_vocab_prep<<<grid, 256, 0, s>>>(G->dt, cs.ss, smeta);
    const LongView lv{G->dt.lref, G->dt.loff, G->dt.llen, G->dt.arena};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = sort_entries(cs.ss, smeta, lv, kSortPasses, s, sort_skip_mask(0, 0));
    if (e == cudaSuccess) {
        k_vocab_place<<<grid, 256, 0, s>>>(G->dt, cs.ss, V->dt, vg);
        k_vocab_ids<<<grid, 256, 0, s>>>(b->args, vg, static_cast<uint32_t *>(ids), b->entries);
        e = cudaGetLastError();
    }
    ctx->launches += 4 + (uint64_t)sort_entries_launches(kSortPasses, cs.ss.cap, sort_skip_mask(0, 0));
    ctx->release(dmeta, 64, s);
    ctx->release(cs.mem, cs.bytes, s);
    table_mark_done(V, s);
    if (e != cudaSuccess) {
        ctx->release(ids, ib, s);
        free_owned_table(V);
        return ctx->cuda_fail(e, "vocabulary ids");
    }
    if ((st = table_sync(V)) != WC_OK) {  // an overflowing id table is reported, never used
        ctx->release(ids, ib, s);
        free_owned_table(V);
        return st;
    }
    b->vocab = V;
    b->d_ids = static_cast<uint32_t *>(ids);
    b->ids_bytes = ib;
    return WC_OK;
}

wc_status wc_batch_vocab(const wc_batch *cb, const wc_table **out) {
    if (!cb || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    wc_batch *b = const_cast<wc_batch *>(cb);
    cudaSetDevice(b->ctx->device);
    const wc_status st = build_vocab(b);
    if (st != WC_OK) return st;
    *out = b->vocab;
    return WC_OK;
}

wc_status wc_batch_export_ids(const wc_batch *cb, uint64_t *h_doc_start, uint32_t *h_doc_n, uint32_t *h_ids,
                              uint32_t *h_counts, cudaStream_t stream) {
    if (!cb) return WC_ERR_INVALID_ARG;
    wc_batch *b = const_cast<wc_batch *>(cb);
    cudaSetDevice(b->ctx->device);
    wc_status st = build_vocab(b);
    if (st != WC_OK) return st;
    cudaStreamWaitEvent(stream, b->vocab->done, 0);
    cudaError_t e = cudaSuccess;
    if (h_doc_start && b->ndocs)
        e = cudaMemcpyAsync(h_doc_start, b->args.doc_start, 8ull * b->ndocs, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && h_doc_n && b->ndocs)
        e = cudaMemcpyAsync(h_doc_n, b->args.doc_n, 4ull * b->ndocs, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && h_ids && b->entries)
        e = cudaMemcpyAsync(h_ids, b->d_ids, 4ull * b->entries, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && h_counts && b->entries)
        e = cudaMemcpyAsync(h_counts, b->args.out_cnt, 4ull * b->entries, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return b->ctx->cuda_fail(e, "id export");
    return WC_OK;
}
