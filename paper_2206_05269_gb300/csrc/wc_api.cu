// C-ABI entry points (include/wc.h): contexts, tables, counting, merge,
// top-k and export.  Device memory comes from a per-context stream-ordered
// pool and is charged against the context's budget.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wc.h"
#include "wc_internal.h"
#include "wc_batch.h"
#include "wc_host.h"

using namespace wc;

// ---------------------------------------------------------------- context
const char *wc_status_str(wc_status s) {
    switch (s) {
    case WC_OK: return "ok";
    case WC_ERR_INVALID_ARG: return "invalid argument";
    case WC_ERR_OOM: return "out of device memory";
    case WC_ERR_BUDGET: return "device-memory budget exceeded";
    case WC_ERR_CAPACITY: return "table capacity exceeded";
    case WC_ERR_CUDA: return "CUDA error";
    case WC_ERR_TIMEOUT: return "device wait timed out";
    case WC_ERR_INTERNAL: return "internal error";
    case WC_ERR_UNSUPPORTED: return "unsupported input";
    }
    return "unknown status";
}

const char *wc_last_error(const wc_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

wc_status wc_ctx::fail(wc_status s, const char *what) {
    last_error = std::string(wc_status_str(s)) + ": " + what;
    return s;
}
wc_status wc_ctx::cuda_fail(cudaError_t e, const char *what) {
    last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return WC_ERR_OOM;
    return WC_ERR_CUDA;
}

wc_status wc_ctx::alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    // reserve the bytes against the budget first (compare-and-swap: two
    // callers can never both pass a budget that holds only one of them)
    uint64_t cur = used.load();
    do {
        if (budget && cur + bytes > budget) return fail(WC_ERR_BUDGET, "allocation over the context budget");
    } while (!used.compare_exchange_weak(cur, cur + bytes));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        used -= bytes;
        *p = nullptr;
        return cuda_fail(e, "cudaMallocFromPoolAsync");
    }
    uint64_t pk = peak.load();
    while (cur + bytes > pk && !peak.compare_exchange_weak(pk, cur + bytes)) {
    }
    return WC_OK;
}
namespace {
struct ReleaseArg {
    wc_ctx *ctx;
    size_t bytes;
};
void CUDART_CB release_done(void *a) {  // runs once the stream has passed the free
    ReleaseArg *r = static_cast<ReleaseArg *>(a);
    r->ctx->used -= r->bytes;
    delete r;
}
}  // namespace

// Stream-ordered free: the bytes stay charged to the budget until the stream
// has passed the free (a host callback after it), because work enqueued
// before it may still use them.  While the stream is being captured into a
// graph the charge is dropped at once (the graph's own allocation and free
// nodes balance on every replay).
void wc_ctx::release(void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    cudaFreeAsync(p, s);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;  // unknown: do not defer
    }
    if (cap == cudaStreamCaptureStatusNone) {
        ReleaseArg *r = new ReleaseArg{this, bytes};
        if (cudaLaunchHostFunc(s, release_done, r) == cudaSuccess) return;
        cudaGetLastError();
        delete r;
    }
    used -= bytes;
}

void wc_ctx::prof_mark(std::vector<cudaEvent_t> &v, cudaStream_t s) {
    cudaEvent_t e = prof_event(v);
    if (e) cudaEventRecord(e, s);
}

cudaEvent_t wc_ctx::prof_event(std::vector<cudaEvent_t> &v) {
    if (!profile) return nullptr;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    v.push_back(e);
    return e;
}

static void prof_clear(wc_ctx *ctx) {
    for (auto e : ctx->ev_head) cudaEventDestroy(e);
    for (auto e : ctx->ev_count) cudaEventDestroy(e);
    for (auto e : ctx->ev_finish) cudaEventDestroy(e);
    ctx->ev_head.clear();
    ctx->ev_count.clear();
    ctx->ev_finish.clear();
    ctx->launches = 0;
}

wc_status wc_profile_enable(wc_ctx *ctx, int enable) {
    if (!ctx) return WC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    prof_clear(ctx);
    ctx->profile = enable != 0;
    return WC_OK;
}

static double sum_pairs(wc_ctx *ctx, const std::vector<cudaEvent_t> &v, cudaError_t *err) {
    double tot = 0;
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        float ms = 0;
        cudaError_t e = cudaEventSynchronize(v[i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, v[i], v[i + 1]);
        if (e != cudaSuccess) *err = e;
        tot += ms;
    }
    return tot;
}

wc_status wc_profile_read(wc_ctx *ctx, double *ms_head, double *ms_count, double *ms_finish,
                          uint64_t *count_launches, uint64_t *kernel_launches) {
    if (!ctx) return WC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaError_t err = cudaSuccess;
    double h = sum_pairs(ctx, ctx->ev_head, &err);
    double a = sum_pairs(ctx, ctx->ev_count, &err), b = sum_pairs(ctx, ctx->ev_finish, &err);
    if (err != cudaSuccess) return ctx->cuda_fail(err, "wc_profile_read");
    if (ms_head) *ms_head = h;
    if (ms_count) *ms_count = a;
    if (ms_finish) *ms_finish = b;
    if (count_launches) *count_launches = ctx->ev_count.size() / 2;
    if (kernel_launches) *kernel_launches = ctx->launches;
    return WC_OK;
}

// Autotuner cache: a JSON object keyed by GPU name, e.g.
//   {"NVIDIA GB300": {"small": 0, "medium": 3, "large": 4}}
// (shape indices of the per-document kernel per size class).  An entry for
// this GPU is used as it is: plans then skip the timing.
void wc_ctx::tune_load() {
    if (tune_cache_path.empty()) return;
    FILE *f = fopen(tune_cache_path.c_str(), "rb");
    if (!f) return;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
    fclose(f);
    size_t k = txt.find("\"" + gpu_name + "\"");
    if (k == std::string::npos) return;
    auto num = [&](const char *field, int *dst) {
        size_t q = txt.find(std::string("\"") + field + "\"", k);
        if (q == std::string::npos) return;
        q = txt.find(':', q);
        if (q == std::string::npos) return;
        int v = atoi(txt.c_str() + q + 1);
        if (v >= 0 && v < kNumDocShapes) *dst = v;
    };
    num("small", &tuned_small);
    num("medium", &tuned_medium);
    num("large", &tuned_large);
    tuned = true;
}

void wc_ctx::tune_save() const {
    if (tune_cache_path.empty()) return;
    FILE *f = fopen(tune_cache_path.c_str(), "wb");
    if (!f) return;
    fprintf(f, "{\"%s\": {\"small\": %d, \"medium\": %d, \"large\": %d}}\n", gpu_name.c_str(), tuned_small,
            tuned_medium, tuned_large);
    fclose(f);
}

wc_status wc_create(const wc_config *cfg, wc_ctx **out) {
    if (!out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    wc_config c{0, 0, 64, 0, nullptr};
    if (cfg) c = *cfg;
    if (c.count_bits != 32 && c.count_bits != 64) return WC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return WC_ERR_INVALID_ARG;
    }
    wc_ctx *ctx = new wc_ctx();
    ctx->device = c.device;
    ctx->budget = c.mem_budget_bytes;
    ctx->count_bits = c.count_bits;
    ctx->autotune = c.autotune;
    if (c.tune_cache_path) ctx->tune_cache_path = c.tune_cache_path;
    cudaSetDevice(c.device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c.device;
    cudaError_t e = cudaMemPoolCreate(&ctx->pool, &props);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return WC_ERR_CUDA;
    }
    uint64_t keep = UINT64_MAX;  // keep freed memory cached in the pool
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, c.device);
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, c.device) == cudaSuccess) ctx->gpu_name = prop.name;
    ctx->tune_load();
    *out = ctx;
    return WC_OK;
}

void wc_destroy(wc_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    prof_clear(ctx);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->meta_host) cudaFreeHost(ctx->meta_host);
    cudaMemPoolDestroy(ctx->pool);
    delete ctx;
}

// ---------------------------------------------------------------- numeric MapReduce
wc_status wc_series_sum(wc_ctx *ctx, int series, uint64_t n, double *d_out, cudaStream_t stream) {
    if (!ctx || !d_out) return WC_ERR_INVALID_ARG;
    if (series != WC_SERIES_SQRT && series != WC_SERIES_ALT_HARMONIC)
        return ctx->fail(WC_ERR_INVALID_ARG, "unknown series");
    if (n >= (1ull << 53)) return ctx->fail(WC_ERR_UNSUPPORTED, "n of 2^53 or more (indices not exact in double)");
    cudaSetDevice(ctx->device);
    const int nb = series_blocks(n);
    void *part = nullptr;
    wc_status st = ctx->alloc(&part, sizeof(double2) * (size_t)nb, stream);
    if (st != WC_OK) return st;
    const cudaError_t e = launch_series(series, n, static_cast<double2 *>(part), nb, d_out, stream);
    ctx->release(part, sizeof(double2) * (size_t)nb, stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "series sum");
    ctx->launches += 2;
    return WC_OK;
}

// ---------------------------------------------------------------- hybrid pipeline reduce
wc_status wc_row_sums(const uint32_t *d_matrix, uint64_t rows, uint64_t cols, uint64_t *d_sums, cudaStream_t stream) {
    if (rows && (!d_sums || (cols && !d_matrix))) return WC_ERR_INVALID_ARG;
    if (rows && cols > UINT64_MAX / 4 / rows) return WC_ERR_INVALID_ARG;
    const cudaError_t e = launch_row_sums(d_matrix, rows, cols, reinterpret_cast<unsigned long long *>(d_sums), stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return WC_ERR_CUDA;
    }
    return WC_OK;
}

// ---------------------------------------------------------------- budgeted buffers
wc_status wc_buffer_alloc(wc_ctx *ctx, uint64_t bytes, cudaStream_t stream, void **out) {
    if (!ctx || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    return ctx->alloc(out, bytes, stream);
}

wc_status wc_buffer_free(wc_ctx *ctx, void *p, uint64_t bytes, cudaStream_t stream) {
    if (!ctx) return WC_ERR_INVALID_ARG;
    if (!p) return WC_OK;
    cudaSetDevice(ctx->device);
    ctx->release(p, bytes, stream);
    return WC_OK;
}

wc_status wc_mem_usage(wc_ctx *ctx, uint64_t *used, uint64_t *peak, int reset) {
    if (!ctx) return WC_ERR_INVALID_ARG;
    const uint64_t u = ctx->used.load();
    if (used) *used = u;
    if (peak) *peak = ctx->peak.load();
    if (reset) ctx->peak.store(u);
    return WC_OK;
}

// ---------------------------------------------------------------- wait self-test
static wc_status status_from_bits(uint32_t bits);

wc_status wc_selftest_wait(wc_ctx *ctx, uint32_t polls, int arrive, cudaStream_t stream) {
    if (!ctx) return WC_ERR_INVALID_ARG;
    if (polls < 1 || polls > (1u << 22)) return ctx->fail(WC_ERR_INVALID_ARG, "polls outside 1 .. 2^22");
    cudaSetDevice(ctx->device);
    void *d = nullptr;
    wc_status st = ctx->alloc(&d, 256, stream);
    if (st != WC_OK) return st;
    uint32_t *d_status = static_cast<uint32_t *>(d);
    uint32_t h = 0;
    cudaError_t e = cudaMemsetAsync(d_status, 0, 4, stream);
    if (e == cudaSuccess) e = launch_wait_selftest(d_status, polls, arrive, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    ctx->release(d, 256, stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "wait self-test");
    ctx->launches++;
    st = status_from_bits(h);
    if (st != WC_OK) return ctx->fail(st, "bounded device wait gave up (self-test)");
    return WC_OK;
}

// ---------------------------------------------------------------- tables
static size_t table_bytes(uint64_t cap, uint64_t lcap, uint64_t arena, int bits) {
    auto r = [](size_t n) { return (n + 255) & ~(size_t)255; };
    return r(8 * 8) + r(4) + r(cap * 8) * 2 + r(cap * (bits / 8)) + r(cap * 4) + r(lcap * 8) * 2 + r(arena);
}

wc_status table_create(wc_ctx *ctx, uint64_t cap, uint64_t lcap, uint64_t arena, int bits, cudaStream_t s,
                       wc_table **out) {
    wc_table *t = new wc_table();
    t->ctx = ctx;
    t->bytes = table_bytes(cap, lcap, arena, bits);
    wc_status st = ctx->alloc(&t->mem, t->bytes, s);
    if (st != WC_OK) { delete t; return st; }
    uint8_t *p = static_cast<uint8_t *>(t->mem);
    auto take = [&](size_t n) { uint8_t *q = p; p += (n + 255) & ~(size_t)255; return q; };
    DevTable &d = t->dt;
    d.cap = cap;
    d.lcap = lcap;
    d.arena_cap = arena;
    d.count_bits = bits;
    d.d_meta = reinterpret_cast<unsigned long long *>(take(8 * 8));
    d.d_status = reinterpret_cast<uint32_t *>(take(4));
    d.khi = reinterpret_cast<unsigned long long *>(take(cap * 8));
    d.klo = reinterpret_cast<unsigned long long *>(take(cap * 8));
    d.cnt = take(cap * (bits / 8));
    d.lref = reinterpret_cast<uint32_t *>(take(cap * 4));
    d.loff = reinterpret_cast<unsigned long long *>(take(lcap * 8));
    d.llen = reinterpret_cast<unsigned long long *>(take(lcap * 8));
    d.arena = take(arena);
    cudaMemsetAsync(t->mem, 0, 512, s);  // meta + status
    t->stream = s;
    cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming);
    *out = t;
    return WC_OK;
}

int wc_ctx::meta_take() {
    std::lock_guard<std::mutex> g(meta_mu);
    if (!meta_host) {
        void *p = nullptr;
        if (cudaHostAlloc(&p, (size_t)kMetaSlots * kMetaSlotBytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        meta_host = static_cast<uint8_t *>(p);
        meta_free.reserve(kMetaSlots);
        for (int i = kMetaSlots - 1; i >= 0; i--) meta_free.push_back(i);
    }
    if (meta_free.empty()) return -1;
    const int slot = meta_free.back();
    meta_free.pop_back();
    return slot;
}

void wc_ctx::meta_give(int slot) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> g(meta_mu);
    meta_free.push_back(slot);
}

// The table's work is all enqueued on s: its metadata and status follow it
// into a pinned slot, then the done event.
void table_mark_done(wc_table *t, cudaStream_t s) {
    t->stream = s;
    if (t->meta_slot < 0) t->meta_slot = t->ctx->meta_take();
    if (t->meta_slot >= 0) {
        uint8_t *h = t->ctx->meta_host + (size_t)t->meta_slot * wc_ctx::kMetaSlotBytes;
        cudaMemcpyAsync(h, t->dt.d_meta, 64, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h + 64, t->dt.d_status, 4, cudaMemcpyDeviceToHost, s);
    }
    cudaEventRecord(t->done, s);
}

static wc_status status_from_bits(uint32_t bits) {
    if (bits & (ST_TABLE_FULL | ST_LONG_FULL | ST_ARENA_FULL | ST_OUT_FULL)) return WC_ERR_CAPACITY;
    if (bits & ST_TIMEOUT) return WC_ERR_TIMEOUT;
    if (bits & ST_TOO_LONG) return WC_ERR_UNSUPPORTED;
    if (bits & ST_BAD_CLASS) return WC_ERR_INVALID_ARG;
    return WC_OK;
}

wc_status table_sync(const wc_table *ct) {
    wc_table *t = const_cast<wc_table *>(ct);
    if (t->synced) return t->sync_status;
    cudaError_t e = cudaEventSynchronize(t->done);
    if (e != cudaSuccess) return t->ctx->cuda_fail(e, "cudaEventSynchronize");
    unsigned long long meta[8];
    uint32_t status = 0;
    if (t->meta_slot >= 0) {  // landed with the table's work
        const uint8_t *h = t->ctx->meta_host + (size_t)t->meta_slot * wc_ctx::kMetaSlotBytes;
        memcpy(meta, h, sizeof(meta));
        memcpy(&status, h + 64, 4);
    } else {
        e = cudaMemcpy(meta, t->dt.d_meta, sizeof(meta), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&status, t->dt.d_status, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return t->ctx->cuda_fail(e, "reading table metadata");
    }
    t->n = meta[0];
    t->nlong = meta[1];
    t->tokens = meta[3];
    t->word_bytes = meta[4];
    t->status_bits = status;
    t->sync_status = status_from_bits(status);
    if (t->sync_status != WC_OK) {
        t->n = t->tokens = t->word_bytes = 0;
        t->ctx->fail(t->sync_status, ("device table overflow or wait limit (status bits " + std::to_string(status) +
                                      "); count again with larger capacities").c_str());
    }
    if (t->sync_status == WC_OK && t->src_bytes) {
        wc_ctx *c = t->ctx;
        c->hist_bytes = t->src_bytes;
        c->hist_n8 = meta[5];
        c->hist_n16 = meta[6];
        c->hist_nlong = meta[1];
        c->hist_arena = meta[2];
    }
    t->synced = true;
    return t->sync_status;
}

wc_status wc_table_status(const wc_table *t) {
    if (!t) return WC_ERR_INVALID_ARG;
    return table_sync(t);
}

int wc_table_count_bits(const wc_table *t) { return t ? t->dt.count_bits : 0; }

wc_status wc_table_size(const wc_table *t, uint64_t *nwords, uint64_t *ntokens, uint64_t *word_bytes) {
    if (!t) return WC_ERR_INVALID_ARG;
    wc_status s = table_sync(t);
    if (nwords) *nwords = t->n;
    if (ntokens) *ntokens = t->tokens;
    if (word_bytes) *word_bytes = t->word_bytes;
    return s;
}

wc_status wc_table_export(const wc_table *t, uint8_t *h_words, uint64_t *h_word_offsets, void *h_counts,
                          cudaStream_t stream) {
    if (!t) return WC_ERR_INVALID_ARG;
    wc_ctx *ctx = t->ctx;
    wc_status s = table_sync(t);
    if (s != WC_OK) return s;
    const DevTable &d = t->dt;
    const uint64_t n = t->n;
    cudaError_t e = cudaSuccess;
    // the counts go to the host on the context's copy stream while the word
    // bytes and offsets are built on `stream` (overlapped when h_counts is pinned)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    const bool side = h_counts && n && (h_words || h_word_offsets) &&
                      (ctx->copy_stream || cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) ==
                                               cudaSuccess) &&
                      cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess &&
                      cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess;
    if (h_counts && n) {
        if (side) {
            cudaEventRecord(ev[0], stream);
            cudaStreamWaitEvent(ctx->copy_stream, ev[0], 0);
        }
        e = cudaMemcpyAsync(h_counts, d.cnt, n * (d.count_bits / 8), cudaMemcpyDeviceToHost,
                            side ? ctx->copy_stream : stream);
        if (side) cudaEventRecord(ev[1], ctx->copy_stream);
        if (e != cudaSuccess) {
            for (auto x : ev)
                if (x) cudaEventDestroy(x);
            return ctx->cuda_fail(e, "copying counts");
        }
    }
    auto abandon = [&](wc_status st) {  // an allocation failed: let the counts copy land first
        if (side) cudaStreamSynchronize(ctx->copy_stream);
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
        return st;
    };
    if (h_words || h_word_offsets) {
        size_t sb = export_scratch_bytes(d.cap);
        size_t wb = t->word_bytes ? t->word_bytes : 1;
        void *scratch = nullptr, *dwords = nullptr, *doffs = nullptr;
        if ((s = ctx->alloc(&scratch, sb, stream)) != WC_OK) return abandon(s);
        if ((s = ctx->alloc(&dwords, wb, stream)) != WC_OK) {
            ctx->release(scratch, sb, stream);
            return abandon(s);
        }
        if ((s = ctx->alloc(&doffs, (d.cap + 1) * 8, stream)) != WC_OK) {
            ctx->release(scratch, sb, stream);
            ctx->release(dwords, wb, stream);
            return abandon(s);
        }
        e = launch_export(d, scratch, static_cast<uint8_t *>(dwords), static_cast<unsigned long long *>(doffs), stream);
        if (e == cudaSuccess && h_words && t->word_bytes)
            e = cudaMemcpyAsync(h_words, dwords, t->word_bytes, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess && h_word_offsets)
            e = cudaMemcpyAsync(h_word_offsets, doffs, (n + 1) * 8, cudaMemcpyDeviceToHost, stream);
        ctx->release(scratch, sb, stream);
        ctx->release(dwords, wb, stream);
        ctx->release(doffs, (d.cap + 1) * 8, stream);
    }
    if (side) cudaStreamWaitEvent(stream, ev[1], 0);
    const cudaError_t es = cudaStreamSynchronize(stream);
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "export");
    if (es != cudaSuccess) return ctx->cuda_fail(es, "cudaStreamSynchronize (export)");
    return WC_OK;
}

void wc_table_free(wc_table *t) {
    if (!t) return;
    if (t->owner) return;  // borrowed from a batch
    cudaSetDevice(t->ctx->device);
    cudaEventSynchronize(t->done);
    t->ctx->release(t->mem, t->bytes, t->stream);
    t->ctx->meta_give(t->meta_slot);
    cudaEventDestroy(t->done);
    delete t;
}

// ---------------------------------------------------------------- counting
static uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Automatic capacities.  Distinct words of a text of B bytes are estimated
// from T = B/5 tokens as the larger of a Heaps'-law term 16 * T^0.6 (a small
// vocabulary) and T/4 (a large vocabulary in a mid-sized text, where most
// tokens of the Zipf tail are still first occurrences), the latter capped at
// 2M distinct words so huge texts keep L2-sized tables, and never above the
// exact bound ceil(B/2).  When the context has counted a text within 8x of
// this size before, the distinct counts it saw (per key width) are used
// instead, twice over and scaled up (never down) by size: distinct words
// grow more slowly than the text.  Overflow is reported, never silent:
// callers count again with larger capacities.
CapPlan plan_capacity(const wc_ctx *ctx, uint64_t nbytes, const wc_count_opts *o) {
    double tokens = (double)nbytes / 5.0 + 1.0;
    double est = std::min(tokens, std::max(16.0 * std::pow(tokens, 0.6), std::min(tokens / 4.0, 2097152.0)));
    uint64_t bound = nbytes / 2 + 1;
    uint64_t d = std::min<uint64_t>((uint64_t)est + 64, bound);
    CapPlan p;
    p.cap8 = pow2_at_least(std::max<uint64_t>(1024, d + d / 5));
    p.cap16 = pow2_at_least(std::max<uint64_t>(1024, d * 3 / 5));
    p.caplong = pow2_at_least(std::max<uint64_t>(256, 2 * (d / 16 + 16)));
    p.arena = std::max<uint64_t>(4096, std::min<uint64_t>(nbytes + nbytes / 16 + 16, p.caplong * 24));
    if (ctx && ctx->hist_bytes && nbytes <= 8 * ctx->hist_bytes && 8 * nbytes >= ctx->hist_bytes) {
        double r = (double)nbytes / (double)ctx->hist_bytes;
        auto scaled = [&](uint64_t n) { return (uint64_t)((double)n * std::max(1.0, r)) + 64; };
        p.cap8 = pow2_at_least(std::max<uint64_t>(1024, 2 * scaled(ctx->hist_n8)));
        p.cap16 = pow2_at_least(std::max<uint64_t>(1024, 2 * scaled(ctx->hist_n16)));
        p.caplong = pow2_at_least(std::max<uint64_t>(256, 2 * scaled(ctx->hist_nlong)));
        p.arena = std::max<uint64_t>(4096, 2 * scaled(ctx->hist_arena));
    }
    if (o) {
        if (o->table_slots) {
            p.cap8 = pow2_at_least(std::max<uint64_t>(64, o->table_slots));
            p.cap16 = pow2_at_least(std::max<uint64_t>(64, o->table_slots));
        }
        if (o->long_slots) p.caplong = pow2_at_least(std::max<uint64_t>(64, o->long_slots));
        if (o->arena_bytes) p.arena = std::max<uint64_t>(64, o->arena_bytes);
    }
    return p;
}

// Allocates the hash tables (+ head-selection scratch) + sort scratch in one block.
wc_status scratch_create(wc_ctx *ctx, const CapPlan &p, bool head, cudaStream_t s, CountScratch &cs) {
    cs.gcap8 = p.cap8;
    cs.gcap = p.cap16;
    cs.glcap = p.caplong;
    auto r = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t b8 = r(p.cap8 * sizeof(G8Slot)), b16 = r(p.cap16 * sizeof(GSlot)), bl = r(p.caplong * sizeof(LSlot));
    const size_t hb = b8 + b16 + bl;
    const size_t bh = head ? r(head_scratch_bytes()) : 0;
    cs.bytes = hb + bh + sort_scratch_bytes(cs.entries(), true) + 512;
    wc_status st = ctx->alloc(&cs.mem, cs.bytes, s);
    if (st != WC_OK) return st;
    uint8_t *q = static_cast<uint8_t *>(cs.mem);
    cs.slots8 = reinterpret_cast<G8Slot *>(q);
    cs.slots = reinterpret_cast<GSlot *>(q + b8);
    cs.lslots = reinterpret_cast<LSlot *>(q + b8 + b16);
    cs.head = head ? q + hb : nullptr;
    sort_scratch_carve(cs.ss, q + hb + bh, cs.entries(), true);
    cudaMemsetAsync(cs.mem, 0, hb, s);
    return WC_OK;
}

wc_status wc_count_ex(wc_ctx *ctx, const uint8_t *d_text, uint64_t nbytes, const wc_count_opts *opts,
                      cudaStream_t stream, wc_table **out) {
    if (!ctx || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d_text && nbytes) return ctx->fail(WC_ERR_INVALID_ARG, "null text");
    if (nbytes >= (1ull << 40)) return ctx->fail(WC_ERR_UNSUPPORTED, "text of 2^40 bytes or more");
    if (ctx->count_bits == 32 && nbytes >= (1ull << 33))
        return ctx->fail(WC_ERR_UNSUPPORTED, "32-bit counts need inputs under 2^33 bytes");
    cudaSetDevice(ctx->device);
    const CapPlan plan = plan_capacity(ctx, nbytes, opts);
    CountScratch cs;
    // head scratch only for texts long enough to sample a head from
    wc_status st = scratch_create(ctx, plan, nbytes >= count_global_head_min(), stream, cs);
    if (st != WC_OK) return st;
    wc_table *t = nullptr;
    st = table_create(ctx, cs.entries(), plan.caplong, plan.arena, ctx->count_bits, stream, &t);
    if (st != WC_OK) { ctx->release(cs.mem, cs.bytes, stream); return st; }
    t->src_bytes = nbytes;
    const GTable g = cs.gtable(t->dt.d_status);
    CountLaunch cl{d_text, 0, nbytes, g, 0, cs.head, {nullptr, nullptr}};
    cl.no_level1 = opts && opts->no_level1 ? 1 : 0;
    // stages: head selection (sampling pass + head kernels), then the main counting kernel
    ctx->prof_mark(ctx->ev_head, stream);
    cl.main_ev[0] = ctx->prof_event(ctx->ev_head);
    cl.main_ev[1] = ctx->prof_event(ctx->ev_count);
    cudaError_t e = launch_count_global(cl, stream);
    ctx->prof_mark(ctx->ev_count, stream);
    ctx->launches += count_global_launches(nbytes, !cl.no_level1, cs.head != nullptr);
    ctx->prof_mark(ctx->ev_finish, stream);
    const uint32_t skip = sort_skip_mask(nbytes / 2 + 1, 0);  // no count exceeds the token bound
    if (e == cudaSuccess) e = finish_table(g, cs.gcap8, cs.gcap, cs.glcap, cs.ss, t->dt, stream, skip);
    ctx->prof_mark(ctx->ev_finish, stream);
    ctx->launches += finish_table_launches(cs.ss, skip);
    ctx->release(cs.mem, cs.bytes, stream);
    table_mark_done(t, stream);
    if (e != cudaSuccess) {
        wc_table_free(t);
        return ctx->cuda_fail(e, "count launch");
    }
    *out = t;
    return WC_OK;
}

wc_status wc_count(wc_ctx *ctx, const uint8_t *d_text, uint64_t nbytes, cudaStream_t stream, wc_table **out) {
    return wc_count_ex(ctx, d_text, nbytes, nullptr, stream, out);
}

// ---------------------------------------------------------------- counting from host memory
static bool host_letter(uint8_t b) { return (uint8_t)((b | 0x20) - 0x61) < 26 && b < 0x80; }

wc_status wc_count_host(wc_ctx *ctx, const uint8_t *h_text, uint64_t nbytes, uint8_t *d_buf, uint64_t piece_bytes,
                        const wc_count_opts *opts, cudaStream_t stream, wc_table **out) {
    if (!ctx || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h_text && nbytes) return ctx->fail(WC_ERR_INVALID_ARG, "null text");
    if (nbytes >= (1ull << 40)) return ctx->fail(WC_ERR_UNSUPPORTED, "text of 2^40 bytes or more");
    if (ctx->count_bits == 32 && nbytes >= (1ull << 33))
        return ctx->fail(WC_ERR_UNSUPPORTED, "32-bit counts need inputs under 2^33 bytes");
    cudaSetDevice(ctx->device);
    if (!ctx->copy_stream && cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->copy_stream = nullptr;
        return ctx->fail(WC_ERR_CUDA, "cudaStreamCreate (copy stream)");
    }
    // pieces cut where a letter is not followed by a letter: no word spans two
    if (!piece_bytes) piece_bytes = std::max<uint64_t>(64ull << 20, (nbytes + 31) / 32);
    std::vector<uint64_t> cut{0};
    while (cut.back() < nbytes) {
        uint64_t e = std::min(nbytes, cut.back() + piece_bytes);
        while (e < nbytes && host_letter(h_text[e - 1]) && host_letter(h_text[e])) e++;
        cut.push_back(e);
    }
    // the device copy of the text, tables for the whole text, the output table
    void *own = nullptr;
    uint8_t *dt = d_buf;
    wc_status st = WC_OK;
    if (!dt && (st = ctx->alloc(&own, std::max<uint64_t>(nbytes, 16), stream)) != WC_OK) return st;
    if (!dt) dt = static_cast<uint8_t *>(own);
    const CapPlan plan = plan_capacity(ctx, nbytes, opts);
    CountScratch cs;
    if ((st = scratch_create(ctx, plan, true, stream, cs)) != WC_OK) {
        if (own) ctx->release(own, std::max<uint64_t>(nbytes, 16), stream);
        return st;
    }
    wc_table *t = nullptr;
    if ((st = table_create(ctx, cs.entries(), plan.caplong, plan.arena, ctx->count_bits, stream, &t)) != WC_OK) {
        ctx->release(cs.mem, cs.bytes, stream);
        if (own) ctx->release(own, std::max<uint64_t>(nbytes, 16), stream);
        return st;
    }
    t->src_bytes = nbytes;
    const GTable g = cs.gtable(t->dt.d_status);
    // copies on the copy stream (after the caller's earlier work); each piece
    // is counted on the caller's stream once it has landed, so later copies
    // overlap earlier counts
    const size_t np = cut.size() - 1;
    std::vector<cudaEvent_t> ev(np + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[np], stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ev[np], 0);
    for (size_t i = 0; i < np && e == cudaSuccess; i++) {
        e = cudaMemcpyAsync(dt + cut[i], h_text + cut[i], cut[i + 1] - cut[i], cudaMemcpyHostToDevice, ctx->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i], ctx->copy_stream);
    }
    const bool head = np && cut[1] - cut[0] >= count_global_head_min();  // the first piece picks the head
    for (size_t i = 0; i < np && e == cudaSuccess; i++) {
        e = cudaStreamWaitEvent(stream, ev[i], 0);
        CountLaunch cl{dt, cut[i], cut[i + 1], g, 0, cs.head, {nullptr, nullptr}, i == 0 ? 0 : (head ? 1 : 2)};
        cl.no_level1 = opts && opts->no_level1 ? 1 : 0;
        if (e == cudaSuccess) e = launch_count_global(cl, stream);
        ctx->launches += count_global_launches(cut[i + 1] - cut[i], i == 0 && head && !cl.no_level1, cs.head != nullptr);
    }
    const uint32_t skip = sort_skip_mask(nbytes / 2 + 1, 0);  // no count exceeds the token bound
    if (e == cudaSuccess) e = finish_table(g, cs.gcap8, cs.gcap, cs.glcap, cs.ss, t->dt, stream, skip);
    ctx->launches += finish_table_launches(cs.ss, skip);
    for (auto x : ev)
        if (x) cudaEventDestroy(x);  // released once their work completes
    ctx->release(cs.mem, cs.bytes, stream);
    if (own) ctx->release(own, std::max<uint64_t>(nbytes, 16), stream);
    table_mark_done(t, stream);
    if (e != cudaSuccess) {
        wc_table_free(t);
        return ctx->cuda_fail(e, "count from host memory");
    }
    *out = t;
    return WC_OK;
}

// ---------------------------------------------------------------- merge / top-k
wc_status wc_merge(wc_ctx *ctx, const wc_table *const *in, uint32_t n, cudaStream_t stream, wc_table **out) {
    if (!ctx || !out || (n && !in)) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    uint64_t sum_cap = 0, sum_lcap = 0, sum_arena = 0, chunks = 0;
    std::vector<MergeSrc> src(n);
    std::vector<uint64_t> cstart(n + 1, 0);
    for (uint32_t i = 0; i < n; i++) {
        if (!in[i]) return ctx->fail(WC_ERR_INVALID_ARG, "null input table");
        const DevTable &d = in[i]->dt;
        src[i] = MergeSrc{d.d_meta, d.khi, d.klo, d.cnt, d.lref, d.loff, d.llen, d.arena, d.count_bits, d.cap,
                          d.arena_cap};
        // a table already waited for gives its sizes, any other its capacities
        const bool known = in[i]->synced && in[i]->sync_status == WC_OK;
        sum_cap += known ? in[i]->n : d.cap;
        sum_lcap += known ? in[i]->nlong : d.lcap;
        sum_arena += known ? in[i]->word_bytes + in[i]->nlong : d.arena_cap;
        cstart[i] = chunks;
        chunks += (d.cap + kMergeChunk - 1) / kMergeChunk;
        cudaStreamWaitEvent(stream, in[i]->done, 0);
    }
    cstart[n] = chunks;
    CapPlan plan;
    plan.cap8 = pow2_at_least(std::max<uint64_t>(1024, 2 * sum_cap));
    plan.cap16 = plan.cap8;
    plan.caplong = pow2_at_least(std::max<uint64_t>(256, 2 * sum_lcap));
    plan.arena = std::max<uint64_t>(4096, sum_arena);
    CountScratch cs;
    wc_status st = scratch_create(ctx, plan, false, stream, cs);
    if (st != WC_OK) return st;
    wc_table *t = nullptr;
    st = table_create(ctx, cs.entries(), plan.caplong, plan.arena, ctx->count_bits, stream, &t);
    if (st != WC_OK) { ctx->release(cs.mem, cs.bytes, stream); return st; }
    void *dsrc = nullptr;
    size_t sb = sizeof(MergeSrc) * std::max<uint32_t>(n, 1) + 8 * (n + 1);
    if ((st = ctx->alloc(&dsrc, sb, stream)) != WC_OK) {
        ctx->release(cs.mem, cs.bytes, stream);
        wc_table_free(t);
        return st;
    }
    std::vector<uint8_t> host(sb);
    memcpy(host.data(), src.data(), sizeof(MergeSrc) * n);
    memcpy(host.data() + sizeof(MergeSrc) * std::max<uint32_t>(n, 1), cstart.data(), 8 * (n + 1));
    // pageable source: the call returns once the bytes are staged, so `host` may go
    cudaError_t e = cudaMemcpyAsync(dsrc, host.data(), sb, cudaMemcpyHostToDevice, stream);
    const GTable g = cs.gtable(t->dt.d_status);
    if (e == cudaSuccess)
        e = launch_merge_insert(static_cast<MergeSrc *>(dsrc),
                                reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(dsrc) + sizeof(MergeSrc) * std::max<uint32_t>(n, 1)),
                                n, chunks, g, stream);
    ctx->launches += chunks ? 1 : 0;
    ctx->prof_mark(ctx->ev_finish, stream);
    if (e == cudaSuccess) e = finish_table(g, cs.gcap8, cs.gcap, cs.glcap, cs.ss, t->dt, stream);
    ctx->prof_mark(ctx->ev_finish, stream);
    ctx->launches += finish_table_launches(cs.ss);
    ctx->release(dsrc, sb, stream);
    ctx->release(cs.mem, cs.bytes, stream);
    table_mark_done(t, stream);
    if (e != cudaSuccess) {
        wc_table_free(t);
        return ctx->cuda_fail(e, "merge");
    }
    *out = t;
    return WC_OK;
}

// ---------------------------------------------------------------- streaming count
wc_status wc_count_stream(wc_ctx *ctx, const uint8_t *h_text, uint64_t nbytes, uint64_t chunk_bytes,
                          cudaStream_t stream, wc_table **out) {
    if (!ctx || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h_text && nbytes) return ctx->fail(WC_ERR_INVALID_ARG, "null text");
    if (!chunk_bytes) chunk_bytes = 512ull << 20;
    if (chunk_bytes < (1ull << 20)) return ctx->fail(WC_ERR_INVALID_ARG, "chunk_bytes below 1 MB");
    cudaSetDevice(ctx->device);
    void *buf = nullptr;
    uint64_t bufb = 0;
    wc_table *acc = nullptr;
    wc_status st = WC_OK;
    for (uint64_t lo = 0; st == WC_OK && (lo < nbytes || !acc);) {
        // a chunk ends after a non-letter byte (a word running past it extends it)
        uint64_t hi = std::min(nbytes, lo + chunk_bytes);
        while (hi < nbytes && host_letter(h_text[hi - 1]) && host_letter(h_text[hi])) hi++;
        const uint64_t n = hi - lo;
        if (n + 16 > bufb) {
            if (buf) ctx->release(buf, bufb, stream);
            buf = nullptr;
            bufb = std::max<uint64_t>(n, chunk_bytes) + 16;
            if ((st = ctx->alloc(&buf, bufb, stream)) != WC_OK) {
                bufb = 0;
                break;
            }
        }
        // the chunk's table, counted again with larger capacities on overflow
        wc_count_opts o{0, 0, 0};
        wc_table *t = nullptr;
        for (int attempt = 0;; attempt++) {
            st = wc_count_host(ctx, n ? h_text + lo : nullptr, n, static_cast<uint8_t *>(buf), 0,
                               attempt ? &o : nullptr, stream, &t);
            if (st == WC_OK) st = wc_table_status(t);
            if (st != WC_ERR_CAPACITY || attempt == 4) break;
            wc_table_free(t);
            t = nullptr;
            if (!attempt) o = wc_count_opts{std::max<uint64_t>(1024, n / 4), std::max<uint64_t>(256, n / 64),
                                            std::max<uint64_t>(4096, n / 8)};
            o.table_slots *= 4;
            o.long_slots *= 4;
            o.arena_bytes *= 4;
        }
        if (st != WC_OK) {
            if (t) wc_table_free(t);
            break;
        }
        if (!acc) {
            acc = t;
        } else {  // the running total plus this chunk (both freed once the merge has read them)
            const wc_table *pair[2] = {acc, t};
            wc_table *m = nullptr;
            st = wc_merge(ctx, pair, 2, stream, &m);
            if (st == WC_OK) st = wc_table_status(m);
            wc_table_free(acc);
            wc_table_free(t);
            acc = st == WC_OK ? m : nullptr;
            if (st != WC_OK && m) wc_table_free(m);
        }
        lo = hi;
        if (!nbytes) break;
    }
    if (buf) ctx->release(buf, bufb, stream);
    if (st != WC_OK) {
        if (acc) wc_table_free(acc);
        return st;
    }
    *out = acc;
    return WC_OK;
}

wc_status wc_topk(wc_ctx *ctx, const wc_table *in, uint32_t k, cudaStream_t stream, wc_table **out) {
    if (!ctx || !in || !out) return WC_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    const DevTable &d = in->dt;
    uint64_t cap = std::max<uint64_t>(1, std::min<uint64_t>(k, d.cap));
    wc_table *t = nullptr;
    wc_status st = table_create(ctx, cap, std::max<uint64_t>(1, d.lcap), std::max<uint64_t>(16, d.arena_cap),
                                d.count_bits, stream, &t);
    if (st != WC_OK) return st;
    cudaStreamWaitEvent(stream, in->done, 0);
    cudaError_t e = launch_topk_copy(d, k, t->dt, stream);
    ctx->launches += 1;
    table_mark_done(t, stream);
    if (e != cudaSuccess) {
        wc_table_free(t);
        return ctx->cuda_fail(e, "topk");
    }
    *out = t;
    return WC_OK;
}
