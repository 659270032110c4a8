// Host-side object layouts behind the opaque C-ABI handles.
#pragma once
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/wc.h"
#include "wc_internal.h"

struct wc_ctx {
    int device = 0;
    int sms = 1;
    uint64_t budget = 0;
    std::atomic<uint64_t> used{0};   // device bytes the context holds (pool allocations not yet released)
    std::atomic<uint64_t> peak{0};   // the largest `used` since creation or the last wc_mem_usage reset
    int count_bits = 64;
    int autotune = 0;
    std::string tune_cache_path;
    cudaMemPool_t pool = nullptr;
    cudaStream_t copy_stream = nullptr;  // host -> device copies of wc_count_host (created on first use)
    std::string last_error;
    // stage tracing
    bool profile = false;
    std::vector<cudaEvent_t> ev_head, ev_count, ev_finish;  // (start, stop) pairs
    uint64_t launches = 0;
    void prof_mark(std::vector<cudaEvent_t> &v, cudaStream_t s);
    cudaEvent_t prof_event(std::vector<cudaEvent_t> &v);  // a new event kept in v (not yet recorded), or null
    // per-document kernel shapes picked by the autotuner (indices into kDocShapes)
    int tuned_small = 1, tuned_medium = 3, tuned_large = 4;
    bool tuned = false;  // shapes known (from the cache, or timed by a plan of this context)
    std::string gpu_name;
    void tune_load();
    void tune_save() const;
    // distinct words seen by the last synced single-document count (capacity hints)
    uint64_t hist_bytes = 0, hist_n8 = 0, hist_n16 = 0, hist_nlong = 0, hist_arena = 0;

    // pinned host slots that receive each table's metadata and status by an
    // asynchronous copy when its work completes, so that reading them waits
    // for that table only, not for work enqueued after it
    static constexpr int kMetaSlots = 4096, kMetaSlotBytes = 128;
    uint8_t *meta_host = nullptr;
    std::vector<int> meta_free;
    std::mutex meta_mu;
    int meta_take();          // a free slot, or -1 (then tables read their metadata synchronously)
    void meta_give(int slot);

    wc_status fail(wc_status s, const char *what);
    wc_status cuda_fail(cudaError_t e, const char *what);
    wc_status alloc(void **p, size_t bytes, cudaStream_t s);
    void release(void *p, size_t bytes, cudaStream_t s);
};

struct wc_table {
    wc_ctx *ctx = nullptr;
    const void *owner = nullptr;   // non-null: a view owned by a batch
    void *mem = nullptr;
    size_t bytes = 0;
    wc::DevTable dt{};
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // filled by table_sync
    bool synced = false;
    wc_status sync_status = WC_OK;
    uint64_t n = 0, nlong = 0, tokens = 0, word_bytes = 0;
    uint32_t status_bits = 0;
    uint64_t src_bytes = 0;  // input size of a single-document count (capacity hints)
    int meta_slot = -1;      // pinned slot of wc_ctx::meta_host, or -1
};

// Hash tables and sort scratch of one count or merge.
struct CountScratch {
    void *mem = nullptr;
    size_t bytes = 0;
    uint64_t gcap8 = 0, gcap = 0, glcap = 0;
    wc::G8Slot *slots8 = nullptr;
    wc::GSlot *slots = nullptr;
    wc::LSlot *lslots = nullptr;
    void *head = nullptr;
    wc::SortScratch ss{};
    wc::GTable gtable(uint32_t *status) const {
        return wc::GTable{slots, gcap - 1, lslots, glcap - 1, status, slots8, gcap8 - 1};
    }
    uint64_t entries() const { return gcap8 + gcap + glcap; }
};

// Capacities of one count.
struct CapPlan {
    uint64_t cap8, cap16, caplong, arena;
};

wc_status table_create(wc_ctx *ctx, uint64_t cap, uint64_t lcap, uint64_t arena, int bits, cudaStream_t s,
                       wc_table **out);
void table_mark_done(wc_table *t, cudaStream_t s);
wc_status table_sync(const wc_table *t);
CapPlan plan_capacity(const wc_ctx *ctx, uint64_t nbytes, const wc_count_opts *o);
wc_status scratch_create(wc_ctx *ctx, const CapPlan &p, bool head, cudaStream_t s, CountScratch &cs);
