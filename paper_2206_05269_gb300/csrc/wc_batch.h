// Batched counting: device-side argument blocks shared by the kernels and
// the host code.
#pragma once
#include "wc_internal.h"

namespace wc {

// One unit of work: a whole document (kind 0) or a byte range of a large
// document (kind 1).  lo/hi are offsets into the text; words that start in
// [lo, hi) belong to the item.
struct DocItem {
    unsigned long long lo, hi;
    uint32_t doc;
    uint32_t kind;
};

struct BatchArgs {
    const uint8_t *text;
    const unsigned long long *doc_off;   // [ndocs + 1] device offsets
    uint32_t ndocs;
    const DocItem *items;
    uint32_t nitems;
    uint32_t *next_item;                 // work-queue cursor (zeroed before the launch)
    GTable g;                            // (document, word) tables for ranges and spills
    unsigned long long *out_khi, *out_klo;
    uint32_t *out_cnt, *out_lref;
    unsigned long long out_cap;
    unsigned long long *doc_start;
    uint32_t *doc_n, *doc_flags;
    unsigned long long *loff, *llen;
    uint8_t *arena;
    unsigned long long lcap, arena_cap;
    unsigned long long *meta;            // [0] entries, [1] long words, [2] arena bytes
    uint32_t *status;
};

// Template shapes of the per-document kernel (threads, log2 shared slots).
struct DocShape {
    int block, logc1;
};
extern const DocShape kDocShapes[];
extern const int kNumDocShapes;

// dependent: launched as a programmatic dependent of the previous size
// class's kernel in the stream (independent work; it waits for that kernel
// only at its end).
cudaError_t launch_docs(const BatchArgs &a, int shape, cudaStream_t s, bool dependent = false);
cudaError_t launch_segmented_finish(const BatchArgs &a, const GTable &g, uint64_t cap8, uint64_t cap16,
                                    uint64_t caplong, SortScratch &ss, unsigned long long *smeta, cudaStream_t s,
                                    uint32_t skip = 0);
int segmented_finish_launches(uint64_t cap, uint32_t skip = 0);

}  // namespace wc
