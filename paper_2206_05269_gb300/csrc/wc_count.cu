// Map + level-1 reduce: the fused tokenise-and-count kernel.
//
// The paper maps on the CPU (Sec. 3.1: remove punctuation, lowercase, split,
// one dictionary per document) and reduces on the GPU (Sec. 3.3); its
// conclusion (Sec. 5.2) asks for a GPU dictionary so the whole map and reduce
// run on the device.  This file is that design for one document:
//
//  0. Head selection (texts of 16 MB or more): a sampling pass counts 64
//     evenly spaced 64 KB pieces into a small table; the most frequent
//     words of at most 8 letters are placed in a bucketised two-choice hash
//     image (4 keys per bucket, a key lives in one of two buckets).
//  1. One persistent 512-thread block per SM copies that image into shared
//     memory (keys read-only, counts zeroed) and walks its chunks through a
//     ring of four buffers.  Each chunk window (16 bytes before, 64 after,
//     16-byte aligned in absolute address space) is staged by a TMA bulk
//     copy that completes a "full" mbarrier; windows that touch the
//     document's edges are staged by plain loads with the outside masked to
//     spaces (a document edge separates words).  Warps never wait for each
//     other: each warp releases a buffer when its words there are consumed,
//     and the last warp to release it issues the copy of the chunk four
//     places ahead.
//  2. A warp classifies 512-byte strips: one 16-bit letter mask per lane
//     (SWAR), word starts = letter & !previous letter, the previous byte
//     carried across lanes, strips and chunks; a word belongs to the chunk
//     holding its first byte and is read through the window's lookahead.
//  3. Words of <= 16 letters are queued per warp and processed 32 at a time:
//     a word of <= 8 letters in the head image adds 1 to its shared count
//     (fingerprints of two buckets, then the matching key); every other word goes to a per-warp tail queue,
//     flushed 32 at a time into the global 8-byte-key or 16-byte-key table
//     (plain load of the key, fire-and-forget reduction; CAS only the first
//     time a word is seen).
//  4. Words of 17+ letters are queued per warp and inserted 32 at a time,
//     one per lane, into the global long-word table.
//  5. At the end each block adds its head counts into the global table.
#include <algorithm>
#include <mutex>
#include <set>
#include <tuple>

#include "wc_internal.h"

namespace wc {

constexpr int kBlock = 512;           // threads of the main counting kernel
constexpr int kWarps = kBlock / 32;
constexpr int kChunk = kWarps * 512;  // bytes per chunk: one 512-byte strip per warp
// Chunk buffers in flight per block (32 KB per SM).  More stages measured
// slower: shared memory and L1 share one array per SM, and the L1 left over
// holds the lines of the tail inserts' scattered loads in flight.
constexpr int kStages = 4;
constexpr int kLead = 16;             // window bytes before the chunk
constexpr int kWinB = kChunk + 96;    // lead + chunk + 64 lookahead + 16 slack
constexpr int kTokCap = 32 + 256;     // per-warp word queue (< 32 left + <= 256 per strip)
constexpr int kTailCap = 64;          // per-warp tail queue
constexpr int kLongCap = 48;          // per-warp queue of words of 17+ letters (< 16 left + <= 32 per step)
constexpr int kHeadBuckets = 2048;    // 8192 head slots
constexpr int kSamplePieces = 64;
constexpr int kSamplePieceBytes = 65536;
constexpr uint64_t kHeadMinBytes = 16ull << 20;
constexpr unsigned long long kSampleSlots = 1ull << 19;
constexpr int kSampleLocalBits = 13;  // per-block table of the sampling pass (the head area)
static_assert((1u << kSampleLocalBits) <= kHeadBuckets * 4, "sampling table fits the head area");
constexpr uint32_t kHeadSortN = kHeadBuckets * 4;  // >= candidates, a multiple of 1024
constexpr uint32_t kHeadIdxBits = 13;
constexpr uint32_t kHeadCntMax = (1u << (32 - kHeadIdxBits)) - 1u;  // sample counts are clamped here
static_assert(kHeadSortN % 1024 == 0, "head candidates per build thread");

struct Count2Args {
    const uint8_t *text;
    unsigned long long lo, hi;        // document bytes text[lo, hi)
    uintptr_t base_al;                // absolute address of chunk 0 (16-aligned, <= text + lo)
    uint32_t nchunks;
    uint32_t piece_chunks;            // chunks per piece (sampling) or nchunks
    unsigned long long piece_stride;  // bytes between pieces (sampling) or 0
    GTable g;
    const uint8_t *lbegin;            // long-word representatives lie in [lbegin, text + hi)
    const unsigned long long *head;   // head image (nb * 4 keys) or null
    const uint32_t *head_fp;          // its fingerprints (nb words of 4 bytes)
    uint32_t nb;
};

// ---------------------------------------------------------------- TMA + mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Arms `bar` for `bytes` and starts the bulk copy global -> shared.
__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                         unsigned long long policy) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}
// Bounded wait for the phase `parity` of `bar` (at most `polls` polls);
// false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t polls = 1u << 22) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < polls; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---------------------------------------------------------------- staging
__device__ __forceinline__ uint4 spaces16() { return make_uint4(0x20202020u, 0x20202020u, 0x20202020u, 0x20202020u); }

// Plain-load staging of the window at absolute (aligned) address w0: bytes
// outside [vb, ve) become spaces; 16-byte blocks holding no valid byte are
// not read at all.
__device__ __forceinline__ void stage_masked(uint8_t *win, uintptr_t w0, uintptr_t vb, uintptr_t ve) {
    for (int t = threadIdx.x; t < kWinB / 16; t += blockDim.x) {
        uintptr_t a = w0 + 16 * (uintptr_t)t;
        uint4 v = spaces16();
        if (a < ve && a + 16 > vb) {
            v = ld_stream16(reinterpret_cast<const void *>(a));
            if (a < vb || a + 16 > ve) v = mask_outside_doc(v, a, vb, ve);
        }
        *reinterpret_cast<uint4 *>(win + 16 * t) = v;
    }
}

// ---------------------------------------------------------------- keys
// 8 lowercased bytes of win[p, p+len), zero padded (1 <= len <= 8), little endian.
__device__ __forceinline__ unsigned long long load_key8(const uint8_t *win, uint32_t p, uint32_t len) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(win + (p & ~3u));
    const uint32_t sh = (p & 3u) * 8u;
    const uint32_t a0 = w[0], a1 = w[1], a2 = w[2];
    const unsigned long long v = ((unsigned long long)__funnelshift_r(a1, a2, sh) << 32) | __funnelshift_r(a0, a1, sh);
    return (v | 0x2020202020202020ull) & (~0ull >> (64u - 8u * len));
}

__device__ __forceinline__ uint32_t head_bucket(unsigned long long key, unsigned long long mul, uint32_t nb) {
    if (kOneSlot) return 0u;  // test build: one bucket for every head word
    return __umulhi((uint32_t)((key * mul) >> 32), nb);
}
constexpr unsigned long long kHeadMulA = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kHeadMulB = 0xC2B2AE3D27D4EB4Full;

// One-byte fingerprint of a head key (never 0: 0 marks an empty slot), from
// bits of the first bucket hash below the ones that pick the bucket.
__device__ __forceinline__ uint32_t head_fp(unsigned long long key) {
    const uint32_t f = (uint32_t)((key * kHeadMulA) >> 40) & 0xFFu;
    return f ? f : 1u;
}

// Slot of key in the shared head image, or -1 (two buckets of four).  The
// two buckets' fingerprint words (one byte a slot) are read first; only a
// slot whose fingerprint matches has its key read and compared.  Most words
// outside the head stop at the fingerprints, and a word in the head costs
// two 4-byte and one 8-byte shared load.
__device__ __forceinline__ int head_find(const unsigned long long *hkey, const uint32_t *hfp,
                                         unsigned long long key, uint32_t nb) {
    const uint32_t b1 = head_bucket(key, kHeadMulA, nb), b2 = head_bucket(key, kHeadMulB, nb);
    const uint32_t f4 = head_fp(key) * 0x01010101u;
    const uint32_t x1 = hfp[b1] ^ f4, x2 = hfp[b2] ^ f4;  // a zero byte = a matching fingerprint
    // 0x80 in each zero byte (and possibly in bytes above one: those fail the key compare)
    unsigned long long mm = ((unsigned long long)((x2 - 0x01010101u) & ~x2 & 0x80808080u) << 32) |
                            ((x1 - 0x01010101u) & ~x1 & 0x80808080u);
    while (mm) {
        const int bit = __ffsll((long long)mm) - 1;  // 8 * byte + 7
        const uint32_t slot = bit < 32 ? b1 * 4 + (uint32_t)(bit >> 3) : b2 * 4 + (uint32_t)((bit - 32) >> 3);
        if (hkey[slot] == key) return (int)slot;
        mm &= mm - 1;
    }
    return -1;
}

// Run length of the letters at w (w is a letter), capped at `end`: the warp
// scans 32 bytes per step.  All lanes call with the same w.
__device__ __forceinline__ unsigned long long run_length_warp(const uint8_t *w, const uint8_t *end) {
    const int lane = threadIdx.x & 31;
    for (unsigned long long off = 0;; off += 32) {
        const uint8_t *q = w + off + lane;
        uint32_t b = q < end ? *q : 0x20u;
        uint32_t m = __ballot_sync(kFull, !is_letter(b));
        if (m) return off + (unsigned long long)(__ffs(m) - 1);
    }
}

// ---------------------------------------------------------------- kernel
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <bool SAMPLE>
struct Counter2 {
    const Count2Args &a;
    unsigned long long *hkey;  // head image keys (read only) or the sampling table
    uint32_t *hcnt;
    const uint32_t *hfp;       // head fingerprints
    uint4 *tailq;
    uint32_t nslots;
    uint32_t tailn;
    int lane;

    // One queued word per lane (have = lane holds one): a word of <= 8
    // letters found in the head image adds 1 to its shared count; any other
    // word is pushed to the tail queue, which is flushed 32 at a time.
    __device__ __forceinline__ void word(const uint8_t *win, bool have, uint32_t e) {
        bool tail = false;
        uint4 tk = make_uint4(0, 0, 0, 0);
        if (SAMPLE) {
            if (have && (e & 31u) <= 8u) {
                const unsigned long long key = load_key8(win, e >> 5, e & 31u);
                tail = !sample_add(key);
                tk = make_uint4((uint32_t)key, (uint32_t)(key >> 32), 0u, 0u);
            }
            push(tail, tk);
            return;
        }
        const int hs = lookup(win, have, e, tail, tk);
        if (hs >= 0) atomicAdd(hcnt + hs, 1u);
        push(tail, tk);
    }
    // The head slot of a queued word (-1 if none) and, when it is not in the
    // head, the key it goes to the tail queue with.
    __device__ __forceinline__ int lookup(const uint8_t *win, bool have, uint32_t e, bool &tail, uint4 &tk) {
        tail = false;
        tk = make_uint4(0, 0, 0, 0);
        int hs = -1;
        if (have) {
            const uint32_t p = e >> 5, len = e & 31u;
            tail = true;
            // one key load for every length (no divergent paths): a word of
            // <= 8 letters has a zero upper half, and its lower half is its
            // 8-byte key
            tk = load_key16(win, p, len);
            if (len <= 8 && nslots) {
                hs = head_find(hkey, hfp, ((unsigned long long)tk.y << 32) | tk.x, a.nb);
                tail = hs < 0;
            }
        }
        return hs;
    }
    __device__ __forceinline__ void push(bool tail, uint4 tk) {
        const uint32_t tb = __ballot_sync(kFull, tail);
        if (tail) tailq[tailn + __popc(tb & ((1u << lane) - 1u))] = tk;
        tailn += __popc(tb);
        __syncwarp();
        if (tailn >= 32) {
            tailn -= 32;
            const uint4 k = tailq[tailn + lane];
            __syncwarp();
            complete();  // the previous 32: their slot loads have had time to land
            issue(k);
        }
    }
    // Sampling pass: the shared head area is a per-block open-addressing table
    // (keys claimed by CAS), so frequent words cost one shared atomic each
    // instead of a global atomic on one hot slot; false when the probe limit
    // is reached (the word then goes to the global sample table).
    __device__ __forceinline__ bool sample_add(unsigned long long key) {
        uint32_t s = (uint32_t)(hash8(key) >> (64 - kSampleLocalBits));
        for (int probe = 0; probe < 16; probe++) {
            unsigned long long k = hkey[s];
            if (k == 0ull) k = atomicCAS(&hkey[s], 0ull, key);
            if (k == 0ull || k == key) {
                atomicAdd(hcnt + s, 1u);
                return true;
            }
            s = (s + 1u) & ((1u << kSampleLocalBits) - 1u);
        }
        return false;
    }
    __device__ __forceinline__ void insert(uint4 k) {
        if (!SAMPLE) table_insert_key(a.g, k, 1ull);
        else global_insert8(a.g, ((unsigned long long)k.y << 32) | k.x, 1ull);
    }

    // Tail inserts in two halves.  issue() computes the home slot of the key
    // and starts loading the keys stored there and in the next slot (the
    // first two probe positions); complete() (called when the next 32 words
    // are ready, so the loads had time to arrive) finishes the insert.  A
    // matching key is final wherever it was seen (keys are written once and
    // never move), so it gets a fire-and-forget add.  Otherwise the probe
    // resumes with fresh loads at the first position that the early loads did
    // not show holding another key for good: an empty or half-written slot is
    // settled there by the CAS.
    bool pend = false, p16 = false;
    uint4 pk;
    unsigned long long pslot = 0, pv0 = 0, pv1 = 0, pv2 = 0, pv3 = 0;
    __device__ __forceinline__ void issue(uint4 k) {
        pk = k;
        pend = true;
        p16 = !SAMPLE && (k.z | k.w) != 0u;
        if (!p16) {
            const unsigned long long key = ((unsigned long long)k.y << 32) | k.x;
            pslot = hash8(key) >> __clzll((long long)a.g.mask8);
            pv0 = ld_u64(&a.g.slots8[pslot].key);
            pv1 = ld_u64(&a.g.slots8[(pslot + 1) & a.g.mask8].key);
        } else {
            pslot = hash_key(k) & a.g.mask;
            const unsigned long long *kp = reinterpret_cast<const unsigned long long *>(&a.g.slots[pslot].key);
            const unsigned long long *kq =
                reinterpret_cast<const unsigned long long *>(&a.g.slots[(pslot + 1) & a.g.mask].key);
            pv0 = ld_u64(kp);
            pv1 = ld_u64(kp + 1);
            pv2 = ld_u64(kq);
            pv3 = ld_u64(kq + 1);
        }
    }
    __device__ __forceinline__ void complete() {
        if (!pend) return;
        pend = false;
        if (!p16) {
            const unsigned long long key = ((unsigned long long)pk.y << 32) | pk.x, m = a.g.mask8;
            if (pv0 == key) { red_add_u64(&a.g.slots8[pslot].cnt, 1ull); return; }
            if (pv1 == key) { red_add_u64(&a.g.slots8[(pslot + 1) & m].cnt, 1ull); return; }
            const unsigned long long from = pv0 == 0ull ? pslot : (pv1 == 0ull ? pslot + 1 : pslot + 2);
            global_insert8_from(a.g, key, 1ull, from & m);
        } else {
            const unsigned long long k0 = ((unsigned long long)pk.y << 32) | pk.x;
            const unsigned long long k1 = ((unsigned long long)pk.w << 32) | pk.z, m = a.g.mask;
            if (pv0 == k0 && pv1 == k1) { red_add_u64(&a.g.slots[pslot].cnt, 1ull); return; }
            if (pv2 == k0 && pv3 == k1) { red_add_u64(&a.g.slots[(pslot + 1) & m].cnt, 1ull); return; }
            // both halves non-zero: the slot holds another key for good
            const bool other0 = pv0 != 0ull && pv1 != 0ull, other1 = pv2 != 0ull && pv3 != 0ull;
            const unsigned long long from = !other0 ? pslot : (!other1 ? pslot + 1 : pslot + 2);
            global_insert16_from(a.g, pk, 1ull, from & m);
        }
    }
};

template <bool SAMPLE>
struct Ring {
    const Count2Args &a;
    uint8_t *buf;          // kStages x kWinB
    uint64_t *full;        // kStages mbarriers
    uint32_t *done;        // kStages release counters
    uintptr_t vb, ve;
    unsigned long long policy;

    __device__ __forceinline__ uintptr_t win_start(uint32_t c) const {
        uint32_t q = c / a.piece_chunks, r = c % a.piece_chunks;
        return a.base_al + (uintptr_t)q * a.piece_stride + (uintptr_t)r * kChunk - kLead;
    }
    __device__ __forceinline__ bool interior(uintptr_t w0) const { return w0 >= vb && w0 + kWinB <= ve; }

    // The calling warp stages this block's i-th chunk into buffer i % kStages.
    __device__ __forceinline__ void produce(uint32_t i) {
        const uint32_t c = blockIdx.x + i * gridDim.x;
        if (c >= a.nchunks) return;
        const int b = (int)(i % kStages);
        const uintptr_t w0 = win_start(c);
        const int lane = threadIdx.x & 31;
        if (interior(w0)) {
            if (lane == 0) {
                fence_proxy_async();
                tma_load(buf + b * kWinB, reinterpret_cast<const void *>(w0), kWinB, &full[b], policy);
            }
        } else {
            uint8_t *win = buf + b * kWinB;
            for (int t = lane; t < kWinB / 16; t += 32) {
                uintptr_t ad = w0 + 16 * (uintptr_t)t;
                uint4 v = spaces16();
                if (ad < ve && ad + 16 > vb) {
                    v = ld_stream16(reinterpret_cast<const void *>(ad));
                    if (ad < vb || ad + 16 > ve) v = mask_outside_doc(v, ad, vb, ve);
                }
                *reinterpret_cast<uint4 *>(win + 16 * t) = v;
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                mbar_arrive(&full[b]);
            }
        }
        __syncwarp();
    }
    // The calling warp is done with chunk i; the last warp refills the buffer.
    __device__ __forceinline__ void release(uint32_t i) {
        const int b = (int)(i % kStages);
        const int lane = threadIdx.x & 31;
        __syncwarp();
        uint32_t last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&done[b], 1u) == kWarps - 1;
            if (last) done[b] = 0;
        }
        if (__shfl_sync(kFull, last, 0)) produce(i + kStages);
    }
};

template <bool SAMPLE>
__global__ void __launch_bounds__(kBlock, 1) k_count2(Count2Args a) {
    extern __shared__ __align__(128) uint8_t smem[];
    unsigned long long *hkey = reinterpret_cast<unsigned long long *>(smem);        // nb*4
    uint32_t *hcnt = reinterpret_cast<uint32_t *>(hkey + kHeadBuckets * 4);           // nb*4
    uint8_t *ring = reinterpret_cast<uint8_t *>(hcnt + kHeadBuckets * 4);             // kStages x kWinB
    uint32_t *tokall = reinterpret_cast<uint32_t *>(ring + kStages * kWinB);         // warps x kTokCap
    uint4 *tailall = reinterpret_cast<uint4 *>(tokall + kWarps * kTokCap);           // warps x kTailCap
    uint4 *longall = tailall + kWarps * kTailCap;                                     // warps x kLongCap
    uint64_t *full = reinterpret_cast<uint64_t *>(longall + kWarps * kLongCap);     // kStages
    uint32_t *done = reinterpret_cast<uint32_t *>(full + kStages);                   // kStages
    uint32_t *hfp = done + kStages;                                                   // nb
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *tok = tokall + warp * kTokCap;
    uint4 *longq = longall + warp * kLongCap;
    // head image (counting) or an empty local table (sampling)
    const uint32_t nslots = SAMPLE ? (1u << kSampleLocalBits) : (a.head ? a.nb * 4 : 0);
    Counter2<SAMPLE> ctr{a, hkey, hcnt, hfp, tailall + warp * kTailCap, nslots, 0u, lane};

    for (uint32_t i = threadIdx.x; i < nslots; i += kBlock) {
        hkey[i] = SAMPLE ? 0ull : a.head[i];
        hcnt[i] = 0u;
    }
    if (!SAMPLE && nslots)
        for (uint32_t i = threadIdx.x; i < a.nb; i += kBlock) hfp[i] = a.head_fp[i];
    if (threadIdx.x < kStages) done[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kStages; b++) mbar_init(&full[b], 1);
        fence_barrier_init();
    }
    __syncthreads();

    Ring<SAMPLE> rg{a, ring, full, done, reinterpret_cast<uintptr_t>(a.text) + a.lo,
                    reinterpret_cast<uintptr_t>(a.text) + a.hi, policy_evict_first()};
    const uint8_t *begin = reinterpret_cast<const uint8_t *>(rg.vb);
    const uint8_t *end = reinterpret_cast<const uint8_t *>(rg.ve);
    if (warp == 0)
        for (uint32_t i = 0; i < kStages; i++) rg.produce(i);

    uint32_t tcount = 0;   // queued words (warp-uniform)
    uint32_t tprev = 0;    // how many of them belong to the previous chunk
    uint32_t longn = 0;    // queued long words
    bool timed_out = false;
    auto flush_long = [&](uint32_t base, uint32_t n) {
        if ((uint32_t)lane < n) {
            uint4 e = longq[base + lane];
            const uint8_t *w = reinterpret_cast<const uint8_t *>(((unsigned long long)e.y << 32) | e.x);
            unsigned long long len = e.z;
            if (len == 0) {  // longer than the window showed: scan to the end of the run
                len = 17;
                while (w + len < end && is_letter(w[len])) len++;
            }
            long_insert2(a.g, w, len, long_hash(w, len), 1ull, a.lbegin, end);
        }
        __syncwarp();
    };

    uint32_t i = 0;
    for (uint32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x, i++) {
        const int b = (int)(i % kStages);
        if (!mbar_wait(&full[b], (i / kStages) & 1u)) { timed_out = true; break; }
        const uint8_t *win = ring + b * kWinB;
        const uintptr_t w0 = rg.win_start(c);
        // ---- this warp's 512-byte strip
        const int sbase = kLead + 512 * warp;
        const uint32_t prevL = is_letter(win[sbase - 1]) ? 1u : 0u;  // the window holds the byte before
        const uint32_t L = letter_mask16(*reinterpret_cast<const uint4 *>(win + sbase + 16 * lane));
        const uint32_t Ln = letter_mask16(*reinterpret_cast<const uint4 *>(win + sbase + 512));  // first 16 bytes after
        const uint32_t up = __shfl_up_sync(kFull, L, 1);
        const uint32_t dn = __shfl_down_sync(kFull, L, 1);
        const uint32_t pbit = lane == 0 ? prevL : ((up >> 15) & 1u);
        const uint32_t W = L | ((lane == 31 ? Ln : dn) << 16);
        const uint32_t S = L & ~((L << 1) | pbit) & 0xFFFFu;
        uint32_t x = W;
        x &= x >> 1; x &= x >> 2; x &= x >> 4; x &= x >> 8; x &= W >> 16;  // starts of 17+ letter runs
        uint32_t Ss = S & ~x, Sl = S & x;

        const uint32_t c1 = __popc(Ss);
        uint32_t incl = c1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        uint32_t off = tcount + incl - c1;
        const uint32_t pbase = (uint32_t)(sbase + 16 * lane);
        static_assert(kStages <= 8 && (kStages & (kStages - 1)) == 0, "3-bit buffer tag in queued words");
        const uint32_t btag = (uint32_t)b << 19;
        // a warp-uniform trip count: no divergent loop to reconverge
        const uint32_t nmax = __reduce_max_sync(kFull, c1);
        for (uint32_t r = 0; r < nmax; r++) {
            if (Ss) {
                const int j = __ffs(Ss) - 1;
                Ss &= Ss - 1;
                const uint32_t len = (uint32_t)__ffs(~(W >> j)) - 1u;
                tok[off++] = btag | ((pbase + (uint32_t)j) << 5) | len;
            }
        }
        const uint32_t tnew = total;
        tcount += total;
        if (!SAMPLE && __any_sync(kFull, Sl != 0)) {
            // 48 bits of letter mask from this lane on: run lengths up to 32 letters are read here
            const uint32_t Ln2 = letter_mask16(*reinterpret_cast<const uint4 *>(win + sbase + 528));
            const uint32_t dn2 = __shfl_down_sync(kFull, L, 2);
            const unsigned long long W48 =
                (unsigned long long)W | ((unsigned long long)(lane == 31 ? Ln2 : (lane == 30 ? Ln : dn2)) << 32);
            while (__any_sync(kFull, Sl != 0)) {
                const bool act = Sl != 0;
                uint4 e = make_uint4(0, 0, 0, 0);
                if (act) {
                    int j = __ffs(Sl) - 1;
                    Sl &= Sl - 1;
                    unsigned long long wa = (unsigned long long)(w0 + pbase + (uint32_t)j);
                    // letters seen in W48 (< 48 - j), else 0: the run continues past it
                    const uint32_t run = (uint32_t)__ffsll((long long)~(W48 >> j)) - 1u;
                    e = make_uint4((uint32_t)wa, (uint32_t)(wa >> 32), run < 48u - (uint32_t)j ? run : 0u, 0u);
                }
                const uint32_t lb = __ballot_sync(kFull, act);
                if (act) longq[longn + __popc(lb & ((1u << lane) - 1u))] = e;
                longn += __popc(lb);
                __syncwarp();
                if (longn >= 16) {  // insert them all, one per lane, 32 at a time
                    flush_long(0, longn < 32 ? longn : 32);
                    if (longn > 32) flush_long(32, longn - 32);
                    longn = 0;
                }
            }
        }
        __syncwarp();
        // ---- queued words, 32 at a time
        uint32_t bq = 0;
        for (; bq + 32 <= tcount; bq += 32) {
            const uint32_t e = tok[bq + lane];
            ctr.word(ring + ((e >> 19) & (uint32_t)(kStages - 1)) * kWinB, true, e & 0x7FFFFu);
        }
        uint32_t rem = tcount - bq;
        const uint32_t old_left = tprev > bq ? tprev - bq : 0u;
        if (old_left) {  // words of the previous chunk still queued: finish them all now
            const uint32_t e = (uint32_t)lane < rem ? tok[bq + lane] : 0u;
            ctr.word(ring + ((e >> 19) & (uint32_t)(kStages - 1)) * kWinB, (uint32_t)lane < rem, e & 0x7FFFFu);
            rem = 0;
        } else if (bq) {
            uint32_t e = (uint32_t)lane < rem ? tok[bq + lane] : 0u;
            __syncwarp();
            if ((uint32_t)lane < rem) tok[lane] = e;
            __syncwarp();
        }
        tcount = rem;
        tprev = rem < tnew ? rem : tnew;
        if (i > 0) rg.release(i - 1);
    }
    // ---- drain: queued words of the last chunk, then the tail and long queues
    if (!timed_out) {
        const uint32_t e = (uint32_t)lane < tcount ? tok[lane] : 0u;
        ctr.word(ring + ((e >> 19) & (uint32_t)(kStages - 1)) * kWinB, (uint32_t)lane < tcount, e & 0x7FFFFu);
        if (!SAMPLE) {
            flush_long(0, longn < 32 ? longn : 32);
            if (longn > 32) flush_long(32, longn - 32);
        }
        ctr.complete();
        if ((uint32_t)lane < ctr.tailn) ctr.insert(ctr.tailq[lane]);
        __syncwarp();
    }
    if (__syncthreads_or(timed_out)) {
        if (threadIdx.x == 0) {
            atomicOr(a.g.status, ST_TIMEOUT);
            for (int b = 0; b < kStages; b++) mbar_wait(&full[b], 0u);  // bounded: let copies in flight land
        }
        return;
    }
    for (uint32_t k = threadIdx.x; k < nslots; k += kBlock)
        if (hcnt[k]) global_insert8(a.g, hkey[k], (unsigned long long)hcnt[k]);
}

constexpr size_t kCountSmem = (size_t)kHeadBuckets * 4 * 8 + (size_t)kHeadBuckets * 4 * 4 + kStages * (size_t)kWinB +
                              (size_t)kWarps * kTokCap * 4 + (size_t)kWarps * kTailCap * 16 +
                              (size_t)kWarps * kLongCap * 16 + kStages * 8 + kStages * 4 + (size_t)kHeadBuckets * 4;
static_assert(kCountSmem <= 227 * 1024, "counting kernel shared memory");

// ---------------------------------------------------------------- head selection
// Histogram of sample counts (clamped to 4095).
__global__ void k_head_hist(const G8Slot *s, unsigned long long cap, uint32_t *hist) {
    __shared__ uint32_t h[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long c = s[i].cnt;
        if (s[i].key && c >= 2) atomicAdd(&h[c > 4095 ? 4095 : c], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Smallest count threshold t >= 2 that keeps at most kmax words: suffix sums
// of the histogram (one block of 1024 threads, 4 bins each).
__global__ void __launch_bounds__(1024) k_head_threshold(const uint32_t *hist, uint32_t kmax, uint32_t *meta) {
    __shared__ uint32_t part[1024];
    __shared__ uint32_t best;
    const uint32_t t = threadIdx.x;
    // bins of thread t, from high counts down: 4095-4t .. 4092-4t
    uint32_t v[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int c = 4095 - 4 * (int)t - j;
        v[j] = c >= 2 ? hist[c] : 0u;
        s += v[j];
    }
    part[t] = s;
    if (t == 0) best = 4096;
    __syncthreads();
    for (int w = 1; w < 1024; w <<= 1) {  // inclusive prefix over threads = suffix over counts
        uint32_t x = t >= (uint32_t)w ? part[t - w] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    uint32_t acc = part[t] - s;  // words with a count above this thread's bins
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int c = 4095 - 4 * (int)t - j;
        acc += v[j];
        if (c >= 2 && acc <= kmax) atomicMin(&best, (uint32_t)c);
    }
    __syncthreads();
    if (t == 0) {
        meta[0] = best;  // threshold
        meta[1] = 0;     // candidates
    }
}

__global__ void k_head_collect(const G8Slot *s, unsigned long long cap, uint32_t *meta, unsigned long long *cand,
                               uint32_t *ccnt, uint32_t kmax) {
    const uint32_t t = meta[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long c = s[i].cnt;
        if (s[i].key && c >= t) {
            uint32_t k = atomicAdd(&meta[1], 1u);
            if (k < kmax) {
                cand[k] = s[i].key;
                ccnt[k] = c < kHeadCntMax ? (uint32_t)c : kHeadCntMax;
            }
        }
    }
}

// Two-choice placement of the candidates into nb buckets of 4 (one block),
// most frequent first: candidates are placed in tiers of equal floor(log2
// sample count), highest tier first, all candidates of a tier in parallel.
// A key whose two buckets are both full is left out of the head and counted
// in the global table.  Placing by frequency makes sure that only the rarest
// candidates can be left out: a frequent word missing from the head would
// send all its occurrences to one global slot, whose atomics then serialise.
__global__ void __launch_bounds__(1024) k_head_build(const unsigned long long *cand, const uint32_t *ccnt,
                                                     const uint32_t *meta, uint32_t kmax, uint32_t nb,
                                                     unsigned long long *image, uint32_t *image_fp) {
    constexpr int kPer = (int)(kHeadSortN / 1024);  // candidates per thread
    __shared__ uint32_t fill[kHeadBuckets];
    __shared__ uint32_t fps[kHeadBuckets];
    const uint32_t n = meta[1] < kmax ? meta[1] : kmax;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        fill[i] = 0;
        fps[i] = 0;
    }
    for (uint32_t i = threadIdx.x; i < nb * 4; i += blockDim.x) image[i] = 0ull;
    int tier[kPer];
    unsigned long long key[kPer];
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        const uint32_t i = threadIdx.x + (uint32_t)k * 1024u;
        tier[k] = i < n ? 31 - __clz((int)ccnt[i]) : -1;  // counts >= 2: tier >= 1
        key[k] = i < n ? cand[i] : 0ull;
    }
    __syncthreads();
    for (int t = 31 - kHeadIdxBits; t >= 1; t--) {
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            if (tier[k] != t) continue;
            const uint32_t b1 = head_bucket(key[k], kHeadMulA, nb), b2 = head_bucket(key[k], kHeadMulB, nb);
            const uint32_t first = fill[b1] <= fill[b2] ? b1 : b2, second = first == b1 ? b2 : b1;
            uint32_t slot = atomicAdd(&fill[first], 1u), bk = first;
            if (slot >= 4) {
                slot = atomicAdd(&fill[second], 1u);
                bk = second;
            }
            if (slot < 4) {
                image[bk * 4 + slot] = key[k];
                atomicOr(&fps[bk], head_fp(key[k]) << (8 * slot));
            }
        }
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) image_fp[i] = fps[i];
}

size_t head_scratch_bytes() {
    return (size_t)kSampleSlots * sizeof(G8Slot) + 4096 * 4 + 64 + (size_t)kHeadBuckets * 4 * (8 * 2 + 4) +
           (size_t)kHeadBuckets * 4 + 1024;
}

static int sm_count_dev() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int count_global_launches(uint64_t nbytes, bool head) {
    return (nbytes >= kHeadMinBytes && head) ? 6 : (nbytes ? 1 : 0);
}

cudaError_t ensure_smem_limit(const void *func, int bytes) {
    static std::mutex mu;
    static std::set<std::tuple<const void *, int, int>> done;  // (kernel, device, bytes)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(func, dev, bytes);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

cudaError_t launch_count_global(const CountLaunch &c, cudaStream_t s) {
    cudaError_t ea = ensure_smem_limit((const void *)k_count2<false>, (int)kCountSmem);
    if (ea == cudaSuccess) ea = ensure_smem_limit((const void *)k_count2<true>, (int)kCountSmem);
    if (ea != cudaSuccess) return ea;
    if (c.hi <= c.lo) return cudaSuccess;
    const int sms = sm_count_dev();
    const uintptr_t tb = reinterpret_cast<uintptr_t>(c.text);
    Count2Args a;
    a.text = c.text;
    a.lo = c.lo;
    a.hi = c.hi;
    a.base_al = (tb + c.lo) & ~(uintptr_t)15;
    const unsigned long long span = tb + c.hi - a.base_al;
    a.nchunks = (uint32_t)((span + kChunk - 1) / kChunk);
    a.piece_chunks = a.nchunks;
    a.piece_stride = 0;
    a.g = c.g;
    a.lbegin = c.text;
    a.head = nullptr;
    a.head_fp = nullptr;
    a.nb = kHeadBuckets;
    const uint64_t n = c.hi - c.lo;
    if (c.head_mode == 1 && c.head_scratch) {  // the head an earlier launch built
        uint8_t *p = static_cast<uint8_t *>(c.head_scratch);
        unsigned long long *cand =
            reinterpret_cast<unsigned long long *>(p + kSampleSlots * sizeof(G8Slot) + 4096 * 4 + 64);
        unsigned long long *image = cand + kHeadBuckets * 4;
        a.head = image;
        a.head_fp = reinterpret_cast<uint32_t *>(image + kHeadBuckets * 4) + kHeadBuckets * 4;
    } else if (c.head_mode == 0 && n >= kHeadMinBytes && c.head_scratch) {
        // sampling pass into its own small 8-byte-key table
        uint8_t *p = static_cast<uint8_t *>(c.head_scratch);
        G8Slot *sample = reinterpret_cast<G8Slot *>(p);
        uint32_t *hist = reinterpret_cast<uint32_t *>(p + kSampleSlots * sizeof(G8Slot));
        uint32_t *meta = hist + 4096;
        unsigned long long *cand = reinterpret_cast<unsigned long long *>(meta + 16);
        unsigned long long *image = cand + kHeadBuckets * 4;
        uint32_t *ccnt = reinterpret_cast<uint32_t *>(image + kHeadBuckets * 4);
        uint32_t *image_fp = ccnt + kHeadBuckets * 4;
        cudaMemsetAsync(p, 0, kSampleSlots * sizeof(G8Slot) + 4096 * 4 + 64, s);
        Count2Args sa = a;
        sa.g.slots8 = sample;
        sa.g.mask8 = kSampleSlots - 1;
        const uint32_t pc = kSamplePieceBytes / kChunk;
        sa.piece_chunks = pc;
        sa.piece_stride = (span / kSamplePieces) & ~(unsigned long long)15;
        sa.nchunks = pc * kSamplePieces;
        int g = (int)std::min<uint32_t>(sa.nchunks, (uint32_t)sms);
        k_count2<true><<<g, kBlock, kCountSmem, s>>>(sa);
        const uint32_t kmax = kHeadBuckets * 4 * 88 / 100;
        k_head_hist<<<sms, 256, 0, s>>>(sample, kSampleSlots, hist);
        k_head_threshold<<<1, 1024, 0, s>>>(hist, kmax, meta);
        k_head_collect<<<sms * 2, 256, 0, s>>>(sample, kSampleSlots, meta, cand, ccnt, kmax);
        k_head_build<<<1, 1024, 0, s>>>(cand, ccnt, meta, kmax, kHeadBuckets, image, image_fp);
        a.head = image;
        a.head_fp = image_fp;
    }
    int grid = c.grid > 0 ? c.grid : sms;
    if ((uint32_t)grid > a.nchunks) grid = (int)a.nchunks;
    for (cudaEvent_t e : c.main_ev)
        if (e) cudaEventRecord(e, s);
    k_count2<false><<<grid, kBlock, kCountSmem, s>>>(a);
    return cudaGetLastError();
}

int count_global_chunk_bytes() { return kChunk; }
uint64_t count_global_head_min() { return kHeadMinBytes; }

// ---------------------------------------------------------------- wait self-test
// The counting kernel's bounded wait, on a barrier expecting one arrival:
// with `arrive` thread 0 makes it first and the wait succeeds; without, no
// one does, the wait gives up after `polls` polls and the timeout is recorded
// in *status as the counting kernel records it.  Nothing else waits, so the
// block always finishes.
__global__ void k_wait_selftest(uint32_t *status, uint32_t polls, int arrive) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) mbar_arrive(&bar);
        if (!mbar_wait(&bar, 0u, polls)) atomicOr(status, ST_TIMEOUT);
    }
}

cudaError_t launch_wait_selftest(uint32_t *d_status, uint32_t polls, int arrive, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(d_status, polls, arrive);
    return cudaGetLastError();
}

}  // namespace wc
