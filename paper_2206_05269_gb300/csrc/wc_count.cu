// Map + level-1 reduce: the fused tokenise-and-count kernel.
//
// The paper maps on the CPU (Sec. 3.1: remove punctuation, lowercase, split,
// one dictionary per document) and reduces on the GPU (Sec. 3.3); its
// conclusion (Sec. 5.2) asks for a GPU dictionary so the whole map and reduce
// run on the device.  This file is that design for one document.
//
// Work split.  The document is cut into 512-byte strips (16-byte aligned in
// absolute address space).  Every warp of the grid owns every
// (grid x warps)-th strip and stages its strips through a private ring of
// four buffers: a strip's window (16 bytes before it, the strip, 32 bytes
// after it) arrives by one TMA bulk copy that completes an mbarrier of that
// warp; windows touching the document's edges are loaded by the warp with
// plain loads and the outside masked to spaces (a document edge separates
// words).  No warp ever waits for another.
//
// Per strip a lane classifies 16 bytes (SWAR letter mask); word starts are
// letters whose previous byte is not one (carried across lanes, and from the
// window's lead byte across strips); a word belongs to the strip holding its
// first byte and is read through the window's lookahead.  Starts of words of
// at most 16 letters go to a per-warp queue (window position and length) and
// are processed 32 at a time, one per lane (with a HEAD table, two batches of
// 32 at once, their lookups interleaved):
//   * level 1 (shared memory): a word of at most 8 letters is looked up in
//     the block's table of 8,192 keys and, if there, its shared count is
//     incremented.  Two table kinds:
//       HEAD  (texts of 16 MB or more): a read-only image of the words a
//             sampling pass found most frequent, placed by hash-and-displace
//             (one displacement byte per bucket of keys), so a lookup is one
//             displacement load and one key compare;
//       LOCAL (smaller texts, and the sampling pass itself): an empty table
//             whose slots words claim by 64-bit CAS as they come (linear
//             probing, at most four probes).
//   * level 2 (global memory): every other word goes to a per-warp tail
//     queue of 16-byte keys, flushed 32 at a time into the global 8-byte-key
//     or 16-byte-key open-addressing table (slot loads issued one flush
//     ahead, fire-and-forget reductions, CAS only for a word's first claim).
// Words of 17+ letters are queued by address and, with head scratch (texts
// of 16 MB or more), appended to a global queue that k_long_deferred drains
// after this kernel; otherwise (or when that queue is full) they are inserted
// 32 at a time here.  Either way into the global long-word table, bytes
// compared, never only hashes.  At the end each block adds its nonzero
// level-1 counts into the global table.
#include <algorithm>
#include <cstddef>
#include <mutex>
#include <set>
#include <tuple>

#include "wc_internal.h"

namespace wc {

constexpr int kWarps = 20;                // warps of the counting kernel, each with its own ring
constexpr int kBlock = kWarps * 32;
constexpr int kStrip = 512;               // bytes a warp classifies per step (16 per lane)
constexpr int kLead = 16;                 // window bytes before the strip (the previous byte, aligned)
constexpr int kWinB = kLead + kStrip + 32;  // + 32 lookahead: 560 bytes, a multiple of 16
constexpr int kStages = 4;                // ring buffers per warp
constexpr int kTokCap = 32 + 256;         // queued words: < 32 left over + at most 256 starts a strip
constexpr int kTailCap = 64;
constexpr int kLongCap = 48;              // < 16 left over + at most 32 starts a step
constexpr int kHeadSlots = 8192;          // level-1 table keys
constexpr int kHeadBuckets = 2048;        // hash-and-displace buckets of the HEAD image
constexpr int kLocalProbes = 4;
constexpr int kSamplePieces = 32;
constexpr int kSamplePieceBytes = 65536;
constexpr uint64_t kHeadMinBytes = 16ull << 20;
constexpr unsigned long long kSampleSlots = 1ull << 19;
constexpr int kHeadRegions = 16;          // the image is placed region by region, one warp each
constexpr int kRegionSlots = kHeadSlots / kHeadRegions;
constexpr uint32_t kHeadMax = kHeadSlots * 80 / 100;  // head candidates (load factor of the image)
constexpr uint32_t kHotMax = 512;                     // candidates placed first (the sample's most frequent)
constexpr unsigned long long kLongQCap = 1ull << 21;  // deferred long words per launch
static_assert(kWinB % 16 == 0, "TMA bulk copies move multiples of 16 bytes");
static_assert(kStages == 4, "2-bit stage tag in queued words");

enum : int { MODE_HEAD = 0, MODE_LOCAL = 1, MODE_SAMPLE = 2 };

struct Count2Args {
    const uint8_t *text;
    unsigned long long lo, hi;        // document bytes text[lo, hi)
    uintptr_t base_al;                // absolute address of strip 0 (16-aligned, <= text + lo)
    unsigned long long nstrips;
    uint32_t piece_strips;            // strips per piece (sampling) or 0 (contiguous)
    unsigned long long piece_stride;  // bytes between pieces (sampling)
    GTable g;
    const uint8_t *lbegin;            // long-word representatives lie in [lbegin, text + hi)
    const unsigned long long *head;   // HEAD image: kHeadSlots keys
    const uint8_t *head_disp;         // HEAD image: kHeadBuckets displacements
    unsigned long long *lq;           // deferred long words (kLongQCap entries), or null: inserted in place
    unsigned long long *lqn;          // entries appended to lq (may pass kLongQCap: the rest were inserted in place)
    int l1_off;                       // LOCAL: no level-1 table (every word to the global tables)
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
// Arms `bar` for `bytes` and starts the bulk copy global -> shared.  Both
// addresses are 16-byte aligned and bytes is a multiple of 16.
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
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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

__device__ __forceinline__ uint4 spaces16() { return make_uint4(0x20202020u, 0x20202020u, 0x20202020u, 0x20202020u); }

// ---------------------------------------------------------------- level-1 tables
// Both table kinds hold kHeadSlots 8-byte keys (words of at most 8 letters,
// lowercased, zero padded; never 0) and 32-bit counts.  One block's counts
// stay below 2^32: a block reads at most 2^40 / 128 bytes (texts are under
// 2^40 bytes and grids have at least 128 blocks), so it sees fewer than 2^32
// words.
//
// Level-1 hash of an 8-byte key: the high letters folded onto the low bits,
// times an odd constant, so that every bit of the product depends on every
// letter.
__device__ __forceinline__ unsigned long long l1_mix(unsigned long long key) {
    if (kOneSlot) return 0ull;  // test build: one home slot, one bucket
    return (key ^ (key >> 29)) * 0xBF58476D1CE4E5B9ull;
}
// HEAD image (hash and displace): a key's bucket is the top 11 bits of its
// hash and its region the bucket's low 4 bits; every key of a bucket is
// placed in its region at base + d * step (mod 512) for the bucket's one
// displacement d, with base and odd step taken from other bits of the hash,
// so the slots of one key for d = 0, 1, ... are all distinct.
static_assert(kHeadSlots == 8192 && kHeadBuckets == 2048 && kRegionSlots == 512, "hash bit fields below");
__device__ __forceinline__ uint32_t head_bucket(unsigned long long h) { return (uint32_t)(h >> 53); }
__device__ __forceinline__ uint32_t head_slot(unsigned long long h, uint32_t d) {
    const uint32_t base = (uint32_t)(h >> 32), step = ((uint32_t)h >> 12) | 1u;
    return ((head_bucket(h) & (uint32_t)(kHeadRegions - 1)) << 9) | ((base + d * step) & (uint32_t)(kRegionSlots - 1));
}
// LOCAL table: home slot = the top 13 bits of the hash.
__device__ __forceinline__ uint32_t local_home(unsigned long long h) { return (uint32_t)(h >> 51); }

// The LOCAL slot holding `key`, claiming the first empty slot on its probe
// path by 64-bit CAS; -1 after kLocalProbes occupied slots of other keys.
// Keys are written once (CAS from 0) and never move, so a load that sees a
// non-zero key sees that slot's final key.
__device__ __forceinline__ int local_slot(unsigned long long *skey, unsigned long long key) {
    uint32_t s = local_home(l1_mix(key));
#pragma unroll 1
    for (int p = 0; p < kLocalProbes; p++) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(&skey[s]);
        if (k == 0ull) k = atomicCAS(&skey[s], 0ull, key);
        if (k == 0ull || k == key) return (int)s;
        s = (s + 1u) & (uint32_t)(kHeadSlots - 1);
    }
    return -1;
}

// ---------------------------------------------------------------- keys
__device__ __forceinline__ unsigned long long key_lo(uint4 k) { return ((unsigned long long)k.y << 32) | k.x; }
// 16 lowercased bytes of the word win[p, p + len) (len <= 16), zero padded:
// a word of at most 8 letters has a zero upper half, and its lower half is
// its 8-byte key.  mask[len] keeps the low len bytes; lowercasing and masking
// take one three-input logic operation per word.  Reads win[p & ~3, +20).
__device__ __forceinline__ uint4 window_key16(const uint8_t *win, uint32_t p, uint32_t len, const uint4 *mask) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(win + (p & ~3u));
    const uint32_t sh = (p & 3u) * 8u;
    const uint32_t a0 = w[0], a1 = w[1], a2 = w[2], a3 = w[3], a4 = w[4];
    const uint4 m = mask[len];
    return make_uint4((__funnelshift_r(a0, a1, sh) | 0x20202020u) & m.x, (__funnelshift_r(a1, a2, sh) | 0x20202020u) & m.y,
                      (__funnelshift_r(a2, a3, sh) | 0x20202020u) & m.z, (__funnelshift_r(a3, a4, sh) | 0x20202020u) & m.w);
}

// ---------------------------------------------------------------- level 2
// Per-warp tail inserts, 32 words at a time (one per lane), as a state
// machine that never waits for a dependent round trip inside a flush.  A
// lane takes a word from the tail queue, computes its home slot and starts
// loading the first 16 bytes of that slot and of the next one; at the next
// flush (when the next 32 tail words are ready, so the loads had time to
// land) it advances one step:
//   * the key is in one of the two slots: a fire-and-forget add, done;
//   * else the first of them not holding another key for good is empty (or,
//     for 16-byte keys, half written): a CAS claims it, and its result is
//     checked at the following flush (the word is done if the CAS won or
//     found the same key, else probing resumes after that slot);
//   * both slots hold other keys: loads of the next two slots are started.
// Keys are written once and never move, so a key seen in a slot is final.
// Both key sizes take the same path: the table (8-byte slots of 16 bytes,
// 16-byte slots of 32 bytes) is chosen by address arithmetic, the slot hash
// is shared, and a 16-byte load covers either slot's key (for an 8-byte slot,
// key and count; the count is ignored).  Only the claim differs (64- or
// 128-bit CAS); claims are rare.  Lanes still busy keep their word across
// flushes; free lanes take new words.
static_assert(sizeof(G8Slot) == 16 && offsetof(G8Slot, cnt) == 8, "8-byte slot layout");
static_assert(sizeof(GSlot) == 32 && offsetof(GSlot, cnt) == 16, "16-byte slot layout");
template <int MODE>
struct Tail {
    const GTable &g;
    uint32_t st = 0;  // 0 free, 1 loads in flight, 2 CAS in flight
    bool p16 = false;
    uint32_t probes = 0;
    unsigned long long k0 = 0, k1 = 0;  // key halves (k1 = 0 for 8-byte keys)
    unsigned long long pslot = 0;
    uint4 v0, v1;  // slots pslot and pslot + 1 (first 16 bytes), or the CAS result in v0

    __device__ __forceinline__ explicit Tail(const GTable &gt) : g(gt) {}

    __device__ __forceinline__ uint8_t *tab() const {
        return p16 ? reinterpret_cast<uint8_t *>(g.slots) : reinterpret_cast<uint8_t *>(g.slots8);
    }
    __device__ __forceinline__ unsigned long long msk() const { return p16 ? g.mask : g.mask8; }
    __device__ __forceinline__ uint32_t shf() const { return p16 ? 5u : 4u; }

    __device__ __forceinline__ void load() {
        uint8_t *t = tab();
        v0 = ld_relaxed_v2(t + (pslot << shf()));
        v1 = ld_relaxed_v2(t + (((pslot + 1) & msk()) << shf()));
        st = 1;
    }
    __device__ __forceinline__ void take(uint4 k) {
        k0 = key_lo(k);
        k1 = ((unsigned long long)k.w << 32) | k.z;
        p16 = MODE != MODE_SAMPLE && k1 != 0ull;
        pslot = hash_slot(k0, k1) >> __clzll((long long)msk());
        probes = 0;
        load();
    }
    __device__ __forceinline__ void add_at(unsigned long long s) {
        red_add_u64(reinterpret_cast<unsigned long long *>(tab() + (s << shf()) + (p16 ? 16u : 8u)), 1ull);
        st = 0;
    }
    __device__ __forceinline__ void claim(unsigned long long s) {
        pslot = s;
        if (!p16) {
            const unsigned long long old = atomicCAS(&g.slots8[s].key, 0ull, k0);
            v0 = make_uint4((uint32_t)old, (uint32_t)(old >> 32), 0u, 0u);
        } else {
            const uint4 want = make_uint4((uint32_t)k0, (uint32_t)(k0 >> 32), (uint32_t)k1, (uint32_t)(k1 >> 32));
            v0 = cas128_global(&g.slots[s].key, make_uint4(0u, 0u, 0u, 0u), want);
        }
        st = 2;
    }
    __device__ __forceinline__ void next(unsigned long long from) {
        probes += 2;
        if (probes >= (uint32_t)kGlobalProbeLimit) {  // the table is full: reported, the word dropped
            atomicOr(g.status, ST_TABLE_FULL);
            st = 0;
            return;
        }
        pslot = from & msk();
        load();
    }
    // One step of a busy lane with what its last step fetched.
    __device__ __forceinline__ void step() {
        const unsigned long long m = msk();
        const unsigned long long a0 = key_lo(v0), a1 = ((unsigned long long)v0.w << 32) | v0.z;
        if (st == 2) {  // the CAS result (an 8-byte claim left a1 = 0 = k1)
            const bool mine = (a0 == 0ull && a1 == 0ull) || (a0 == k0 && a1 == k1);
            if (mine) add_at(pslot);
            else next(pslot + 1);
            return;
        }
        const unsigned long long b0 = key_lo(v1), b1 = ((unsigned long long)v1.w << 32) | v1.z;
        // an 8-byte slot's second word is its count: only 16-byte keys compare it
        const bool m0 = a0 == k0 && (!p16 || a1 == k1), m1 = b0 == k0 && (!p16 || b1 == k1);
        if (m0 || m1) { add_at(m0 ? pslot : ((pslot + 1) & m)); return; }
        // a 16-byte slot with both halves non-zero holds another key for good
        const bool e0 = a0 == 0ull || (p16 && a1 == 0ull), e1 = b0 == 0ull || (p16 && b1 == 0ull);
        if (e0 || e1) { claim(e0 ? pslot : ((pslot + 1) & m)); return; }
        next(pslot + 2);
    }
    // One flush round: busy lanes step, free lanes take words from the end of
    // the queue (tailn, warp-uniform, is updated).
    __device__ __forceinline__ void round(const uint4 *tailq, uint32_t &tailn, int lane) {
        if (st) step();
        const uint32_t freem = __ballot_sync(kFull, st == 0u);
        const uint32_t nf = __popc(freem);
        const uint32_t tk = nf < tailn ? nf : tailn;
        const uint32_t r = __popc(freem & ((1u << lane) - 1u));
        if (st == 0u && r < tk) take(tailq[tailn - tk + r]);
        tailn -= tk;
        __syncwarp();
    }
};

// ---------------------------------------------------------------- kernel
constexpr size_t kSmemKeys = (size_t)kHeadSlots * 8;
constexpr size_t kSmemCnts = (size_t)kHeadSlots * 4;
constexpr size_t kSmemDisp = (size_t)kHeadBuckets;
constexpr size_t kSmemRing = (size_t)kWarps * kStages * kWinB;
constexpr size_t kSmemTok = (size_t)kWarps * kTokCap * 4;
constexpr size_t kSmemTail = (size_t)kWarps * kTailCap * 16;
constexpr size_t kSmemLong = (size_t)kWarps * kLongCap * 8;
constexpr size_t kSmemBars = (size_t)kWarps * kStages * 8;
constexpr size_t kCountSmem = kSmemKeys + kSmemCnts + kSmemDisp + kSmemRing + kSmemTok + kSmemTail + kSmemLong + kSmemBars;
static_assert((kSmemKeys + kSmemCnts + kSmemDisp) % 16 == 0 && kSmemRing % 16 == 0 && kSmemTok % 16 == 0,
              "16-byte aligned ring buffers and queues");
static_assert(kCountSmem <= 227 * 1024, "counting kernel shared memory");
// Measured: the dynamic shared memory plus the static 384 bytes and the 1 KB
// the SM reserves per block must stay within the 196 KB shared-memory
// carveout.  The next carveout (228 KB) leaves 28 KB of L1 instead of 60 KB,
// and the tail's global loads then miss L1 (a 10 KB larger tail queue made
// the kernel 29 % slower).
static_assert(kCountSmem + 384 + 1024 <= 196 * 1024, "keep the 196 KB shared-memory carveout");

template <int MODE>
__global__ void __launch_bounds__(kBlock, 1) k_count3(Count2Args a) {
    extern __shared__ __align__(128) uint8_t smem[];
    // an ordinary launch (measured: as a dependent of the head kernels, with
    // its blocks scheduled early, the kernel ran about 1 % slower); no early
    // trigger, so the deferred long-word kernel launches as its blocks exit
    grid_dependency_wait();
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *scnt = reinterpret_cast<uint32_t *>(smem + kSmemKeys);
    uint8_t *sdisp = smem + kSmemKeys + kSmemCnts;
    uint8_t *ring_all = sdisp + kSmemDisp;
    uint32_t *tok_all = reinterpret_cast<uint32_t *>(ring_all + kSmemRing);
    uint4 *tail_all = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(tok_all) + kSmemTok);
    unsigned long long *long_all = reinterpret_cast<unsigned long long *>(reinterpret_cast<uint8_t *>(tail_all) + kSmemTail);
    uint64_t *bar_all = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(long_all) + kSmemLong);

    __shared__ uint4 kmask[17];  // kmask[n]: the low n bytes of 16 kept
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *ring = ring_all + (size_t)warp * kStages * kWinB;
    uint64_t *full = bar_all + warp * kStages;
    uint32_t *tok = tok_all + warp * kTokCap;
    uint4 *tailq = tail_all + warp * kTailCap;
    unsigned long long *longq = long_all + warp * kLongCap;

    for (int i = threadIdx.x; i < kHeadSlots; i += kBlock) {
        skey[i] = MODE == MODE_HEAD ? a.head[i] : 0ull;
        scnt[i] = 0u;
    }
    if (MODE == MODE_HEAD)
        for (int i = threadIdx.x; i < kHeadBuckets; i += kBlock) sdisp[i] = a.head_disp[i];
    if (threadIdx.x <= 16) {
        const int n = threadIdx.x;
        kmask[n] = make_uint4(byte_keep_mask(n), byte_keep_mask(n - 4), byte_keep_mask(n - 8), byte_keep_mask(n - 12));
    }
    if (lane == 0) {
        for (int b = 0; b < kStages; b++) mbar_init(&full[b], 1);
        fence_barrier_init();
    }
    __syncthreads();

    const uintptr_t vb = reinterpret_cast<uintptr_t>(a.text) + a.lo, ve = reinterpret_cast<uintptr_t>(a.text) + a.hi;
    const uint8_t *end = reinterpret_cast<const uint8_t *>(ve);
    const unsigned long long policy = policy_evict_first();
    // this warp's strips: s0, s0 + stride, ...
    const unsigned long long stride = (unsigned long long)gridDim.x * kWarps;
    const unsigned long long s0 = (unsigned long long)blockIdx.x * kWarps + (unsigned long long)warp;
    const unsigned long long nk = s0 < a.nstrips ? (a.nstrips - s0 + stride - 1) / stride : 0ull;

    auto win_start = [&](unsigned long long k) -> uintptr_t {
        const unsigned long long s = s0 + k * stride;
        if (a.piece_strips == 0u) return a.base_al + (uintptr_t)(s * kStrip) - kLead;
        const unsigned long long q = s / a.piece_strips, r = s % a.piece_strips;
        return a.base_al + (uintptr_t)(q * a.piece_stride + r * kStrip) - kLead;
    };
    // Stages this warp's k-th strip into ring buffer k % kStages (strips are
    // produced in order; `issued` is one past the last one).
    unsigned long long issued = 0;
    auto produce = [&](unsigned long long k) {
        if (k >= nk) return;
        issued = k + 1;
        const int b = (int)(k % kStages);
        uint8_t *win = ring + b * kWinB;
        const uintptr_t w0 = win_start(k);
        if (w0 >= vb && w0 + kWinB <= ve) {
            if (lane == 0) {
                fence_proxy_async();
                tma_load(win, reinterpret_cast<const void *>(w0), kWinB, &full[b], policy);
            }
        } else {  // a document edge: plain loads, the outside read as spaces
            for (int t = lane; t < kWinB / 16; t += 32) {
                const uintptr_t ad = w0 + 16 * (uintptr_t)t;
                uint4 v = spaces16();
                if (ad < ve && ad + 16 > vb) {
                    v = ld_stream16(reinterpret_cast<const void *>(ad));
                    if (ad < vb || ad + 16 > ve) v = mask_outside_doc(v, ad, vb, ve);
                }
                *reinterpret_cast<uint4 *>(win + 16 * t) = v;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[b]);
        }
        __syncwarp();
    };

    Tail<MODE> tl(a.g);
    uint32_t tailn = 0;
    // One queued word per lane (have: this lane holds one).
    auto process = [&](uint32_t e, bool have) {
        bool tail = false;
        uint4 tk = make_uint4(0u, 0u, 0u, 0u);
        if (have) {
            const uint32_t len = e & 31u, p = (e >> 5) & 0x3FFu;
            const uint8_t *w = ring + (e >> 27) * kWinB;
            // one key load for every length (no divergent paths)
            tk = window_key16(w, p, len, kmask);
            tail = true;
            if (len <= 8u && (MODE != MODE_LOCAL || !a.l1_off)) {
                const unsigned long long key = key_lo(tk);
                int s;
                if (MODE == MODE_HEAD) {
                    const unsigned long long h = l1_mix(key);
                    const uint32_t hs = head_slot(h, sdisp[head_bucket(h)]);
                    s = skey[hs] == key ? (int)hs : -1;
                } else {
                    s = local_slot(skey, key);
                }
                if (s >= 0) {
                    atomicAdd(&scnt[s], 1u);
                    tail = false;
                }
            } else if (MODE == MODE_SAMPLE) {
                tail = false;  // the sampling pass looks for frequent words of <= 8 letters only
            }
        }
        const uint32_t tb = __ballot_sync(kFull, tail);
        if (tail) tailq[tailn + __popc(tb & ((1u << lane) - 1u))] = tk;
        tailn += __popc(tb);
        __syncwarp();
        // flush: the lanes' previous words advance (their loads have had time
        // to land), free lanes take new ones; the queue ends below 32 words
        while (tailn >= 32) tl.round(tailq, tailn, lane);
    };
    // HEAD mode, two full batches of queued words: the two words' head
    // lookups are independent, so they run interleaved (every load issued
    // before the compares; a word of more than 8 letters never hits), then
    // each batch's misses are queued and flushed as process does.
    auto push_tail = [&](bool tail, uint4 tk) {
        const uint32_t tb = __ballot_sync(kFull, tail);
        if (tail) tailq[tailn + __popc(tb & ((1u << lane) - 1u))] = tk;
        tailn += __popc(tb);
        __syncwarp();
        while (tailn >= 32) tl.round(tailq, tailn, lane);
    };
    auto process2 = [&](uint32_t e0, uint32_t e1) {
        const uint32_t n0 = e0 & 31u, n1 = e1 & 31u;
        const uint4 k0 = window_key16(ring + (e0 >> 27) * kWinB, (e0 >> 5) & 0x3FFu, n0, kmask);
        const uint4 k1 = window_key16(ring + (e1 >> 27) * kWinB, (e1 >> 5) & 0x3FFu, n1, kmask);
        const unsigned long long y0 = key_lo(k0), y1 = key_lo(k1);
        const unsigned long long h0 = l1_mix(y0), h1 = l1_mix(y1);
        const uint32_t s0 = head_slot(h0, sdisp[head_bucket(h0)]), s1 = head_slot(h1, sdisp[head_bucket(h1)]);
        const unsigned long long v0 = skey[s0], v1 = skey[s1];
        const bool hit0 = n0 <= 8u && v0 == y0, hit1 = n1 <= 8u && v1 == y1;
        if (hit0) atomicAdd(&scnt[s0], 1u);
        if (hit1) atomicAdd(&scnt[s1], 1u);
        push_tail(!hit0, k0);
        push_tail(!hit1, k1);
    };

    // Words of 17+ letters: (address << 16 | run length, or 0 when the window
    // did not show the run's end).  With a deferred queue they are appended to
    // it (one atomic a flush) and inserted by k_long_deferred after this
    // kernel, so the warp never waits on their table round trips; entries the
    // queue cannot hold, or all of them without a queue, are inserted here,
    // one per lane.
    uint32_t longn = 0;
    auto flush_long = [&](uint32_t base, uint32_t n) {
        unsigned long long qb = kLongQCap;
        if (a.lq) {
            if (lane == 0) qb = atomicAdd(a.lqn, (unsigned long long)n);
            qb = __shfl_sync(kFull, qb, 0);
        }
        if ((uint32_t)lane < n && qb + (unsigned long long)lane < kLongQCap) {
            a.lq[qb + lane] = longq[base + lane];
        } else if ((uint32_t)lane < n) {
            const unsigned long long e = longq[base + lane];
            const uint8_t *w = reinterpret_cast<const uint8_t *>(e >> 16);
            unsigned long long len = e & 0xFFFFull;
            if (len == 0) {  // longer than the window showed: scan to the end of the run
                len = 17;
                while (w + len < end && is_letter(w[len])) len++;
            }
            uint4 fl[2];
            long_ends(w, len, fl[0], fl[1]);
            long_insert2(a.g, w, len, long_hash_mix(fl[0], fl[1], len), 1ull, a.lbegin, end, fl);
        }
        __syncwarp();
    };

    for (unsigned long long k = 0; k < kStages; k++) produce(k);

    uint32_t tcount = 0;  // queued words (warp-uniform)
    uint32_t tprev = 0;   // how many of them belong to the previous strip
    unsigned long long k = 0;
    bool timed_out = false;
    for (; k < nk; k++) {
        const int b = (int)(k % kStages);
        if (!mbar_wait(&full[b], (uint32_t)(k / kStages) & 1u)) { timed_out = true; break; }
        const uint8_t *win = ring + b * kWinB;
        // ---- classify this lane's 16 bytes
        const uint32_t L = letter_mask16(*reinterpret_cast<const uint4 *>(win + kLead + 16 * lane));
        // the 32 lookahead bytes after the strip, one per lane, as one mask
        const uint32_t A = __ballot_sync(kFull, is_letter(win[kLead + kStrip + lane]));
        const uint32_t prevL = is_letter(win[kLead - 1]) ? 1u : 0u;
        const uint32_t up = __shfl_up_sync(kFull, L, 1);
        const uint32_t dn = __shfl_down_sync(kFull, L, 1);
        const uint32_t pbit = lane == 0 ? prevL : ((up >> 15) & 1u);
        const uint32_t W = L | ((lane == 31 ? (A & 0xFFFFu) : dn) << 16);  // this lane's and the next 16 bytes
        const uint32_t S = L & ~((L << 1) | pbit) & 0xFFFFu;                // word starts
        uint32_t x = W;
        x &= x >> 1; x &= x >> 2; x &= x >> 4; x &= x >> 8; x &= W >> 16;  // starts of 17+ letter runs
        uint32_t Ss = S & ~x, Sl = S & x;
        const uint32_t E = W & ~(W >> 1);  // last letters of runs (bits 0..30 are exact)

        const uint32_t c1 = __popc(Ss);
        uint32_t incl = c1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        // this lane's c1 queue slots are [lo, hi): each step takes its highest
        // start into the top and its lowest into the bottom (two independent
        // chains; queue order does not matter)
        uint32_t lo = tcount + incl - c1, hi = tcount + incl;
        const uint32_t tag = ((uint32_t)b << 27) | ((uint32_t)(kLead + 16 * lane) << 5);
        const uint32_t nmax = (__reduce_max_sync(kFull, c1) + 1u) >> 1;  // a warp-uniform trip count
        for (uint32_t r = 0; r < nmax; r++) {
            if (Ss) {
                const uint32_t j = 31u - (uint32_t)__clz(Ss), i = (uint32_t)__ffs(Ss) - 1u;
                Ss &= ~((1u << j) | (1u << i));
                // a short word ends within the 32 bits
                tok[--hi] = tag + (j << 5) + (uint32_t)__ffs(E >> j);
                if (i != j) tok[lo++] = tag + (i << 5) + (uint32_t)__ffs(E >> i);
            }
        }
        tcount += total;
        if (MODE != MODE_SAMPLE && __any_sync(kFull, Sl != 0)) {
            // 48 bits of letter mask from this lane on: runs shorter than 48 - j are measured here
            const uint32_t dn2 = __shfl_down_sync(kFull, L, 2);
            const uint32_t third = lane == 31 ? (A >> 16) : (lane == 30 ? (A & 0xFFFFu) : dn2);
            const unsigned long long W48 = (unsigned long long)W | ((unsigned long long)third << 32);
            const uintptr_t lbase = win_start(k) + kLead + 16 * (uintptr_t)lane;
            while (__any_sync(kFull, Sl != 0)) {
                const bool act = Sl != 0;
                unsigned long long e = 0;
                if (act) {
                    const int j = __ffs(Sl) - 1;
                    Sl &= Sl - 1;
                    const uint32_t run = (uint32_t)__ffsll((long long)~(W48 >> j)) - 1u;
                    e = ((unsigned long long)(lbase + (uintptr_t)j) << 16) | (run < 48u - (uint32_t)j ? run : 0u);
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
        if (MODE == MODE_HEAD)
            for (; bq + 64 <= tcount; bq += 64) process2(tok[bq + lane], tok[bq + 32 + lane]);
        for (; bq + 32 <= tcount; bq += 32) process(tok[bq + lane], true);
        uint32_t rem = tcount - bq;
        if (tprev > bq) {  // words of the previous strip still queued: finish them all now
            const uint32_t e = (uint32_t)lane < rem ? tok[bq + lane] : 0u;
            process(e, (uint32_t)lane < rem);
            rem = 0;
        } else if (bq) {
            const uint32_t e = (uint32_t)lane < rem ? tok[bq + lane] : 0u;
            __syncwarp();
            if ((uint32_t)lane < rem) tok[lane] = e;
            __syncwarp();
        }
        tcount = rem;
        tprev = rem;
        // the previous strip's buffer holds no queued word any more: refill it
        if (k > 0) produce(k - 1 + kStages);
    }
    // ---- drain: the last strip's queued words, then the long and tail queues
    if (!timed_out) {
        const uint32_t e = (uint32_t)lane < tcount ? tok[lane] : 0u;
        process(e, (uint32_t)lane < tcount);
        if (MODE != MODE_SAMPLE) {
            flush_long(0, longn < 32 ? longn : 32);
            if (longn > 32) flush_long(32, longn - 32);
        }
        while (tailn > 0 || __any_sync(kFull, tl.st != 0u)) tl.round(tailq, tailn, lane);
    }
    if (__syncthreads_or(timed_out)) {
        if (lane == 0) {
            if (timed_out) atomicOr(a.g.status, ST_TIMEOUT);
            // let this warp's copies in flight land before the block exits
            // (bounded): strips k .. issued - 1 were staged but not waited for
            for (unsigned long long j = k; j < issued; j++)
                mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
        }
        return;
    }
    for (int i = threadIdx.x; i < kHeadSlots; i += kBlock)
        if (scnt[i]) global_insert8(a.g, skey[i], (unsigned long long)scnt[i]);
}

// Inserts the long words k_count3 queued (Count2Args::lq).  A block takes
// chunks of kDefChunk queued words, one a thread: each thread computes its
// word's ends and hash, and the chunk's words of at most 32 letters are
// counted in a shared table first.  Two queued words are the same word
// exactly when hash, length and first and last 16 letters agree, since those
// cover every letter.  The thread that claimed a word's shared slot then makes
// its one global insert, carrying the chunk count, so a frequent long word
// costs one table update per chunk instead of one per occurrence.  Words of
// more than 32 letters are inserted one by one (the insert compares bytes).
constexpr int kDefChunk = 512;  // = threads per block (two blocks per SM)
constexpr int kDefSlots = 2 * kDefChunk;
constexpr size_t kDefSmem = (size_t)kDefChunk * (16 + 16 + 8 + 8 + 4) + (size_t)kDefSlots * 8;
__global__ void __launch_bounds__(kDefChunk) k_long_deferred(const unsigned long long *lq,
                                                             const unsigned long long *lqn, GTable g,
                                                             const uint8_t *lbegin, const uint8_t *end) {
    extern __shared__ __align__(16) uint8_t dsm[];
    grid_dependency_wait();  // the counting kernel's queue
    grid_dependency_trigger();
    uint4 *ef = reinterpret_cast<uint4 *>(dsm);
    uint4 *el = ef + kDefChunk;
    unsigned long long *eh = reinterpret_cast<unsigned long long *>(el + kDefChunk);
    unsigned long long *ea = eh + kDefChunk;
    uint32_t *elen = reinterpret_cast<uint32_t *>(ea + kDefChunk);
    uint32_t *tidx = elen + kDefChunk;  // 1 + entry index, 0 = empty
    uint32_t *tcnt = tidx + kDefSlots;
    const unsigned long long n = *lqn < kLongQCap ? *lqn : kLongQCap;
    const int i = threadIdx.x;
    for (unsigned long long c0 = (unsigned long long)blockIdx.x * kDefChunk; c0 < n;
         c0 += (unsigned long long)gridDim.x * kDefChunk) {
        tidx[i] = 0u;
        tidx[i + kDefChunk] = 0u;
        tcnt[i] = 0u;
        tcnt[i + kDefChunk] = 0u;
        uint32_t mylen = 0;
        if (c0 + i < n) {
            const unsigned long long e = lq[c0 + i];
            const uint8_t *w = reinterpret_cast<const uint8_t *>(e >> 16);
            unsigned long long len = e & 0xFFFFull;
            if (len == 0) {  // longer than the window showed: scan to the end of the run
                len = 17;
                while (w + len < end && is_letter(w[len])) len++;
            }
            uint4 fl[2];
            long_ends(w, len, fl[0], fl[1]);
            const unsigned long long h = long_hash_mix(fl[0], fl[1], len);
            if (len > 32) {
                long_insert2(g, w, len, h, 1ull, lbegin, end, fl);
            } else {
                ef[i] = fl[0];
                el[i] = fl[1];
                eh[i] = h;
                ea[i] = (unsigned long long)reinterpret_cast<uintptr_t>(w);
                mylen = (uint32_t)len;
            }
        }
        elen[i] = mylen;
        __syncthreads();
        // count the chunk's words in the shared table (at most half full)
        int mine = -1;  // the slot this thread claimed
        if (mylen) {
            uint32_t sl = (uint32_t)(eh[i] >> 40) & (uint32_t)(kDefSlots - 1);
            for (int probe = 0; probe < kDefSlots; probe++) {
                uint32_t cur = tidx[sl];
                if (cur == 0u) cur = atomicCAS(&tidx[sl], 0u, (uint32_t)i + 1u);
                const uint32_t j = cur ? cur - 1u : (uint32_t)i;
                if (j == (uint32_t)i || (eh[j] == eh[i] && elen[j] == mylen && key_eq(ef[j], ef[i]) &&
                                         key_eq(el[j], el[i]))) {
                    if (j == (uint32_t)i) mine = (int)sl;
                    atomicAdd(&tcnt[sl], 1u);
                    break;
                }
                sl = (sl + 1u) & (uint32_t)(kDefSlots - 1);
            }
        }
        __syncthreads();
        if (mine >= 0) {  // the word's one global insert, with its count in the chunk
            const uint4 fl[2] = {ef[i], el[i]};
            long_insert2(g, reinterpret_cast<const uint8_t *>(ea[i]), mylen, eh[i], tcnt[mine], lbegin, end, fl);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- head selection
// Histogram of sample counts (clamped to 4095).
__global__ void k_head_hist(const G8Slot *s, unsigned long long cap, uint32_t *hist) {
    __shared__ uint32_t h[4096];
    grid_dependency_wait();
    grid_dependency_trigger();
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
    __shared__ uint32_t best, hot;
    grid_dependency_wait();
    grid_dependency_trigger();
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
    if (t == 0) {
        best = 4096;
        hot = 4096;
    }
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
        if (c >= 2 && acc <= kHotMax) atomicMin(&hot, (uint32_t)c);
    }
    __syncthreads();
    if (t == 0) {
        meta[0] = best;  // threshold
        meta[1] = 0;     // candidates
        meta[2] = hot;   // the sample count from which a candidate is placed first
    }
}

__global__ void k_head_collect(const G8Slot *s, unsigned long long cap, uint32_t *meta, unsigned long long *cand,
                               uint32_t *ccnt, uint32_t kmax) {
    grid_dependency_wait();
    grid_dependency_trigger();
    const uint32_t t = meta[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long c = s[i].cnt;
        if (s[i].key && c >= t) {
            uint32_t k = atomicAdd(&meta[1], 1u);
            if (k < kmax) {
                cand[k] = s[i].key;
                ccnt[k] = c < 0xFFFFFFFFull ? (uint32_t)c : 0xFFFFFFFFu;
            }
        }
    }
}

// Places the head candidates into the HEAD image by hash and displace.  The
// image's regions of 512 slots are independent (a key's region is fixed by
// its bucket), so block r builds region r alone: its eight warps pick out
// the candidates whose bucket lies in the region and group them by bucket,
// and its first warp places the buckets in two passes, first those holding one of the sample's
// kHotMax most frequent words (the region is then nearly empty, so they
// always find room), then the rest, each pass largest bucket first.  A bucket
// of at most 8 keys tries 32 displacements at once, one per lane: a lane's
// displacement qualifies when its keys land on distinct slots that the
// region's occupancy bitmap shows free, and the lowest qualifying lane takes
// it.  Larger buckets try one displacement at a time, one key per lane.  A
// bucket with no displacement in 0..255, or with more than 32 keys, is left
// out (as are candidates beyond the region's 512 slots): their words are then
// counted in the global table, never wrongly, because a lookup always
// compares the whole key.  Empty slots keep key 0, which no word has.
constexpr int kRegionBuckets = kHeadBuckets / kHeadRegions;  // 128
static_assert(kRegionBuckets == 128, "four buckets a lane");

template <int S>
__device__ __forceinline__ bool chd_place_small(const unsigned long long *bk, uint32_t *used, unsigned long long *rimage,
                                                uint8_t *disp, uint32_t lane) {
    unsigned long long key[S], h[S];
#pragma unroll
    for (int i = 0; i < S; i++) {
        key[i] = bk[i];
        h[i] = l1_mix(key[i]);
    }
    for (uint32_t dbase = 0; dbase < 256; dbase += 32) {
        const uint32_t d = dbase + lane;
        uint32_t slot[S];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < S; i++) {
            slot[i] = head_slot(h[i], d) & (uint32_t)(kRegionSlots - 1);
            ok = ok && !((used[slot[i] >> 5] >> (slot[i] & 31u)) & 1u);
#pragma unroll
            for (int j = 0; j < i; j++) ok = ok && slot[j] != slot[i];
        }
        const uint32_t win = __ballot_sync(kFull, ok);
        if (win) {
            if ((int)lane == __ffs(win) - 1) {  // the region is this warp's alone
#pragma unroll
                for (int i = 0; i < S; i++) {
                    used[slot[i] >> 5] |= 1u << (slot[i] & 31u);
                    rimage[slot[i]] = key[i];
                }
                *disp = (uint8_t)d;
            }
            __syncwarp();
            return true;
        }
    }
    return false;
}

constexpr int kChdThreads = 256;
__global__ void __launch_bounds__(kChdThreads) k_head_chd(const unsigned long long *cand, const uint32_t *ccnt,
                                                          const uint32_t *meta, unsigned long long *image,
                                                          uint8_t *disp) {
    __shared__ unsigned long long sel[kRegionSlots], rkey[kRegionSlots], rimage[kRegionSlots];
    grid_dependency_wait();
    grid_dependency_trigger();
    __shared__ uint32_t selb[kRegionSlots];  // local bucket, bit 31: hot
    __shared__ uint32_t bsize[kRegionBuckets], bstart[kRegionBuckets], bfill[kRegionBuckets];
    __shared__ uint32_t used[kRegionSlots / 32];
    __shared__ uint8_t sdisp[kRegionBuckets];
    __shared__ uint32_t nsel_sh;
    constexpr uint32_t kHot = 1u << 31;
    const uint32_t r = blockIdx.x, t = threadIdx.x, lane = t & 31;
    const uint32_t n = meta[1] < kHeadMax ? meta[1] : kHeadMax, hot_min = meta[2];
    for (uint32_t i = t; i < kRegionBuckets; i += kChdThreads) {
        bsize[i] = 0;
        bfill[i] = 0;
        sdisp[i] = 0;
    }
    for (uint32_t i = t; i < kRegionSlots; i += kChdThreads) rimage[i] = 0ull;
    if (t < kRegionSlots / 32) used[t] = 0;
    if (t == 0) nsel_sh = 0;
    __syncthreads();
    // ---- this region's candidates (in any order), every thread a share
    for (uint32_t i = t; i < n; i += kChdThreads) {
        const unsigned long long key = cand[i];
        const uint32_t g = head_bucket(l1_mix(key));
        if ((g & (uint32_t)(kHeadRegions - 1)) == r) {
            const uint32_t pos = atomicAdd(&nsel_sh, 1u);
            if (pos < (uint32_t)kRegionSlots) {
                sel[pos] = key;
                selb[pos] = (g / kHeadRegions) | (ccnt[i] >= hot_min ? kHot : 0u);
            }
        }
    }
    __syncthreads();
    const uint32_t nsel = nsel_sh < (uint32_t)kRegionSlots ? nsel_sh : (uint32_t)kRegionSlots;
    for (uint32_t j = t; j < nsel; j += kChdThreads) {
        const uint32_t lb = selb[j] & ~kHot;
        atomicAdd(&bsize[lb], 1u);
        if (selb[j] & kHot) atomicOr(&bsize[lb], kHot);
    }
    __syncthreads();
    if (t >= 32) return;  // grouping and placement: the first warp alone (warp barriers only)
    // bucket starts: four buckets a lane, then a shuffle scan
    uint32_t own = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) own += bsize[lane * 4 + q] & 0xFFFFu;
    uint32_t incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += x;
    }
    uint32_t run = incl - own;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        bstart[lane * 4 + q] = run;
        run += bsize[lane * 4 + q] & 0xFFFFu;
    }
    __syncwarp();
    for (uint32_t j = lane; j < nsel; j += 32) {
        const uint32_t lb = selb[j] & ~kHot;
        rkey[bstart[lb] + atomicAdd(&bfill[lb], 1u)] = sel[j];
    }
    __syncwarp();
    uint32_t maxsize = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) maxsize = max(maxsize, bsize[lane * 4 + q] & 0xFFFFu);
    maxsize = __reduce_max_sync(kFull, maxsize);
    // ---- placement
    for (int pass = 0; pass < 2; pass++) {
        for (uint32_t size = maxsize < 32u ? maxsize : 32u; size >= 1; size--) {
            for (uint32_t i0 = 0; i0 < (uint32_t)kRegionBuckets; i0 += 32) {
                const uint32_t bs = bsize[i0 + lane];
                uint32_t todo = __ballot_sync(kFull, (bs & 0xFFFFu) == size && ((bs & kHot) != 0) == (pass == 0));
                while (todo) {
                    const uint32_t lb = i0 + (uint32_t)(__ffs(todo) - 1);
                    todo &= todo - 1;
                    const unsigned long long *bk = rkey + bstart[lb];
                    switch (size) {  // warp-uniform
                    case 1: chd_place_small<1>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 2: chd_place_small<2>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 3: chd_place_small<3>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 4: chd_place_small<4>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 5: chd_place_small<5>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 6: chd_place_small<6>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 7: chd_place_small<7>(bk, used, rimage, &sdisp[lb], lane); continue;
                    case 8: chd_place_small<8>(bk, used, rimage, &sdisp[lb], lane); continue;
                    default: break;
                    }
                    const bool mine = lane < size;
                    const unsigned long long key = mine ? bk[lane] : 0ull;
                    const unsigned long long h = l1_mix(key);
                    for (uint32_t d = 0; d < 256; d++) {
                        // dummy slots of idle lanes never clash; every lane takes part in the match
                        const uint32_t slot = mine ? (head_slot(h, d) & (uint32_t)(kRegionSlots - 1)) : 1024u + lane;
                        const uint32_t peers = __match_any_sync(kFull, slot);
                        const bool ok = (!mine || !((used[slot >> 5] >> (slot & 31u)) & 1u)) && peers == (1u << lane);
                        if (!__all_sync(kFull, ok)) continue;
                        if (mine) {
                            atomicOr(&used[slot >> 5], 1u << (slot & 31u));  // lanes may share a bitmap word
                            rimage[slot] = key;
                        }
                        if (lane == 0) sdisp[lb] = (uint8_t)d;
                        __syncwarp();
                        break;
                    }
                }
            }
        }
    }
    __syncwarp();
    for (uint32_t i = lane; i < kRegionSlots; i += 32) image[r * kRegionSlots + i] = rimage[i];
    for (uint32_t i = lane; i < (uint32_t)kRegionBuckets; i += 32) disp[r + kHeadRegions * i] = sdisp[i];
}

// ---------------------------------------------------------------- launch
// Head scratch: the sample table, its histogram and metadata (the deferred
// long-word count at byte 32), the candidates and the HEAD image (keys, then
// displacements), then the deferred long-word queue.
constexpr size_t kHsSample = (size_t)kSampleSlots * sizeof(G8Slot);
constexpr size_t kHsHist = 4096 * 4;
constexpr size_t kHsMeta = 64;
constexpr size_t kHsCand = (size_t)kHeadSlots * 8;
constexpr size_t kHsCcnt = (size_t)kHeadSlots * 4;
constexpr size_t kHsImage = (size_t)kHeadSlots * 8;
constexpr size_t kHsLongQ =
    (kHsSample + kHsHist + kHsMeta + kHsCand + kHsCcnt + kHsImage + kHeadBuckets + 255) & ~(size_t)255;
size_t head_scratch_bytes() { return kHsLongQ + (size_t)kLongQCap * 8; }

static int sm_count_dev() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int count_global_launches(uint64_t nbytes, bool head, bool scratch) {
    if (!nbytes) return 0;
    return ((nbytes >= kHeadMinBytes && head) ? 6 : 1) + (scratch ? 1 : 0);
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
    cudaError_t e = ensure_smem_limit((const void *)k_count3<MODE_HEAD>, (int)kCountSmem);
    if (e == cudaSuccess) e = ensure_smem_limit((const void *)k_count3<MODE_LOCAL>, (int)kCountSmem);
    if (e == cudaSuccess) e = ensure_smem_limit((const void *)k_count3<MODE_SAMPLE>, (int)kCountSmem);
    if (e == cudaSuccess) e = ensure_smem_limit((const void *)k_long_deferred, (int)kDefSmem);
    if (e != cudaSuccess) return e;
    if (c.hi <= c.lo) return cudaSuccess;
    const int sms = sm_count_dev();
    const uintptr_t tb = reinterpret_cast<uintptr_t>(c.text);
    Count2Args a;
    a.text = c.text;
    a.lo = c.lo;
    a.hi = c.hi;
    a.base_al = (tb + c.lo) & ~(uintptr_t)15;
    const unsigned long long span = tb + c.hi - a.base_al;
    a.nstrips = (span + kStrip - 1) / kStrip;
    a.piece_strips = 0;
    a.piece_stride = 0;
    a.g = c.g;
    a.lbegin = c.text;
    a.head = nullptr;
    a.head_disp = nullptr;
    a.lq = nullptr;
    a.lqn = nullptr;
    a.l1_off = c.no_level1 ? 1 : 0;
    const uint64_t n = c.hi - c.lo;
    uint8_t *hs = static_cast<uint8_t *>(c.head_scratch);
    unsigned long long *image =
        hs ? reinterpret_cast<unsigned long long *>(hs + kHsSample + kHsHist + kHsMeta + kHsCand + kHsCcnt) : nullptr;
    uint8_t *image_disp = hs ? reinterpret_cast<uint8_t *>(image + kHeadSlots) : nullptr;
    bool head = false, sampled = false;
    if (c.no_level1) {  // LOCAL kernel with its table switched off
    } else if (c.head_mode == 1 && hs) {  // the head an earlier launch built
        head = true;
    } else if (c.head_mode == 0 && n >= kHeadMinBytes && hs) {
        // sampling pass (LOCAL tables per block, spills into the sample table)
        G8Slot *sample = reinterpret_cast<G8Slot *>(hs);
        uint32_t *hist = reinterpret_cast<uint32_t *>(hs + kHsSample);
        uint32_t *meta = reinterpret_cast<uint32_t *>(hs + kHsSample + kHsHist);
        unsigned long long *cand = reinterpret_cast<unsigned long long *>(hs + kHsSample + kHsHist + kHsMeta);
        uint32_t *ccnt = reinterpret_cast<uint32_t *>(hs + kHsSample + kHsHist + kHsMeta + kHsCand);
        e = cudaMemsetAsync(hs, 0, kHsSample + kHsHist + kHsMeta, s);
        if (e != cudaSuccess) return e;
        Count2Args sa = a;
        sa.g.slots8 = sample;
        sa.g.mask8 = kSampleSlots - 1;
        sa.piece_strips = kSamplePieceBytes / kStrip;
        sa.piece_stride = (span / kSamplePieces) & ~(unsigned long long)15;
        sa.nstrips = (unsigned long long)sa.piece_strips * kSamplePieces;
        k_count3<MODE_SAMPLE><<<sms, kBlock, kCountSmem, s>>>(sa);
        // each head kernel overlaps its launch with the tail of the one before
        launch_dependent(k_head_hist, dim3(sms), dim3(256), 0, s, (const G8Slot *)sample, kSampleSlots, hist);
        launch_dependent(k_head_threshold, dim3(1), dim3(1024), 0, s, (const uint32_t *)hist, kHeadMax, meta);
        launch_dependent(k_head_collect, dim3(sms * 2), dim3(256), 0, s, (const G8Slot *)sample, kSampleSlots, meta,
                         cand, ccnt, kHeadMax);
        launch_dependent(k_head_chd, dim3(kHeadRegions), dim3(kChdThreads), 0, s, (const unsigned long long *)cand,
                         (const uint32_t *)ccnt, (const uint32_t *)meta, image, image_disp);
        head = true;
        sampled = true;
    }
    if (hs && !sampled) {  // the deferred long-word count (the sampling memset zeroes it otherwise)
        e = cudaMemsetAsync(hs + kHsSample + kHsHist + 32, 0, 8, s);
        if (e != cudaSuccess) return e;
    }
    if (hs) {
        a.lq = reinterpret_cast<unsigned long long *>(hs + kHsLongQ);
        a.lqn = reinterpret_cast<unsigned long long *>(hs + kHsSample + kHsHist + 32);
    }
    if (head) {
        a.head = image;
        a.head_disp = image_disp;
    }
    // one persistent block per SM (fewer for short texts); each block's
    // level-1 counts stay below 2^32 because a block reads under 2^33 bytes
    unsigned long long grid = c.grid > 0 ? (unsigned long long)c.grid : (unsigned long long)sms;
    const unsigned long long need = (a.nstrips + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    while ((a.nstrips + grid * kWarps - 1) / (grid * kWarps) * kWarps * kStrip >= (1ull << 33)) grid *= 2;
    for (cudaEvent_t ev : c.main_ev)
        if (ev) cudaEventRecord(ev, s);
    if (head) k_count3<MODE_HEAD><<<(unsigned)grid, kBlock, kCountSmem, s>>>(a);
    else k_count3<MODE_LOCAL><<<(unsigned)grid, kBlock, kCountSmem, s>>>(a);
    if (a.lq)
        launch_dependent(k_long_deferred, dim3(sms * 2), dim3(kDefChunk), kDefSmem, s, (const unsigned long long *)a.lq,
                         (const unsigned long long *)a.lqn, a.g, a.lbegin, reinterpret_cast<const uint8_t *>(tb + c.hi));
    return cudaGetLastError();
}

int count_global_chunk_bytes() { return kStrip; }
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
