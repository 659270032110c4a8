// Compaction, sort, merge, top-k and export of count tables.
//
// After the counting kernel the global hash tables hold each distinct word
// once with its exact count (Sec. 3.3's reduced dictionary).  This file turns
// them into the sorted output: compact the occupied slots, copy long words
// into the table's own byte arena, then sort.  A single table whose counts
// are below 2^32 is merge-sorted by one 128-bit key per entry (the
// complemented count, then the 16-letter prefix packed 5 bits a letter: 0 for
// padding, 1..26 for a..z, so integer order is lexicographic order and a
// proper prefix sorts first).  Other sorts (batched, merged and allocation-
// free tables) are an LSD radix sort over a permutation: 10 byte-digits of
// the packed prefix and up to 8 digits of the complemented count (count
// descending).  Either is followed by a fix-up that orders long words sharing
// count and 16-letter prefix by their remaining bytes; every radix pass is
// stable, so the final order is (count desc, word asc).  Digits that are equal for every
// element are skipped, detected on the device from one histogram pass; those
// the host's bounds already show constant (count bytes above the token bound,
// document bytes above the document count) are not launched at all.
#include <algorithm>
#include <vector>

#include "wc_internal.h"

namespace wc {

constexpr int kSortTile = (int)kSortTileElems;  // elements per block in a radix pass
constexpr int kSortThreads = 256;
constexpr int kItems = kSortTile / kSortThreads;  // 16
constexpr int kPasses = kSortPasses;
constexpr int kPassesSeg = kSortPassesSeg;

__device__ __forceinline__ unsigned long long be64(uint32_t x, uint32_t y) {
    return ((unsigned long long)__byte_perm(x, 0, 0x0123) << 32) | __byte_perm(y, 0, 0x0123);
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

size_t sort_scratch_bytes(uint64_t cap, bool with_msort) {
    uint64_t ntiles = (cap + kSortTile - 1) / kSortTile;
    return cap * (8 + 8 + 8 + 8 + 4 + 4 + 4 + 4 + 4) + 4 * kPassesSeg * 256 + 4 * 256 * ntiles + 4 * 32 +
           2 * 4 * 256 * (ntiles <= kSortFusedMaxTiles ? sort_group_stride(ntiles) : 1) + 4096 +
           2 * (4 * 256 * ntiles + 256) + 256 + (with_msort ? 4 * (cap * 8 + 256) : 0);
}

void sort_scratch_carve(SortScratch &s, void *base, uint64_t cap, bool with_msort) {
    uint64_t ntiles = (cap + kSortTile - 1) / kSortTile;
    uint8_t *p = static_cast<uint8_t *>(base);
    auto take = [&](size_t n) { uint8_t *r = p; p += (n + 255) & ~(size_t)255; return r; };
    s.cap = cap;
    s.khi = reinterpret_cast<unsigned long long *>(take(cap * 8));
    s.klo = reinterpret_cast<unsigned long long *>(take(cap * 8));
    s.cnt = reinterpret_cast<unsigned long long *>(take(cap * 8));
    s.pk = reinterpret_cast<unsigned long long *>(take(cap * 8));
    s.pk2 = reinterpret_cast<uint32_t *>(take(cap * 4));
    s.lref = reinterpret_cast<uint32_t *>(take(cap * 4));
    s.perm[0] = reinterpret_cast<uint32_t *>(take(cap * 4));
    s.perm[1] = reinterpret_cast<uint32_t *>(take(cap * 4));
    s.doc = reinterpret_cast<uint32_t *>(take(cap * 4));
    s.hist_all = reinterpret_cast<uint32_t *>(take(4 * kPassesSeg * 256));
    s.tile_hist = reinterpret_cast<uint32_t *>(take(4 * 256 * ntiles));
    s.cur = reinterpret_cast<uint32_t *>(take(4 * 32));
    s.group_stride = (uint32_t)(ntiles <= kSortFusedMaxTiles ? sort_group_stride(ntiles) : 1);
    s.group_hist[0] = reinterpret_cast<uint32_t *>(take(2 * 4 * 256 * (size_t)s.group_stride));  // both, adjacent
    s.group_hist[1] = s.group_hist[0] + 256 * (size_t)s.group_stride;
    s.look[0] = reinterpret_cast<uint32_t *>(take(4 * 256 * ntiles));
    s.look[1] = reinterpret_cast<uint32_t *>(take(4 * 256 * ntiles));
    s.tile_ctr = reinterpret_cast<uint32_t *>(take(4 * 2));
    for (int i = 0; i < 4; i++)
        s.mk[i] = with_msort ? reinterpret_cast<unsigned long long *>(take(cap * 8)) : nullptr;
}

// ---------------------------------------------------------------- compaction
// The sort's key for an entry: the 16-letter prefix packed 5 bits a letter
// (80 bits: pk low 64, pk2 high 16) and the count inverted (descending), and
// the counts of each of their digits in a block's histogram h (one row of 256
// per pass), from which a pass with a single digit value is skipped.
__device__ __forceinline__ void sort_key_prep(const SortScratch &s, unsigned long long i, unsigned long long khi,
                                              unsigned long long klo, unsigned long long cnt, uint32_t *h) {
    const unsigned long long ph = pack5(khi), pl = pack5(klo), c = ~cnt;
    const unsigned long long lo = (ph << 40) | pl;  // the 80-bit code: ph:pl
    const uint32_t hi = (uint32_t)(ph >> 24);
    s.perm[0][i] = (uint32_t)i;
    s.pk[i] = lo;
    s.pk2[i] = hi;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        atomicAdd(&h[b * 256 + ((lo >> (8 * b)) & 0xFF)], 1u);
        atomicAdd(&h[(kSortKeyPasses + b) * 256 + ((c >> (8 * b)) & 0xFF)], 1u);
    }
    atomicAdd(&h[8 * 256 + (hi & 0xFF)], 1u);
    atomicAdd(&h[9 * 256 + ((hi >> 8) & 0xFF)], 1u);
}

// The merge sort's 128-bit key of an entry (counts below 2^32): the count
// inverted in the high 32 bits (count descending), then the 80-bit packed
// prefix, then 16 zero bits.  A count of at least 1 keeps the high word below
// all ones, the key of the sort's padding.
__device__ __forceinline__ void ms_key_prep(const SortScratch &s, unsigned long long i, unsigned long long khi,
                                            unsigned long long klo, unsigned long long cnt) {
    const unsigned long long ph = pack5(khi), pl = pack5(klo);
    const unsigned long long lo = (ph << 40) | pl, hi16 = ph >> 24;  // the 80-bit code: hi16:lo
    s.mk[0][i] = ((unsigned long long)(~(uint32_t)cnt) << 32) | (hi16 << 16) | (lo >> 48);
    s.mk[1][i] = lo << 16;
}

// How a compaction prepares the sort: nothing (the sort packs its own keys),
// the radix sort's keys and digit counts (into the block histogram h), or the
// merge sort's keys.
enum KeyPrep : int { kPrepNone = 0, kPrepRadix = 1, kPrepMerge = 2 };

// One entry of a compaction, with the sort keys `prep` asks for.
__device__ __forceinline__ void emit_entry(const SortScratch &ss, unsigned long long pos, unsigned long long khi,
                                           unsigned long long klo, unsigned long long cnt, uint32_t lref, uint32_t *h,
                                           int prep) {
    ss.khi[pos] = khi;
    ss.klo[pos] = klo;
    ss.cnt[pos] = cnt;
    ss.lref[pos] = lref;
    if (prep == kPrepRadix) sort_key_prep(ss, pos, khi, klo, cnt, h);
    else if (prep == kPrepMerge) ms_key_prep(ss, pos, khi, klo, cnt);
}

// Occupied 16-byte-key slots -> entries (big-endian key halves); block bid of nb.
__device__ __forceinline__ void compact_short_body(const GSlot *slots, unsigned long long cap, const SortScratch &ss,
                                                   unsigned long long *meta, unsigned bid, unsigned nb, uint32_t *h,
                                                   int prep) {
    __shared__ BlockTake sh;
    const unsigned long long step = (unsigned long long)nb * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)bid * blockDim.x * kScanUnroll; b < cap; b += step) {
        uint4 k[kScanUnroll];
        unsigned long long c[kScanUnroll], tok = 0;
        uint32_t mine = 0;
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            k[u] = make_uint4(0, 0, 0, 0);
            c[u] = 0;
            if (i < cap) {
                k[u] = slots[i].key;
                c[u] = slots[i].cnt;
            }
            if (!key_zero(k[u])) {
                mine++;
                tok += c[u];
            }
        }
        unsigned long long pos = block_take(sh, mine, tok, &meta[0], &meta[3], &meta[6]);
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            if (key_zero(k[u])) continue;
            emit_entry(ss, pos, be64(k[u].x, k[u].y), be64(k[u].z, k[u].w), c[u], 0u, h, prep);
            pos++;
        }
    }
}

// Occupied 8-byte-key slots -> entries; block bid of nb.
__device__ __forceinline__ void compact8_body(const G8Slot *slots, unsigned long long cap, const SortScratch &ss,
                                              unsigned long long *meta, unsigned bid, unsigned nb, uint32_t *h,
                                              int prep) {
    __shared__ BlockTake sh;
    const unsigned long long step = (unsigned long long)nb * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)bid * blockDim.x * kScanUnroll; b < cap; b += step) {
        ulonglong2 v[kScanUnroll];
        unsigned long long tok = 0;
        uint32_t mine = 0;
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            v[u] = i < cap ? *reinterpret_cast<const ulonglong2 *>(&slots[i]) : make_ulonglong2(0ull, 0ull);
            if (v[u].x) {
                mine++;
                tok += v[u].y;
            }
        }
        unsigned long long pos = block_take(sh, mine, tok, &meta[0], &meta[3], &meta[5]);
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long key = v[u].x;
            if (!key) continue;
            emit_entry(ss, pos, be64((uint32_t)key, (uint32_t)(key >> 32)), 0ull, v[u].y, 0u, h, prep);
            pos++;
        }
    }
}

// Byte i (0..15) of 16 bytes held as a uint4 (little-endian words).
__device__ __forceinline__ uint32_t byte16(uint4 v, uint32_t i) {
    const uint32_t w = i < 8u ? (i < 4u ? v.x : v.y) : (i < 12u ? v.z : v.w);
    return (w >> (8u * (i & 3u))) & 0xFFu;
}

// One lane per long-word slot: a warp's occupied slots take their entry
// positions, long-word indices and arena bytes with one atomic each.  Each
// word is copied (lowercased, followed by one 0 byte so a run in the arena
// ends where the word ends) into the arena, by its own lane up to 64 bytes
// and by the whole warp beyond, and emits an entry.  A word of at most 32
// letters whose slot holds its first and last 16 letters (kLongReady) is
// written from the slot, without reading its occurrence in the text.
__device__ __forceinline__ void compact_long_body(const LSlot *ls, unsigned long long lcap, const SortScratch &ss,
                                                  const DevTable &out, unsigned bid, unsigned nb, uint32_t *hist,
                                                  int prep) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = ((unsigned long long)nb * blockDim.x) >> 5;
    unsigned long long *meta = out.d_meta;
    for (unsigned long long w0 = (((unsigned long long)bid * blockDim.x + threadIdx.x) >> 5) * 32; w0 < lcap;
         w0 += nw * 32) {
        const unsigned long long w = w0 + lane;
        unsigned long long h = 0, addr = 0, len = 0, c = 0, lr = 0;
        uint4 f = make_uint4(0u, 0u, 0u, 0u), l = f;
        if (w < lcap) {
            h = ls[w].h;
            addr = ls[w].addr;
            lr = ls[w].len;
            len = long_len(lr);
            c = ls[w].cnt;
        }
        const bool occ = !(h == 0 && addr == 0);
        const uint32_t m = __ballot_sync(kFull, occ);
        if (!m) continue;
        const bool from_slot = occ && (lr & kLongReady) && len <= 32;
        if (from_slot) {
            f = ls[w].f;
            l = ls[w].l;
        }
        const unsigned long long rank = __popc(m & lanemask_lt()), nocc = __popc(m);
        const unsigned long long bytes = occ ? len + 1 : 0ull;
        unsigned long long incl = bytes, tok = occ ? c : 0ull;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += t;
        }
        for (int d = 16; d; d >>= 1) tok += __shfl_xor_sync(kFull, tok, d);
        const unsigned long long total = __shfl_sync(kFull, incl, 31);
        unsigned long long boff = 0, blidx = 0, bpos = 0;
        if (lane == 0) {
            boff = atomicAdd(&meta[2], total);
            blidx = atomicAdd(&meta[1], nocc);
            bpos = atomicAdd(&meta[0], nocc);
            atomicAdd(&meta[3], tok);
        }
        const unsigned long long off = __shfl_sync(kFull, boff, 0) + incl - bytes;
        const unsigned long long lidx = __shfl_sync(kFull, blidx, 0) + rank;
        const unsigned long long pos = __shfl_sync(kFull, bpos, 0) + rank;
        // The arena or the long index is full: the table fails (status), but
        // the entry slot taken above is still filled (prefix key, no long
        // reference) so that the sort that follows reads only valid entries.
        const bool full = occ && (off + len + 1 > out.arena_cap || lidx >= out.lcap);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(addr);
        if (from_slot && !full)  // word byte j: f[j] below 16, else l[j - (len - 16)]
            for (uint32_t j = 0; j < (uint32_t)len; j++)
                out.arena[off + j] = (uint8_t)(j < 16u ? byte16(f, j) : byte16(l, j + 16u - (uint32_t)len));
        else if (occ && !full && len <= 64)
            for (unsigned long long j = 0; j < len; j++) out.arena[off + j] = (uint8_t)(src[j] | 0x20u);
        uint32_t big = __ballot_sync(kFull, occ && !full && len > 64);
        while (big) {
            const int l = __ffs(big) - 1;
            big &= big - 1;
            const uint8_t *bs = reinterpret_cast<const uint8_t *>(__shfl_sync(kFull, addr, l));
            const unsigned long long bo = __shfl_sync(kFull, off, l), bl = __shfl_sync(kFull, len, l);
            for (unsigned long long j = lane; j < bl; j += 32) out.arena[bo + j] = (uint8_t)(bs[j] | 0x20u);
        }
        if (occ) {
            if (full) {
                atomicOr(out.d_status, ST_ARENA_FULL);
            } else {
                out.arena[off + len] = 0;
                out.loff[lidx] = off;
                out.llen[lidx] = len;
            }
            unsigned long long hi = 0, lo = 0;
            if (from_slot) {  // f holds the first 16 letters, lowercased, little-endian words
                hi = ((unsigned long long)__byte_perm(f.x, 0, 0x0123) << 32) | __byte_perm(f.y, 0, 0x0123);
                lo = ((unsigned long long)__byte_perm(f.z, 0, 0x0123) << 32) | __byte_perm(f.w, 0, 0x0123);
            } else {
                for (int j = 0; j < 8; j++) hi = (hi << 8) | (unsigned long long)(src[j] | 0x20u);
                for (int j = 8; j < 16; j++) lo = (lo << 8) | (unsigned long long)(src[j] | 0x20u);
            }
            emit_entry(ss, pos, hi, lo, c, full ? 0u : (uint32_t)(lidx + 1), hist, prep);
        }
    }
}

// All three tables' occupied slots -> entries in one launch: blocks
// [0, nb8) scan the 8-byte table, the next nb16 the 16-byte table and the
// rest the long-word table.  The per-kind entry counts go to meta[5] (8-byte)
// and meta[6] (16-byte).  In a single table's finish the entries' sort keys
// are prepared here as well (`prep`; for the radix sort with the digit
// histograms of its passes).
__global__ void __launch_bounds__(256) k_compact_all(GTable g, unsigned long long cap8, unsigned long long cap16,
                                                     unsigned long long lcap, SortScratch ss, DevTable out,
                                                     unsigned nb8, unsigned nb16, int prep) {
    __shared__ uint32_t h[kPasses * 256];
    grid_dependency_wait();
    grid_dependency_trigger();
    const bool hist = prep == kPrepRadix;
    if (hist) {
        for (int i = threadIdx.x; i < kPasses * 256; i += blockDim.x) h[i] = 0u;
        __syncthreads();
    }
    uint32_t *hp = hist ? h : nullptr;
    const unsigned b = blockIdx.x;
    if (b < nb8) compact8_body(g.slots8, cap8, ss, out.d_meta, b, nb8, hp, prep);
    else if (b < nb8 + nb16) compact_short_body(g.slots, cap16, ss, out.d_meta, b - nb8, nb16, hp, prep);
    else compact_long_body(g.lslots, lcap, ss, out, b - nb8 - nb16, gridDim.x - nb8 - nb16, hp, prep);
    if (hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < kPasses * 256; i += blockDim.x)
            if (h[i]) atomicAdd(&ss.hist_all[i], h[i]);
    }
}

// ---------------------------------------------------------------- radix sort
// The sort kernels take one table's arguments as their parameter (OneJob) or
// several tables' from a device array, table blockIdx.y (JobList): a batch's
// class and global tables are sorted by one launch per pass.
struct OneJob {
    SortJob j;
    __device__ __forceinline__ const SortJob &get() const { return j; }
};
struct JobList {
    const SortJob *j;
    __device__ __forceinline__ const SortJob &get() const { return j[blockIdx.y]; }
};

__device__ __forceinline__ uint32_t sort_digit(const SortScratch &s, uint32_t idx, int p) {
    if (p >= kPasses) return (s.doc[idx] >> (8 * (p - kPasses))) & 0xFFu;
    if (p < 8) return (uint32_t)(s.pk[idx] >> (8 * p)) & 0xFFu;
    if (p < kSortKeyPasses) return (s.pk2[idx] >> (8 * (p - 8))) & 0xFFu;
    return (uint32_t)(~s.cnt[idx] >> (8 * (p - kSortKeyPasses))) & 0xFFu;
}

// Packs the prefix keys, and takes the histograms of all digit positions
// (for skipping constant digits) and the identity permutation.
template <class J>
__global__ void k_hist_all(J job, int passes) {
    const SortScratch &s = job.get().s;
    const unsigned long long *meta = job.get().meta;
    __shared__ uint32_t h[kPassesSeg * 256];
    for (int i = threadIdx.x; i < kPassesSeg * 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long n = meta[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        sort_key_prep(s, i, s.khi[i], s.klo[i], s.cnt[i], h);
        if (passes > kPasses) {
            const uint32_t d = s.doc[i];
#pragma unroll
            for (int b = 0; b < 4; b++) atomicAdd(&h[(kPasses + b) * 256 + ((d >> (8 * b)) & 0xFF)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
        if (h[i]) atomicAdd(&s.hist_all[i], h[i]);
}

// A pass is skipped when one digit value holds every element.
__device__ __forceinline__ bool pass_skipped(const SortScratch &s, int p, unsigned long long n) {
    bool mine = false;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) mine |= (s.hist_all[p * 256 + d] == n);
    return __syncthreads_or(mine) != 0;
}

template <class J>
__global__ void __launch_bounds__(kSortThreads) k_pass_count(J job, int p, int e, int fused) {
    const SortScratch &s = job.get().s;
    const unsigned long long *meta = job.get().meta;
    __shared__ uint32_t h[256];
    const unsigned long long n = meta[0];
    const unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    if (blockIdx.x >= ntiles) return;
    if (pass_skipped(s, p, n)) return;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t *in = s.perm_buf(s.cur[e]);
    const unsigned long long t0 = (unsigned long long)blockIdx.x * kSortTile + threadIdx.x;
    // all loads first (16 independent gathers in flight per thread), then the histogram
    uint32_t dig[kItems];
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + (unsigned long long)it * kSortThreads;
        dig[it] = i < n ? in[i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int it = 0; it < kItems; it++)
        if (dig[it] != 0xFFFFFFFFu) dig[it] = sort_digit(s, dig[it], p);
#pragma unroll
    for (int it = 0; it < kItems; it++)
        if (dig[it] != 0xFFFFFFFFu) atomicAdd(&h[dig[it]], 1u);
    __syncthreads();
    const uint32_t c = h[threadIdx.x];
    s.tile_hist[(unsigned long long)threadIdx.x * ntiles + blockIdx.x] = c;
    if (fused && c)
        atomicAdd(&s.group_buf((uint32_t)e & 1u)[(unsigned long long)threadIdx.x * s.group_stride +
                                                 blockIdx.x / sort_group_tiles(ntiles)],
                  c);
}

// Sorts of more than kSortFusedMaxTiles tiles: exclusive scan of the
// digit-major tile histogram: block d scans digit d's
// row of tile counts, starting from the number of elements with a smaller
// digit (from the all-pass histogram).  256 blocks of 256 threads.
template <class J>
__global__ void __launch_bounds__(256) k_pass_scan(J job, int p, int e, int last) {
    const SortScratch &s = job.get().s;
    const unsigned long long *meta = job.get().meta;
    __shared__ uint32_t part[256];
    __shared__ uint32_t base_s;
    const unsigned long long n = meta[0];
    const bool skip = pass_skipped(s, p, n) || n == 0;
    if (skip) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            s.cur[e + 1] = s.cur[e];
            if (last) s.cur[kCurFinal] = s.cur[e];
        }
        return;
    }
    const uint32_t d = blockIdx.x, t = threadIdx.x;
    // base = elements whose digit is below d
    part[t] = t < d ? s.hist_all[p * 256 + t] : 0u;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (t < (uint32_t)w) part[t] += part[t + w];
        __syncthreads();
    }
    if (t == 0) base_s = part[0];
    __syncthreads();
    uint32_t run = base_s;
    const unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    uint32_t *row = s.tile_hist + (unsigned long long)d * ntiles;
    for (unsigned long long c0 = 0; c0 < ntiles; c0 += 256) {
        const unsigned long long i = c0 + t;
        const uint32_t v = i < ntiles ? row[i] : 0u;
        __syncthreads();
        part[t] = v;
        __syncthreads();
        for (int w = 1; w < 256; w <<= 1) {
            uint32_t x = t >= (uint32_t)w ? part[t - w] : 0u;
            __syncthreads();
            part[t] += x;
            __syncthreads();
        }
        if (i < ntiles) row[i] = run + part[t] - v;
        run += part[255];
    }
    if (d == 0 && t == 0) {
        s.cur[e + 1] = 1u - s.cur[e];
        if (last) s.cur[kCurFinal] = 1u - s.cur[e];
    }
}

// Stable scatter: warp w ranks its 512 consecutive elements in order with
// match_any; warps are combined in order, so equal digits keep their order.
template <class J>
__global__ void __launch_bounds__(kSortThreads) k_pass_scatter(J job, int p, int e, int fused, int last) {
    const SortScratch &s = job.get().s;
    const unsigned long long *meta = job.get().meta;
    constexpr int WARPS = kSortThreads / 32;
    static_assert(kSortThreads == 256, "one thread per digit");
    __shared__ uint32_t wcount[WARPS][256];
    __shared__ uint32_t wtot[WARPS];
    const unsigned long long n = meta[0];
    const unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    const bool skip = pass_skipped(s, p, n);
    if (fused) {  // (the scan pass does both otherwise)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const uint32_t c = skip ? s.cur[e] : 1u - s.cur[e];
            s.cur[e + 1] = c;
            if (last) s.cur[kCurFinal] = c;
        }
        // the next pass's group counts start from zero (this pass's are in the other buffer)
        uint32_t *gn = s.group_buf(((uint32_t)e + 1u) & 1u);
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
             i < 256ull * s.group_stride; i += (unsigned long long)gridDim.x * blockDim.x)
            gn[i] = 0u;
    }
    if (skip || blockIdx.x >= ntiles) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * 256; i += kSortThreads) (&wcount[0][0])[i] = 0;
    // This tile's first position for digit d = threadIdx.x: scanned by the
    // scan pass, or (fused) the entries with a smaller digit, then digit d's
    // entries in the earlier tile groups and in the earlier tiles of this
    // tile's group.
    const int d = threadIdx.x;
    uint32_t run;
    if (fused) {
        const uint32_t own = s.hist_all[p * 256 + d];
        uint32_t incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) wtot[warp] = incl;
        run = incl - own;
        const uint32_t G = (uint32_t)sort_group_tiles(ntiles), g = blockIdx.x / G;
        const uint32_t *gb = s.group_buf((uint32_t)e & 1u) + (unsigned long long)d * s.group_stride;
#pragma unroll 4
        for (uint32_t q = 0; q < g; q++) run += gb[q];
        const uint32_t *tb = s.tile_hist + (unsigned long long)d * ntiles;
#pragma unroll 4
        for (uint32_t t2 = g * G; t2 < blockIdx.x; t2++) run += tb[t2];
    } else {
        run = s.tile_hist[(unsigned long long)d * ntiles + blockIdx.x];
    }
    __syncthreads();
    if (fused)
        for (int w = 0; w < warp; w++) run += wtot[w];
    const uint32_t cur = s.cur[e];
    const uint32_t *in = s.perm_buf(cur);
    uint32_t *out = s.perm_buf(1 - cur);
    const unsigned long long t0 = (unsigned long long)blockIdx.x * kSortTile + (unsigned long long)warp * (kSortTile / WARPS);
    uint32_t idx[kItems], dig[kItems], rank[kItems];
    // all loads first (independent gathers in flight), then the in-order ranking
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        idx[it] = i < n ? in[i] : 0u;
    }
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        dig[it] = i < n ? sort_digit(s, idx[it], p) : 256u + lane;  // invalid lanes never match real digits
    }
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        const bool valid = i < n;
        uint32_t peers = __match_any_sync(kFull, dig[it]);
        int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader && valid) {
            before = wcount[warp][dig[it]];
            wcount[warp][dig[it]] = before + __popc(peers);
        }
        before = __shfl_sync(kFull, before, leader);
        rank[it] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // exclusive prefix over warps, per digit (thread d handles digit d)
    {
        for (int w = 0; w < WARPS; w++) {
            uint32_t v = wcount[w][d];
            wcount[w][d] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        unsigned long long i = t0 + it * 32 + lane;
        if (i < n) out[wcount[warp][dig[it]] + rank[it]] = idx[it];
    }
}

// One radix pass in one launch, with a decoupled look-back for the tile
// offsets.  Blocks take tiles in launch order from a counter (so every tile
// a block waits for belongs to a block that is already running), rank their
// entries per digit as k_pass_scatter does, publish their per-digit counts
// (flag "aggregate"), and learn the counts of all earlier tiles by walking
// back over the published values until one carries a complete prefix (flag
// "inclusive"), which they then publish for their own tile.  Each wait is
// bounded: a look-back that gives up records kCurSortError (reported as a
// timeout by the finish) instead of hanging.  The block also zeroes its row
// of the other parity's look-back buffer and block 0 the other tile counter,
// for the next pass.
constexpr uint32_t kLookAgg = 1u << 30, kLookInc = 2u << 30, kLookVal = kLookAgg - 1u;
constexpr uint32_t kLookSpins = 1u << 22;  // look-back rounds before giving up
constexpr int kLookWin = 8;                // earlier tiles read per round
// A published word carries its flag and value together, and nothing else is
// read on its account (the next pass is ordered by the kernel boundary), so
// relaxed GPU-scope accesses suffice.
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
template <class J>
__global__ void __launch_bounds__(kSortThreads) k_pass_one(J job, int p, int e, int last) {
    grid_dependency_wait();
    grid_dependency_trigger();
    const SortScratch &s = job.get().s;
    const unsigned long long *meta = job.get().meta;
    constexpr int WARPS = kSortThreads / 32;
    __shared__ uint32_t wcount[WARPS][256];
    __shared__ uint32_t wtot[WARPS];
    __shared__ uint32_t tile_sh;
    const unsigned long long n = meta[0];
    // loads that do not depend on n go out with it: digit d's count over all
    // entries (thread d) and the order this pass reads
    const int d = threadIdx.x;
    const uint32_t own = s.hist_all[p * 256 + d];
    const uint32_t cur = s.cur[e];
    const unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    // the grid is sized by capacity: blocks past the entries leave at once
    // (block 0 stays: it records this pass's order even for an empty table)
    if (blockIdx.x >= ntiles && blockIdx.x != 0) return;
    const uint32_t par = (uint32_t)e & 1u;
    // the tile is taken before the skip test is known (a skipped pass's count
    // is zeroed by the next pass like any other)
    if (blockIdx.x < ntiles && threadIdx.x == 0) tile_sh = atomicAdd(&s.tile_ctr[par], 1u);
    if (blockIdx.x < ntiles) s.look_buf(par ^ 1u)[(unsigned long long)blockIdx.x * 256 + threadIdx.x] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) s.tile_ctr[par ^ 1u] = 0u;
    // a pass is skipped when one digit value holds every entry
    const bool skip = __syncthreads_or(own == n) != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t c = skip ? cur : 1u - cur;
        s.cur[e + 1] = c;
        if (last) s.cur[kCurFinal] = c;
    }
    if (skip || blockIdx.x >= ntiles) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * 256; i += kSortThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = tile_sh;
    const uint32_t *in = s.perm_buf(cur);
    uint32_t *out = s.perm_buf(1 - cur);
    const unsigned long long t0 = (unsigned long long)tile * kSortTile + (unsigned long long)warp * (kSortTile / WARPS);
    uint32_t idx[kItems], dig[kItems], rank[kItems];
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        idx[it] = i < n ? in[i] : 0u;
    }
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        dig[it] = i < n ? sort_digit(s, idx[it], p) : 256u + lane;  // invalid lanes never match real digits
    }
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        const bool valid = i < n;
        const uint32_t peers = __match_any_sync(kFull, dig[it]);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader && valid) {
            before = wcount[warp][dig[it]];
            wcount[warp][dig[it]] = before + __popc(peers);
        }
        before = __shfl_sync(kFull, before, leader);
        rank[it] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // thread d: this tile's count of digit d, published, then the look-back
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) cnt += wcount[w][d];
    uint32_t *look = s.look_buf(par);
    uint32_t excl = 0;
    if (tile == 0) {
        st_relaxed_u32(&look[d], kLookInc | cnt);
    } else {
        st_relaxed_u32(&look[(unsigned long long)tile * 256 + d], kLookAgg | cnt);
        // look back kLookWin tiles per round trip: add published counts from
        // the nearest tile down until one carries a complete prefix; a tile not
        // yet published ends the round, and the next round starts from it
        long long t = (long long)tile - 1;
        uint32_t rounds = 0;
        bool done = false;
        while (!done) {
            uint32_t v[kLookWin];
#pragma unroll
            for (int j = 0; j < kLookWin; j++)
                v[j] = t - j >= 0 ? ld_relaxed_u32(&look[(unsigned long long)(t - j) * 256 + d]) : 0u;
            int j = 0;
#pragma unroll
            for (; j < kLookWin; j++) {
                if (!(v[j] & (kLookAgg | kLookInc))) break;
                excl += v[j] & kLookVal;
                if (v[j] & kLookInc) { done = true; break; }
            }
            if (done) break;
            t -= j;
            if (++rounds >= kLookSpins) {  // gave up: recorded, the order is not used
                atomicOr(&s.cur[kCurSortError], 1u);
                break;
            }
        }
        st_relaxed_u32(&look[(unsigned long long)tile * 256 + d], kLookInc | (excl + cnt));
    }
    // this tile's first position for digit d: the entries with a smaller
    // digit (the all-pass histogram) plus digit d's entries in earlier tiles
    uint32_t incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    uint32_t run = incl - own + excl;
    for (int w = 0; w < warp; w++) run += wtot[w];
    for (int w = 0; w < WARPS; w++) {
        const uint32_t v = wcount[w][d];
        wcount[w][d] = run;
        run += v;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const unsigned long long i = t0 + it * 32 + lane;
        if (i < n) out[wcount[warp][dig[it]] + rank[it]] = idx[it];
    }
}

// ---------------------------------------------------------------- merge sort
// A single table's finish (counts below 2^32) sorts its entries by one
// 128-bit key each (ms_key_prep: count descending, then the 16-letter
// prefix); the entry index travels with the key.  Keys that tie belong to
// long words sharing count and prefix, which the long-word fix-up orders
// afterwards, so ties may come out in any order.  Blocks first sort runs of
// kMsTile entries: each thread sorts kMsPer entries in registers (a bitonic
// network), then the block merges pairs of sorted pieces in shared memory
// until the run is whole.  Each round then merges pairs of runs into runs
// twice as long, until one run holds every entry: ceil(log2(n / kMsTile))
// rounds, each one launch in which no block waits for another.  A block of a
// round writes kMsTile consecutive outputs of one merged pair: it finds how
// many of them come from the first run at its first and last output (the
// merge path split; each search step tests kMsThreads candidates at once, one
// a thread, and keeps the interval between the last that goes first and the
// first that does not), stages the two input pieces in shared memory, and
// merges kMsPer outputs a thread.  Every merge takes the first run's entry on
// a tie, and every search counts the same way.  Keys and indices alternate
// between two buffers: the run sort writes buffer 1, round r reads buffer
// r & 1.
constexpr int kMsTile = 4096;
constexpr int kMsThreads = 256;
constexpr int kMsPer = kMsTile / kMsThreads;  // entries a thread sorts or merges
static_assert(kMsPer == 16 && (kMsTile & (kMsTile - 1)) == 0, "16 entries a thread, power-of-two runs");
// Shared memory: slot i at i + i / 16, so that the 16 consecutive entries of
// each of a warp's threads fall in different banks.
constexpr int kMsSlots = kMsTile + kMsTile / 16;
constexpr size_t kMsSmem = (size_t)kMsSlots * (8 + 8 + 4);
__host__ __device__ __forceinline__ int ms_rounds(unsigned long long n) {
    int r = 0;
    for (unsigned long long len = kMsTile; len < n; len <<= 1) r++;
    return r;
}
struct MsKey {
    unsigned long long h, l;
    uint32_t x;  // entry index (not compared)
};
// A run sort's key: the index within the run in the 16 free low bits of l.
struct MsKey2 {
    unsigned long long h, l;
};
__device__ __forceinline__ bool ms_less(const MsKey &a, const MsKey &b) { return a.h != b.h ? a.h < b.h : a.l < b.l; }
__device__ __forceinline__ bool ms_less(const MsKey2 &a, const MsKey2 &b) { return a.h != b.h ? a.h < b.h : a.l < b.l; }
struct MsShared {
    unsigned long long *h, *l;
    uint32_t *x;
    __device__ __forceinline__ explicit MsShared(unsigned long long *base)
        : h(base), l(base + kMsSlots), x(reinterpret_cast<uint32_t *>(base + 2 * kMsSlots)) {}
    __device__ __forceinline__ static uint32_t at(uint32_t i) { return i + (i >> 4); }
    __device__ __forceinline__ void get(uint32_t i, MsKey &k) const {
        const uint32_t j = at(i);
        k = MsKey{h[j], l[j], x[j]};
    }
    __device__ __forceinline__ void get(uint32_t i, MsKey2 &k) const {
        const uint32_t j = at(i);
        k = MsKey2{h[j], l[j]};
    }
    __device__ __forceinline__ void put(uint32_t i, const MsKey &k) const {
        const uint32_t j = at(i);
        h[j] = k.h;
        l[j] = k.l;
        x[j] = k.x;
    }
    __device__ __forceinline__ void put(uint32_t i, const MsKey2 &k) const {
        const uint32_t j = at(i);
        h[j] = k.h;
        l[j] = k.l;
    }
};
// How many of sm[a0, a0 + na) lead the first d outputs of merging them with
// sm[b0, b0 + nb) (the first piece first on ties), by bisection.
template <class K>
__device__ __forceinline__ uint32_t ms_split(const MsShared &sm, uint32_t a0, uint32_t na, uint32_t b0, uint32_t nb,
                                             uint32_t d) {
    uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        K ka, kb;
        sm.get(a0 + m, ka);
        sm.get(b0 + d - 1 - m, kb);
        if (!ms_less(kb, ka)) lo = m + 1;
        else hi = m;
    }
    return lo;
}
// cnt (<= kMsPer) outputs of merging sm[a0, a0 + na) with sm[b0, b0 + nb),
// starting ia entries into the first and ib into the second, into v.
template <class K>
__device__ __forceinline__ void ms_merge_into(const MsShared &sm, uint32_t a0, uint32_t na, uint32_t b0, uint32_t nb,
                                              uint32_t ia, uint32_t ib, uint32_t cnt, K (&v)[kMsPer]) {
    K ka{}, kb{};
    if (ia < na) sm.get(a0 + ia, ka);
    if (ib < nb) sm.get(b0 + ib, kb);
#pragma unroll
    for (int k = 0; k < kMsPer; k++) {
        if ((uint32_t)k < cnt) {  // ia + ib < na + nb: one of the pieces has an entry left
            const bool fromA = ib >= nb || (ia < na && !ms_less(kb, ka));
            v[k] = fromA ? ka : kb;
            // one load path for either piece (lanes taking from different
            // pieces do not diverge): the taken piece's next entry
            ia += fromA ? 1u : 0u;
            ib += fromA ? 0u : 1u;
            const uint32_t nx = fromA ? ia : ib;
            if (nx < (fromA ? na : nb)) {
                K nk;
                sm.get((fromA ? a0 : b0) + nx, nk);
                if (fromA) ka = nk;
                else kb = nk;
            }
        }
    }
}

// Sorts entries [kMsTile * b, kMsTile * (b + 1)) of buffer 0 into buffer 1;
// block 0 records which buffer the last round leaves the order in.
__global__ void __launch_bounds__(kMsThreads) k_ms_runs(SortScratch s, const unsigned long long *meta) {
    extern __shared__ __align__(16) unsigned long long ms_smem[];
    const MsShared sm(ms_smem);
    grid_dependency_wait();
    grid_dependency_trigger();
    const unsigned long long n = meta[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) s.cur[kCurFinal] = (ms_rounds(n) & 1) ? 0u : 1u;
    const unsigned long long base = (unsigned long long)blockIdx.x * kMsTile;
    if (base >= n) return;
    const uint32_t m = (uint32_t)(n - base < (unsigned long long)kMsTile ? n - base : (unsigned long long)kMsTile);
    const uint32_t t = threadIdx.x;
    // coalesced loads into shared memory (padding past m sorts last), then
    // each thread's kMsPer consecutive entries into registers
    MsKey2 v[kMsPer];
#pragma unroll
    for (int k = 0; k < kMsPer; k++) {
        const uint32_t i = t + (uint32_t)k * kMsThreads;
        v[k] = i < m ? MsKey2{s.mk[0][base + i], s.mk[1][base + i] | i} : MsKey2{~0ull, ~0ull};
    }
#pragma unroll
    for (int k = 0; k < kMsPer; k++) sm.put(t + (uint32_t)k * kMsThreads, v[k]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMsPer; k++) sm.get(kMsPer * t + k, v[k]);
    // bitonic network over the thread's entries (ascending)
#pragma unroll
    for (int k = 2; k <= kMsPer; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < kMsPer; i++) {
                const int p = i ^ j;
                if (p > i && ms_less(v[p], v[i]) == ((i & k) == 0)) {
                    const MsKey2 w = v[i];
                    v[i] = v[p];
                    v[p] = w;
                }
            }
    // merge sorted pieces of sz entries in pairs until the run is whole;
    // thread t produces outputs [kMsPer * t, kMsPer * (t + 1)) of its pair
    for (uint32_t sz = kMsPer; sz < (uint32_t)kMsTile; sz <<= 1) {
        __syncthreads();  // every thread has read the previous level
#pragma unroll
        for (int k = 0; k < kMsPer; k++) sm.put(kMsPer * t + k, v[k]);
        __syncthreads();
        const uint32_t g0 = (kMsPer * t) & ~(2 * sz - 1), d = kMsPer * t - g0;
        const uint32_t ia = ms_split<MsKey2>(sm, g0, sz, g0 + sz, sz, d);
        ms_merge_into(sm, g0, sz, g0 + sz, sz, ia, d - ia, kMsPer, v);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMsPer; k++) sm.put(kMsPer * t + k, v[k]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMsPer; k++) {
        const uint32_t i = t + (uint32_t)k * kMsThreads;
        if (i < m) {
            MsKey2 w;
            sm.get(i, w);
            s.mk[2][base + i] = w.h;
            s.mk[3][base + i] = w.l & ~0xFFFFull;
            s.perm[1][base + i] = (uint32_t)(base + (w.l & 0xFFFFull));
        }
    }
}

// Round r: runs of kMsTile << (r - 1) entries merged in pairs.
__global__ void __launch_bounds__(kMsThreads) k_ms_merge(SortScratch s, const unsigned long long *meta, int r) {
    extern __shared__ __align__(16) unsigned long long ms_smem[];
    const MsShared sm(ms_smem);
    grid_dependency_wait();
    grid_dependency_trigger();
    const unsigned long long n = meta[0];
    const unsigned long long R = (unsigned long long)kMsTile << (r - 1);
    const unsigned long long out0 = (unsigned long long)blockIdx.x * kMsTile;
    if (R >= n || out0 >= n) return;  // one run holds everything already / no tile
    const uint32_t src = (uint32_t)r & 1u;
    const unsigned long long *ih = s.mk[src ? 2 : 0], *il = s.mk[src ? 3 : 1];
    const uint32_t *ix = s.perm_buf(src);
    unsigned long long *oh = s.mk[src ? 0 : 2], *ol = s.mk[src ? 1 : 3];
    uint32_t *ox = s.perm_buf(1u - src);
    // this tile's pair: run A = [p0, ae), run B = [ae, be); outputs [out0, out1)
    const unsigned long long out1 = out0 + kMsTile < n ? out0 + kMsTile : n;
    const unsigned long long p0 = out0 / (2 * R) * (2 * R);
    const unsigned long long ae = p0 + R < n ? p0 + R : n, be = p0 + 2 * R < n ? p0 + 2 * R : n;
    const uint32_t la = (uint32_t)(ae - p0), lb = (uint32_t)(be - ae);
    const uint32_t d0 = (uint32_t)(out0 - p0), d1 = (uint32_t)(out1 - p0);
    // A[a] goes before B[d - 1 - a]: its key is not above (A first on ties)
    auto first = [&](uint32_t d, uint32_t a) {
        const unsigned long long bh = ih[ae + d - 1 - a], bl = il[ae + d - 1 - a];
        const unsigned long long ah = ih[p0 + a], al = il[p0 + a];
        return !(bh != ah ? bh < ah : bl < al);
    };
    // the splits of outputs d0 and d1, searched together: a in
    // [max(0, d - lb), min(d, la)], every bound block-uniform.  An interval
    // of w <= E candidates is tested whole (thread i tests lo + i); a wider
    // one at the P = E - 1 points lo + (i + 1) w / E (no division: E = 256)
    constexpr uint32_t E = kMsThreads, P = E - 1;
    static_assert(kMsThreads == 256, "candidates placed by a shift of 8");
    auto cand = [](uint32_t lo, uint32_t w, uint32_t i) -> uint32_t {
        return w <= E ? lo + i : lo + (uint32_t)(((unsigned long long)(i + 1) * w) >> 8);
    };
    uint32_t lo0 = d0 > lb ? d0 - lb : 0u, hi0 = d0 < la ? d0 : la;
    uint32_t lo1 = d1 > lb ? d1 - lb : 0u, hi1 = d1 < la ? d1 : la;
    const uint32_t t = threadIdx.x;
    while (lo0 < hi0 || lo1 < hi1) {  // each step leaves at most w / E + 1 of w > E candidates, 0 of fewer
        const uint32_t w0 = hi0 - lo0, w1 = hi1 - lo1;
        const bool b0 = t < (w0 <= E ? w0 : P) && first(d0, cand(lo0, w0, t));
        const bool b1 = t < (w1 <= E ? w1 : P) && first(d1, cand(lo1, w1, t));
        const uint32_t c0 = (uint32_t)__syncthreads_count(b0), c1 = (uint32_t)__syncthreads_count(b1);
        if (w0 <= E) {
            lo0 += c0;
            hi0 = lo0;
        } else {
            const uint32_t nl = c0 ? cand(lo0, w0, c0 - 1) + 1 : lo0;
            if (c0 < P) hi0 = cand(lo0, w0, c0);
            lo0 = nl;
        }
        if (w1 <= E) {
            lo1 += c1;
            hi1 = lo1;
        } else {
            const uint32_t nl = c1 ? cand(lo1, w1, c1 - 1) + 1 : lo1;
            if (c1 < P) hi1 = cand(lo1, w1, c1);
            lo1 = nl;
        }
    }
    // the tile's inputs, A[lo0, lo1) then B[d0 - lo0, d1 - lo1): na + nb = L
    const uint32_t L = d1 - d0, na = lo1 - lo0, nb = L - na;
    const unsigned long long ga = p0 + lo0, gb = ae + (d0 - lo0);
    MsKey v[kMsPer];
#pragma unroll
    for (int k = 0; k < kMsPer; k++) {
        const uint32_t i = t + (uint32_t)k * kMsThreads;
        if (i < L) {
            const unsigned long long g = i < na ? ga + i : gb + (i - na);
            v[k] = MsKey{ih[g], il[g], ix[g]};
        }
    }
#pragma unroll
    for (int k = 0; k < kMsPer; k++) {
        const uint32_t i = t + (uint32_t)k * kMsThreads;
        if (i < L) sm.put(i, v[k]);
    }
    __syncthreads();
    // thread t: outputs [kMsPer * t, ...) of the tile, from its own split
    const uint32_t dt = kMsPer * t < L ? kMsPer * t : L, cnt = L - dt < (uint32_t)kMsPer ? L - dt : (uint32_t)kMsPer;
    const uint32_t ia = ms_split<MsKey>(sm, 0, na, na, nb, dt);
    ms_merge_into(sm, 0, na, na, nb, ia, dt - ia, cnt, v);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMsPer; k++)
        if ((uint32_t)k < cnt) sm.put(dt + k, v[k]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMsPer; k++) {
        const uint32_t i = t + (uint32_t)k * kMsThreads;
        if (i < L) {
            MsKey w;
            sm.get(i, w);
            oh[out0 + i] = w.h;
            ol[out0 + i] = w.l;
            ox[out0 + i] = w.x;
        }
    }
}

// Compares two entries whose 16-byte prefixes are equal by the bytes after
// the prefix (a word that fits the prefix is a proper prefix of a longer one).
__device__ __forceinline__ bool tail_less(const LongView &v, uint32_t a, uint32_t b) {
    uint32_t ra = v.lref[a], rb = v.lref[b];
    if (ra == 0) return rb != 0;   // the 16-letter (or shorter) word is a prefix
    if (rb == 0) return false;
    const uint8_t *pa = v.arena + v.loff[ra - 1], *pb = v.arena + v.loff[rb - 1];
    unsigned long long la = v.llen[ra - 1], lb = v.llen[rb - 1];
    unsigned long long m = la < lb ? la : lb;
    for (unsigned long long i = 16; i < m; i++)
        if (pa[i] != pb[i]) return pa[i] < pb[i];
    return la < lb;
}

// After the last pass, entries are in (document, count desc, 16-letter prefix
// asc) order; only a long word can share its prefix with another word, so
// the runs left to order are the entries of one document with equal count
// and prefix that hold a long word, ordered here by their full bytes.  The
// first long entry of such a run sorts it by insertion; the runs are tiny.
__device__ __forceinline__ bool same_run(const SortScratch &s, uint32_t a, uint32_t b, bool seg) {
    return s.khi[a] == s.khi[b] && s.klo[a] == s.klo[b] && s.cnt[a] == s.cnt[b] && (!seg || s.doc[a] == s.doc[b]);
}
template <class J>
__global__ void k_fix_long(J job, int passes) {
    grid_dependency_wait();
    grid_dependency_trigger();
    const SortScratch &s = job.get().s;
    const LongView &v = job.get().v;
    const unsigned long long *meta = job.get().meta;
    const unsigned long long n = meta[0];
    if (meta[1] == 0) return;
    const bool seg = passes > kPasses;
    uint32_t *perm = s.perm_buf(s.cur[kCurFinal]);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t e = perm[i];
        if (v.lref[e] == 0u) continue;
        unsigned long long lo = i;
        bool leader = true;
        while (lo > 0) {
            const uint32_t q = perm[lo - 1];
            if (!same_run(s, q, e, seg)) break;
            if (v.lref[q] != 0u) { leader = false; break; }  // an earlier long entry sorts the run
            lo--;
        }
        if (!leader) continue;
        unsigned long long j = i + 1;
        while (j < n && same_run(s, perm[j], e, seg)) j++;
        if (j - lo < 2) continue;
        const unsigned long long i0 = lo;
        for (unsigned long long a = i0 + 1; a < j; a++) {
            uint32_t x = perm[a];
            unsigned long long b = a;
            while (b > i0 && tail_less(v, x, perm[b - 1])) { perm[b] = perm[b - 1]; b--; }
            perm[b] = x;
        }
    }
}

__device__ __forceinline__ unsigned long long short_len(unsigned long long hi, unsigned long long lo) {
    if (lo) return 16 - (__ffsll((long long)lo) - 1) / 8;
    return 8 - (__ffsll((long long)hi) - 1) / 8;
}

template <class J>
__global__ void k_gather_final(J job) {
    grid_dependency_wait();
    grid_dependency_trigger();
    const SortScratch &s = job.get().s;
    const DevTable &out = job.get().out;
    const unsigned long long n = out.d_meta[0];
    if (blockIdx.x == 0 && threadIdx.x == 0 && s.cur[kCurSortError]) atomicOr(out.d_status, ST_TIMEOUT);
    const uint32_t *perm = s.perm_buf(s.cur[kCurFinal]);
    unsigned long long bytes = 0;
    // kScanUnroll entries a thread per step, all gathers issued before the stores
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x * kScanUnroll; b < n; b += step) {
        uint32_t e[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            e[u] = i < n ? perm[i] : 0u;
        }
        unsigned long long hi[kScanUnroll], lo[kScanUnroll], c[kScanUnroll];
        uint32_t r[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            hi[u] = s.khi[e[u]];
            lo[u] = s.klo[e[u]];
            c[u] = s.cnt[e[u]];
            r[u] = s.lref[e[u]];
        }
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            if (i >= n) continue;
            out.khi[i] = hi[u];
            out.klo[i] = lo[u];
            out.lref[i] = r[u];
            if (out.count_bits == 32) static_cast<uint32_t *>(out.cnt)[i] = (uint32_t)c[u];
            else static_cast<unsigned long long *>(out.cnt)[i] = c[u];
            bytes += r[u] ? out.llen[r[u] - 1] : short_len(hi[u], lo[u]);
        }
    }
    for (int d = 16; d; d >>= 1) bytes += __shfl_xor_sync(kFull, bytes, d);
    if ((threadIdx.x & 31) == 0 && bytes) atomicAdd(&out.d_meta[4], bytes);
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

static int grid_for(unsigned long long n, int threads, int max_blocks) {
    unsigned long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (unsigned long long)max_blocks) g = max_blocks;
    return (int)g;
}

// A single table's finish merge-sorts when the scratch has the key buffers
// and every count is below 2^32 (the radix sort's count digits 4..7 skipped).
static bool use_msort(const SortScratch &ss, uint32_t skip) {
    return ss.mk[0] && ((skip >> (kSortKeyPasses + 4)) & 0xFu) == 0xFu;
}

// reset + fused compaction + (run sort + merge rounds + long-word fix-up, or
// the sort without its key pass) + gather
int finish_table_launches(const SortScratch &ss, uint32_t skip) {
    if (use_msort(ss, skip)) return 2 + 1 + ms_rounds(ss.cap) + 1 + 1;
    return 2 + sort_entries_launches(kPasses, ss.cap, skip) - 1 + 1;
}

// The passes of one sort, for one table (J = OneJob) or a list of them;
// keyed: the compaction has prepared the sort keys and histograms already.
template <class J>
static void launch_sort(const J &job, uint64_t cap, int ntab, int passes, uint32_t skip, cudaStream_t st,
                        bool keyed = false) {
    const int sms = sm_count();
    if (!keyed) k_hist_all<<<dim3(grid_for(cap, 256, sms * 2), ntab), 256, 0, st>>>(job, passes);
    const int ntiles = (int)((cap + kSortTile - 1) / kSortTile);
    const int fused = (uint64_t)ntiles <= kSortFusedMaxTiles;
    int lastp = -1;
    for (int p = 0; p < passes; p++)
        if (!((skip >> p) & 1u)) lastp = p;
    // e counts the launched passes: pass e reads its order from cur[e].
    // Counts below 2^30 fit the look-back words: one launch a pass; larger
    // sorts count, (scan) and scatter in separate launches.
    const bool onesweep = cap < (1ull << 30);
    for (int p = 0, e = 0; p < passes; p++) {
        if ((skip >> p) & 1u) continue;
        const int last = p == lastp;
        if (onesweep) {  // overlaps its launch with the tail of the kernel before
            launch_dependent(k_pass_one<J>, dim3(ntiles, ntab), dim3(kSortThreads), 0, st, job, p, e, last);
        } else {
            k_pass_count<<<dim3(ntiles, ntab), kSortThreads, 0, st>>>(job, p, e, fused);
            if (!fused) k_pass_scan<<<dim3(256, ntab), 256, 0, st>>>(job, p, e, last);
            k_pass_scatter<<<dim3(ntiles, ntab), kSortThreads, 0, st>>>(job, p, e, fused, last);
        }
        e++;
    }
    launch_dependent(k_fix_long<J>, dim3(grid_for(cap, 256, sms * 4), ntab), dim3(256), 0, st, job, passes);
}

// Merge sort of a single table's entries (keys from the compaction): the
// runs, every round the capacity may need (rounds beyond the entries' own
// return at once), then the long-word fix-up.
static void launch_msort(const OneJob &job, uint64_t cap, cudaStream_t st) {
    const int grid = (int)std::max<uint64_t>(1, (cap + kMsTile - 1) / kMsTile);
    ensure_smem_limit((const void *)k_ms_runs, (int)kMsSmem);
    ensure_smem_limit((const void *)k_ms_merge, (int)kMsSmem);
    launch_dependent(k_ms_runs, dim3(grid), dim3(kMsThreads), kMsSmem, st, job.j.s, job.j.meta);
    for (int r = 1; r <= ms_rounds(cap); r++)
        launch_dependent(k_ms_merge, dim3(grid), dim3(kMsThreads), kMsSmem, st, job.j.s, job.j.meta, r);
    launch_dependent(k_fix_long<OneJob>, dim3(grid_for(cap, 256, sm_count() * 4)), dim3(256), 0, st, job, kPasses);
}

// LSD radix sort of the entries in ss (count n = meta[0]) into ss.perm_buf(ss.cur[passes]).
cudaError_t sort_entries(SortScratch &ss, const unsigned long long *meta, const LongView &v, int passes,
                         cudaStream_t st, uint32_t skip) {
    OneJob job{SortJob{ss, meta, v, DevTable{}}};
    launch_sort(job, ss.cap, 1, passes, skip, st);
    return cudaGetLastError();
}
int sort_entries_launches(int passes, uint64_t cap, uint32_t skip) {
    const bool fused = (cap + kSortTile - 1) / kSortTile <= kSortFusedMaxTiles;
    const uint32_t mask = passes >= 32 ? ~0u : ((1u << passes) - 1u);
    const int per = cap < (1ull << 30) ? 1 : (fused ? 2 : 3);
    return 1 + 1 + per * (passes - __builtin_popcount(skip & mask));
}

uint32_t sort_skip_mask(uint64_t max_count, uint64_t ndocs) {
    auto bytes_of = [](uint64_t x) {
        int b = 0;
        while (x) { b++; x >>= 8; }
        return b;
    };
    uint32_t m = 0;
    for (int b = bytes_of(max_count); b < 8; b++) m |= 1u << (kSortKeyPasses + b);
    const int db = std::max(1, bytes_of(ndocs ? ndocs - 1 : 0));
    for (int b = db; b < 4; b++) m |= 1u << (kPasses + b);
    return m;
}

// Zeroes a sort's state in one launch: the digit histograms, the pass
// order words, the group histograms, the first look-back buffer and the tile
// counters (the second look-back buffer is zeroed by the first pass).
__global__ void k_sort_reset(SortScratch ss, uint64_t nlook) {
    const uint64_t n0 = (uint64_t)kPassesSeg * 256, n1 = n0 + 32, n2 = n1 + 2ull * 256 * ss.group_stride,
                   n3 = n2 + nlook, n4 = n3 + 2;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < n0) ss.hist_all[i] = 0u;
        else if (i < n1) ss.cur[i - n0] = 0u;
        else if (i < n2) ss.group_hist[0][i - n1] = 0u;
        else if (i < n3) ss.look[0][i - n2] = 0u;
        else ss.tile_ctr[i - n3] = 0u;
    }
}

void sort_state_reset(SortScratch &ss, cudaStream_t st) {
    const uint64_t ntiles = (ss.cap + kSortTile - 1) / kSortTile;
    const uint64_t n = (uint64_t)kPassesSeg * 256 + 32 + 2ull * 256 * ss.group_stride + 256 * ntiles + 2;
    k_sort_reset<<<grid_for(n, 256, sm_count() * 2), 256, 0, st>>>(ss, 256 * ntiles);
}

// Resets the sort state and compacts the three tables in one launch (with
// `keyed`, also preparing the sort keys and histograms).
static void launch_compaction(const GTable &g, uint64_t gcap8, uint64_t gcap, uint64_t glcap, SortScratch &ss,
                              DevTable &out, cudaStream_t st, int prep) {
    const int sms = sm_count();
    sort_state_reset(ss, st);
    const int nb8 = grid_for(gcap8, 256 * kScanUnroll, sms * 8), nb16 = grid_for(gcap, 256 * kScanUnroll, sms * 8),
              nbl = grid_for(glcap, 256, sms * 8);
    launch_dependent(k_compact_all, dim3(nb8 + nb16 + nbl), dim3(256), 0, st, g, (unsigned long long)gcap8,
                     (unsigned long long)gcap, (unsigned long long)glcap, ss, out, (unsigned)nb8, (unsigned)nb16, prep);
}

cudaError_t finish_table(const GTable &g, uint64_t gcap8, uint64_t gcap, uint64_t glcap, SortScratch &ss,
                         DevTable &out, cudaStream_t st, uint32_t skip) {
    const bool ms = use_msort(ss, skip);
    launch_compaction(g, gcap8, gcap, glcap, ss, out, st, ms ? kPrepMerge : kPrepRadix);
    OneJob job{SortJob{ss, out.d_meta, LongView{ss.lref, out.loff, out.llen, out.arena}, out}};
    if (ms) launch_msort(job, ss.cap, st);
    else launch_sort(job, ss.cap, 1, kPasses, skip, st, true);
    launch_dependent(k_gather_final<OneJob>, dim3(grid_for(ss.cap, 256 * kScanUnroll, sm_count() * 8)), dim3(256), 0,
                     st, job);
    return cudaGetLastError();
}

size_t finish_tables_job_bytes(int n) { return sizeof(SortJob) * (size_t)(n > 0 ? n : 1); }
int finish_tables_launches(int n, uint64_t cap, uint32_t skip) {
    return 2 * n + sort_entries_launches(kPasses, cap, skip) + 1;
}

cudaError_t finish_tables(const FinishSpec *spec, int n, void *d_jobs, cudaStream_t st, uint32_t skip) {
    if (n <= 0) return cudaSuccess;
    std::vector<SortJob> jobs((size_t)n);
    uint64_t cap = 0;
    for (int t = 0; t < n; t++) {
        const FinishSpec &f = spec[t];
        launch_compaction(f.g, f.gcap8, f.gcap, f.glcap, *f.ss, *f.out, st, kPrepNone);
        jobs[t] = SortJob{*f.ss, f.out->d_meta, LongView{f.ss->lref, f.out->loff, f.out->llen, f.out->arena}, *f.out};
        cap = std::max<uint64_t>(cap, f.ss->cap);
    }
    cudaError_t e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(SortJob) * jobs.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    JobList list{static_cast<const SortJob *>(d_jobs)};
    launch_sort(list, cap, n, kPasses, skip, st);
    launch_dependent(k_gather_final<JobList>, dim3(grid_for(cap, 256 * kScanUnroll, sm_count() * 8), n), dim3(256), 0,
                     st, list);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- merge
__global__ void k_merge_insert(const MergeSrc *src, const unsigned long long *chunk_start, uint32_t nsrc, GTable g) {
    // table t owns blocks [chunk_start[t], chunk_start[t+1])
    uint32_t lo = 0, hi = nsrc;
    const unsigned long long b = blockIdx.x;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (chunk_start[mid] <= b) lo = mid; else hi = mid;
    }
    const MergeSrc t = src[lo];
    const unsigned long long n = t.meta[0];
    const unsigned long long i0 = (b - chunk_start[lo]) * kMergeChunk;
    for (unsigned long long ib = i0 + (threadIdx.x & ~31u); ib < i0 + kMergeChunk && ib < n; ib += blockDim.x) {
        const unsigned long long i = ib + (threadIdx.x & 31);  // whole warps iterate together
        const bool valid = i < i0 + kMergeChunk && i < n;
        unsigned long long c = 0;
        uint32_t r = 0;
        if (valid) {
            c = t.count_bits == 32 ? static_cast<const uint32_t *>(t.cnt)[i]
                                   : static_cast<const unsigned long long *>(t.cnt)[i];
            r = t.lref[i];
        }
        if (valid && r == 0) {
            unsigned long long hi8 = t.khi[i], lo8 = t.klo[i];
            uint4 k;
            k.x = __byte_perm((uint32_t)(hi8 >> 32), 0, 0x0123);
            k.y = __byte_perm((uint32_t)hi8, 0, 0x0123);
            k.z = __byte_perm((uint32_t)(lo8 >> 32), 0, 0x0123);
            k.w = __byte_perm((uint32_t)lo8, 0, 0x0123);
            table_insert_key(g, k, c);
        }
        if (valid && r != 0)
            long_insert(g, t.arena + t.loff[r - 1], t.llen[r - 1], c, nullptr, nullptr);
    }
}

cudaError_t launch_merge_insert(const MergeSrc *d_src, const uint64_t *d_chunk_start, uint32_t nsrc,
                                uint64_t total_chunks, const GTable &g, cudaStream_t s) {
    if (total_chunks == 0) return cudaSuccess;
    k_merge_insert<<<(unsigned)total_chunks, 256, 0, s>>>(d_src, reinterpret_cast<const unsigned long long *>(d_chunk_start), nsrc, g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- top-k
__global__ void k_topk_copy(DevTable in, unsigned long long k, DevTable out) {
    const unsigned long long n = in.d_meta[0];
    const unsigned long long m = n < k ? n : k;
    const unsigned long long nl = in.d_meta[1], ab = in.d_meta[2];
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        out.d_meta[0] = m;
        out.d_meta[1] = nl;
        out.d_meta[2] = ab;
        *out.d_status = *in.d_status;
    }
    unsigned long long tok = 0, bytes = 0;
    for (unsigned long long i = t; i < m; i += stride) {
        out.khi[i] = in.khi[i];
        out.klo[i] = in.klo[i];
        uint32_t r = in.lref[i];
        out.lref[i] = r;
        unsigned long long c;
        if (in.count_bits == 32) c = static_cast<const uint32_t *>(in.cnt)[i];
        else c = static_cast<const unsigned long long *>(in.cnt)[i];
        if (out.count_bits == 32) static_cast<uint32_t *>(out.cnt)[i] = (uint32_t)c;
        else static_cast<unsigned long long *>(out.cnt)[i] = c;
        tok += c;
        bytes += r ? in.llen[r - 1] : short_len(in.khi[i], in.klo[i]);
    }
    for (unsigned long long i = t; i < nl; i += stride) {
        out.loff[i] = in.loff[i];
        out.llen[i] = in.llen[i];
    }
    for (unsigned long long i = t; i < ab; i += stride) out.arena[i] = in.arena[i];
    for (int d = 16; d; d >>= 1) {
        tok += __shfl_xor_sync(kFull, tok, d);
        bytes += __shfl_xor_sync(kFull, bytes, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (tok) atomicAdd(&out.d_meta[3], tok);
        if (bytes) atomicAdd(&out.d_meta[4], bytes);
    }
}

cudaError_t launch_topk_copy(const DevTable &in, uint64_t k, DevTable &out, cudaStream_t s) {
    uint64_t work = in.cap > in.arena_cap ? in.cap : in.arena_cap;
    k_topk_copy<<<grid_for(work, 256, sm_count() * 8), 256, 0, s>>>(in, k, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- export
constexpr int kScanBlock = 1024;  // elements per scan block (256 threads x 4)

size_t export_scratch_bytes(uint64_t cap) {
    uint64_t nb = (cap + kScanBlock - 1) / kScanBlock;
    return (nb + 8) * 8 + 256;
}

__global__ void k_export_lens(DevTable t, unsigned long long *offs, unsigned long long *blocksum) {
    __shared__ unsigned long long part[256];
    const unsigned long long n = t.d_meta[0];
    const unsigned long long b0 = (unsigned long long)blockIdx.x * kScanBlock;
    if (b0 >= n && !(n == 0 && blockIdx.x == 0)) return;
    unsigned long long v[4], sum = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        unsigned long long i = b0 + threadIdx.x * 4 + j;
        unsigned long long len = 0;
        if (i < n) {
            uint32_t r = t.lref[i];
            len = r ? t.llen[r - 1] : short_len(t.khi[i], t.klo[i]);
        }
        v[j] = len;
        sum += len;
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < 256; d <<= 1) {
        unsigned long long x = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0ull;
        __syncthreads();
        part[threadIdx.x] += x;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - sum;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        unsigned long long i = b0 + threadIdx.x * 4 + j;
        if (i < n) offs[i] = run;
        run += v[j];
    }
    if (threadIdx.x == 255) blocksum[blockIdx.x] = part[255];
}

// Exclusive scan of the scan blocks' byte counts, in one block: each thread
// sums a contiguous run of them, the run totals are scanned in shared
// memory, and each thread writes its run's prefixes.
constexpr int kBlockSumThreads = 1024;
__global__ void __launch_bounds__(kBlockSumThreads) k_export_blocksums(const DevTable t, unsigned long long *blocksum,
                                                                       unsigned long long *offs) {
    __shared__ unsigned long long part[kBlockSumThreads];
    const unsigned long long n = t.d_meta[0];
    const unsigned long long nb = (n + kScanBlock - 1) / kScanBlock;
    const unsigned long long per = (nb + kBlockSumThreads - 1) / kBlockSumThreads;
    const unsigned long long lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    unsigned long long own = 0;
    for (unsigned long long b = lo; b < hi; b++) own += blocksum[b];
    part[threadIdx.x] = own;
    __syncthreads();
    for (int o = 1; o < kBlockSumThreads; o <<= 1) {
        const unsigned long long x = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
        __syncthreads();
        part[threadIdx.x] += x;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - own;
    for (unsigned long long b = lo; b < hi; b++) {
        const unsigned long long v = blocksum[b];
        blocksum[b] = run;
        run += v;
    }
    if (threadIdx.x == kBlockSumThreads - 1) offs[n] = part[kBlockSumThreads - 1];
}

__global__ void k_export_write(DevTable t, unsigned long long *offs, const unsigned long long *blocksum, uint8_t *words) {
    const unsigned long long n = t.d_meta[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long o = offs[i] + blocksum[i / kScanBlock];
        offs[i] = o;
        uint32_t r = t.lref[i];
        if (r) {
            const uint8_t *p = t.arena + t.loff[r - 1];
            unsigned long long len = t.llen[r - 1];
            for (unsigned long long j = 0; j < len; j++) words[o + j] = p[j];
        } else {
            unsigned long long hi = t.khi[i], lo = t.klo[i];
            unsigned long long len = short_len(hi, lo);
            for (unsigned long long j = 0; j < len; j++)
                words[o + j] = (uint8_t)((j < 8 ? hi >> (56 - 8 * j) : lo >> (56 - 8 * (j - 8))) & 0xFF);
        }
    }
}

cudaError_t launch_export(const DevTable &t, void *scratch, uint8_t *d_words, unsigned long long *d_offs,
                          cudaStream_t s) {
    unsigned long long *blocksum = static_cast<unsigned long long *>(scratch);
    const int nb = (int)((t.cap + kScanBlock - 1) / kScanBlock);
    k_export_lens<<<nb > 0 ? nb : 1, 256, 0, s>>>(t, d_offs, blocksum);
    k_export_blocksums<<<1, kBlockSumThreads, 0, s>>>(t, blocksum, d_offs);
    k_export_write<<<grid_for(t.cap, 256, sm_count() * 8), 256, 0, s>>>(t, d_offs, blocksum, d_words);
    return cudaGetLastError();
}

}  // namespace wc
