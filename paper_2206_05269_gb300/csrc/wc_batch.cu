// Batched counting: many documents of uneven size in one pass.
//
// Sec. 3.1 of the paper builds one dictionary per document and Sec. 3.3 sums
// them; here every document's table is built on the GPU.  One persistent
// kernel per size class walks a device work queue of items:
//  - a whole document (sizes up to the split threshold): one block counts it
//    into a shared-memory table (dynamic inserts, 16-byte keys) with words of
//    17+ letters in a small shared list, sorts the entries by (count desc,
//    word asc) with a bitonic network in shared memory and writes them into
//    the CSR output at an atomically reserved offset;
//  - a byte range of a large document: the block counts the range (words
//    that start in it, read past its end as needed) and adds its table into
//    global tables keyed by (document, word).
// A whole document whose shared table fills up spills the rest of its words
// (and, at the end, its shared table) to the same global tables.  Documents
// counted there are finished by a segmented pass: compaction, a radix sort
// with the document as most significant key, and a CSR write.
#include "wc_batch.h"

namespace wc {

// ---------------------------------------------------------------- (doc, word) keys
// Letter bytes are 0x61..0x7A: their low 5 bits (1..26) name the letter and
// bits 5-7 are always 011; padding bytes are 0.  So bits 5-7 of each key byte
// can carry 3 bits of the document number and be restored afterwards.
constexpr unsigned long long kCodeMask = 0x1F1F1F1F1F1F1F1Full;
__device__ __forceinline__ unsigned long long spread_doc(uint32_t d) {  // 24 bits -> bits 5..7 of 8 bytes
    unsigned long long r = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) r |= (unsigned long long)((d >> (3 * i)) & 7u) << (8 * i + 5);
    return r;
}
__device__ __forceinline__ uint32_t gather_doc(unsigned long long k) {
    uint32_t d = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) d |= (uint32_t)((k >> (8 * i + 5)) & 7u) << (3 * i);
    return d;
}
__device__ __forceinline__ unsigned long long restore_letters(unsigned long long k) {
    unsigned long long c = k & kCodeMask;
    unsigned long long nz = (c + 0x7F7F7F7F7F7F7F7Full) & 0x8080808080808080ull;  // 0x80 where code != 0
    return c | (nz >> 1) | (nz >> 2);
}
__device__ __forceinline__ unsigned long long long_doc_hash(unsigned long long h, uint32_t d) {
    if (kOneSlot) return h;  // test build: one home slot for every document's long words
    return h ^ fmix64((unsigned long long)d + 0x632BE59BD9B4E019ull);
}

// Adds `add` to word k (<= 16 letters) of document d in the global tables.
__device__ __forceinline__ void doc_insert_key(const GTable &g, uint32_t d, uint4 k, unsigned long long add) {
    const unsigned long long lo = ((unsigned long long)k.y << 32) | k.x, hi = ((unsigned long long)k.w << 32) | k.z;
    if (hi == 0ull) {
        global_insert8(g, (lo & kCodeMask) | spread_doc(d & 0xFFFFFFu), add);
    } else {
        const unsigned long long l2 = (lo & kCodeMask) | spread_doc(d & 0xFFFFFFu);
        const unsigned long long h2 = (hi & kCodeMask) | spread_doc(d >> 24);
        global_insert16(g, make_uint4((uint32_t)l2, (uint32_t)(l2 >> 32), (uint32_t)h2, (uint32_t)(h2 >> 32)), add);
    }
}
__device__ __forceinline__ void doc_insert_long(const GTable &g, uint32_t d, const uint8_t *w, unsigned long long len,
                                                unsigned long long add, const uint8_t *begin, const uint8_t *end) {
    long_insert2(g, w, len, long_doc_hash(long_hash(w, len), d), add, begin, end);
}

__device__ __forceinline__ unsigned long long be64b(uint32_t x, uint32_t y) {
    return ((unsigned long long)__byte_perm(x, 0, 0x0123) << 32) | __byte_perm(y, 0, 0x0123);
}
__device__ __forceinline__ unsigned long long be_bytes16(const uint8_t *src, int from) {  // lowercased, big endian
    unsigned long long v = 0;
    for (int j = from; j < from + 8; j++) v = (v << 8) | (unsigned long long)(src[j] | 0x20u);
    return v;
}

// 128-bit sort composite of a per-document entry: count (16 bits, stored as
// 0xFFFF - count so that a larger count sorts first), the 16-letter prefix
// packed 5 bits a letter (80 bits, pack5 of the big-endian key halves), a
// long-word flag and the long word's index.  Documents counted in shared
// memory hold at most 64 KB, so counts stay below 2^16.
__device__ __forceinline__ ulonglong2 doc_composite(unsigned long long khi, unsigned long long klo, uint32_t cnt,
                                                   bool is_long, uint32_t idx) {
    const unsigned long long ph = pack5(khi), pl = pack5(klo);  // 40 bits each
    const unsigned long long c = 0xFFFFull - (cnt > 0xFFFFu ? 0xFFFFu : cnt);
    const unsigned long long hi = (c << 48) | (ph << 8) | (pl >> 32);
    const unsigned long long lo = ((pl & 0xFFFFFFFFull) << 32) | ((unsigned long long)is_long << 31) | (idx & 0x7FFFFFFFu);
    return make_ulonglong2(hi, lo);
}
__device__ __forceinline__ void doc_decompose(ulonglong2 k, unsigned long long *khi, unsigned long long *klo,
                                              uint32_t *cnt) {
    *cnt = 0xFFFFu - (uint32_t)(k.x >> 48);
    *khi = unpack5((k.x >> 8) & 0xFFFFFFFFFFull);
    *klo = unpack5(((k.x & 0xFFull) << 32) | (k.y >> 32));
}

// ---------------------------------------------------------------- per-document shared table
// A document's shared table holds 16-byte keys claimed whole by a 128-bit
// CAS, so a word can never occupy two slots.  A word of at most 8 letters is
// stored with byte 8 set to 1 (never a letter), so neither half of a stored
// key is ever zero: a 16-byte load that shows a zero half is empty or a
// claim in flight (possibly of this very word), settled by the CAS, which
// returns the whole key; a load that shows two non-zero halves equal to the
// word's can only come from that word's slot.
__device__ __forceinline__ uint4 mark_key(uint4 k) {
    if ((k.z | k.w) == 0u) k.z = 1u;
    return k;
}
__device__ __forceinline__ uint4 unmark_key(uint4 k) {
    if (k.z == 1u && k.w == 0u) k.z = 0u;
    return k;
}
__device__ __forceinline__ ulonglong2 lds128(const uint4 *p) {
    ulonglong2 v;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ uint4 cas128_shared(uint4 *p, uint4 val) {  // compare with zero
    const uint64_t v0 = ((uint64_t)val.y << 32) | val.x, v1 = ((uint64_t)val.w << 32) | val.z;
    uint64_t r0, r1;
    asm volatile(
        "{\n\t.reg .b128 c, v, d;\n\t"
        "mov.b128 c, {%2, %2};\n\t"
        "mov.b128 v, {%3, %4};\n\t"
        "atom.relaxed.cta.shared::cta.cas.b128 d, [%5], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(r0), "=l"(r1)
        : "l"(0ull), "l"(v0), "l"(v1), "r"((uint32_t)__cvta_generic_to_shared(p))
        : "memory");
    return make_uint4((uint32_t)r0, (uint32_t)(r0 >> 32), (uint32_t)r1, (uint32_t)(r1 >> 32));
}
// Adds 1 to marked key km from home slot s; false when the word must spill
// (the probe limit, or an empty slot found with the table filled to its limit).
__device__ __forceinline__ bool doc_table_add(uint4 *skey, uint32_t *scnt, uint32_t *nfill, uint32_t mask,
                                              uint32_t fill_limit, uint4 km, uint32_t s, int max_probe) {
    const unsigned long long k0 = ((unsigned long long)km.y << 32) | km.x, k1 = ((unsigned long long)km.w << 32) | km.z;
    for (int probe = 0; probe < max_probe; probe++) {
        const ulonglong2 c = lds128(skey + s);
        bool hit = c.x == k0 && c.y == k1;
        if (!hit && (c.x == 0ull || c.y == 0ull)) {
            if (c.x == 0ull && c.y == 0ull && *(volatile uint32_t *)nfill >= fill_limit) return false;
            const uint4 old = cas128_shared(skey + s, km);
            if (key_zero(old)) {
                atomicAdd(nfill, 1u);
                hit = true;
            } else {
                hit = key_eq(old, km);
            }
        }
        if (hit) {
            atomicAdd(scnt + s, 1u);
            return true;
        }
        s = (s + 1u) & mask;
    }
    return false;
}

// ---------------------------------------------------------------- per-document kernel
template <int BLOCK, int LOGC1>
struct DocCfg {
    static constexpr int W = BLOCK / 32;
    static constexpr int CH = W * 512;         // one strip per warp
    static constexpr int WINB = CH + 96;
    static constexpr int C1 = 1 << LOGC1;
    static constexpr int TOKCAP = 32 + 256;
    static constexpr int LCAP = 64;            // distinct long words per document in shared memory
    static constexpr uint32_t FILL = C1 * 3 / 4;
    static constexpr size_t SMEM = (size_t)WINB + (size_t)W * TOKCAP * 4 +  // window + queues (sort buffer)
                                   (size_t)C1 * 16 + (size_t)C1 * 4 +  // keys, counts
                                   (size_t)LCAP * (8 + 8 + 4 + 4 + 16) + 16 + 64;
    static_assert((size_t)WINB + (size_t)W * TOKCAP * 4 >= (size_t)C1 * 2, "sort buffer must fit");
    // blocks per SM that the shared memory allows: the register budget follows
    static constexpr int MINB = (int)((227u * 1024u) / SMEM) < 1 ? 1 : ((int)((227u * 1024u) / SMEM) > 8 ? 8 : (int)((227u * 1024u) / SMEM));
    static_assert(C1 <= 32768, "16-bit sort indices");
};

struct DocShared {  // per-block scalars
    uint32_t item;
    uint32_t lcount;
    uint32_t nfill;
    uint32_t spilled;
    uint32_t nent;
    uint32_t nlong;
    unsigned long long base, lbase, abase;
    uint32_t ok;
};

template <int BLOCK, int LOGC1>
__global__ void __launch_bounds__(BLOCK, (DocCfg<BLOCK, LOGC1>::MINB)) k_docs(BatchArgs a) {
    using C = DocCfg<BLOCK, LOGC1>;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *win = smem;
    uint32_t *tokall = reinterpret_cast<uint32_t *>(smem + C::WINB);
    uint16_t *sidx = reinterpret_cast<uint16_t *>(smem);  // sort buffer, reuses window + queues
    uint4 *skey = reinterpret_cast<uint4 *>(smem + C::WINB + (size_t)C::W * C::TOKCAP * 4);
    uint32_t *scnt = reinterpret_cast<uint32_t *>(skey + C::C1);
    unsigned long long *laddr = reinterpret_cast<unsigned long long *>(scnt + C::C1);
    unsigned long long *llen = laddr + C::LCAP;
    uint32_t *lcnt = reinterpret_cast<uint32_t *>(llen + C::LCAP);
    uint32_t *lrank = lcnt + C::LCAP;
    ulonglong2 *lkey = reinterpret_cast<ulonglong2 *>(lrank + C::LCAP);
    __shared__ DocShared sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *tok = tokall + warp * C::TOKCAP;
    const uintptr_t tb = reinterpret_cast<uintptr_t>(a.text);
    // The size classes' kernels work on separate item queues: a later one
    // may start as soon as this one's blocks have all started (its blocks
    // then fill the SMs this one's finished blocks leave), and waits for this
    // one only at its end, so that its completion implies this one's.
    grid_dependency_trigger();

    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(a.next_item, 1u);
        __syncthreads();
        const uint32_t item = sh.item;
        if (item >= a.nitems) break;
        const DocItem it = a.items[item];
        const uint32_t d = it.doc;
        const uintptr_t vb = tb + a.doc_off[d], ve = tb + a.doc_off[d + 1];
        const uintptr_t own_lo = tb + it.lo, own_hi = tb + it.hi;
        const uint8_t *dbeg = reinterpret_cast<const uint8_t *>(vb);
        const uint8_t *dend = reinterpret_cast<const uint8_t *>(ve);
        // The slots this item uses: a whole document takes a power of two
        // of about a quarter of its bytes (at least BLOCK; three quarters of
        // it may fill before words spill), so that the clearing, merging and
        // composite passes below scale with the document; ranges take all.
        uint32_t ceff = C::C1;
        if (!it.kind) {
            const unsigned long long want = (it.hi - it.lo) / 4;
            ceff = BLOCK;
            while (ceff < (uint32_t)C::C1 && ceff < want) ceff <<= 1;
        }
        const uint32_t fill_limit = ceff / 4u * 3u;
        for (int i = threadIdx.x; i < (int)ceff; i += BLOCK) {
            skey[i] = make_uint4(0u, 0u, 0u, 0u);
            scnt[i] = 0u;
        }
        if (threadIdx.x == 0) {
            sh.lcount = 0;
            sh.nfill = 0;
            sh.spilled = it.kind;  // ranges always go to the global tables
        }
        for (int i = threadIdx.x; i < C::LCAP; i += BLOCK) laddr[i] = 0ull;
        __syncthreads();

        auto process = [&](bool have, uint32_t e) {
            if (have) {
                const uint32_t p = e >> 5, len = e & 31u;
                uint4 k = load_key16(win, p, len);
                if (!doc_table_add(skey, scnt, &sh.nfill, ceff - 1u, fill_limit, mark_key(k),
                                   (uint32_t)(hash_key(k) >> 40) & (ceff - 1u), (int)ceff)) {
                    doc_insert_key(a.g, d, k, 1ull);
                    sh.spilled = 1u;
                }
            }
        };

        // The window of the next chunk is loaded one chunk ahead: each thread
        // keeps its (at most two) 16-byte pieces in registers while the
        // current chunk is processed, and masks the document's edges when
        // it stores them.
        static_assert(C::WINB / 16 <= 2 * BLOCK, "two window pieces per thread");
        const int t1 = threadIdx.x + BLOCK;
        auto fetch = [&](uintptr_t w0, uint4 &v0, uint4 &v1) {
            const uintptr_t a0 = w0 + 16 * (uintptr_t)threadIdx.x, a1 = w0 + 16 * (uintptr_t)t1;
            v0 = v1 = make_uint4(0x20202020u, 0x20202020u, 0x20202020u, 0x20202020u);
            if (a0 < ve && a0 + 16 > vb) v0 = ld_stream16(reinterpret_cast<const void *>(a0));
            if (t1 < C::WINB / 16 && a1 < ve && a1 + 16 > vb) v1 = ld_stream16(reinterpret_cast<const void *>(a1));
        };
        auto stage = [&](uintptr_t w0, uint4 v0, uint4 v1) {
            const uintptr_t a0 = w0 + 16 * (uintptr_t)threadIdx.x, a1 = w0 + 16 * (uintptr_t)t1;
            if (a0 < ve && a0 + 16 > vb && (a0 < vb || a0 + 16 > ve)) v0 = mask_outside_doc(v0, a0, vb, ve);
            *reinterpret_cast<uint4 *>(win + 16 * threadIdx.x) = v0;
            if (t1 < C::WINB / 16) {
                if (a1 < ve && a1 + 16 > vb && (a1 < vb || a1 + 16 > ve)) v1 = mask_outside_doc(v1, a1, vb, ve);
                *reinterpret_cast<uint4 *>(win + 16 * t1) = v1;
            }
        };
        uint4 nx0, nx1;
        fetch((own_lo & ~(uintptr_t)15) - 16, nx0, nx1);
        for (uintptr_t cs = own_lo & ~(uintptr_t)15; cs < own_hi; cs += C::CH) {
            const uintptr_t w0 = cs - 16;
            stage(w0, nx0, nx1);
            __syncthreads();
            if (cs + C::CH < own_hi) fetch(w0 + C::CH, nx0, nx1);
            // ---- this warp's strip
            const int sbase = 16 + 512 * warp;
            const uint32_t prevL = is_letter(win[sbase - 1]) ? 1u : 0u;
            const uint32_t L = letter_mask16(*reinterpret_cast<const uint4 *>(win + sbase + 16 * lane));
            const uint32_t Ln = letter_mask16(*reinterpret_cast<const uint4 *>(win + sbase + 512));
            const uint32_t up = __shfl_up_sync(kFull, L, 1);
            const uint32_t dn = __shfl_down_sync(kFull, L, 1);
            const uint32_t pbit = lane == 0 ? prevL : ((up >> 15) & 1u);
            const uint32_t Wm = L | ((lane == 31 ? Ln : dn) << 16);
            uint32_t S = L & ~((L << 1) | pbit) & 0xFFFFu;
            {   // only words that start inside this item's byte range
                const uintptr_t A = w0 + sbase + 16 * lane;
                long long lo = (long long)(own_lo - A), hi = (long long)(own_hi - A);
                int klo = (int)(lo < 0 ? 0 : (lo > 16 ? 16 : lo)), khi = (int)(hi < 0 ? 0 : (hi > 16 ? 16 : hi));
                uint32_t m = (khi > klo) ? (((1u << khi) - 1u) & ~((1u << klo) - 1u)) : 0u;
                S &= m;
            }
            uint32_t x = Wm;
            x &= x >> 1; x &= x >> 2; x &= x >> 4; x &= x >> 8; x &= Wm >> 16;
            uint32_t Ss = S & ~x, Sl = S & x;
            const uint32_t c1 = __popc(Ss);
            uint32_t incl = c1;
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                uint32_t t = __shfl_up_sync(kFull, incl, dd);
                if (lane >= dd) incl += t;
            }
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            uint32_t off = incl - c1;
            const uint32_t pbase = (uint32_t)(sbase + 16 * lane);
            while (Ss) {
                int j = __ffs(Ss) - 1;
                Ss &= Ss - 1;
                tok[off++] = ((pbase + (uint32_t)j) << 5) | ((uint32_t)__ffs(~(Wm >> j)) - 1u);
            }
            // long words: the whole warp handles each in turn
            uint32_t pend = __ballot_sync(kFull, Sl != 0);
            while (pend) {
                const int who = __ffs(pend) - 1;
                unsigned long long wa = 0;
                if (lane == who) {
                    int j = __ffs(Sl) - 1;
                    Sl &= Sl - 1;
                    wa = (unsigned long long)(w0 + pbase + (uint32_t)j);
                }
                wa = __shfl_sync(kFull, wa, who);
                pend = __ballot_sync(kFull, Sl != 0);
                const uint8_t *w = reinterpret_cast<const uint8_t *>(wa);
                unsigned long long len = 0;
                for (unsigned long long o = 0;; o += 32) {
                    const uint8_t *q = w + o + lane;
                    uint32_t bb = q < dend ? *q : 0x20u;
                    uint32_t m = __ballot_sync(kFull, !is_letter(bb));
                    if (m) { len = o + (unsigned long long)(__ffs(m) - 1); break; }
                }
                bool found = false;
                const uint32_t lc = *(volatile uint32_t *)&sh.lcount;
                for (uint32_t j = 0; j < lc && j < (uint32_t)C::LCAP && !found; j++) {
                    const unsigned long long ra = *(volatile unsigned long long *)&laddr[j];
                    if (!ra || *(volatile unsigned long long *)&llen[j] != len) continue;
                    const uint8_t *r = reinterpret_cast<const uint8_t *>(ra);
                    bool ok = true;
                    for (unsigned long long q = lane; q < len; q += 32) ok &= ((r[q] | 0x20u) == (w[q] | 0x20u));
                    if (__all_sync(kFull, ok)) {
                        if (lane == 0) atomicAdd(&lcnt[j], 1u);
                        found = true;
                    }
                }
                if (!found) {
                    uint32_t slot = 0;
                    if (lane == 0) slot = atomicAdd(&sh.lcount, 1u);
                    slot = __shfl_sync(kFull, slot, 0);
                    if (slot < (uint32_t)C::LCAP) {
                        if (lane == 0) {
                            llen[slot] = len;
                            lcnt[slot] = 1u;
                            __threadfence_block();
                            *(volatile unsigned long long *)&laddr[slot] = wa;
                        }
                    } else {
                        if (lane == 0) {
                            doc_insert_long(a.g, d, w, len, 1ull, dbeg, dend);
                            sh.spilled = 1u;
                        }
                    }
                }
                __syncwarp();
            }
            __syncwarp();
            uint32_t bq = 0;
            for (; bq + 32 <= total; bq += 32) process(true, tok[bq + lane]);
            process((uint32_t)lane < total - bq, (uint32_t)lane < total - bq ? tok[bq + lane] : 0u);
            __syncthreads();  // the window is about to be overwritten
        }
        if (threadIdx.x == 0 && sh.lcount > (uint32_t)C::LCAP) sh.lcount = C::LCAP;
        __syncthreads();

        if (sh.spilled) {
            // ---- range or overflowing document: add everything to the global tables
            for (int i = threadIdx.x; i < (int)ceff; i += BLOCK)
                if (!key_zero(skey[i])) doc_insert_key(a.g, d, unmark_key(skey[i]), (unsigned long long)scnt[i]);
            for (uint32_t j = threadIdx.x; j < sh.lcount; j += BLOCK)
                doc_insert_long(a.g, d, reinterpret_cast<const uint8_t *>(laddr[j]), llen[j],
                                (unsigned long long)lcnt[j], dbeg, dend);
            if (threadIdx.x == 0) atomicOr(&a.doc_flags[d], 1u);
            __syncthreads();
            continue;
        }

        // merge duplicate long entries (warp 0)
        const uint32_t nl = sh.lcount;
        if (warp == 0) {
            for (uint32_t i = 1; i < nl; i++) {
                for (uint32_t j = 0; j < i; j++) {
                    if (lcnt[j] == 0u || llen[j] != llen[i]) continue;
                    const uint8_t *p = reinterpret_cast<const uint8_t *>(laddr[i]);
                    const uint8_t *q = reinterpret_cast<const uint8_t *>(laddr[j]);
                    bool ok = true;
                    for (unsigned long long k = lane; k < llen[i]; k += 32) ok &= ((p[k] | 0x20u) == (q[k] | 0x20u));
                    if (__all_sync(kFull, ok)) {
                        if (lane == 0) { lcnt[j] += lcnt[i]; lcnt[i] = 0u; }
                        __syncwarp();
                        break;
                    }
                }
            }
        }
        // Every live entry becomes a 128-bit composite in place (its count,
        // its 16-letter prefix packed 5 bits a letter, a long-word flag and
        // index): integer order on composites is the output order (count
        // desc, word asc) except among long words sharing a prefix, which a
        // fix-up orders below.  The sort then moves 16-bit indices and
        // compares composites.
        if (threadIdx.x == 0) {
            sh.nent = 0;
            sh.nlong = 0;
        }
        __syncthreads();
        // composites in place, and the index list of live entries (its order
        // is fixed by the sort below): one shared atomic per warp and step
        static_assert(C::C1 % BLOCK == 0, "whole steps over the shared table");
        for (int i0 = 0; i0 < (int)ceff; i0 += BLOCK) {
            const int i = i0 + threadIdx.x;
            const uint4 km = skey[i];
            const bool live = !key_zero(km);
            if (live) {
                const uint4 k = unmark_key(km);
                reinterpret_cast<ulonglong2 *>(skey)[i] =
                    doc_composite(be64b(k.x, k.y), be64b(k.z, k.w), scnt[i], false, 0u);
            }
            const uint32_t m = __ballot_sync(kFull, live);
            uint32_t base = 0;
            if (lane == 0 && m) base = atomicAdd(&sh.nent, (uint32_t)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (live) sidx[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)i;
        }
        for (uint32_t j = threadIdx.x; j < nl; j += BLOCK) {
            const uint8_t *p = reinterpret_cast<const uint8_t *>(laddr[j]);
            lkey[j] = doc_composite(be_bytes16(p, 0), be_bytes16(p, 8), lcnt[j], true, j);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t r = 0;
            for (uint32_t j = 0; j < nl; j++) {
                if (lcnt[j]) { lrank[j] = r++; sidx[sh.nent++] = (uint16_t)(C::C1 + j); }
            }
            sh.nlong = r;
        }
        __syncthreads();
        const uint32_t n = sh.nent;
        uint32_t N = 1;
        while (N < n) N <<= 1;
        __syncthreads();
        auto key_of = [&](uint32_t s) -> ulonglong2 {
            return s < (uint32_t)C::C1 ? reinterpret_cast<const ulonglong2 *>(skey)[s] : lkey[s - C::C1];
        };
        // Bitonic network over N = 2^m >= n positions, every merge ascending:
        // its first stage compares each position of a block's lower half with
        // its mirror in the upper half, the later stages with the position j
        // above.  Positions from n on stand for entries above every real
        // one, so a pair that reaches one never swaps and is skipped: the
        // padding is never touched.  The pairs of thread t lie in the 64
        // positions from 64 * (t / 32) while a stage works within blocks of
        // at most 64, so a warp owns the same positions through consecutive
        // such stages and only a change to or from a wider stage needs a
        // block-wide barrier.
        for (uint32_t k = 2; k <= N; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const bool mirror = j == (k >> 1);
                for (uint32_t t = threadIdx.x; t < N / 2; t += BLOCK) {
                    const uint32_t i = 2 * t - (t & (j - 1)), q = mirror ? (i ^ (k - 1)) : i + j;
                    if (q >= n) continue;
                    const uint32_t x = sidx[i], y = sidx[q];
                    const ulonglong2 kx = key_of(x), ky = key_of(y);
                    if (ky.x != kx.x ? ky.x < kx.x : ky.y < kx.y) { sidx[i] = (uint16_t)y; sidx[q] = (uint16_t)x; }
                }
                const uint32_t span = 2 * j, span_next = j > 1 ? j : 2 * k;  // block sizes of this and the next stage
                if (span <= 64 && span_next <= 64) __syncwarp();
                else __syncthreads();
            }
        }
        __syncthreads();
        // long words with equal count and prefix: order by their remaining
        // bytes (insertion over each such run; runs are rare and short)
        if (sh.nlong) {
            if (threadIdx.x == 0) sh.ok = 0u;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i + 1 < n; i += BLOCK) {
                const ulonglong2 a0 = key_of(sidx[i]), a1 = key_of(sidx[i + 1]);
                if ((a1.y >> 31) & 1u && a0.x == a1.x && (a0.y >> 32) == (a1.y >> 32)) sh.ok = 2u;
            }
            __syncthreads();
            if (sh.ok == 2u && threadIdx.x == 0) {
                for (uint32_t a = 1; a < n; a++) {
                    const uint32_t x = sidx[a];
                    const ulonglong2 kx = key_of(x);
                    if (!((kx.y >> 31) & 1u)) continue;  // only long words move
                    uint32_t b = a;
                    while (b > 0) {
                        const uint32_t y = sidx[b - 1];
                        const ulonglong2 ky = key_of(y);
                        if (ky.x != kx.x || (ky.y >> 32) != (kx.y >> 32) || !((ky.y >> 31) & 1u)) break;
                        const uint32_t jx = x - C::C1, jy = y - C::C1;
                        const uint8_t *px = reinterpret_cast<const uint8_t *>(laddr[jx]);
                        const uint8_t *py = reinterpret_cast<const uint8_t *>(laddr[jy]);
                        const unsigned long long nx = llen[jx], ny = llen[jy], m = nx < ny ? nx : ny;
                        int c = 0;
                        for (unsigned long long q = 16; q < m && !c; q++) {
                            const uint32_t bx = px[q] | 0x20u, by = py[q] | 0x20u;
                            c = bx < by ? -1 : (bx > by ? 1 : 0);
                        }
                        if (!(c < 0 || (c == 0 && nx < ny))) break;
                        sidx[b] = (uint16_t)y;
                        b--;
                    }
                    sidx[b] = (uint16_t)x;
                }
            }
            __syncthreads();
        }
        // reserve output: entries, long words, arena bytes
        if (threadIdx.x == 0) {
            unsigned long long ab = 0;
            for (uint32_t j = 0; j < nl; j++)
                if (lcnt[j]) ab += llen[j] + 1;
            sh.base = atomicAdd(&a.meta[0], (unsigned long long)n);
            sh.lbase = sh.nlong ? atomicAdd(&a.meta[1], (unsigned long long)sh.nlong) : 0ull;
            sh.abase = ab ? atomicAdd(&a.meta[2], ab) : 0ull;
            sh.ok = (sh.base + n <= a.out_cap && sh.lbase + sh.nlong <= a.lcap && sh.abase + ab <= a.arena_cap);
            if (!sh.ok) atomicOr(a.status, ST_OUT_FULL);
            a.doc_start[d] = sh.base;
            a.doc_n[d] = sh.ok ? n : 0u;
        }
        __syncthreads();
        if (sh.ok) {
            const unsigned long long base = sh.base;
            for (uint32_t i = threadIdx.x; i < n; i += BLOCK) {
                const uint32_t s = sidx[i];
                unsigned long long khi, klo;
                uint32_t cnt;
                doc_decompose(key_of(s), &khi, &klo, &cnt);
                a.out_khi[base + i] = khi;
                a.out_klo[base + i] = klo;
                a.out_cnt[base + i] = cnt;
                a.out_lref[base + i] = s < (uint32_t)C::C1 ? 0u : (uint32_t)(sh.lbase + lrank[s - C::C1] + 1);
            }
            if (warp == 0 && sh.nlong) {
                unsigned long long ao = sh.abase;
                for (uint32_t j = 0; j < nl; j++) {
                    if (!lcnt[j]) continue;
                    const uint8_t *p = reinterpret_cast<const uint8_t *>(laddr[j]);
                    const unsigned long long len = llen[j];
                    for (unsigned long long q = lane; q < len; q += 32) a.arena[ao + q] = (uint8_t)(p[q] | 0x20u);
                    if (lane == 0) {
                        a.arena[ao + len] = 0;
                        a.loff[sh.lbase + lrank[j]] = ao;
                        a.llen[sh.lbase + lrank[j]] = len;
                    }
                    ao += len + 1;
                }
            }
        }
        __syncthreads();
    }
    grid_dependency_wait();  // the previous size class's kernel has completed (a no-op after an ordinary launch)
}

template <int BLOCK, int LOGC1>
cudaError_t launch_docs_t(const BatchArgs &a, int grid, cudaStream_t s, bool dependent) {
    using C = DocCfg<BLOCK, LOGC1>;
    const cudaError_t ea = ensure_smem_limit((const void *)k_docs<BLOCK, LOGC1>, (int)C::SMEM);
    if (ea != cudaSuccess) return ea;
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_docs<BLOCK, LOGC1>, BLOCK, C::SMEM);
        grid = sms * (per > 0 ? per : 1);
    }
    if (dependent) return launch_dependent(k_docs<BLOCK, LOGC1>, dim3(grid), dim3(BLOCK), C::SMEM, s, a);
    k_docs<BLOCK, LOGC1><<<grid, BLOCK, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

const DocShape kDocShapes[] = {
    {128, 10}, {256, 11}, {256, 12}, {512, 12}, {512, 13}, {1024, 13}, {64, 10}, {32, 9},
};
const int kNumDocShapes = sizeof(kDocShapes) / sizeof(kDocShapes[0]);

cudaError_t launch_docs(const BatchArgs &a, int shape, cudaStream_t s, bool dependent) {
    switch (shape) {
    case 0: return launch_docs_t<128, 10>(a, 0, s, dependent);
    case 1: return launch_docs_t<256, 11>(a, 0, s, dependent);
    case 2: return launch_docs_t<256, 12>(a, 0, s, dependent);
    case 3: return launch_docs_t<512, 12>(a, 0, s, dependent);
    case 4: return launch_docs_t<512, 13>(a, 0, s, dependent);
    case 5: return launch_docs_t<1024, 13>(a, 0, s, dependent);
    case 6: return launch_docs_t<64, 10>(a, 0, s, dependent);
    default: return launch_docs_t<32, 9>(a, 0, s, dependent);
    }
}

// ---------------------------------------------------------------- segmented finish
__device__ __forceinline__ uint32_t doc_of_pos(const unsigned long long *off, uint32_t ndocs, unsigned long long pos) {
    uint32_t lo = 0, hi = ndocs;  // last doc with off[doc] <= pos
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (off[mid] <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_bcompact8(const G8Slot *slots, unsigned long long cap, SortScratch ss, unsigned long long *meta) {
    __shared__ BlockTake sh;
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x * kScanUnroll; b < cap; b += step) {
        ulonglong2 v[kScanUnroll];
        uint32_t mine = 0;
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            v[u] = i < cap ? *reinterpret_cast<const ulonglong2 *>(&slots[i]) : make_ulonglong2(0ull, 0ull);
            mine += v[u].x != 0ull;
        }
        unsigned long long pos = block_take(sh, mine, 0ull, &meta[0], nullptr);
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long k = v[u].x;
            if (!k) continue;
            const unsigned long long w = restore_letters(k);
            ss.khi[pos] = be64b((uint32_t)w, (uint32_t)(w >> 32));
            ss.klo[pos] = 0ull;
            ss.cnt[pos] = v[u].y;
            ss.lref[pos] = 0u;
            ss.doc[pos] = gather_doc(k);
            pos++;
        }
    }
}

__global__ void k_bcompact16(const GSlot *slots, unsigned long long cap, SortScratch ss, unsigned long long *meta) {
    __shared__ BlockTake sh;
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x * kScanUnroll; b < cap; b += step) {
        uint4 k[kScanUnroll];
        unsigned long long c[kScanUnroll];
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
            mine += !key_zero(k[u]);
        }
        unsigned long long pos = block_take(sh, mine, 0ull, &meta[0], nullptr);
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            if (key_zero(k[u])) continue;
            const unsigned long long lo = ((unsigned long long)k[u].y << 32) | k[u].x;
            const unsigned long long hi = ((unsigned long long)k[u].w << 32) | k[u].z;
            const unsigned long long wl = restore_letters(lo), wh = restore_letters(hi);
            ss.khi[pos] = be64b((uint32_t)wl, (uint32_t)(wl >> 32));
            ss.klo[pos] = be64b((uint32_t)wh, (uint32_t)(wh >> 32));
            ss.cnt[pos] = c[u];
            ss.lref[pos] = 0u;
            ss.doc[pos] = gather_doc(lo) | (gather_doc(hi) << 24);
            pos++;
        }
    }
}

// One lane per long slot, a warp's slots reserving entries, long indices
// and arena bytes with one atomic each: document from the representative's
// position, bytes copied (lowercased, 0-terminated) into the batch arena by
// the slot's lane up to 64 bytes and by the whole warp beyond.
__global__ void k_bcompact_long(const LSlot *ls, unsigned long long lcap, SortScratch ss, BatchArgs a,
                                unsigned long long *meta) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long w0 = (((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; w0 < lcap;
         w0 += nw * 32) {
        const unsigned long long w = w0 + lane;
        unsigned long long h = 0, addr = 0, len = 0, c = 0;
        if (w < lcap) {
            h = ls[w].h;
            addr = ls[w].addr;
            len = long_len(ls[w].len);
            c = ls[w].cnt;
        }
        const bool occ = !(h == 0 && addr == 0);
        const uint32_t m = __ballot_sync(kFull, occ);
        if (!m) continue;
        const unsigned long long rank = __popc(m & ((1u << lane) - 1u)), nocc = __popc(m);
        const unsigned long long bytes = occ ? len + 1 : 0ull;
        unsigned long long incl = bytes;
        for (int dd = 1; dd < 32; dd <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, incl, dd);
            if (lane >= dd) incl += t;
        }
        const unsigned long long total = __shfl_sync(kFull, incl, 31);
        unsigned long long boff = 0, blidx = 0, bpos = 0;
        if (lane == 0) {
            boff = atomicAdd(&a.meta[2], total);
            blidx = atomicAdd(&a.meta[1], nocc);
            bpos = atomicAdd(&meta[0], nocc);
            atomicAdd(&meta[1], nocc);  // long entries present: the sort orders shared prefixes by full bytes
        }
        const unsigned long long off = __shfl_sync(kFull, boff, 0) + incl - bytes;
        const unsigned long long lidx = __shfl_sync(kFull, blidx, 0) + rank;
        const unsigned long long pos = __shfl_sync(kFull, bpos, 0) + rank;
        const bool fits = off + len + 1 <= a.arena_cap && lidx < a.lcap;
        const uint8_t *src = reinterpret_cast<const uint8_t *>(addr);
        if (occ && fits && len <= 64)
            for (unsigned long long j = 0; j < len; j++) a.arena[off + j] = (uint8_t)(src[j] | 0x20u);
        uint32_t big = __ballot_sync(kFull, occ && fits && len > 64);
        while (big) {
            const int l = __ffs(big) - 1;
            big &= big - 1;
            const uint8_t *bs = reinterpret_cast<const uint8_t *>(__shfl_sync(kFull, addr, l));
            const unsigned long long bo = __shfl_sync(kFull, off, l), bl = __shfl_sync(kFull, len, l);
            for (unsigned long long j = lane; j < bl; j += 32) a.arena[bo + j] = (uint8_t)(bs[j] | 0x20u);
        }
        if (occ) {
            if (!fits) atomicOr(a.status, ST_OUT_FULL);
            else {
                a.arena[off + len] = 0;
                a.loff[lidx] = off;
                a.llen[lidx] = len;
            }
            ss.khi[pos] = be_bytes16(src, 0);
            ss.klo[pos] = be_bytes16(src, 8);
            ss.cnt[pos] = c;
            ss.lref[pos] = fits ? (uint32_t)(lidx + 1) : 0u;
            ss.doc[pos] = doc_of_pos(a.doc_off, a.ndocs, addr - reinterpret_cast<uintptr_t>(a.text));
        }
    }
}

__global__ void k_seg_base(BatchArgs a, unsigned long long *meta) {
    const unsigned long long n = meta[0];
    const unsigned long long base = n ? atomicAdd(&a.meta[0], n) : 0ull;
    meta[8] = base;
    if (base + n > a.out_cap) {
        atomicOr(a.status, ST_OUT_FULL);
        meta[9] = 0;
    } else {
        meta[9] = 1;
    }
}

// The sorted (document, word) entries -> the CSR output, and each
// document's first row; kScanUnroll entries a thread per step, all loads
// issued before the stores.
__global__ void k_seg_write(SortScratch ss, BatchArgs a, const unsigned long long *meta, int passes) {
    const unsigned long long n = meta[0], base = meta[8];
    if (!meta[9]) return;
    const uint32_t *perm = ss.perm_buf(ss.cur[kCurFinal]);
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x * kScanUnroll; b < n; b += step) {
        uint32_t e[kScanUnroll], ep[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            e[u] = i < n ? perm[i] : 0u;
            ep[u] = i < n && i > 0 ? perm[i - 1] : 0u;
        }
        unsigned long long kh[kScanUnroll], kl[kScanUnroll], c[kScanUnroll];
        uint32_t lr[kScanUnroll], d[kScanUnroll], dp[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            kh[u] = ss.khi[e[u]];
            kl[u] = ss.klo[e[u]];
            c[u] = ss.cnt[e[u]];
            lr[u] = ss.lref[e[u]];
            d[u] = ss.doc[e[u]];
            dp[u] = ss.doc[ep[u]];
        }
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            if (i >= n) continue;
            a.out_khi[base + i] = kh[u];
            a.out_klo[base + i] = kl[u];
            a.out_cnt[base + i] = (uint32_t)c[u];
            a.out_lref[base + i] = lr[u];
            if (i == 0 || dp[u] != d[u]) a.doc_start[d[u]] = base + i;
        }
    }
}

__global__ void k_seg_ends(SortScratch ss, BatchArgs a, const unsigned long long *meta, int passes) {
    const unsigned long long n = meta[0], base = meta[8];
    if (!meta[9]) return;
    const uint32_t *perm = ss.perm_buf(ss.cur[kCurFinal]);
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x * kScanUnroll;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x * kScanUnroll; b < n; b += step) {
        uint32_t d[kScanUnroll], dn[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            d[u] = i < n ? ss.doc[perm[i]] : 0u;
            dn[u] = i + 1 < n ? ss.doc[perm[i + 1]] : ~0u;
        }
#pragma unroll
        for (int u = 0; u < kScanUnroll; u++) {
            const unsigned long long i = b + (unsigned long long)u * blockDim.x + threadIdx.x;
            if (i < n && dn[u] != d[u]) a.doc_n[d[u]] = (uint32_t)(base + i + 1 - a.doc_start[d[u]]);
        }
    }
}

static int gridn(unsigned long long n, int t, int maxb) {
    unsigned long long g = (n + t - 1) / t;
    if (g < 1) g = 1;
    if (g > (unsigned long long)maxb) g = maxb;
    return (int)g;
}

cudaError_t launch_segmented_finish(const BatchArgs &a, const GTable &g, uint64_t cap8, uint64_t cap16,
                                    uint64_t caplong, SortScratch &ss, unsigned long long *smeta, cudaStream_t s,
                                    uint32_t skip) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaMemsetAsync(smeta, 0, 16 * 8, s);
    sort_state_reset(ss, s);
    k_bcompact8<<<gridn(cap8, 256 * kScanUnroll, sms * 8), 256, 0, s>>>(g.slots8, cap8, ss, smeta);
    k_bcompact16<<<gridn(cap16, 256 * kScanUnroll, sms * 8), 256, 0, s>>>(g.slots, cap16, ss, smeta);
    k_bcompact_long<<<gridn(caplong, 256, sms * 8), 256, 0, s>>>(g.lslots, caplong, ss, a, smeta);
    LongView v{ss.lref, a.loff, a.llen, a.arena};
    cudaError_t e = sort_entries(ss, smeta, v, kSortPassesSeg, s, skip);
    if (e != cudaSuccess) return e;
    k_seg_base<<<1, 1, 0, s>>>(a, smeta);
    k_seg_write<<<gridn(ss.cap, 256 * kScanUnroll, sms * 8), 256, 0, s>>>(ss, a, smeta, kSortPassesSeg);
    k_seg_ends<<<gridn(ss.cap, 256 * kScanUnroll, sms * 8), 256, 0, s>>>(ss, a, smeta, kSortPassesSeg);
    return cudaGetLastError();
}
int segmented_finish_launches(uint64_t cap, uint32_t skip) {
    return 4 + sort_entries_launches(kSortPassesSeg, cap, skip) + 3;
}

}  // namespace wc
