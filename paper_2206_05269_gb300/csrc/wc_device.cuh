// Device primitives shared by the counting, table and sort kernels.
//
// Word rule (the paper's normalisation of Sec. 2 / Sec. 3.1 fixed as a byte
// rule): a word is a maximal run of ASCII letters; letters are lowercased;
// every other byte and every document edge separates words.
//
// Keys: a word of at most 16 letters is keyed by its 16 lowercased bytes,
// zero padded (4 x u32, little-endian byte order).  Letters are never zero,
// so the key is unique per word and empty slots are the all-zero key.  Words
// of 17 or more letters ("long" words) are keyed by (64-bit hash, length) in
// a separate table whose slots point at one occurrence of the word; an equal
// (hash, length) pair is always confirmed by comparing the bytes, so a hash
// collision never merges two words.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wc {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kShortMax = 16;  // letters that fit the in-table key

// Test build switch (compile with -DWC_TEST_ONE_SLOT; never the product
// library): every hash below returns one constant, so every key of a table
// starts probing at the same home slot and only the exact key comparison
// keeps distinct words apart.  The parity tests run small inputs through
// that build against the oracle.  The global probe limit is raised so that a
// few thousand distinct words still fit one probe chain.
#ifdef WC_TEST_ONE_SLOT
constexpr bool kOneSlot = true;
#else
constexpr bool kOneSlot = false;
#endif

// status bits written by kernels (OR-ed into one device word)
enum : uint32_t {
    ST_TABLE_FULL = 1u,   // short-word table probe limit reached
    ST_LONG_FULL = 2u,    // long-word table probe limit reached
    ST_ARENA_FULL = 4u,   // long-word byte arena too small
    ST_TIMEOUT = 8u,      // a bounded wait gave up
    ST_TOO_LONG = 16u,    // a word or position beyond the documented limits
    ST_OUT_FULL = 32u,    // a per-document output region overflowed
    ST_BAD_CLASS = 64u,   // a document's class id is not below the class count
};

// ---------------------------------------------------------------- bytes
// 0x80 in every byte lane that holds an ASCII letter: fold case with |0x20,
// then test 0x61 <= y <= 0x7A with two carry-free byte adds; bytes >= 0x80
// are excluded by the original high bit.
__device__ __forceinline__ uint32_t letter_bits(uint32_t w) {
    uint32_t y = (w | 0x20202020u) & 0x7F7F7F7Fu;
    uint32_t a = y + 0x1F1F1F1Fu;  // bit 7 set iff y >= 0x61
    uint32_t b = y + 0x05050505u;  // bit 7 set iff y >= 0x7B
    return a & ~b & ~w & 0x80808080u;
}
// Gathers the four lane bits of letter_bits into bits 0..3 (one multiply; the
// partial products land on distinct bit positions, so nothing carries).
__device__ __forceinline__ uint32_t letter_mask4(uint32_t w) {
    return ((letter_bits(w) >> 7) * 0x00204081u) >> 21 & 0xFu;
}
__device__ __forceinline__ uint32_t letter_mask16(uint4 v) {
    return letter_mask4(v.x) | (letter_mask4(v.y) << 4) | (letter_mask4(v.z) << 8) |
           (letter_mask4(v.w) << 12);
}
__device__ __forceinline__ bool is_letter(uint32_t b) {
    uint32_t y = (b | 0x20u) - 0x61u;
    return b < 0x80u && y < 26u;
}
__device__ __forceinline__ uint32_t lower_byte(uint32_t b) { return b | 0x20u; }

// Mask of the low r bytes of a word (none for r <= 0, all for r >= 4): the
// high word of 0:0xFFFFFFFF shifted left by 8r bits, the shift clamped to 32.
__device__ __forceinline__ uint32_t byte_keep_mask(int r) {
    return __funnelshift_lc(0xFFFFFFFFu, 0u, 8u * (uint32_t)(r > 0 ? r : 0));
}

// 16 lowercased bytes of win[p, p+len), zero padded (len <= 16).  Reads
// win[p & ~3, (p & ~3) + 20): the window must hold 4 bytes of slack.
__device__ __forceinline__ uint4 load_key16(const uint8_t *win, uint32_t p, uint32_t len) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(win + (p & ~3u));
    uint32_t sh = (p & 3u) * 8u;
    uint32_t a0 = w[0], a1 = w[1], a2 = w[2], a3 = w[3], a4 = w[4];
    uint4 k;
    int n = (int)len;
    k.x = (__funnelshift_r(a0, a1, sh) | 0x20202020u) & byte_keep_mask(n);
    k.y = (__funnelshift_r(a1, a2, sh) | 0x20202020u) & byte_keep_mask(n - 4);
    k.z = (__funnelshift_r(a2, a3, sh) | 0x20202020u) & byte_keep_mask(n - 8);
    k.w = (__funnelshift_r(a3, a4, sh) | 0x20202020u) & byte_keep_mask(n - 12);
    return k;
}

// 8 big-endian key bytes (0, or a letter) -> 8 five-bit codes (0 for
// padding, 1..26 for a..z), the first byte in the highest code (40 bits):
// integer order on codes is byte order on lowercase words.
__device__ __forceinline__ unsigned long long pack5(unsigned long long be) {
    unsigned long long r = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint32_t b = (uint32_t)(be >> (56 - 8 * i)) & 0xFFu;
        r = (r << 5) | (b ? ((b | 0x20u) - 0x60u) & 31u : 0u);
    }
    return r;
}
// The inverse of pack5: 40 bits of codes -> 8 big-endian lowercase bytes.
__device__ __forceinline__ unsigned long long unpack5(unsigned long long c) {
    unsigned long long r = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint32_t v = (uint32_t)(c >> (35 - 5 * i)) & 31u;
        r = (r << 8) | (v ? v + 0x60u : 0u);
    }
    return r;
}

__device__ __forceinline__ bool key_eq(uint4 a, uint4 b) {
    return ((a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w)) == 0u;
}
__device__ __forceinline__ bool key_zero(uint4 a) { return (a.x | a.y | a.z | a.w) == 0u; }

// 64-bit slot hash of a 16-byte key: MurmurHash3's fmix64 finalizer
// (Appleby, public domain) over the two halves folded together.  It only picks
// slots; equality is always decided on the full key.
__device__ __forceinline__ uint64_t hash_key(uint4 k) {
    if (kOneSlot) return 0ull;
    uint64_t lo = ((uint64_t)k.y << 32) | k.x;
    uint64_t hi = ((uint64_t)k.w << 32) | k.z;
    uint64_t x = lo ^ (hi * 0x9E3779B97F4A7C15ull);
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDull;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ unsigned long long fmix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDull;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ull;
    x ^= x >> 33;
    return x;
}

// 16 lowercased bytes of the letter run at p[0, n), zero padded (n <= 0: all
// zero).  Reads only the aligned 4-byte words that hold some of those bytes,
// so it never touches memory past the run's last aligned word; the loads are
// independent of each other.
__device__ __forceinline__ uint4 load_run16(const uint8_t *p, long long n) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a & ~(uintptr_t)3);
    const uint32_t sh = (uint32_t)(a & 3u) * 8u;
    const long long need = n > 0 ? n + (long long)(a & 3u) : 0;  // bytes needed from the aligned start
    uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0;
    if (need > 0) v0 = __ldg(w);
    if (need > 4) v1 = __ldg(w + 1);
    if (need > 8) v2 = __ldg(w + 2);
    if (need > 12) v3 = __ldg(w + 3);
    if (need > 16) v4 = __ldg(w + 4);
    const int m = n < 0 ? 0 : (n > 16 ? 16 : (int)n);
    uint4 k;
    k.x = (__funnelshift_r(v0, v1, sh) | 0x20202020u) & byte_keep_mask(m);
    k.y = (__funnelshift_r(v1, v2, sh) | 0x20202020u) & byte_keep_mask(m - 4);
    k.z = (__funnelshift_r(v2, v3, sh) | 0x20202020u) & byte_keep_mask(m - 8);
    k.w = (__funnelshift_r(v3, v4, sh) | 0x20202020u) & byte_keep_mask(m - 12);
    return k;
}
// Hash of a long word (17+ letters): its first and last 16 lowercased bytes
// and its length, mixed by MurmurHash3's fmix64 finalizer (Appleby, public
// domain).  It only picks slots (equality is always decided on every byte),
// so the two ends suffice; every table holding long words uses this one
// function, from the text or from a table's arena alike.
__device__ __forceinline__ unsigned long long long_hash_mix(uint4 f, uint4 l, unsigned long long len) {
    if (kOneSlot) return 1ull;  // a claimed slot keeps a non-zero hash word
    const unsigned long long f0 = ((unsigned long long)f.y << 32) | f.x, f1 = ((unsigned long long)f.w << 32) | f.z;
    const unsigned long long l0 = ((unsigned long long)l.y << 32) | l.x, l1 = ((unsigned long long)l.w << 32) | l.z;
    return fmix64(f0 * 0x9E3779B97F4A7C15ull ^ f1 * 0xC2B2AE3D27D4EB4Full ^ l0 * 0x165667B19E3779F9ull ^
                  l1 * 0xD6E8FEB86659FD93ull ^ len * 0xFF51AFD7ED558CCDull);
}
// The first and last 16 lowercased letters of the run w[0, len) (len >= 16).
__device__ __forceinline__ void long_ends(const uint8_t *w, unsigned long long len, uint4 &f, uint4 &l) {
    f = load_run16(w, 16);
    l = load_run16(w + (len - 16ull), 16);
}
__device__ __forceinline__ unsigned long long long_hash(const uint8_t *w, unsigned long long len) {
    const long long m = len < 16 ? (long long)len : 16;
    return long_hash_mix(load_run16(w, m), load_run16(w + (len - (unsigned long long)m), m), len);
}
// Whether the letter runs a[0, len) and b[0, len) are equal (case folded).
__device__ inline bool runs_equal(const uint8_t *a, const uint8_t *b, unsigned long long len) {
    for (unsigned long long off = 0; off < len; off += 32) {
        const long long n = (long long)(len - off);
        const uint4 a0 = load_run16(a + off, n), b0 = load_run16(b + off, n);
        const uint4 a1 = load_run16(a + off + 16, n - 16), b1 = load_run16(b + off + 16, n - 16);
        if (!key_eq(a0, b0) || !key_eq(a1, b1)) return false;
    }
    return true;
}

// ---------------------------------------------------------------- atomics
// A 64-bit load that sees other SMs' atomics (not served from a stale L1 line).
__device__ __forceinline__ unsigned long long ld_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// 128-bit compare-and-swap (sm_90+): returns the previous value.
__device__ __forceinline__ uint4 cas128_global(void *addr, uint4 cmp, uint4 val) {
    uint64_t c0 = ((uint64_t)cmp.y << 32) | cmp.x, c1 = ((uint64_t)cmp.w << 32) | cmp.z;
    uint64_t v0 = ((uint64_t)val.y << 32) | val.x, v1 = ((uint64_t)val.w << 32) | val.z;
    uint64_t r0, r1;
    asm volatile(
        "{\n\t.reg .b128 c, v, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.relaxed.gpu.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(r0), "=l"(r1)
        : "l"(c0), "l"(c1), "l"(v0), "l"(v1), "l"(addr)
        : "memory");
    uint4 r;
    r.x = (uint32_t)r0; r.y = (uint32_t)(r0 >> 32);
    r.z = (uint32_t)r1; r.w = (uint32_t)(r1 >> 32);
    return r;
}

__device__ __forceinline__ void red_add_u64_dev(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint4 ld_stream16(const void *p) {  // read-once text
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Replaces the bytes of 16 aligned bytes at absolute address a that lie
// outside [vb, ve) by spaces (a document edge separates words).
__device__ __forceinline__ uint4 mask_outside_doc(uint4 v, uintptr_t a, uintptr_t vb, uintptr_t ve) {
    long long lo = (long long)(vb - a), hi = (long long)(ve - a);  // keep bytes in [lo, hi)
    int klo = (int)(lo < 0 ? 0 : (lo > 16 ? 16 : lo));
    int khi = (int)(hi < 0 ? 0 : (hi > 16 ? 16 : hi));
    uint32_t m0 = byte_keep_mask(khi) & ~byte_keep_mask(klo);
    uint32_t m1 = byte_keep_mask(khi - 4) & ~byte_keep_mask(klo - 4);
    uint32_t m2 = byte_keep_mask(khi - 8) & ~byte_keep_mask(klo - 8);
    uint32_t m3 = byte_keep_mask(khi - 12) & ~byte_keep_mask(klo - 12);
    v.x = (v.x & m0) | (0x20202020u & ~m0);
    v.y = (v.y & m1) | (0x20202020u & ~m1);
    v.z = (v.z & m2) | (0x20202020u & ~m2);
    v.w = (v.w & m3) | (0x20202020u & ~m3);
    return v;
}

// ---------------------------------------------------------------- tables
// Global short-word slot: one 32-byte sector (key, count, spare).
struct __align__(32) GSlot {
    uint4 key;
    unsigned long long cnt;
    unsigned long long spare;
};
// Global long-word slot: (hash, address of the first occurrence) is the
// 128-bit CAS target, so a slot is published whole in one atomic step.  The
// claimer then writes the length and, when it knows them, the word's first
// and last 16 lowercased letters (f, l) followed by kLongReady in len with a
// release store: for a word of at most 32 letters (f, l, length) is the
// whole word, so later inserts that read kLongReady (acquire) compare
// against the slot instead of reading the first occurrence's bytes.  Length
// readers mask kLongReady off (long_len).
constexpr unsigned long long kLongReady = 1ull << 63;
struct __align__(64) LSlot {
    unsigned long long h;
    unsigned long long addr;
    unsigned long long cnt;
    unsigned long long len;
    uint4 f, l;
};
__device__ __forceinline__ unsigned long long long_len(unsigned long long len_field) { return len_field & ~kLongReady; }
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 16 bytes at a 16-byte aligned address as one vector load of two relaxed
// 64-bit elements (each half single-copy atomic, as two separate loads).
__device__ __forceinline__ uint4 ld_relaxed_v2(const void *p) {
    unsigned long long a, b;
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
    return make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
}
__device__ __forceinline__ uint4 ld_relaxed_u128(const uint4 *p) {
    const unsigned long long *q = reinterpret_cast<const unsigned long long *>(p);
    const unsigned long long a = ld_u64(q), b = ld_u64(q + 1);
    return make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
}

// Global 8-byte-key slot (words of at most 8 letters): key, count.
struct __align__(16) G8Slot {
    unsigned long long key;
    unsigned long long cnt;
};

struct GTable {
    GSlot *slots;                // words of 9..16 letters
    unsigned long long mask;     // capacity - 1 (power of two)
    LSlot *lslots;               // words of 17+ letters
    unsigned long long lmask;
    uint32_t *status;
    G8Slot *slots8;              // words of 1..8 letters
    unsigned long long mask8;
};

constexpr int kGlobalProbeLimit = kOneSlot ? (1 << 20) : 4096;
// Lowercased byte comparison of two runs of `len` letters.
__device__ __forceinline__ bool bytes_eq_lower(const uint8_t *a, const uint8_t *b, uint64_t len) {
    for (uint64_t i = 0; i < len; i++)
        if ((a[i] | 0x20u) != (b[i] | 0x20u)) return false;
    return true;
}
__device__ __forceinline__ bool bytes_eq_lower_warp(const uint8_t *a, const uint8_t *b, uint64_t len) {
    bool ok = true;
    for (uint64_t i = threadIdx.x & 31; i < len; i += 32) ok &= ((a[i] | 0x20u) == (b[i] | 0x20u));
    return __all_sync(kFull, ok);
}

// Adds `add` to the long word w[0, len) (a maximal letter run, len >= 17),
// given its hash h (which includes the length, and the document in batched
// counting).  fl (may be null) holds the word's first and last 16 lowercased
// letters: a claimer publishes them in the slot, and a word of at most 32
// letters is then matched against a ready slot without reading text.  `end` bounds the buffer holding w: a word ends at its first
// non-letter or at `end`.  The slot's (hash, address) pair is claimed with one
// 128-bit CAS; a thread finding the same hash compares the representative's
// bytes with its own and checks that the representative's run ends after
// exactly len letters, so a hash collision never merges two words and no
// thread ever waits for another.  In text, [begin, end) is the document: a
// representative outside it belongs to another document and never matches.
// With begin == null the words live in arenas where each word is followed by
// a 0 byte; the compare stops at the first difference, so it never reads past
// a representative's terminator.
__device__ inline void long_insert2(const GTable &g, const uint8_t *w, unsigned long long len,
                                    unsigned long long h, unsigned long long add, const uint8_t *begin,
                                    const uint8_t *end, const uint4 *fl = nullptr) {
    unsigned long long s = h & g.lmask;
    const unsigned long long wa = (unsigned long long)reinterpret_cast<uintptr_t>(w);
    const uint4 want = make_uint4((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)wa, (uint32_t)(wa >> 32));
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (int probe = 0; probe < kGlobalProbeLimit; probe++) {
        LSlot *slot = g.lslots + s;
        // relaxed loads first, the whole slot in one round trip: a claimed slot
        // (both key words non-zero, written by one 128-bit CAS) is settled; an
        // empty or half-seen one goes to the CAS
        uint4 old = ld_relaxed_v2(&slot->h);
        const uint4 clen = ld_relaxed_v2(&slot->cnt);
        uint4 sf = make_uint4(0u, 0u, 0u, 0u), sl = sf;
        if (fl) {
            sf = ld_relaxed_v2(&slot->f);
            sl = ld_relaxed_v2(&slot->l);
        }
        const unsigned long long h0 = ((unsigned long long)old.y << 32) | old.x,
                                 a0 = ((unsigned long long)old.w << 32) | old.z;
        if (h0 == 0ull || a0 == 0ull) old = cas128_global(&slot->h, zero, want);
        if (key_zero(old)) {
            if (fl) {
                slot->f = fl[0];
                slot->l = fl[1];
                st_release_u64(&slot->len, len | kLongReady);
            } else {
                slot->len = len;
            }
            red_add_u64_dev(&slot->cnt, add);
            return;
        }
        if (fl && old.x == want.x && old.y == want.y) {
            // the length word seen with the slot: when ready, the ends read
            // with it are the published ones or (if read before publication)
            // still zero, which no word's ends are; a mismatch is confirmed
            // by reading the ends again after an acquire of the length word
            unsigned long long lr = ((unsigned long long)clen.w << 32) | clen.z;
            bool ends = (lr & kLongReady) && long_len(lr) == len && key_eq(sf, fl[0]) && key_eq(sl, fl[1]);
            if (!ends) {
                lr = ld_acquire_u64(&slot->len);
                ends = (lr & kLongReady) && long_len(lr) == len && key_eq(ld_relaxed_u128(&slot->f), fl[0]) &&
                       key_eq(ld_relaxed_u128(&slot->l), fl[1]);
            }
            if (lr & kLongReady) {
                if (ends && len <= 32) {  // the ends and the length are the whole word
                    red_add_u64_dev(&slot->cnt, add);
                    return;
                }
                if (!ends) {  // another word with the same hash
                    s = (s + 1) & g.lmask;
                    continue;
                }
            }
        }
        if (old.x == want.x && old.y == want.y) {
            const uint8_t *rep = reinterpret_cast<const uint8_t *>(((unsigned long long)old.w << 32) | old.z);
            bool cand;
            if (begin) cand = rep >= begin && rep + len <= end;  // text: same document, in bounds
            else cand = true;  // arena: 0-terminated words, the early-exit compare stays inside them
            if (cand) {
                bool eq = true;
                if (begin) {  // text: both runs are readable for len bytes
                    const bool term = rep + len == end || !is_letter(rep[len]);
                    eq = term && runs_equal(rep, w, len);
                } else {
                    for (unsigned long long i = 0; i < len && eq; i++) eq = (rep[i] | 0x20u) == (w[i] | 0x20u);
                    if (eq) eq = !is_letter(rep[len]);
                }
                if (eq) {
                    red_add_u64_dev(&slot->cnt, add);
                    return;
                }
            }
        }
        s = (s + 1) & g.lmask;
    }
    atomicOr(g.status, ST_LONG_FULL);
}

// One thread inserts a long word (computes the hash itself).
__device__ inline void long_insert(const GTable &g, const uint8_t *w, uint64_t len, unsigned long long add,
                                   const uint8_t *begin, const uint8_t *end) {
    long_insert2(g, w, len, long_hash(w, len), add, begin, end);
}

// ---------------------------------------------------------------- 8-byte keys
// Words of at most 8 letters: key = the 8 lowercased bytes, zero padded,
// little-endian (never 0).  Keys are written once (CAS from 0) and never
// change, so a plain 64-bit load that sees a non-zero key sees the final key.
// Slot hash of a word of at most 16 letters, given as its key halves k0 (the
// first 8 letters) and k1 (the next 8, or 0): multiplicative (Fibonacci)
// hashing of k0 ^ (k1 * c); a table of 2^b slots takes the top b bits.  With
// k1 = 0 it is k0 times the golden-ratio constant.  Both global key tables
// use it, so one probe sequence serves either key size.
__device__ __forceinline__ unsigned long long hash_slot(unsigned long long k0, unsigned long long k1) {
    if (kOneSlot) return 0ull;
    return (k0 ^ (k1 * 0xC2B2AE3D27D4EB4Full)) * 0x9E3779B97F4A7C15ull;
}
__device__ __forceinline__ unsigned long long hash8(unsigned long long key) { return hash_slot(key, 0ull); }
// The home slot of a 16-byte key in a table of mask + 1 (a power of two, at least 2) slots.
__device__ __forceinline__ unsigned long long home16(uint4 k, unsigned long long mask) {
    return hash_slot(((unsigned long long)k.y << 32) | k.x, ((unsigned long long)k.w << 32) | k.z) >>
           __clzll((long long)mask);
}
__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) { red_add_u64_dev(p, v); }
// Probes from slot s onwards (s = the home slot, or a later slot of its chain).
__device__ __forceinline__ void global_insert8_from(const GTable &g, unsigned long long key, unsigned long long add,
                                                    unsigned long long s) {
    for (int probe = 0; probe < kGlobalProbeLimit; probe++) {
        G8Slot *slot = g.slots8 + s;
        unsigned long long cur = ld_u64(&slot->key);
        if (cur == 0ull) cur = atomicCAS(&slot->key, 0ull, key);
        if (cur == 0ull || cur == key) {
            red_add_u64(&slot->cnt, add);
            return;
        }
        s = (s + 1) & g.mask8;
    }
    atomicOr(g.status, ST_TABLE_FULL);
}
__device__ __forceinline__ void global_insert8(const GTable &g, unsigned long long key, unsigned long long add) {
    global_insert8_from(g, key, add, hash8(key) >> __clzll((long long)g.mask8));  // top bits
}

// Words of 9..16 letters: both key halves are non-zero, so two 64-bit loads
// that each see the corresponding half of `k` can only come from a slot that
// holds exactly `k` (halves are written once, by one 128-bit CAS).  Loads that
// see a zero half may have caught a claim in flight (possibly of this very
// word), so that case is settled by the CAS, which returns the whole key.
__device__ __forceinline__ void global_insert16_from(const GTable &g, uint4 k, unsigned long long add,
                                                     unsigned long long s) {
    const unsigned long long k0 = ((unsigned long long)k.y << 32) | k.x, k1 = ((unsigned long long)k.w << 32) | k.z;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (int probe = 0; probe < kGlobalProbeLimit; probe++) {
        GSlot *slot = g.slots + s;
        const unsigned long long *kp = reinterpret_cast<const unsigned long long *>(&slot->key);
        unsigned long long c0 = ld_u64(kp), c1 = ld_u64(kp + 1);
        bool hit = (c0 == k0 && c1 == k1);
        if (!hit && (c0 == 0ull || c1 == 0ull)) {  // empty, or a key being written: ask the CAS
            uint4 old = cas128_global(&slot->key, zero, k);
            hit = key_zero(old) || key_eq(old, k);
        }
        if (hit) {
            red_add_u64(&slot->cnt, add);
            return;
        }
        s = (s + 1) & g.mask;
    }
    atomicOr(g.status, ST_TABLE_FULL);
}
__device__ __forceinline__ void global_insert16(const GTable &g, uint4 k, unsigned long long add) {
    global_insert16_from(g, k, add, home16(k, g.mask));
}

// Any word of at most 16 letters given as a 16-byte key.
__device__ __forceinline__ void table_insert_key(const GTable &g, uint4 k, unsigned long long add) {
    if ((k.z | k.w) == 0u) global_insert8(g, ((unsigned long long)k.y << 32) | k.x, add);
    else global_insert16(g, k, add);
}

}  // namespace wc
