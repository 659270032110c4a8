// Map + level-1 reduce: the fused tokenise-and-count kernel.
//
// The paper maps on the CPU (Sec. 3.1: remove punctuation, lowercase, split,
// one dictionary per document) and reduces on the GPU (Sec. 3.3); its
// conclusion (Sec. 5.2) asks for a GPU dictionary so the whole map and reduce
// can run on the device.  This kernel is that design for one document:
//
//  1. a persistent block stages a chunk of text (plus 16 bytes before and 64
//     after) into shared memory with 16-byte loads;
//  2. each warp classifies 512-byte strips: one 16-bit letter mask per lane
//     (SWAR), word starts = letter & !previous-letter, with the previous
//     byte carried across lanes, strips and chunk edges; a word belongs to
//     the chunk that holds its first byte;
//  3. words of <= 16 letters are queued per warp and processed 32 at a time:
//     16-byte lowercased key, 64-bit hash, insert into the block's
//     shared-memory table; a full table or a long probe spills the word to
//     the global open-addressing table;
//  4. words of >= 17 letters go to the global long-word table;
//  5. at the end each block flushes its shared table into the global table.
#include "wc_internal.h"

namespace wc {

struct CountArgs {
    const uint8_t *text;
    unsigned long long lo, hi;
    uint32_t nchunks;
    GTable g;
};

__device__ __forceinline__ uint4 spaces16() { return make_uint4(0x20202020u, 0x20202020u, 0x20202020u, 0x20202020u); }

// Loads the aligned 16-byte block at address a0 if it holds any byte of the
// valid range [vb, ve) (then it lies inside the caller's allocation pages);
// otherwise returns spaces.
__device__ __forceinline__ uint4 load_block(uintptr_t a0, uintptr_t vb, uintptr_t ve) {
    if (a0 < ve && a0 + 16 > vb) return ld_stream16(reinterpret_cast<const void *>(a0));
    return spaces16();
}

// bytes [m, m+16) of the 32-byte concatenation (w0, w1), m in 1..15
__device__ __forceinline__ uint4 shift_bytes(uint4 w0, uint4 w1, uint32_t m) {
    uint32_t q = m >> 2, sh = (m & 3u) * 8u;
    uint32_t s0, s1, s2, s3, s4;
    if (q == 0) { s0 = w0.x; s1 = w0.y; s2 = w0.z; s3 = w0.w; s4 = w1.x; }
    else if (q == 1) { s0 = w0.y; s1 = w0.z; s2 = w0.w; s3 = w1.x; s4 = w1.y; }
    else if (q == 2) { s0 = w0.z; s1 = w0.w; s2 = w1.x; s3 = w1.y; s4 = w1.z; }
    else { s0 = w0.w; s1 = w1.x; s2 = w1.y; s3 = w1.z; s4 = w1.w; }
    uint4 r;
    r.x = __funnelshift_r(s0, s1, sh);
    r.y = __funnelshift_r(s1, s2, sh);
    r.z = __funnelshift_r(s2, s3, sh);
    r.w = __funnelshift_r(s3, s4, sh);
    return r;
}

// Replaces the bytes of a 16-byte word (logical positions q0..q0+15) that lie
// outside [vlo, vhi) by spaces: a document edge is a separator.
__device__ __forceinline__ uint4 mask_outside(uint4 v, long long q0, long long vlo, long long vhi) {
    long long a = vlo - q0, b = vhi - q0;
    int klo = (int)(a < 0 ? 0 : (a > 16 ? 16 : a));
    int khi = (int)(b < 0 ? 0 : (b > 16 ? 16 : b));
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

// win[j] = text[ws + j] for ws + j in [vlo, vhi), else ' ', for j < nbytes (multiple of 16).
template <int BLOCK>
__device__ __forceinline__ void stage_window(uint8_t *win, int nbytes, const uint8_t *text, long long ws,
                                             unsigned long long vlo, unsigned long long vhi) {
    const uintptr_t base = reinterpret_cast<uintptr_t>(text);
    const uintptr_t vb = base + vlo, ve = base + vhi;
    for (int t = threadIdx.x; t < nbytes / 16; t += BLOCK) {
        long long q0 = ws + 16LL * t;
        uintptr_t a = base + (uintptr_t)q0;  // modular arithmetic; only dereferenced when valid
        uintptr_t a0 = a & ~(uintptr_t)15;
        uint32_t m = (uint32_t)(a & 15);
        uint4 w0 = load_block(a0, vb, ve);
        uint4 out = w0;
        if (m) out = shift_bytes(w0, load_block(a0 + 16, vb, ve), m);
        if (q0 < (long long)vlo || q0 + 16 > (long long)vhi) out = mask_outside(out, q0, (long long)vlo, (long long)vhi);
        *reinterpret_cast<uint4 *>(win + 16 * t) = out;
    }
}

// Length of the letter run starting at text[pos] (pos is a letter), capped at hi.
__device__ __forceinline__ unsigned long long run_length(const uint8_t *text, unsigned long long pos,
                                                         unsigned long long hi) {
    unsigned long long e = pos;
    while (e < hi && is_letter(text[e])) e++;
    return e - pos;
}

template <int BLOCK, int CHUNK, int LOG_C1>
struct CountCfg {
    static constexpr int WARPS = BLOCK / 32;
    static constexpr int STRIPS = CHUNK / 512;
    static constexpr int SPW = STRIPS / WARPS;
    static constexpr int LEAD = 16;
    static constexpr int WIN = LEAD + CHUNK + 64 + 16;
    static constexpr int TOKCAP = 32 + 256;
    static constexpr int C1 = 1 << LOG_C1;
    static constexpr size_t SMEM = (size_t)WIN + (size_t)C1 * 16 + (size_t)C1 * 8 + (size_t)WARPS * TOKCAP * 4 + 16;
    static_assert(STRIPS % WARPS == 0, "chunk must split evenly into warp strips");
    static_assert(WIN % 16 == 0, "window must be 16-byte aligned");
};

template <int BLOCK, int CHUNK, int LOG_C1, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_count_global(CountArgs a) {
    using C = CountCfg<BLOCK, CHUNK, LOG_C1>;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *win = smem;
    uint4 *skey = reinterpret_cast<uint4 *>(smem + C::WIN);
    uint32_t *stag = reinterpret_cast<uint32_t *>(skey + C::C1);
    uint32_t *scnt = stag + C::C1;
    uint32_t *tokall = scnt + C::C1;
    uint32_t *nfill = tokall + C::WARPS * C::TOKCAP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *tok = tokall + warp * C::TOKCAP;
    STable st{stag, skey, scnt, nfill, (uint32_t)(C::C1 - 1), (uint32_t)(C::C1 * 7 / 10)};

    for (int i = threadIdx.x; i < C::C1; i += BLOCK) stag[i] = 0u;
    if (threadIdx.x == 0) *nfill = 0u;

    auto process = [&](uint32_t e) {
        uint32_t p = e >> 5, len = e & 31u;
        uint4 k = load_key16(win, p, len);
        uint64_t h = hash_key(k);
        if (!shared_insert(st, k, h, 1u, 8)) global_insert(a.g, k, h, 1ull);
    };

    for (uint32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        const unsigned long long lo = a.lo + (unsigned long long)c * CHUNK;
        const long long ws = (long long)lo - C::LEAD;
        __syncthreads();  // previous chunk's window reads are done
        stage_window<BLOCK>(win, C::WIN, a.text, ws, a.lo, a.hi);
        __syncthreads();

        uint32_t tcount = 0;
        const int s0 = warp * C::SPW;
        uint32_t prevL = is_letter(win[C::LEAD + 512 * s0 - 1]) ? 1u : 0u;
        uint32_t L = letter_mask16(*reinterpret_cast<const uint4 *>(win + C::LEAD + 512 * s0 + 16 * lane));
#pragma unroll 1
        for (int k = 0; k < C::SPW; k++) {
            const int sbase = C::LEAD + 512 * (s0 + k);
            int nidx = sbase + 512 + 16 * lane;
            if (nidx > C::LEAD + CHUNK) nidx = C::LEAD + CHUNK;  // past the chunk only lane 0 matters
            const uint32_t Ln = letter_mask16(*reinterpret_cast<const uint4 *>(win + nidx));
            const uint32_t up = __shfl_up_sync(kFull, L, 1);
            const uint32_t dn = __shfl_down_sync(kFull, L, 1);
            const uint32_t n0 = __shfl_sync(kFull, Ln, 0);
            const uint32_t pbit = lane == 0 ? prevL : ((up >> 15) & 1u);
            const uint32_t W = L | ((lane == 31 ? n0 : dn) << 16);
            const uint32_t S = L & ~((L << 1) | pbit) & 0xFFFFu;
            prevL = (__shfl_sync(kFull, L, 31) >> 15) & 1u;
            uint32_t x = W;
            x &= x >> 1; x &= x >> 2; x &= x >> 4; x &= x >> 8; x &= W >> 16;  // 17-letter runs
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
            while (Ss) {
                int j = __ffs(Ss) - 1;
                Ss &= Ss - 1;
                uint32_t len = (uint32_t)__ffs(~(W >> j)) - 1u;
                tok[off++] = ((pbase + (uint32_t)j) << 5) | len;
            }
            tcount += total;
            while (Sl) {  // rare: words of 17+ letters
                int j = __ffs(Sl) - 1;
                Sl &= Sl - 1;
                unsigned long long pos = (unsigned long long)(ws + (long long)pbase + j);
                unsigned long long len = run_length(a.text, pos, a.hi);
                long_insert(a.g, a.text + pos, len, 1ull);
            }
            __syncwarp();
            uint32_t b = 0;
            for (; b + 32 <= tcount; b += 32) process(tok[b + lane]);
            const uint32_t rem = tcount - b;
            if (b) {
                uint32_t e = lane < rem ? tok[b + lane] : 0u;
                __syncwarp();
                if (lane < rem) tok[lane] = e;
                __syncwarp();
            }
            tcount = rem;
            L = Ln;
        }
        if ((uint32_t)lane < tcount) process(tok[lane]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C::C1; i += BLOCK) {
        if (stag[i] > 1u) {
            uint4 k = skey[i];
            global_insert(a.g, k, hash_key(k), (unsigned long long)scnt[i]);
        }
    }
}

// Default shape: 256 threads, 8 KB chunks, 2048-slot level-1 table.
constexpr int kBlock = 256, kChunk = 8192, kLogC1 = 11, kMinBlocks = 3;

int count_global_chunk_bytes() { return kChunk; }

cudaError_t launch_count_global(const CountLaunch &c, cudaStream_t s) {
    using C = CountCfg<kBlock, kChunk, kLogC1>;
    auto kern = k_count_global<kBlock, kChunk, kLogC1, kMinBlocks>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (c.hi <= c.lo) return cudaSuccess;
    CountArgs a;
    a.text = c.text;
    a.lo = c.lo;
    a.hi = c.hi;
    unsigned long long n = c.hi - c.lo;
    a.nchunks = (uint32_t)((n + kChunk - 1) / kChunk);
    a.g = c.g;
    int grid = c.grid;
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBlock, C::SMEM);
        grid = sms * (per > 0 ? per : 1);
    }
    if ((uint32_t)grid > a.nchunks) grid = (int)a.nchunks;
    kern<<<grid, kBlock, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace wc
