// Counting without any device allocation, for callers that may not allocate.
//
// Some callers cannot call cudaMalloc (or any allocating routine): code that
// runs while another component owns all device memory through its own
// allocator, real-time services that forbid allocation after start-up (an
// allocation can block on the device or fail under memory pressure at the
// worst moment), and hosts that embed this library where only the buffers
// they pass in may be touched.  wc_count_noalloc serves them: it runs the
// single-document count with every piece of scratch memory (the hash tables
// and the sort scratch) in one file-scope __device__ array of fixed size, and
// writes the sorted table into buffers the caller provides.
//
// The array is a host-side stand-in in host code: its device address is
// obtained once per device with cudaGetSymbolAddress (on the first call on
// that device, with that device current) and passed to the kernels.  Every
// call on a device shares the one array and leaves its contents behind; each
// call clears what must start at zero.  Calls whose work overlaps on the GPU
// (another stream, or a second call before the first has finished) race on
// the array: keep calls on one device in one stream, in order.
#include <cstring>
#include <mutex>

#include "../../include/wc.h"
#include "wc_internal.h"

namespace {

constexpr uint64_t kNaMaxBytes = 1ull << 20;  // largest document accepted (1 MiB)
constexpr uint64_t kNaCap8 = 1ull << 17;      // 8-byte-key slots
constexpr uint64_t kNaCap16 = 1ull << 16;     // 16-byte-key slots
constexpr uint64_t kNaCapLong = 1ull << 13;   // long-word slots
constexpr uint64_t kNaEntries = kNaCap8 + kNaCap16 + kNaCapLong;
constexpr uint64_t kR = 256;
constexpr uint64_t round256(uint64_t n) { return (n + kR - 1) / kR * kR; }
constexpr uint64_t kBytes8 = round256(kNaCap8 * sizeof(wc::G8Slot));
constexpr uint64_t kBytes16 = round256(kNaCap16 * sizeof(wc::GSlot));
constexpr uint64_t kBytesLong = round256(kNaCapLong * sizeof(wc::LSlot));
// Sort scratch for kNaEntries entries (khi, klo, cnt, packed key (8 + 4 bytes),
// lref, 2 permutations, doc, the digit histograms, tile histograms, pass
// cursors, group counts, the look-back buffers and tile counters), each
// carved at a 256-byte boundary.
constexpr uint64_t kNaTiles = (kNaEntries + wc::kSortTileElems - 1) / wc::kSortTileElems;
constexpr uint64_t kSortBytes = kNaEntries * (8 + 8 + 8 + 8 + 4 + 4 + 4 + 4 + 4) + 4 * wc::kSortPassesSeg * 256 +
                                4 * 256 * kNaTiles + 4 * 32 + 2 * 4 * 256 * wc::sort_group_stride(kNaTiles) + 4096 +
                                2 * (4 * 256 * kNaTiles + 256) + 256 + 20 * kR;
constexpr uint64_t kScratchBytes = kBytes8 + kBytes16 + kBytesLong + kSortBytes;  // about 15.5 MB

}  // namespace

// The scratch: held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {
std::mutex g_na_mu;
void *g_na_ptr[256];  // device address of the scratch, per device ordinal

// Looks up the scratch's device address for the current device (once).
wc_status noalloc_setup(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return WC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return WC_ERR_CUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return WC_OK;
}
}  // namespace

extern "C" wc_status wc_count_noalloc(const uint8_t *d_text, uint64_t nbytes, uint64_t *d_khi, uint64_t *d_klo,
                                      uint64_t *d_cnt, uint32_t *d_lref, uint64_t out_cap, uint64_t *d_loff,
                                      uint64_t *d_llen, uint64_t long_cap, uint8_t *d_arena, uint64_t arena_cap,
                                      uint64_t *d_meta, cudaStream_t stream) {
    if (nbytes > kNaMaxBytes) return WC_ERR_UNSUPPORTED;  // larger documents need wc_count
    if ((nbytes && !d_text) || !d_khi || !d_klo || !d_cnt || !d_lref || !d_loff || !d_llen || !d_arena || !d_meta)
        return WC_ERR_INVALID_ARG;
    if (out_cap < kNaEntries || long_cap < kNaCapLong || arena_cap < nbytes + nbytes / 16 + 16)
        return WC_ERR_INVALID_ARG;
    if (wc::sort_scratch_bytes(kNaEntries) > kSortBytes) return WC_ERR_INTERNAL;
    void *base = nullptr;
    wc_status st = noalloc_setup(&base);
    if (st != WC_OK) return st;
    uint8_t *p = static_cast<uint8_t *>(base);
    wc::GTable g;
    g.slots8 = reinterpret_cast<wc::G8Slot *>(p);
    g.mask8 = kNaCap8 - 1;
    g.slots = reinterpret_cast<wc::GSlot *>(p + kBytes8);
    g.mask = kNaCap16 - 1;
    g.lslots = reinterpret_cast<wc::LSlot *>(p + kBytes8 + kBytes16);
    g.lmask = kNaCapLong - 1;
    g.status = reinterpret_cast<uint32_t *>(d_meta + 7);
    wc::SortScratch ss;
    wc::sort_scratch_carve(ss, p + kBytes8 + kBytes16 + kBytesLong, kNaEntries);
    wc::DevTable out;
    out.cap = out_cap;
    out.lcap = long_cap;
    out.arena_cap = arena_cap;
    out.count_bits = 64;
    out.d_meta = reinterpret_cast<unsigned long long *>(d_meta);
    out.d_status = reinterpret_cast<uint32_t *>(d_meta + 7);
    out.khi = reinterpret_cast<unsigned long long *>(d_khi);
    out.klo = reinterpret_cast<unsigned long long *>(d_klo);
    out.cnt = d_cnt;
    out.lref = d_lref;
    out.loff = reinterpret_cast<unsigned long long *>(d_loff);
    out.llen = reinterpret_cast<unsigned long long *>(d_llen);
    out.arena = d_arena;
    // zero what the previous call left: the output metadata and the hash tables
    cudaError_t e = cudaMemsetAsync(d_meta, 0, 64, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, kBytes8 + kBytes16 + kBytesLong, stream);
    wc::CountLaunch cl{d_text, 0, nbytes, g, 0, nullptr, {nullptr, nullptr}};
    if (e == cudaSuccess) e = wc::launch_count_global(cl, stream);
    if (e == cudaSuccess)
        e = wc::finish_table(g, kNaCap8, kNaCap16, kNaCapLong, ss, out, stream, wc::sort_skip_mask(nbytes / 2 + 1, 0));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return WC_ERR_CUDA;
    }
    return WC_OK;
}
