// Read ceiling: one pass over a text that only reads it.  Any kernel that
// reads the text once is bounded by this pass's time, so it is the practical
// HBM limit the counting kernel is measured against, beside the copy
// bandwidth of the measured peaks.
#include <algorithm>

#include "../../include/wc.h"
#include "wc_internal.h"

namespace wc {

constexpr int kCeilThreads = 512;
constexpr int kCeilUnroll = 4;

// 16-byte loads over the aligned middle (kCeilUnroll in flight a thread),
// byte loads over the ragged ends; every byte is folded into one word a
// block, so no load can be dropped.
__global__ void __launch_bounds__(kCeilThreads) k_read_ceiling(const uint8_t *text, unsigned long long n,
                                                               unsigned long long *sink) {
    const uintptr_t b = reinterpret_cast<uintptr_t>(text);
    const uintptr_t a0 = (b + 15) & ~(uintptr_t)15;
    const unsigned long long head = a0 - b < n ? a0 - b : n;
    const unsigned long long nv = (n - head) / 16;  // 16-byte vectors from a0
    const uint4 *v = reinterpret_cast<const uint4 *>(a0);
    unsigned long long acc = 0;
    const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long nt = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long i = tid;
    for (; i + (kCeilUnroll - 1) * nt < nv; i += kCeilUnroll * nt) {
        uint4 x[kCeilUnroll];
#pragma unroll
        for (int u = 0; u < kCeilUnroll; u++) x[u] = __ldcs(v + i + u * nt);
#pragma unroll
        for (int u = 0; u < kCeilUnroll; u++) acc += (unsigned long long)(x[u].x ^ x[u].y) + (x[u].z ^ x[u].w);
    }
    for (; i < nv; i += nt) {
        const uint4 x = __ldcs(v + i);
        acc += (unsigned long long)(x.x ^ x.y) + (x.z ^ x.w);
    }
    const unsigned long long tail0 = head + nv * 16;
    if (tid < head) acc += text[tid];
    if (tid < n - tail0) acc += text[tail0 + tid];
    for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(sink + blockIdx.x, acc);
}

}  // namespace wc

using namespace wc;

wc_status wc_read_ceiling(const uint8_t *d_text, uint64_t nbytes, uint64_t *d_sink, uint32_t sink_words,
                          cudaStream_t stream) {
    if ((!d_text && nbytes) || !d_sink || sink_words == 0) return WC_ERR_INVALID_ARG;
    if (!nbytes) return WC_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned int grid = std::min<unsigned int>(sink_words, (unsigned int)std::max(1, sms) * 8u);
    cudaMemsetAsync(d_sink, 0, 8ull * grid, stream);
    k_read_ceiling<<<grid, kCeilThreads, 0, stream>>>(d_text, nbytes, reinterpret_cast<unsigned long long *>(d_sink));
    return cudaGetLastError() == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}
