// The reduce of the paper's hybrid pipeline (Sec. 3.3 "Reduce on GPU",
// measured in Sec. 4.1): the host has mapped every document to a dictionary
// and laid the per-document counts of each word out as one row of a
// zero-padded matrix; the GPU sums each row.  Here one warp sums one row
// with coalesced loads and a shuffle reduction and writes one 64-bit total;
// warps take rows in a grid-stride loop.  It reads the matrix once: bound by
// HBM (rows x cols x 4 bytes read, rows x 8 written).
#include <cuda_runtime.h>

#include <cstdint>

#include "wc_internal.h"

namespace wc {

__global__ void k_row_sums(const uint32_t *m, unsigned long long rows, unsigned long long cols,
                           unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long r = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
        const uint32_t *row = m + r * cols;
        unsigned long long s = 0;
        unsigned long long c = lane;
        for (; c + 96 < cols; c += 128)  // four independent loads in flight per lane
            s += (unsigned long long)__ldg(row + c) + __ldg(row + c + 32) + __ldg(row + c + 64) + __ldg(row + c + 96);
        for (; c < cols; c += 32) s += __ldg(row + c);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) out[r] = s;
    }
}

cudaError_t launch_row_sums(const uint32_t *m, unsigned long long rows, unsigned long long cols,
                            unsigned long long *out, cudaStream_t s) {
    if (!rows) return cudaSuccess;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long want = (rows + 7) / 8;  // 8 warps (rows) a block
    const unsigned long long cap = (unsigned long long)(sms > 0 ? sms : 1) * 16;
    k_row_sums<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(m, rows, cols, out);
    return cudaGetLastError();
}

}  // namespace wc
