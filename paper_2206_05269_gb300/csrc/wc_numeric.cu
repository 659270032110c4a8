// The paper's numeric MapReduce (Sec. 4.2): map each i in 1..n to a double
// term and reduce with +,
//   series 0: sum_{i=1}^{n} sqrt(i)
//   series 1: sum_{i=1}^{n} (-1)^(i+1) / i      (which tends to ln 2)
// The paper's kernel adds every term into one accumulator with an atomic; here
// every thread sums a strided share of one block's contiguous range with
// Neumaier's compensated summation, the warp and then the block combine their
// (sum, compensation) pairs through shuffles and shared memory, each block
// writes one pair, and a second one-block launch combines the blocks' pairs in
// a fixed order.  The result is deterministic for a given grid, no atomics.
// Terms are IEEE double: sqrt and the division are correctly rounded.
#include <cuda_runtime.h>

#include <cstdint>

#include "wc_internal.h"

namespace wc {

constexpr int kSeriesThreads = 256;

struct Pair {
    double s, c;  // running sum and the rounding errors it has dropped
};

// Neumaier's step: adds x to (s, c).
__device__ __forceinline__ void nadd(Pair &p, double x) {
    const double t = p.s + x;
    p.c += fabs(p.s) >= fabs(x) ? (p.s - t) + x : (x - t) + p.s;
    p.s = t;
}
__device__ __forceinline__ void nmerge(Pair &p, const Pair &q) {
    nadd(p, q.s);
    p.c += q.c;
}

template <int SERIES>
__device__ __forceinline__ double series_term(unsigned long long i) {
    if (SERIES == 0) return sqrt((double)i);
    const double t = 1.0 / (double)i;
    return (i & 1ull) ? t : -t;
}

// Block b sums the terms of i in [lo_b, hi_b), the b-th of gridDim.x equal
// slices of 1..n, and writes its pair to part[b].
template <int SERIES>
__global__ void __launch_bounds__(kSeriesThreads) k_series_part(unsigned long long n, double2 *part) {
    __shared__ Pair warp_pair[kSeriesThreads / 32];
    const unsigned long long per = (n + gridDim.x - 1) / gridDim.x;
    const unsigned long long lo = 1ull + (unsigned long long)blockIdx.x * per;
    unsigned long long hi = lo + per;
    if (hi > n + 1) hi = n + 1;
    Pair p{0.0, 0.0};
    for (unsigned long long i = lo + threadIdx.x; i < hi; i += kSeriesThreads) nadd(p, series_term<SERIES>(i));
    for (int o = 16; o; o >>= 1) {
        Pair q{__shfl_down_sync(0xFFFFFFFFu, p.s, o), __shfl_down_sync(0xFFFFFFFFu, p.c, o)};
        nmerge(p, q);
    }
    if ((threadIdx.x & 31) == 0) warp_pair[threadIdx.x >> 5] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        Pair b = warp_pair[0];
        for (int w = 1; w < kSeriesThreads / 32; w++) nmerge(b, warp_pair[w]);
        part[blockIdx.x] = make_double2(b.s, b.c);
    }
}

// One block combines nb pairs, in order of block index, into *out.
__global__ void __launch_bounds__(kSeriesThreads) k_series_final(const double2 *part, int nb, double *out) {
    __shared__ Pair tpair[kSeriesThreads];
    Pair p{0.0, 0.0};
    // thread t takes a contiguous run of pairs, so the combination order is fixed
    const int per = (nb + kSeriesThreads - 1) / kSeriesThreads;
    for (int k = threadIdx.x * per; k < nb && k < (int)(threadIdx.x + 1) * per; k++) {
        const double2 v = part[k];
        nmerge(p, Pair{v.x, v.y});
    }
    tpair[threadIdx.x] = p;
    __syncthreads();
    for (int w = kSeriesThreads / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) nmerge(tpair[threadIdx.x], tpair[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = tpair[0].s + tpair[0].c;
}

int series_blocks(unsigned long long n) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about 64 terms a thread at least; at most 8 blocks of 256 threads per SM
    unsigned long long want = (n + 64ull * kSeriesThreads - 1) / (64ull * kSeriesThreads);
    const unsigned long long cap = 8ull * (unsigned long long)(sms > 0 ? sms : 1);
    if (want > cap) want = cap;
    return (int)(want ? want : 1);
}

cudaError_t launch_series(int series, unsigned long long n, double2 *part, int nb, double *d_out, cudaStream_t s) {
    if (series == 0) k_series_part<0><<<nb, kSeriesThreads, 0, s>>>(n, part);
    else k_series_part<1><<<nb, kSeriesThreads, 0, s>>>(n, part);
    k_series_final<<<1, kSeriesThreads, 0, s>>>(part, nb, d_out);
    return cudaGetLastError();
}

}  // namespace wc
