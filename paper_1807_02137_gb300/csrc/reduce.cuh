// reduce.cuh -- deterministic block-wide FP64 reductions shared by the cycle kernels.
#pragma once

namespace segmg {

// Sum of a per-thread double over the block (blockDim.x * blockDim.y <= 1024); the result is
// returned to every thread.  Fixed reduction order: deterministic.
__device__ __forceinline__ double block_sum(double v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        double s = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (tid == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// Sum of a per-thread value of type C over the block, returned to every thread: each warp adds
// its 32 values in C (pairwise, by shuffles), the warp sums are added in FP64 as in block_sum.
// FP64 arithmetic costs much more than FP32 here, so an FP32 value leaves only the block's
// few warp sums to FP64; for C = double this is block_sum.  Fixed order: deterministic.
template <typename C>
__device__ __forceinline__ double block_sum_warps(C v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = (double)v;
    __syncthreads();
    if (tid < 32) {
        double s = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (tid == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// Sums of many per-block partials.  One block adding tens of thousands of FP64 values is bound
// by its loads' latency and by one SM's FP64 rate, so above kSumChunk values the partials are
// first cut into chunks, one block per chunk (k_chunk_sums), and the chunk sums are then added
// in chunk order by one block: a fixed order, as before.
constexpr int kSumChunk = 1024;

// Sum of a[begin, end) over the block, returned to every thread.
__device__ __forceinline__ double chunk_sum(const double *a, int begin, int end, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    double v = 0.0;
    for (int q = begin + tid; q < end; q += nt) v += a[q];
    return block_sum(v, red);
}

// Chunks of the chunked sum of n partials (1: no chunk stage).
inline int sum_blocks(int n) { return n > kSumChunk ? (n + kSumChunk - 1) / kSumChunk : 1; }

__device__ __forceinline__ double block_max(double v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        double s = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
        if (tid == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

template <typename C>
__device__ __forceinline__ C max_t(C a, C b) { return a > b ? a : (b > a ? b : a); }
template <typename C>
__device__ __forceinline__ C abs_t(C a) { return a < C(0) ? -a : a; }

// The same reductions in the type C (FP32 sums stay in FP32); `red` holds 33 doubles.
template <typename C>
__device__ __forceinline__ C block_sum_t(C v, double *red) {
    if (sizeof(C) == 8) return (C)block_sum((double)v, red);
    C *rf = reinterpret_cast<C *>(red);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) rf[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        C s = tid < (nt + 31) / 32 ? rf[tid] : C(0);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (tid == 0) rf[32] = s;
    }
    __syncthreads();
    C r = rf[32];
    __syncthreads();
    return r;
}

template <typename C>
__device__ __forceinline__ C block_max_t(C v, double *red) {
    C *rf = reinterpret_cast<C *>(red);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v = max_t<C>(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((tid & 31) == 0) rf[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        C s = tid < (nt + 31) / 32 ? rf[tid] : C(0);
        for (int o = 16; o > 0; o >>= 1) s = max_t<C>(s, __shfl_down_sync(0xffffffffu, s, o));
        if (tid == 0) rf[32] = s;
    }
    __syncthreads();
    C r = rf[32];
    __syncthreads();
    return r;
}

}  // namespace segmg
