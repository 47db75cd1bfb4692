// snap_scan.cuh — exclusive prefix sum over a device array of uint32 values
// (in place allowed), 64-bit lengths, three launches, no inter-block waits.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace snapgpu {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;  // elements per thread per tile

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem_warp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < (kScanThreads / 32)) ? smem_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kScanThreads / 32)) smem_warp[lane] = w;
    }
    __syncthreads();
    const T warp_prefix = (warp > 0) ? smem_warp[warp - 1] : T(0);
    *total = smem_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

// per-chunk sums
template <typename In, typename Acc>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const In* in, uint64_t n,
                                                                   uint64_t chunk, Acc* partial) {
    __shared__ Acc sw[kScanThreads / 32];
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = min(n, b0 + chunk);
    Acc s = 0;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += kScanThreads) s += (Acc)in[i];
    Acc tot;
    block_exclusive_scan<Acc>(s, sw, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// exclusive scan of the chunk sums (one block); grand total to *total
template <typename Acc>
__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(Acc* partial, int nb,
                                                                     Acc* total) {
    __shared__ Acc sw[kScanThreads / 32];
    Acc carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int i = base + threadIdx.x;
        Acc v = (i < nb) ? partial[i] : Acc(0);
        Acc tot;
        Acc ex = block_exclusive_scan<Acc>(v, sw, &tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// out[i] = partial[chunk] + sum of in[chunk start .. i)
template <typename In, typename Out, typename Acc>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const In* in, Out* out,
                                                                  uint64_t n, uint64_t chunk,
                                                                  const Acc* partial) {
    __shared__ Acc sw[kScanThreads / 32];
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = min(n, b0 + chunk);
    Acc carry = partial[blockIdx.x];
    const uint64_t tile = (uint64_t)kScanThreads * kScanItems;
    for (uint64_t t0 = b0; t0 < b1; t0 += tile) {
        Acc v[kScanItems];
        Acc s = 0;
        const uint64_t i0 = t0 + (uint64_t)threadIdx.x * kScanItems;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const uint64_t i = i0 + j;
            v[j] = (i < b1) ? (Acc)in[i] : Acc(0);
            s += v[j];
        }
        Acc tot;
        Acc ex = block_exclusive_scan<Acc>(s, sw, &tot);
        Acc run = carry + ex;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const uint64_t i = i0 + j;
            if (i < b1) out[i] = (Out)run;
            run += v[j];
        }
        carry += tot;
    }
}

// Exclusive scan of n values; partial must hold >= scan_blocks(n) Acc values;
// *total (device) receives the sum.
inline int scan_blocks(uint64_t n) {
    uint64_t nb = (n + 8191) / 8192;
    if (nb > 8192) nb = 8192;
    if (nb < 1) nb = 1;
    return (int)nb;
}

template <typename In, typename Out, typename Acc>
inline void exclusive_scan(const In* in, Out* out, uint64_t n, Acc* partial, Acc* total,
                           cudaStream_t st) {
    const int nb = scan_blocks(n);
    const uint64_t chunk = (n + nb - 1) / nb;
    scan_reduce_kernel<In, Acc><<<nb, kScanThreads, 0, st>>>(in, n, chunk ? chunk : 1, partial);
    scan_partials_kernel<Acc><<<1, kScanThreads, 0, st>>>(partial, nb, total);
    scan_apply_kernel<In, Out, Acc><<<nb, kScanThreads, 0, st>>>(in, out, n, chunk ? chunk : 1,
                                                                  partial);
}

}  // namespace snapgpu
