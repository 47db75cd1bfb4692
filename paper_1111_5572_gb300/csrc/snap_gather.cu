// snap_gather.cu — the random-gather ceiling that the probe path is measured
// against.  Every index probe, position-list read and genome-window fetch of the
// aligner is a read of a few dozen bytes at an unpredictable address, so a
// streaming copy overstates what HBM can deliver to it; this kernel measures
// what it can: independent reads of one aligned chunk (16 to 128 bytes) each at
// pseudo-random chunk indices of a buffer far larger than L2, at a launch shape
// (chunks in flight per thread, threads per SM) that a sweep can vary.
#include <cuda_runtime.h>

#include <cstdint>

#include "snap_device.cuh"
#include "snap_internal.h"

namespace snapgpu {
namespace {

// Groups of words16 consecutive threads read one chunk together (16 bytes each,
// as a warp reads a bucket or a window), `per_group` chunks per group, ILP at a
// time, at chunk indices mix64(counter) mod n_chunks, folded into one word so
// that no load is dead.
template <int ILP>
__global__ void __launch_bounds__(256) k_gather(const uint4* __restrict__ buf, uint64_t n_chunks,
                                                int words16, uint32_t per_group, uint64_t seed,
                                                uint32_t* __restrict__ sink) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t group = tid / (uint64_t)words16;
    const int part = (int)(tid % (uint64_t)words16);
    uint32_t acc = 0;
    for (uint32_t j0 = 0; j0 < per_group; j0 += ILP) {
        uint4 v[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const uint64_t ctr = (group * per_group + j0 + u) ^ seed;
            const uint64_t chunk = __umul64hi(mix64(ctr), n_chunks);
            v[u] = __ldg(buf + chunk * (uint64_t)words16 + part);
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    sink[tid] = acc;
}

using GatherKernel = void (*)(const uint4*, uint64_t, int, uint32_t, uint64_t, uint32_t*);

}  // namespace
}  // namespace snapgpu

using namespace snapgpu;

extern "C" int snap_measure_gather_config(uint64_t buffer_bytes, uint32_t chunk_bytes,
                                          uint64_t n_reads, int ilp, int threads_per_sm,
                                          double* gbs_out) {
    clear_error();
    if (!gbs_out || (chunk_bytes != 16 && chunk_bytes != 32 && chunk_bytes != 64 &&
                     chunk_bytes != 128) ||
        buffer_bytes < (64ull << 20) || n_reads == 0 ||
        (ilp != 1 && ilp != 2 && ilp != 4 && ilp != 8 && ilp != 16) ||
        threads_per_sm < 256 || threads_per_sm > 2048 || threads_per_sm % 256) {
        set_error("snap_measure_gather: need chunk_bytes 16/32/64/128, buffer_bytes >= 64 MiB, "
                  "n_reads > 0, ilp 1/2/4/8/16, threads_per_sm a multiple of 256 in "
                  "[256, 2048] and an output pointer");
        return SNAP_E_INVAL;
    }
    int dev = 0, sms = 0;
    SNAP_CUDA(cudaGetDevice(&dev), "device");
    SNAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute");
    const int threads = 256;
    const uint64_t blocks = (uint64_t)sms * (threads_per_sm / threads);
    const uint64_t nthreads = blocks * threads;
    const int w16 = (int)(chunk_bytes / 16);
    const uint64_t ngroups = nthreads / w16;
    uint32_t per_group = (uint32_t)((n_reads + ngroups - 1) / ngroups);
    per_group = (per_group + ilp - 1) / ilp * ilp;
    const uint64_t n_chunks = buffer_bytes / chunk_bytes;
    GatherKernel kern = ilp == 1 ? k_gather<1> : ilp == 2 ? k_gather<2> : ilp == 4 ? k_gather<4>
                      : ilp == 8 ? k_gather<8> : k_gather<16>;
    DevBuf buf, sink;
    int rc;
    if ((rc = buf.ensure(n_chunks * chunk_bytes, "gather buffer"))) return rc;
    if ((rc = sink.ensure(nthreads * sizeof(uint32_t), "gather sink"))) {
        buf.release();
        return rc;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto fail = [&](cudaError_t err, const char* what) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        const int code = cuda_fail(err, what);
        buf.release();
        sink.release();
        return code;
    };
    cudaError_t err;
    if ((err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(err, "stream");
    if ((err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess)
        return fail(err, "event");
    if ((err = cudaMemsetAsync(buf.p, 0x5a, n_chunks * chunk_bytes, st)) != cudaSuccess)
        return fail(err, "fill");
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first run warms up
        cudaEventRecord(e0, st);
        kern<<<(unsigned)blocks, threads, 0, st>>>(static_cast<const uint4*>(buf.p), n_chunks, w16,
                                                   per_group, 0x9e3779b97f4a7c15ull * rep,
                                                   static_cast<uint32_t*>(sink.p));
        cudaEventRecord(e1, st);
        if ((err = cudaEventSynchronize(e1)) != cudaSuccess) return fail(err, "gather");
        if ((err = cudaGetLastError()) != cudaSuccess) return fail(err, "gather launch");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    buf.release();  // the buffers are this call's own
    sink.release();
    *gbs_out = (double)ngroups * per_group * chunk_bytes / (best * 1e-3) / 1e9;
    return SNAP_OK;
}

extern "C" int snap_measure_gather(uint64_t buffer_bytes, uint32_t chunk_bytes,
                                   uint64_t n_reads, double* gbs_out) {
    if (chunk_bytes == 128) {  // the four-chunk-size form keeps its original sizes
        clear_error();
        set_error("snap_measure_gather: need chunk_bytes 16/32/64 (128 via "
                  "snap_measure_gather_config)");
        return SNAP_E_INVAL;
    }
    return snap_measure_gather_config(buffer_bytes, chunk_bytes, n_reads, 4, 2048, gbs_out);
}
