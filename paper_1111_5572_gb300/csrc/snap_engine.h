// snap_engine.h — per-index align workspaces shared by the batched and the
// plain form (library-private).
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <mutex>
#include <utility>
#include <vector>

#include "snap_internal.h"

namespace snapgpu {

// A launch shape of the batched form (chosen by the autotuner per batch shape).
struct LaunchShape {
    int light_threads;  // threads per block of the thread-per-read bucket
    int warps;          // warps per block of the warp-per-read kernel
    int scap;           // shared-memory candidate slots per warp
};

// What a tuned shape is keyed on: the kernel variant and the batch statistics
// that decide the layout.
struct TuneKey {
    int lvd, light, mmax, Lmax, nmax, nbucket;
    unsigned long long hits;
};

struct Engine {
    // everything an align call on one index needs; guarded by mu
    std::mutex mu;
    cudaStream_t own_stream = nullptr;
    int sms = 0;
    DevBuf stats, head, packed, gtab, ghits, gdense, heavy;
    DevBuf gseeds[4];  // per-class per-warp seed records of long reads
    DevBuf gqbits[4];  // per-class per-warp q-gram bitmaps (large limits)
    DevBuf hseeds;     // probe records of the reads the thread-per-read kernel hands over
    DevBuf hprobed;    // per read: 1 when hseeds holds its records
    DevBuf rcost;      // per read of a block-per-read class: estimated picks (k_read_cost)
    DevBuf rnd;        // per read of such a class: distinct candidates (or kNoCount)
    DevBuf order2;     // such classes' read lists, largest estimate first
    DevBuf cneed;      // per class: the largest candidate-table need k_read_cost found
    unsigned cost_mask = 0;             // classes of this call counted by k_read_cost
    unsigned len_mask = 0;              // warp-per-read classes ordered by read length
    unsigned cost_need[4] = {0, 0, 0, 0};  // their table needs, on the host
    // class launches that run side by side: one stream per class besides the
    // caller's, forked from and joined into the caller's stream by events
    cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[4] = {nullptr, nullptr, nullptr, nullptr};
    bool gtab_ready = false;  // gtab holds only empty slots
    DevBuf h_reads, h_offsets, h_out, h_dmax;  // device copies for the host-buffer entry points
    PinnedBuf pin;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};  // plain-form stage marks
    bool last_light = false;  // the thread-per-read kernel ran in the last call
    uint64_t launches = 0;
    snap_call_stats last{};
    // autotuner and graph replay of the batched form
    bool autotune = true;
    bool use_graphs = true;
    std::vector<std::pair<TuneKey, LaunchShape>> tuned;
    cudaEvent_t tev[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    LaunchShape last_shape{0, 0, 0};
    int last_graph = 0;
    int last_team = 0;  // classes of the last batch that ran one read per block
    int last_wave = 0;  // of those, classes in wave mode
    int last_wave_warps = 0;
    int team = -1;      // -1 chosen per batch, 0 warp per read, 1 team mode, 2 wave mode
    bool last_plain = false;  // the last call ran the plain form (pev marks are valid)
    // host clock when the batch statistics arrived, and the planning time after it
    std::chrono::steady_clock::time_point t_stats;
    double host_plan_ms = 0;
    uint64_t overflow_budget = 4ull << 30;  // device bytes for per-warp global candidate tables
    // plain-form workspace
    DevBuf p_seeds, p_hits, p_hitoff, p_partial, p_table, p_events, p_hitlist, p_items, p_misc,
        p_dense;
};

// Shared by both forms: batch statistics (one small device-to-host copy and
// a stream sync) and the packed read stream.
struct BatchPrep {
    BatchStats st;
    uint32_t* rwords;
    uint64_t base0;
};

inline int grid_cap(int sms, uint64_t n, int threads) {
    uint64_t want = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sms * 16;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

// thread-per-read kernel (snap_light.cu): limits of the reads it takes
constexpr int kLightBucketMaxM = 128;
constexpr int kLightBucketMaxSeeds = 6;    // probe slots on a plain index
// probe slots on a strided index (stride 2: nine probes for a 100 bp read) or with
// the seeds-first variant; its kernel keeps these records in local memory
constexpr int kLightVariantMaxSeeds = 10;
// probe records per read in the hand-over buffer (room for either kernel)
constexpr int kLightHandoverSlots = 10;
constexpr int kLightBucketMaxL = 15;
int light_prepare();
int launch_light(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                 const snap_params* p, snap_result* d_out, cudaStream_t stream,
                 const BatchPrep& bp, uint32_t* heavy_ids, unsigned long long* heavy_count,
                 int threads, SeedRec* hseeds, uint8_t* hprobed);

int prepare_batch(const snap_index* idx, Engine* e, const uint8_t* d_reads,
                  const uint64_t* d_offsets, uint64_t n, const snap_params* p,
                  cudaStream_t stream, BatchPrep* out, const char* where);

}  // namespace snapgpu
