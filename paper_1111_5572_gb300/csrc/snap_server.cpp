// snap_server.cpp — the serving loop: continuous batching of alignment requests.
//
// A server owns `max_inflight` slots.  Each slot is a host thread with its own
// CUDA stream and its own align workspaces (an Engine), so requests in different
// slots run on the device at the same time.  Slots take requests from one FIFO
// queue in arrival order; the request at the head is admitted when a slot is
// free and its device footprint fits in the server's memory budget (and in the
// device's free memory); a request that could never fit fails with
// SNAP_E_NOMEM.  Slot workspaces grow to the largest request they served and
// are reused, so the admission test charges a slot only for what a request adds
// to it.  Each request's results are computed read by read exactly as by
// snap_align, so they do not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "snap_engine.h"
#include "snap_internal.h"

using namespace snapgpu;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const uint8_t* reads = nullptr;
    const uint64_t* offsets = nullptr;
    uint64_t n = 0;
    snap_params params{};
    uint64_t need = 0;  // device bytes the request needs in a slot
    Clock::time_point submitted, finished;
    int status = SNAP_OK;
    std::string error;
    std::vector<snap_result> out;
    bool done = false;
};

struct Slot {
    Engine* eng = nullptr;
    cudaStream_t stream = nullptr;
    std::thread th;
    uint64_t footprint = 0;  // device bytes this slot's workspaces hold
};

}  // namespace

struct snap_server {
    const snap_index* idx = nullptr;
    uint64_t budget = 0;
    int device = 0;
    std::vector<Slot> slots;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> requests;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t in_use = 0;
    int running = 0;
};

namespace {

constexpr uint64_t kSlotOverflowBudget = 256ull << 20;  // per-slot global candidate tables

// Device bytes a request needs in a slot: its reads, offsets, results and
// per-read limits, the packed reads and the work lists, plus the slot's
// candidate-table allowance when a read can outgrow shared memory.
uint64_t request_need(const snap_index* idx, const uint8_t*, const uint64_t* offsets, uint64_t n,
                      const snap_params* p) {
    const uint64_t bytes = offsets[n] - offsets[0];
    uint64_t mmax = 0;
    for (uint64_t r = 0; r < n; ++r) mmax = std::max(mmax, offsets[r + 1] - offsets[r]);
    const uint64_t nseeds = p->num_seeds > 0 ? (uint64_t)p->num_seeds : mmax / idx->s;
    const uint64_t hits = nseeds * (uint64_t)std::max(0, p->max_hits);
    uint64_t need = bytes + 16 + 8 * (n + 1) + sizeof(snap_result) * n +
                    (p->max_dist_per_read ? 4 * n : 0) + (bytes + 64) / 4 + 64 + 4 * n + 65536;
    if (2 * hits > 128) need += kSlotOverflowBudget;
    return need;
}

void run_request(snap_server* S, Slot& slot, Request* R) {
    clear_error();
    Engine* e = slot.eng;
    cudaSetDevice(S->device);
    int rc = SNAP_OK;
    const uint64_t lo = R->offsets[0], hi = R->offsets[R->n];
    auto fail = [&](int code) {
        R->status = code;
        R->error = snap_last_error();
    };
    do {
        if (hi < lo) {
            set_error("snap_server: read offsets decrease");
            fail(SNAP_E_INVAL);
            break;
        }
        if ((rc = e->h_reads.ensure(hi - lo + 16, "read copy")) ||
            (rc = e->h_offsets.ensure((R->n + 1) * 8, "offset copy")) ||
            (rc = e->h_out.ensure(R->n * sizeof(snap_result), "result buffer"))) {
            fail(rc);
            break;
        }
        cudaError_t ce = cudaMemcpyAsync(e->h_reads.p, R->reads + lo, hi - lo,
                                         cudaMemcpyHostToDevice, slot.stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(e->h_offsets.p, R->offsets, (R->n + 1) * 8,
                                 cudaMemcpyHostToDevice, slot.stream);
        snap_params dp = R->params;
        if (ce == cudaSuccess && R->params.max_dist_per_read) {
            if ((rc = e->h_dmax.ensure(R->n * 4, "max_dist copy"))) {
                fail(rc);
                break;
            }
            ce = cudaMemcpyAsync(e->h_dmax.p, R->params.max_dist_per_read, R->n * 4,
                                 cudaMemcpyHostToDevice, slot.stream);
            dp.max_dist_per_read = static_cast<const int32_t*>(e->h_dmax.p);
        }
        if (ce != cudaSuccess) {
            fail(cuda_fail(ce, "snap_server copy in"));
            break;
        }
        const uint8_t* d_reads = static_cast<const uint8_t*>(e->h_reads.p) - lo;
        rc = align_batch_device(S->idx, e, d_reads, static_cast<const uint64_t*>(e->h_offsets.p),
                                R->n, &dp, static_cast<snap_result*>(e->h_out.p), slot.stream,
                                false);
        if (rc) {
            fail(rc);
            break;
        }
        R->out.resize(R->n);
        ce = cudaMemcpyAsync(R->out.data(), e->h_out.p, R->n * sizeof(snap_result),
                             cudaMemcpyDeviceToHost, slot.stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(slot.stream);
        if (ce != cudaSuccess) fail(cuda_fail(ce, "snap_server copy out"));
    } while (false);
    R->finished = Clock::now();
}

void slot_loop(snap_server* S, int k) {
    Slot& slot = S->slots[k];
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        Request* R = nullptr;
        S->cv_work.wait(lock, [&] {
            if (S->stop && S->queue.empty()) return true;
            if (S->queue.empty()) return false;
            Request* h = S->queue.front();
            if (h->need > S->budget) return true;  // can never fit: fail it
            uint64_t grow = h->need > slot.footprint ? h->need - slot.footprint : 0;
            if (S->in_use + grow > S->budget && S->running == 0 && slot.footprint > 0) {
                // nothing runs and idle workspaces block the head of the queue:
                // this slot gives its workspaces back (the others do the same when
                // they wake up)
                engine_release(slot.eng);
                S->in_use -= std::min(S->in_use, slot.footprint);
                slot.footprint = 0;
                grow = h->need;
                S->cv_work.notify_all();
            }
            if (S->in_use + grow > S->budget) return false;
            size_t free_b = 0, total_b = 0;
            if (grow && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                free_b < grow + (64ull << 20) && S->running > 0)
                return false;
            return true;
        });
        if (S->queue.empty()) break;  // stopping
        R = S->queue.front();
        S->queue.pop_front();
        if (R->need > S->budget) {
            R->status = SNAP_E_NOMEM;
            R->error = "snap_server: request needs more device memory than the server budget";
            R->finished = Clock::now();
            R->done = true;
            S->cv_done.notify_all();
            S->cv_work.notify_all();
            continue;
        }
        const uint64_t grow = R->need > slot.footprint ? R->need - slot.footprint : 0;
        S->in_use += grow;
        slot.footprint += grow;
        S->running++;
        lock.unlock();
        run_request(S, slot, R);
        lock.lock();
        S->running--;
        // charge what the slot really holds now
        const uint64_t held = engine_bytes(slot.eng);
        if (held > slot.footprint) {
            S->in_use += held - slot.footprint;
            slot.footprint = held;
        }
        R->done = true;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" int snap_server_create(const snap_index* idx, uint64_t mem_budget_bytes,
                                  int max_inflight, snap_server** out) {
    clear_error();
    if (!out) {
        set_error("snap_server_create: out is NULL");
        return SNAP_E_INVAL;
    }
    *out = nullptr;
    if (!idx) {
        set_error("snap_server_create: index is NULL");
        return SNAP_E_INVAL;
    }
    if (max_inflight < 1 || max_inflight > 64) {
        set_error("snap_server_create: max_inflight %d outside [1, 64]", max_inflight);
        return SNAP_E_INVAL;
    }
    if (mem_budget_bytes == 0) {
        set_error("snap_server_create: zero memory budget");
        return SNAP_E_INVAL;
    }
    snap_server* S = new snap_server();
    S->idx = idx;
    S->budget = mem_budget_bytes;
    S->device = idx->device;
    S->slots.resize(max_inflight);
    cudaSetDevice(S->device);
    for (auto& sl : S->slots) {
        sl.eng = engine_create();
        sl.eng->overflow_budget = kSlotOverflowBudget;
        const cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto& s2 : S->slots) {
                if (s2.stream) cudaStreamDestroy(s2.stream);
                if (s2.eng) engine_destroy(s2.eng);
            }
            delete S;
            return cuda_fail(e, "snap_server_create stream");
        }
    }
    for (int k = 0; k < max_inflight; ++k) S->slots[k].th = std::thread(slot_loop, S, k);
    *out = S;
    return SNAP_OK;
}

extern "C" int snap_server_submit(snap_server* S, const uint8_t* reads, const uint64_t* offsets,
                                  uint64_t n, const snap_params* params, uint64_t* ticket) {
    clear_error();
    if (!S || !offsets || !params || !ticket || (n > 0 && !reads)) {
        set_error("snap_server_submit: NULL argument");
        return SNAP_E_INVAL;
    }
    int rc = validate_params(S->idx, params);
    if (rc) return rc;
    if (offsets[n] < offsets[0]) {
        set_error("snap_server_submit: read offsets decrease");
        return SNAP_E_INVAL;
    }
    Request* R = new Request();
    R->reads = reads;
    R->offsets = offsets;
    R->n = n;
    R->params = *params;
    R->need = request_need(S->idx, reads, offsets, n, params);
    R->submitted = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) {
            delete R;
            set_error("snap_server_submit: server is stopping");
            return SNAP_E_INVAL;
        }
        R->ticket = S->next_ticket++;
        S->requests[R->ticket] = R;
        if (n == 0) {
            R->finished = R->submitted;
            R->done = true;
        } else {
            S->queue.push_back(R);
        }
    }
    S->cv_work.notify_all();
    *ticket = R->ticket;
    return SNAP_OK;
}

extern "C" int snap_server_wait(snap_server* S, uint64_t ticket, snap_result* out,
                                double* latency_s) {
    clear_error();
    if (!S) {
        set_error("snap_server_wait: server is NULL");
        return SNAP_E_INVAL;
    }
    Request* R = nullptr;
    {
        std::unique_lock<std::mutex> lock(S->mu);
        auto it = S->requests.find(ticket);
        if (it == S->requests.end()) {
            set_error("snap_server_wait: unknown ticket %llu", (unsigned long long)ticket);
            return SNAP_E_INVAL;
        }
        R = it->second;
        S->cv_done.wait(lock, [&] { return R->done; });
        S->requests.erase(it);
    }
    const int status = R->status;
    if (status == SNAP_OK) {
        if (out && R->n) std::memcpy(out, R->out.data(), R->n * sizeof(snap_result));
        if (latency_s)
            *latency_s = std::chrono::duration<double>(R->finished - R->submitted).count();
    } else {
        set_error("%s", R->error.c_str());
    }
    delete R;
    return status;
}

extern "C" int snap_server_destroy(snap_server* S) {
    clear_error();
    if (!S) return SNAP_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& sl : S->slots)
        if (sl.th.joinable()) sl.th.join();
    cudaSetDevice(S->device);
    for (auto& sl : S->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        engine_destroy(sl.eng);
    }
    for (auto& kv : S->requests) delete kv.second;
    delete S;
    return SNAP_OK;
}
