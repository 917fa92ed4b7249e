// Continuous-batching step server (the serving pattern around the rollout step).
//
// A host thread owns one CUDA stream and runs iterations.  Each iteration:
//   1. admission: queued requests join, first come first served, while their
//      agents fit in the batch capacity and the device copy of their inputs
//      fits in the context's memory budget (otherwise they wait);
//   2. one pack kernel gathers every active request's agents into one batch:
//      states (from the previous batch, or from the request's input copy when
//      it was just admitted), this step's commands and scene ids;
//   3. one dynamics launch and one persistent ray-cast launch over the batch;
//   4. images of requests that want them and the final states of requests that
//      ran their last step are copied out, and an event marks each finished
//      request; finished requests leave the batch before the next iteration.
// Up to two iterations are in flight, so the host prepares iteration k+1 while
// the GPU runs k.  Requests arriving at any time join at the next iteration:
// their work overlaps on the device with requests already running.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "visfly_b300.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kRing = 4;

struct PackEntry {
    const float* src_state;  // [17][src_stride], pointing at the request's first agent
    const float* cmd;        // [4][n] commands of this step
    int32_t src_stride;
    int32_t n;
    int32_t off;             // first slot of the request in the new batch
    int32_t scene;
};

// Slot i of the new batch: find its request (entries sorted by off), copy the
// agent's state, this step's command and the scene id.
__global__ void pack_kernel(const PackEntry* __restrict__ tab, int R, int N, float* __restrict__ state,
                            float* __restrict__ cmd, int32_t* __restrict__ ids) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].off <= i) lo = mid;
        else hi = mid - 1;
    }
    const PackEntry e = tab[lo];
    const int j = i - e.off;
#pragma unroll
    for (int k = 0; k < vf::kStateDim; ++k) state[(size_t)k * N + i] = e.src_state[(size_t)k * e.src_stride + j];
#pragma unroll
    for (int k = 0; k < vf::kCmdDim; ++k) cmd[(size_t)k * N + i] = e.cmd[(size_t)k * e.n + j];
    ids[i] = e.scene;
}

enum class St { Queued, Active, Draining, Done };

struct Req {
    int64_t ticket = 0;
    sim_request spec{};
    Clock::time_point t_submit;
    St st = St::Queued;
    int code = SIM_OK;
    bool cancel = false;
    float* d_in = nullptr;  // device copy of the inputs: state0 [17][n] then cmds [T][4][n]
    size_t d_bytes = 0;
    int step = 0;
    int off = -1;           // first slot in the current batch (-1: not yet packed)
    int off_next = 0;
    cudaEvent_t ev = nullptr;
    double latency_ms = 0.0;
};

}  // namespace

struct sim_server {
    sim_ctx* ctx = nullptr;
    int device = 0;
    int cap = 0;
    int W = 0, H = 0;
    cudaStream_t stream = nullptr;
    float* d_state[2] = {nullptr, nullptr};
    float* d_cmd = nullptr;
    int32_t* d_ids = nullptr;
    float* d_depth = nullptr;
    uint8_t* d_rgb = nullptr;
    unsigned* d_counters = nullptr;
    PackEntry* d_tab[kRing] = {};
    PackEntry* h_tab[kRing] = {};
    cudaEvent_t it_ev[kRing] = {};
    std::vector<std::pair<void*, size_t>> owned;
    // per-request input blocks come from this stream-ordered pool: admitting
    // and retiring requests never synchronises the device
    cudaMemPool_t pool = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::unordered_map<int64_t, Req*> all;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread th;

    // server-thread state
    std::vector<Req*> active, draining;
    int cur = 0;
    int n_prev = 0;
    int64_t iter = 0;

    // statistics (under mu)
    int64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, iterations = 0, agent_frames = 0;
    int64_t active_requests = 0, active_agents = 0;
};

namespace {

void finish(sim_server* S, Req* r, int code) {
    // caller holds S->mu
    r->code = code;
    r->st = St::Done;
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    if (code == SIM_OK) ++S->completed;
    else if (r->cancel) ++S->cancelled;
    else ++S->failed;
    S->cv_done.notify_all();
}

void release_inputs(sim_server* S, Req* r) {
    if (r->d_in) vf::ctx_free_pool(S->ctx, r->d_in, r->d_bytes, S->stream);
    r->d_in = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
}

void poll_draining(sim_server* S) {
    std::vector<Req*> still;
    for (Req* r : S->draining) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) {
            still.push_back(r);
            continue;
        }
        release_inputs(S, r);
        std::lock_guard<std::mutex> lk(S->mu);
        finish(S, r, q == cudaSuccess ? (r->cancel ? SIM_ERR_INVALID_ARG : SIM_OK) : SIM_ERR_CUDA);
    }
    S->draining.swap(still);
}

// Admit queued requests while agents and memory allow.
void admit(sim_server* S, int& n_active) {
    for (;;) {
        Req* r = nullptr;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->queue.empty()) return;
            r = S->queue.front();
            if (r->cancel) {
                S->queue.pop_front();
                finish(S, r, SIM_ERR_INVALID_ARG);
                continue;
            }
            if (n_active + r->spec.n_agents > S->cap) return;
        }
        const int n = r->spec.n_agents, T = r->spec.n_steps;
        const size_t bytes = sizeof(float) * ((size_t)vf::kStateDim * n + (size_t)T * vf::kCmdDim * n);
        void* p = nullptr;
        const int rc = vf::ctx_alloc_pool(S->ctx, bytes, &p, S->pool, S->stream);
        // memory admission: wait until memory frees up, unless nothing is running
        // that could free it (then the request can never fit the budget)
        if (rc == SIM_ERR_BUDGET && (!S->active.empty() || !S->draining.empty())) return;
        std::lock_guard<std::mutex> lk(S->mu);
        S->queue.pop_front();
        if (rc != SIM_OK) {
            finish(S, r, rc);
            continue;
        }
        r->d_in = static_cast<float*>(p);
        r->d_bytes = bytes;
        cudaError_t e = cudaMemcpyAsync(r->d_in, r->spec.state0, sizeof(float) * vf::kStateDim * n, cudaMemcpyDefault,
                                        S->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->d_in + (size_t)vf::kStateDim * n, r->spec.cmds,
                                sizeof(float) * (size_t)T * vf::kCmdDim * n, cudaMemcpyDefault, S->stream);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            vf::ctx_free_pool(S->ctx, r->d_in, r->d_bytes, S->stream);
            r->d_in = nullptr;
            finish(S, r, SIM_ERR_CUDA);
            continue;
        }
        r->st = St::Active;
        r->off = -1;
        S->active.push_back(r);
        n_active += n;
        ++S->active_requests;
        S->active_agents += n;
    }
}

void fail_active(sim_server* S, int code) {
    cudaStreamSynchronize(S->stream);
    for (Req* r : S->active) {
        release_inputs(S, r);
        std::lock_guard<std::mutex> lk(S->mu);
        finish(S, r, code);
        --S->active_requests;
        S->active_agents -= r->spec.n_agents;
    }
    S->active.clear();
    S->n_prev = 0;
}

// One batch iteration over the active requests.
void iterate(sim_server* S) {
    // cancelled active requests leave the batch without outputs
    {
        std::vector<Req*> keep;
        for (Req* r : S->active) {
            bool c;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                c = r->cancel;
            }
            if (!c) {
                keep.push_back(r);
                continue;
            }
            cudaEventRecord(r->ev, S->stream);
            r->st = St::Draining;
            S->draining.push_back(r);
            std::lock_guard<std::mutex> lk(S->mu);
            --S->active_requests;
            S->active_agents -= r->spec.n_agents;
        }
        S->active.swap(keep);
    }
    if (S->active.empty()) return;
    const int slot = (int)(S->iter % kRing);
    if (S->iter >= kRing) cudaEventSynchronize(S->it_ev[slot]);  // the pinned table slot is free again
    float* A = S->d_state[S->cur];
    float* Bs = S->d_state[S->cur ^ 1];
    PackEntry* h = S->h_tab[slot];
    int R = 0, N = 0;
    for (Req* r : S->active) {
        const int n = r->spec.n_agents;
        PackEntry& e = h[R++];
        e.src_state = r->off >= 0 ? A + r->off : r->d_in;
        e.src_stride = r->off >= 0 ? S->n_prev : n;
        e.cmd = r->d_in + (size_t)vf::kStateDim * n + (size_t)r->step * vf::kCmdDim * n;
        e.n = n;
        e.off = N;
        e.scene = r->spec.scene_id;
        r->off_next = N;
        N += n;
    }
    cudaError_t e = cudaMemcpyAsync(S->d_tab[slot], h, sizeof(PackEntry) * R, cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) {
        pack_kernel<<<(N + 255) / 256, 256, 0, S->stream>>>(S->d_tab[slot], R, N, Bs, S->d_cmd, S->d_ids);
        e = cudaGetLastError();
    }
    int rc = e == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
    if (rc == SIM_OK) rc = vf::ctx_step(S->ctx, N, Bs, S->d_cmd, S->stream);
    if (rc == SIM_OK) rc = vf::ctx_render_own(S->ctx, N, S->d_ids, Bs, S->d_depth, S->d_rgb, S->d_counters, S->stream);
    if (rc != SIM_OK) {
        fail_active(S, rc);
        return;
    }
    const size_t px = (size_t)S->W * S->H;
    std::vector<Req*> keep;
    for (Req* r : S->active) {
        const int n = r->spec.n_agents;
        const bool last = r->step == r->spec.n_steps - 1;
        const sim_request& q = r->spec;
        if (q.frames == 2 || (q.frames == 1 && last)) {
            const size_t k = q.frames == 2 ? (size_t)r->step : 0;
            if (q.depth_out && e == cudaSuccess)
                e = cudaMemcpyAsync(q.depth_out + k * n * px, S->d_depth + (size_t)r->off_next * px,
                                    sizeof(float) * n * px, cudaMemcpyDefault, S->stream);
            if (q.rgb_out && e == cudaSuccess)
                e = cudaMemcpyAsync(q.rgb_out + k * n * px * 3, S->d_rgb + (size_t)r->off_next * px * 3, 3 * n * px,
                                    cudaMemcpyDefault, S->stream);
        }
        r->off = r->off_next;
        ++r->step;
        if (last) {
            if (q.state_out && e == cudaSuccess)
                e = cudaMemcpy2DAsync(q.state_out, sizeof(float) * n, Bs + r->off, sizeof(float) * N,
                                      sizeof(float) * n, vf::kStateDim, cudaMemcpyDefault, S->stream);
            if (e == cudaSuccess) e = cudaEventRecord(r->ev, S->stream);
            r->st = St::Draining;
            S->draining.push_back(r);
            std::lock_guard<std::mutex> lk(S->mu);
            --S->active_requests;
            S->active_agents -= n;
        } else {
            keep.push_back(r);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail_active(S, SIM_ERR_CUDA);
        return;
    }
    S->active.swap(keep);
    cudaEventRecord(S->it_ev[slot], S->stream);
    S->cur ^= 1;
    S->n_prev = N;
    ++S->iter;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->iterations;
        S->agent_frames += N;
    }
    if (S->iter >= 2) cudaEventSynchronize(S->it_ev[(S->iter - 2) % kRing]);  // two iterations in flight
}

void server_main(sim_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            if (S->active.empty() && S->draining.empty() && S->queue.empty())
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return S->stop || !S->queue.empty(); });
            if (S->stop) break;
        }
        int n_active = 0;
        for (Req* r : S->active) n_active += r->spec.n_agents;
        admit(S, n_active);
        iterate(S);
        poll_draining(S);
        if (S->active.empty() && !S->draining.empty()) {
            // nothing to run: wait for the outstanding copies instead of spinning
            cudaStreamSynchronize(S->stream);
            poll_draining(S);
        }
    }
    cudaStreamSynchronize(S->stream);
    for (Req* r : S->active) S->draining.push_back(r);
    S->active.clear();
    for (Req* r : S->draining) {
        release_inputs(S, r);
        std::lock_guard<std::mutex> lk(S->mu);
        if (r->st != St::Done) {
            r->cancel = true;
            finish(S, r, SIM_ERR_INVALID_ARG);
        }
    }
    S->draining.clear();
}

int alloc_owned(sim_server* S, size_t bytes, void** p) {
    const int rc = vf::ctx_alloc_ext(S->ctx, bytes, p);
    if (rc == SIM_OK) S->owned.emplace_back(*p, bytes);
    return rc;
}

void free_server(sim_server* S) {
    for (auto& pr : S->owned) vf::ctx_free_ext(S->ctx, pr.first, pr.second);
    S->owned.clear();
    for (int k = 0; k < kRing; ++k) {
        if (S->h_tab[k]) cudaFreeHost(S->h_tab[k]);
        if (S->it_ev[k]) cudaEventDestroy(S->it_ev[k]);
    }
    if (S->stream) {
        cudaStreamSynchronize(S->stream);
        cudaStreamDestroy(S->stream);
    }
    if (S->pool) cudaMemPoolDestroy(S->pool);
    for (auto& kv : S->all) {
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        delete kv.second;
    }
    S->all.clear();
    delete S;
}

}  // namespace

extern "C" {

int sim_server_create(sim_ctx* ctx, sim_server** out, int32_t capacity) {
    if (!ctx || !out) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (capacity < 1 || capacity > (1 << 20)) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "capacity out of range");
    sim_server* S = new sim_server();
    S->ctx = ctx;
    S->device = vf::ctx_device(ctx);
    S->cap = capacity;
    vf::ctx_image_size(ctx, &S->W, &S->H);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    const size_t n = (size_t)capacity, px = (size_t)S->W * S->H;
    void* p;
    int rc = SIM_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = SIM_ERR_CUDA;
    if (rc == SIM_OK) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
            cudaGetLastError();
            S->pool = nullptr;
            rc = SIM_ERR_CUDA;
        } else {
            // keep freed blocks in the pool for the next requests
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    for (int k = 0; k < 2 && rc == SIM_OK; ++k)
        if ((rc = alloc_owned(S, sizeof(float) * vf::kStateDim * n, &p)) == SIM_OK) S->d_state[k] = (float*)p;
    if (rc == SIM_OK && (rc = alloc_owned(S, sizeof(float) * vf::kCmdDim * n, &p)) == SIM_OK) S->d_cmd = (float*)p;
    if (rc == SIM_OK && (rc = alloc_owned(S, sizeof(int32_t) * n, &p)) == SIM_OK) S->d_ids = (int32_t*)p;
    if (rc == SIM_OK && (rc = alloc_owned(S, sizeof(float) * n * px, &p)) == SIM_OK) S->d_depth = (float*)p;
    if (rc == SIM_OK && (rc = alloc_owned(S, 3 * n * px, &p)) == SIM_OK) S->d_rgb = (uint8_t*)p;
    if (rc == SIM_OK && (rc = alloc_owned(S, 2 * sizeof(unsigned), &p)) == SIM_OK) S->d_counters = (unsigned*)p;
    for (int k = 0; k < kRing && rc == SIM_OK; ++k) {
        if ((rc = alloc_owned(S, sizeof(PackEntry) * n, &p)) == SIM_OK) S->d_tab[k] = (PackEntry*)p;
        if (rc == SIM_OK && cudaMallocHost((void**)&S->h_tab[k], sizeof(PackEntry) * n) != cudaSuccess) rc = SIM_ERR_OOM;
        if (rc == SIM_OK && cudaEventCreateWithFlags(&S->it_ev[k], cudaEventDisableTiming) != cudaSuccess)
            rc = SIM_ERR_CUDA;
    }
    if (rc == SIM_OK && cudaMemsetAsync(S->d_counters, 0, 2 * sizeof(unsigned), S->stream) != cudaSuccess)
        rc = SIM_ERR_CUDA;
    if (rc == SIM_OK && cudaStreamSynchronize(S->stream) != cudaSuccess) rc = SIM_ERR_CUDA;
    if (prev >= 0) cudaSetDevice(prev);
    if (rc != SIM_OK) {
        free_server(S);
        return rc == SIM_ERR_BUDGET ? rc : vf::ctx_fail(rc, "server set-up failed");
    }
    S->th = std::thread(server_main, S);
    *out = S;
    return SIM_OK;
}

int sim_server_submit(sim_server* S, const sim_request* req, int64_t* ticket) {
    if (!S || !req || !ticket) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "null argument");
    *ticket = 0;
    if (req->n_agents < 1 || req->n_agents > S->cap || req->n_steps < 1 || req->frames < 0 || req->frames > 2 ||
        !req->state0 || !req->cmds)
        return vf::ctx_fail(SIM_ERR_INVALID_ARG, "bad request (agents beyond capacity, steps, frames or inputs)");
    if (!vf::ctx_scene_live(S->ctx, req->scene_id)) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "scene not resident");
    Req* r = new Req();
    r->spec = *req;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return vf::ctx_fail(SIM_ERR_INVALID_ARG, "server stopped");
        }
        r->ticket = S->next_ticket++;
        S->all[r->ticket] = r;
        S->queue.push_back(r);
        ++S->submitted;
    }
    S->cv_work.notify_one();
    *ticket = r->ticket;
    return SIM_OK;
}

int sim_server_wait(sim_server* S, int64_t ticket, int32_t timeout_ms, double* latency_ms) {
    if (!S) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return vf::ctx_fail(SIM_ERR_NOT_FOUND, "unknown ticket");
    Req* r = it->second;
    auto done = [&] { return r->st == St::Done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return vf::ctx_fail(SIM_ERR_TIMEOUT, "request still running");
    if (latency_ms) *latency_ms = r->latency_ms;
    const int code = r->code;
    S->all.erase(it);
    delete r;
    if (code != SIM_OK) return vf::ctx_fail(code, code == SIM_ERR_INVALID_ARG ? "request cancelled" : "request failed");
    return SIM_OK;
}

int sim_server_cancel(sim_server* S, int64_t ticket) {
    if (!S) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return vf::ctx_fail(SIM_ERR_NOT_FOUND, "unknown ticket");
    it->second->cancel = true;
    S->cv_work.notify_one();
    return SIM_OK;
}

int sim_server_stats_get(sim_server* S, sim_server_stats* st) {
    if (!S || !st) return vf::ctx_fail(SIM_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->cancelled = S->cancelled;
    st->failed = S->failed;
    st->iterations = S->iterations;
    st->agent_frames = S->agent_frames;
    st->queued = (int64_t)S->queue.size();
    st->active_requests = S->active_requests;
    st->active_agents = S->active_agents;
    st->mean_batch_agents = S->iterations ? (double)S->agent_frames / S->iterations : 0.0;
    return SIM_OK;
}

int sim_server_destroy(sim_server* S) {
    if (!S) return SIM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Req* r : S->queue) {
            r->cancel = true;
            finish(S, r, SIM_ERR_INVALID_ARG);
        }
        S->queue.clear();
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    free_server(S);
    if (prev >= 0) cudaSetDevice(prev);
    return SIM_OK;
}

}  // extern "C"
