// server.cu -- continuous-batching server on one GPU (include/dc.h, dc_server_*).
//
// The paper has no serving system; this serves the chain to several sensors
// whose frames arrive one at a time.  One worker thread owns all device work:
//   admit     a submitted frame takes a free device slot (room for an input
//             frame of the largest size; the frame lies dense in it, so its
//             copy is contiguous) and is copied in on the upload stream; with
//             no free slot it waits (back-pressure);
//   batch     the uploaded frames form a batch when max_batch are ready or the
//             oldest has waited deadline_us since its submission, and the batch
//             runs as one dc_complete on a free lane (its own context, scratch
//             reserved for a full batch, stream, and an output buffer in which
//             the batch's results lie dense), followed on that stream by the
//             copies of every result into the caller's host buffer;
//   complete  when a lane's kernels have passed, its frames' slots are free
//             again (a slot is held from its copy in to the end of the kernels,
//             not to the end of the copies out); when its copies have passed,
//             its frames are reported done with their latency (submission to
//             result in host memory) and the lane is free again.
// Submission and polling only touch two queues under a mutex, so any thread
// may call them while the worker runs.
#include "../../include/dc.h"
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <utility>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    const float* in = nullptr;
    float* out = nullptr;
    int H = 0, W = 0;
    unsigned long long tag = 0;
    Clock::time_point t0;
    int slot = -1;
    int ev = -1;   // upload event recorded after its copy in
    int ups = -1;  // the upload stream it was copied on
};

// Copies in round-robin over kUploadStreams streams and copies out over
// kDownloadStreams streams per lane, so that several transfers are in flight
// at once and each one's start-up is hidden behind the others.
constexpr int kUploadStreams = 4;
constexpr int kDownloadStreams = 2;

struct Lane {
    dc_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaStream_t down[kDownloadStreams] = {};
    cudaEvent_t down_done[kDownloadStreams] = {};
    cudaEvent_t kernels = nullptr;  // after the batch's kernels: its slots are free
    cudaEvent_t done = nullptr;     // after its copies out
    float* d_out = nullptr;         // the batch's results, dense
    bool busy = false;
    bool slots_held = false;
    std::vector<Req> batch;
};

constexpr int kUploadEvents = 8192;  // more than any number of slots: an event is re-recorded
                                     // only after the frame that last used it was batched

}  // namespace

struct dc_server {
    int device = 0;
    dc_params params{};
    int Hmax = 0, Wmax = 0;
    size_t slot_floats = 0;
    int n_slots = 0;
    int deadline_us = 0;
    int max_batch = 1;
    float* d_in = nullptr;
    cudaStream_t upload[kUploadStreams] = {};
    int up_turn = 0;
    std::vector<cudaEvent_t> up_ev;
    int up_next = 0;
    std::vector<Lane> lanes;
    std::vector<int> free_slots;
    std::deque<Req> waiting, ready;  // worker only

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> submitted;                                   // under mu
    std::deque<std::pair<unsigned long long, double>> finished;  // under mu
    dc_status sticky = DC_OK;                                    // under mu
    bool stopping = false;                                       // under mu
    std::atomic<unsigned long long> n_submitted{0}, n_done{0}, n_batches{0};
    std::thread worker;

    void fail(dc_status s)
    {
        std::lock_guard<std::mutex> g(mu);
        if (sticky == DC_OK) sticky = s;
    }
    void run();
};

void dc_server::run()
{
    cudaSetDevice(device);
    std::vector<dc_frame> frames;
    for (;;) {
        bool progress = false;
        bool stop_now = false;
        {
            std::lock_guard<std::mutex> g(mu);
            while (!submitted.empty()) {
                waiting.push_back(submitted.front());
                submitted.pop_front();
                progress = true;
            }
            stop_now = stopping;
        }
        // admit: copy into free slots
        while (!waiting.empty() && !free_slots.empty()) {
            Req r = waiting.front();
            waiting.pop_front();
            r.slot = free_slots.back();
            free_slots.pop_back();
            // a frame lies dense in its slot (row pitch W): one contiguous copy
            float* dst = d_in + (size_t)r.slot * slot_floats;
            r.ups = up_turn;
            up_turn = (up_turn + 1) % kUploadStreams;
            if (cudaMemcpyAsync(dst, r.in, (size_t)r.H * r.W * sizeof(float), cudaMemcpyHostToDevice,
                                upload[r.ups]) != cudaSuccess ||
                cudaEventRecord(up_ev[up_next], upload[r.ups]) != cudaSuccess) {
                cudaGetLastError();
                fail(DC_ERR_CUDA);
            }
            r.ev = up_next;
            up_next = (up_next + 1) % kUploadEvents;
            ready.push_back(r);
            progress = true;
        }
        // complete: lanes whose kernels have passed give their slots back;
        // lanes whose results are in host memory report them
        const Clock::time_point now = Clock::now();
        for (Lane& l : lanes) {
            if (!l.busy) continue;
            if (l.slots_held) {
                const cudaError_t qk = cudaEventQuery(l.kernels);
                if (qk == cudaErrorNotReady) continue;
                if (qk != cudaSuccess) {
                    cudaGetLastError();
                    fail(DC_ERR_CUDA);
                }
                for (const Req& r : l.batch) free_slots.push_back(r.slot);
                l.slots_held = false;
                progress = true;
            }
            const cudaError_t q = cudaEventQuery(l.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                fail(DC_ERR_CUDA);
            }
            const Clock::time_point t = Clock::now();
            {
                std::lock_guard<std::mutex> g(mu);
                for (const Req& r : l.batch)
                    finished.emplace_back(r.tag, std::chrono::duration<double, std::milli>(t - r.t0).count());
            }
            n_done += l.batch.size();
            ++n_batches;
            l.batch.clear();
            l.busy = false;
            progress = true;
        }
        // batch: full, or the oldest frame at its deadline (or shutting down)
        for (Lane& l : lanes) {
            if (l.busy || ready.empty()) continue;
            const bool due = (int)ready.size() >= max_batch || stop_now ||
                             std::chrono::duration_cast<std::chrono::microseconds>(now - ready.front().t0).count() >=
                                 deadline_us;
            if (!due) break;
            const int n = std::min<int>(max_batch, (int)ready.size());
            l.batch.assign(ready.begin(), ready.begin() + n);
            ready.erase(ready.begin(), ready.begin() + n);
            frames.resize((size_t)n);
            int last_ev[kUploadStreams];
            for (int k = 0; k < kUploadStreams; ++k) last_ev[k] = -1;
            size_t off = 0;  // results lie dense in the lane's output buffer
            for (int i = 0; i < n; ++i) {
                const Req& r = l.batch[(size_t)i];
                frames[(size_t)i] = dc_frame{d_in + (size_t)r.slot * slot_floats, l.d_out + off, r.H, r.W, r.W, r.W};
                off += (size_t)r.H * r.W;
                last_ev[r.ups] = r.ev;  // uploads are in order per stream: its last one covers the batch's
            }
            dc_status s = DC_OK;
            for (int k = 0; s == DC_OK && k < kUploadStreams; ++k)
                if (last_ev[k] >= 0 && cudaStreamWaitEvent(l.st, up_ev[last_ev[k]], 0) != cudaSuccess) s = DC_ERR_CUDA;
            if (s == DC_OK) s = dc_complete(l.ctx, frames.data(), n, &params, l.st);
            if (s == DC_OK && cudaEventRecord(l.kernels, l.st) != cudaSuccess) s = DC_ERR_CUDA;
            for (int k = 0; s == DC_OK && k < kDownloadStreams; ++k)
                if (cudaStreamWaitEvent(l.down[k], l.kernels, 0) != cudaSuccess) s = DC_ERR_CUDA;
            for (int i = 0; s == DC_OK && i < n; ++i) {
                const Req& r = l.batch[(size_t)i];
                if (cudaMemcpyAsync(r.out, frames[(size_t)i].out, (size_t)r.H * r.W * sizeof(float),
                                    cudaMemcpyDeviceToHost, l.down[i % kDownloadStreams]) != cudaSuccess)
                    s = DC_ERR_CUDA;
            }
            for (int k = 0; s == DC_OK && k < kDownloadStreams; ++k)
                if (cudaEventRecord(l.down_done[k], l.down[k]) != cudaSuccess ||
                    cudaStreamWaitEvent(l.st, l.down_done[k], 0) != cudaSuccess)
                    s = DC_ERR_CUDA;
            if (s == DC_OK && cudaEventRecord(l.done, l.st) != cudaSuccess) s = DC_ERR_CUDA;
            l.slots_held = true;
            if (s != DC_OK) {
                cudaGetLastError();
                fail(s);
            }
            l.busy = true;
            progress = true;
        }
        bool busy = !ready.empty() || !waiting.empty();
        for (const Lane& l : lanes) busy = busy || l.busy;
        if (stop_now && !busy) {
            std::lock_guard<std::mutex> g(mu);
            if (submitted.empty()) return;
            continue;
        }
        if (!progress) {
            std::unique_lock<std::mutex> g(mu);
            if (submitted.empty() && !stopping) {
                // work in flight: poll again shortly; idle: sleep until a submission
                if (busy) cv.wait_for(g, std::chrono::microseconds(20));
                else cv.wait(g, [this] { return !submitted.empty() || stopping; });
            }
        }
    }
}

extern "C" {

dc_status dc_server_create(dc_server** out, int device, int max_H, int max_W, size_t budget_bytes,
                           int deadline_us, int max_batch, int lanes, const dc_params* params)
{
    if (!out || !params || max_H < 1 || max_W < 1 || deadline_us < 0 || max_batch < 1 || lanes < 1 || lanes > 16)
        return DC_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return DC_ERR_CUDA;
    }
    if (device < 0 || device >= count) return DC_ERR_INVALID_ARG;
    dc_server* s = new (std::nothrow) dc_server();
    if (!s) return DC_ERR_OOM;
    s->device = device;
    s->params = *params;
    s->Hmax = max_H;
    s->Wmax = max_W;
    s->deadline_us = deadline_us;
    s->max_batch = max_batch;
    s->slot_floats = (size_t)max_H * max_W;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    dc_status st = DC_OK;
    // each lane: scratch for a full batch of the largest frames (the step-4
    // map as 16-bit keys and as floats, column tops, work lists: about 6
    // bytes a pixel) and the batch's results; each slot one input frame
    const size_t cpitch = ((size_t)max_W + 31) / 32 * 32;
    const size_t lane_bytes = (size_t)max_batch * ((size_t)max_H * cpitch + cpitch) * 6 +
                              (size_t)max_batch * s->slot_floats * sizeof(float) + (8u << 20);
    const size_t slot_bytes = s->slot_floats * sizeof(float);
    if (budget_bytes <= (size_t)lanes * lane_bytes + slot_bytes) st = DC_ERR_OOM;
    if (st == DC_OK) {
        size_t slots = (budget_bytes - (size_t)lanes * lane_bytes) / slot_bytes;
        if (slots > 4096) slots = 4096;
        s->n_slots = (int)slots;
        if (cudaMalloc(&s->d_in, slots * s->slot_floats * sizeof(float)) != cudaSuccess) st = DC_ERR_OOM;
        for (int k = 0; st == DC_OK && k < kUploadStreams; ++k)
            if (cudaStreamCreateWithFlags(&s->upload[k], cudaStreamNonBlocking) != cudaSuccess) st = DC_ERR_CUDA;
        for (int i = 0; i < s->n_slots; ++i) s->free_slots.push_back(s->n_slots - 1 - i);
    }
    if (st == DC_OK) {
        s->up_ev.assign(kUploadEvents, nullptr);
        for (cudaEvent_t& e : s->up_ev)
            if (st == DC_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = DC_ERR_CUDA;
    }
    for (int i = 0; st == DC_OK && i < lanes; ++i) {
        s->lanes.emplace_back();
        Lane& l = s->lanes.back();
        st = dc_create(&l.ctx, device, 0);
        if (st == DC_OK) st = dc_reserve(l.ctx, max_batch, max_H, max_W);
        if (st == DC_OK && cudaMalloc(&l.d_out, (size_t)max_batch * s->slot_floats * sizeof(float)) != cudaSuccess)
            st = DC_ERR_OOM;
        if (st == DC_OK && (cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess ||
                            cudaEventCreateWithFlags(&l.kernels, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess))
            st = DC_ERR_CUDA;
        for (int k = 0; st == DC_OK && k < kDownloadStreams; ++k)
            if (cudaStreamCreateWithFlags(&l.down[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&l.down_done[k], cudaEventDisableTiming) != cudaSuccess)
                st = DC_ERR_CUDA;
    }
    cudaSetDevice(prev);
    if (st != DC_OK) {
        cudaGetLastError();
        dc_server_destroy(s);
        return st;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return DC_OK;
}

dc_status dc_server_submit(dc_server* s, const float* host_in, float* host_out, int H, int W,
                           unsigned long long tag)
{
    if (!s || !host_in || !host_out || H < 1 || W < 1 || H > s->Hmax || W > s->Wmax) return DC_ERR_INVALID_ARG;
    Req r;
    r.in = host_in;
    r.out = host_out;
    r.H = H;
    r.W = W;
    r.tag = tag;
    r.t0 = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->sticky != DC_OK) return s->sticky;
        if (s->stopping) return DC_ERR_INVALID_ARG;
        s->submitted.push_back(r);
    }
    ++s->n_submitted;
    s->cv.notify_one();
    return DC_OK;
}

dc_status dc_server_poll(dc_server* s, unsigned long long* tags, double* latency_ms, int max, int* n_done)
{
    if (!s || !n_done || max < 0 || (max > 0 && !tags)) return DC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    int n = 0;
    while (n < max && !s->finished.empty()) {
        tags[n] = s->finished.front().first;
        if (latency_ms) latency_ms[n] = s->finished.front().second;
        s->finished.pop_front();
        ++n;
    }
    *n_done = n;
    return s->sticky;
}

dc_status dc_server_get_stats(dc_server* s, dc_server_stats* st)
{
    if (!s || !st) return DC_ERR_INVALID_ARG;
    st->submitted = s->n_submitted.load();
    st->done = s->n_done.load();
    st->batches = s->n_batches.load();
    st->slots = s->n_slots;
    st->lanes = (int)s->lanes.size();
    std::lock_guard<std::mutex> g(s->mu);
    return s->sticky;
}

void dc_server_destroy(dc_server* s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stopping = true;
        }
        s->cv.notify_all();
        s->worker.join();
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (Lane& l : s->lanes) {
        if (l.st) cudaStreamSynchronize(l.st);
        if (l.ctx) dc_destroy(l.ctx);
        cudaFree(l.d_out);
        if (l.kernels) cudaEventDestroy(l.kernels);
        if (l.done) cudaEventDestroy(l.done);
        for (int k = 0; k < kDownloadStreams; ++k) {
            if (l.down[k]) {
                cudaStreamSynchronize(l.down[k]);
                cudaStreamDestroy(l.down[k]);
            }
            if (l.down_done[k]) cudaEventDestroy(l.down_done[k]);
        }
        if (l.st) cudaStreamDestroy(l.st);
    }
    for (int k = 0; k < kUploadStreams; ++k)
        if (s->upload[k]) {
            cudaStreamSynchronize(s->upload[k]);
            cudaStreamDestroy(s->upload[k]);
        }
    for (cudaEvent_t e : s->up_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(s->d_in);
    cudaGetLastError();
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
