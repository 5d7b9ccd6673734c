// server.cu -- serving loop with continuous batching over camera streams.
//
// No counterpart in the paper (one camera there).  Streams are admitted by
// an HBM budget: a stream needs its device-resident models plus a ring of six
// input and mask frames; a stream that does not fit waits (FIFO) until others
// leave.  fos_server_submit copies a frame into one of the stream's pinned
// input slots and returns at once; with no free slot, or before admission,
// it refuses the frame (backpressure).  A worker thread runs ticks: each tick
// takes the oldest pending frames of every admitted stream (up to three per
// stream, in order), copies them to the device, runs ONE batched launch over
// all of them (fos_batch: one graph step per frame slot, back to back), and
// copies the masks back.  Three ticks are in flight, on three CUDA streams (input copies,
// kernels, mask copies): frames that arrive while a tick runs are admitted
// into the next one.  Completed frames are delivered into the caller's mask
// buffers and reported by fos_server_poll with their latency.
//
// No allocation or free runs on the worker thread.  A housekeeping thread
// creates an admitted stream's context and device buffers and hands them to
// the worker, which only puts them into a batch slot between ticks; when a
// stream leaves, the worker takes it out of its slot and the housekeeper
// frees its memory (cudaFree waits for the device, which would otherwise
// drain the pipeline).  Pinned host staging (the input slots of copying
// submits, the mask staging for pageable mask buffers) is allocated by the
// first submit of the stream that needs it, on the submitting thread.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"
#include "fos.h"
#include "fos_internal.h"

using namespace fos;

namespace {

using Clock = std::chrono::steady_clock;

double now_us()
{
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Frame {
    int64_t tag;
    uint8_t* host_in;    // pinned slot: rgb (P*3), depth (P*2) at depth_offset(P); or NULL
    const uint8_t* ext_rgb;     // caller's buffers (zero-copy submit) when host_in is NULL
    const uint16_t* ext_depth;
    uint8_t* out_gmm;    // caller's buffers (nullable per method)
    uint8_t* out_pbas;
    bool direct_out;     // the caller's mask buffers are pinned: masks are copied
                         // straight into them (no staging, no host memcpy)
    double t_submit;
};

size_t round16(size_t n) { return (n + 15) / 16 * 16; }

// Byte offset of the depth plane in an input buffer (host slot or device):
// 16-byte aligned whatever the pixel count.
size_t depth_offset(size_t P) { return round16(P * 3); }

// Ticks in flight: the input copies of one tick, the kernels of another and
// the mask copies of a third run at the same time.
constexpr int kTicks = 3;
// Per stream: a ring of kRing device frame buffers (inputs and masks); a tick
// takes up to kTickFrames of a stream's pending frames (consecutive ring
// slots), so a stream has at most kRing frames in flight.
constexpr int kRing = 6, kTickFrames = 3;
size_t round256(size_t n) { return (n + 255) / 256 * 256; }

// True for NULL and for page-locked host memory (cudaHostAlloc /
// cudaHostRegister), which the copy engines can write directly.
bool host_pinned(const void* p)
{
    if (!p) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}
size_t input_bytes(size_t P) { return depth_offset(P) + P * 2; }

struct Stream {
    int id;              // server handle
    int32_t W, H;
    uint32_t stream_id;
    size_t bytes = 0;    // device bytes charged against the budget
    int slot = -1;       // batch slot once admitted
    bool admitting = false;  // the housekeeper is allocating its memory
    bool closing = false;
    fos_ctx* ctx = nullptr;  // its models, from the housekeeper
    std::deque<Frame> pending;
    int inflight = 0;    // frames of this stream in ticks not yet completed
    // by frame number mod kRing; each ring is contiguous (frame k at k
    // frames' bytes), as the batched multi-frame launch takes it
    uint8_t* dbuf = nullptr;                   // the device rings below, one allocation
    uint8_t* d_rgb = nullptr;                  // [kRing][P*3]
    uint16_t* d_dep = nullptr;                 // [kRing][P]
    uint8_t* d_mg = nullptr;                   // [kRing][P]
    uint8_t* d_mp = nullptr;                   // [kRing][P]
    uint8_t* hstage = nullptr;                 // pinned mask staging [kRing][2][P], on first need
    int64_t nframes = 0;
    uint8_t* arena = nullptr;                  // pinned input slots, on the first copying submit
    bool host_alloc = false;                   // a submit is allocating arena or staging now
    int copying = 0;                           // submits writing into a slot (or allocating) now
    std::vector<uint8_t*> free_in;             // free slots of the arena
};

struct TickItem {
    int stream;
    int ring;    // ring slot of the frame
    Frame f;
};

struct Tick {
    std::vector<TickItem> items;
    cudaEvent_t in = nullptr;    // inputs on the device (copy-in stream)
    cudaEvent_t k0 = nullptr;    // kernels start (compute stream, after the input wait)
    cudaEvent_t k = nullptr;     // kernels done (compute stream)
    cudaEvent_t done = nullptr;  // masks in host memory (copy-out stream)
    double t_launch = 0.0;
};

}  // namespace

struct fos_server {
    fos_params prm{};
    size_t budget = 0, used = 0;      // used: device bytes held, freed ones excluded
    int max_streams = 0;
    int resident = 0;                 // streams holding (or being given) a batch slot
    int queue_depth = 16;             // pinned input slots per stream
    fos_batch* batch = nullptr;
    cudaStream_t cs = nullptr;        // batched kernels
    cudaStream_t cin = nullptr;       // input copies
    cudaStream_t cout = nullptr;      // mask copies
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker (and waiting submitters)
    std::condition_variable hcv;      // wakes the housekeeper
    std::vector<Stream*> streams;     // by handle (nullptr once gone)
    std::deque<int> waiting;          // handles waiting for admission
    std::vector<int> ready;           // handles whose memory is ready for a slot
    std::deque<Stream*> dead;         // left their slot; memory to be freed
    bool admit_blocked = false;       // an allocation failed: retry once memory comes back
    std::deque<fos_server_result> results;
    std::thread worker, housekeeper;
    bool stop = false;
    std::string err;
    int64_t ticks = 0, frames_done = 0;
    double busy_us = 0.0, house_us = 0.0, kernel_us = 0.0;
    std::vector<cudaEvent_t> events;  // free tick events (created once, reused)
};

namespace {

// Device bytes of a stream's frame rings (the model is fos_stream_device_bytes).
size_t ring_bytes(size_t P) { return round256(kRing * P * 3) + round256(kRing * P * 2) + 2 * round256(kRing * P); }

size_t stream_bytes(const fos_params* prm, int32_t W, int32_t H)
{
    return fos_stream_device_bytes(W, H, prm) + ring_bytes(size_t(W) * size_t(H));
}

size_t slot_bytes(size_t P) { return round16(input_bytes(P)); }

// Context and device buffers of an admitted stream (housekeeper thread, no lock).
bool allocate_stream(fos_server* s, Stream* st, std::string& why)
{
    fos_params p = s->prm;
    p.stream_id = st->stream_id;
    st->ctx = fos_create(st->W, st->H, &p);
    if (!st->ctx) {
        why = std::string("admission: ") + fos_last_error(nullptr);
        return false;
    }
    const size_t P = size_t(st->W) * size_t(st->H);
    if (dev_alloc(reinterpret_cast<void**>(&st->dbuf), ring_bytes(P)) != cudaSuccess) {
        cudaGetLastError();
        fos_destroy(st->ctx);
        st->ctx = nullptr;
        st->dbuf = nullptr;
        why = "admission: device memory exhausted (frame buffers)";
        return false;
    }
    st->d_rgb = st->dbuf;
    st->d_dep = reinterpret_cast<uint16_t*>(st->dbuf + round256(kRing * P * 3));
    st->d_mg = st->dbuf + round256(kRing * P * 3) + round256(kRing * P * 2);
    st->d_mp = st->d_mg + round256(kRing * P);
    return true;
}

// Everything a stream holds, device and host (housekeeper or destroy; no lock).
void release_stream(Stream* st)
{
    if (st->ctx) fos_destroy(st->ctx);
    st->ctx = nullptr;
    cudaFree(st->dbuf);
    cudaFreeHost(st->arena);
    cudaFreeHost(st->hstage);
    st->dbuf = st->arena = st->hstage = nullptr;
    st->free_in.clear();
}

// Frees what streams that left held and allocates the memory of waiting
// streams, FIFO, while they fit the budget and a batch slot is free.
void housekeeper_main(fos_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (!s->dead.empty()) {
            Stream* st = s->dead.front();
            s->dead.pop_front();
            lk.unlock();
            const double t0 = now_us();
            release_stream(st);
            const double dt = now_us() - t0;
            lk.lock();
            s->used -= st->bytes;
            s->house_us += dt;
            s->admit_blocked = false;  // memory came back: a failed admission may fit now
            delete st;
            continue;
        }
        if (s->stop) break;
        Stream* next = nullptr;
        while (!s->waiting.empty() && !(next = s->streams[s->waiting.front()])) s->waiting.pop_front();
        if (next && !s->admit_blocked && s->resident < s->max_streams && s->used + next->bytes <= s->budget) {
            s->waiting.pop_front();
            s->used += next->bytes;
            s->resident += 1;
            next->admitting = true;
            lk.unlock();
            const double t0 = now_us();
            std::string why;
            const bool ok = allocate_stream(s, next, why);
            const double dt = now_us() - t0;
            lk.lock();
            s->house_us += dt;
            next->admitting = false;
            if (ok) {
                s->ready.push_back(next->id);
                s->cv.notify_all();
            } else {
                s->used -= next->bytes;
                s->resident -= 1;
                s->waiting.push_front(next->id);
                s->err = why;
                s->admit_blocked = true;
            }
            continue;
        }
        s->hcv.wait(lk);
    }
}

// Streams whose memory is ready take a batch slot (worker thread, lock held).
void attach_ready(fos_server* s)
{
    for (int h : s->ready) {
        Stream* st = s->streams[h];
        const int slot = batch_attach(s->batch, st->ctx);
        if (slot < 0) {  // cannot happen: resident streams never exceed the slots
            s->err = "admission: no free batch slot";
            s->resident -= 1;
            s->streams[h] = nullptr;
            s->dead.push_back(st);
            s->hcv.notify_all();
            continue;
        }
        st->slot = slot;
    }
    s->ready.clear();
}

// Streams that asked to close and have nothing left leave their slot; the
// housekeeper frees their memory (worker thread, lock held).
void retire(fos_server* s)
{
    for (size_t h = 0; h < s->streams.size(); ++h) {
        Stream* st = s->streams[h];
        if (!st || !st->closing || !st->pending.empty() || st->inflight > 0 || st->copying > 0 ||
            st->admitting || (st->ctx && st->slot < 0))
            continue;
        s->streams[h] = nullptr;
        if (st->slot >= 0) {
            // all of its ticks have completed, so no step in flight uses it
            batch_detach(s->batch, st->slot);
            st->slot = -1;
            s->resident -= 1;
            s->dead.push_back(st);
            s->hcv.notify_all();
        } else {
            delete st;  // never admitted: holds nothing
        }
    }
}

void publish(fos_server* s, Tick& t)
{
    const double done = now_us();
    for (TickItem& it : t.items) {
        Stream* st = s->streams[it.stream];
        const size_t P = size_t(st->W) * size_t(st->H);
        if (!it.f.direct_out) {
            if (it.f.out_gmm) std::memcpy(it.f.out_gmm, st->hstage + (2 * size_t(it.ring)) * P, P);
            if (it.f.out_pbas) std::memcpy(it.f.out_pbas, st->hstage + (2 * size_t(it.ring) + 1) * P, P);
        }
        if (it.f.host_in) st->free_in.push_back(it.f.host_in);
        fos_server_result r{};
        r.stream = it.stream;
        r.tag = it.f.tag;
        r.status = FOS_OK;
        r.latency_us = done - it.f.t_submit;
        r.queue_us = t.t_launch - it.f.t_submit;
        s->results.push_back(r);
        st->inflight -= 1;
        s->frames_done += 1;
    }
    float ms = 0.f;
    if (t.k0 && t.k && cudaEventElapsedTime(&ms, t.k0, t.k) == cudaSuccess) s->kernel_us += 1e3 * double(ms);
    for (cudaEvent_t* e : {&t.in, &t.k0, &t.k, &t.done})
        if (*e) {
            s->events.push_back(*e);
            *e = nullptr;
        }
}

cudaError_t take_event(fos_server* s, cudaEvent_t* e)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->events.empty()) {
            *e = s->events.back();
            s->events.pop_back();
            return cudaSuccess;
        }
    }
    return cudaEventCreate(e);  // timing enabled: the kernels of a tick are timed
}

void worker_main(fos_server* s)
{
    cudaSetDevice(s->device);
    std::deque<Tick> inflight;
    std::vector<int32_t> slots, counts, ks;
    std::vector<const uint8_t*> rgb, kr;
    std::vector<const uint16_t*> dep, kd;
    std::vector<uint8_t*> mg, mp, kg, kp;
    for (;;) {
        Tick t;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            attach_ready(s);
            retire(s);
            auto ready = [&] {
                if (s->stop || !s->ready.empty()) return true;
                for (Stream* st : s->streams)
                    if (st && st->slot >= 0 && (!st->pending.empty() || st->closing)) return true;
                return false;
            };
            // idle: sleep until a frame arrives, memory is ready for a stream,
            // or a stream asks to close (or re-check every millisecond)
            if (inflight.empty()) s->cv.wait_for(lk, std::chrono::milliseconds(1), ready);
            if (s->stop && inflight.empty()) break;
            attach_ready(s);
            // continuous batching: the oldest frames of every admitted stream,
            // up to kTickFrames consecutive ring slots that no frame in flight
            // still uses (items of one stream are adjacent, in frame order)
            for (size_t h = 0; h < s->streams.size(); ++h) {
                Stream* st = s->streams[h];
                if (!st || st->slot < 0 || st->pending.empty()) continue;
                const int r0 = int(st->nframes % kRing);
                const int take = std::min({int(st->pending.size()), kTickFrames, kRing - st->inflight, kRing - r0});
                for (int k = 0; k < take; ++k) {
                    TickItem it;
                    it.stream = int(h);
                    it.ring = r0 + k;
                    it.f = st->pending.front();
                    st->pending.pop_front();
                    st->nframes += 1;
                    st->inflight += 1;
                    t.items.push_back(it);
                }
            }
        }
        if (!t.items.empty()) {
            slots.clear(); counts.clear(); rgb.clear(); dep.clear(); mg.clear(); mp.clear();
            cudaError_t e = cudaSuccess;
            bool multi = false;
            for (size_t q = 0; q < t.items.size(); ++q) {
                TickItem& it = t.items[q];
                Stream* st = s->streams[it.stream];
                const size_t P = size_t(st->W) * size_t(st->H);
                uint8_t* dr = st->d_rgb + size_t(it.ring) * P * 3;
                uint16_t* dd = st->d_dep + size_t(it.ring) * P;
                const uint8_t* hr = it.f.host_in ? it.f.host_in : it.f.ext_rgb;
                const uint16_t* hd = it.f.host_in ? reinterpret_cast<const uint16_t*>(it.f.host_in + depth_offset(P))
                                                  : it.f.ext_depth;
                if (e == cudaSuccess) e = cudaMemcpyAsync(dr, hr, P * 3, cudaMemcpyHostToDevice, s->cin);
                if (e == cudaSuccess) e = cudaMemcpyAsync(dd, hd, P * 2, cudaMemcpyHostToDevice, s->cin);
                if (q == 0 || t.items[q - 1].stream != it.stream) {  // the stream's first frame in the tick
                    slots.push_back(st->slot);
                    counts.push_back(1);
                    rgb.push_back(dr);
                    dep.push_back(dd);
                    mg.push_back(st->d_mg + size_t(it.ring) * P);
                    mp.push_back(st->d_mp + size_t(it.ring) * P);
                } else {
                    counts.back() += 1;
                    multi = true;
                }
            }
            // the input copies of this tick overlap the previous tick's kernels,
            // its mask copies the next tick's (at most kTicks ticks in flight,
            // and a stream's frames in them use different ring slots)
            if (e == cudaSuccess) e = take_event(s, &t.in);
            if (e == cudaSuccess) e = take_event(s, &t.k0);
            if (e == cudaSuccess) e = take_event(s, &t.k);
            if (e == cudaSuccess) e = take_event(s, &t.done);
            if (e == cudaSuccess) e = cudaEventRecord(t.in, s->cin);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cs, t.in, 0);
            if (e == cudaSuccess) e = cudaEventRecord(t.k0, s->cs);
            t.t_launch = now_us();
            fos_status bst = FOS_OK;
            // one batched graph step per frame slot, back to back on the
            // kernel stream (a stream with k frames takes part in the first k)
            for (int k = 0; e == cudaSuccess && bst == FOS_OK && (k == 0 || multi); ++k) {
                ks.clear(); kr.clear(); kd.clear(); kg.clear(); kp.clear();
                for (size_t j = 0; j < slots.size(); ++j) {
                    if (counts[j] <= k) continue;
                    const fos_ctx* c = fos_batch_stream(s->batch, slots[j]);
                    const size_t P = size_t(c->P);
                    ks.push_back(slots[j]);
                    kr.push_back(rgb[j] + size_t(k) * P * 3);
                    kd.push_back(dep[j] + size_t(k) * P);
                    kg.push_back(mg[j] + size_t(k) * P);
                    kp.push_back(mp[j] + size_t(k) * P);
                }
                if (ks.empty()) break;
                bst = fos_batch_process_device(s->batch, int32_t(ks.size()), ks.data(), kr.data(), kd.data(),
                                               kg.data(), kp.data(), s->cs);
            }
            if (e == cudaSuccess && bst == FOS_OK) e = cudaEventRecord(t.k, s->cs);
            if (e == cudaSuccess && bst == FOS_OK) e = cudaStreamWaitEvent(s->cout, t.k, 0);
            for (TickItem& it : t.items) {
                Stream* st = s->streams[it.stream];
                const size_t P = size_t(st->W) * size_t(st->H);
                uint8_t* og = it.f.direct_out ? it.f.out_gmm : st->hstage + 2 * size_t(it.ring) * P;
                uint8_t* op = it.f.direct_out ? it.f.out_pbas : st->hstage + (2 * size_t(it.ring) + 1) * P;
                if (e == cudaSuccess && bst == FOS_OK && (s->prm.methods & FOS_METHOD_GMM) && og)
                    e = cudaMemcpyAsync(og, st->d_mg + size_t(it.ring) * P, P, cudaMemcpyDeviceToHost, s->cout);
                if (e == cudaSuccess && bst == FOS_OK && (s->prm.methods & FOS_METHOD_PBAS) && op)
                    e = cudaMemcpyAsync(op, st->d_mp + size_t(it.ring) * P, P, cudaMemcpyDeviceToHost, s->cout);
            }
            if (e == cudaSuccess && bst == FOS_OK) e = cudaEventRecord(t.done, s->cout);
            if (e != cudaSuccess || bst != FOS_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->err = e != cudaSuccess ? cudaGetErrorString(e) : fos_batch_last_error(s->batch);
                s->stop = true;
                for (TickItem& it : t.items) {
                    fos_server_result r{};
                    r.stream = it.stream;
                    r.tag = it.f.tag;
                    r.status = e != cudaSuccess ? FOS_ERR_CUDA : bst;
                    s->results.push_back(r);
                    s->streams[it.stream]->inflight -= 1;
                    if (it.f.host_in) s->streams[it.stream]->free_in.push_back(it.f.host_in);
                }
                for (cudaEvent_t ev : {t.in, t.k0, t.k, t.done})
                    if (ev) s->events.push_back(ev);
                s->hcv.notify_all();
                break;
            }
            inflight.push_back(std::move(t));
        }
        // deliver finished ticks; keep at most kTicks in flight
        while (!inflight.empty()) {
            Tick& old = inflight.front();
            const bool full = inflight.size() >= size_t(kTicks);
            const cudaError_t q = full ? cudaEventSynchronize(old.done) : cudaEventQuery(old.done);
            if (q == cudaErrorNotReady) break;
            std::lock_guard<std::mutex> lk(s->mu);
            s->busy_us += now_us() - old.t_launch;
            s->ticks += 1;
            publish(s, old);
            inflight.pop_front();
        }
        if (!inflight.empty() && t.items.empty()) {
            // nothing new to launch: wait for the oldest tick or a new frame
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
    for (Tick& t : inflight) {
        cudaEventSynchronize(t.done);
        std::lock_guard<std::mutex> lk(s->mu);
        publish(s, t);
    }
}

Stream* live_stream(fos_server* s, int32_t stream)
{
    if (stream < 0 || stream >= int32_t(s->streams.size())) return nullptr;
    Stream* st = s->streams[stream];
    return st && !st->closing ? st : nullptr;
}

// Allocates, on first need, a stream's pinned input slots (copying submits)
// and its pinned mask staging (masks bound for pageable buffers), on the
// calling thread without the lock held.  FOS_ERR_BUSY while another submit of
// the stream is allocating them.
fos_status ensure_host_memory(fos_server* s, int32_t stream, bool arena, bool stage)
{
    size_t P;
    bool need_arena, need_stage;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Stream* st = live_stream(s, stream);
        if (!st) return FOS_ERR_INVALID_ARG;
        if (s->stop) return FOS_ERR_STATE;
        if (st->slot < 0) return FOS_ERR_BUDGET;  // still waiting for admission
        need_arena = arena && !st->arena;
        need_stage = stage && !st->hstage;
        if (!need_arena && !need_stage) return FOS_OK;
        if (st->host_alloc) return FOS_ERR_BUSY;
        st->host_alloc = true;
        st->copying += 1;  // keeps the stream from leaving meanwhile
        P = size_t(st->W) * size_t(st->H);
    }
    uint8_t* a = nullptr;
    uint8_t* g = nullptr;
    bool ok = true;
    if (need_arena)
        ok = cudaHostAlloc(reinterpret_cast<void**>(&a), size_t(s->queue_depth) * slot_bytes(P),
                           cudaHostAllocDefault) == cudaSuccess;
    if (ok && need_stage)
        ok = cudaHostAlloc(reinterpret_cast<void**>(&g), kRing * 2 * P, cudaHostAllocDefault) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFreeHost(a);
        a = nullptr;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Stream* st = s->streams[stream];
    st->host_alloc = false;
    st->copying -= 1;
    if (!ok) {
        s->err = "submit: pinned host memory exhausted";
        set_thread_error(s->err.c_str());
        return FOS_ERR_OOM;
    }
    if (a) {
        st->arena = a;
        st->free_in.clear();
        for (int q = 0; q < s->queue_depth; ++q) st->free_in.push_back(a + size_t(q) * slot_bytes(P));
    }
    if (g) st->hstage = g;
    return FOS_OK;
}

}  // namespace

extern "C" {

fos_server* fos_server_create(const fos_params* params, size_t hbm_budget_bytes, int32_t max_streams,
                              int32_t queue_depth)
{
    std::string why;
    if (ctx_validate_params(params, why) != FOS_OK || max_streams < 1 || hbm_budget_bytes == 0 ||
        queue_depth < 1 || queue_depth > 1024) {
        set_thread_error(why.empty() ? "fos_server_create: bad arguments" : why.c_str());
        return nullptr;
    }
    fos_server* s = new fos_server();
    s->prm = *params;
    s->budget = hbm_budget_bytes;
    s->max_streams = max_streams;
    s->queue_depth = queue_depth;
    cudaGetDevice(&s->device);
    s->batch = fos_batch_create(max_streams, params);
    if (!s->batch || cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cout, cudaStreamNonBlocking) != cudaSuccess) {
        if (s->batch) fos_batch_destroy(s->batch);
        for (cudaStream_t q : {s->cs, s->cin, s->cout})
            if (q) cudaStreamDestroy(q);
        delete s;
        return nullptr;
    }
    s->worker = std::thread(worker_main, s);
    s->housekeeper = std::thread(housekeeper_main, s);
    return s;
}

void fos_server_destroy(fos_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    s->hcv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->housekeeper.joinable()) s->housekeeper.join();
    // the worker has finished every tick: take the streams out of their slots
    // (the batch would otherwise free their contexts) and free them here
    for (Stream* st : s->dead) {
        release_stream(st);
        delete st;
    }
    for (Stream* st : s->streams) {
        if (!st) continue;
        if (st->slot >= 0) batch_detach(s->batch, st->slot);
        release_stream(st);
        delete st;
    }
    fos_batch_destroy(s->batch);
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    cudaStreamDestroy(s->cs);
    cudaStreamDestroy(s->cin);
    cudaStreamDestroy(s->cout);
    delete s;
}

const char* fos_server_last_error(const fos_server* s) { return s ? s->err.c_str() : ""; }

size_t fos_server_stream_bytes(int32_t width, int32_t height, const fos_params* params)
{
    if (!params || width < 1 || height < 1) return 0;
    return stream_bytes(params, width, height);
}

int32_t fos_server_open_stream(fos_server* s, int32_t width, int32_t height, uint32_t stream_id)
{
    if (!s || width < 1 || height < 1) return -1;
    Stream* st = new Stream();
    st->W = width;
    st->H = height;
    st->stream_id = stream_id;
    st->bytes = stream_bytes(&s->prm, width, height);
    std::lock_guard<std::mutex> lk(s->mu);
    if (st->bytes > s->budget) {
        s->err = "stream needs more device memory than the whole budget";
        delete st;
        return -1;
    }
    st->id = int(s->streams.size());
    s->streams.push_back(st);
    s->waiting.push_back(st->id);
    s->hcv.notify_all();
    return st->id;
}

fos_status fos_server_close_stream(fos_server* s, int32_t stream)
{
    if (!s) return FOS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (stream < 0 || stream >= int32_t(s->streams.size()) || !s->streams[stream]) return FOS_ERR_INVALID_ARG;
    s->streams[stream]->closing = true;
    s->cv.notify_all();
    return FOS_OK;
}

fos_status fos_server_submit(fos_server* s, int32_t stream, const uint8_t* rgb, const uint16_t* depth,
                             uint8_t* mask_gmm, uint8_t* mask_pbas, int64_t tag)
{
    if (!s || !rgb || !depth) return FOS_ERR_INVALID_ARG;
    Frame f{};
    f.tag = tag;
    f.out_gmm = mask_gmm;
    f.out_pbas = mask_pbas;
    f.direct_out = host_pinned(mask_gmm) && host_pinned(mask_pbas);
    const fos_status hs = ensure_host_memory(s, stream, true, !f.direct_out);
    if (hs != FOS_OK) return hs;
    size_t P;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Stream* st = live_stream(s, stream);
        if (!st) return FOS_ERR_INVALID_ARG;
        if (s->stop) return FOS_ERR_STATE;
        if (int(st->pending.size()) + st->inflight + st->copying >= s->queue_depth || st->free_in.empty())
            return FOS_ERR_BUSY;  // queue full
        f.host_in = st->free_in.back();
        st->free_in.pop_back();
        st->copying += 1;
        P = size_t(st->W) * size_t(st->H);
    }
    // the slot belongs to this call until it is queued
    std::memcpy(f.host_in, rgb, P * 3);
    std::memcpy(f.host_in + depth_offset(P), depth, P * 2);
    f.t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->streams[stream]->pending.push_back(f);
        s->streams[stream]->copying -= 1;
    }
    s->cv.notify_all();
    return FOS_OK;
}

fos_status fos_server_submit_nocopy(fos_server* s, int32_t stream, const uint8_t* rgb, const uint16_t* depth,
                                    uint8_t* mask_gmm, uint8_t* mask_pbas, int64_t tag)
{
    if (!s || !rgb || !depth) return FOS_ERR_INVALID_ARG;
    Frame f{};
    f.tag = tag;
    f.ext_rgb = rgb;
    f.ext_depth = depth;
    f.out_gmm = mask_gmm;
    f.out_pbas = mask_pbas;
    f.direct_out = host_pinned(mask_gmm) && host_pinned(mask_pbas);
    const fos_status hs = ensure_host_memory(s, stream, false, !f.direct_out);
    if (hs != FOS_OK) return hs;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Stream* st = live_stream(s, stream);
        if (!st) return FOS_ERR_INVALID_ARG;
        if (s->stop) return FOS_ERR_STATE;
        if (int(st->pending.size()) + st->inflight + st->copying >= s->queue_depth) return FOS_ERR_BUSY;
        f.t_submit = now_us();
        st->pending.push_back(f);
    }
    s->cv.notify_all();
    return FOS_OK;
}

int32_t fos_server_poll(fos_server* s, fos_server_result* out, int32_t max_results)
{
    if (!s || !out || max_results < 1) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    int32_t n = 0;
    while (n < max_results && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    return n;
}

fos_status fos_server_stats(fos_server* s, fos_server_stats_t* out)
{
    if (!s || !out) return FOS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->ticks = s->ticks;
    out->frames_done = s->frames_done;
    out->device_bytes_used = s->used;
    int32_t active = 0, waiting = 0;
    for (Stream* st : s->streams)
        if (st) (st->slot >= 0 ? active : waiting) += 1;
    out->streams_active = active;
    out->streams_waiting = waiting;
    out->busy_us = s->busy_us;
    out->housekeeping_us = s->house_us;
    out->kernel_us = s->kernel_us;
    return s->stop && !s->err.empty() ? FOS_ERR_CUDA : FOS_OK;
}

}  // extern "C"
