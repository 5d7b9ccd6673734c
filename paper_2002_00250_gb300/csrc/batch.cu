// batch.cu -- many camera streams in one launch per frame step.
//
// A batch owns up to max_streams stream contexts (ordinary fos_ctx objects,
// so every single-stream call -- state export, reset, options -- works on
// them).  One frame step of any subset of the streams is one CUDA graph
// replay: a copy of the per-stream kernel arguments from pinned host memory,
// a persistent GMM kernel and a persistent PBAS kernel that walk the
// (stream, tile) work of the step with a grid stride.  The counts are read
// from device memory, so the same graph serves every composition; two graphs
// alternate over two argument buffers so the host can fill one while the
// other is in flight.  Results are bit-identical to processing each stream
// alone: every pixel runs the same code on the same data.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"
#include "fos.h"
#include "fos_internal.h"

using namespace fos;

struct fos_batch {
    fos_params prm{};
    int max_streams = 0;
    int sms = 0;
    std::vector<fos_ctx*> slot;
    // argument buffers: [2] x (gmm entries | pbas entries | header)
    size_t gmm_bytes = 0, pbas_bytes = 0, buf_bytes = 0;
    uint8_t* dev = nullptr;
    uint8_t* host = nullptr;  // pinned
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_key[2] = {-1, -1};
    cudaStream_t cap = nullptr;
    int tick = 0;
    int gmm_px = 2, pbas_px = 2, pbas_ty = 8;  // tuned shapes
    std::string err;
};

namespace {

fos_status bfail(fos_batch* b, fos_status st, const std::string& msg)
{
    if (b) b->err = msg;
    set_thread_error(msg.c_str());
    return st;
}

fos_status bcuda(fos_batch* b, const char* what, cudaError_t e)
{
    char buf[400];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return bfail(b, e == cudaErrorMemoryAllocation ? FOS_ERR_OOM : FOS_ERR_CUDA, buf);
}

#define FOS_BTRY(b, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(b, #call, e_); \
    } while (0)

GmmBatchEntry* dev_gmm(fos_batch* b, int k) { return reinterpret_cast<GmmBatchEntry*>(b->dev + k * b->buf_bytes); }
PbasBatchEntry* dev_pbas(fos_batch* b, int k)
{
    return reinterpret_cast<PbasBatchEntry*>(b->dev + k * b->buf_bytes + b->gmm_bytes);
}
int* dev_hdr(fos_batch* b, int k) { return reinterpret_cast<int*>(b->dev + k * b->buf_bytes + b->gmm_bytes + b->pbas_bytes); }
uint8_t* host_buf(fos_batch* b, int k) { return b->host + k * b->buf_bytes; }

bool gmm_on(const fos_batch* b) { return b->prm.methods & FOS_METHOD_GMM; }
bool pbas_on(const fos_batch* b) { return b->prm.methods & FOS_METHOD_PBAS; }
// Both methods with the 3+3 model: every tile runs GMM and PBAS in one kernel.
bool fused(const fos_batch* b) { return gmm_on(b) && pbas_on(b) && b->prm.K_rgb == 3 && b->prm.K_d == 3; }

// Shapes usable for this set of streams: vector paths need every width to be
// a multiple of the pixels per thread.
int effective_pbas_px(const fos_batch* b, int n, const int32_t* slots)
{
    for (int i = 0; i < n; ++i)
        if (b->slot[slots[i]]->W % b->pbas_px != 0) return 1;
    return b->pbas_px;
}

// Captures (or reuses) the graph of argument buffer k for the shapes in use.
fos_status ensure_graph(fos_batch* b, int k, int pbas_px)
{
    const int gpx = gmm_batch_px(b->prm.K_rgb, b->prm.K_d, b->gmm_px);
    const int key = gpx * 10000 + pbas_px * 100 + b->pbas_ty;
    if (b->graph[k] && b->graph_key[k] == key) return FOS_OK;
    if (b->graph[k]) {
        cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
    }
    int gblocks = 0, pblocks = 0;
    const bool fz = fused(b);
    if (gmm_on(b) && !fz) gblocks = b->sms * std::max(1, gmm_batch_blocks_per_sm(b->prm.K_rgb, b->prm.K_d, b->gmm_px));
    if (pbas_on(b)) pblocks = b->sms * std::max(1, pbas_batch_blocks_per_sm(b->prm.N, pbas_px, b->pbas_ty, fz));
    FOS_BTRY(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(b->dev + k * b->buf_bytes, host_buf(b, k), b->buf_bytes,
                                    cudaMemcpyHostToDevice, b->cap);
    LaunchResult r = kLaunchOk;
    if (e == cudaSuccess && gmm_on(b) && !fz)
        r = launch_gmm_batch(dev_gmm(b, k), dev_hdr(b, k), gblocks, b->prm.K_rgb, b->prm.K_d, b->gmm_px, b->cap);
    if (e == cudaSuccess && r == kLaunchOk && pbas_on(b))
        r = launch_pbas_batch(dev_pbas(b, k), fz ? dev_gmm(b, k) : nullptr, dev_hdr(b, k), pblocks, b->prm.N,
                              pbas_px, b->pbas_ty, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, "cudaMemcpyAsync (capture)", e);
    }
    if (r != kLaunchOk) {
        if (g) cudaGraphDestroy(g);
        return r == kLaunchUnsupported ? bfail(b, FOS_ERR_UNSUPPORTED, "batch: shape not compiled in")
                                       : bcuda(b, "batch launch (capture)", cudaGetLastError());
    }
    if (e2 != cudaSuccess) return bcuda(b, "cudaStreamEndCapture", e2);
    e = cudaGraphInstantiate(&b->graph[k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, "cudaGraphInstantiate", e);
    b->graph_key[k] = key;
    return FOS_OK;
}

}  // namespace

extern "C" {

size_t fos_stream_device_bytes(int32_t width, int32_t height, const fos_params* p)
{
    if (!p || width < 1 || height < 1) return 0;
    const size_t P = size_t(width) * size_t(height);
    const size_t plane = (P + 127) / 128 * 128;
    const size_t Wp = (size_t(width) + kSeg - 1) / kSeg * kSeg, pp = Wp * size_t(height);
    size_t bytes = 16 * sizeof(unsigned long long);
    if (p->methods & FOS_METHOD_GMM) bytes += size_t(5 * p->K_rgb + 3 * p->K_d) * plane * 4;
    if (p->methods & FOS_METHOD_PBAS)
        bytes += 2 * 4 * size_t(p->N) * pp * 2 + 3 * 4 * pp * 4 + 2 * pp * 4 +
                 (p->pbas_propagate ? 2 * 8 + 4 : 8) * pp;
    return bytes;
}

fos_batch* fos_batch_create(int32_t max_streams, const fos_params* params)
{
    std::string why;
    if (max_streams < 1 || max_streams > 4096) {
        bfail(nullptr, FOS_ERR_INVALID_ARG, "max_streams must be in 1..4096");
        return nullptr;
    }
    if (ctx_validate_params(params, why) != FOS_OK) {
        bfail(nullptr, FOS_ERR_INVALID_ARG, why);
        return nullptr;
    }
    if ((params->methods & FOS_METHOD_GMM) && params->gmm_literal) {
        bfail(nullptr, FOS_ERR_UNSUPPORTED, "batched launches take the FP32 GMM only (gmm_literal = 0)");
        return nullptr;
    }
    if ((params->methods & FOS_METHOD_PBAS) && params->pbas_joint) {
        bfail(nullptr, FOS_ERR_UNSUPPORTED, "batched launches take the per-channel PBAS only (pbas_joint = 0)");
        return nullptr;
    }
    fos_batch* b = new fos_batch();
    b->prm = *params;
    b->max_streams = max_streams;
    b->slot.assign(size_t(max_streams), nullptr);
    auto round = [](size_t v) { return (v + 255) / 256 * 256; };
    b->gmm_bytes = round(sizeof(GmmBatchEntry) * size_t(max_streams));
    b->pbas_bytes = round(sizeof(PbasBatchEntry) * size_t(max_streams));
    b->buf_bytes = b->gmm_bytes + b->pbas_bytes + 256;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&b->dev, 2 * b->buf_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->host, 2 * b->buf_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        bcuda(nullptr, "fos_batch_create", e);
        fos_batch_destroy(b);
        return nullptr;
    }
    std::memset(b->host, 0, 2 * b->buf_bytes);
    return b;
}

void fos_batch_destroy(fos_batch* b)
{
    if (!b) return;
    for (int k = 0; k < 2; ++k)
        if (b->done[k] && b->used[k]) cudaEventSynchronize(b->done[k]);
    for (fos_ctx* c : b->slot) fos_destroy(c);
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        if (b->done[k]) cudaEventDestroy(b->done[k]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->dev);
    cudaFreeHost(b->host);
    delete b;
}

const char* fos_batch_last_error(const fos_batch* b) { return b ? b->err.c_str() : ""; }

int32_t fos_batch_add_stream(fos_batch* b, int32_t width, int32_t height, uint32_t stream_id)
{
    if (!b) return -1;
    int free_slot = -1;
    for (int i = 0; i < b->max_streams; ++i)
        if (!b->slot[i]) { free_slot = i; break; }
    if (free_slot < 0) {
        bfail(b, FOS_ERR_BUDGET, "batch is full");
        return -1;
    }
    fos_params p = b->prm;
    p.stream_id = stream_id;
    fos_ctx* c = fos_create(width, height, &p);
    if (!c) {
        b->err = fos_last_error(nullptr);
        return -1;
    }
    b->slot[free_slot] = c;
    return free_slot;
}

fos_status fos_batch_remove_stream(fos_batch* b, int32_t slot)
{
    if (!b || slot < 0 || slot >= b->max_streams || !b->slot[slot])
        return bfail(b, FOS_ERR_INVALID_ARG, "no stream in that slot");
    // a step still in flight may use the stream's memory
    for (int k = 0; k < 2; ++k)
        if (b->used[k]) FOS_BTRY(b, cudaEventSynchronize(b->done[k]));
    fos_destroy(b->slot[slot]);
    b->slot[slot] = nullptr;
    return FOS_OK;
}

fos_ctx* fos_batch_stream(fos_batch* b, int32_t slot)
{
    if (!b || slot < 0 || slot >= b->max_streams) return nullptr;
    return b->slot[slot];
}

fos_status fos_batch_process_device(fos_batch* b, int32_t n, const int32_t* slots,
                                    const uint8_t* const* d_rgb, const uint16_t* const* d_depth,
                                    uint8_t* const* d_mask_gmm, uint8_t* const* d_mask_pbas,
                                    void* stream)
{
    NvtxRange nvtx("fos_batch_process_device");
    if (!b) return FOS_ERR_INVALID_ARG;
    if (n < 0 || n > b->max_streams) return bfail(b, FOS_ERR_INVALID_ARG, "n out of range");
    if (n == 0) return FOS_OK;
    if (!slots || !d_rgb || !d_depth || (gmm_on(b) && !d_mask_gmm) || (pbas_on(b) && !d_mask_pbas))
        return bfail(b, FOS_ERR_INVALID_ARG, "NULL array argument");
    std::vector<char> seen(size_t(b->max_streams), 0);
    for (int i = 0; i < n; ++i) {
        const int s = slots[i];
        if (s < 0 || s >= b->max_streams || !b->slot[s]) return bfail(b, FOS_ERR_INVALID_ARG, "bad slot");
        if (seen[s]) return bfail(b, FOS_ERR_INVALID_ARG, "a stream appears twice in one step");
        seen[s] = 1;
        if (!d_rgb[i] || !d_depth[i] || (gmm_on(b) && !d_mask_gmm[i]) || (pbas_on(b) && !d_mask_pbas[i]))
            return bfail(b, FOS_ERR_INVALID_ARG, "NULL frame pointer");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int k = b->tick & 1;
    if (b->used[k]) FOS_BTRY(b, cudaEventSynchronize(b->done[k]));  // host buffer k is free again
    const int px = effective_pbas_px(b, n, slots);
    fos_status st = ensure_graph(b, k, px);
    if (st != FOS_OK) return st;

    // per-stream arguments of this step
    uint8_t* hb = host_buf(b, k);
    GmmBatchEntry* ge = reinterpret_cast<GmmBatchEntry*>(hb);
    PbasBatchEntry* pe = reinterpret_cast<PbasBatchEntry*>(hb + b->gmm_bytes);
    int* hdr = reinterpret_cast<int*>(hb + b->gmm_bytes + b->pbas_bytes);
    const int gpx = gmm_batch_px(b->prm.K_rgb, b->prm.K_d, b->gmm_px);
    int gblocks = 0, ptiles = 0;
    for (int i = 0; i < n; ++i) {
        fos_ctx* c = b->slot[slots[i]];
        if (c->t == 0) FOS_BTRY(b, cudaMemsetAsync(c->aux, 0, 12 * sizeof(unsigned long long), s));
        if (gmm_on(b)) {
            ge[i].a = ctx_gmm_args(c, d_rgb[i], d_depth[i], d_mask_gmm[i]);
            ge[i].block_off = gblocks;
            gblocks += int((c->P + int64_t(kGmmBatchThreads) * gpx - 1) / (int64_t(kGmmBatchThreads) * gpx));
        }
        if (pbas_on(b)) {
            pe[i].a = ctx_pbas_args(c, d_rgb[i], d_depth[i], d_mask_pbas[i]);
            pe[i].a.mask_vec = (reinterpret_cast<uintptr_t>(d_mask_pbas[i]) % uintptr_t(px)) == 0 ? 1 : 0;
            pe[i].tile_off = ptiles;
            pe[i].tiles_x = (c->W + 32 * px - 1) / (32 * px);
            pe[i].init = c->t == 0 ? 1 : 0;
            ptiles += pe[i].tiles_x * ((c->H + b->pbas_ty - 1) / b->pbas_ty);
        }
    }
    hdr[0] = n;
    hdr[1] = ptiles;
    hdr[2] = gblocks;
    hdr[3] = 0;  // tile counter of the PBAS kernel (copied in with the arguments)
    FOS_BTRY(b, cudaGraphLaunch(b->graph[k], s));
    FOS_BTRY(b, cudaEventRecord(b->done[k], s));
    b->used[k] = true;
    b->tick += 1;
    for (int i = 0; i < n; ++i) ctx_frame_done(b->slot[slots[i]]);
    return FOS_OK;
}

fos_status fos_batch_set_shape(fos_batch* b, int32_t gmm_px, int32_t pbas_px, int32_t pbas_ty)
{
    if (!b) return FOS_ERR_INVALID_ARG;
    const bool ok = (gmm_px == 1 || gmm_px == 2) &&
                    ((pbas_px == 2 && (pbas_ty == 4 || pbas_ty == 8)) ||
                     (pbas_px == 4 && (pbas_ty == 4 || pbas_ty == 8)) || (pbas_px == 1 && pbas_ty == 8));
    if (!ok) return bfail(b, FOS_ERR_UNSUPPORTED, "batch shape not compiled in");
    b->gmm_px = gmm_px;
    b->pbas_px = pbas_px;
    b->pbas_ty = pbas_ty;
    return FOS_OK;
}

fos_status fos_batch_autotune(fos_batch* b, int32_t n, const int32_t* slots,
                              const uint8_t* const* d_rgb, const uint16_t* const* d_depth,
                              void* stream, fos_batch_tuning* out)
{
    if (!b || n < 1 || !slots || !d_rgb || !d_depth) return bfail(b, FOS_ERR_INVALID_ARG, "autotune: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // throwaway batch with the same streams, fed the given frame repeatedly
    fos_batch* t = fos_batch_create(n, &b->prm);
    if (!t) return bfail(b, FOS_ERR_CUDA, std::string("autotune: ") + fos_last_error(nullptr));
    std::vector<int32_t> ts(static_cast<size_t>(n), -1);
    std::vector<uint8_t*> mg(size_t(n), nullptr), mp(size_t(n), nullptr);
    fos_status st = FOS_OK;
    for (int i = 0; i < n && st == FOS_OK; ++i) {
        const fos_ctx* c = b->slot[slots[i]];
        if (!c) st = bfail(b, FOS_ERR_INVALID_ARG, "autotune: bad slot");
        else if ((ts[i] = fos_batch_add_stream(t, c->W, c->H, c->prm.stream_id)) < 0)
            st = bfail(b, FOS_ERR_OOM, "autotune: " + t->err);
        else if (cudaMalloc(&mg[i], size_t(c->P)) != cudaSuccess || cudaMalloc(&mp[i], size_t(c->P)) != cudaSuccess)
            st = bfail(b, FOS_ERR_OOM, "autotune: mask buffers");
    }
    struct Cand { int g, p, y; };
    const Cand cands[] = {{2, 2, 8}, {2, 2, 4}, {2, 4, 4}, {2, 4, 8}, {1, 2, 8}};
    float best = 1e30f;
    Cand pick = {b->gmm_px, b->pbas_px, b->pbas_ty};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == FOS_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = bfail(b, FOS_ERR_CUDA, "autotune: events");
    if (st == FOS_OK) st = fos_batch_process_device(t, n, ts.data(), d_rgb, d_depth, mg.data(), mp.data(), s);
    for (const Cand& c : cands) {
        if (st != FOS_OK) break;
        bool widths_ok = true;
        for (int i = 0; i < n; ++i) widths_ok &= (b->slot[slots[i]]->W % c.p) == 0;
        if (!widths_ok || fos_batch_set_shape(t, c.g, c.p, c.y) != FOS_OK) continue;
        st = fos_batch_process_device(t, n, ts.data(), d_rgb, d_depth, mg.data(), mp.data(), s);  // warm-up, capture
        if (st != FOS_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && st == FOS_OK; ++r)
            st = fos_batch_process_device(t, n, ts.data(), d_rgb, d_depth, mg.data(), mp.data(), s);
        cudaEventRecord(e1, s);
        if (st != FOS_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / 3.f < best) {
            best = ms / 3.f;
            pick = c;
        }
    }
    if (st != FOS_OK && t->err.size()) b->err = t->err;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    for (int i = 0; i < n; ++i) {
        cudaFree(mg[i]);
        cudaFree(mp[i]);
    }
    fos_batch_destroy(t);
    if (st != FOS_OK) return st;
    fos_batch_set_shape(b, pick.g, pick.p, pick.y);
    if (out) {
        out->gmm_px = pick.g;
        out->pbas_px = pick.p;
        out->pbas_ty = pick.y;
        out->ms_per_step = best;
    }
    return FOS_OK;
}

}  // extern "C"
