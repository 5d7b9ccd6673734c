// batch.cu -- many camera streams in one launch per frame step.
//
// A batch owns up to max_streams stream contexts (ordinary fos_ctx objects,
// so every single-stream call -- state export, reset, options -- works on
// them).  One frame step of up to kBatchLaunchMax streams is one replay of a
// CUDA graph holding one kernel launch (GMM and PBAS of every tile, or one
// per method when they do not run together) with one block per tile of every
// stream (the GMM-only kernel: a persistent grid over the streams' blocks).
// The per-stream arguments of the step form a table that rides in the kernel
// node's parameters, updated in the instantiated graph together with the
// grid size before each replay, so the kernels read them from the constant
// bank; larger steps take one replay per kBatchLaunchMax streams.
// Results are bit-identical to processing each stream alone: every pixel runs
// the same code on the same data.
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
    cudaEvent_t done = nullptr;  // after the last step's kernels
    bool used = false;
    // the step graph: its kernel nodes (GMM, PBAS; null where unused) and the
    // parameters they were captured with
    cudaGraph_t graph_src = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_key = -1;
    cudaGraphNode_t node[2] = {nullptr, nullptr};
    cudaKernelNodeParams kp[2] = {};
    int blocks[2] = {0, 0};
    cudaStream_t cap = nullptr;
    int gmm_px = 2, pbas_px = 2, pbas_ty = 8;  // tuned shapes
    GmmBatchTable gt{};
    PbasBatchTable pt{};
    // several frames per call (fos_batch_process_frames_device): the launch
    // table and its device scratch (claim counter, error word, scratch sums,
    // completion words, gradient sums), grown on demand
    SeqBatchTable qt{};
    uint8_t* seq = nullptr;
    size_t seq_bytes = 0;
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

#define FOS_BSTEP(call)                \
    do {                               \
        const fos_status st_ = (call); \
        if (st_ != FOS_OK) return st_; \
    } while (0)

#define FOS_BTRY(b, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(b, #call, e_); \
    } while (0)

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

void drop_graph(fos_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_src) cudaGraphDestroy(b->graph_src);
    b->graph = nullptr;
    b->graph_src = nullptr;
    b->node[0] = b->node[1] = nullptr;
    b->graph_key = -1;
}

// Captures (or reuses) the step graph for the shapes in use: one launch of
// each kernel the methods need, with the (empty) tables as parameters; the
// kernel nodes are kept so each step can write its tables into them.
fos_status ensure_graph(fos_batch* b, int pbas_px)
{
    const int gpx = gmm_batch_px(b->prm.K_rgb, b->prm.K_d, b->gmm_px);
    const int key = gpx * 10000 + pbas_px * 100 + b->pbas_ty;
    if (b->graph && b->graph_key == key) return FOS_OK;
    drop_graph(b);
    const bool fz = fused(b);
    b->blocks[0] = b->blocks[1] = 0;
    // one block per tile / per block of pixels: the grid is set at each replay
    if (gmm_on(b) && !fz) b->blocks[0] = 1;
    if (pbas_on(b)) b->blocks[1] = 1;
    b->gt.n = b->gt.total = 0;
    b->pt.n = b->pt.total = 0;
    FOS_BTRY(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    LaunchResult r = kLaunchOk;
    if (b->blocks[0])
        r = launch_gmm_batch(b->gt, b->blocks[0], b->prm.K_rgb, b->prm.K_d, b->gmm_px, b->cap);
    if (r == kLaunchOk && b->blocks[1])
        r = launch_pbas_batch(b->pt, fz, b->blocks[1], b->prm.N, pbas_px, b->pbas_ty, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (r != kLaunchOk) {
        if (g) cudaGraphDestroy(g);
        return r == kLaunchUnsupported ? bfail(b, FOS_ERR_UNSUPPORTED, "batch: shape not compiled in")
                                       : bcuda(b, "batch launch (capture)", cudaGetLastError());
    }
    if (e != cudaSuccess) return bcuda(b, "cudaStreamEndCapture", e);
    b->graph_src = g;
    // the kernel nodes in launch order (a chain: GMM first when present)
    size_t n = 0;
    FOS_BTRY(b, cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    FOS_BTRY(b, cudaGraphGetNodes(g, nodes.data(), &n));
    int k = b->blocks[0] ? 0 : 1;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        FOS_BTRY(b, cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeKernel || k > 1) continue;
        b->node[k] = nd;
        FOS_BTRY(b, cudaGraphKernelNodeGetParams(nd, &b->kp[k]));
        k = (k == 0 && b->blocks[1]) ? 1 : 2;
    }
    if ((b->blocks[0] && !b->node[0]) || (b->blocks[1] && !b->node[1])) {
        drop_graph(b);
        return bfail(b, FOS_ERR_CUDA, "batch: kernel node missing from the captured graph");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    if (e != cudaSuccess) {
        drop_graph(b);
        return bcuda(b, "cudaGraphInstantiate", e);
    }
    b->graph_key = key;
    return FOS_OK;
}

// Writes the step's tables into the graph's kernel nodes and replays it.
fos_status replay(fos_batch* b, cudaStream_t s)
{
    void* gargs[1] = {&b->gt};
    void* pargs[1] = {&b->pt};
    if (b->node[0]) {
        cudaKernelNodeParams p = b->kp[0];
        p.kernelParams = gargs;
        p.extra = nullptr;
        p.gridDim = dim3(unsigned(std::max(1, b->gt.total)));
        FOS_BTRY(b, cudaGraphExecKernelNodeSetParams(b->graph, b->node[0], &p));
    }
    if (b->node[1]) {
        cudaKernelNodeParams p = b->kp[1];
        p.kernelParams = pargs;
        p.extra = nullptr;
        p.gridDim = dim3(unsigned(std::max(1, b->pt.total)));  // one block per tile
        FOS_BTRY(b, cudaGraphExecKernelNodeSetParams(b->graph, b->node[1], &p));
    }
    FOS_BTRY(b, cudaGraphLaunch(b->graph, s));
    return FOS_OK;
}

}  // namespace

namespace fos {

int32_t batch_attach(fos_batch* b, fos_ctx* c)
{
    if (!b || !c) return -1;
    for (int i = 0; i < b->max_streams; ++i)
        if (!b->slot[i]) {
            b->slot[i] = c;
            return i;
        }
    return -1;
}

fos_ctx* batch_detach(fos_batch* b, int32_t slot)
{
    if (!b || slot < 0 || slot >= b->max_streams) return nullptr;
    fos_ctx* c = b->slot[slot];
    b->slot[slot] = nullptr;
    return c;
}

}  // namespace fos

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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        bcuda(nullptr, "fos_batch_create", e);
        fos_batch_destroy(b);
        return nullptr;
    }
    return b;
}

void fos_batch_destroy(fos_batch* b)
{
    if (!b) return;
    if (b->done && b->used) cudaEventSynchronize(b->done);
    for (fos_ctx* c : b->slot) fos_destroy(c);
    drop_graph(b);
    cudaFree(b->seq);
    if (b->done) cudaEventDestroy(b->done);
    if (b->cap) cudaStreamDestroy(b->cap);
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
    if (b->used) FOS_BTRY(b, cudaEventSynchronize(b->done));
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
    const int px = effective_pbas_px(b, n, slots);
    fos_status st = ensure_graph(b, px);
    if (st != FOS_OK) return st;

    // per-stream arguments of this step, kBatchLaunchMax streams per replay
    const int gpx = gmm_batch_px(b->prm.K_rgb, b->prm.K_d, b->gmm_px);
    const bool fz = fused(b);
    for (int i0 = 0; i0 < n; i0 += kBatchLaunchMax) {
        const int m = std::min(n - i0, kBatchLaunchMax);
        int gblocks = 0, ptiles = 0;
        for (int j = 0; j < m; ++j) {
            const int i = i0 + j;
            fos_ctx* c = b->slot[slots[i]];
            if (c->t == 0) FOS_BTRY(b, cudaMemsetAsync(c->aux, 0, 12 * sizeof(unsigned long long), s));
            if (gmm_on(b)) {
                const GmmArgs ga = ctx_gmm_args(c, d_rgb[i], d_depth[i], d_mask_gmm[i]);
                if (fz) {
                    b->pt.g[j] = ga;
                } else {
                    b->gt.e[j].a = ga;
                    b->gt.e[j].block_off = gblocks;
                    gblocks += int((c->P + int64_t(kGmmBatchThreads) * gpx - 1) / (int64_t(kGmmBatchThreads) * gpx));
                }
            }
            if (pbas_on(b)) {
                PbasBatchEntry& e = b->pt.e[j];
                e.a = ctx_pbas_args(c, d_rgb[i], d_depth[i], d_mask_pbas[i]);
                e.a.mask_vec = (reinterpret_cast<uintptr_t>(d_mask_pbas[i]) % uintptr_t(px)) == 0 ? 1 : 0;
                e.tile_off = ptiles;
                e.tiles_x = (c->W + 32 * px - 1) / (32 * px);
                e.init = c->t == 0 ? 1 : 0;
                ptiles += e.tiles_x * ((c->H + b->pbas_ty - 1) / b->pbas_ty);
            }
        }
        b->gt.n = gmm_on(b) && !fz ? m : 0;
        b->gt.total = gblocks;
        b->pt.n = pbas_on(b) ? m : 0;
        b->pt.total = ptiles;
        st = replay(b, s);
        if (st != FOS_OK) return st;
    }
    FOS_BTRY(b, cudaEventRecord(b->done, s));
    b->used = true;
    for (int i = 0; i < n; ++i) ctx_frame_done(b->slot[slots[i]]);
    return FOS_OK;
}

fos_status fos_batch_process_frames_device(fos_batch* b, int32_t n, const int32_t* slots, const int32_t* n_frames,
                                           const uint8_t* const* d_rgb, const uint16_t* const* d_depth,
                                           uint8_t* const* d_mask_gmm, uint8_t* const* d_mask_pbas, void* stream)
{
    NvtxRange nvtx("fos_batch_process_frames_device");
    if (!b) return FOS_ERR_INVALID_ARG;
    if (n < 0 || n > b->max_streams) return bfail(b, FOS_ERR_INVALID_ARG, "n out of range");
    if (n == 0) return FOS_OK;
    if (!slots || !n_frames || !d_rgb || !d_depth || (gmm_on(b) && !d_mask_gmm) || (pbas_on(b) && !d_mask_pbas))
        return bfail(b, FOS_ERR_INVALID_ARG, "NULL array argument");
    int maxf = 0;
    for (int i = 0; i < n; ++i) {
        if (n_frames[i] < 0) return bfail(b, FOS_ERR_INVALID_ARG, "negative frame count");
        maxf = std::max(maxf, int(n_frames[i]));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> sl;
    std::vector<const uint8_t*> r;
    std::vector<const uint16_t*> d;
    std::vector<uint8_t*> g, p;
    // frame k of stream i (k < n_frames[i])
    auto frame_of = [&](int i, int k) {
        const fos_ctx* c = b->slot[slots[i]];
        r.push_back(d_rgb[i] + size_t(k) * size_t(c->P) * 3);
        d.push_back(d_depth[i] + size_t(k) * size_t(c->Pd));
        g.push_back(gmm_on(b) ? d_mask_gmm[i] + size_t(k) * size_t(c->P) : nullptr);
        p.push_back(pbas_on(b) ? d_mask_pbas[i] + size_t(k) * size_t(c->P) : nullptr);
    };
    auto step = [&]() -> fos_status {
        const fos_status st = sl.empty() ? FOS_OK
                                         : fos_batch_process_device(b, int32_t(sl.size()), sl.data(), r.data(), d.data(),
                                                                    gmm_on(b) ? g.data() : nullptr,
                                                                    pbas_on(b) ? p.data() : nullptr, stream);
        sl.clear(); r.clear(); d.clear(); g.clear(); p.clear();
        return st;
    };
    for (int i = 0; i < n; ++i)  // validates slots and pointers (and runs nothing)
        if (slots[i] < 0 || slots[i] >= b->max_streams || !b->slot[slots[i]])
            return bfail(b, FOS_ERR_INVALID_ARG, "bad slot");
    if (!fused(b)) {  // one batched step per frame slot
        for (int k = 0; k < maxf; ++k) {
            for (int i = 0; i < n; ++i)
                if (n_frames[i] > k) {
                    sl.push_back(slots[i]);
                    frame_of(i, k);
                }
            FOS_BSTEP(step());
        }
        return FOS_OK;
    }
    // frame 0 of streams that start here: one batched step
    std::vector<int> first(size_t(n), 0);
    for (int i = 0; i < n; ++i)
        if (n_frames[i] > 0 && b->slot[slots[i]]->t == 0) {
            sl.push_back(slots[i]);
            frame_of(i, 0);
            first[i] = 1;
        }
    FOS_BSTEP(step());
    // the rest: entries sorted by remaining frames (descending), in launches of
    // at most kSeqBatchMax streams
    std::vector<int> order;
    for (int i = 0; i < n; ++i)
        if (n_frames[i] - first[i] > 0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return n_frames[x] - first[x] > n_frames[y] - first[y]; });
    int px = b->pbas_px == 2 ? 2 : 1;
    for (int i : order)
        if (b->slot[slots[i]]->W % 2 != 0) px = 1;
    const int ty = px == 2 && b->pbas_ty == 4 ? 4 : 8;
    for (size_t c0 = 0; c0 < order.size(); c0 += kSeqBatchMax) {
        const int m = int(std::min(order.size() - c0, size_t(kSeqBatchMax)));
        SeqBatchTable& T = b->qt;
        T.n = m;
        // scratch: header, completion words, gradient sums
        size_t words = 0, sums = 0;
        for (int j = 0; j < m; ++j) {
            const fos_ctx* c = b->slot[slots[order[c0 + j]]];
            const int tx = (c->W + 32 * px - 1) / (32 * px), tyy = (c->H + ty - 1) / ty;
            words += size_t(tx) * tyy;
            sums += size_t(n_frames[order[c0 + j]] - first[order[c0 + j]] + 1) * 4;
        }
        const size_t need = 256 + sums * 8 + words * 4;
        if (need > b->seq_bytes) {
            FOS_BTRY(b, cudaDeviceSynchronize());  // an earlier launch may still use the old scratch
            cudaFree(b->seq);
            b->seq = nullptr;
            b->seq_bytes = 0;
            FOS_BTRY(b, dev_alloc(reinterpret_cast<void**>(&b->seq), need));
            b->seq_bytes = need;
        }
        T.claim = reinterpret_cast<unsigned int*>(b->seq);
        T.err = reinterpret_cast<int*>(b->seq + 4);
        T.gscratch = reinterpret_cast<unsigned long long*>(b->seq + 64);
        unsigned long long* gs = reinterpret_cast<unsigned long long*>(b->seq + 256);
        int* dn = reinterpret_cast<int*>(b->seq + 256 + sums * 8);
        T.done_all = dn;
        T.done_words = int(words);
        int tile_off = 0, gtile_off = 0;
        for (int j = 0; j < m; ++j) {
            const int i = order[c0 + j];
            fos_ctx* c = b->slot[slots[i]];
            const int nf = n_frames[i] - first[i], f0 = first[i];
            SeqBatchEntry& E = T.e[j];
            const uint8_t* rgb = d_rgb[i] + size_t(f0) * size_t(c->P) * 3;
            const uint16_t* dep = d_depth[i] + size_t(f0) * size_t(c->Pd);
            uint8_t* mg = d_mask_gmm[i] + size_t(f0) * size_t(c->P);
            uint8_t* mp = d_mask_pbas[i] + size_t(f0) * size_t(c->P);
            E.a = ctx_pbas_args(c, rgb, dep, mp);
            T.g[j] = ctx_gmm_args(c, rgb, dep, mg);
            E.n = nf;
            E.tiles_x = (c->W + 32 * px - 1) / (32 * px);
            E.tiles_y = (c->H + ty - 1) / ty;
            E.tile_off = tile_off;
            E.gtile_off = gtile_off;
            tile_off += E.tiles_x * E.tiles_y;
            gtile_off += ((c->W + 31) / 32) * ((c->H + kGradStripRows - 1) / kGradStripRows);
            E.rgb_stride = c->P * 3;
            E.depth_stride = c->Pd;
            E.mask_stride = c->P;
            E.req_base = c->req;
            E.prev_base = c->prev;
            E.gprev = gs;
            gs += 4 * size_t(nf + 1);
            E.gsum_src = E.a.gsum_prev;
            E.gsum_last = c->aux + ((c->t + nf - 1) % 3) * 4;
            E.gsum_zero = c->aux + ((c->t + nf) % 3) * 4;
            E.done = dn;
            dn += size_t(E.tiles_x) * E.tiles_y;
        }
        T.gtiles = gtile_off;
        T.maxn = T.e[0].n;
        if (T.maxn > 65535) return bfail(b, FOS_ERR_INVALID_ARG, "at most 65535 frames per stream and call");
        // runs of frame slots with the same active entries (a prefix of the order)
        T.segs = 0;
        long long claims = 0;
        int slot0 = 0;
        for (int mm = m; mm > 0; --mm) {
            const int slot1 = T.e[mm - 1].n;  // entries 0 .. mm-1 have at least slot1 frames
            if (slot1 <= slot0) continue;
            const int tiles = T.e[mm - 1].tile_off + T.e[mm - 1].tiles_x * T.e[mm - 1].tiles_y;
            T.seg_slot0[T.segs] = slot0;
            T.seg_m[T.segs] = mm;
            T.seg_tiles[T.segs] = tiles;
            T.seg_claim0[T.segs] = claims;
            claims += static_cast<long long>(slot1 - slot0) * tiles;
            slot0 = slot1;
            T.segs += 1;
        }
        T.seg_slot0[T.segs] = slot0;
        T.seg_claim0[T.segs] = claims;
        if (claims >= (1ll << 32)) return bfail(b, FOS_ERR_INVALID_ARG, "too many tiles x frames in one call");
        const LaunchResult lr = launch_batch_sequence(T, px, ty, s);
        if (lr == kLaunchUnsupported) return bfail(b, FOS_ERR_UNSUPPORTED, "batch sequence: shape not compiled in");
        if (lr != kLaunchOk) return bcuda(b, "batch sequence launch", cudaGetLastError());
        for (int j = 0; j < m; ++j) {
            fos_ctx* c = b->slot[slots[order[c0 + j]]];
            for (int k = 0; k < T.e[j].n; ++k) ctx_frame_done(c);
        }
    }
    FOS_BTRY(b, cudaEventRecord(b->done, s));
    b->used = true;
    return FOS_OK;
}

fos_status fos_batch_sequence_status(fos_batch* b)
{
    if (!b) return FOS_ERR_INVALID_ARG;
    if (!b->seq) return FOS_OK;
    FOS_BTRY(b, cudaDeviceSynchronize());
    int e = 0;
    FOS_BTRY(b, cudaMemcpy(&e, b->seq + 4, 4, cudaMemcpyDeviceToHost));
    if (e) return bfail(b, FOS_ERR_TIMEOUT, "batch sequence: a tile's wait for its neighbours gave up");
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
