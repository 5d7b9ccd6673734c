// api.cu -- the C ABI (include/fos.h): contexts, device state, frame loop,
// state export/import, timing and counters.
//
// The paper's heterogeneous frame loop (Sec. 4.2): the host allocates the
// background model, copies each frame to the GPU, the GPU classifies and
// updates every pixel in parallel, and the mask is copied back.  Here the
// context owns the device-resident model (SoA planes, padded to 128 elements
// so every plane starts 256-byte aligned); frames come either from device
// memory (asynchronous, caller's stream) or from host memory (synchronous,
// with the next frame's copy overlapping the current frame's kernels).
#include <cstdio>
#include <cstring>
#include <atomic>
#include <cstdlib>
#include <string>
#include <vector>

#include "ctx.h"
#include "fos.h"
#include "fos_internal.h"
#include "philox.cuh"

using namespace fos;

void fos::pbas_args_finish(PbasArgs& a)
{
    philox_round_keys(a.seed, a.stream_id, a.rk);
    depth_divisor(a.depth_fs, a.depth_m, a.depth_sh);
}

namespace {

thread_local std::string g_create_error;
thread_local fos_status g_create_status = FOS_OK;

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

constexpr int kAuxWords = 32;  // aux: gsum[3][4], counters[3], GMM error word 15, OobWord at word 16

// The context's violation record in range-checked builds (none otherwise).
fos::OobWord* oob_of(fos_ctx* c)
{
#ifdef FOS_DEBUG_BOUNDS
    return reinterpret_cast<fos::OobWord*>(c->aux + 16);
#else
    (void)c;
    return nullptr;
#endif
}

}  // namespace


namespace {

fos_status fail(fos_ctx* c, fos_status st, const std::string& msg)
{
    if (c) {
        c->err = msg;
        c->last_status = st;
    } else {
        g_create_error = msg;
        g_create_status = st;
    }
    return st;
}

fos_status cuda_fail(fos_ctx* c, const char* what, cudaError_t e)
{
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return fail(c, e == cudaErrorMemoryAllocation ? FOS_ERR_OOM : FOS_ERR_CUDA, buf);
}

#define FOS_TRY(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, #call, e_); \
    } while (0)

#define FOS_TRY_ST(call)                      \
    do {                                      \
        const fos_status st_ = (call);        \
        if (st_ != FOS_OK) return st_;        \
    } while (0)

bool gmm_on(const fos_ctx* c) { return c->prm.methods & FOS_METHOD_GMM; }
bool pbas_on(const fos_ctx* c) { return c->prm.methods & FOS_METHOD_PBAS; }

bool k_supported(int Kr, int Kd)
{
    const bool r = Kr == 1 || Kr == 2 || Kr == 3 || Kr == 5 || Kr == 7;
    const bool d = Kd >= 1 && Kd <= 3;
    return r && d;
}

fos_status validate_params(const fos_params* p, std::string& why)
{
    if (!p) { why = "params is NULL"; return FOS_ERR_INVALID_ARG; }
    if (p->methods == 0 || (p->methods & ~(FOS_METHOD_GMM | FOS_METHOD_PBAS))) {
        why = "methods must be a non-empty subset of GMM|PBAS"; return FOS_ERR_INVALID_ARG;
    }
    if (p->gmm_literal != 0 && p->gmm_literal != 1) {
        why = "gmm_literal must be 0 or 1"; return FOS_ERR_INVALID_ARG;
    }
    if ((p->methods & FOS_METHOD_GMM) && p->gmm_literal) {
        if (!gmm_literal_supported(p->K_rgb, p->K_d)) {
            why = "the literal GMM takes (K_rgb, K_d) = (7, 3) or (3, 3)"; return FOS_ERR_UNSUPPORTED;
        }
        if (!(p->density_scale > 0.f) || !(p->density_threshold > 0.f)) {
            why = "density_scale and density_threshold must be > 0"; return FOS_ERR_INVALID_ARG;
        }
    }
    if (p->methods & FOS_METHOD_GMM) {
        if (!p->gmm_literal && !k_supported(p->K_rgb, p->K_d)) {
            why = "unsupported (K_rgb, K_d); K_rgb in {1,2,3,5,7}, K_d in {1,2,3}";
            return FOS_ERR_UNSUPPORTED;
        }
        if (!(p->alpha > 0.f && p->alpha <= 1.f) || !(p->lambda > 0.f) || !(p->T_bg > 0.f) ||
            !(p->w_depth >= 0.f && p->w_depth <= 1.f) || !(p->v_init_rgb > 0.f) ||
            !(p->v_init_d > 0.f) || !(p->v_min_rgb > 0.f) || !(p->v_min_d > 0.f)) {
            why = "GMM parameter out of range"; return FOS_ERR_INVALID_ARG;
        }
    }
    if (p->methods & FOS_METHOD_PBAS) {
        // a neighbour request is one byte per channel: 1 + j*N + k2 <= 8N <= 255
        if (p->N < 1 || p->N > 31 || p->n_min < 1 || p->n_min > p->N) {
            why = "PBAS needs 1 <= n_min <= N <= 31"; return FOS_ERR_INVALID_ARG;
        }
        if ((p->pbas_propagate != 0 && p->pbas_propagate != 1) || (p->pbas_joint != 0 && p->pbas_joint != 1) ||
            p->forced_rng < 0 || p->forced_rng > 3) {
            why = "pbas_propagate and pbas_joint must be 0 or 1, forced_rng 0..3"; return FOS_ERR_INVALID_ARG;
        }
        if (!(p->T_lower > 0.f) || !(p->T_upper >= p->T_lower) || !(p->eps_d > 0.f) ||
            !(p->R_lower_rgb > 0.f) || !(p->R_lower_d > 0.f) || !(p->R_incdec >= 0.f && p->R_incdec < 1.f)) {
            why = "PBAS parameter out of range"; return FOS_ERR_INVALID_ARG;
        }
    }
    if (p->depth_full_scale_mm == 0 || p->depth_full_scale_mm > 65535u * 4u) {
        why = "depth_full_scale_mm out of range"; return FOS_ERR_INVALID_ARG;
    }
    return FOS_OK;
}

cudaEvent_t pool_event(fos_ctx* c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// Records events around one launch when its kind is being timed.
struct TimedScope {
    fos_ctx* c;
    cudaStream_t s;
    TimedLaunch tl{};
    bool on;
    TimedScope(fos_ctx* c_, int kind, cudaStream_t s_, int64_t frames = 1) : c(c_), s(s_), on(false)
    {
        if (c->timing_mask & (1u << kind)) {
            tl.kind = kind;
            tl.frames = frames;
            tl.start = pool_event(c);
            tl.stop = pool_event(c);
            if (tl.start && tl.stop) {
                cudaEventRecord(tl.start, s);
                on = true;
            }
        }
    }
    ~TimedScope()
    {
        if (on) {
            cudaEventRecord(tl.stop, s);
            c->timed.push_back(tl);
        }
    }
};

fos_status launch_result(fos_ctx* c, LaunchResult r, const char* what)
{
    if (r == kLaunchOk) return FOS_OK;
    if (r == kLaunchUnsupported) return fail(c, FOS_ERR_UNSUPPORTED, std::string(what) + ": unsupported configuration");
    return cuda_fail(c, what, cudaGetLastError());
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

PbasArgs pbas_args(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mask)
{
    PbasArgs a{};
    const fos_params& p = c->prm;
    a.W = c->W; a.H = c->H; a.P = c->P;
    a.Wd = c->Wd; a.Hd = c->Hd;
    a.Wp = c->Wp; a.spr = c->spr; a.nseg = c->nseg; a.plane = c->pplane;
    a.rgb = rgb; a.depth = depth; a.mask = mask;
    a.samp = c->samp; a.Dq = c->Dq; a.R = c->R; a.T = c->T; a.S = c->S;
    const int64_t t = c->t;
    a.propagate = p.pbas_propagate;
    if (p.pbas_propagate) {  // planes by frame parity: write frame t, read frame t-1
        a.prev = c->prev + (t & 1) * c->pplane;
        a.prev_src = c->prev + ((t + 1) & 1) * c->pplane;
        a.own = reinterpret_cast<uint32_t*>(c->prev + 2 * c->pplane);
    } else {
        a.prev = c->prev;
        a.prev_src = c->prev;
    }
    a.req_cur = c->req + (t & 1) * c->pplane;
    a.req_prev = c->req + ((t + 1) & 1) * c->pplane;      // buffer of frame t-1
    a.gsum_prev = c->aux + ((t + 2) % 3) * 4;             // frame t-1
    a.gsum_cur = c->aux + (t % 3) * 4;
    a.gsum_next = c->aux + ((t + 1) % 3) * 4;
    a.counters = c->aux + 12;
    a.apply = c->pending ? 1 : 0;
    a.R_lower_rgb = p.R_lower_rgb; a.R_lower_d = p.R_lower_d; a.R_scale = p.R_scale;
    a.R_incdec = p.R_incdec; a.T_lower = p.T_lower; a.T_upper = p.T_upper;
    a.T_inc = p.T_inc; a.T_dec = p.T_dec; a.alpha_g = p.alpha_g; a.eps_d = p.eps_d;
    a.N = p.N; a.n_min = p.n_min; a.seed = p.seed; a.stream_id = p.stream_id;
    a.forced = p.forced_rng; a.depth_fs = p.depth_full_scale_mm;
    a.t = uint32_t(c->t);
    a.px = c->opt[FOS_OPT_PBAS_PX];
    a.ty = c->opt[FOS_OPT_PBAS_TY];
    a.mask_vec = aligned(mask, uintptr_t(a.px)) ? 1 : 0;
    a.oob = oob_of(c);
    pbas_args_finish(a);
    return a;
}

GmmArgs gmm_args(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mg)
{
    GmmArgs a{};
    const fos_params& p = c->prm;
    a.P = c->P; a.plane = c->plane; a.state = c->gmm;
    a.rgb = rgb; a.depth = depth; a.mask = mg;
    a.alpha = p.alpha; a.lam2 = p.lambda * p.lambda; a.w_depth = p.w_depth; a.T_bg = p.T_bg;
    a.v_init_rgb = p.v_init_rgb; a.v_init_d = p.v_init_d;
    a.v_min_rgb = p.v_min_rgb; a.v_min_d = p.v_min_d;
    a.depth_fs = p.depth_full_scale_mm;
    a.init = c->t == 0 ? 1 : 0;
    a.W = c->W; a.H = c->H; a.Wd = c->Wd; a.Hd = c->Hd;
    // the vector path reads depth as it lies in memory: equal sizes only
    a.vec_ok = aligned(rgb, 4) && aligned(depth, 8) && aligned(mg, 4) && c->Wd == c->W && c->Hd == c->H;
    a.px = c->opt[FOS_OPT_GMM_PX];
    a.tpb = c->opt[FOS_OPT_GMM_TPB];
    a.oob = oob_of(c);
    a.stream = c->opt[FOS_OPT_GMM_STREAM];
    a.err = reinterpret_cast<int*>(c->aux + 15);
    return a;
}

// GMM and PBAS of a frame in one launch: both methods, the 3+3 model, option on.
bool ctx_fused(const fos_ctx* c)
{
    return gmm_on(c) && pbas_on(c) && !c->prm.gmm_literal && !c->prm.pbas_joint && c->prm.K_rgb == 3 &&
           c->prm.K_d == 3 && c->opt[FOS_OPT_FUSE] != 0;
}

fos_status process_device(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mg,
                          uint8_t* mp, cudaStream_t s)
{
    if (!rgb || !depth) return fail(c, FOS_ERR_INVALID_ARG, "rgb and depth must be non-NULL");
    if (gmm_on(c) && !mg) return fail(c, FOS_ERR_INVALID_ARG, "GMM enabled: mask_gmm must be non-NULL");
    if (pbas_on(c) && !mp) return fail(c, FOS_ERR_INVALID_ARG, "PBAS enabled: mask_pbas must be non-NULL");
    const bool first = c->t == 0;
    if (first) FOS_TRY(c, cudaMemsetAsync(c->aux, 0, 12 * sizeof(unsigned long long), s));
    if (!first && ctx_fused(c)) {
        const GmmArgs g = gmm_args(c, rgb, depth, mg);
        const PbasArgs a = pbas_args(c, rgb, depth, mp);
        TimedScope ts(c, FOS_KERNEL_FUSED, s);
        fos_status st = launch_result(c, launch_fused_classify(a, g, s), "fused_classify");
        if (st != FOS_OK) return st;
        c->pending = true;
        c->t += 1;
        c->frames_since_counters += 1;
        return FOS_OK;
    }
    if (gmm_on(c)) {
        const fos_params& p = c->prm;
        TimedScope ts(c, first ? FOS_KERNEL_INIT : FOS_KERNEL_GMM, s);
        fos_status st;
        if (p.gmm_literal) {
            GmmLiteralArgs a{};
            a.P = c->P; a.plane = c->plane; a.state = reinterpret_cast<double*>(c->gmm);
            a.rgb = rgb; a.depth = depth; a.mask = mg;
            a.alpha = p.alpha; a.lam2 = double(p.lambda) * double(p.lambda); a.T_bg = p.T_bg;
            a.v_init_rgb = p.v_init_rgb; a.v_init_d = p.v_init_d; a.v_min_rgb = p.v_min_rgb; a.v_min_d = p.v_min_d;
            a.s = p.density_scale; a.theta = p.density_threshold;
            a.depth_fs = p.depth_full_scale_mm; a.init = first ? 1 : 0;
            a.W = c->W; a.H = c->H; a.Wd = c->Wd; a.Hd = c->Hd;
            st = launch_result(c, launch_gmm_literal(a, p.K_rgb, p.K_d, s), "gmm_literal");
        } else {
            const GmmArgs a = gmm_args(c, rgb, depth, mg);
            st = launch_result(c, launch_gmm(a, p.K_rgb, p.K_d, s), "gmm");
        }
        if (st != FOS_OK) return st;
    }
    if (pbas_on(c)) {
        const PbasArgs a = pbas_args(c, rgb, depth, mp);
        if (first) {
            TimedScope ts(c, FOS_KERNEL_INIT, s);
            fos_status st = launch_result(c, launch_pbas_init(a, s), "pbas_init");
            if (st != FOS_OK) return st;
            c->pending = false;
        } else {
            TimedScope ts(c, FOS_KERNEL_PBAS_CLASSIFY, s);
            fos_status st = c->prm.pbas_joint ? launch_result(c, launch_pbas_joint(a, s), "pbas_joint")
                                              : launch_result(c, launch_pbas_classify(a, s), "pbas_classify");
            if (st != FOS_OK) return st;
            c->pending = true;
        }
    }
    c->t += 1;
    c->frames_since_counters += 1;
    return FOS_OK;
}

// --- several frames in one persistent launch ---------------------------------

constexpr size_t kSeqHeader = 256;  // tile counter, error word; scratch sums at byte 64

bool seq_on(const fos_ctx* c) { return ctx_fused(c) && c->opt[FOS_OPT_SEQUENCE] != 0; }

// Buffers of the sequence launch for n frames and `tiles` tiles (grown on
// demand; an earlier launch using them has been ordered before on the stream
// or synchronised).
fos_status ensure_seq(fos_ctx* c, int n, int tiles)
{
    if (c->seq && c->seq_frames >= n && c->seq_tiles >= tiles) return FOS_OK;
    const int nf = std::max(n, c->seq_frames), nt = std::max(tiles, c->seq_tiles);
    FOS_TRY(c, cudaDeviceSynchronize());  // an earlier launch may still use the old buffers
    cudaFree(c->seq);
    c->seq = nullptr;
    c->seq_frames = c->seq_tiles = 0;
    const size_t bytes = kSeqHeader + size_t(nf + 1) * 32 + size_t(nt) * 4;
    FOS_TRY(c, dev_alloc(reinterpret_cast<void**>(&c->seq), bytes));
    FOS_TRY(c, cudaMemset(c->seq, 0, kSeqHeader));
    c->seq_frames = nf;
    c->seq_tiles = nt;
    return FOS_OK;
}

// Frames t .. t+n-1 (t >= 1) of a fused context in one persistent launch:
// frame f's inputs at rgb + f*rgb_stride bytes and depth + f*depth_stride
// elements, its masks at f*mask_stride bytes.  Same bits as n process_device calls.
fos_status process_device_seq(fos_ctx* c, int32_t n, const uint8_t* rgb, size_t rgb_stride,
                              const uint16_t* depth, size_t depth_stride, uint8_t* mg, uint8_t* mp,
                              size_t mask_stride, cudaStream_t s)
{
    const PbasArgs a = pbas_args(c, rgb, depth, mp);
    const GmmArgs g = gmm_args(c, rgb, depth, mg);
    int tx = 0, ty = 0;
    fused_sequence_tiles(a, tx, ty);
    FOS_TRY_ST(ensure_seq(c, n, tx * ty));
    SeqArgs q{};
    q.n = n;
    q.tiles_x = tx;
    q.tiles_y = ty;
    q.rgb_stride = int64_t(rgb_stride);
    q.depth_stride = int64_t(depth_stride);
    q.mask_stride = int64_t(mask_stride);
    q.req_base = c->req;
    q.prev_base = c->prev;
    q.claim = reinterpret_cast<unsigned int*>(c->seq);
    q.err = reinterpret_cast<int*>(c->seq + 4);
    q.gscratch = reinterpret_cast<unsigned long long*>(c->seq + 64);
    unsigned long long* gprev = reinterpret_cast<unsigned long long*>(c->seq + kSeqHeader);
    q.gprev = gprev;
    q.done = reinterpret_cast<int*>(c->seq + kSeqHeader + size_t(c->seq_frames + 1) * 32);
    const int64_t t0 = c->t;
    unsigned long long* last = c->aux + ((t0 + n - 1) % 3) * 4;   // read by frame t0+n
    unsigned long long* next = c->aux + ((t0 + n) % 3) * 4;       // accumulated by frame t0+n
    {
        TimedScope ts(c, FOS_KERNEL_FUSED_SEQUENCE, s, n);
        // gprev[0]: sums of frame t0-1 (from the last launch); gprev[1 + f]:
        // sums of frame t0+f, f = 0 .. n-1, by the pre-pass
        FOS_TRY(c, cudaMemsetAsync(c->seq, 0, 8, s));  // tile counter, error word
        FOS_TRY(c, cudaMemsetAsync(q.done, 0, size_t(tx) * ty * 4, s));
        FOS_TRY(c, cudaMemcpyAsync(gprev, a.gsum_prev, 32, cudaMemcpyDeviceToDevice, s));
        FOS_TRY(c, cudaMemsetAsync(gprev + 4, 0, size_t(n) * 32, s));
        fos_status st = launch_result(c, launch_grad_sums(a, q, gprev + 4, s), "grad_sums");
        if (st != FOS_OK) return st;
        st = launch_result(c, launch_fused_sequence(a, g, q, s), "fused_sequence");
        if (st != FOS_OK) return st;
    }
    // where a per-frame launch of frame t0+n expects the gradient sums
    FOS_TRY(c, cudaMemcpyAsync(last, gprev + 4 * size_t(n), 32, cudaMemcpyDeviceToDevice, s));
    FOS_TRY(c, cudaMemsetAsync(next, 0, 32, s));
    c->pending = true;
    c->t += n;
    c->frames_since_counters += uint64_t(n);
    return FOS_OK;
}

// n frames through the per-frame path, or (fused, option on, n >= 2) the
// first through it when the context is at frame 0 and the rest in one
// sequence launch.
fos_status process_device_frames(fos_ctx* c, int32_t n, const uint8_t* rgb, size_t rgb_stride,
                                 const uint16_t* depth, size_t depth_stride, uint8_t* mg, uint8_t* mp,
                                 size_t mask_stride, cudaStream_t s)
{
    int32_t f = 0;
    if (seq_on(c) && n >= 2) {
        if (!rgb || !depth || !mg || !mp)
            return fail(c, FOS_ERR_INVALID_ARG, "rgb, depth and both masks must be non-NULL");
        if (c->t == 0) {
            FOS_TRY_ST(process_device(c, rgb, depth, mg, mp, s));
            f = 1;
        }
        if (n - f >= 2)
            return process_device_seq(c, n - f, rgb + size_t(f) * rgb_stride, rgb_stride,
                                      depth + size_t(f) * depth_stride, depth_stride, mg + size_t(f) * mask_stride,
                                      mp + size_t(f) * mask_stride, mask_stride, s);
    }
    for (; f < n; ++f) {
        FOS_TRY_ST(process_device(c, rgb + size_t(f) * rgb_stride, depth + size_t(f) * depth_stride,
                                  mg ? mg + size_t(f) * mask_stride : nullptr,
                                  mp ? mp + size_t(f) * mask_stride : nullptr, s));
    }
    return FOS_OK;
}

// Error word of the last sequence launch (after a synchronisation).
fos_status seq_check(fos_ctx* c)
{
    int e = 0;
    FOS_TRY(c, cudaMemcpy(&e, c->aux + 15, 4, cudaMemcpyDeviceToHost));
    if (e) {
        FOS_TRY(c, cudaMemset(c->aux + 15, 0, 4));
        return fail(c, FOS_ERR_TIMEOUT, "gmm: a bulk copy's wait gave up");
    }
    if (!c->seq) return FOS_OK;
    FOS_TRY(c, cudaMemcpy(&e, c->seq + 4, 4, cudaMemcpyDeviceToHost));
    if (e) {
        FOS_TRY(c, cudaMemset(c->seq + 4, 0, 4));
        return fail(c, FOS_ERR_TIMEOUT, "fused_sequence: a tile's wait for its neighbours gave up");
    }
    return FOS_OK;
}

// Staging for `frames` host frames per slot (grown on demand; callers of the
// host-pointer API have synchronised every earlier use before this runs).
constexpr int kHostChunk = 16;  // host frames per staging slot (8: 1.6 % slower end to end, 64: 2 %)

fos_status ensure_staging(fos_ctx* c, int frames)
{
    if (!c->ev_in[0]) {
        for (int b = 0; b < 2; ++b) {
            FOS_TRY(c, cudaEventCreateWithFlags(&c->ev_in[b], cudaEventDisableTiming));
            FOS_TRY(c, cudaEventCreateWithFlags(&c->ev_k[b], cudaEventDisableTiming));
            FOS_TRY(c, cudaEventCreateWithFlags(&c->ev_done[b], cudaEventDisableTiming));
        }
    }
    if (c->stage_frames >= frames) return FOS_OK;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    c->stage_rgb = up(size_t(c->P) * 3);
    c->stage_depth = up(size_t(c->Pd) * 2);
    c->stage_mask = up(size_t(c->P));
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->h_rgb[b]); cudaFree(c->h_depth[b]); cudaFree(c->h_mg[b]); cudaFree(c->h_mp[b]);
        c->h_rgb[b] = nullptr; c->h_depth[b] = nullptr; c->h_mg[b] = nullptr; c->h_mp[b] = nullptr;
    }
    c->stage_frames = 0;
    const size_t f = size_t(frames);
    for (int b = 0; b < 2; ++b) {
        FOS_TRY(c, dev_alloc(reinterpret_cast<void**>(&c->h_rgb[b]), f * c->stage_rgb));
        FOS_TRY(c, dev_alloc(reinterpret_cast<void**>(&c->h_depth[b]), f * c->stage_depth));
        FOS_TRY(c, dev_alloc(reinterpret_cast<void**>(&c->h_mg[b]), f * c->stage_mask));
        FOS_TRY(c, dev_alloc(reinterpret_cast<void**>(&c->h_mp[b]), f * c->stage_mask));
    }
    c->stage_frames = frames;
    return FOS_OK;
}

// GMM state planes and bytes per element: FP32 isotropic, or the FP64
// literal model with per-channel variances.
size_t gmm_nplanes(const fos_ctx* c)
{
    return size_t(c->prm.gmm_literal ? gmm_literal_planes(c->prm.K_rgb, c->prm.K_d)
                                     : gmm_planes(c->prm.K_rgb, c->prm.K_d));
}
size_t gmm_elem(const fos_ctx* c) { return c->prm.gmm_literal ? 8 : 4; }

size_t gmm_bytes(const fos_ctx* c)
{
    return gmm_on(c) ? gmm_nplanes(c) * size_t(c->P) * gmm_elem(c) : 0;
}

size_t pbas_bytes(const fos_ctx* c)
{
    if (!pbas_on(c)) return 0;
    const size_t P = size_t(c->P), N = size_t(c->prm.N);
    return 4 * N * P * 2 * 2 + 3 * 4 * P * 4 + 4 * 8;
}

void free_all(fos_ctx* c)
{
    cudaFree(c->gmm); cudaFree(c->samp); cudaFree(c->Dq); cudaFree(c->R); cudaFree(c->T);
    cudaFree(c->S); cudaFree(c->req); cudaFree(c->prev); cudaFree(c->aux); cudaFree(c->seq);
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->h_rgb[b]); cudaFree(c->h_depth[b]); cudaFree(c->h_mg[b]); cudaFree(c->h_mp[b]);
        if (c->ev_in[b]) cudaEventDestroy(c->ev_in[b]);
        if (c->ev_k[b]) cudaEventDestroy(c->ev_k[b]);
        if (c->ev_done[b]) cudaEventDestroy(c->ev_done[b]);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->out_stream) cudaStreamDestroy(c->out_stream);
}

// Sample / D planes: blocked device layout <-> unpadded [c][k][P] export layout.
int64_t blocked_index(const fos_ctx* c, int ch, int k, int x, int y)
{
    const int64_t seg = int64_t(y) * c->spr + x / kSeg;
    return ((int64_t(ch) * c->nseg + seg) * c->prm.N + k) * kSeg + x % kSeg;
}

void unblock_samples(const fos_ctx* c, const uint16_t* blocked, uint16_t* planes)
{
    const int N = c->prm.N;
    for (int ch = 0; ch < 4; ++ch)
        for (int k = 0; k < N; ++k)
            for (int y = 0; y < c->H; ++y)
                for (int x = 0; x < c->W; ++x)
                    planes[(int64_t(ch) * N + k) * c->P + int64_t(y) * c->W + x] =
                        blocked[blocked_index(c, ch, k, x, y)];
}

void block_samples(const fos_ctx* c, const uint16_t* planes, uint16_t* blocked)
{
    const int N = c->prm.N;
    for (int ch = 0; ch < 4; ++ch)
        for (int k = 0; k < N; ++k)
            for (int y = 0; y < c->H; ++y)
                for (int x = 0; x < c->W; ++x)
                    blocked[blocked_index(c, ch, k, x, y)] =
                        planes[(int64_t(ch) * N + k) * c->P + int64_t(y) * c->W + x];
}

}  // namespace

void fos::set_thread_error(const char* msg) { g_create_error = msg; }

cudaError_t fos::dev_alloc(void** p, size_t bytes)
{
    static const long long fail_after = [] {
        const char* v = std::getenv("FOS_FAIL_ALLOC_AFTER");
        return v ? std::atoll(v) : -1LL;
    }();
    static std::atomic<long long> count{0};
    if (fail_after >= 0 && count.fetch_add(1) >= fail_after) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

GmmArgs fos::ctx_gmm_args(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mask)
{
    return gmm_args(c, rgb, depth, mask);
}

PbasArgs fos::ctx_pbas_args(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mask)
{
    return pbas_args(c, rgb, depth, mask);
}

void fos::ctx_frame_done(fos_ctx* c)
{
    if (pbas_on(c)) c->pending = c->t > 0;
    c->t += 1;
    c->frames_since_counters += 1;
}

bool fos::ctx_gmm_on(const fos_ctx* c) { return gmm_on(c); }
bool fos::ctx_pbas_on(const fos_ctx* c) { return pbas_on(c); }

fos_status fos::ctx_validate_params(const fos_params* p, std::string& why)
{
    return validate_params(p, why);
}

extern "C" {

void fos_default_params(fos_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->methods = FOS_METHOD_GMM | FOS_METHOD_PBAS;
    p->K_rgb = 3; p->K_d = 3;
    p->alpha = 0.001f; p->lambda = 2.5f; p->w_depth = 0.5f; p->T_bg = 0.7f;
    p->v_init_rgb = 36.f; p->v_init_d = 4.f; p->v_min_rgb = 4.f; p->v_min_d = 0.25f;
    p->N = 20; p->n_min = 2;
    p->R_lower_rgb = 18.f; p->R_lower_d = 4.f; p->R_scale = 5.f; p->R_incdec = 0.05f;
    p->T_lower = 2.f; p->T_upper = 200.f; p->T_inc = 1.f; p->T_dec = 0.05f;
    p->alpha_g = 10.f; p->eps_d = 1.f / 16.f;
    p->seed = 0; p->stream_id = 0; p->forced_rng = 0;
    p->depth_full_scale_mm = 10000;
    p->gmm_literal = 0; p->density_scale = 10000.f; p->density_threshold = 1.f;
}

int32_t fos_abi_version(void) { return FOS_ABI_VERSION; }

fos_ctx* fos_create(int32_t width, int32_t height, const fos_params* params)
{
    return fos_create_rgbd(width, height, width, height, params);
}

fos_ctx* fos_create_rgbd(int32_t width, int32_t height, int32_t depth_width, int32_t depth_height,
                         const fos_params* params)
{
    g_create_error.clear();
    g_create_status = FOS_OK;
    if (width < 1 || height < 1 || width > 16384 || height > 16384 || depth_width < 1 || depth_height < 1 ||
        depth_width > 16384 || depth_height > 16384) {
        fail(nullptr, FOS_ERR_INVALID_ARG, "width, height, depth_width, depth_height must be in 1..16384");
        return nullptr;
    }
    std::string why;
    if (validate_params(params, why) != FOS_OK) {
        fail(nullptr, FOS_ERR_INVALID_ARG, why);
        return nullptr;
    }
    fos_ctx* c = new fos_ctx();
    c->W = width; c->H = height;
    c->P = int64_t(width) * height;
    c->Wd = depth_width; c->Hd = depth_height;
    c->Pd = int64_t(depth_width) * depth_height;
    c->plane = round_up(c->P, 128);
    c->spr = (width + kSeg - 1) / kSeg;
    c->Wp = c->spr * kSeg;
    c->nseg = int64_t(c->spr) * height;
    c->pplane = int64_t(c->Wp) * height;
    c->prm = *params;
    auto bail = [&](const char* what, cudaError_t e) -> fos_ctx* {
        cuda_fail(nullptr, what, e);
        free_all(c);
        delete c;
        return nullptr;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return bail("cudaGetDevice", e);
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("cudaStreamCreate", e);
    if ((e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("cudaStreamCreate", e);
    if ((e = cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("cudaStreamCreate", e);
    const size_t pl = size_t(c->plane);
    if (gmm_on(c)) {
        const size_t n = gmm_nplanes(c) * pl * gmm_elem(c);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->gmm), n)) != cudaSuccess) return bail("cudaMalloc(gmm)", e);
    }
    if (pbas_on(c)) {
        const size_t N = size_t(params->N), ns = size_t(c->nseg) * kSeg, pp = size_t(c->pplane);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->samp), 4 * N * ns * 2)) != cudaSuccess) return bail("cudaMalloc(samples)", e);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->Dq), 4 * N * ns * 2)) != cudaSuccess) return bail("cudaMalloc(D)", e);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->R), 4 * pp * 4)) != cudaSuccess) return bail("cudaMalloc(R)", e);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->T), 4 * pp * 4)) != cudaSuccess) return bail("cudaMalloc(T)", e);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->S), 4 * pp * 4)) != cudaSuccess) return bail("cudaMalloc(S)", e);
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->req), 2 * pp * 4)) != cudaSuccess) return bail("cudaMalloc(req)", e);
        // with propagation two planes by frame parity (the requesters' values of
        // frame t-1 are read while frame t's values are written) and, behind
        // them, a uint32 plane with the slots of each pixel's own updates
        const size_t prev_bytes = params->pbas_propagate ? pp * (2 * 8 + 4) : pp * 8;
        if ((e = dev_alloc(reinterpret_cast<void**>(&c->prev), prev_bytes)) != cudaSuccess) return bail("cudaMalloc(prev)", e);
    }
    // gradient sums, counters, and at word 16 the range-checked build's OobWord
    if ((e = dev_alloc(reinterpret_cast<void**>(&c->aux), kAuxWords * sizeof(unsigned long long))) != cudaSuccess) return bail("cudaMalloc(aux)", e);
    if ((e = cudaMemset(c->aux, 0, kAuxWords * sizeof(unsigned long long))) != cudaSuccess) return bail("cudaMemset(aux)", e);
    return c;
}

void fos_destroy(fos_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamSynchronize(ctx->out_stream);
    free_all(ctx);
    delete ctx;
}

const char* fos_last_error(const fos_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

fos_status fos_last_status(const fos_ctx* ctx)
{
    return ctx ? ctx->last_status : g_create_status;
}

fos_status fos_reset(fos_ctx* ctx)
{
    if (!ctx) return FOS_ERR_INVALID_ARG;
    ctx->t = 0;
    ctx->pending = false;
    return FOS_OK;
}

int64_t fos_frame_index(const fos_ctx* ctx) { return ctx ? ctx->t : -1; }

fos_status fos_process_frame_device(fos_ctx* ctx, const uint8_t* d_rgb, const uint16_t* d_depth,
                                    uint8_t* d_mask_gmm, uint8_t* d_mask_pbas, void* stream)
{
    NvtxRange nvtx("fos_process_frame_device");
    if (!ctx) return FOS_ERR_INVALID_ARG;
    return process_device(ctx, d_rgb, d_depth, d_mask_gmm, d_mask_pbas, static_cast<cudaStream_t>(stream));
}

fos_status fos_process_frames_device(fos_ctx* ctx, int32_t n_frames, const uint8_t* d_rgb,
                                     const uint16_t* d_depth, uint8_t* d_mask_gmm,
                                     uint8_t* d_mask_pbas, void* stream)
{
    NvtxRange nvtx("fos_process_frames_device");
    if (!ctx) return FOS_ERR_INVALID_ARG;
    if (n_frames < 0) return fail(ctx, FOS_ERR_INVALID_ARG, "n_frames < 0");
    const int64_t P = ctx->P, Pd = ctx->Pd;
    const fos_params& p = ctx->prm;
    if (n_frames > 1 && gmm_on(ctx) && !pbas_on(ctx) && !p.gmm_literal &&
        ctx->opt[FOS_OPT_TEMPORAL] && gmm_frames_supported(p.K_rgb, p.K_d)) {
        // GMM alone over frames already on the device: one launch for all of them
        if (!d_rgb || !d_depth || !d_mask_gmm)
            return fail(ctx, FOS_ERR_INVALID_ARG, "rgb, depth and mask_gmm must be non-NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (ctx->t == 0) FOS_TRY(ctx, cudaMemsetAsync(ctx->aux, 0, 12 * sizeof(unsigned long long), s));
        GmmArgs a = gmm_args(ctx, d_rgb, d_depth, d_mask_gmm);
        TimedScope ts(ctx, FOS_KERNEL_GMM, s);
        fos_status st = launch_result(ctx, launch_gmm_frames(a, n_frames, p.K_rgb, p.K_d, s), "gmm_frames");
        if (st != FOS_OK) return st;
        ctx->t += n_frames;
        ctx->frames_since_counters += uint64_t(n_frames);
        return FOS_OK;
    }
    return process_device_frames(ctx, n_frames, d_rgb, size_t(P) * 3, d_depth, size_t(Pd), d_mask_gmm, d_mask_pbas,
                                 size_t(P), static_cast<cudaStream_t>(stream));
}

fos_status fos_process_frames_host(fos_ctx* ctx, int32_t n_frames, const uint8_t* rgb,
                                   const uint16_t* depth, uint8_t* mask_gmm, uint8_t* mask_pbas)
{
    NvtxRange nvtx("fos_process_frames_host");
    if (!ctx) return FOS_ERR_INVALID_ARG;
    if (n_frames < 0) return fail(ctx, FOS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames > 0 && (!rgb || !depth)) return fail(ctx, FOS_ERR_INVALID_ARG, "rgb and depth must be non-NULL");
    if (gmm_on(ctx) && !mask_gmm && n_frames > 0) return fail(ctx, FOS_ERR_INVALID_ARG, "mask_gmm must be non-NULL");
    if (pbas_on(ctx) && !mask_pbas && n_frames > 0) return fail(ctx, FOS_ERR_INVALID_ARG, "mask_pbas must be non-NULL");
    if (n_frames == 0) return FOS_OK;
    // Three streams, two staging slots of up to kHostChunk frames: the input
    // copy of chunk g+1 and the mask copy of chunk g-1 run while chunk g's
    // kernels do, and the kernels of one chunk run back to back (one
    // cross-stream wait per chunk, not per frame).  Slot b is reused by
    // chunk g+2 only after chunk g's kernels have read its inputs (ev_k) and
    // its masks have left the device (ev_done).
    const int chunk = n_frames < kHostChunk ? n_frames : kHostChunk;
    fos_status st = ensure_staging(ctx, chunk);
    if (st != FOS_OK) return st;
    const size_t P = size_t(ctx->P), Pd = size_t(ctx->Pd);
    const size_t rp = ctx->stage_rgb, dp = ctx->stage_depth, mp = ctx->stage_mask;
    for (int32_t f0 = 0, g = 0; f0 < n_frames; f0 += chunk, ++g) {
        const int b = g & 1;
        const size_t m = size_t(n_frames - f0 < chunk ? n_frames - f0 : chunk);
        FOS_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_k[b], 0));
        FOS_TRY(ctx, cudaMemcpy2DAsync(ctx->h_rgb[b], rp, rgb + size_t(f0) * P * 3, P * 3, P * 3, m,
                                       cudaMemcpyHostToDevice, ctx->copy_stream));
        FOS_TRY(ctx, cudaMemcpy2DAsync(ctx->h_depth[b], dp, depth + size_t(f0) * Pd, Pd * 2, Pd * 2, m,
                                       cudaMemcpyHostToDevice, ctx->copy_stream));
        FOS_TRY(ctx, cudaEventRecord(ctx->ev_in[b], ctx->copy_stream));
        FOS_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_in[b], 0));
        FOS_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_done[b], 0));
        st = process_device_frames(ctx, int32_t(m), ctx->h_rgb[b], rp, ctx->h_depth[b], dp / 2, ctx->h_mg[b],
                                   ctx->h_mp[b], mp, ctx->stream);
        if (st != FOS_OK) return st;
        FOS_TRY(ctx, cudaEventRecord(ctx->ev_k[b], ctx->stream));
        FOS_TRY(ctx, cudaStreamWaitEvent(ctx->out_stream, ctx->ev_k[b], 0));
        if (gmm_on(ctx))
            FOS_TRY(ctx, cudaMemcpy2DAsync(mask_gmm + size_t(f0) * P, P, ctx->h_mg[b], mp, P, m,
                                           cudaMemcpyDeviceToHost, ctx->out_stream));
        if (pbas_on(ctx))
            FOS_TRY(ctx, cudaMemcpy2DAsync(mask_pbas + size_t(f0) * P, P, ctx->h_mp[b], mp, P, m,
                                           cudaMemcpyDeviceToHost, ctx->out_stream));
        FOS_TRY(ctx, cudaEventRecord(ctx->ev_done[b], ctx->out_stream));
    }
    FOS_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    FOS_TRY(ctx, cudaStreamSynchronize(ctx->out_stream));
    return seq_check(ctx);
}

fos_status fos_process_frame2(fos_ctx* ctx, const uint8_t* rgb, const uint16_t* depth,
                              uint8_t* mask_gmm, uint8_t* mask_pbas)
{
    return fos_process_frames_host(ctx, 1, rgb, depth, mask_gmm, mask_pbas);
}

fos_status fos_process_frame(fos_ctx* ctx, const uint8_t* rgb, const uint16_t* depth, uint8_t* mask_out)
{
    if (!ctx) return FOS_ERR_INVALID_ARG;
    if (!mask_out) return fail(ctx, FOS_ERR_INVALID_ARG, "mask_out must be non-NULL");
    // the mask of the method not returned goes to a host buffer of its own
    if (gmm_on(ctx)) {
        if (!pbas_on(ctx)) return fos_process_frames_host(ctx, 1, rgb, depth, mask_out, nullptr);
        std::vector<uint8_t> unused(size_t(ctx->P));
        return fos_process_frames_host(ctx, 1, rgb, depth, mask_out, unused.data());
    }
    return fos_process_frames_host(ctx, 1, rgb, depth, nullptr, mask_out);
}

fos_status fos_state_size(const fos_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return FOS_ERR_INVALID_ARG;
    *bytes = sizeof(fos_state_header) + gmm_bytes(ctx) + pbas_bytes(ctx);
    return FOS_OK;
}

fos_status fos_get_state(fos_ctx* ctx, void* host_buf, size_t bytes)
{
    if (!ctx || !host_buf) return FOS_ERR_INVALID_ARG;
    size_t need;
    fos_state_size(ctx, &need);
    if (bytes < need) return fail(ctx, FOS_ERR_INVALID_ARG, "state buffer too small");
    FOS_TRY(ctx, cudaDeviceSynchronize());
    if (pbas_on(ctx) && ctx->pending) {
        // the last frame's neighbour updates are applied lazily by the next
        // frame; apply them now so the exported state is complete
        const PbasArgs a = pbas_args(ctx, nullptr, nullptr, nullptr);
        TimedScope ts(ctx, FOS_KERNEL_PBAS_FLUSH, nullptr);
        fos_status st = launch_result(ctx, launch_pbas_flush(a, nullptr), "pbas_flush");
        if (st != FOS_OK) return st;
        ctx->pending = false;
        FOS_TRY(ctx, cudaDeviceSynchronize());
    }
    uint8_t* out = static_cast<uint8_t*>(host_buf);
    fos_state_header h{};
    h.magic = 0x53534F46u; h.abi_version = FOS_ABI_VERSION;
    h.width = ctx->W; h.height = ctx->H; h.methods = ctx->prm.methods;
    h.K_rgb = ctx->prm.K_rgb; h.K_d = ctx->prm.K_d; h.N = ctx->prm.N;
    h.frame_index = ctx->t; h.gmm_bytes = gmm_bytes(ctx); h.pbas_bytes = pbas_bytes(ctx);
    std::memcpy(out, &h, sizeof h);
    out += sizeof h;
    const size_t P = size_t(ctx->P), pl = size_t(ctx->plane);
    if (gmm_on(ctx)) {
        const size_t np = gmm_nplanes(ctx), el = gmm_elem(ctx);
        FOS_TRY(ctx, cudaMemcpy2D(out, P * el, ctx->gmm, pl * el, P * el, np, cudaMemcpyDeviceToHost));
        out += np * P * el;
    }
    if (pbas_on(ctx)) {
        const size_t N4 = 4 * size_t(ctx->prm.N);
        const size_t W = size_t(ctx->W), Wp = size_t(ctx->Wp), H4 = 4 * size_t(ctx->H);
        std::vector<uint16_t> tmp(N4 * size_t(ctx->nseg) * kSeg);
        for (uint16_t* dev : {ctx->samp, ctx->Dq}) {
            FOS_TRY(ctx, cudaMemcpy(tmp.data(), dev, tmp.size() * 2, cudaMemcpyDeviceToHost));
            unblock_samples(ctx, tmp.data(), reinterpret_cast<uint16_t*>(out));
            out += N4 * P * 2;
        }
        for (void* dev : {static_cast<void*>(ctx->R), static_cast<void*>(ctx->T), static_cast<void*>(ctx->S)}) {
            FOS_TRY(ctx, cudaMemcpy2D(out, W * 4, dev, Wp * 4, W * 4, H4, cudaMemcpyDeviceToHost));
            out += 4 * P * 4;
        }
        if (ctx->t > 0) {
            FOS_TRY(ctx, cudaMemcpy(out, ctx->aux + ((ctx->t + 2) % 3) * 4, 32, cudaMemcpyDeviceToHost));
        } else {
            std::memset(out, 0, 32);
        }
    }
    return FOS_OK;
}

fos_status fos_set_state(fos_ctx* ctx, const void* host_buf, size_t bytes)
{
    if (!ctx || !host_buf) return FOS_ERR_INVALID_ARG;
    size_t need;
    fos_state_size(ctx, &need);
    if (bytes < need) return fail(ctx, FOS_ERR_INVALID_ARG, "state buffer too small");
    const uint8_t* in = static_cast<const uint8_t*>(host_buf);
    fos_state_header h;
    std::memcpy(&h, in, sizeof h);
    if (h.magic != 0x53534F46u || h.width != ctx->W || h.height != ctx->H ||
        h.methods != ctx->prm.methods || h.K_rgb != ctx->prm.K_rgb || h.K_d != ctx->prm.K_d ||
        h.N != ctx->prm.N || h.frame_index < 0)
        return fail(ctx, FOS_ERR_INVALID_ARG, "state blob does not match this context");
    in += sizeof h;
    FOS_TRY(ctx, cudaDeviceSynchronize());
    const size_t P = size_t(ctx->P), pl = size_t(ctx->plane);
    if (gmm_on(ctx)) {
        const size_t np = gmm_nplanes(ctx), el = gmm_elem(ctx);
        FOS_TRY(ctx, cudaMemcpy2D(ctx->gmm, pl * el, in, P * el, P * el, np, cudaMemcpyHostToDevice));
        in += np * P * el;
    }
    if (pbas_on(ctx)) {
        const size_t N4 = 4 * size_t(ctx->prm.N);
        const size_t W = size_t(ctx->W), Wp = size_t(ctx->Wp), H4 = 4 * size_t(ctx->H);
        std::vector<uint16_t> tmp(N4 * size_t(ctx->nseg) * kSeg, 0);
        for (uint16_t* dev : {ctx->samp, ctx->Dq}) {
            block_samples(ctx, reinterpret_cast<const uint16_t*>(in), tmp.data());
            FOS_TRY(ctx, cudaMemcpy(dev, tmp.data(), tmp.size() * 2, cudaMemcpyHostToDevice));
            in += N4 * P * 2;
        }
        for (void* dev : {static_cast<void*>(ctx->R), static_cast<void*>(ctx->T), static_cast<void*>(ctx->S)}) {
            FOS_TRY(ctx, cudaMemcpy2D(dev, Wp * 4, in, W * 4, W * 4, H4, cudaMemcpyHostToDevice));
            in += 4 * P * 4;
        }
        // gsum of the last frame goes where the next frame reads it; the
        // other buffers are accumulators and start at zero; nothing pending
        const int64_t t = h.frame_index;
        unsigned long long g[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (t > 0) std::memcpy(g + ((t + 2) % 3) * 4, in, 32);
        FOS_TRY(ctx, cudaMemcpy(ctx->aux, g, sizeof g, cudaMemcpyHostToDevice));
        ctx->pending = false;
    }
    ctx->t = h.frame_index;
    return FOS_OK;
}

fos_status fos_set_timing(fos_ctx* ctx, uint32_t kernel_mask)
{
    if (!ctx) return FOS_ERR_INVALID_ARG;
    ctx->timing_mask = kernel_mask;
    return FOS_OK;
}

fos_status fos_get_timing(fos_ctx* ctx, fos_kernel_timing out[FOS_KERNEL_COUNT])
{
    if (!ctx || !out) return FOS_ERR_INVALID_ARG;
    for (int k = 0; k < FOS_KERNEL_COUNT; ++k) { out[k].launches = 0; out[k].total_ms = 0.0; out[k].frames = 0; }
    for (const TimedLaunch& tl : ctx->timed) {
        FOS_TRY(ctx, cudaEventSynchronize(tl.stop));
        float ms = 0.f;
        FOS_TRY(ctx, cudaEventElapsedTime(&ms, tl.start, tl.stop));
        out[tl.kind].launches += 1;
        out[tl.kind].total_ms += ms;
        out[tl.kind].frames += tl.frames;
    }
    ctx->timed.clear();
    ctx->ev_used = 0;
    return FOS_OK;
}

fos_status fos_set_option(fos_ctx* ctx, int32_t option, int32_t value)
{
    if (!ctx) return FOS_ERR_INVALID_ARG;
    bool ok = false;
    switch (option) {
    case FOS_OPT_GMM_PX: ok = value == 1 || value == 2 || value == 4; break;
    case FOS_OPT_GMM_TPB: ok = value == 64 || value == 128 || value == 256; break;
    case FOS_OPT_PBAS_PX: ok = value == 1 || value == 2 || value == 4; break;
    case FOS_OPT_PBAS_TY: ok = value == 2 || value == 4 || value == 8; break;
    case FOS_OPT_FUSE: ok = value == 0 || value == 1; break;
    case FOS_OPT_TEMPORAL: ok = value == 0 || value == 1; break;
    case FOS_OPT_SEQUENCE: ok = value == 0 || value == 1; break;
    case FOS_OPT_GMM_STREAM: ok = value == 0 || value == 1; break;
    default: return fail(ctx, FOS_ERR_INVALID_ARG, "unknown option");
    }
    if (!ok) return fail(ctx, FOS_ERR_INVALID_ARG, "option value not supported");
    if (option == FOS_OPT_PBAS_PX || option == FOS_OPT_PBAS_TY) {
        const int px = option == FOS_OPT_PBAS_PX ? value : ctx->opt[FOS_OPT_PBAS_PX];
        const int ty = option == FOS_OPT_PBAS_TY ? value : ctx->opt[FOS_OPT_PBAS_TY];
        if (px == 2 && ty == 2) return fail(ctx, FOS_ERR_UNSUPPORTED, "PBAS tile 2 x 2 not compiled in");
    }
    ctx->opt[option] = value;
    return FOS_OK;
}

int32_t fos_get_option(const fos_ctx* ctx, int32_t option)
{
    if (!ctx || option < 1 || option >= FOS_OPT_COUNT) return -1;
    return ctx->opt[option];
}

fos_status fos_get_counters(fos_ctx* ctx, uint64_t out[4])
{
    if (!ctx || !out) return FOS_ERR_INVALID_ARG;
    FOS_TRY(ctx, cudaDeviceSynchronize());
    FOS_TRY_ST(seq_check(ctx));
    unsigned long long c[4];
    FOS_TRY(ctx, cudaMemcpy(c, ctx->aux + 12, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = ctx->frames_since_counters;
    FOS_TRY(ctx, cudaMemset(ctx->aux + 12, 0, 3 * sizeof(unsigned long long)));
    ctx->frames_since_counters = 0;
    return FOS_OK;
}

}  // extern "C"

extern "C" int32_t fos_bounds_checked(void)
{
#ifdef FOS_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

extern "C" fos_status fos_bounds_status(fos_ctx* ctx, uint32_t* violations, uint32_t* first_site,
                                        int64_t* first_index)
{
    if (!ctx || !violations) return FOS_ERR_INVALID_ARG;
#ifdef FOS_DEBUG_BOUNDS
    FOS_TRY(ctx, cudaSetDevice(ctx->device));
    FOS_TRY(ctx, cudaDeviceSynchronize());
    fos::OobWord w{};
    FOS_TRY(ctx, cudaMemcpy(&w, oob_of(ctx), sizeof w, cudaMemcpyDeviceToHost));
    FOS_TRY(ctx, cudaMemset(oob_of(ctx), 0, sizeof w));
    *violations = w.count;
    if (first_site) *first_site = w.site;
    if (first_index) *first_index = w.index;
    return FOS_OK;
#else
    *violations = 0;
    return fail(ctx, FOS_ERR_UNSUPPORTED, "fos_bounds_status: not a range-checked build (FOS_DEBUG_BOUNDS)");
#endif
}

#ifdef FOS_DEBUG_BOUNDS
namespace {
// Reads element i of a 16-element buffer through the checked accessor with a
// declared extent of n: for i >= n the check records the violation and the
// read goes to the sink, so the buffer is never accessed out of its range.
__global__ void bounds_selftest_kernel(const uint32_t* buf, int64_t i, int64_t n, fos::OobWord* w, uint32_t* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = fos::at(buf, i, n, 99, w);
}
}  // namespace
#endif

extern "C" fos_status fos_bounds_selftest(uint32_t* violations, uint32_t* first_site, int64_t* first_index)
{
    if (!violations) return FOS_ERR_INVALID_ARG;
    *violations = 0;
#ifdef FOS_DEBUG_BOUNDS
    uint32_t* buf = nullptr;
    fos::OobWord w{};
    cudaError_t e = cudaMalloc(&buf, 64 * sizeof(uint32_t) + sizeof(fos::OobWord));
    fos::OobWord* dw = reinterpret_cast<fos::OobWord*>(buf + 32);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, 64 * sizeof(uint32_t) + sizeof(fos::OobWord));
    if (e == cudaSuccess) {
        bounds_selftest_kernel<<<1, 32>>>(buf, 12, 8, dw, buf + 16);  // element 12 is in the buffer, above 8
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&w, dw, sizeof w, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return FOS_ERR_CUDA;
    }
    *violations = w.count;
    if (first_site) *first_site = w.site;
    if (first_index) *first_index = w.index;
    return FOS_OK;
#else
    (void)first_site;
    (void)first_index;
    set_thread_error("fos_bounds_selftest: not a range-checked build (FOS_DEBUG_BOUNDS)");
    return FOS_ERR_UNSUPPORTED;
#endif
}
