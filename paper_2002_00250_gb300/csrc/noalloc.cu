// noalloc.cu -- fos_pbas_step_noalloc: one PBAS frame step that allocates no
// memory at all.
//
// Some callers cannot allocate device memory at the moment they process a
// frame: a plug-in running inside a host framework that owns every device
// allocation and forbids allocation while a pipeline runs, a hard real-time
// capture callback where cudaMalloc's implicit synchronisation and unbounded
// latency are not acceptable, or code that must not touch the allocator while
// other work may be capturing streams.  For them this entry point takes the
// model and the frame in caller-owned device memory and keeps its own scratch
// (the per-pixel neighbour-request words, the frame's (value, gradient)
// words and three counters) in one file-scope __device__ array of fixed size.
//
// The kernels are the library's PBAS kernels unchanged: the classify pass of
// the frame, then the pass that applies this frame's neighbour requests, so
// the model the call leaves behind already contains them.
#include <cstdio>
#include <mutex>
#include <string>

#include "ctx.h"
#include "fos.h"
#include "fos_internal.h"

using namespace fos;

namespace {

// Scratch layout: request words (uint32) for FOS_NOALLOC_MAX_PIXELS padded
// pixels, then (value | gradient << 8) words (uint64) for as many, then three
// uint64 counters.  Every GPU that loads the library holds it until exit.
constexpr size_t kReqBytes = size_t(FOS_NOALLOC_MAX_PIXELS) * 4;
constexpr size_t kPrevBytes = size_t(FOS_NOALLOC_MAX_PIXELS) * 8;
constexpr size_t kScratchBytes = kReqBytes + kPrevBytes + 256;
__device__ __align__(256) unsigned char g_pbas_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device.  In host
// code g_pbas_scratch names a host-side stand-in, not device memory, so the
// kernels are only ever given the address cudaGetSymbolAddress returns.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pbas_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// The message goes where fos_last_error(NULL) reads it on this thread.
fos_status noalloc_fail(fos_status st, const char* msg, cudaError_t e = cudaSuccess)
{
    char buf[320];
    if (e != cudaSuccess)
        std::snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else
        std::snprintf(buf, sizeof buf, "%s", msg);
    set_thread_error(buf);
    return st;
}

}  // namespace

extern "C" fos_status fos_pbas_step_noalloc(int32_t width, int32_t height, const fos_params* params,
                                            int64_t frame_index, const uint8_t* d_rgb,
                                            const uint16_t* d_depth, void* d_model, uint8_t* d_mask,
                                            void* stream)
{
    set_thread_error("");
    if (!params || !d_rgb || !d_depth || !d_model || !d_mask)
        return noalloc_fail(FOS_ERR_INVALID_ARG, "fos_pbas_step_noalloc: NULL argument");
    if (width < 1 || height < 1 || frame_index < 0)
        return noalloc_fail(FOS_ERR_INVALID_ARG, "fos_pbas_step_noalloc: bad size or frame index");
    const int spr = (width + kSeg - 1) / kSeg;
    const int64_t padded = int64_t(spr) * kSeg * height;
    if (padded > int64_t(FOS_NOALLOC_MAX_PIXELS))
        return noalloc_fail(FOS_ERR_INVALID_ARG,
                            "fos_pbas_step_noalloc: frame too large: 128*ceil(width/128)*height "
                            "exceeds FOS_NOALLOC_MAX_PIXELS (2097152)");
    if (reinterpret_cast<uintptr_t>(d_model) % 256 != 0)
        return noalloc_fail(FOS_ERR_INVALID_ARG, "fos_pbas_step_noalloc: d_model must be 256-byte aligned");
    // the same parameter checks as a PBAS-only context (methods is ignored here)
    fos_params pv = *params;
    pv.methods = FOS_METHOD_PBAS;
    pv.gmm_literal = 0;
    std::string why;
    const fos_status vs = ctx_validate_params(&pv, why);
    if (vs != FOS_OK) return noalloc_fail(vs, ("fos_pbas_step_noalloc: " + why).c_str());
    const fos_params& p = *params;
    if (p.pbas_propagate)
        return noalloc_fail(FOS_ERR_UNSUPPORTED,
                            "fos_pbas_step_noalloc: spatial propagation needs a second value plane (not in the scratch)");
    if (p.pbas_joint)
        return noalloc_fail(FOS_ERR_UNSUPPORTED, "fos_pbas_step_noalloc: the per-channel PBAS only (pbas_joint = 0)");

    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return noalloc_fail(FOS_ERR_CUDA, "fos_pbas_step_noalloc: scratch set-up", e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* sc = static_cast<uint8_t*>(scratch);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(sc + kReqBytes + kPrevBytes);
    // the counters accumulate: start them at zero (request and value words are
    // fully rewritten by the classify pass before anything reads them)
    e = cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return noalloc_fail(FOS_ERR_CUDA, "fos_pbas_step_noalloc: cudaMemsetAsync", e);

    // caller's model buffer (layout documented with the declaration)
    const int64_t N = p.N;
    uint8_t* m = static_cast<uint8_t*>(d_model);
    PbasArgs a{};
    a.W = width; a.H = height; a.P = int64_t(width) * height;
    a.Wd = width; a.Hd = height;
    a.propagate = 0;
    a.Wp = spr * kSeg; a.spr = spr; a.nseg = int64_t(spr) * height; a.plane = padded;
    a.rgb = d_rgb; a.depth = d_depth; a.mask = d_mask;
    a.samp = reinterpret_cast<uint16_t*>(m);
    a.Dq = reinterpret_cast<uint16_t*>(m + 8 * N * padded);
    a.R = reinterpret_cast<float*>(m + 16 * N * padded);
    a.T = reinterpret_cast<float*>(m + 16 * N * padded + 16 * padded);
    a.S = reinterpret_cast<uint32_t*>(m + 16 * N * padded + 32 * padded);
    unsigned long long* gsum = reinterpret_cast<unsigned long long*>(m + 16 * N * padded + 48 * padded);
    a.prev = reinterpret_cast<uint64_t*>(sc + kReqBytes);
    a.prev_src = a.prev;
    a.req_cur = reinterpret_cast<uint32_t*>(sc);
    a.req_prev = reinterpret_cast<uint32_t*>(sc);
    const int64_t t = frame_index;
    a.gsum_prev = gsum + ((t + 2) % 3) * 4;
    a.gsum_cur = gsum + (t % 3) * 4;
    a.gsum_next = gsum + ((t + 1) % 3) * 4;
    a.counters = counters;
    a.R_lower_rgb = p.R_lower_rgb; a.R_lower_d = p.R_lower_d; a.R_scale = p.R_scale;
    a.R_incdec = p.R_incdec; a.T_lower = p.T_lower; a.T_upper = p.T_upper;
    a.T_inc = p.T_inc; a.T_dec = p.T_dec; a.alpha_g = p.alpha_g; a.eps_d = p.eps_d;
    a.N = p.N; a.n_min = p.n_min; a.seed = p.seed; a.stream_id = p.stream_id;
    a.forced = p.forced_rng; a.depth_fs = p.depth_full_scale_mm;
    a.t = uint32_t(t);
    a.px = 2;
    a.ty = 8;
    a.mask_vec = (reinterpret_cast<uintptr_t>(d_mask) % 2) == 0 ? 1 : 0;
    pbas_args_finish(a);

    LaunchResult r;
    if (t == 0) {
        e = cudaMemsetAsync(gsum, 0, 12 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return noalloc_fail(FOS_ERR_CUDA, "fos_pbas_step_noalloc: cudaMemsetAsync", e);
        a.apply = 0;
        r = launch_pbas_init(a, s);
    } else {
        a.apply = 0;  // the previous call already applied its requests
        r = launch_pbas_classify(a, s);
        if (r == kLaunchOk) r = launch_pbas_flush(a, s);
    }
    if (r == kLaunchUnsupported) return noalloc_fail(FOS_ERR_UNSUPPORTED, "fos_pbas_step_noalloc: unsupported shape");
    if (r != kLaunchOk) return noalloc_fail(FOS_ERR_CUDA, "fos_pbas_step_noalloc: launch", cudaGetLastError());
    return FOS_OK;
}
