// ctx.h -- the context object behind fos_ctx (internal to the library).
#pragma once

#include <string>
#include <vector>

#include "fos.h"
#include "fos_internal.h"

namespace fos {
struct TimedLaunch {
    int kind;
    int64_t frames;  // frames the launch processed
    cudaEvent_t start, stop;
};
}  // namespace fos

struct fos_ctx {
    int W = 0, H = 0;
    int64_t P = 0, plane = 0;       // GMM planes: P padded to 128
    int Wp = 0, spr = 0;            // PBAS: row pitch, 128-pixel segments per row
    int Wd = 0, Hd = 0;             // depth frames (read through the resampling map when they differ)
    int64_t Pd = 0;
    int64_t nseg = 0, pplane = 0;   // PBAS: segments, plane stride (Wp * H)
    fos_params prm{};
    int64_t t = 0;
    int device = 0;
    cudaStream_t stream = nullptr;       // host-pointer API: kernels
    cudaStream_t copy_stream = nullptr;  // host-pointer API: input copies
    cudaStream_t out_stream = nullptr;   // host-pointer API: mask copies
    float* gmm = nullptr;
    uint16_t* samp = nullptr;
    uint16_t* Dq = nullptr;
    float* R = nullptr;
    float* T = nullptr;
    uint32_t* S = nullptr;
    uint32_t* req = nullptr;            // [2][pplane] requests of even / odd frames
    uint64_t* prev = nullptr;           // [pplane]
    bool pending = false;               // requests of the last frame not yet applied
    int opt[FOS_OPT_COUNT] = {0, 4, 128, 2, 8, 1, 1, 1, 1};  // kernel shapes (fos_set_option)
    unsigned long long* aux = nullptr;  // gsum[3][4], counters[3]
    // several frames in one launch (grown on demand): a 256-byte header (tile
    // counter, error word, 8 scratch sums), gradient sums [frames + 1][4],
    // tile completion words [tiles]
    uint8_t* seq = nullptr;
    int seq_frames = 0, seq_tiles = 0;
    // device staging for host frames: two slots of stage_frames frames each,
    // frame pitches rounded up to 256 bytes
    int stage_frames = 0;
    size_t stage_rgb = 0, stage_depth = 0, stage_mask = 0;
    uint8_t* h_rgb[2] = {nullptr, nullptr};
    uint16_t* h_depth[2] = {nullptr, nullptr};
    uint8_t* h_mg[2] = {nullptr, nullptr};
    uint8_t* h_mp[2] = {nullptr, nullptr};
    // by staging slot: inputs copied in, kernel done (inputs free, masks
    // ready), masks copied out (mask staging free)
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_k[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    uint32_t timing_mask = 0;
    std::vector<fos::TimedLaunch> timed;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    uint64_t frames_since_counters = 0;
    std::string err;
    fos_status last_status = FOS_OK;    // status of the last failed call (fos_last_status)
};

namespace fos {
// Kernel arguments of one frame of a context (device frame pointers).
GmmArgs ctx_gmm_args(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mask);
PbasArgs ctx_pbas_args(fos_ctx* c, const uint8_t* rgb, const uint16_t* depth, uint8_t* mask);
// Book-keeping after a frame of the context ran (by any launch path).
void ctx_frame_done(fos_ctx* c);
bool ctx_gmm_on(const fos_ctx* c);
bool ctx_pbas_on(const fos_ctx* c);
// Parameter validation shared by every creation path; returns FOS_OK or an
// error with the reason in `why`.
fos_status ctx_validate_params(const fos_params* p, std::string& why);
}  // namespace fos
