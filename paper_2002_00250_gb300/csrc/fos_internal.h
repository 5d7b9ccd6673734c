// fos_internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/fos.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fos {

// Launch status of an internal launcher.
enum LaunchResult { kLaunchOk = 0, kLaunchUnsupported = 1, kLaunchCudaError = 2 };

// Plane layout of the GMM state (float32, one plane of `plane` elements each):
// colour model  w[k]=k, mu_r[k]=Kr+k, mu_g[k]=2Kr+k, mu_b[k]=3Kr+k, v[k]=4Kr+k;
// depth model   w[k]=5Kr+k, mu[k]=5Kr+Kd+k, v[k]=5Kr+2Kd+k.
inline int gmm_planes(int Kr, int Kd) { return 5 * Kr + 3 * Kd; }

struct GmmArgs {
    int64_t P;          // pixels
    int64_t plane;      // plane stride in elements (multiple of 128)
    float* state;       // gmm_planes(Kr,Kd) * plane floats
    const uint8_t* rgb; // P*3
    const uint16_t* depth;  // P
    uint8_t* mask;      // P
    float alpha, lam2, w_depth, T_bg;
    float v_init_rgb, v_init_d, v_min_rgb, v_min_d;
    uint32_t depth_fs;  // depth full scale (mm)
    int init;           // 1: frame 0 (bootstrap)
    int vec_ok;         // 1: pointers aligned for the vectorised path
};

LaunchResult launch_gmm(const GmmArgs& a, int Kr, int Kd, cudaStream_t s);

// PBAS device state.  Frames are cut into row segments of kSeg = 128 pixels
// (spr = ceil(W / 128) segments per row, nseg = H * spr).  Samples and D are
// uint16 in a blocked layout: element (c, k, x, y) sits at
//   ((c * nseg + y * spr + x / 128) * N + k) * 128 + x % 128,
// so the N slots of one channel of one segment are 256-byte rows of one
// contiguous block: a warp reads each slot with one coalesced 256-byte access
// and its random own/neighbour slot writes land in the block it just read.
// R, T, S (per channel) and the request word are planes with row pitch
// Wp = spr * 128; plane stride `plane` = Wp * H.  Request byte c of a pixel:
// 0 none, else 1 + j * N + k2.
constexpr int kSeg = 128;

struct PbasArgs {
    int W, H;
    int64_t P;
    int Wp, spr;
    int64_t nseg, plane;
    const uint8_t* rgb;
    const uint16_t* depth;
    uint8_t* mask;
    uint16_t* samp;
    uint16_t* Dq;
    float* R;
    float* T;
    uint32_t* S;
    uint32_t* req;
    unsigned long long* gsum_prev;  // [4] gradient sums of the previous frame
    unsigned long long* gsum_cur;   // [4] accumulated for this frame (zeroed beforehand)
    unsigned long long* counters;   // [3] own updates, neighbour writes, requests
    float R_lower_rgb, R_lower_d, R_scale, R_incdec;
    float T_lower, T_upper, T_inc, T_dec, alpha_g, eps_d;
    int N, n_min;
    uint32_t seed, stream_id;
    int forced;
    uint32_t depth_fs;
    uint32_t t;   // frame index
    int vec_ok;   // W % 4 == 0 and a 4-byte aligned mask
};

LaunchResult launch_pbas_init(const PbasArgs& a, cudaStream_t s);
LaunchResult launch_pbas_classify(const PbasArgs& a, cudaStream_t s);
LaunchResult launch_pbas_neighbour(const PbasArgs& a, cudaStream_t s);

}  // namespace fos
