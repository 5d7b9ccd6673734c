// gmm.cu -- GMM classify-and-update over RGB and depth (paper Sec. 3.1, Eq. 1).
//
// One thread owns PX consecutive pixels.  The model state is structure-of-
// arrays (one float32 plane per component parameter), so each plane is read
// and written with PX-wide vector accesses that coalesce across the warp; the
// whole per-pixel update runs in registers (components are compile-time
// unrolled, the re-ranking is a stable bubble network of compare-and-swap).
// Input conversion (Sec. 4.2 depth rescale) is fused.  The kernel is bound by
// HBM: (5*Kr + 3*Kd) * 4 bytes of state are read and written per pixel-frame.
#include <algorithm>
#include <cmath>

#include "bulk.cuh"
#include "fos_internal.h"
#include "gmm_dev.cuh"

namespace fos {
namespace {
using namespace gmmdev;

// Depth reading of colour pixel p (through the resampling map when the depth
// frame has another size).
__device__ __forceinline__ uint32_t depth_at(const GmmArgs& a, int64_t p)
{
    const uint16_t* d = a.depth;
    const int64_t nd = int64_t(a.Wd) * a.Hd;
    if (a.Wd == a.W && a.Hd == a.H) return at(d, p, nd, 44, a.oob);
    const int y = int(uint32_t(p) / uint32_t(a.W)), x = int(p) - y * a.W;  // P < 2^28
    return at(d, depth_index(x, y, a.W, a.H, a.Wd, a.Hd), nd, 44, a.oob);
}

// PX consecutive pixels per thread starting at pixel p0 of one stream.
template <int KR, int KD, int PX>
__device__ __forceinline__ void gmm_pixels(const GmmArgs& a, int64_t p0)
{
    if (p0 >= a.P) return;
    const int64_t ne = int64_t(5 * KR + 3 * KD) * a.plane;  // state extent (range-checked builds)
    // PX = 4 reads the inputs as 32/64-bit words: needs aligned frame buffers
    if (PX > 1 && (PX != 4 || a.vec_ok) && p0 + PX <= a.P) {
        Mix<KR, 3> mr[PX];
        Mix<KD, 1> md[PX];
        if (!a.init) move_state<KR, KD, PX, false>(a.state, a.plane, p0, mr, md, ne, a.oob);
        uint32_t rgbw[3 * PX / 4 > 0 ? 3 * PX / 4 : 1];
        uint16_t dv[PX];
        uint8_t rgbb[3 * PX];
        if constexpr (PX == 4) {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(a.rgb + 3 * p0);
            rgbw[0] = at(src, 0, 3 * (a.P - p0) / 4, 45, a.oob);
            rgbw[1] = at(src, 1, 3 * (a.P - p0) / 4, 45, a.oob);
            rgbw[2] = at(src, 2, 3 * (a.P - p0) / 4, 45, a.oob);
#pragma unroll
            for (int j = 0; j < 12; ++j) rgbb[j] = uint8_t(rgbw[j >> 2] >> (8 * (j & 3)));
            const uint2 dd = vat<const uint2>(a.depth, p0, 4, a.P, 46, a.oob);
            dv[0] = uint16_t(dd.x); dv[1] = uint16_t(dd.x >> 16);
            dv[2] = uint16_t(dd.y); dv[3] = uint16_t(dd.y >> 16);
        } else {
#pragma unroll
            for (int j = 0; j < 3 * PX; ++j) rgbb[j] = at(a.rgb, 3 * p0 + j, 3 * a.P, 47, a.oob);
#pragma unroll
            for (int i = 0; i < PX; ++i) dv[i] = uint16_t(depth_at(a, p0 + i));
        }
        uint8_t m[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i)
            m[i] = gmm_pixel<KR, KD>(mr[i], md[i], rgbb[3 * i], rgbb[3 * i + 1], rgbb[3 * i + 2],
                                     dv[i], a);
        move_state<KR, KD, PX, true>(a.state, a.plane, p0, mr, md, ne, a.oob);
        if constexpr (PX == 4) {
            vat<uint32_t>(a.mask, p0, 4, a.P, 48, a.oob) =
                uint32_t(m[0]) | (uint32_t(m[1]) << 8) | (uint32_t(m[2]) << 16) | (uint32_t(m[3]) << 24);
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i) at(a.mask, p0 + i, a.P, 48, a.oob) = m[i];
        }
        return;
    }
    // scalar path: ragged tail or unaligned buffers
    for (int64_t p = p0; p < p0 + PX && p < a.P; ++p) {
        Mix<KR, 3> mr[1];
        Mix<KD, 1> md[1];
        if (!a.init) move_state<KR, KD, 1, false>(a.state, a.plane, p, mr, md, ne, a.oob);
        const uint8_t m = gmm_pixel<KR, KD>(mr[0], md[0], at(a.rgb, 3 * p, 3 * a.P, 49, a.oob),
                                            at(a.rgb, 3 * p + 1, 3 * a.P, 49, a.oob),
                                            at(a.rgb, 3 * p + 2, 3 * a.P, 49, a.oob), depth_at(a, p), a);
        move_state<KR, KD, 1, true>(a.state, a.plane, p, mr, md, ne, a.oob);
        at(a.mask, p, a.P, 50, a.oob) = m;
    }
}

template <int KR, int KD, int PX>
__global__ void __launch_bounds__(256) gmm_kernel(const GmmArgs a)
{
    gmm_pixels<KR, KD, PX>(a, (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * PX);
}

// Many streams in one launch: entry i of the table (a __grid_constant__
// parameter, read from the constant bank) holds stream i's arguments and its
// first block in the launch; one block per block of pixels of every stream.
template <int KR, int KD, int PX>
__global__ void __launch_bounds__(kGmmBatchThreads) gmm_batch_kernel(const __grid_constant__ GmmBatchTable T)
{
    const int it = int(blockIdx.x);
    if (it >= T.total) return;
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.e[mid].block_off <= it) lo = mid;
        else hi = mid - 1;
    }
    gmm_pixels<KR, KD, PX>(T.e[lo].a, (int64_t(it - T.e[lo].block_off) * blockDim.x + threadIdx.x) * PX);
}

// Two pixels per thread through gmm_pair (frames >= 1, depth of the colour
// frame's size): the two colour mixtures, then the two depth mixtures, each
// parameter plane moved with one 8-byte access; a lower register peak than
// gmm_pixels (more warps resident to hide the plane loads).  Same arithmetic
// (mix_step) and bits.
template <int KR, int KD, int MINB>
__global__ void __launch_bounds__(256, MINB) gmm_pair_kernel(const GmmArgs a)
{
    const int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 2;
    if (p >= a.P) return;
    if (p + 2 > a.P) {  // odd pixel count: the last pixel alone
        gmm_pixels<KR, KD, 1>(a, p);
        return;
    }
    uint32_t r[2], g[2], b[2], d8[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        r[i] = at(a.rgb, 3 * (p + i), 3 * a.P, 47, a.oob);
        g[i] = at(a.rgb, 3 * (p + i) + 1, 3 * a.P, 47, a.oob);
        b[i] = at(a.rgb, 3 * (p + i) + 2, 3 * a.P, 47, a.oob);
        d8[i] = depth_to_u8(at(a.depth, p + i, a.P, 46, a.oob), a.depth_fs);
    }
    const uint32_t m = gmm_pair<KR, KD>(a, p, r, g, b, d8);
    if ((reinterpret_cast<uintptr_t>(a.mask) & 1u) == 0) {
        vat<uint16_t>(a.mask, p, 2, a.P, 48, a.oob) = uint16_t(m);
    } else {
        at(a.mask, p, a.P, 48, a.oob) = uint8_t(m);
        at(a.mask, p + 1, a.P, 48, a.oob) = uint8_t(m >> 8);
    }
}

// --- frames >= 1 through a bulk-copy pipeline -------------------------------
//
// The per-frame GMM is a pure stream (96 B of state read and written per
// pixel), but its per-pixel update needs ~110 registers, which leaves too few
// warps resident to keep enough plane loads in flight.  Here the loads are
// decoupled from the registers: a persistent block walks chunks of pixels
// (one per thread); one thread issues bulk asynchronous copies of the next
// chunks' planes, colour and depth into a ring of shared-memory stages
// (completing on an mbarrier per stage) and every thread updates one pixel
// of the current stage (the arithmetic of gmm_pixel: same bits as the other
// GMM kernels).  stages - 1 chunks are in flight per block while one computes.
// 128-pixel chunks, 3 stages (38.8 KB of shared memory per block): five
// blocks per SM, 20 warps.  At 1280x720: 32.3 us per frame against 35.6 with
// 256-pixel chunks (two blocks per SM), 33.6 with 224 (three), 32.7 with 96
// (seven) and 35.0 with 128 and 4 stages (four); the register kernels took
// 44.9 (4 pixels per thread, 161 registers, three 128-thread blocks per SM).
constexpr int kGsPx = 128;     // pixels per chunk = threads per block
constexpr int kGsStages = 3;   // ring depth: chunks k+1, k+2 load while k computes
constexpr int kGsMinBlocks = 4;
constexpr uint32_t kGsSpinLimit = 1u << 22;  // bounded mbarrier polls (far beyond any copy)

template <int KR, int KD>
struct GsStage {
    static constexpr int NP = 5 * KR + 3 * KD;
    float st[NP * kGsPx];        // plane q of the chunk at st[q * kGsPx]
    uint8_t rgb[3 * kGsPx];
    uint16_t depth[kGsPx];
    static constexpr uint32_t kInBytes = NP * kGsPx * 4 + 3 * kGsPx + 2 * kGsPx;
};

// Each thread writes its pixel's updated planes and mask byte straight from
// registers (a warp stores 128 contiguous bytes per plane), so a stage is
// free for the next loads as soon as its chunk has been computed.
template <int KR, int KD>
__global__ void __launch_bounds__(kGsPx, kGsMinBlocks) gmm_stream_kernel(const GmmArgs a)
{
    using St = GsStage<KR, KD>;
    constexpr int NP = St::NP;
    extern __shared__ __align__(128) uint8_t gs_raw[];
    St* S = reinterpret_cast<St*>(gs_raw);
    __shared__ __align__(8) uint64_t full[kGsStages];
    const int tid = threadIdx.x;
    const int64_t nchunk = a.P / kGsPx;
    const int64_t G = gridDim.x;
    const int64_t mine = nchunk > int64_t(blockIdx.x) ? (nchunk - 1 - blockIdx.x) / G + 1 : 0;
    if (tid == 0) {
        for (int q = 0; q < kGsStages; ++q) mbar_init(&full[q], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // thread 0: the loads of this block's k-th chunk into stage k % kGsStages
    auto issue = [&](int64_t k) {
        St& T = S[k % kGsStages];
        uint64_t* bar = &full[k % kGsStages];
        const int64_t p0 = (int64_t(blockIdx.x) + k * G) * kGsPx;
        mbar_arrive_expect_tx(bar, St::kInBytes);
#pragma unroll 1
        for (int q = 0; q < NP; ++q) bulk_load(T.st + q * kGsPx, a.state + int64_t(q) * a.plane + p0, kGsPx * 4, bar);
        bulk_load(T.rgb, a.rgb + 3 * p0, 3 * kGsPx, bar);
        bulk_load(T.depth, a.depth + p0, 2 * kGsPx, bar);
    };
    if (tid == 0)
        for (int64_t k = 0; k < kGsStages && k < mine; ++k) issue(k);
    int64_t failed = -1;  // chunk whose wait gave up
    const int64_t ne = int64_t(NP) * a.plane;
    for (int64_t k = 0; k < mine; ++k) {
        const int q = int(k % kGsStages);
        const bool ok = bulk_wait(&full[q], uint32_t(k / kGsStages) & 1u, kGsSpinLimit);
        if (__syncthreads_or(!ok)) {
            failed = k;
            break;
        }
        St& T = S[q];
        Mix<KR, 3> mr[1];
        Mix<KD, 1> md[1];
        constexpr int64_t ns = int64_t(NP) * kGsPx;
        move_state<KR, KD, 1, false>(T.st, kGsPx, tid, mr, md, ns, a.oob);
        const uint32_t r = at(T.rgb, 3 * tid, 3 * kGsPx, 54, a.oob), g = at(T.rgb, 3 * tid + 1, 3 * kGsPx, 54, a.oob);
        const uint32_t b = at(T.rgb, 3 * tid + 2, 3 * kGsPx, 54, a.oob), d = at(T.depth, tid, kGsPx, 54, a.oob);
        __syncthreads();  // the stage has been read: its next loads may start
        if (tid == 0 && k + kGsStages < mine) issue(k + kGsStages);
        const int64_t p = (int64_t(blockIdx.x) + k * G) * kGsPx + tid;
        const uint8_t m = gmm_pixel<KR, KD>(mr[0], md[0], r, g, b, d, a);
        move_state<KR, KD, 1, true>(a.state, a.plane, p, mr, md, ne, a.oob);
        at(a.mask, p, a.P, 54, a.oob) = m;
    }
    if (failed >= 0 && tid == 0) {
        // report, and let the loads already issued (chunks failed ..
        // failed + stages - 1) land, bounded, before the shared memory goes away
        atomicExch(a.err, 1);
        for (int64_t j = failed; j < failed + kGsStages && j < mine; ++j)
            bulk_wait(&full[j % kGsStages], uint32_t(j / kGsStages) & 1u, kGsSpinLimit);
    }
    // the pixels after the last whole chunk: one thread each, straight from global memory
    const int64_t tail0 = nchunk * kGsPx;
    if (blockIdx.x == gridDim.x - 1 && tail0 + tid < a.P) gmm_pixels<KR, KD, 1>(a, tail0 + tid);
}

template <int KR, int KD, int PX>
LaunchResult launch_k(const GmmArgs& a, cudaStream_t s)
{
    const int tpb = (a.tpb == 64 || a.tpb == 256) ? a.tpb : 128;
    const int64_t threads = (a.P + PX - 1) / PX;
    const int64_t blocks = (threads + tpb - 1) / tpb;
    gmm_kernel<KR, KD, PX><<<dim3(unsigned(blocks)), tpb, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

}  // namespace

// Pixels per thread: the requested px for the 3+3 model; mixtures with more
// components keep fewer pixels per thread so the state stays in registers.
// The bulk-copy kernel for frames >= 1 of the 3+3 model: depth of the colour
// frame's size and 16-byte aligned frame buffers (every copy starts on a
// 16-byte boundary).  As many blocks as fit per SM, one chunk each at a time.
LaunchResult launch_gmm_stream(const GmmArgs& a, cudaStream_t s)
{
    using St = GsStage<3, 3>;
    auto k = gmm_stream_kernel<3, 3>;
    constexpr int smem = kGsStages * int(sizeof(St));
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kGsPx, smem) != cudaSuccess || per_sm < 1)
            return kLaunchCudaError;
    }
    const int64_t chunks = a.P / kGsPx;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(chunks, int64_t(per_sm) * sms)));
    k<<<grid, kGsPx, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

bool gmm_stream_ok(const GmmArgs& a, int Kr, int Kd)
{
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return a.stream && !a.init && Kr == 3 && Kd == 3 && a.Wd == a.W && a.Hd == a.H && a.err && al(a.rgb) &&
           al(a.depth) && al(a.mask) && al(a.state);
}

LaunchResult launch_gmm(const GmmArgs& a, int Kr, int Kd, cudaStream_t s)
{
    if (a.P == 0) return kLaunchOk;
    if (gmm_stream_ok(a, Kr, Kd)) return launch_gmm_stream(a, s);
    if (Kr == 3 && Kd == 3) {
        if (a.px == 1) return launch_k<3, 3, 1>(a, s);
        if (a.px == 2) {
            if (a.init || a.Wd != a.W || a.Hd != a.H) return launch_k<3, 3, 2>(a, s);
            const int64_t blocks = ((a.P + 1) / 2 + 255) / 256;
            gmm_pair_kernel<3, 3, 2><<<dim3(unsigned(blocks)), 256, 0, s>>>(a);
            return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
        }
        return launch_k<3, 3, 4>(a, s);
    }
#define FOS_CASE(R, D, PX) \
    if (Kr == R && Kd == D) return launch_k<R, D, PX>(a, s);
    FOS_CASE(7, 3, 2) FOS_CASE(5, 3, 2) FOS_CASE(2, 2, 4) FOS_CASE(1, 1, 4)
    FOS_CASE(2, 1, 4) FOS_CASE(3, 1, 4) FOS_CASE(3, 2, 4) FOS_CASE(5, 2, 2) FOS_CASE(7, 2, 2)
    FOS_CASE(1, 2, 4) FOS_CASE(1, 3, 4) FOS_CASE(2, 3, 4) FOS_CASE(5, 1, 2) FOS_CASE(7, 1, 2)
#undef FOS_CASE
    return kLaunchUnsupported;
}

// Pixels per thread of the batched launch: the kernel keeps the per-stream
// arguments in registers, so the 3+3 model runs 1 or 2 pixels per thread
// (px option, default 2) and larger mixtures one pixel per thread.
int gmm_batch_px(int Kr, int Kd, int px)
{
    if (Kr == 3 && Kd == 3) return px == 1 ? 1 : 2;
    return 1;
}

#define FOS_GMM_BATCH_CASES(X)                                                        \
    X(3, 3, 2) X(3, 3, 1) X(7, 3, 1) X(5, 3, 1) X(2, 2, 1) X(1, 1, 1) X(2, 1, 1)        \
    X(3, 1, 1) X(3, 2, 1) X(5, 2, 1) X(7, 2, 1) X(1, 2, 1) X(1, 3, 1) X(2, 3, 1)        \
    X(5, 1, 1) X(7, 1, 1)

LaunchResult launch_gmm_batch(const GmmBatchTable& t, int blocks, int Kr, int Kd, int px, cudaStream_t s)
{
    const int p = gmm_batch_px(Kr, Kd, px);
#define FOS_B(R, D, PX)                                                                    \
    if (Kr == R && Kd == D && p == PX) {                                                   \
        gmm_batch_kernel<R, D, PX><<<blocks, kGmmBatchThreads, 0, s>>>(t);                 \
        return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;           \
    }
    FOS_GMM_BATCH_CASES(FOS_B)
#undef FOS_B
    return kLaunchUnsupported;
}

#undef FOS_GMM_BATCH_CASES

namespace {

// Many frames of one stream in one launch (the frames already in device
// memory): every pixel's mixtures stay in registers across the frames, so
// the state is read and written once per launch instead of once per frame
// and each frame costs only its 5 input bytes and 1 mask byte per pixel.
// The per-pixel arithmetic is gmm_pixel's, so the results are the bits of
// frame-by-frame processing.  The next frame's inputs are loaded while the
// current one is processed.
constexpr int kFramesThreads = 128;

template <int KR, int KD>
__global__ void __launch_bounds__(kFramesThreads) gmm_frames_kernel(const GmmArgs a, int n)
{
    const int64_t p = int64_t(blockIdx.x) * kFramesThreads + threadIdx.x;
    if (p >= a.P) return;
    Mix<KR, 3> mr[1];
    Mix<KD, 1> md[1];
    const int64_t ne = int64_t(5 * KR + 3 * KD) * a.plane;  // state extent (range-checked builds)
    if (!a.init) move_state<KR, KD, 1, false>(a.state, a.plane, p, mr, md, ne, a.oob);
    GmmArgs b = a;
    // the pixel's depth reading (the same index in every frame) and the depth frame stride
    const int y = int(uint32_t(p) / uint32_t(a.W)), x = int(p) - y * a.W;
    const int64_t pd = depth_index(x, y, a.W, a.H, a.Wd, a.Hd), Pd = int64_t(a.Wd) * a.Hd;
    const int64_t nrgb = 3 * a.P * n, nd = Pd * n, nm = a.P * n;
    uint32_t r = at(a.rgb, 3 * p, nrgb, 51, a.oob), g = at(a.rgb, 3 * p + 1, nrgb, 51, a.oob);
    uint32_t bl = at(a.rgb, 3 * p + 2, nrgb, 51, a.oob), d = at(a.depth, pd, nd, 52, a.oob);
    for (int f = 0; f < n; ++f) {
        uint32_t r1 = 0, g1 = 0, b1 = 0, d1 = 0;
        if (f + 1 < n) {
            const int64_t q = int64_t(f + 1) * a.P + p;
            r1 = at(a.rgb, 3 * q, nrgb, 51, a.oob);
            g1 = at(a.rgb, 3 * q + 1, nrgb, 51, a.oob);
            b1 = at(a.rgb, 3 * q + 2, nrgb, 51, a.oob);
            d1 = at(a.depth, int64_t(f + 1) * Pd + pd, nd, 52, a.oob);
        }
        b.init = (f == 0) ? a.init : 0;
        at(a.mask, int64_t(f) * a.P + p, nm, 53, a.oob) = gmm_pixel<KR, KD>(mr[0], md[0], r, g, bl, d, b);
        r = r1; g = g1; bl = b1; d = d1;
    }
    move_state<KR, KD, 1, true>(a.state, a.plane, p, mr, md, ne, a.oob);
}

}  // namespace

bool gmm_frames_supported(int Kr, int Kd) { return (Kr == 3 && Kd == 3) || (Kr == 7 && Kd == 3); }

LaunchResult launch_gmm_frames(const GmmArgs& a, int n, int Kr, int Kd, cudaStream_t s)
{
    if (a.P == 0 || n <= 0) return kLaunchOk;
    const unsigned blocks = unsigned((a.P + kFramesThreads - 1) / kFramesThreads);
    if (Kr == 3 && Kd == 3) gmm_frames_kernel<3, 3><<<blocks, kFramesThreads, 0, s>>>(a, n);
    else if (Kr == 7 && Kd == 3) gmm_frames_kernel<7, 3><<<blocks, kFramesThreads, 0, s>>>(a, n);
    else return kLaunchUnsupported;
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

}  // namespace fos
