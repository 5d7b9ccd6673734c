// fos_internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/fos.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

struct fos_batch;
struct fos_ctx;

namespace fos {

// Launch status of an internal launcher.
enum LaunchResult { kLaunchOk = 0, kLaunchUnsupported = 1, kLaunchCudaError = 2 };

// Range-checked builds.  Compiled with -DFOS_DEBUG_BOUNDS (libfos_bounds.so),
// every global and shared-memory index of the GMM and PBAS kernels is checked
// against the extent of its buffer before the access.  A violation is counted
// in the context's OobWord (the first one's site and index are kept) and the
// access goes to a scratch sink instead, so the kernel neither faults nor
// traps; fos_bounds_status reads the word back.  In release builds at()
// and vat() are plain indexing.
struct OobWord {
    unsigned int count;  // violations since the last read
    unsigned int site;   // site code of the first one
    long long index;     // its index (elements) or, for a vector access, its start
};

#ifdef FOS_DEBUG_BOUNDS
__device__ __align__(16) static unsigned long long g_oob_sink[2];
__device__ __forceinline__ void oob_record(OobWord* w, int site, int64_t i)
{
    if (w && atomicAdd(&w->count, 1u) == 0u) {
        w->site = unsigned(site);
        w->index = i;
    }
}
template <class T>
__device__ __forceinline__ T& at(T* base, int64_t i, int64_t n, int site, OobWord* w)
{
    if (i >= 0 && i < n) return base[i];
    oob_record(w, site, i);
    return *reinterpret_cast<T*>(g_oob_sink);
}
// element i..i+width-1 of base as one vector V (also checks V's alignment)
template <class V, class T>
__device__ __forceinline__ V& vat(T* base, int64_t i, int width, int64_t n, int site, OobWord* w)
{
    V* p = reinterpret_cast<V*>(base + i);
    if (i >= 0 && i + width <= n && (reinterpret_cast<uintptr_t>(p) % sizeof(V)) == 0) return *p;
    oob_record(w, site, i);
    return *reinterpret_cast<V*>(g_oob_sink);
}
#else
template <class T>
__device__ __forceinline__ T& at(T* base, int64_t i, int64_t, int, OobWord*)
{
    return base[i];
}
template <class V, class T>
__device__ __forceinline__ V& vat(T* base, int64_t i, int, int64_t, int, OobWord*)
{
    return *reinterpret_cast<V*>(base + i);
}
#endif

// Index of the depth reading used for colour pixel (x, y) of a W x H frame
// when depth frames are Wd x Hd: the same pixel at equal sizes, else the
// nearest-neighbour source with floor mapping (Sec. 4.3; the resampling that
// fos_depth_resample_device performs as a separate pass).
__host__ __device__ inline int64_t depth_index(int x, int y, int W, int H, int Wd, int Hd)
{
    if (Wd == W && Hd == H) return int64_t(y) * W + x;
    // sizes up to 16384: the products stay below 2^28, 32-bit arithmetic
    return int64_t(uint32_t(y * Hd) / uint32_t(H)) * Wd + int64_t(uint32_t(x * Wd) / uint32_t(W));
}

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
    int px;             // pixels per thread: 1, 2 or 4
    int tpb;            // threads per block: 64, 128 or 256
    int W, H, Wd, Hd;   // colour frame; depth frame (resampled on read when it differs)
    OobWord* oob;       // range-checked builds: the context's violation record
    int stream;         // 1: frames >= 1 of the 3+3 model through the bulk-copy kernel
    int* err;           // set to 1 by the bulk-copy kernel if a bounded wait gave up
};

LaunchResult launch_gmm(const GmmArgs& a, int Kr, int Kd, cudaStream_t s);
// n consecutive frames (rgb, depth, mask of frame f at f * P) in one launch,
// the mixtures held in registers across the frames; same bits as n launches.
bool gmm_frames_supported(int Kr, int Kd);
LaunchResult launch_gmm_frames(const GmmArgs& a, int n, int Kr, int Kd, cudaStream_t s);

// The paper-literal GMM (FP64, per-channel variances, density-product
// decision); plane layout with the kernel in gmm_literal.cu.
struct GmmLiteralArgs {
    int64_t P, plane;
    double* state;          // gmm_literal_planes(Kr, Kd) * plane doubles
    const uint8_t* rgb;
    const uint16_t* depth;
    uint8_t* mask;
    double alpha, lam2, T_bg, v_init_rgb, v_init_d, v_min_rgb, v_min_d, s, theta;
    uint32_t depth_fs;
    int init;
    int W, H, Wd, Hd;       // colour frame; depth frame (resampled on read when it differs)
};
int gmm_literal_planes(int Kr, int Kd);
bool gmm_literal_supported(int Kr, int Kd);
LaunchResult launch_gmm_literal(const GmmLiteralArgs& a, int Kr, int Kd, cudaStream_t s);

// Streams per batched launch: the argument table of a launch travels as a
// __grid_constant__ kernel parameter (below the 32 KB parameter limit), so
// the kernels read every stream's arguments from the constant bank with
// block-uniform indexed loads and nothing is staged through device memory.
// A step with more streams takes several launches.
constexpr int kBatchLaunchMax = 48;

// One stream of a batched GMM launch.
struct GmmBatchEntry {
    GmmArgs a;
    int block_off;  // first block of this stream in the launch
    int pad[3];
};
struct GmmBatchTable {
    int n, total;  // entries, blocks of kGmmBatchThreads threads
    int pad[2];
    GmmBatchEntry e[kBatchLaunchMax];
};
// Batched GMM launch over t.n entries and t.total blocks of kGmmBatchThreads
// threads (`blocks` >= t.total); every stream uses the same (Kr, Kd) and
// pixels per thread.
constexpr int kGmmBatchThreads = 128;
LaunchResult launch_gmm_batch(const GmmBatchTable& t, int blocks, int Kr, int Kd, int px, cudaStream_t s);
int gmm_batch_px(int Kr, int Kd, int px);

// PBAS device state.  Frames are cut into row segments of kSeg = 128 pixels
// (spr = ceil(W / 128) segments per row, nseg = H * spr).  Samples and D are
// uint16 in a blocked layout: element (c, k, x, y) sits at
//   ((c * nseg + y * spr + x / 128) * N + k) * 128 + x % 128,
// so the N slots of one channel of one segment are 256-byte rows of one
// contiguous block: a warp reads each slot with one coalesced 256-byte access
// and its random own/neighbour slot writes land in the block it just read.
// R, T, S (per channel), prev and the request words are planes with row pitch
// Wp = spr * 128; plane stride `plane` = Wp * H.
// Request word of a pixel: byte c = (direction << 5) | slot for channel c, or
// 0x1F for no request.  prev holds, per pixel, 16 bits (value | gradient << 8)
// for each channel c at bit 16c, of the last processed frame (the value the
// neighbour requests write).
constexpr int kSeg = 128;
constexpr uint32_t kReqNone4 = 0x1F1F1F1Fu;

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
    uint64_t* prev;                 // [pplane] 4 x (value | gradient << 8) of frame t-1
    const uint32_t* req_prev;       // requests of frame t-1 (read)
    uint32_t* req_cur;              // requests of frame t (written)
    unsigned long long* gsum_prev;  // [4] gradient sums of frame t-1
    unsigned long long* gsum_cur;   // [4] accumulated for frame t (zero on entry)
    unsigned long long* gsum_next;  // [4] zeroed for frame t+1
    unsigned long long* counters;   // [3] own updates, neighbour writes, requests
    float R_lower_rgb, R_lower_d, R_scale, R_incdec;
    float T_lower, T_upper, T_inc, T_dec, alpha_g, eps_d;
    int N, n_min;
    uint32_t seed, stream_id;
    int forced;
    uint32_t depth_fs;
    uint32_t t;    // frame index
    int apply;     // 1: requests of frame t-1 are pending
    int px, ty;    // tile shape: pixels per thread (used when W % px == 0), rows
    int mask_vec;  // mask pointer aligned for PX-wide stores
    int Wd, Hd;    // depth frame size (resampled on staging when it differs from W x H)
    int propagate;               // 1: a neighbour update writes the requester's value
    const uint64_t* prev_src;    // values of frame t-1 the pending requests write: the
                                 // requesters' (propagate; a second plane) or prev itself
    uint32_t* own;               // [plane] propagate only: byte c = slot of the pixel's own
                                 // update in channel c of the last frame (0x1F none)
    OobWord* oob;                // range-checked builds: the context's violation record
    uint32_t rk[20];             // Philox round keys of (seed, stream_id) (pbas_args_finish)
    uint32_t depth_m;            // depth rescale: floor(x / depth_fs) = (x * depth_m) >> depth_sh
    int depth_sh;                //   (pbas_args_finish)
};

// floor(x / fs) = (x * m) >> sh for every 0 <= x < 2^25 and 1 <= fs <= 2^18:
// the round-up multiplier of Granlund and Montgomery ("Division by invariant
// integers using multiplication", PLDI 1994): with l = ceil(log2 fs),
// sh = 25 + l and m = ceil(2^sh / fs), m fs lies in [2^sh, 2^sh + 2^l], which
// makes the quotient exact for 25-bit x; m < 2^26 + 1 and x m < 2^51.  The
// depth rescale's numerator d * 255 + fs / 2 stays below 2^25 for 16-bit d.
inline void depth_divisor(uint32_t fs, uint32_t& m, int& sh)
{
    int l = 0;
    while ((uint64_t(1) << l) < uint64_t(fs)) ++l;
    sh = 25 + l;
    m = uint32_t(((uint64_t(1) << sh) + fs - 1) / fs);
}

// The fields of a PbasArgs derived from others: the Philox round keys of
// (seed, stream_id) and the depth rescale's multiplier (depth_fs >= 1).
void pbas_args_finish(PbasArgs& a);

// Extents (elements) of the PBAS buffers, for the range-checked build.
__host__ __device__ inline int64_t samp_extent(const PbasArgs& a) { return 4 * a.nseg * a.N * kSeg; }
__host__ __device__ inline int64_t rts_extent(const PbasArgs& a) { return 4 * a.plane; }
__host__ __device__ inline int64_t depth_extent(const PbasArgs& a) { return int64_t(a.Wd) * a.Hd; }

// Frames t0 .. t0+n-1 (t0 = a0.t >= 1) of one fused (3+3 GMM + PBAS) context
// in one persistent launch.  Tiles are claimed in frame-major order from a
// counter; a tile of frame t0+i (i >= 1) starts once its 3x3 neighbourhood of
// tiles has finished frame t0+i-1 (per-tile completion words), so the next
// frame's tiles fill the SMs that the end of the previous frame leaves idle.
// Every cross-tile read of a tile is of the input (read-only), of the request
// planes of frame t-1 or, with propagation, of the value planes of frame t-1
// (both double-buffered by frame parity): the 3x3 dependency covers them.
// The gradient sums that weight frame t0+i come from a pre-pass (gprev).
struct SeqArgs {
    int n;                             // frames in the launch
    int tiles_x, tiles_y;              // tile grid of one frame
    int64_t rgb_stride;                // bytes between frames
    int64_t depth_stride;              // elements between frames
    int64_t mask_stride;               // bytes between frames (both masks)
    uint32_t* req_base;                // [2][plane] request planes by frame parity
    uint64_t* prev_base;               // propagation: [2][plane] value planes by frame parity
    const unsigned long long* gprev;   // [n][4] gradient sums of frame t0+i-1, weighting frame t0+i
    unsigned long long* gscratch;      // [8] sink for the tiles' own gradient sums
    unsigned int* claim;               // tile counter, zero on entry
    int* done;                         // [tiles] frames of this launch each tile has finished, zero on entry
    int* err;                          // set to 1 if a bounded wait gave up
};
LaunchResult launch_fused_sequence(const PbasArgs& a0, const GmmArgs& g0, const SeqArgs& q, cudaStream_t s);
// The tile grid launch_fused_sequence expects for this context's shape options.
void fused_sequence_tiles(const PbasArgs& a, int& tiles_x, int& tiles_y);
// Gradient sums (R, G, B, depth; the Sobel magnitudes the classify pass
// computes) of the n frames at a0's input pointers with q's strides into
// out[n][4] (zero on entry).
LaunchResult launch_grad_sums(const PbasArgs& a0, const SeqArgs& q, unsigned long long* out, cudaStream_t s);

// Several frames of many fused streams in one persistent launch: the
// sequence launch above generalised over the streams of a batch.  Entries are
// sorted by frame count, descending, so that at frame slot i the streams with
// more than i frames are entries 0 .. m_i-1; the claim order is slot-major,
// then entry, then tile, and a tile waits for its own stream's 3x3 tiles of
// the previous slot.
struct SeqBatchEntry {
    PbasArgs a;                        // frame t0 of the stream
    int n;                             // frames
    int tiles_x, tiles_y;              // tile grid (sequence tile shape)
    int tile_off;                      // first tile of the stream within a slot
    int gtile_off;                     // first 32 x kGradStripRows strip of the stream in the gradient pre-pass
    int pad[3];
    int64_t rgb_stride, depth_stride, mask_stride;
    uint32_t* req_base;
    uint64_t* prev_base;
    unsigned long long* gprev;         // [n + 1][4]: frame t0-1 (copied from gsum_src), then frames t0 .. t0+n-1
    const unsigned long long* gsum_src;  // the context's sums of frame t0-1
    unsigned long long* gsum_last;     // where the context keeps frame t0+n-1's sums
    unsigned long long* gsum_zero;     // the context's accumulator of frame t0+n (zeroed)
    int* done;                         // [tiles]
};
constexpr int kSeqBatchMax = 48;
constexpr int kGradStripRows = 64;  // rows of one block of the gradient pre-pass (32 pixels wide)
struct SeqBatchTable {
    int n;                             // entries (sorted by n, descending)
    int segs;                          // runs of slots with the same active entries
    int gtiles;                        // pre-pass tiles of all entries
    int maxn;                          // frames of entry 0
    // run r: slots [seg_slot0[r], seg_slot0[r+1]) with entries 0 .. seg_m[r]-1
    // active (seg_tiles[r] tiles per slot), claims from seg_claim0[r]
    int seg_slot0[kSeqBatchMax + 1];
    int seg_m[kSeqBatchMax];
    int seg_tiles[kSeqBatchMax];
    long long seg_claim0[kSeqBatchMax + 1];
    unsigned int* claim;
    int* err;
    unsigned long long* gscratch;      // [8]
    int* done_all;                     // every entry's completion words
    int done_words;
    int pad;
    SeqBatchEntry e[kSeqBatchMax];
    GmmArgs g[kSeqBatchMax];
};
// Zero the counter and completion words, gradient sums set up, pre-pass,
// the persistent launch, and the sums left where per-frame launches expect
// them; all on stream s.
LaunchResult launch_batch_sequence(const SeqBatchTable& t, int px, int ty, cudaStream_t s);

LaunchResult launch_pbas_init(const PbasArgs& a, cudaStream_t s);
LaunchResult launch_pbas_classify(const PbasArgs& a, cudaStream_t s);
LaunchResult launch_pbas_flush(const PbasArgs& a, cudaStream_t s);
// Joint-channel variant of the classify pass (pbas_joint.cu).
LaunchResult launch_pbas_joint(const PbasArgs& a, cudaStream_t s);

// GMM (3+3 components) and PBAS of one frame in one launch (frames >= 1).
LaunchResult launch_fused_classify(const PbasArgs& a, const GmmArgs& g, cudaStream_t s);

// One stream of a batched launch (one entry per stream).
struct PbasBatchEntry {
    PbasArgs a;
    int tile_off;  // first tile of this stream in the launch
    int tiles_x;   // tiles per row
    int init;      // 1: frame 0 of this stream
    int pad;
};
struct PbasBatchTable {
    int n, total;  // entries, tiles
    int pad[2];
    PbasBatchEntry e[kBatchLaunchMax];
    GmmArgs g[kBatchLaunchMax];  // fused launches: the GMM arguments of entry i
};
// Batched PBAS launch over t.n entries and t.total tiles, one block per tile
// (`blocks` >= t.total).  fused (3+3-component GMM): each tile also runs the
// GMM of its pixels.
LaunchResult launch_pbas_batch(const PbasBatchTable& t, bool fused, int blocks, int N, int px, int ty,
                               cudaStream_t s);

// Depth frame sw x sh resampled onto dw x dh (nearest, floor mapping).
LaunchResult launch_depth_resample(const uint16_t* src, int sw, int sh, uint16_t* dst, int dw, int dh,
                                   cudaStream_t s);

// NVTX range over a host call (frame steps, batch ticks, server ticks, the
// soft-GMM passes), visible on the timeline of a profiler that collects
// NVTX; costs nothing without one.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device allocation of the library's long-lived buffers.  The environment
// variable FOS_FAIL_ALLOC_AFTER=n makes every allocation after the first n
// of the process fail with cudaErrorMemoryAllocation (host-side fault
// injection for the error-path tests; unset, it is cudaMalloc).
cudaError_t dev_alloc(void** p, size_t bytes);

// Sets the text fos_last_error(NULL) returns on the calling thread.
void set_thread_error(const char* msg);

// Puts an existing context (same parameters as the batch) into a free slot of
// the batch without allocating; returns the slot, or -1 if none is free.
int32_t batch_attach(fos_batch* b, fos_ctx* c);
// Takes the context out of the slot without freeing it (NULL if empty).  The
// caller guarantees that no step still in flight uses it.
fos_ctx* batch_detach(fos_batch* b, int32_t slot);

}  // namespace fos
