/*
 * fos.h -- C ABI of the GB300 (sm_103a) RGB-D foreground segmentation library.
 *
 * Foreground object segmentation in RGB-D video with two per-pixel background
 * models (Janus, Kryjak, Gorgon, "Foreground object segmentation in RGB-D data
 * implemented on GPU"):
 *   GMM   Sec. 3.1 (Eq. 1): two separate Gaussian mixtures per pixel, one over
 *         colour and one over depth; the depth model is used only where the
 *         depth reading is valid (> 0); the two results are combined.
 *   PBAS  Sec. 3.2: N background samples per pixel, each holding R, G, B and
 *         depth, every channel processed separately with its own adaptive
 *         decision threshold R(x), learning parameter T(x) and minimal-distance
 *         record D(x); random update of the pixel's own and its neighbours'
 *         samples; depth used only where valid.
 *   Depth is rescaled from 16 to 8 bits as Sec. 4.2 describes.  The host owns
 *   acquisition and copies frames to the GPU; the GPU classifies every pixel
 *   in parallel and returns a binary mask (Sec. 4.2, "Application architecture").
 *
 * Conventions for every entry point:
 *   - Frames are row-major.  rgb: H*W*3 bytes, interleaved R,G,B.  depth: H*W
 *     uint16 millimetres, 0 = invalid.  masks: H*W bytes, 0 = background,
 *     255 = foreground.
 *   - "host" pointers are ordinary (pageable or pinned) CPU memory; "device"
 *     pointers are CUDA global memory of the current device.  The caller owns
 *     every frame buffer; the library does not keep a pointer after returning.
 *   - A context owns its device state and is not thread-safe: one thread (and
 *     one stream at a time) per context.
 *   - Errors never abort.  Each call returns a fos_status; the text of the last
 *     error is available from fos_last_error().  CUDA errors map to
 *     FOS_ERR_CUDA.  A sticky CUDA error leaves the context unusable.
 *   - The first frame a context processes (frame 0) initialises the models;
 *     its masks are all background.
 */
#ifndef FOS_H
#define FOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FOS_ABI_VERSION 1

/* Method selection bits (fos_params.methods). */
#define FOS_METHOD_GMM 1u  /* Sec. 3.1 */
#define FOS_METHOD_PBAS 2u /* Sec. 3.2 */

typedef enum fos_status {
    FOS_OK = 0,
    FOS_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or parameter */
    FOS_ERR_CUDA = 2,        /* a CUDA call failed; see fos_last_error */
    FOS_ERR_OOM = 3,         /* device or pinned host allocation failed */
    FOS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    FOS_ERR_BUDGET = 5,      /* admission refused: memory budget exceeded */
    FOS_ERR_STATE = 6,       /* call not valid in the context's current state */
    FOS_ERR_UNSUPPORTED = 7, /* parameter combination not compiled in */
    FOS_ERR_BUSY = 8         /* queue full: the call took nothing, retry later */
} fos_status;

/*
 * Parameters.  fos_default_params() fills the values the library is tuned and
 * tested with; the paper fixes N = 20 (Sec. 3.2) and alpha = 0.001 (Sec. 3.1);
 * the other constants follow the cited base methods (Stauffer-Grimson GMM,
 * Hofmann PBAS) or are readings of the paper documented with the library.
 */
typedef struct fos_params {
    uint32_t methods;          /* FOS_METHOD_GMM | FOS_METHOD_PBAS */
    /* ---- GMM (Sec. 3.1) ---- */
    int32_t K_rgb;             /* components of the colour model: 1,2,3,5,7 */
    int32_t K_d;               /* components of the depth model: 1,2,3 */
    float alpha;               /* learning rate (paper: 0.001) */
    float lambda;              /* match threshold on the Mahalanobis distance */
    float w_depth;             /* weight of the depth model in the combined score */
    float T_bg;                /* background weight fraction */
    float v_init_rgb, v_init_d;/* variance of a new component */
    float v_min_rgb, v_min_d;  /* variance floor */
    /* ---- PBAS (Sec. 3.2) ---- */
    int32_t N;                 /* samples per pixel, 1..31 (paper: 20) */
    int32_t n_min;             /* matches needed for background */
    float R_lower_rgb, R_lower_d, R_scale, R_incdec;
    float T_lower, T_upper, T_inc, T_dec;
    float alpha_g;             /* gradient weight numerator */
    float eps_d;               /* floor of the mean minimal distance */
    uint32_t seed;             /* Philox4x32-10 key word 0 */
    uint32_t stream_id;        /* Philox4x32-10 key word 1 (camera stream) */
    int32_t forced_rng;        /* 0: Philox; 1..3: deterministic test draws (every coin fires,
                                  own slot t mod N, neighbour slot (t+1) mod N; direction t mod 8;
                                  with 2 east from columns 0,1 mod 4 and west from 2,3; with 3
                                  north from even columns, south-east from odd ones, and pixels
                                  of even rows ask for slot t mod N) */
    /* ---- input conversion (Sec. 4.2) ---- */
    uint32_t depth_full_scale_mm; /* depth mapped onto 1..255, 0 = invalid */
    /* ---- GMM as the paper prints it (Sec. 3.1, Eq. 1) ---- */
    int32_t gmm_literal;       /* 1: FP64 state, one variance per colour channel, decision on the
                                  product of the s-scaled Eq. 1 densities (K = 7+3 or 3+3);
                                  0: the FP32 isotropic model with the distance score */
    float density_scale;       /* s (paper: 10000) */
    float density_threshold;   /* background iff the product of the factors >= this */
    /* ---- PBAS neighbour update variant ---- */
    int32_t pbas_propagate;    /* 0: a chosen neighbour takes its own value (the base method);
                                  1: it takes the updating pixel's value (spatial propagation,
                                  as in ViBe); a slot the neighbour's own update of the same
                                  frame wrote keeps that value, and among requests for one
                                  slot the requester at the lowest direction index seen from
                                  the neighbour (N, NE, E, SE, S, SW, W, NW) wins */
    /* ---- PBAS channel coupling variant ---- */
    int32_t pbas_joint;        /* 0: every channel has its own R, T, D and decision, foreground
                                  if any channel is (the base method); 1: one R, T, D per pixel
                                  and one decision on the mean of the per-channel distances
                                  over the active channels (R, G, B, and depth where valid),
                                  computed as their FP32 sum in channel order times fl(1/n);
                                  one draw per pixel; updates write whole samples; R, T, S
                                  and D are kept in channel 0's entries of the state, the
                                  other channels' entries keep their bootstrap values.
                                  Not available in batches or the no-alloc entry point. */
} fos_params;

typedef struct fos_ctx fos_ctx;

/* Fills *p with the defaults (both methods enabled). NULL-safe. */
void fos_default_params(fos_params* p);

/* ABI version of the loaded library (FOS_ABI_VERSION it was built with). */
int32_t fos_abi_version(void);

/*
 * Creates a context for width x height frames (1..16384 each) and allocates
 * its device state on the current CUDA device.  Returns NULL on error; the
 * reason is then available from fos_last_error(NULL) on the calling thread.
 */
fos_ctx* fos_create(int32_t width, int32_t height, const fos_params* params);

/*
 * Like fos_create, for a sensor whose depth frames are depth_width x
 * depth_height (1..16384 each) while colour frames are width x height
 * (Sec. 4.3: processing runs at the colour resolution).  Every depth frame
 * passed to this context has the depth size (a frame batch is
 * n * depth_width * depth_height values); the kernels read each colour
 * pixel's depth through the nearest-neighbour map of fos_depth_resample_device
 * while they stage their input (no separate pass, no extra buffer).  With
 * equal sizes this is fos_create.  The batch and serving APIs take equal
 * sizes only.
 */
fos_ctx* fos_create_rgbd(int32_t width, int32_t height, int32_t depth_width, int32_t depth_height,
                         const fos_params* params);

/*
 * Depth frame d_src (src_width x src_height uint16, device) resampled onto
 * d_dst (dst_width x dst_height uint16, device), nearest neighbour:
 * dst(x, y) = src(floor(x * src_width / dst_width),
 * floor(y * src_height / dst_height)); every output is an input value, so
 * the invalid reading 0 is never blended into a valid depth (Sec. 4.3 brings
 * depth to the colour resolution without saying how).  Sizes 1..16384.
 * Asynchronous on `stream` (cudaStream_t; NULL = legacy default stream).
 * FOS_ERR_INVALID_ARG on NULL pointers or sizes out of range, FOS_ERR_CUDA if
 * the launch fails (text in fos_last_error(NULL)).  Allocates nothing.
 */
fos_status fos_depth_resample_device(const uint16_t* d_src, int32_t src_width, int32_t src_height,
                                     uint16_t* d_dst, int32_t dst_width, int32_t dst_height, void* stream);

/* Frees the context and its device memory.  NULL-safe. */
void fos_destroy(fos_ctx* ctx);

/* Text of the context's last error ("" if none); ctx == NULL gives the calling
 * thread's last fos_create or fos_pbas_step_noalloc error.  The pointer stays valid until the next call
 * on the same context / thread. */
const char* fos_last_error(const fos_ctx* ctx);

/* Status of the context's last failed call (FOS_OK if none); ctx == NULL
 * gives the status of the calling thread's last failed fos_create /
 * fos_create_rgbd (for example FOS_ERR_OOM when device memory ran out, which
 * the NULL return alone does not tell). */
fos_status fos_last_status(const fos_ctx* ctx);

/* Restarts the sequence: the next processed frame is frame 0 again. */
fos_status fos_reset(fos_ctx* ctx);

/* Number of frames processed since creation or the last reset. */
int64_t fos_frame_index(const fos_ctx* ctx);

/*
 * One frame from HOST memory, synchronous: copies rgb and depth to the
 * device, runs the enabled methods, copies the mask back and waits.
 * mask_out receives the GMM mask when GMM is enabled, else the PBAS mask.
 */
fos_status fos_process_frame(fos_ctx* ctx, const uint8_t* rgb, const uint16_t* depth,
                             uint8_t* mask_out);

/* As fos_process_frame, returning both masks (either may be NULL if its
 * method is disabled). */
fos_status fos_process_frame2(fos_ctx* ctx, const uint8_t* rgb, const uint16_t* depth,
                              uint8_t* mask_gmm, uint8_t* mask_pbas);

/*
 * One frame from DEVICE memory, asynchronous on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  mask_gmm / mask_pbas must be non-NULL for
 * each enabled method.  Any alignment is accepted; 16-byte aligned buffers
 * whose width is a multiple of 4 take the vectorised kernels.
 */
fos_status fos_process_frame_device(fos_ctx* ctx, const uint8_t* d_rgb, const uint16_t* d_depth,
                                    uint8_t* d_mask_gmm, uint8_t* d_mask_pbas, void* stream);

/*
 * n_frames consecutive frames from DEVICE memory, asynchronous on `stream`.
 * Frame f starts at d_rgb + f*H*W*3, d_depth + f*H*W, and writes its masks at
 * d_mask_gmm + f*H*W, d_mask_pbas + f*H*W.
 */
fos_status fos_process_frames_device(fos_ctx* ctx, int32_t n_frames, const uint8_t* d_rgb,
                                     const uint16_t* d_depth, uint8_t* d_mask_gmm,
                                     uint8_t* d_mask_pbas, void* stream);

/*
 * n_frames consecutive frames from HOST memory (same strides as above),
 * pipelined in chunks of up to 16 frames on three streams: the input copy of
 * chunk g+1 and the mask copy of chunk g-1 overlap the kernels of chunk g.
 * Pinned host buffers give the overlap; pageable ones still work, serialised.
 * The context keeps device staging for two chunks (allocated on first use,
 * grown when a call needs more: about 2 * 16 * 7 bytes per pixel).
 * Synchronous: returns when every mask is in host memory.
 */
fos_status fos_process_frames_host(fos_ctx* ctx, int32_t n_frames, const uint8_t* rgb,
                                   const uint16_t* depth, uint8_t* mask_gmm, uint8_t* mask_pbas);

/* ---------------------------------------------------------------------------
 * Model state export / import (checkpoint, resume, step-by-step testing).
 * Blob layout: fos_state_header, then the GMM section (if enabled), then the
 * PBAS section (if enabled); every plane holds P = W*H values, unpadded.
 *   GMM  (float32): for the colour model with K = K_rgb components, planes
 *        w[k], mu_r[k], mu_g[k], mu_b[k], v[k] (in that order, each k = 0..K-1),
 *        then for the depth model with K = K_d: w[k], mu[k], v[k].
 *        Components are stored in ranked order (k = 0 ranks highest).
 *        With gmm_literal = 1 the section is float64 with one variance per
 *        colour channel: w[k], mu_r[k], mu_g[k], mu_b[k], v_r[k], v_g[k],
 *        v_b[k], then depth w[k], mu[k], v[k] (gmm_bytes tells them apart).
 *   PBAS: samples  uint16 planes [c][k] (c = R,G,B,D; k = 0..N-1), value in the
 *                  low byte, gradient magnitude in the high byte;
 *         D        uint16 planes [c][k]: minimal distance x16 (rounded);
 *         R, T     float32 planes [c];
 *         S        uint32 planes [c]: sum over k of D[c][k];
 *         gsum     uint64[4]: gradient-magnitude sums of the last frame.
 * ------------------------------------------------------------------------- */
typedef struct fos_state_header {
    uint32_t magic;      /* 0x53534F46 ("FOSS") */
    uint32_t abi_version;
    int32_t width, height;
    uint32_t methods;
    int32_t K_rgb, K_d, N;
    int64_t frame_index;
    uint64_t gmm_bytes, pbas_bytes;
} fos_state_header;

/* Size in bytes of the blob fos_get_state writes. */
fos_status fos_state_size(const fos_ctx* ctx, size_t* bytes);
/* Writes the blob into host memory (synchronises the context's work). */
fos_status fos_get_state(fos_ctx* ctx, void* host_buf, size_t bytes);
/* Replaces the device state with a blob from fos_get_state of a context with
 * the same size, methods, K_rgb, K_d and N. */
fos_status fos_set_state(fos_ctx* ctx, const void* host_buf, size_t bytes);

/* ---------------------------------------------------------------------------
 * Measurement hooks.
 * ------------------------------------------------------------------------- */
#define FOS_KERNEL_GMM 0        /* GMM classify + update (Sec. 3.1) */
#define FOS_KERNEL_PBAS_CLASSIFY 1 /* PBAS: the previous frame's neighbour
                                      updates, gradient, classify, own update */
#define FOS_KERNEL_PBAS_FLUSH 2  /* PBAS pending neighbour updates applied
                                    outside a frame (before a state export) */
#define FOS_KERNEL_INIT 3       /* frame-0 initialisation */
#define FOS_KERNEL_FUSED 4      /* GMM and PBAS of a frame in one launch */
#define FOS_KERNEL_FUSED_SEQUENCE 5 /* GMM and PBAS of several frames in one
                                       persistent launch (with the gradient-sum
                                       pre-pass it needs) */
#define FOS_KERNEL_COUNT 6

typedef struct fos_kernel_timing {
    int64_t launches;
    double total_ms;  /* sum of CUDA-event durations on the launch stream */
    int64_t frames;   /* frames those launches processed */
} fos_kernel_timing;

/* Bit k of mask enables CUDA-event timing around every launch of kernel k. */
fos_status fos_set_timing(fos_ctx* ctx, uint32_t kernel_mask);
/* Waits for the timed launches and writes FOS_KERNEL_COUNT entries; then
 * clears the accumulators. */
fos_status fos_get_timing(fos_ctx* ctx, fos_kernel_timing out[FOS_KERNEL_COUNT]);

/* ---------------------------------------------------------------------------
 * Kernel shapes (tuning).  Results do not depend on them: every shape computes
 * the same bits.  Defaults: GMM 4 pixels per thread, 128 threads per block;
 * PBAS 2 pixels per thread (when the width is a multiple of it), 8 rows.
 * ------------------------------------------------------------------------- */
#define FOS_OPT_GMM_PX 1   /* GMM pixels per thread: 1, 2, 4 (3+3 components) */
#define FOS_OPT_GMM_TPB 2  /* GMM threads per block: 64, 128, 256 */
#define FOS_OPT_PBAS_PX 3  /* PBAS pixels per thread: 1, 2, 4 */
#define FOS_OPT_PBAS_TY 4  /* PBAS tile rows: 2, 4, 8 (2 only with 4 px/thread) */
#define FOS_OPT_FUSE 5     /* 1 (default): with both methods and K = 3+3, frames >= 1
                              run GMM and PBAS in one fused launch; 0: two launches */
#define FOS_OPT_TEMPORAL 6 /* 1 (default): fos_process_frames_device with GMM alone (FP32, K = 3+3
                              or 7+3, equal colour/depth size) runs all its frames in one launch,
                              each pixel's mixtures kept in registers; 0: one launch per frame.
                              Same bits either way. */
#define FOS_OPT_SEQUENCE 7 /* 1 (default): fos_process_frames_device / _host with both methods
                              fused (FOS_OPT_FUSE, K = 3+3) run the frames after the first of a
                              call in one persistent launch, in which a tile of frame t+1 starts
                              as soon as the 3x3 tiles around it have finished frame t; 0: one
                              launch per frame.  Same bits either way. */
#define FOS_OPT_GMM_STREAM 8 /* 1 (default): GMM frames >= 1 of the 3+3 model (depth of the colour
                              frame's size, 16-byte aligned frame buffers) through the bulk-copy
                              kernel, which stages 256-pixel chunks of the state planes and inputs
                              in shared memory while the previous chunks compute; 0: the
                              register kernels shaped by FOS_OPT_GMM_PX / _TPB.  Same bits. */
#define FOS_OPT_COUNT 9

/* Sets a kernel-shape option; FOS_ERR_INVALID_ARG for unknown options or
 * values, FOS_ERR_UNSUPPORTED for shapes not compiled in. */
fos_status fos_set_option(fos_ctx* ctx, int32_t option, int32_t value);
/* Current value of an option, -1 for an unknown option or NULL ctx. */
int32_t fos_get_option(const fos_ctx* ctx, int32_t option);

/*
 * PBAS update counters since the last call (then cleared):
 * out[0] own-sample updates, out[1] neighbour-sample writes applied,
 * out[2] neighbour requests issued, out[3] frames.
 */
fos_status fos_get_counters(fos_ctx* ctx, uint64_t out[4]);

/* ---------------------------------------------------------------------------
 * Quality indicators (Sec. 5): confusion counts of foreground masks against
 * ground truth, and the percentage of wrong classifications (PWC), the false
 * negative rate (FNR), the false positive rate (FPR) and the similarity (Si)
 * derived from them.  A byte is foreground when it is non-zero.
 *
 * fos_quality_counts_device: d_mask, d_gt are device arrays of n_pixels bytes
 * (any number of frames laid end to end); the counts TP, TN, FP, FN are ADDED
 * to d_counts[0..3] (device uint64; zero them to start a new total).
 * Asynchronous on `stream` (cudaStream_t; NULL = legacy default stream).
 * FOS_ERR_INVALID_ARG for NULL pointers or n_pixels < 0; FOS_ERR_CUDA if the
 * launch fails (text in fos_last_error(NULL)).  Allocates nothing.
 *
 * fos_quality_metrics: out = {PWC = 100 (FN+FP)/(TP+FN+FP+TN),
 * FNR = FN/(TP+FN), FPR = FP/(FP+TN), Si = TP/(TP+FP+FN)} from host counts
 * (a ratio with a zero denominator is NaN).
 * ------------------------------------------------------------------------- */
fos_status fos_quality_counts_device(const uint8_t* d_mask, const uint8_t* d_gt, int64_t n_pixels,
                                     uint64_t* d_counts, void* stream);
void fos_quality_metrics(const uint64_t counts[4], double out[4]);

/* ---------------------------------------------------------------------------
 * Batched multi-stream processing.  No counterpart in the paper (one stream
 * there); many camera streams share one GPU.
 *
 * A batch owns up to max_streams stream contexts that share every parameter
 * except stream_id.  fos_batch_process_device runs one frame of any subset of
 * them as ONE CUDA graph replay on the caller's stream: a copy of the
 * per-stream kernel arguments, then a persistent GMM kernel and a persistent
 * PBAS kernel that walk all streams' tiles.  Per-stream results are
 * bit-identical to fos_process_frame_device on a lone context.  Streams may
 * join at any time (their first frame is their frame 0) and leave between
 * steps.  A batch is not thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct fos_batch fos_batch;

typedef struct fos_batch_tuning {
    int32_t gmm_px;     /* GMM pixels per thread in the batched kernel (1, 2) */
    int32_t pbas_px;    /* PBAS pixels per thread (1, 2, 4) */
    int32_t pbas_ty;    /* PBAS tile rows (4, 8) */
    float ms_per_step;  /* measured time of one step with that shape */
} fos_batch_tuning;

/* Device memory one stream context of this size holds (its models and
 * scratch planes; frame and mask buffers not included).  0 on bad input. */
size_t fos_stream_device_bytes(int32_t width, int32_t height, const fos_params* params);

/* Creates an empty batch (device argument buffers, pinned host buffers).
 * NULL on error (reason in fos_last_error(NULL)). */
fos_batch* fos_batch_create(int32_t max_streams, const fos_params* params);
/* Destroys the batch and every stream it still holds.  NULL-safe. */
void fos_batch_destroy(fos_batch* b);
/* Last error of the batch ("" if none). */
const char* fos_batch_last_error(const fos_batch* b);
/* Adds a width x height stream with the batch's parameters and this Philox
 * stream id; returns its slot (>= 0), or -1 (batch full: the batch error says
 * so; device memory exhausted: FOS_ERR_OOM text). */
int32_t fos_batch_add_stream(fos_batch* b, int32_t width, int32_t height, uint32_t stream_id);
/* Removes a stream between steps (waits for steps in flight) and frees it. */
fos_status fos_batch_remove_stream(fos_batch* b, int32_t slot);
/* The context of a slot (owned by the batch): for fos_get_state, fos_reset,
 * fos_frame_index.  NULL for an empty slot. */
fos_ctx* fos_batch_stream(fos_batch* b, int32_t slot);
/*
 * One frame of n distinct streams: for i < n, stream slots[i] processes the
 * device frame d_rgb[i], d_depth[i] and writes d_mask_gmm[i] / d_mask_pbas[i]
 * (host arrays of device pointers; mask arrays may be NULL for a disabled
 * method).  Asynchronous on `stream`; the pointer arrays are read before the
 * call returns.
 */
fos_status fos_batch_process_device(fos_batch* b, int32_t n, const int32_t* slots,
                                    const uint8_t* const* d_rgb, const uint16_t* const* d_depth,
                                    uint8_t* const* d_mask_gmm, uint8_t* const* d_mask_pbas,
                                    void* stream);
/*
 * Several frames of n distinct streams: stream slots[i] processes n_frames[i]
 * (>= 0) consecutive device frames, frame k at d_rgb[i] + k*W*H*3,
 * d_depth[i] + k*Wd*Hd, and writes its masks at d_mask_*[i] + k*W*H.  With
 * both methods and the 3+3 GMM (the fused model): the first frame of streams
 * at frame 0 runs as one batched step, then all remaining frames of all
 * streams run in ONE persistent launch (per 48 streams) in which a tile of
 * frame t+1 of a stream starts as soon as that stream's 3x3 tiles around it
 * have finished frame t (a bounded wait; the gradient-weight sums of every
 * frame come from a pre-pass over the inputs).  Otherwise one batched step
 * per frame slot.  Per-stream results are bit-identical to processing each
 * stream alone.  Asynchronous on `stream`; the arrays are read before the
 * call returns.  Errors: FOS_ERR_INVALID_ARG (bad slot, count or pointer;
 * more than 65535 frames of one stream), FOS_ERR_UNSUPPORTED, FOS_ERR_CUDA,
 * FOS_ERR_OOM (its scratch is grown on demand; growing synchronises the device).
 */
fos_status fos_batch_process_frames_device(fos_batch* b, int32_t n, const int32_t* slots, const int32_t* n_frames,
                                           const uint8_t* const* d_rgb, const uint16_t* const* d_depth,
                                           uint8_t* const* d_mask_gmm, uint8_t* const* d_mask_pbas,
                                           void* stream);
/* Waits for the device; FOS_ERR_TIMEOUT if a wait of the last persistent
 * launch of fos_batch_process_frames_device gave up (it cannot while every
 * block is resident, as the cooperative launch guarantees), else FOS_OK. */
fos_status fos_batch_sequence_status(fos_batch* b);
/* Sets the kernel shapes of the batched launch (see fos_batch_tuning). */
fos_status fos_batch_set_shape(fos_batch* b, int32_t gmm_px, int32_t pbas_px, int32_t pbas_ty);
/*
 * Autotuner: times every compiled shape on copies of the listed streams fed
 * the given frames (throwaway contexts; the batch's own models are not
 * touched), picks the fastest and sets it on the batch.  Synchronous;
 * allocates temporary device memory.  `out` (nullable) receives the choice.
 */
fos_status fos_batch_autotune(fos_batch* b, int32_t n, const int32_t* slots,
                              const uint8_t* const* d_rgb, const uint16_t* const* d_depth,
                              void* stream, fos_batch_tuning* out);

/* ---------------------------------------------------------------------------
 * Serving loop with continuous batching.  No counterpart in the paper.
 *
 * A server owns a batch and a worker thread.  Streams (cameras) are admitted
 * by a device-memory budget: each needs fos_server_stream_bytes (its models
 * plus a ring of six device frames of inputs and masks, 6 * 7 bytes per pixel
 * rounded up to 256-byte regions); a stream that does not fit, or finds no
 * free slot, waits in FIFO order until others close.  A housekeeping thread
 * allocates an admitted stream's memory and frees that of streams that left,
 * so the worker's ticks never wait on an allocation or a free.
 * fos_server_submit copies a frame into one of the stream's queue_depth
 * pinned input slots (allocated by its first copying submit) and returns at
 * once.  Each worker tick takes
 * the oldest pending frames of every admitted stream (up to three per stream,
 * in order; frames of one stream run in order), runs them as batched graph
 * steps back to back (one per frame slot), and writes the masks into the
 * caller's buffers given at submit time; three ticks are in flight (the
 * input copies of one, the kernels of another and the mask copies of a third
 * overlap), so frames that arrive while one runs join the next.  Results are identical to
 * processing each stream alone.  All calls are thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct fos_server fos_server;

typedef struct fos_server_result {
    int32_t stream;      /* handle from fos_server_open_stream */
    int32_t status;      /* fos_status of the frame */
    int64_t tag;         /* caller's tag from fos_server_submit */
    double latency_us;   /* submit -> masks written */
    double queue_us;     /* submit -> its tick launched */
} fos_server_result;

typedef struct fos_server_stats_t {
    int64_t ticks, frames_done;
    size_t device_bytes_used;
    int32_t streams_active, streams_waiting;
    double busy_us;      /* sum over ticks of launch -> completion */
    double housekeeping_us;  /* time the housekeeping thread spent allocating
                                and freeing streams' memory */
    double kernel_us;    /* sum over ticks of the batched kernels' device time */
} fos_server_stats_t;

/* Device bytes the server charges against its budget for one width x height
 * stream with these parameters (0 on bad input). */
size_t fos_server_stream_bytes(int32_t width, int32_t height, const fos_params* params);
/* Server over one device-memory budget (bytes), at most max_streams admitted
 * streams, and queue_depth (1..1024) queued-or-running frames per stream.
 * NULL on error (fos_last_error(NULL)). */
fos_server* fos_server_create(const fos_params* params, size_t hbm_budget_bytes, int32_t max_streams,
                              int32_t queue_depth);
/* Stops the worker (frames in flight complete; pending ones are dropped). */
void fos_server_destroy(fos_server* s);
const char* fos_server_last_error(const fos_server* s);
/* Registers a camera; returns its handle (admitted now or when memory frees
 * up), -1 if it can never fit the budget. */
int32_t fos_server_open_stream(fos_server* s, int32_t width, int32_t height, uint32_t stream_id);
/* The stream leaves after its submitted frames complete; its memory is freed. */
fos_status fos_server_close_stream(fos_server* s, int32_t stream);
/* Queues one host frame of the stream (copied before returning).  The masks
 * (either may be NULL) are written when the frame completes: keep those
 * buffers valid until fos_server_poll reports the tag.  Pinned mask buffers
 * are written by DMA; pageable ones through the stream's pinned staging.
 * The stream's first submit that needs its pinned input slots or its mask
 * staging allocates them (FOS_ERR_OOM if pinned memory is exhausted).  The frame is not
 * taken (drop it or retry) with FOS_ERR_BUDGET while the stream still waits
 * for admission, and with FOS_ERR_BUSY while it has queue_depth frames queued
 * or running. */
fos_status fos_server_submit(fos_server* s, int32_t stream, const uint8_t* rgb, const uint16_t* depth,
                             uint8_t* mask_gmm, uint8_t* mask_pbas, int64_t tag);

/* Zero-copy variant of fos_server_submit: the frame is not copied; the
 * server reads rgb (H*W*3) and depth (H*W) straight from the caller's buffers
 * when the frame's tick runs, so they must stay valid and unchanged until
 * fos_server_poll reports the tag.  Pinned buffers (cudaHostAlloc /
 * cudaHostRegister) are copied by DMA; pageable ones work but are staged by
 * the driver.  When both mask buffers are pinned (or NULL) the masks are
 * copied straight into them, without the server's staging and host copy.  Same refusals (FOS_ERR_BUDGET, FOS_ERR_BUSY) as
 * fos_server_submit; frames of both kinds share the stream's queue_depth. */
fos_status fos_server_submit_nocopy(fos_server* s, int32_t stream, const uint8_t* rgb, const uint16_t* depth,
                                    uint8_t* mask_gmm, uint8_t* mask_pbas, int64_t tag);
/* Up to max_results completed frames, oldest first; returns how many. */
int32_t fos_server_poll(fos_server* s, fos_server_result* out, int32_t max_results);
/* Counters; FOS_ERR_CUDA once the worker has stopped on an error. */
fos_status fos_server_stats(fos_server* s, fos_server_stats_t* out);

/* ---------------------------------------------------------------------------
 * Differentiable (soft) GMM: parameter tuning against ground-truth masks.
 * No counterpart in the paper, which runs the hard GMM of Sec. 3.1 with fixed
 * parameters.  The hard match test d_k < L is replaced by sigmoid((L - d_k)/tau)
 * (first-match and no-match weights follow from it), the mask by
 * sigmoid((Q - L)/tau), and the loss is the mean binary cross-entropy against
 * ground truth over frames 1..T-1 of every sequence.  Gradients are taken
 * with respect to theta = (alpha, L = lambda^2, w_depth, v_init_rgb); the
 * depth model starts at v_init_rgb * v_init_d_ratio.  Ranks, background sets,
 * arg-mins and the v_min floor are decisions of the forward pass.  As tau -> 0
 * the forward equals the hard GMM (colour K = 3, depth K = 3).
 * ------------------------------------------------------------------------- */
typedef struct fos_softgmm_params {
    float alpha, lambda2, w_depth, v_init_rgb;  /* theta */
    float tau;                                  /* sigmoid temperature */
    float T_bg, v_min_rgb, v_min_d, v_init_d_ratio;
    int32_t K_rgb, K_d;                         /* must be 3 and 3 */
    int32_t ckpt_every;                         /* frames between checkpoints, 1..16 */
    uint32_t depth_full_scale_mm;
    int32_t fp64;                               /* 0: FP32 state and adjoint (fast);
                                                   1: FP64 throughout (checkpoints 8 B) */
} fos_softgmm_params;

typedef struct fos_softgmm fos_softgmm;

void fos_softgmm_default_params(fos_softgmm_params* p);
/* Workspace for `batch` sequences of `frames` frames of width x height:
 * checkpoints of the model every ckpt_every frames (24 values per pixel each,
 * 4 or 8 bytes by params->fp64). */
fos_softgmm* fos_softgmm_create(int32_t width, int32_t height, int32_t batch, int32_t frames,
                                const fos_softgmm_params* params);
void fos_softgmm_destroy(fos_softgmm* g);
const char* fos_softgmm_last_error(const fos_softgmm* g);
/* Replaces theta (alpha, lambda2, w_depth, v_init_rgb); the next backward
 * needs a forward with the new values. */
fos_status fos_softgmm_set_theta(fos_softgmm* g, const float theta[4]);
/* The same with double values: with fp64 = 1 the kernels use them unrounded
 * (finite differences of the loss need steps below float resolution). */
fos_status fos_softgmm_set_theta64(fos_softgmm* g, const double theta[4]);
/*
 * Forward over device sequences rgb [batch][frames][H][W][3] u8,
 * depth [batch][frames][H][W] u16 (mm, 0 invalid), gt [batch][frames][H][W]
 * u8 (nonzero = foreground; frame 0 unused).  Stores the checkpoints and
 * writes the loss to *loss_out (host).  Synchronous on `stream`.
 */
fos_status fos_softgmm_forward(fos_softgmm* g, const uint8_t* d_rgb, const uint16_t* d_depth,
                               const uint8_t* d_gt, double* loss_out, void* stream);
/*
 * Adjoint of the last forward (same inputs): writes d loss / d theta to
 * grad_out[4] (host); d_pixel_grad (nullable, device, [batch][H][W][4] float)
 * receives every pixel's contribution.  Sums are reduced in a fixed order
 * (deterministic).  Synchronous on `stream`.
 */
fos_status fos_softgmm_backward(fos_softgmm* g, const uint8_t* d_rgb, const uint16_t* d_depth,
                                const uint8_t* d_gt, double grad_out[4], float* d_pixel_grad,
                                void* stream);

/* ---------------------------------------------------------------------------
 * Range-checked builds.  The paper has no counterpart: this is a testing aid.
 * The library built with FOS_DEBUG_BOUNDS defined (libfos_bounds.so; the
 * build script makes it on request) checks every global and shared-memory
 * index of the GMM, PBAS (per-channel), fused, batched, frame-0 and flush
 * kernels against the extent of its buffer before the access.  A violation
 * does not fault or trap: it is counted in the context's device-side record,
 * the first one's site code and index are kept, and the access goes to a
 * scratch word instead (its result is then meaningless).  Other kernels
 * (joint-channel PBAS, literal GMM, soft GMM, quality counts, resampling,
 * the no-allocation entry point) are not instrumented.
 *
 * fos_bounds_checked: 1 in a range-checked build, else 0.
 * fos_bounds_status: waits for the device, writes the context's violation
 *     count (and, if the pointers are non-NULL, the first violation's site
 *     code and element index) and clears the record.  FOS_ERR_UNSUPPORTED in
 *     a release build (*violations set to 0).
 * fos_bounds_selftest: exercises the check itself: a one-thread kernel reads
 *     element 12 of a 64-element buffer through the checked accessor told
 *     that the buffer has 8 elements; the check must record one violation
 *     (site 99, index 12) and send the read to the scratch word, so nothing
 *     outside the declared range is touched.  Allocates and frees its own
 *     buffer (error text from fos_last_error(NULL)); FOS_ERR_UNSUPPORTED in a
 *     release build.
 * ------------------------------------------------------------------------- */
int32_t fos_bounds_checked(void);
fos_status fos_bounds_status(fos_ctx* ctx, uint32_t* violations, uint32_t* first_site,
                             int64_t* first_index);
fos_status fos_bounds_selftest(uint32_t* violations, uint32_t* first_site, int64_t* first_index);

/* ---------------------------------------------------------------------------
 * One PBAS frame step that allocates nothing.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they process frames -- plug-ins whose
 * host framework owns all device memory and forbids allocation while its
 * pipeline runs, real-time capture callbacks that cannot afford cudaMalloc's
 * implicit synchronisation and latency, and code that must leave the
 * allocator alone while other work may be capturing streams.  The caller owns
 * the model and the frame buffers; the library keeps its per-frame scratch
 * (neighbour-request words, the frame's value/gradient words, counters) in a
 * fixed array in device memory that every GPU loading the library holds until
 * the process exits (about 24 MB).  No cudaMalloc, cudaFree or other
 * allocating call is made.
 *
 * Computes exactly what a context with methods = FOS_METHOD_PBAS computes for
 * frame `frame_index` (same parameters, same bits), and additionally applies
 * this frame's neighbour updates before returning, so the model it leaves
 * equals fos_get_state of such a context after the same frame.
 *
 * width, height: 128*ceil(width/128)*height must not exceed
 *     FOS_NOALLOC_MAX_PIXELS, else FOS_ERR_INVALID_ARG.
 * params: PBAS fields are used (methods is ignored).
 * frame_index: 0 initialises the model from the frame; later calls must come
 *     in order 1, 2, ... on the same model.
 * d_rgb, d_depth, d_mask: device frame buffers as for fos_process_frame_device.
 * d_model: caller-allocated device buffer of
 *     16*N*Sp + 48*Sp + 96 bytes, Sp = 128*ceil(width/128)*height, holding
 *     (offsets in bytes) samples uint16 [4][Sp/128 segments][N][128] at 0,
 *     D uint16 (same shape) at 8*N*Sp, R float32 [4][Sp] at 16*N*Sp,
 *     T float32 [4][Sp] at 16*N*Sp + 16*Sp, S uint32 [4][Sp] at
 *     16*N*Sp + 32*Sp, gradient sums uint64 [3][4] at 16*N*Sp + 48*Sp.
 *     Must be 256-byte aligned (else FOS_ERR_INVALID_ARG).  Its contents
 *     need no initialisation before frame 0.
 * params: checked as fos_create checks them for a PBAS-only context; spatial
 *     propagation and the joint-channel variant give FOS_ERR_UNSUPPORTED.
 * stream: cudaStream_t (NULL = legacy default stream); asynchronous.
 *
 * First call on a device: the CUDA runtime loads the library's device code
 * on a device when it is first used there (lazy module loading), and that
 * load is when the scratch array is allocated; it may also synchronise the
 * device.  The first call on each device therefore allocates implicitly and
 * can fail with FOS_ERR_CUDA if the device has no room for the array.  It
 * also looks up the array's device address.  Callers with a no-allocation
 * window should make one call on every device they will use (frame 0 of any
 * model will do) before that window opens, and before any stream capture.
 * All calls share the one scratch array: calls whose kernels may overlap on
 * the GPU (other streams, other threads) race on it and must be serialised
 * by the caller.
 * Errors: status code, text from fos_last_error(NULL) on the calling thread.
 * ------------------------------------------------------------------------- */
#define FOS_NOALLOC_MAX_PIXELS 2097152

fos_status fos_pbas_step_noalloc(int32_t width, int32_t height, const fos_params* params,
                                 int64_t frame_index, const uint8_t* d_rgb,
                                 const uint16_t* d_depth, void* d_model, uint8_t* d_mask,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FOS_H */
