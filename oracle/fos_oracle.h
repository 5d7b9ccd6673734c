/*
 * fos_oracle.h -- plain CPU oracle for the RGB-D GMM and PBAS background models.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load it.  It shares no code, header, table or constant generator with
 * the CUDA path (paper_2002_00250_gb300/csrc) and must never be called from it.
 *
 * What it computes (paper: Janus, Kryjak, Gorgon, "Foreground object
 * segmentation in RGB-D data implemented on GPU"):
 *   - depth u16 -> u8 rescale                        Sec. 4.2
 *   - depth resampled to the colour resolution       Sec. 4.3
 *   - GMM with two separate models (RGB, depth)       Sec. 3.1, Eq. 1
 *   - PBAS with samples holding RGB and depth         Sec. 3.2
 *   - quality indicators PWC, FNR, FPR, Si            Sec. 5
 * The paper cites Stauffer-Grimson (GMM) and Hofmann et al. (PBAS) for the base
 * algorithms and does not restate them; the steps below restate those published
 * methods with the RGB-D adaptation the paper describes.  Every reading taken
 * where the paper is silent is listed in the repository's design notes.
 *
 * Precision: GMM in IEEE double.  PBAS in IEEE single precision and integers,
 * compiled with -ffp-contract=off so that every float operation is rounded
 * once, in the order written.
 */
#ifndef FOS_ORACLE_H
#define FOS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x32-10 counter-based generator (Salmon et al., SC'11). ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n independent evaluations; ctr is n x 4, key is n x 2, out is n x 4. */
void or_philox_many(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* ---- Sec. 4.2: depth u16 (mm, 0 = invalid) -> u8 (0 = invalid, 1..255). ---- */
void or_depth_to_u8(int64_t n, const uint16_t* depth, uint32_t full_scale_mm, uint8_t* out);

/* Depth frame of sw x sh resampled onto the colour grid dw x dh (Sec. 4.3:
 * depth is brought to the colour resolution when the two differ; the paper
 * does not say how).  Nearest neighbour: out(x, y) = src(floor(x*sw/dw),
 * floor(y*sh/dh)), so the invalid value 0 is never blended into a valid depth. */
void or_depth_resample(int sw, int sh, const uint16_t* src, int dw, int dh, uint16_t* out);

/* ---- gradient magnitude feature used by PBAS: 3x3 Sobel, L1, >>3, clamp. ---- */
void or_sobel_grad_u8(int W, int H, const uint8_t* img, uint8_t* g);

/* ---- Sec. 3.1: GMM over RGB and over depth (two models), FP64. ---- */
typedef struct {
    int K_rgb, K_d;             /* components per model, 1..8 */
    double alpha;               /* learning rate */
    double lambda;              /* match threshold on the Mahalanobis distance */
    double w_depth;             /* weight of the depth model in the combined score */
    double T_bg;                /* background weight fraction */
    double v_init_rgb, v_init_d;
    double v_min_rgb, v_min_d;
    uint32_t depth_full_scale_mm;
} or_gmm_params;

/*
 * State layout (oracle's own; pixel-major, then component):
 *   w_rgb [P*K_rgb], mu_rgb[P*K_rgb*3], v_rgb[P*K_rgb]
 *   w_d   [P*K_d],   mu_d  [P*K_d],    v_d  [P*K_d]
 * Components are stored in ranked order (slot 0 = highest rank).
 * t == 0 initialises the model from the frame; t >= 1 classifies and updates.
 * mask gets 0 (background) or 255 (foreground).
 * margin (nullable) gets, per pixel, the smallest relative distance of any
 * discrete decision taken this frame from its threshold (match tests,
 * background-set prefix sums, the final score, the ranking comparisons);
 * +inf when no decision was close to a tie.
 */
void or_gmm_frame(const or_gmm_params* p, int W, int H, int64_t t,
                  const uint8_t* rgb, const uint16_t* depth,
                  double* w_rgb, double* mu_rgb, double* v_rgb,
                  double* w_d, double* mu_d, double* v_d,
                  uint8_t* mask, double* margin, int nthreads);

/* ---- Sec. 3.1 as printed: the paper-literal GMM variant (FP64). ----
 * K_rgb = 7 / K_d = 3 in the paper; one variance per colour channel
 * ("a single value is used for each colour component"); the decision uses
 * the Eq. 1 density scaled by s: per model the factor
 *   F = s * sum_{k in B} w_k eta_k(x) / sum_{k in B} w_k,
 *   eta_k = exp(-D_k / 2) / (2 pi g_k),  D_k = sum_c (x_c - mu_kc)^2 / v_kc,
 *   g_k = (prod_c v_kc)^(1/C)
 * over the background set B of the model before this frame's update (for one
 * channel this is Eq. 1 with sigma read as the variance); the two factors are
 * multiplied (depth only where valid) and the pixel is foreground when the
 * product is below theta.  The update is the default one per channel: match =
 * first ranked k with D_k / C < lambda^2; matched: rho = alpha / w_k,
 * mu_kc += rho (x_c - mu_kc), v_kc <- max(v_min, v_kc + rho ((x_c - mu_kc)^2
 * - v_kc)); no match: last-ranked <- (alpha, x, v_init in every channel);
 * normalise; stable re-rank by w / sqrt(mean_c v_kc).
 * State (pixel-major, then component, ranked): w_rgb[P*Kr], mu_rgb[P*Kr*3],
 * v_rgb[P*Kr*3], w_d[P*Kd], mu_d[P*Kd], v_d[P*Kd].  margin as or_gmm_frame
 * (the final decision's margin is |log(F / theta)|). */
typedef struct {
    or_gmm_params base;
    double s;       /* density scale, 10000 in the paper */
    double theta;   /* background iff the product of the factors >= theta */
} or_gmm_literal_params;

void or_gmm_literal_frame(const or_gmm_literal_params* p, int W, int H, int64_t t,
                          const uint8_t* rgb, const uint16_t* depth,
                          double* w_rgb, double* mu_rgb, double* v_rgb,
                          double* w_d, double* mu_d, double* v_d,
                          uint8_t* mask, double* margin, int nthreads);

/* 1 when the oracle was built with OpenMP, else 0 (every loop single-threaded). */
int or_openmp(void);
/* Threads a parallel loop runs on for an nthreads argument (0: the OpenMP default). */
int or_threads(int nthreads);

/* ---- Sec. 3.2: PBAS with samples holding (R, G, B, D), FP32 + integers. ---- */
typedef struct {
    int N;                      /* samples per pixel, 1..32 */
    int n_min;                  /* #min: matches needed for background */
    float R_lower_rgb, R_lower_d, R_scale, R_incdec;
    float T_lower, T_upper, T_inc, T_dec;
    float alpha_g;              /* gradient weight numerator */
    float eps_d;                /* floor of the mean minimal distance */
    uint32_t seed, stream_id;   /* Philox key */
    int forced_rng;             /* 1..3: test-only deterministic draws (see or_pbas_draws) */
    uint32_t depth_full_scale_mm;
    int propagate;              /* neighbour update: 0 = the neighbour takes its own value
                                   (the base method); 1 = it takes the updating pixel's value
                                   (spatial propagation as in ViBe); a slot the pixel's own
                                   update of the same frame wrote keeps that value, and among
                                   neighbours asking for the same slot the one with the
                                   lowest direction index as seen from the pixel wins */
    int joint;                  /* 0: each channel has its own R, T, D and decision (the
                                   base method; foreground if any channel is); 1: one R, T,
                                   D per pixel (channel 0's entries) and one decision on the
                                   joint distance over the active channels (see
                                   or_pbas_frame) */
} or_pbas_params;

/*
 * State layout (oracle's own): for pixel p, channel c in {0:R,1:G,2:B,3:D},
 * slot k:  sv[(p*4+c)*N+k] (u8 value), sg[...] (u8 gradient), sD[...] (u16,
 * minimal distance x16); R[p*4+c], T[p*4+c] (float), S[p*4+c] (u32, sum of
 * the N D values).  gsum[4] holds the gradient sums of the previous frame
 * (read at t >= 1, rewritten every frame).
 *
 * Joint-channel variant (p->joint): the active channels A of a pixel are R,
 * G, B, and D where the depth reading is valid; n = |A|.  The distance of
 * sample k is the mean over A of the per-channel distances: the FP32 sum of
 * fl(fl(wg_c |dg|) + |dv|) in channel order, times fl(1/n).  One decision
 * per pixel (fewer than #min samples within R: foreground), one draw per
 * pixel (channel word 0 of the counter), and the pixel's R, T, S and D are
 * those of channel 0 (R floor R_lower_rgb); the entries of channels 1..3
 * keep their bootstrap values.  The own update writes every channel of A
 * into the slot; a neighbour request covers all four channels (with
 * propagation, the requester's active ones).
 */
void or_pbas_frame(const or_pbas_params* p, int W, int H, int64_t t,
                   const uint8_t* rgb, const uint16_t* depth,
                   uint8_t* sv, uint8_t* sg, uint16_t* sD,
                   float* R, float* T, uint32_t* S, uint64_t gsum[4],
                   uint8_t* mask, int nthreads);

/* ---- Sec. 5: quality indicators.  out = {TP, TN, FP, FN, PWC, FNR, FPR, Si}. ---- */
void or_quality(int64_t n, const uint8_t* mask, const uint8_t* gt, double out[8]);

#ifdef __cplusplus
}
#endif
#endif
