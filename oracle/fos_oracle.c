/*
 * fos_oracle.c -- plain CPU oracle (TEST INFRASTRUCTURE ONLY; see fos_oracle.h).
 *
 * Written to be read against the paper, not to be fast: one pixel at a time,
 * the steps in the order the method defines them.  The only concession to
 * speed is an OpenMP loop over pixels (each iteration touches its own pixel's
 * state only); the PBAS neighbour writes run serially in raster order.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math [-fopenmp] -shared -fPIC
 */
#include "fos_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define OR_THREADS(n) ((n) > 0 ? (n) : omp_get_max_threads())
#else
#define OR_THREADS(n) 1
#endif

/* 1 when built with OpenMP (the pixel loops then run on the host's cores). */
int or_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Threads a parallel loop of the oracle runs on for an nthreads argument. */
int or_threads(int nthreads) { return OR_THREADS(nthreads); }

/* ======================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications     */
/* with the published multipliers, key bumped by the published Weyl          */
/* constants between rounds.                                                 */
/* ======================================================================== */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_W0;
            k1 += OR_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void or_philox_many(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i)
        or_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* ======================================================================== */
/* Sec. 4.2: the 16-bit depth (mm) is rescaled to 8 bits.  Reading: the     */
/* sensor's 10 m range maps to 1..255 (about 4 cm per step, as the paper    */
/* states), rounding half up in integers; 0 stays 0 and marks an invalid    */
/* reading ("valid if greater than 0", Sec. 3.1).                           */
/* ======================================================================== */
static uint8_t or_depth_u8_one(uint16_t d, uint32_t full_scale_mm)
{
    if (d == 0) return 0;
    uint64_t q = ((uint64_t)d * 255u + full_scale_mm / 2u) / full_scale_mm;
    if (q < 1) q = 1;
    if (q > 255) q = 255;
    return (uint8_t)q;
}

void or_depth_to_u8(int64_t n, const uint16_t* depth, uint32_t full_scale_mm, uint8_t* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_depth_u8_one(depth[i], full_scale_mm);
}

/* ======================================================================== */
/* Gradient magnitude feature (PBAS uses the gradient magnitude beside the  */
/* value): 3x3 Sobel, |gx| + |gy|, shifted right by 3 and clamped to 255;   */
/* borders repeat the edge pixel.                                           */
/* ======================================================================== */
static int or_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int or_px(const uint8_t* img, int W, int H, int x, int y)
{
    return img[(int64_t)or_clampi(y, 0, H - 1) * W + or_clampi(x, 0, W - 1)];
}

void or_depth_resample(int sw, int sh, const uint16_t* src, int dw, int dh, uint16_t* out)
{
    for (int y = 0; y < dh; ++y) {
        const int ys = (int)(((int64_t)y * sh) / dh);
        for (int x = 0; x < dw; ++x) {
            const int xs = (int)(((int64_t)x * sw) / dw);
            out[(int64_t)y * dw + x] = src[(int64_t)ys * sw + xs];
        }
    }
}

void or_sobel_grad_u8(int W, int H, const uint8_t* img, uint8_t* g)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int gx = (or_px(img, W, H, x + 1, y - 1) + 2 * or_px(img, W, H, x + 1, y) +
                      or_px(img, W, H, x + 1, y + 1)) -
                     (or_px(img, W, H, x - 1, y - 1) + 2 * or_px(img, W, H, x - 1, y) +
                      or_px(img, W, H, x - 1, y + 1));
            int gy = (or_px(img, W, H, x - 1, y + 1) + 2 * or_px(img, W, H, x, y + 1) +
                      or_px(img, W, H, x + 1, y + 1)) -
                     (or_px(img, W, H, x - 1, y - 1) + 2 * or_px(img, W, H, x, y - 1) +
                      or_px(img, W, H, x + 1, y - 1));
            int m = (abs(gx) + abs(gy)) >> 3;
            g[(int64_t)y * W + x] = (uint8_t)(m > 255 ? 255 : m);
        }
}

/* ======================================================================== */
/* Sec. 3.1: GMM, two separate models (RGB with C = 3, depth with C = 1).   */
/* Each model: K components (w, mu[C], v) in ranked order, v one variance   */
/* shared by the channels.  The per-frame update follows the Stauffer-      */
/* Grimson method the paper builds on; the depth model is skipped entirely  */
/* when the depth reading is invalid; the two models' distances are         */
/* combined into one score compared with the match threshold.               */
/* ======================================================================== */
typedef struct {
    double w;
    double mu[3];
    double v;
} or_comp;

static void or_margin_min(double* m, double a, double threshold)
{
    double r = fabs(a - threshold) / fabs(threshold);
    if (r < *m) *m = r;
}

/*
 * One model, one pixel, one frame t >= 1.  Returns the background-set
 * distance of the model as it was before this frame's update.
 */
static double or_gmm_model_step(int K, int C, const or_gmm_params* p, double v_init, double v_min,
                                 const double* x, or_comp* c, double* margin)
{
    const double lam2 = p->lambda * p->lambda;
    const double alpha = p->alpha;
    double d2[8], ss[8], diff[8][3];

    /* 1. squared Mahalanobis distance of x to each component (old params). */
    for (int k = 0; k < K; ++k) {
        ss[k] = 0.0;
        for (int ch = 0; ch < C; ++ch) {
            diff[k][ch] = x[ch] - c[k].mu[ch];
            ss[k] += diff[k][ch] * diff[k][ch];
        }
        d2[k] = ss[k] / ((double)C * c[k].v);
    }

    /* 2. background set B: shortest ranked prefix whose weight exceeds T_bg;
     *    the pixel's distance to the background is the smallest over B. */
    double cum = 0.0, dB = INFINITY;
    for (int k = 0; k < K; ++k) {
        if (d2[k] < dB) dB = d2[k];
        cum += c[k].w;
        or_margin_min(margin, cum, p->T_bg);
        if (cum > p->T_bg) break;
    }

    /* 3. match: first component in ranked order within the threshold. */
    int match = -1;
    for (int k = 0; k < K; ++k) {
        or_margin_min(margin, d2[k], lam2);
        if (d2[k] < lam2) {
            match = k;
            break;
        }
    }

    /* 4. weights: w <- (1 - alpha) w + alpha [k = match]. */
    for (int k = 0; k < K; ++k) c[k].w = (1.0 - alpha) * c[k].w + (k == match ? alpha : 0.0);

    if (match >= 0) {
        /* 5. matched component moves toward x with rate rho = alpha / w. */
        or_comp* m = &c[match];
        double rho = alpha / m->w;
        for (int ch = 0; ch < C; ++ch) m->mu[ch] = m->mu[ch] + rho * diff[match][ch];
        double v = m->v + rho * (ss[match] / (double)C - m->v);
        m->v = v > v_min ? v : v_min;
    } else {
        /* 6. no match: the last-ranked component is replaced by x. */
        or_comp* m = &c[K - 1];
        m->w = alpha;
        for (int ch = 0; ch < C; ++ch) m->mu[ch] = x[ch];
        for (int ch = C; ch < 3; ++ch) m->mu[ch] = 0.0;
        m->v = v_init;
    }

    /* 7. normalise the weights (sum in index order). */
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += c[k].w;
    for (int k = 0; k < K; ++k) c[k].w = c[k].w / s;

    /* 8. re-rank by w / sqrt(v), descending, stable (ties keep their order). */
    double key[8];
    for (int k = 0; k < K; ++k) key[k] = c[k].w / sqrt(c[k].v);
    for (int a = 0; a < K; ++a)
        for (int b = a + 1; b < K; ++b) {
            if (key[a] == 0.0 && key[b] == 0.0) continue; /* untouched slots: exact tie */
            double mx = fabs(key[a]) > fabs(key[b]) ? fabs(key[a]) : fabs(key[b]);
            double r = fabs(key[a] - key[b]) / mx;
            if (r < *margin) *margin = r;
        }
    for (int i = 1; i < K; ++i) {
        int j = i;
        while (j > 0 && key[j] > key[j - 1]) {
            or_comp tc = c[j];
            c[j] = c[j - 1];
            c[j - 1] = tc;
            double tk = key[j];
            key[j] = key[j - 1];
            key[j - 1] = tk;
            --j;
        }
    }
    return dB;
}

static void or_gmm_load(int K, int C, const double* w, const double* mu, const double* v, or_comp* c)
{
    for (int k = 0; k < K; ++k) {
        c[k].w = w[k];
        for (int ch = 0; ch < 3; ++ch) c[k].mu[ch] = ch < C ? mu[k * C + ch] : 0.0;
        c[k].v = v[k];
    }
}

static void or_gmm_store(int K, int C, const or_comp* c, double* w, double* mu, double* v)
{
    for (int k = 0; k < K; ++k) {
        w[k] = c[k].w;
        for (int ch = 0; ch < C; ++ch) mu[k * C + ch] = c[k].mu[ch];
        v[k] = c[k].v;
    }
}

void or_gmm_frame(const or_gmm_params* p, int W, int H, int64_t t,
                  const uint8_t* rgb, const uint16_t* depth,
                  double* w_rgb, double* mu_rgb, double* v_rgb,
                  double* w_d, double* mu_d, double* v_d,
                  uint8_t* mask, double* margin, int nthreads)
{
    const int64_t P = (int64_t)W * H;
    const int Kr = p->K_rgb, Kd = p->K_d;
    const double lam2 = p->lambda * p->lambda;
    (void)nthreads;

#pragma omp parallel for schedule(static) num_threads(OR_THREADS(nthreads))
    for (int64_t i = 0; i < P; ++i) {
        double xr[3] = {rgb[3 * i + 0], rgb[3 * i + 1], rgb[3 * i + 2]};
        int valid = depth[i] != 0;
        double xd[1] = {(double)or_depth_u8_one(depth[i], p->depth_full_scale_mm)};
        or_comp cr[8], cd[8];
        double mg = INFINITY;

        if (t == 0) {
            /* bootstrap: first component takes the first frame, the rest are empty. */
            for (int k = 0; k < Kr; ++k) {
                cr[k].w = k == 0 ? 1.0 : 0.0;
                for (int ch = 0; ch < 3; ++ch) cr[k].mu[ch] = k == 0 ? xr[ch] : 0.0;
                cr[k].v = p->v_init_rgb;
            }
            for (int k = 0; k < Kd; ++k) {
                cd[k].w = k == 0 ? 1.0 : 0.0;
                cd[k].mu[0] = k == 0 ? xd[0] : 0.0;
                cd[k].mu[1] = cd[k].mu[2] = 0.0;
                cd[k].v = p->v_init_d;
            }
            mask[i] = 0;
        } else {
            or_gmm_load(Kr, 3, w_rgb + i * Kr, mu_rgb + i * Kr * 3, v_rgb + i * Kr, cr);
            or_gmm_load(Kd, 1, w_d + i * Kd, mu_d + i * Kd, v_d + i * Kd, cd);
            double dB_rgb = or_gmm_model_step(Kr, 3, p, p->v_init_rgb, p->v_min_rgb, xr, cr, &mg);
            double Q = dB_rgb;
            if (valid) {
                double dB_d = or_gmm_model_step(Kd, 1, p, p->v_init_d, p->v_min_d, xd, cd, &mg);
                Q = (1.0 - p->w_depth) * dB_rgb + p->w_depth * dB_d;
            }
            or_margin_min(&mg, Q, lam2);
            mask[i] = Q >= lam2 ? 255 : 0;
        }
        or_gmm_store(Kr, 3, cr, w_rgb + i * Kr, mu_rgb + i * Kr * 3, v_rgb + i * Kr);
        or_gmm_store(Kd, 1, cd, w_d + i * Kd, mu_d + i * Kd, v_d + i * Kd);
        if (margin) margin[i] = mg;
    }
}

/* ---- the paper-literal GMM variant (declaration comment in the header) ---- */
typedef struct {
    double w, mu[3], v[3];
} or_dcomp;

/* One model, one pixel, one frame t >= 1: returns the model's density factor
 * F = s * (background-set mixture density of x) before this frame's update. */
static double or_gmm_literal_model_step(int K, int C, const or_gmm_literal_params* lp, double v_init,
                                        double v_min, const double* x, or_dcomp* c, double* margin)
{
    const or_gmm_params* p = &lp->base;
    const double lam2 = p->lambda * p->lambda, alpha = p->alpha;
    const double two_pi = 6.283185307179586476925286766559;
    double D[8], diff[8][3];
    for (int k = 0; k < K; ++k) {
        D[k] = 0.0;
        for (int ch = 0; ch < C; ++ch) {
            diff[k][ch] = x[ch] - c[k].mu[ch];
            D[k] += diff[k][ch] * diff[k][ch] / c[k].v[ch];
        }
    }
    /* background set and its normalised mixture density (old parameters) */
    double cum = 0.0, num = 0.0, den = 0.0;
    for (int k = 0; k < K; ++k) {
        double g = 1.0;
        for (int ch = 0; ch < C; ++ch) g *= c[k].v[ch];
        g = pow(g, 1.0 / (double)C);
        num += c[k].w * exp(-0.5 * D[k]) / (two_pi * g);
        den += c[k].w;
        cum += c[k].w;
        or_margin_min(margin, cum, p->T_bg);
        if (cum > p->T_bg) break;
    }
    const double F = lp->s * num / den;
    /* match on the per-channel Mahalanobis distance, averaged over channels */
    int match = -1;
    for (int k = 0; k < K; ++k) {
        const double dm = D[k] / (double)C;
        or_margin_min(margin, dm, lam2);
        if (dm < lam2) {
            match = k;
            break;
        }
    }
    for (int k = 0; k < K; ++k) c[k].w = (1.0 - alpha) * c[k].w + (k == match ? alpha : 0.0);
    if (match >= 0) {
        or_dcomp* m = &c[match];
        const double rho = alpha / m->w;
        for (int ch = 0; ch < C; ++ch) {
            m->mu[ch] = m->mu[ch] + rho * diff[match][ch];
            const double v = m->v[ch] + rho * (diff[match][ch] * diff[match][ch] - m->v[ch]);
            m->v[ch] = v > v_min ? v : v_min;
        }
    } else {
        or_dcomp* m = &c[K - 1];
        m->w = alpha;
        for (int ch = 0; ch < 3; ++ch) {
            m->mu[ch] = ch < C ? x[ch] : 0.0;
            m->v[ch] = ch < C ? v_init : 0.0;
        }
    }
    double sum = 0.0;
    for (int k = 0; k < K; ++k) sum += c[k].w;
    for (int k = 0; k < K; ++k) c[k].w = c[k].w / sum;
    double key[8];
    for (int k = 0; k < K; ++k) {
        double vb = 0.0;
        for (int ch = 0; ch < C; ++ch) vb += c[k].v[ch];
        key[k] = c[k].w / sqrt(vb / (double)C);
    }
    for (int a = 0; a < K; ++a)
        for (int b = a + 1; b < K; ++b) {
            if (key[a] == 0.0 && key[b] == 0.0) continue;
            const double mx = fabs(key[a]) > fabs(key[b]) ? fabs(key[a]) : fabs(key[b]);
            const double r = fabs(key[a] - key[b]) / mx;
            if (r < *margin) *margin = r;
        }
    for (int i = 1; i < K; ++i) {
        int j = i;
        while (j > 0 && key[j] > key[j - 1]) {
            or_dcomp tc = c[j]; c[j] = c[j - 1]; c[j - 1] = tc;
            double tk = key[j]; key[j] = key[j - 1]; key[j - 1] = tk;
            --j;
        }
    }
    return F;
}

void or_gmm_literal_frame(const or_gmm_literal_params* lp, int W, int H, int64_t t,
                          const uint8_t* rgb, const uint16_t* depth,
                          double* w_rgb, double* mu_rgb, double* v_rgb,
                          double* w_d, double* mu_d, double* v_d,
                          uint8_t* mask, double* margin, int nthreads)
{
    const or_gmm_params* p = &lp->base;
    const int64_t P = (int64_t)W * H;
    const int Kr = p->K_rgb, Kd = p->K_d;
    (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(OR_THREADS(nthreads))
    for (int64_t i = 0; i < P; ++i) {
        const double xr[3] = {rgb[3 * i + 0], rgb[3 * i + 1], rgb[3 * i + 2]};
        const int valid = depth[i] != 0;
        const double xd[1] = {(double)or_depth_u8_one(depth[i], p->depth_full_scale_mm)};
        or_dcomp cr[8], cd[8];
        double mg = INFINITY;
        if (t == 0) {
            for (int k = 0; k < Kr; ++k) {
                cr[k].w = k == 0 ? 1.0 : 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    cr[k].mu[ch] = k == 0 ? xr[ch] : 0.0;
                    cr[k].v[ch] = p->v_init_rgb;
                }
            }
            for (int k = 0; k < Kd; ++k) {
                cd[k].w = k == 0 ? 1.0 : 0.0;
                cd[k].mu[0] = k == 0 ? xd[0] : 0.0;
                cd[k].v[0] = p->v_init_d;
            }
            mask[i] = 0;
        } else {
            for (int k = 0; k < Kr; ++k) {
                cr[k].w = w_rgb[i * Kr + k];
                for (int ch = 0; ch < 3; ++ch) {
                    cr[k].mu[ch] = mu_rgb[(i * Kr + k) * 3 + ch];
                    cr[k].v[ch] = v_rgb[(i * Kr + k) * 3 + ch];
                }
            }
            for (int k = 0; k < Kd; ++k) {
                cd[k].w = w_d[i * Kd + k];
                cd[k].mu[0] = mu_d[i * Kd + k];
                cd[k].v[0] = v_d[i * Kd + k];
            }
            double F = or_gmm_literal_model_step(Kr, 3, lp, p->v_init_rgb, p->v_min_rgb, xr, cr, &mg);
            if (valid) F *= or_gmm_literal_model_step(Kd, 1, lp, p->v_init_d, p->v_min_d, xd, cd, &mg);
            const double r = fabs(log(F / lp->theta));
            if (r < mg) mg = r;
            mask[i] = F >= lp->theta ? 0 : 255;
        }
        for (int k = 0; k < Kr; ++k) {
            w_rgb[i * Kr + k] = cr[k].w;
            for (int ch = 0; ch < 3; ++ch) {
                mu_rgb[(i * Kr + k) * 3 + ch] = cr[k].mu[ch];
                v_rgb[(i * Kr + k) * 3 + ch] = cr[k].v[ch];
            }
        }
        for (int k = 0; k < Kd; ++k) {
            w_d[i * Kd + k] = cd[k].w;
            mu_d[i * Kd + k] = cd[k].mu[0];
            v_d[i * Kd + k] = cd[k].v[0];
        }
        if (margin) margin[i] = mg;
    }
}

/* ======================================================================== */
/* Sec. 3.2: PBAS (Hofmann et al.) with a sample holding R, G, B and D,     */
/* each channel processed separately with its own decision threshold R,     */
/* learning parameter T and minimal-distance record D; the depth channel    */
/* only where the depth reading is valid; the pixel is foreground if any    */
/* processed channel says so.  Two phases: every pixel is classified        */
/* against the model as it stood after the previous frame, then the         */
/* neighbour updates are applied.                                           */
/* ======================================================================== */
static const int OR_DIRX[8] = {0, 1, 1, 1, 0, -1, -1, -1}; /* N NE E SE S SW W NW */
static const int OR_DIRY[8] = {-1, -1, 0, 1, 1, 1, 0, -1};

typedef struct {
    int coin1, k1, coin2, j, k2;
} or_draws;

static or_draws or_pbas_draws(const or_pbas_params* p, int W, int64_t pix, int64_t t, int c, float prob)
{
    or_draws d;
    if (p->forced_rng) {
        /* mode 1: every pixel the same direction t mod 8; mode 2: east from
         * columns 0, 1 (mod 4) and west from columns 2, 3, so a pixel can
         * receive two requests for the same slot (tests the conflict rule);
         * mode 3: north from even columns, south-east from odd ones, so every
         * even column is asked from below and from the north-west; pixels of
         * even rows ask for the slot of their own update (t mod N), odd rows
         * for (t + 1) mod N */
        const int64_t col = pix % W, row = pix / W;
        d.coin1 = 1;
        d.coin2 = 1;
        d.k1 = (int)(t % p->N);
        d.k2 = (int)((t + 1) % p->N);
        if (p->forced_rng == 1) {
            d.j = (int)(t % 8);
        } else if (p->forced_rng == 2) {
            d.j = ((col >> 1) & 1) == 0 ? 2 : 6;
        } else {
            d.j = (col & 1) == 0 ? 0 : 3;
            if ((row & 1) == 0) d.k2 = d.k1;
        }
        return d;
    }
    uint32_t ctr[4] = {(uint32_t)pix, (uint32_t)t, (uint32_t)c, 0u};
    uint32_t key[2] = {p->seed, p->stream_id};
    uint32_t u[4];
    or_philox4x32_10(ctr, key, u);
    const float two_m24 = 1.0f / 16777216.0f;
    d.coin1 = (float)(u[0] >> 8) * two_m24 < prob;
    d.k1 = (int)(((uint64_t)u[1] * (uint64_t)p->N) >> 32);
    d.coin2 = (float)(u[2] >> 8) * two_m24 < prob;
    d.j = (int)(u[3] >> 29);
    d.k2 = (int)(((uint64_t)(u[3] & 0x1FFFFFFFu) * (uint64_t)p->N) >> 29);
    return d;
}

void or_pbas_frame(const or_pbas_params* p, int W, int H, int64_t t,
                   const uint8_t* rgb, const uint16_t* depth,
                   uint8_t* sv, uint8_t* sg, uint16_t* sD,
                   float* R, float* T, uint32_t* S, uint64_t gsum[4],
                   uint8_t* mask, int nthreads)
{
    const int64_t P = (int64_t)W * H;
    const int N = p->N;
    (void)nthreads;

    /* channel images (R, G, B, depth rescaled) and their gradient magnitudes. */
    uint8_t* ch = (uint8_t*)malloc((size_t)(4 * P));
    uint8_t* gr = (uint8_t*)malloc((size_t)(4 * P));
    uint8_t* valid = (uint8_t*)malloc((size_t)P);
    int8_t* req_j = (int8_t*)malloc((size_t)(4 * P));
    int8_t* req_k = (int8_t*)malloc((size_t)(4 * P));
    int8_t* own_k = (int8_t*)malloc((size_t)(4 * P));   /* slot of this frame's own update */
    for (int64_t i = 0; i < P; ++i) {
        ch[0 * P + i] = rgb[3 * i + 0];
        ch[1 * P + i] = rgb[3 * i + 1];
        ch[2 * P + i] = rgb[3 * i + 2];
        ch[3 * P + i] = or_depth_u8_one(depth[i], p->depth_full_scale_mm);
        valid[i] = depth[i] != 0;
    }
    for (int c = 0; c < 4; ++c) or_sobel_grad_u8(W, H, ch + c * P, gr + c * P);

    if (t == 0) {
        /* bootstrap: every sample slot takes the first frame. */
        for (int64_t i = 0; i < P; ++i) {
            for (int c = 0; c < 4; ++c) {
                int64_t b = (i * 4 + c) * N;
                for (int k = 0; k < N; ++k) {
                    sv[b + k] = ch[c * P + i];
                    sg[b + k] = gr[c * P + i];
                    sD[b + k] = 0;
                }
                R[i * 4 + c] = c < 3 ? p->R_lower_rgb : p->R_lower_d;
                T[i * 4 + c] = p->T_lower;
                S[i * 4 + c] = 0;
            }
            mask[i] = 0;
        }
    } else {
        /* gradient weight: alpha / (mean gradient magnitude of the previous frame). */
        float wg[4];
        for (int c = 0; c < 4; ++c) {
            float mean = (float)gsum[c] / (float)P;
            if (mean < 1.0f) mean = 1.0f;
            wg[c] = p->alpha_g / mean;
        }
        const float one_minus_r = 1.0f - p->R_incdec;
        const float one_plus_r = 1.0f + p->R_incdec;
        const float n16 = (float)(16 * N);

        /* phase 1, joint-channel variant: one distance per sample over the
         * active channels, one decision, one draw and one R, T, D per pixel
         * (kept in channel 0's entries). */
        const int64_t P_joint = p->joint ? P : 0, P_sep = p->joint ? 0 : P;
#pragma omp parallel for schedule(static) num_threads(OR_THREADS(nthreads))
        for (int64_t i = 0; i < P_joint; ++i) {
            const int nc = valid[i] ? 4 : 3;
            const float inv_nc = 1.0f / (float)nc;
            for (int c = 0; c < 4; ++c) {
                req_j[i * 4 + c] = -1;
                req_k[i * 4 + c] = -1;
                own_k[i * 4 + c] = -1;
            }
            float Rx = R[i * 4];
            int count = 0;
            float dmin = INFINITY;
            for (int k = 0; k < N; ++k) {
                float sum = 0.0f;
                for (int c = 0; c < nc; ++c) {
                    int64_t b = (i * 4 + c) * N + k;
                    float a = wg[c] * (float)abs((int)gr[c * P + i] - (int)sg[b]);
                    float dist_c = a + (float)abs((int)ch[c * P + i] - (int)sv[b]);
                    sum = sum + dist_c;
                }
                float dist = sum * inv_nc;
                if (dist < Rx) ++count;
                if (dist < dmin) dmin = dist;
            }
            int fg = count < p->n_min;
            float Tx = T[i * 4];
            or_draws d = or_pbas_draws(p, W, i, t, 0, 1.0f / Tx);
            if (!fg && d.coin1) {
                for (int c = 0; c < nc; ++c) {
                    int64_t b = (i * 4 + c) * N + d.k1;
                    sv[b] = ch[c * P + i];
                    sg[b] = gr[c * P + i];
                    own_k[i * 4 + c] = (int8_t)d.k1;
                }
                float q16 = dmin * 16.0f;
                uint32_t q = q16 >= 65535.0f ? 65535u : (uint32_t)rintf(q16);
                S[i * 4] = S[i * 4] + q - sD[i * 4 * N + d.k1];
                sD[i * 4 * N + d.k1] = (uint16_t)q;
            }
            float dbar = (float)S[i * 4] / n16;
            if (dbar < p->eps_d) dbar = p->eps_d;
            float Rs = dbar * p->R_scale;
            Rx = Rx > Rs ? Rx * one_minus_r : Rx * one_plus_r;
            if (Rx < p->R_lower_rgb) Rx = p->R_lower_rgb;
            R[i * 4] = Rx;
            if (fg) Tx = Tx + p->T_inc / dbar;
            else Tx = Tx - p->T_dec / dbar;
            if (Tx < p->T_lower) Tx = p->T_lower;
            if (Tx > p->T_upper) Tx = p->T_upper;
            T[i * 4] = Tx;
            if (!fg && d.coin2) {
                /* the whole sample: all four channels (phase 2 writes the
                 * asked pixel's depth only where it is valid); with
                 * propagation the requester's active channels */
                const int nreq = p->propagate ? nc : 4;
                for (int c = 0; c < nreq; ++c) {
                    req_j[i * 4 + c] = (int8_t)d.j;
                    req_k[i * 4 + c] = (int8_t)d.k2;
                }
            }
            mask[i] = fg ? 255 : 0;
        }

        /* phase 1: classify every pixel and update its own model. */
#pragma omp parallel for schedule(static) num_threads(OR_THREADS(nthreads))
        for (int64_t i = 0; i < P_sep; ++i) {
            int any_fg = 0;
            for (int c = 0; c < 4; ++c) {
                req_j[i * 4 + c] = -1;
                req_k[i * 4 + c] = -1;
                own_k[i * 4 + c] = -1;
                if (c == 3 && !valid[i]) continue;
                int64_t b = (i * 4 + c) * N;
                int v = ch[c * P + i], g = gr[c * P + i];
                float Rx = R[i * 4 + c];
                int count = 0;
                float dmin = INFINITY;
                for (int k = 0; k < N; ++k) {
                    float a = wg[c] * (float)abs(g - (int)sg[b + k]);
                    float dist = a + (float)abs(v - (int)sv[b + k]);
                    if (dist < Rx) ++count;
                    if (dist < dmin) dmin = dist;
                }
                int fg = count < p->n_min;
                any_fg |= fg;

                float Tx = T[i * 4 + c];
                float prob = 1.0f / Tx;
                or_draws d = or_pbas_draws(p, W, i, t, c, prob);

                if (!fg && d.coin1) {
                    own_k[i * 4 + c] = (int8_t)d.k1;
                    sv[b + d.k1] = (uint8_t)v;
                    sg[b + d.k1] = (uint8_t)g;
                    float q16 = dmin * 16.0f;
                    uint32_t q = q16 >= 65535.0f ? 65535u : (uint32_t)rintf(q16);
                    S[i * 4 + c] = S[i * 4 + c] + q - sD[b + d.k1];
                    sD[b + d.k1] = (uint16_t)q;
                }
                float dbar = (float)S[i * 4 + c] / n16;
                if (dbar < p->eps_d) dbar = p->eps_d;

                /* decision threshold R: shrink when above R_scale * dbar, else grow. */
                float Rs = dbar * p->R_scale;
                Rx = Rx > Rs ? Rx * one_minus_r : Rx * one_plus_r;
                float Rlo = c < 3 ? p->R_lower_rgb : p->R_lower_d;
                if (Rx < Rlo) Rx = Rlo;
                R[i * 4 + c] = Rx;

                /* learning parameter T: grows on foreground, shrinks on background. */
                if (fg) Tx = Tx + p->T_inc / dbar;
                else Tx = Tx - p->T_dec / dbar;
                if (Tx < p->T_lower) Tx = p->T_lower;
                if (Tx > p->T_upper) Tx = p->T_upper;
                T[i * 4 + c] = Tx;

                if (!fg && d.coin2) {
                    req_j[i * 4 + c] = (int8_t)d.j;
                    req_k[i * 4 + c] = (int8_t)d.k2;
                }
            }
            mask[i] = any_fg ? 255 : 0;
        }

        /* phase 2, spatial propagation: a requested neighbour y takes the
         * requesting pixel's value.  A slot that y's own update of this frame
         * wrote keeps y's value; the other slots go to the first request met
         * when y looks at its neighbours in direction order N, NE, ..., NW
         * (the neighbour r = y + dir(jy) made request j = jy ^ 4, the
         * opposite direction, if it points at y). */
        if (p->propagate) {
            for (int64_t n = 0; n < P; ++n) {
                const int tx = (int)(n % W), ty = (int)(n / W);
                for (int c = 0; c < 4; ++c) {
                    char taken[32] = {0};
                    if (own_k[n * 4 + c] >= 0) taken[(int)own_k[n * 4 + c]] = 1;
                    for (int jy = 0; jy < 8; ++jy) {
                        const int rx = tx + OR_DIRX[jy], ry = ty + OR_DIRY[jy];
                        if (rx < 0 || rx >= W || ry < 0 || ry >= H) continue;
                        const int64_t r = (int64_t)ry * W + rx;
                        if (req_j[r * 4 + c] != (jy ^ 4)) continue;
                        const int k = req_k[r * 4 + c];
                        if (taken[k]) continue;
                        taken[k] = 1;
                        const int64_t b = (n * 4 + c) * N + k;
                        sv[b] = ch[c * P + r];
                        sg[b] = gr[c * P + r];
                    }
                }
            }
        }
        /* phase 2: neighbour updates; the neighbour y takes its own current value. */
        for (int64_t i = 0; i < P && !p->propagate; ++i) {
            int x = (int)(i % W), y = (int)(i / W);
            for (int c = 0; c < 4; ++c) {
                int j = req_j[i * 4 + c];
                if (j < 0) continue;
                int nx = x + OR_DIRX[j], ny = y + OR_DIRY[j];
                if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
                int64_t n = (int64_t)ny * W + nx;
                if (c == 3 && !valid[n]) continue;
                int64_t b = (n * 4 + c) * N + req_k[i * 4 + c];
                sv[b] = ch[c * P + n];
                sg[b] = gr[c * P + n];
            }
        }
    }

    /* gradient sums of this frame, for the next frame's weight. */
    for (int c = 0; c < 4; ++c) {
        uint64_t s = 0;
        for (int64_t i = 0; i < P; ++i) s += gr[c * P + i];
        gsum[c] = s;
    }
    free(ch);
    free(gr);
    free(valid);
    free(req_j);
    free(req_k);
    free(own_k);
}

/* ======================================================================== */
/* Sec. 5: percentage of wrong classifications, false negative rate, false  */
/* positive rate and similarity from the confusion counts.                  */
/* ======================================================================== */
void or_quality(int64_t n, const uint8_t* mask, const uint8_t* gt, double out[8])
{
    double tp = 0, tn = 0, fp = 0, fn = 0;
    for (int64_t i = 0; i < n; ++i) {
        int m = mask[i] != 0, g = gt[i] != 0;
        if (m && g) tp += 1;
        else if (!m && !g) tn += 1;
        else if (m && !g) fp += 1;
        else fn += 1;
    }
    out[0] = tp;
    out[1] = tn;
    out[2] = fp;
    out[3] = fn;
    out[4] = 100.0 * (fn + fp) / (tp + fn + fp + tn);
    out[5] = fn / (tp + fn);
    out[6] = fp / (fp + tn);
    out[7] = tp / (tp + fp + fn);
}
