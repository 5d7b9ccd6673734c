// gmm_dev.cuh -- per-pixel GMM device code shared by the GMM kernels and the
// fused GMM+PBAS tile kernel (paper Sec. 3.1, Eq. 1).
//
// Every floating-point operation is written as an explicit intrinsic (fused
// multiply-adds where intended), so the result does not depend on the
// compiler's contraction setting of the including file: all kernels produce
// the same bits for the same pixel.  Quotients use the hardware reciprocal
// approximation (__fdividef, at most 2 ulp) rather than the correctly rounded
// division, which costs about twenty instructions each: the FP32 model is held
// to the FP64 definition only within 1e-4 relative, and fourteen divisions per
// pixel made the update a quarter of the fused kernel's instructions.
#pragma once
#include <cmath>

#include "fos_internal.h"

namespace fos {
namespace gmmdev {

template <int K, int C>
struct Mix {
    float w[K];
    float mu[C][K];
    float v[K];
};

// Depth u16 (mm) -> u8 as Sec. 4.2 describes: 0 stays 0 (invalid), the full
// scale maps onto 1..255 with round-half-up.
__device__ __forceinline__ uint32_t depth_to_u8(uint32_t d, uint32_t fs)
{
    if (d == 0) return 0;
    uint32_t q = (d * 255u + (fs >> 1)) / fs;
    return q < 1u ? 1u : (q > 255u ? 255u : q);
}

template <int K, int C>
__device__ __forceinline__ void mix_init(Mix<K, C>& m, const float (&x)[C], float v_init)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        m.w[k] = k == 0 ? 1.f : 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) m.mu[c][k] = k == 0 ? x[c] : 0.f;
        m.v[k] = v_init;
    }
}

// One frame of one mixture at one pixel.  Returns the distance of x to the
// background set of the model as it stood before this frame's update.
// Steps: squared Mahalanobis distance per component; background set = shortest
// ranked prefix whose weight exceeds T_bg; first ranked match within lambda^2;
// weight decay toward the match; matched component moves toward x with
// rho = alpha / w (else the last-ranked component is replaced by x);
// normalisation; stable re-ranking by w / sqrt(v).
template <int K, int C>
__device__ __forceinline__ float mix_step(Mix<K, C>& m, const float (&x)[C], float alpha,
                                          float lam2, float T_bg, float v_init, float v_min)
{
    float ss[K], d2[K], diff[C][K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            diff[c][k] = __fsub_rn(x[c], m.mu[c][k]);
            s = __fmaf_rn(diff[c][k], diff[c][k], s);
        }
        ss[k] = s;
        d2[k] = __fdividef(s, __fmul_rn(float(C), m.v[k]));
    }
    float cum = 0.f, dB = INFINITY;
    bool open = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (open) {
            dB = fminf(dB, d2[k]);
            cum = __fadd_rn(cum, m.w[k]);
            open = !(cum > T_bg);
        }
    }
    int match = -1;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (match < 0 && d2[k] < lam2) match = k;

    const float oma = __fsub_rn(1.f, alpha);
#pragma unroll
    for (int k = 0; k < K; ++k) m.w[k] = __fmaf_rn(oma, m.w[k], k == match ? alpha : 0.f);
    if (match >= 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k == match) {
                const float rho = __fdividef(alpha, m.w[k]);
#pragma unroll
                for (int c = 0; c < C; ++c) m.mu[c][k] = __fmaf_rn(rho, diff[c][k], m.mu[c][k]);
                const float dv = __fsub_rn(__fmul_rn(ss[k], 1.f / float(C)), m.v[k]);
                const float v = __fmaf_rn(rho, dv, m.v[k]);
                m.v[k] = fmaxf(v, v_min);
            }
        }
    } else {
        m.w[K - 1] = alpha;
#pragma unroll
        for (int c = 0; c < C; ++c) m.mu[c][K - 1] = x[c];
        m.v[K - 1] = v_init;
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) s = __fadd_rn(s, m.w[k]);
    const float inv = __fdividef(1.f, s);
#pragma unroll
    for (int k = 0; k < K; ++k) m.w[k] = __fmul_rn(m.w[k], inv);

    float key[K];
    bool ranked = true;  // already in order: the network below would not swap
#pragma unroll
    for (int k = 0; k < K; ++k) {
        key[k] = __fmul_rn(m.w[k], rsqrtf(m.v[k]));
        if (k > 0) ranked &= !(key[k] > key[k - 1]);
    }
    if (ranked) return dB;
#pragma unroll
    for (int pass = 0; pass < K - 1; ++pass) {
#pragma unroll
        for (int j = 0; j < K - 1 - pass; ++j) {
            if (key[j + 1] > key[j]) {
                float t;
                t = key[j]; key[j] = key[j + 1]; key[j + 1] = t;
                t = m.w[j]; m.w[j] = m.w[j + 1]; m.w[j + 1] = t;
                t = m.v[j]; m.v[j] = m.v[j + 1]; m.v[j + 1] = t;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    t = m.mu[c][j]; m.mu[c][j] = m.mu[c][j + 1]; m.mu[c][j + 1] = t;
                }
            }
        }
    }
    return dB;
}

// PX floats of a state plane from element i (extent n: range-checked builds).
template <int PX>
__device__ __forceinline__ void ldv(const float* st, int64_t i, int64_t n, OobWord* w, float (&o)[PX])
{
    if constexpr (PX == 4) {
        const float4 v = vat<const float4>(st, i, 4, n, 40, w);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (PX == 2) {
        const float2 v = vat<const float2>(st, i, 2, n, 40, w);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = at(st, i, n, 40, w);
    }
}

template <int PX>
__device__ __forceinline__ void stv(float* st, int64_t i, int64_t n, OobWord* w, const float (&o)[PX])
{
    if constexpr (PX == 4) {
        vat<float4>(st, i, 4, n, 41, w) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (PX == 2) {
        vat<float2>(st, i, 2, n, 41, w) = make_float2(o[0], o[1]);
    } else {
        at(st, i, n, 41, w) = o[0];
    }
}

// Per-plane load/store of PX pixels of one parameter into the mixtures
// (n: elements of the whole state, for range-checked builds).
template <int KR, int KD, int PX, bool STORE>
__device__ __forceinline__ void move_state(float* st, int64_t plane, int64_t p0,
                                           Mix<KR, 3> (&mr)[PX], Mix<KD, 1> (&md)[PX],
                                           int64_t n = int64_t(1) << 62, OobWord* w = nullptr)
{
    float tmp[PX];
#define FOS_MOVE(QIDX, FIELD_I)                                            \
    {                                                                      \
        const int64_t idx = (int64_t)(QIDX) * plane + p0;                  \
        if (STORE) {                                                       \
            _Pragma("unroll") for (int i = 0; i < PX; ++i) tmp[i] = FIELD_I; \
            stv<PX>(st, idx, n, w, tmp);                                   \
        } else {                                                           \
            ldv<PX>(st, idx, n, w, tmp);                                   \
            _Pragma("unroll") for (int i = 0; i < PX; ++i) FIELD_I = tmp[i]; \
        }                                                                  \
    }
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        FOS_MOVE(k, mr[i].w[k]);
        FOS_MOVE(KR + k, mr[i].mu[0][k]);
        FOS_MOVE(2 * KR + k, mr[i].mu[1][k]);
        FOS_MOVE(3 * KR + k, mr[i].mu[2][k]);
        FOS_MOVE(4 * KR + k, mr[i].v[k]);
    }
#pragma unroll
    for (int k = 0; k < KD; ++k) {
        FOS_MOVE(5 * KR + k, md[i].w[k]);
        FOS_MOVE(5 * KR + KD + k, md[i].mu[0][k]);
        FOS_MOVE(5 * KR + 2 * KD + k, md[i].v[k]);
    }
#undef FOS_MOVE
}

// One pixel, inputs already converted: colour bytes and the 8-bit depth
// (0 = invalid reading).  Returns the mask byte.
template <int KR, int KD>
__device__ __forceinline__ uint8_t gmm_pixel_d8(Mix<KR, 3>& mr, Mix<KD, 1>& md, uint32_t r,
                                                uint32_t g, uint32_t b, uint32_t d8,
                                                const GmmArgs& a)
{
    const float xr[3] = {float(r), float(g), float(b)};
    const float xd[1] = {float(d8)};
    if (a.init) {
        mix_init(mr, xr, a.v_init_rgb);
        mix_init(md, xd, a.v_init_d);
        return 0;
    }
    const float dB_rgb = mix_step(mr, xr, a.alpha, a.lam2, a.T_bg, a.v_init_rgb, a.v_min_rgb);
    float Q = dB_rgb;
    if (d8 != 0) {
        const float dB_d = mix_step(md, xd, a.alpha, a.lam2, a.T_bg, a.v_init_d, a.v_min_d);
        Q = __fmaf_rn(a.w_depth, dB_d, __fmul_rn(__fsub_rn(1.f, a.w_depth), dB_rgb));
    }
    return Q >= a.lam2 ? 255 : 0;
}

// One mixture of one pixel moved between registers and its planes
// (first plane index q0: colour model 0, depth model 5*Kr).
template <int K, int C, bool STORE>
__device__ __forceinline__ void move_mix(float* st, int64_t plane, int64_t p, int q0, Mix<K, C>& m,
                                         int64_t n = int64_t(1) << 62, OobWord* ob = nullptr)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float& w = at(st, int64_t(q0 + k) * plane + p, n, 42, ob);
        float& v = at(st, int64_t(q0 + (1 + C) * K + k) * plane + p, n, 42, ob);
        if (STORE) { w = m.w[k]; v = m.v[k]; }
        else { m.w[k] = w; m.v[k] = v; }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float& mu = at(st, int64_t(q0 + (1 + c) * K + k) * plane + p, n, 42, ob);
            if (STORE) mu = m.mu[c][k];
            else m.mu[c][k] = mu;
        }
    }
}

// One mixture of two adjacent pixels (p even, plane 8-byte aligned) moved
// between registers and its planes with one 8-byte access per parameter.
template <int K, int C, bool STORE>
__device__ __forceinline__ void move_mix2(float* st, int64_t plane, int64_t p, int q0, Mix<K, C> (&m)[2],
                                          int64_t n = int64_t(1) << 62, OobWord* ob = nullptr)
{
    auto mv = [&](int q, float& a0, float& a1) {
        float2& ref = vat<float2>(st, int64_t(q) * plane + p, 2, n, 43, ob);
        if (STORE) {
            ref = make_float2(a0, a1);
        } else {
            const float2 v = ref;
            a0 = v.x;
            a1 = v.y;
        }
    };
#pragma unroll
    for (int k = 0; k < K; ++k) {
        mv(q0 + k, m[0].w[k], m[1].w[k]);
        mv(q0 + (1 + C) * K + k, m[0].v[k], m[1].v[k]);
#pragma unroll
        for (int c = 0; c < C; ++c) mv(q0 + (1 + c) * K + k, m[0].mu[c][k], m[1].mu[c][k]);
    }
}

// Two adjacent pixels (p even, inputs already converted: colour bytes r, g, b
// and the 8-bit depth, 0 = invalid reading), frames >= 1: the colour mixtures
// of both, then the depth mixtures of both (moved only if either reading is
// valid; a pixel with an invalid reading writes its model back unchanged).
// Returns the two mask bytes in bits 0-7 and 8-15.
template <int KR, int KD>
__device__ __forceinline__ uint32_t gmm_pair(const GmmArgs& a, int64_t p, const uint32_t (&r)[2],
                                             const uint32_t (&g)[2], const uint32_t (&b)[2],
                                             const uint32_t (&d8)[2])
{
    const int64_t ne = int64_t(5 * KR + 3 * KD) * a.plane;
    float Q[2];
    {
        Mix<KR, 3> mr[2];
        move_mix2<KR, 3, false>(a.state, a.plane, p, 0, mr, ne, a.oob);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float xr[3] = {float(r[i]), float(g[i]), float(b[i])};
            Q[i] = mix_step(mr[i], xr, a.alpha, a.lam2, a.T_bg, a.v_init_rgb, a.v_min_rgb);
        }
        move_mix2<KR, 3, true>(a.state, a.plane, p, 0, mr, ne, a.oob);
    }
    if (d8[0] | d8[1]) {
        Mix<KD, 1> md[2];
        move_mix2<KD, 1, false>(a.state, a.plane, p, 5 * KR, md, ne, a.oob);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            if (d8[i] != 0) {
                const float xd[1] = {float(d8[i])};
                const float dB_d = mix_step(md[i], xd, a.alpha, a.lam2, a.T_bg, a.v_init_d, a.v_min_d);
                Q[i] = __fmaf_rn(a.w_depth, dB_d, __fmul_rn(__fsub_rn(1.f, a.w_depth), Q[i]));
            }
        }
        move_mix2<KD, 1, true>(a.state, a.plane, p, 5 * KR, md, ne, a.oob);
    }
    return (Q[0] >= a.lam2 ? 0xFFu : 0u) | (Q[1] >= a.lam2 ? 0xFF00u : 0u);
}

// One pixel with the two mixtures handled one after the other (lower
// register peak than gmm_pixel_d8; same arithmetic, same bits).
template <int KR, int KD>
__device__ __forceinline__ uint8_t gmm_pixel_lowreg(const GmmArgs& a, int64_t p, uint32_t r,
                                                    uint32_t g, uint32_t b, uint32_t d8)
{
    const int64_t ne = int64_t(5 * KR + 3 * KD) * a.plane;
    float dB_rgb;
    {
        Mix<KR, 3> mr;
        const float xr[3] = {float(r), float(g), float(b)};
        if (a.init) {
            mix_init(mr, xr, a.v_init_rgb);
            dB_rgb = 0.f;
        } else {
            move_mix<KR, 3, false>(a.state, a.plane, p, 0, mr, ne, a.oob);
            dB_rgb = mix_step(mr, xr, a.alpha, a.lam2, a.T_bg, a.v_init_rgb, a.v_min_rgb);
        }
        move_mix<KR, 3, true>(a.state, a.plane, p, 0, mr, ne, a.oob);
    }
    float Q = dB_rgb;
    {
        Mix<KD, 1> md;
        const float xd[1] = {float(d8)};
        if (a.init) {
            mix_init(md, xd, a.v_init_d);
            move_mix<KD, 1, true>(a.state, a.plane, p, 5 * KR, md, ne, a.oob);
        } else if (d8 != 0) {
            move_mix<KD, 1, false>(a.state, a.plane, p, 5 * KR, md, ne, a.oob);
            const float dB_d = mix_step(md, xd, a.alpha, a.lam2, a.T_bg, a.v_init_d, a.v_min_d);
            move_mix<KD, 1, true>(a.state, a.plane, p, 5 * KR, md, ne, a.oob);
            Q = __fmaf_rn(a.w_depth, dB_d, __fmul_rn(__fsub_rn(1.f, a.w_depth), dB_rgb));
        }
    }
    if (a.init) return 0;
    return Q >= a.lam2 ? 255 : 0;
}

template <int KR, int KD>
__device__ __forceinline__ uint8_t gmm_pixel(Mix<KR, 3>& mr, Mix<KD, 1>& md, uint32_t r,
                                             uint32_t g, uint32_t b, uint32_t d16,
                                             const GmmArgs& a)
{
    return gmm_pixel_d8<KR, KD>(mr, md, r, g, b, depth_to_u8(d16, a.depth_fs), a);
}

}  // namespace gmmdev
}  // namespace fos
