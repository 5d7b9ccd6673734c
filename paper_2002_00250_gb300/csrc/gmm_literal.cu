// gmm_literal.cu -- the GMM of Sec. 3.1 as the paper prints it: K = 7 colour
// and 3 depth components in IEEE double ("float numbers on a 64 bit
// machine"), one variance per colour channel ("a single value for each colour
// component"), and a decision on the product of the two models' density
// factors, each the Eq. 1 density scaled by s.
//
// Per model (C channels; the depth model only where the reading is valid),
// pixel x, frame t >= 1, with the model before this frame's update:
//   D_k = sum_c (x_c - mu_kc)^2 / v_kc,   g_k = (prod_c v_kc)^(1/C)
//   background set B = shortest ranked prefix whose weight exceeds T_bg
//   F = s * sum_{k in B} w_k exp(-D_k / 2) / (2 pi g_k) / sum_{k in B} w_k
// (for one channel the density is Eq. 1 with sigma read as the variance).
// Foreground when F_rgb * F_d (depth valid) or F_rgb is below theta.
// Update per channel: match = first ranked k with D_k / C < lambda^2;
// w <- (1 - alpha) w + alpha [k = match]; matched: rho = alpha / w_k,
// mu_kc += rho (x_c - mu_kc), v_kc <- max(v_min, v_kc + rho ((x_c - mu_kc)^2
// - v_kc)); no match: the last-ranked component becomes (alpha, x, v_init);
// normalise; stable re-rank by w / sqrt(mean_c v_kc).
//
// State: double planes of `plane` elements; colour component k has planes
// w = k, mu_r/g/b = (1..3) Kr + k, v_r/g/b = (4..6) Kr + k; depth component
// k: w = 7 Kr + k, mu = 7 Kr + Kd + k, v = 7 Kr + 2 Kd + k.  One thread per
// pixel; the kernel is bound by FP64 arithmetic (exp, pow) rather than HBM.
#include <cmath>

#include "fos.h"
#include "fos_internal.h"

namespace fos {
namespace {

constexpr int kLitThreads = 128;

template <int K, int C>
struct DMix {
    double w[K];
    double mu[K][C];
    double v[K][C];
};

__device__ __forceinline__ uint32_t lit_depth_u8(uint32_t d, uint32_t fs)
{
    if (d == 0) return 0;
    const uint32_t q = (d * 255u + (fs >> 1)) / fs;
    return q < 1u ? 1u : (q > 255u ? 255u : q);
}

// One model, one frame: returns the density factor F of x under the
// pre-update background set, then updates m in place.
template <int K, int C>
__device__ double lit_step(DMix<K, C>& m, const double (&x)[C], const GmmLiteralArgs& a, double v_init,
                           double v_min)
{
    const double two_pi = 6.283185307179586476925286766559;
    double D[K], diff[K][C];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        D[k] = 0.0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            diff[k][c] = x[c] - m.mu[k][c];
            D[k] += diff[k][c] * diff[k][c] / m.v[k][c];
        }
    }
    double cum = 0.0, num = 0.0, den = 0.0;
    bool open = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (open) {
            double g = 1.0;
#pragma unroll
            for (int c = 0; c < C; ++c) g *= m.v[k][c];
            if (C > 1) g = pow(g, 1.0 / double(C));
            num += m.w[k] * exp(-0.5 * D[k]) / (two_pi * g);
            den += m.w[k];
            cum += m.w[k];
            open = !(cum > a.T_bg);
        }
    }
    const double F = a.s * num / den;
    int match = -1;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (match < 0 && D[k] / double(C) < a.lam2) match = k;
#pragma unroll
    for (int k = 0; k < K; ++k) m.w[k] = (1.0 - a.alpha) * m.w[k] + (k == match ? a.alpha : 0.0);
    if (match >= 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k != match) continue;
            const double rho = a.alpha / m.w[k];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                m.mu[k][c] = m.mu[k][c] + rho * diff[k][c];
                const double v = m.v[k][c] + rho * (diff[k][c] * diff[k][c] - m.v[k][c]);
                m.v[k][c] = v > v_min ? v : v_min;
            }
        }
    } else {
        m.w[K - 1] = a.alpha;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            m.mu[K - 1][c] = x[c];
            m.v[K - 1][c] = v_init;
        }
    }
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) sum += m.w[k];
#pragma unroll
    for (int k = 0; k < K; ++k) m.w[k] = m.w[k] / sum;
    double key[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double vb = 0.0;
#pragma unroll
        for (int c = 0; c < C; ++c) vb += m.v[k][c];
        key[k] = m.w[k] / sqrt(vb / double(C));
    }
    // stable insertion sort, descending (equal keys keep their order)
#pragma unroll
    for (int i = 1; i < K; ++i) {
#pragma unroll
        for (int j = i; j > 0; --j) {
            if (!(key[j] > key[j - 1])) break;
            double t = key[j]; key[j] = key[j - 1]; key[j - 1] = t;
            t = m.w[j]; m.w[j] = m.w[j - 1]; m.w[j - 1] = t;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                t = m.mu[j][c]; m.mu[j][c] = m.mu[j - 1][c]; m.mu[j - 1][c] = t;
                t = m.v[j][c]; m.v[j][c] = m.v[j - 1][c]; m.v[j - 1][c] = t;
            }
        }
    }
    return F;
}

template <int K, int C, bool STORE>
__device__ __forceinline__ void lit_move(double* st, int64_t plane, int64_t p, int q0, DMix<K, C>& m)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double* w = st + int64_t(q0 + k) * plane + p;
        if (STORE) *w = m.w[k];
        else m.w[k] = *w;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            double* mu = st + int64_t(q0 + (1 + c) * K + k) * plane + p;
            double* v = st + int64_t(q0 + (1 + C + c) * K + k) * plane + p;
            if (STORE) { *mu = m.mu[k][c]; *v = m.v[k][c]; }
            else { m.mu[k][c] = *mu; m.v[k][c] = *v; }
        }
    }
}

template <int KR, int KD>
__global__ void __launch_bounds__(kLitThreads) gmm_literal_kernel(const GmmLiteralArgs a)
{
    const int64_t p = int64_t(blockIdx.x) * kLitThreads + threadIdx.x;
    if (p >= a.P) return;
    const double xr[3] = {double(a.rgb[3 * p]), double(a.rgb[3 * p + 1]), double(a.rgb[3 * p + 2])};
    const int y = int(p / a.W), x = int(p - int64_t(y) * a.W);
    const uint32_t d8 = lit_depth_u8(a.depth[depth_index(x, y, a.W, a.H, a.Wd, a.Hd)], a.depth_fs);
    const double xd[1] = {double(d8)};
    double F;
    {
        DMix<KR, 3> mr;
        if (a.init) {
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                mr.w[k] = k == 0 ? 1.0 : 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    mr.mu[k][c] = k == 0 ? xr[c] : 0.0;
                    mr.v[k][c] = a.v_init_rgb;
                }
            }
            F = a.theta;
        } else {
            lit_move<KR, 3, false>(a.state, a.plane, p, 0, mr);
            F = lit_step<KR, 3>(mr, xr, a, a.v_init_rgb, a.v_min_rgb);
        }
        lit_move<KR, 3, true>(a.state, a.plane, p, 0, mr);
    }
    {
        DMix<KD, 1> md;
        if (a.init) {
#pragma unroll
            for (int k = 0; k < KD; ++k) {
                md.w[k] = k == 0 ? 1.0 : 0.0;
                md.mu[k][0] = k == 0 ? xd[0] : 0.0;
                md.v[k][0] = a.v_init_d;
            }
            lit_move<KD, 1, true>(a.state, a.plane, p, 7 * KR, md);
        } else if (d8 != 0) {
            lit_move<KD, 1, false>(a.state, a.plane, p, 7 * KR, md);
            F *= lit_step<KD, 1>(md, xd, a, a.v_init_d, a.v_min_d);
            lit_move<KD, 1, true>(a.state, a.plane, p, 7 * KR, md);
        }
    }
    a.mask[p] = (a.init || F >= a.theta) ? 0 : 255;
}

}  // namespace

int gmm_literal_planes(int Kr, int Kd) { return 7 * Kr + 3 * Kd; }

bool gmm_literal_supported(int Kr, int Kd) { return (Kr == 7 && Kd == 3) || (Kr == 3 && Kd == 3); }

LaunchResult launch_gmm_literal(const GmmLiteralArgs& a, int Kr, int Kd, cudaStream_t s)
{
    if (a.P == 0) return kLaunchOk;
    const unsigned blocks = unsigned((a.P + kLitThreads - 1) / kLitThreads);
    if (Kr == 7 && Kd == 3) gmm_literal_kernel<7, 3><<<blocks, kLitThreads, 0, s>>>(a);
    else if (Kr == 3 && Kd == 3) gmm_literal_kernel<3, 3><<<blocks, kLitThreads, 0, s>>>(a);
    else return kLaunchUnsupported;
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

}  // namespace fos
