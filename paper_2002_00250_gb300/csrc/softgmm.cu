// softgmm.cu -- differentiable (soft) GMM over RGB-D sequences: forward with
// checkpoints, and its hand-written adjoint.
//
// The paper's GMM (Sec. 3.1, Eq. 1) decides hard matches; here the match test
// is a sigmoid of (L - d_k) / tau so a mask loss (mean BCE against ground
// truth) has gradients with respect to theta = (alpha, L = lambda^2, w, v0).
// Per model and frame (see the oracle's docstring for the same definition):
//   d_k = ||x - mu_k||^2 / (C v_k); m_k = sigmoid((L - d_k) / tau);
//   r_k = m_k prod_{j<k}(1 - m_j); q = prod_k (1 - m_k);
//   w1 = (1-alpha) w + alpha r; rho = alpha r / w1 (1 for a never-used component);
//   mu1 = mu + rho (x - mu); v1 = max(v_min, v + rho(||x-mu||^2/C - v));
//   last-ranked component blended with weight q toward (alpha, x, v_init);
//   normalise; stable re-rank by w / sqrt(v).
// Classification uses the pre-update model: delta = d at the first arg-min
// over the hard background set; Q = (1-w) delta_rgb + w delta_d (depth valid);
// p = sigmoid((Q - L) / tau).  Ranks, background sets, arg-mins and v_min
// clamps are decisions of the forward, held constant in the adjoint.
//
// One thread owns one pixel of one sequence for the whole sequence.  The
// forward stores the state every `ckpt` frames; the adjoint walks the
// segments from last to first, recomputes the segment's states from its
// checkpoint into thread-local storage, then runs the frames backwards.
// Loss and parameter gradients are reduced per block into fixed slots and
// summed by one block in a fixed order (deterministic).
//
// Every routine is written once for the real type R: R = float is the fast
// path; R = double (fos_softgmm_params.fp64) runs the same recurrence, its
// checkpoints and its adjoint in double precision, so that its gradient can be
// held to finite differences of its own forward and to the FP64 definition at
// 1e-5 relative (an FP32 recurrence over tens of frames drifts to 1e-4).
#include <cstdio>
#include <string>

#include "fos.h"
#include "fos_internal.h"

namespace fos {
namespace {

constexpr int KR = 3, KD = 3;          // components (colour, depth)
constexpr int NQ = 5 * KR + 3 * KD;    // state floats per pixel (24)
constexpr int kMaxSeg = 16;            // largest checkpoint interval
constexpr int kThreads = 128;

template <typename R>
struct Theta {
    R alpha, L, w, v0, tau, T_bg, vmin_rgb, vmin_d, ratio;
    uint32_t depth_fs;
};

template <typename R>
struct SoftArgs {
    int64_t P;         // pixels per frame
    int B, T, ck;      // sequences, frames, checkpoint interval
    const uint8_t* rgb;     // [B][T][P][3]
    const uint16_t* depth;  // [B][T][P]
    const uint8_t* gt;      // [B][T][P]
    R* chk;                 // [ceil..][NQ][B*P]
    int nchk;
    double* part;           // [gridDim][5] per-block partial sums
    float* pixel_grad;      // nullable [B*P][4]
    Theta<R> th;
    double scale;           // 1 / (B (T-1) P)
};

template <int K, int C, typename R>
struct SMix {
    R w[K];
    R mu[K][C];
    R v[K];
};

template <int K, int C, typename R>
struct SFwd {
    R e[K][C], s[K], d[K], m[K], Pp[K + 1], r[K], q, w1[K], rho[K];
    bool clamp[K], unused[K];
    R mu1[K][C], v1[K], w2[K], v2[K], sum, w3[K];
    int rank[K];  // output position of component k after the re-rank
};

template <typename R>
struct State {
    SMix<KR, 3, R> c;
    SMix<KD, 1, R> d;
};

// exp, log1p, sqrt of the working precision
__device__ __forceinline__ float rexp(float x) { return expf(x); }
__device__ __forceinline__ double rexp(double x) { return exp(x); }
__device__ __forceinline__ float rlog1p(float x) { return log1pf(x); }
__device__ __forceinline__ double rlog1p(double x) { return log1p(x); }
__device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }

__device__ __forceinline__ uint32_t depth_u8(uint32_t d, uint32_t fs)
{
    if (d == 0) return 0;
    uint32_t q = (d * 255u + (fs >> 1)) / fs;
    return q < 1u ? 1u : (q > 255u ? 255u : q);
}

template <typename R>
__device__ __forceinline__ R sigm(R z) { return R(1) / (R(1) + rexp(-z)); }

// log(1 + e^a) without overflow
template <typename R>
__device__ __forceinline__ R softplus(R a) { return a > R(0) ? a + rlog1p(rexp(-a)) : rlog1p(rexp(a)); }

template <int K, int C, typename R>
__device__ __forceinline__ void mix_init(SMix<K, C, R>& m, const R (&x)[C], R v_init)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        m.w[k] = k == 0 ? R(1) : R(0);
#pragma unroll
        for (int c = 0; c < C; ++c) m.mu[k][c] = k == 0 ? x[c] : R(0);
        m.v[k] = v_init;
    }
}

// Pre-update distances and the background-set arg-min (first on ties).
template <int K, int C, typename R>
__device__ __forceinline__ R classify(const SMix<K, C, R>& m, const R (&x)[C], R T_bg, int& kstar)
{
    R cum = R(0), best = R(INFINITY);
    bool open = true;
    kstar = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        R s = R(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const R e = x[c] - m.mu[k][c];
            s = fma(e, e, s);
        }
        const R d = s / (R(C) * m.v[k]);
        if (open && d < best) {
            best = d;
            kstar = k;
        }
        cum += m.w[k];
        open = open && !(cum > T_bg);
    }
    return best;
}

template <int K, int C, typename R>
__device__ __forceinline__ void mix_fwd(const SMix<K, C, R>& in, const R (&x)[C], R alpha, R L,
                                        R tau, R v_init, R v_min, SFwd<K, C, R>& f, SMix<K, C, R>& out)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        R s = R(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            f.e[k][c] = x[c] - in.mu[k][c];
            s = fma(f.e[k][c], f.e[k][c], s);
        }
        f.s[k] = s;
        f.d[k] = s / (R(C) * in.v[k]);
        f.m[k] = sigm((L - f.d[k]) / tau);
    }
    f.Pp[0] = R(1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        f.r[k] = f.m[k] * f.Pp[k];
        f.Pp[k + 1] = f.Pp[k] * (R(1) - f.m[k]);
    }
    f.q = f.Pp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        f.w1[k] = (R(1) - alpha) * in.w[k] + alpha * f.r[k];
        f.unused[k] = in.w[k] == R(0);
        f.rho[k] = f.unused[k] ? (f.r[k] > R(0) ? R(1) : R(0)) : alpha * f.r[k] / f.w1[k];
#pragma unroll
        for (int c = 0; c < C; ++c) f.mu1[k][c] = in.mu[k][c] + f.rho[k] * f.e[k][c];
        const R u = in.v[k] + f.rho[k] * (f.s[k] / R(C) - in.v[k]);
        f.clamp[k] = u > v_min;
        f.v1[k] = f.clamp[k] ? u : v_min;
        f.w2[k] = f.w1[k];
        f.v2[k] = f.v1[k];
    }
    R mu2[K][C];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < C; ++c) mu2[k][c] = f.mu1[k][c];
    {
        constexpr int l = K - 1;
        const R q = f.q;
        f.w2[l] = (R(1) - q) * f.w1[l] + q * alpha;
#pragma unroll
        for (int c = 0; c < C; ++c) mu2[l][c] = (R(1) - q) * f.mu1[l][c] + q * x[c];
        f.v2[l] = (R(1) - q) * f.v1[l] + q * v_init;
    }
    f.sum = R(0);
#pragma unroll
    for (int k = 0; k < K; ++k) f.sum += f.w2[k];
    R key[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        f.w3[k] = f.w2[k] / f.sum;
        key[k] = f.w3[k] / rsqrt_(f.v2[k]);
    }
    // stable descending order of the keys: component k goes to position
    // #{j < k: key_j >= key_k} + #{j > k: key_j > key_k}.  Ranks come from
    // comparisons and the outputs from predicated selects, so that no array
    // is indexed by a run-time value (which would move the state to local memory).
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (j != k) r += (j < k ? key[j] >= key[k] : key[j] > key[k]) ? 1 : 0;
        f.rank[k] = r;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        R w = f.w3[0], v = f.v2[0], mu[C];
#pragma unroll
        for (int c = 0; c < C; ++c) mu[c] = mu2[0][c];
#pragma unroll
        for (int kk = 1; kk < K; ++kk) {
            const bool here = f.rank[kk] == i;
            w = here ? f.w3[kk] : w;
            v = here ? f.v2[kk] : v;
#pragma unroll
            for (int c = 0; c < C; ++c) mu[c] = here ? mu2[kk][c] : mu[c];
        }
        out.w[i] = w;
        out.v[i] = v;
#pragma unroll
        for (int c = 0; c < C; ++c) out.mu[i][c] = mu[c];
    }
}

// Adjoint of one model step.  gout: adjoint of the (ranked) output;
// gcls_k: adjoint of d_k from the classification.  Writes the adjoint of the
// input state and adds to the parameter gradients.
template <int K, int C, typename R>
__device__ __forceinline__ void mix_bwd(const SMix<K, C, R>& in, const R (&x)[C], R alpha, R tau,
                                        R v_init, const SFwd<K, C, R>& f, const SMix<K, C, R>& gout,
                                        const R (&gcls)[K], SMix<K, C, R>& gin, R& ga, R& gL,
                                        R& gvi)
{
    R gw3[K], gmu2[K][C], gv2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        R w = gout.w[0], v = gout.v[0], mu[C];
#pragma unroll
        for (int c = 0; c < C; ++c) mu[c] = gout.mu[0][c];
#pragma unroll
        for (int i = 1; i < K; ++i) {
            const bool here = f.rank[k] == i;
            w = here ? gout.w[i] : w;
            v = here ? gout.v[i] : v;
#pragma unroll
            for (int c = 0; c < C; ++c) mu[c] = here ? gout.mu[i][c] : mu[c];
        }
        gw3[k] = w;
        gv2[k] = v;
#pragma unroll
        for (int c = 0; c < C; ++c) gmu2[k][c] = mu[c];
    }
    // w3 = w2 / sum
    R dot = R(0);
#pragma unroll
    for (int k = 0; k < K; ++k) dot += gw3[k] * f.w3[k];
    R gw1[K], gmu1[K][C], gv1[K], gq = R(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        gw1[k] = (gw3[k] - dot) / f.sum;
        gv1[k] = gv2[k];
#pragma unroll
        for (int c = 0; c < C; ++c) gmu1[k][c] = gmu2[k][c];
    }
    {
        constexpr int l = K - 1;
        const R q = f.q, gw2l = gw1[l];
        gw1[l] = (R(1) - q) * gw2l;
        gq += (alpha - f.w1[l]) * gw2l;
        ga += q * gw2l;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            gq += (x[c] - f.mu1[l][c]) * gmu2[l][c];
            gmu1[l][c] = (R(1) - q) * gmu2[l][c];
        }
        gq += (v_init - f.v1[l]) * gv2[l];
        gvi += q * gv2[l];
        gv1[l] = (R(1) - q) * gv2[l];
    }
    R gr[K], gs[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        // v1 = clamp ? v + rho (s/C - v) : v_min
        const R gu = f.clamp[k] ? gv1[k] : R(0);
        R grho = gu * (f.s[k] / R(C) - in.v[k]);
        gs[k] = gu * f.rho[k] / R(C);
        gin.v[k] = gu * (R(1) - f.rho[k]);
        // mu1 = mu + rho (x - mu)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            gin.mu[k][c] = gmu1[k][c] * (R(1) - f.rho[k]);
            grho += f.e[k][c] * gmu1[k][c];
        }
        // rho = alpha r / w1 (constant for a never-used component)
        gr[k] = R(0);
        if (!f.unused[k]) {
            ga += grho * f.r[k] / f.w1[k];
            gr[k] += grho * alpha / f.w1[k];
            gw1[k] -= grho * f.rho[k] / f.w1[k];
        }
        // w1 = (1 - alpha) w + alpha r
        gin.w[k] = (R(1) - alpha) * gw1[k];
        ga += (f.r[k] - in.w[k]) * gw1[k];
        gr[k] += alpha * gw1[k];
    }
    // r_k = m_k P_k, P_{k+1} = P_k (1 - m_k), q = P_K
    R gP = gq;
    R gm[K];
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        gm[k] = f.Pp[k] * gr[k] - f.Pp[k] * gP;
        gP = f.m[k] * gr[k] + (R(1) - f.m[k]) * gP;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        // m = sigmoid((L - d) / tau)
        const R gz = f.m[k] * (R(1) - f.m[k]) * gm[k];
        gL += gz / tau;
        const R gd = -gz / tau + gcls[k];
        // d = s / (C v)
        gs[k] += gd / (R(C) * in.v[k]);
        gin.v[k] -= gd * f.d[k] / in.v[k];
        // s = sum (x - mu)^2
#pragma unroll
        for (int c = 0; c < C; ++c) gin.mu[k][c] -= R(2) * f.e[k][c] * gs[k];
    }
}

template <typename R>
__device__ __forceinline__ void load_frame(const SoftArgs<R>& a, int b, int t, int64_t p, R (&xc)[3],
                                           R (&xd)[1], bool& valid, R& y)
{
    const int64_t o = (int64_t(b) * a.T + t) * a.P + p;
    xc[0] = a.rgb[3 * o];
    xc[1] = a.rgb[3 * o + 1];
    xc[2] = a.rgb[3 * o + 2];
    const uint32_t d8 = depth_u8(a.depth[o], a.th.depth_fs);
    xd[0] = R(d8);
    valid = d8 != 0;
    y = a.gt[o] ? R(1) : R(0);
}

template <typename R>
__device__ __forceinline__ void state_io(R* base, int64_t stride, State<R>& s, bool store)
{
    int q = 0;
#define FOS_IO(v)                                                \
    {                                                            \
        if (store) base[int64_t(q) * stride] = (v);              \
        else (v) = base[int64_t(q) * stride];                    \
        ++q;                                                     \
    }
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        FOS_IO(s.c.w[k]) FOS_IO(s.c.v[k])
#pragma unroll
        for (int c = 0; c < 3; ++c) FOS_IO(s.c.mu[k][c])
    }
#pragma unroll
    for (int k = 0; k < KD; ++k) { FOS_IO(s.d.w[k]) FOS_IO(s.d.v[k]) FOS_IO(s.d.mu[k][0]) }
#undef FOS_IO
}

// One frame forward: returns the loss term; advances the state.
template <typename R>
__device__ __forceinline__ R frame_fwd(const SoftArgs<R>& a, State<R>& s, const R (&xc)[3],
                                           const R (&xd)[1], bool valid, R y)
{
    const Theta<R>& th = a.th;
    int kc, kd;
    const R dc = classify(s.c, xc, th.T_bg, kc);
    R Q = dc;
    if (valid) {
        const R dd = classify(s.d, xd, th.T_bg, kd);
        Q = (R(1) - th.w) * dc + th.w * dd;
    }
    const R z = (Q - th.L) / th.tau;
    const R loss = softplus(z) - y * z;
    SFwd<KR, 3, R> fc;
    SMix<KR, 3, R> oc;
    mix_fwd(s.c, xc, th.alpha, th.L, th.tau, th.v0, th.vmin_rgb, fc, oc);
    s.c = oc;
    if (valid) {
        SFwd<KD, 1, R> fd;
        SMix<KD, 1, R> od;
        mix_fwd(s.d, xd, th.alpha, th.L, th.tau, th.v0 * th.ratio, th.vmin_d, fd, od);
        s.d = od;
    }
    return loss;
}

template <typename R>
__device__ __forceinline__ void frame0(const SoftArgs<R>& a, State<R>& s, const R (&xc)[3], const R (&xd)[1])
{
    mix_init(s.c, xc, a.th.v0);
    mix_init(s.d, xd, a.th.v0 * a.th.ratio);
}

template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* out)
{
    __shared__ double red[NV][kThreads / 32];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
        out[int64_t(blockIdx.x) * NV + threadIdx.x] = s;
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) soft_forward_kernel(const SoftArgs<R> a)
{
    const int64_t gid = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t BP = int64_t(a.B) * a.P;
    double part[1] = {0.0};
    if (gid < BP) {
        const int b = int(gid / a.P);
        const int64_t p = gid - int64_t(b) * a.P;
        State<R> s;
        R xc[3], xd[1], y;
        bool valid;
        load_frame(a, b, 0, p, xc, xd, valid, y);
        frame0(a, s, xc, xd);
        state_io(a.chk + gid, BP, s, true);
        double acc = 0.0;
        for (int t = 1; t < a.T; ++t) {
            load_frame(a, b, t, p, xc, xd, valid, y);
            acc += frame_fwd(a, s, xc, xd, valid, y);
            if (t % a.ck == 0 && t / a.ck < a.nchk)
                state_io(a.chk + int64_t(t / a.ck) * NQ * BP + gid, BP, s, true);
        }
        part[0] = acc * a.scale;
    }
    block_partials<1>(part, a.part);
}

// Adjoint of one frame: ga (adjoint of the state after the frame) becomes the
// adjoint of the state before it; parameter gradients accumulate in g[4].
template <typename R>
__device__ __forceinline__ void frame_bwd(const SoftArgs<R>& a, const State<R>& sp, const R (&xc)[3],
                                          const R (&xd)[1], bool valid, R y, State<R>& ga, R (&g)[4])
{
    const Theta<R>& th = a.th;
    int kc = 0, kd = 0;
    const R dc = classify(sp.c, xc, th.T_bg, kc);
    R dd = R(0), Q = dc;
    if (valid) {
        dd = classify(sp.d, xd, th.T_bg, kd);
        Q = (R(1) - th.w) * dc + th.w * dd;
    }
    const R z = (Q - th.L) / th.tau;
    const R gz = (sigm(z) - y) * R(a.scale);  // d loss / d z
    const R gQ = gz / th.tau;
    g[1] -= gz / th.tau;
    R gcls_c[KR], gcls_d[KD];
#pragma unroll
    for (int k = 0; k < KR; ++k) gcls_c[k] = R(0);
#pragma unroll
    for (int k = 0; k < KD; ++k) gcls_d[k] = R(0);
    const R gdc = valid ? (R(1) - th.w) * gQ : gQ;
#pragma unroll
    for (int k = 0; k < KR; ++k)
        if (k == kc) gcls_c[k] = gdc;
    if (valid) {
        g[2] += (dd - dc) * gQ;
#pragma unroll
        for (int k = 0; k < KD; ++k)
            if (k == kd) gcls_d[k] = th.w * gQ;
    }
    R gvi_c = R(0), gvi_d = R(0);
    {
        SFwd<KR, 3, R> f;
        SMix<KR, 3, R> out, gin;
        mix_fwd(sp.c, xc, th.alpha, th.L, th.tau, th.v0, th.vmin_rgb, f, out);
        mix_bwd(sp.c, xc, th.alpha, th.tau, th.v0, f, ga.c, gcls_c, gin, g[0], g[1], gvi_c);
        ga.c = gin;
    }
    if (valid) {
        SFwd<KD, 1, R> f;
        SMix<KD, 1, R> out, gin;
        mix_fwd(sp.d, xd, th.alpha, th.L, th.tau, th.v0 * th.ratio, th.vmin_d, f, out);
        mix_bwd(sp.d, xd, th.alpha, th.tau, th.v0 * th.ratio, f, ga.d, gcls_d, gin, g[0], g[1], gvi_d);
        ga.d = gin;
    }
    g[3] += gvi_c + th.ratio * gvi_d;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) soft_backward_kernel(const SoftArgs<R> a)
{
    const int64_t gid = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t BP = int64_t(a.B) * a.P;
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    if (gid < BP) {
        const int b = int(gid / a.P);
        const int64_t p = gid - int64_t(b) * a.P;
        State<R> ga;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            ga.c.w[k] = ga.c.v[k] = R(0);
            ga.c.mu[k][0] = ga.c.mu[k][1] = ga.c.mu[k][2] = R(0);
        }
#pragma unroll
        for (int k = 0; k < KD; ++k) ga.d.w[k] = ga.d.v[k] = ga.d.mu[k][0] = R(0);
        R g[4] = {R(0), R(0), R(0), R(0)};
        State<R> seg[kMaxSeg];  // states before each frame of the segment
        R xc[3], xd[1], y;
        bool valid;
        for (int j = a.nchk - 1; j >= 0; --j) {
            const int t0 = j * a.ck + 1, t1 = min(a.T - 1, (j + 1) * a.ck);
            if (t0 > t1) continue;
            State<R> s;
            state_io(a.chk + int64_t(j) * NQ * BP + gid, BP, s, false);
            for (int t = t0; t <= t1; ++t) {
                seg[t - t0] = s;
                load_frame(a, b, t, p, xc, xd, valid, y);
                frame_fwd(a, s, xc, xd, valid, y);
            }
            for (int t = t1; t >= t0; --t) {
                load_frame(a, b, t, p, xc, xd, valid, y);
                frame_bwd(a, seg[t - t0], xc, xd, valid, y, ga, g);
            }
        }
        // frame 0: every component starts with v = v_init (colour v0, depth v0 * ratio)
#pragma unroll
        for (int k = 0; k < KR; ++k) g[3] += ga.c.v[k];
#pragma unroll
        for (int k = 0; k < KD; ++k) g[3] += a.th.ratio * ga.d.v[k];
        if (a.pixel_grad) {
#pragma unroll
            for (int q = 0; q < 4; ++q) a.pixel_grad[gid * 4 + q] = float(g[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) part[q] = g[q];
    }
    block_partials<4>(part, a.part);
}

// Sums nb rows of nv partials in a fixed order (one block).
__global__ void reduce_partials_kernel(const double* part, int nb, int nv, double* out)
{
    __shared__ double buf[256];
    for (int q = 0; q < nv; ++q) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[int64_t(i) * nv + q];
        buf[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = buf[0];
        __syncthreads();
    }
}

}  // namespace
}  // namespace fos

using namespace fos;

struct fos_softgmm {
    int W = 0, H = 0, B = 0, T = 0;
    fos_softgmm_params prm{};
    double theta[4] = {0, 0, 0, 0};  // alpha, lambda2, w_depth, v_init_rgb as given
    void* chk = nullptr;              // checkpoints, float or double (prm.fp64)
    int nchk = 0;
    double* part = nullptr;  // [blocks][4] + result [8]
    int blocks = 0;
    bool have_forward = false;
    std::string err;
};

namespace {

fos_status sg_fail(fos_softgmm* g, fos_status st, const char* what, cudaError_t e = cudaSuccess)
{
    char buf[400];
    if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    else std::snprintf(buf, sizeof buf, "%s", what);
    if (g) g->err = buf;
    set_thread_error(buf);
    return st;
}

template <typename R>
SoftArgs<R> make_args(fos_softgmm* g, const uint8_t* rgb, const uint16_t* depth, const uint8_t* gt, float* pixel_grad)
{
    SoftArgs<R> a{};
    const fos_softgmm_params& p = g->prm;
    a.P = int64_t(g->W) * g->H;
    a.B = g->B; a.T = g->T; a.ck = p.ckpt_every;
    a.rgb = rgb; a.depth = depth; a.gt = gt;
    a.chk = static_cast<R*>(g->chk); a.nchk = g->nchk; a.part = g->part; a.pixel_grad = pixel_grad;
    a.th.alpha = R(g->theta[0]); a.th.L = R(g->theta[1]); a.th.w = R(g->theta[2]); a.th.v0 = R(g->theta[3]);
    a.th.tau = p.tau; a.th.T_bg = p.T_bg; a.th.vmin_rgb = p.v_min_rgb; a.th.vmin_d = p.v_min_d;
    a.th.ratio = p.v_init_d_ratio; a.th.depth_fs = p.depth_full_scale_mm;
    a.scale = 1.0 / (double(g->B) * double(g->T - 1) * double(a.P));
    return a;
}

void launch_forward(fos_softgmm* g, const uint8_t* rgb, const uint16_t* depth, const uint8_t* gt, cudaStream_t s)
{
    if (g->prm.fp64) soft_forward_kernel<double><<<g->blocks, kThreads, 0, s>>>(make_args<double>(g, rgb, depth, gt, nullptr));
    else soft_forward_kernel<float><<<g->blocks, kThreads, 0, s>>>(make_args<float>(g, rgb, depth, gt, nullptr));
}

void launch_backward(fos_softgmm* g, const uint8_t* rgb, const uint16_t* depth, const uint8_t* gt, float* pg,
                     cudaStream_t s)
{
    if (g->prm.fp64) soft_backward_kernel<double><<<g->blocks, kThreads, 0, s>>>(make_args<double>(g, rgb, depth, gt, pg));
    else soft_backward_kernel<float><<<g->blocks, kThreads, 0, s>>>(make_args<float>(g, rgb, depth, gt, pg));
}

}  // namespace

extern "C" {

void fos_softgmm_default_params(fos_softgmm_params* p)
{
    if (!p) return;
    p->alpha = 0.001f;
    p->lambda2 = 6.25f;
    p->w_depth = 0.5f;
    p->v_init_rgb = 36.f;
    p->tau = 0.25f;
    p->T_bg = 0.7f;
    p->v_min_rgb = 4.f;
    p->v_min_d = 0.25f;
    p->v_init_d_ratio = 4.f / 36.f;
    p->K_rgb = 3;
    p->K_d = 3;
    p->ckpt_every = 8;
    p->depth_full_scale_mm = 10000;
    p->fp64 = 0;
}

fos_softgmm* fos_softgmm_create(int32_t width, int32_t height, int32_t batch, int32_t frames,
                                const fos_softgmm_params* params)
{
    if (!params || width < 1 || height < 1 || batch < 1 || frames < 2) {
        sg_fail(nullptr, FOS_ERR_INVALID_ARG, "fos_softgmm_create: bad size");
        return nullptr;
    }
    if (params->K_rgb != KR || params->K_d != KD || params->ckpt_every < 1 || params->ckpt_every > kMaxSeg ||
        !(params->tau > 0.f) || params->depth_full_scale_mm == 0 || (params->fp64 != 0 && params->fp64 != 1)) {
        sg_fail(nullptr, FOS_ERR_UNSUPPORTED,
                "fos_softgmm_create: needs K = 3 + 3, 1 <= ckpt_every <= 16, tau > 0, fp64 0 or 1");
        return nullptr;
    }
    fos_softgmm* g = new fos_softgmm();
    g->W = width; g->H = height; g->B = batch; g->T = frames; g->prm = *params;
    g->theta[0] = params->alpha; g->theta[1] = params->lambda2;
    g->theta[2] = params->w_depth; g->theta[3] = params->v_init_rgb;
    g->nchk = (frames - 1) / params->ckpt_every + 1;
    const int64_t BP = int64_t(batch) * width * height;
    g->blocks = int((BP + kThreads - 1) / kThreads);
    const size_t elem = params->fp64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaMalloc(&g->chk, size_t(g->nchk) * NQ * size_t(BP) * elem);
    if (e == cudaSuccess) e = cudaMalloc(&g->part, (size_t(g->blocks) * 4 + 8) * sizeof(double));
    if (e != cudaSuccess) {
        sg_fail(nullptr, e == cudaErrorMemoryAllocation ? FOS_ERR_OOM : FOS_ERR_CUDA, "fos_softgmm_create", e);
        fos_softgmm_destroy(g);
        return nullptr;
    }
    return g;
}

void fos_softgmm_destroy(fos_softgmm* g)
{
    if (!g) return;
    cudaFree(g->chk);
    cudaFree(g->part);
    delete g;
}

const char* fos_softgmm_last_error(const fos_softgmm* g) { return g ? g->err.c_str() : ""; }

fos_status fos_softgmm_set_theta(fos_softgmm* g, const float theta[4])
{
    if (!g || !theta) return FOS_ERR_INVALID_ARG;
    const double t64[4] = {theta[0], theta[1], theta[2], theta[3]};
    return fos_softgmm_set_theta64(g, t64);
}

fos_status fos_softgmm_set_theta64(fos_softgmm* g, const double theta[4])
{
    if (!g || !theta) return FOS_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i) g->theta[i] = theta[i];
    g->prm.alpha = float(theta[0]);
    g->prm.lambda2 = float(theta[1]);
    g->prm.w_depth = float(theta[2]);
    g->prm.v_init_rgb = float(theta[3]);
    g->have_forward = false;
    return FOS_OK;
}

fos_status fos_softgmm_forward(fos_softgmm* g, const uint8_t* d_rgb, const uint16_t* d_depth,
                               const uint8_t* d_gt, double* loss_out, void* stream)
{
    if (!g || !d_rgb || !d_depth || !d_gt || !loss_out) return sg_fail(g, FOS_ERR_INVALID_ARG, "fos_softgmm_forward: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_forward(g, d_rgb, d_depth, d_gt, s);
    reduce_partials_kernel<<<1, 256, 0, s>>>(g->part, g->blocks, 1, g->part + size_t(g->blocks) * 4);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss_out, g->part + size_t(g->blocks) * 4, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sg_fail(g, FOS_ERR_CUDA, "fos_softgmm_forward", e);
    g->have_forward = true;
    return FOS_OK;
}

fos_status fos_softgmm_backward(fos_softgmm* g, const uint8_t* d_rgb, const uint16_t* d_depth,
                                const uint8_t* d_gt, double grad_out[4], float* d_pixel_grad, void* stream)
{
    if (!g || !d_rgb || !d_depth || !d_gt || !grad_out) return sg_fail(g, FOS_ERR_INVALID_ARG, "fos_softgmm_backward: NULL argument");
    if (!g->have_forward) return sg_fail(g, FOS_ERR_STATE, "fos_softgmm_backward: run fos_softgmm_forward with these parameters first");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_backward(g, d_rgb, d_depth, d_gt, d_pixel_grad, s);
    reduce_partials_kernel<<<1, 256, 0, s>>>(g->part, g->blocks, 4, g->part + size_t(g->blocks) * 4);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad_out, g->part + size_t(g->blocks) * 4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sg_fail(g, FOS_ERR_CUDA, "fos_softgmm_backward", e);
    return FOS_OK;
}

}  // extern "C"
