// pbas_joint.cu -- joint-channel PBAS, a variant of the paper's Sec. 3.2
// model: one decision threshold R(x), learning parameter T(x) and minimal-
// distance record D(x) per pixel instead of one per channel, and one
// decision per pixel on the joint distance of each sample.
//
// Active channels A(x): R, G, B, and D where the depth reading is valid;
// n = |A|.  Distance of sample k: the mean over A of the per-channel PBAS
// distances fl(fl(wg_c |dg|) + |dv|), computed as their FP32 sum in channel
// order times fl(1/n).  Fewer than #min samples closer than R: foreground.
// One Philox draw per pixel (counter channel word 0).  The own update writes
// every channel of A into slot k1 and D/S as in the base method; a neighbour
// request covers the whole sample (with propagation, the requester's active
// channels).  R, T, S and D live in channel 0's planes of the usual layout
// (R floor R_lower_rgb); the entries of channels 1..3 keep their bootstrap
// values, so the state exports unchanged.  Bootstrap, pending-request
// application and the flush are the base method's kernels.
//
// Same two-phase schedule and explicit single-rounding arithmetic as the
// per-channel kernel; this translation unit is compiled without contraction.
#include "pbas_dev.cuh"

namespace fos {
namespace {

template <int NT, int PX, int TY>
__global__ void __launch_bounds__(32 * TY, 1024 / (32 * TY)) pbas_joint_kernel(const PbasArgs a)
{
    using G = Geo<PX, TY>;
    constexpr int NW = SWords<PX>::NW;
    constexpr float kThird = 1.0f / 3.0f;  // fl(1/3)
    constexpr int kAhead = 4;              // sample rows prefetched into L1 ahead of use
    __shared__ ClassifySmem<PX, TY> S;
    __shared__ float wtab[4][256];  // fl(wg_c * dg) for every gradient difference dg
    uint8_t* sm = S.sm;
    uint32_t* sreq = S.sreq;
    const int N = NT > 0 ? NT : a.N;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int x0 = blockIdx.x * G::TW, y0 = blockIdx.y * TY;

    {
        // L1 prefetch of R, T, S and the first kAhead sample rows of every channel
        const int px = x0 + int(threadIdx.x) * PX, py = y0 + int(threadIdx.y);
        if (py < a.H && px < a.W) {
            const int64_t q = int64_t(py) * a.Wp + px;
            prefetch_l1(a.R + q); prefetch_l1(a.T + q); prefetch_l1(a.S + q);
            const int64_t sb = sidx(a, N, 0, 0, px, py), cs = a.nseg * int64_t(N) * kSeg;
#pragma unroll
            for (int k = 0; k < kAhead; ++k)
                if (k < N)
#pragma unroll
                    for (int c = 0; c < 4; ++c) prefetch_l1(a.samp + sb + c * cs + int64_t(k) * kSeg);
        }
    }
    stage_input<PX, TY>(a, x0, y0, sm);
    if (a.apply) stage_requests<PX, TY>(a, x0, y0, sreq);
    if (tid < 4) {
        // gradient weight: alpha_g / mean gradient magnitude of the previous frame
        float mean = __fdiv_rn(__ull2float_rn(a.gsum_prev[tid]), __ll2float_rn(a.P));
        mean = fmaxf(mean, 1.0f);
        S.wgs[tid] = __fdiv_rn(a.alpha_g, mean);
    }
    if (x0 == 0 && y0 == 0 && tid >= 4 && tid < 8) a.gsum_next[tid - 4] = 0ull;
    __syncthreads();
    for (int e = tid; e < 1024; e += 32 * TY)
        wtab[e >> 8][e & 255] = __fmul_rn(S.wgs[e >> 8], __int2float_rn(e & 255));
    __syncthreads();

    const int lx0 = threadIdx.x * PX, ly = threadIdx.y;
    const int x = x0 + lx0, y = y0 + ly;
    bool inb[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) inb[i] = (y < a.H) && (x + i < a.W);
    const int64_t q0 = int64_t(y) * a.Wp + x;
    const uint32_t pix0 = uint32_t(y) * uint32_t(a.W) + uint32_t(x);
    const bool vec = (PX > 1) && inb[0];  // W % PX == 0 on this path
    uint32_t cnt5[5] = {0, 0, 0, 0, 0};  // gsum R,G,B,D; neighbour writes
    uint32_t cnt2[2] = {0, 0};           // own-update sample writes; requests

    // R, and the words the neighbour updates need, are loaded before any of
    // this thread's stores (a load behind scattered stores waits for them)
    float Rv[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) Rv[i] = 0.f;
    if (vec) {
        ldf<PX>(a.R + q0, Rv);
    } else {
#pragma unroll
        for (int i = 0; i < PX; ++i) Rv[i] = inb[i] ? a.R[q0 + i] : 0.f;
    }

    // neighbour updates requested during frame t-1 (whole samples)
    if (a.apply) {
        uint32_t mm[PX];
        uint64_t pw[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            mm[i] = inb[i] ? request_matches<G::SW>(sreq, ly, lx0 + i + 1) : 0u;
            // base method: the pixel's own value; propagation: its own-slot word
            pw[i] = mm[i] ? (a.propagate ? uint64_t(a.own[q0 + i]) : a.prev[q0 + i]) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if (!mm[i]) continue;
            if (a.propagate)
                cnt5[4] += apply_propagated<G::SW>(a, N, sreq, ly, lx0 + i + 1, x + i, y, mm[i], uint32_t(pw[i]));
            else
                cnt5[4] += apply_own_value<G::SW>(a, N, sreq, ly, lx0 + i + 1, x + i, y, mm[i], pw[i]);
        }
    }

    // this frame's features: (value | gradient << 8) per channel and pixel,
    // pixel i in half i & 1 of word own[c][i >> 1] (the only copy kept live
    // through the distance loop, so that registers go to loads in flight)
    uint32_t own[4][NW];
    bool dval[PX];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int w = 0; w < NW; ++w) own[c][w] = 0u;
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        const int col = lx0 + i + 1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t v = sm[c * G::CH + (ly + 1) * G::SWP + col];
            const uint32_t g = sobel(sm + c * G::CH, G::SWP, ly + 1, col);
            own[c][i >> 1] |= (v | (g << 8)) << (16 * (i & 1));
            if (inb[i]) cnt5[c] += g;
        }
        dval[i] = inb[i] && sm[3 * G::CH + (ly + 1) * G::SWP + col] != 0;
    }
    block_add<TY, 5>(cnt5, [&](int q) { return q < 4 ? a.gsum_cur + q : a.counters + 1; });

    if (inb[0]) {
        // joint distances to the N samples: count within R, minimum
        float inv[PX];
        int cnt[PX];
        float dmin[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) { inv[i] = dval[i] ? 0.25f : kThird; cnt[i] = 0; dmin[i] = INFINITY; }
        const int64_t sb = sidx(a, N, 0, 0, x, y);
        const int64_t cstride = a.nseg * int64_t(N) * kSeg;  // channel c + 1 lies this far after c
#pragma unroll(NT > 0 ? NT : 4)
        for (int k = 0; k < N; ++k) {
            if (k + kAhead < N)
#pragma unroll
                for (int c = 0; c < 4; ++c) prefetch_l1(a.samp + sb + int64_t(c) * cstride + int64_t(k + kAhead) * kSeg);
            uint32_t s[4][NW];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint16_t* p = a.samp + sb + int64_t(c) * cstride + int64_t(k) * kSeg;
                if (vec) ldw<PX>(p, s[c]);
                else s[c][0] = *p;
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint32_t d[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) d[c] = __vabsdiffu4(s[c][w], own[c][w]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = 2 * w + h;
                    if (i >= PX) break;
                    float sum = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t dv = (d[c] >> (16 * h)) & 0xFFu;
                        const uint32_t dg = (d[c] >> (16 * h + 8)) & 0xFFu;
                        const float dc = __fadd_rn(wtab[c][dg], __uint2float_rn(dv));
                        if (c == 0) sum = dc;
                        else if (c < 3 || dval[i]) sum = __fadd_rn(sum, dc);
                    }
                    const float dist = __fmul_rn(sum, inv[i]);
                    cnt[i] += dist < Rv[i] ? 1 : 0;
                    dmin[i] = fminf(dmin[i], dist);
                }
            }
        }

        float Tv[PX];
        uint32_t Sv[PX];
        if (vec) {
            ldf<PX>(a.T + q0, Tv);
            ldu<PX>(a.S + q0, Sv);
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                Tv[i] = inb[i] ? a.T[q0 + i] : 1.f;
                Sv[i] = inb[i] ? a.S[q0 + i] : 0u;
            }
        }
        uint32_t pv[4][PX];
        uint64_t pnew[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            pnew[i] = 0ull;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                pv[c][i] = (own[c][i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                pnew[i] |= uint64_t(pv[c][i]) << (16 * c);
            }
        }
        const float omr = __fsub_rn(1.0f, a.R_incdec), opr = __fadd_rn(1.0f, a.R_incdec);
        const float n16 = __int2float_rn(16 * N);
        // decisions and draws, then every D read before any store: a load
        // issued behind this thread's scattered sample stores waits for them
        uint32_t reqw[PX], ownw[PX];
        uint8_t mk[PX];
        int slot[PX];
        int64_t di[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            reqw[i] = kReqNone4;
            ownw[i] = kReqNone4;
            mk[i] = 0;
            slot[i] = -1;
            di[i] = 0;
            if (!inb[i]) continue;
            const bool fg = cnt[i] < a.n_min;
            mk[i] = fg ? 255 : 0;
            if (fg) continue;
            const Draws d = draws(a, pix0 + uint32_t(i), 0u, __frcp_rn(Tv[i]), N);
            if (d.coin1) {
                slot[i] = int(d.k1);
                di[i] = sidx(a, N, 0, int(d.k1), x + i, y);
            }
            if (d.coin2) {
                // the whole sample; with propagation only the requester's active channels
                reqw[i] = ((d.j << 5) | d.k2) * 0x01010101u;
                if (a.propagate && !dval[i]) reqw[i] = (reqw[i] & 0x00FFFFFFu) | 0x1F000000u;
                cnt2[1] += 1;
            }
        }
        uint32_t dold[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) dold[i] = slot[i] >= 0 ? uint32_t(a.Dq[di[i]]) : 0u;
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if (slot[i] < 0) continue;
            const int nc = dval[i] ? 4 : 3;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c >= nc) break;
                a.samp[di[i] + int64_t(c) * cstride] = uint16_t(pv[c][i]);
                ownw[i] = (ownw[i] & ~(0xFFu << (8 * c))) | (uint32_t(slot[i]) << (8 * c));
            }
            const float q16 = __fmul_rn(dmin[i], 16.0f);
            const uint32_t q = q16 >= 65535.0f ? 65535u : __float2uint_rn(q16);
            Sv[i] = Sv[i] + q - dold[i];
            a.Dq[di[i]] = uint16_t(q);
            cnt2[0] += uint32_t(nc);
        }
        // adaptive threshold R and learning parameter T
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if (!inb[i]) continue;
            const bool fg = mk[i] != 0;
            const float dbar = fmaxf(__fdiv_rn(__uint2float_rn(Sv[i]), n16), a.eps_d);
            const float Rs = __fmul_rn(dbar, a.R_scale);
            const float Rn = Rv[i] > Rs ? __fmul_rn(Rv[i], omr) : __fmul_rn(Rv[i], opr);
            Rv[i] = Rn < a.R_lower_rgb ? a.R_lower_rgb : Rn;
            float Tn = fg ? __fadd_rn(Tv[i], __fdiv_rn(a.T_inc, dbar)) : __fsub_rn(Tv[i], __fdiv_rn(a.T_dec, dbar));
            Tn = Tn < a.T_lower ? a.T_lower : Tn;
            Tv[i] = Tn > a.T_upper ? a.T_upper : Tn;
        }

        const int64_t p0 = int64_t(y) * a.W + x;  // mask index (unpadded frame)
        if (vec) {
            stf<PX>(a.R + q0, Rv);
            stf<PX>(a.T + q0, Tv);
            stu<PX>(a.S + q0, Sv);
            stu<PX>(a.req_cur + q0, reqw);
            if (a.propagate) stu<PX>(a.own + q0, ownw);
            if constexpr (PX == 2) {
                *reinterpret_cast<ulonglong2*>(a.prev + q0) = make_ulonglong2(pnew[0], pnew[1]);
                if ((reinterpret_cast<uintptr_t>(a.mask + p0) & 1u) == 0u)
                    *reinterpret_cast<uint16_t*>(a.mask + p0) = uint16_t(mk[0] | (mk[1] << 8));
                else { a.mask[p0] = mk[0]; a.mask[p0 + 1] = mk[1]; }
            }
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                if (!inb[i]) continue;
                a.R[q0 + i] = Rv[i];
                a.T[q0 + i] = Tv[i];
                a.S[q0 + i] = Sv[i];
                a.req_cur[q0 + i] = reqw[i];
                if (a.propagate) a.own[q0 + i] = ownw[i];
                a.prev[q0 + i] = pnew[i];
                a.mask[p0 + i] = mk[i];
            }
        }
    }

    block_add<TY, 2>(cnt2, [&](int q) { return a.counters + (q == 0 ? 0 : 2); });
}

}  // namespace

// Two pixels per thread (vector accesses) when the width is even, else one;
// 8 rows per block.
LaunchResult launch_pbas_joint(const PbasArgs& a, cudaStream_t s)
{
    if (a.P == 0) return kLaunchOk;
    constexpr int TY = 8;
    const bool two = a.W % 2 == 0;
    const int tw = two ? 64 : 32;
    const dim3 grid(unsigned((a.W + tw - 1) / tw), unsigned((a.H + TY - 1) / TY)), block(32, TY);
    if (two) {
        if (a.N == 20) pbas_joint_kernel<20, 2, TY><<<grid, block, 0, s>>>(a);
        else pbas_joint_kernel<0, 2, TY><<<grid, block, 0, s>>>(a);
    } else {
        if (a.N == 20) pbas_joint_kernel<20, 1, TY><<<grid, block, 0, s>>>(a);
        else pbas_joint_kernel<0, 1, TY><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

}  // namespace fos
