// pbas.cu -- PBAS classify-and-update over R, G, B and depth (paper Sec. 3.2).
//
// Each sample holds R, G, B and D; each channel is processed separately with
// its own decision threshold R(x), learning parameter T(x) and minimal-
// distance record D(x) (base method: Hofmann et al., cited by the paper); the
// depth channel only where the depth reading is valid; the pixel is
// foreground if any processed channel is.
//
// Two-phase semantics (every pixel of frame t is classified against the model
// as it stood after frame t-1, including frame t-1's neighbour updates) with
// one launch per frame:
//   classify(t): stage the frame tile plus a 1-pixel halo in shared memory;
//     apply the neighbour updates requested during frame t-1 to this pixel's
//     slots (each writes the pixel's own frame-(t-1) value, kept in `prev`);
//     Sobel gradient per channel; distance to the N samples; own update;
//     R/T/D update; this frame's neighbour requests; mask; per-channel
//     gradient sums for the next frame's weight.
//   flush: applies pending requests without classifying (before the state is
//     exported).
// The pending writes go to memory just before the same thread reads those
// slots, so they merge into sectors the kernel is reading anyway.
// Arithmetic is IEEE single precision with every operation rounded once
// (explicit _rn intrinsics, no contraction), so results are bit-exact against
// a plain C implementation of the same steps.
#include <algorithm>

#include "pbas_dev.cuh"

namespace fos {
namespace {

// One tile (32*PX x TY pixels at x0, y0) of the classify pass of one stream.
// build_table: recompute the gradient-weight table (the stream changed).
// GPAIR: the GMM part moves two pixels' state with 8-byte accesses (more
// registers live; the persistent batched kernel keeps the one-pixel form).
template <int NT, int PX, int TY, int KR = 0, int KD = 0, bool GPAIR = true>
__device__ __forceinline__ void classify_tile(const PbasArgs& a, const GmmArgs* gm, int x0, int y0,
                                              ClassifySmem<PX, TY>& S, bool build_table)
{
    using G = Geo<PX, TY>;
    constexpr int NW = SWords<PX>::NW;
    uint8_t* sm = S.sm;
    uint32_t* sreq = S.sreq;
    const int N = NT > 0 ? NT : a.N;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    {
        const int px = x0 + int(threadIdx.x) * PX, py = y0 + int(threadIdx.y);
        if (py < a.H && px < a.W) prefetch_channel<NT>(a, N, 0, px, py, int64_t(py) * a.Wp + px);
    }
    stage_input<PX, TY>(a, x0, y0, sm);
    const int lx0 = threadIdx.x * PX, ly = threadIdx.y;
    if (a.apply) stage_requests<PX, TY>(a, x0, y0, sreq);
    if (build_table && tid < 4) {
        // gradient weight: alpha_g / mean gradient magnitude of the previous frame
        float mean = __fdiv_rn(__ull2float_rn(a.gsum_prev[tid]), __ll2float_rn(a.P));
        mean = fmaxf(mean, 1.0f);
        S.wgs[tid] = __fdiv_rn(a.alpha_g, mean);
        if (tid == 0) S.rn16 = __frcp_rn(__int2float_rn(16 * N));
    }
    if (x0 == 0 && y0 == 0 && tid >= 4 && tid < 8) a.gsum_next[tid - 4] = 0ull;
    __syncthreads();

    if constexpr (KR > 0) gmm_tile_part<KR, KD, PX, TY, GPAIR>(*gm, a, x0, y0, sm);

    const int x = x0 + lx0, y = y0 + ly;
    bool inb[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) inb[i] = (y < a.H) && (x + i < a.W);
    const int64_t q0 = int64_t(y) * a.Wp + x;   // index in the pitched planes
    const uint32_t pix0 = uint32_t(y) * uint32_t(a.W) + uint32_t(x);  // Philox counter
    const bool vec = (PX > 1) && inb[0];  // W % PX == 0 on this path: all PX in frame
    uint32_t reqw[PX];
    bool anyfg[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) { reqw[i] = kReqNone4; anyfg[i] = false; }
    uint32_t cnt7[7] = {0, 0, 0, 0, 0, 0, 0};  // gsum R,G,B,D; own; neighbour writes; requests

    // Neighbour updates of frame t-1: this pixel's own frame-(t-1) value (prev,
    // 4 channels x (value | gradient << 8)) goes into every slot a neighbour
    // asked for; depth only if it was valid.  Written before any sample of
    // this pixel is read below, so this frame sees the updated model.
    if (a.apply) {
        uint64_t pw[PX];
        if (vec) {
            if constexpr (PX == 4) {
                const ulonglong2 u0 = vat<const ulonglong2>(a.prev, q0, 2, a.plane, 24, a.oob);
                const ulonglong2 u1 = vat<const ulonglong2>(a.prev, q0 + 2, 2, a.plane, 24, a.oob);
                pw[0] = u0.x; pw[1] = u0.y; pw[2] = u1.x; pw[3] = u1.y;
            } else if constexpr (PX == 2) {
                const ulonglong2 u0 = vat<const ulonglong2>(a.prev, q0, 2, a.plane, 24, a.oob);
                pw[0] = u0.x; pw[1] = u0.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i) pw[i] = inb[i] ? at(a.prev, q0 + i, a.plane, 24, a.oob) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            const uint32_t mm = inb[i] ? request_matches<G::SW>(sreq, ly, lx0 + i + 1, G::SH * G::SW, a.oob) : 0u;
            if (a.propagate) {
                cnt7[5] += apply_propagated<G::SW>(a, N, sreq, ly, lx0 + i + 1, x + i, y, mm,
                                                   mm ? at(a.own, q0 + i, a.plane, 25, a.oob) : kReqNone4,
                                                   G::SH * G::SW);
            } else {
                cnt7[5] += apply_own_value<G::SW>(a, N, sreq, ly, lx0 + i + 1, x + i, y, mm, pw[i], G::SH * G::SW);
            }
        }
    }
    uint64_t pnew[PX];  // this frame's (value | gradient << 8) per channel
#pragma unroll
    for (int i = 0; i < PX; ++i) pnew[i] = 0ull;

    const float omr = __fsub_rn(1.0f, a.R_incdec), opr = __fadd_rn(1.0f, a.R_incdec);
    const float n16 = __int2float_rn(16 * N);


#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        uint32_t pv[PX];   // this frame's (value | gradient << 8)
        bool act[PX];
        bool any = false;
        uint32_t gsc = 0;
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            const int col = lx0 + i + 1;
            const uint32_t v = at(sm, c * G::CH + (ly + 1) * G::SWP + col, 4 * G::CH, 26, a.oob);
            const uint32_t g = sobel(sm + c * G::CH, G::SWP, ly + 1, col, G::CH, a.oob);
            pv[i] = v | (g << 8);
            act[i] = inb[i] && (c < 3 || at(sm, 3 * G::CH + (ly + 1) * G::SWP + col, 4 * G::CH, 26, a.oob) != 0);
            if (inb[i]) gsc += g;
            any |= act[i];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) cnt7[q] += (q == c) ? gsc : 0u;

        const int64_t pc = int64_t(c) * a.plane + q0;
#pragma unroll
        for (int i = 0; i < PX; ++i) pnew[i] |= uint64_t(pv[i]) << (16 * c);
        if (!any) {
            if (a.propagate) put_own_slots<PX>(a, q0, c, inb, nullptr);
            continue;
        }

        float Rv[PX], Tv[PX];
        uint32_t Sv[PX];
        const int64_t ne = rts_extent(a);
        if (vec) {
            ldf<PX>(a.R, pc, ne, 16, a.oob, Rv);
            ldf<PX>(a.T, pc, ne, 17, a.oob, Tv);
            ldu<PX>(a.S, pc, ne, 18, a.oob, Sv);
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                Rv[i] = inb[i] ? at(a.R, pc + i, ne, 16, a.oob) : 0.f;
                Tv[i] = inb[i] ? at(a.T, pc + i, ne, 17, a.oob) : 1.f;
                Sv[i] = inb[i] ? at(a.S, pc + i, ne, 18, a.oob) : 0u;
            }
        }
        if (c < 3 && inb[0]) prefetch_channel<NT>(a, N, c + 1, x, y, q0);

        // distances to the N samples: count within R, minimum.
        // dist = fl(fl(wg * |dg|) + |dv|), each operation rounded once.
        uint32_t own[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) own[w] = pv[2 * w] | (2 * w + 1 < PX ? pv[2 * w + 1] << 16 : 0u);
        int cnt[PX];
        float dmin[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) { cnt[i] = 0; dmin[i] = INFINITY; }
        const int64_t sb = inb[0] ? sidx(a, N, c, 0, x, y) : 0;  // slot 0 of pixel x
        // dist = fl(fl(wg * |dg|) + |dv|): a byte b is the float (2^23 + b) - 2^23
        // exactly (a byte permute and a subtraction instead of a conversion)
        const float wgc = S.wgs[c];
#pragma unroll(NT > 0 ? NT : 4)
        for (int k = 0; k < N; ++k) {
            uint32_t s[NW];
            if (vec) {
                ldw<PX>(a.samp, sb + int64_t(k) * kSeg, samp_extent(a), 23, a.oob, s);
            } else {
                s[0] = inb[0] ? at(a.samp, sidx(a, N, c, k, x, y), samp_extent(a), 23, a.oob) : 0u;
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t d = __vabsdiffu4(s[w], own[w]);  // |dv0| |dg0| |dv1| |dg1|
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = 2 * w + h;
                    if (i >= PX) break;
                    const float fv = __fsub_rn(__uint_as_float(__byte_perm(d, 0x4B000000u, h ? 0x7442 : 0x7440)),
                                               8388608.f);
                    const float fgd = __fsub_rn(__uint_as_float(__byte_perm(d, 0x4B000000u, h ? 0x7443 : 0x7441)),
                                                8388608.f);
                    const float dist = __fadd_rn(__fmul_rn(wgc, fgd), fv);
                    cnt[i] += dist < Rv[i] ? 1 : 0;
                    dmin[i] = fminf(dmin[i], dist);
                }
            }
        }

        // decisions and random draws
        bool fg[PX];
        int slot[PX];
        int64_t oidx[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            fg[i] = act[i] && cnt[i] < a.n_min;
            slot[i] = -1;
            oidx[i] = 0;
            if (act[i] && !fg[i]) {
                const Draws d = draws(a, pix0 + uint32_t(i), uint32_t(c), __frcp_rn(Tv[i]), N);
                if (d.coin1) {
                    slot[i] = int(d.k1);
                    oidx[i] = sidx(a, N, c, int(d.k1), x + i, y);
                }
                if (d.coin2) {
                    const uint32_t byte = (d.j << 5) | d.k2;
                    reqw[i] = (reqw[i] & ~(0xFFu << (8 * c))) | (byte << (8 * c));
                    cnt7[6] += 1;
                }
            }
            anyfg[i] |= fg[i];
        }
        // own updates: all D reads first (independent), then the writes
        uint32_t dold[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) dold[i] = slot[i] >= 0 ? uint32_t(at(a.Dq, oidx[i], samp_extent(a), 27, a.oob)) : 0u;
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if (slot[i] < 0) continue;
            at(a.samp, oidx[i], samp_extent(a), 28, a.oob) = uint16_t(pv[i]);
            const float q16 = __fmul_rn(dmin[i], 16.0f);
            const uint32_t q = q16 >= 65535.0f ? 65535u : __float2uint_rn(q16);
            Sv[i] = Sv[i] + q - dold[i];
            at(a.Dq, oidx[i], samp_extent(a), 29, a.oob) = uint16_t(q);
            cnt7[4] += 1;
        }
        if (a.propagate) put_own_slots<PX>(a, q0, c, inb, slot);
        // adaptive threshold R and learning parameter T
        const float Rlo = c < 3 ? a.R_lower_rgb : a.R_lower_d;
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if (!act[i]) continue;
            // mean quantised minimal distance S / (16 N), correctly rounded
            const float dbar = fmaxf(div_int_const(Sv[i], n16, S.rn16), a.eps_d);
            const float Rs = __fmul_rn(dbar, a.R_scale);
            const float Rn = Rv[i] > Rs ? __fmul_rn(Rv[i], omr) : __fmul_rn(Rv[i], opr);
            Rv[i] = Rn < Rlo ? Rlo : Rn;
            // T + T_inc / dbar or T - T_dec / dbar: one division of the chosen
            // numerator (fl(-x / y) = -fl(x / y))
            float Tn = __fadd_rn(Tv[i], __fdiv_rn(fg[i] ? a.T_inc : -a.T_dec, dbar));
            Tn = Tn < a.T_lower ? a.T_lower : Tn;
            Tv[i] = Tn > a.T_upper ? a.T_upper : Tn;
        }
        if (vec) {
            stf<PX>(a.R, pc, ne, 19, a.oob, Rv);
            stf<PX>(a.T, pc, ne, 20, a.oob, Tv);
            stu<PX>(a.S, pc, ne, 21, a.oob, Sv);
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i)
                if (inb[i]) {
                    at(a.R, pc + i, ne, 19, a.oob) = Rv[i];
                    at(a.T, pc + i, ne, 20, a.oob) = Tv[i];
                    at(a.S, pc + i, ne, 21, a.oob) = Sv[i];
                }
        }
    }

    if (vec) {
        if constexpr (PX == 4) {
            vat<ulonglong2>(a.prev, q0, 2, a.plane, 30, a.oob) = make_ulonglong2(pnew[0], pnew[1]);
            vat<ulonglong2>(a.prev, q0 + 2, 2, a.plane, 30, a.oob) = make_ulonglong2(pnew[2], pnew[3]);
        } else if constexpr (PX == 2) {
            vat<ulonglong2>(a.prev, q0, 2, a.plane, 30, a.oob) = make_ulonglong2(pnew[0], pnew[1]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < PX; ++i)
            if (inb[i]) at(a.prev, q0 + i, a.plane, 30, a.oob) = pnew[i];
    }

    const int64_t p0 = int64_t(y) * a.W + x;  // mask index (unpadded frame)
    if (vec && a.mask_vec) {
        uint32_t m = 0;
#pragma unroll
        for (int i = 0; i < PX; ++i) m |= (anyfg[i] ? 255u : 0u) << (8 * i);
        if constexpr (PX == 4) vat<uint32_t>(a.mask, p0, 4, a.P, 31, a.oob) = m;
        else vat<uint16_t>(a.mask, p0, 2, a.P, 31, a.oob) = uint16_t(m);
    } else {
#pragma unroll
        for (int i = 0; i < PX; ++i)
            if (inb[i]) at(a.mask, p0 + i, a.P, 31, a.oob) = anyfg[i] ? 255 : 0;
    }
    if (vec) {
        stu<PX>(a.req_cur, q0, a.plane, 32, a.oob, reqw);
    } else {
#pragma unroll
        for (int i = 0; i < PX; ++i)
            if (inb[i]) at(a.req_cur, q0 + i, a.plane, 32, a.oob) = reqw[i];
    }

    block_add<TY, 7>(cnt7, [&](int q) {
        return q < 4 ? a.gsum_cur + q : a.counters + (q == 4 ? 0 : (q == 5 ? 1 : 2));
    });
}

template <int NT, int PX, int TY>
// four 256-thread blocks per SM (64 registers): more warps to hide the
// memory latency than the three an unbounded register count leaves room for
__global__ void __launch_bounds__(32 * TY, PX <= 2 ? 1024 / (32 * TY) : 1) pbas_classify_kernel(const PbasArgs a)
{
    __shared__ ClassifySmem<PX, TY> S;
    classify_tile<NT, PX, TY>(a, nullptr, blockIdx.x * Geo<PX, TY>::TW, blockIdx.y * TY, S, true);
}

// GMM and PBAS of one frame in one pass over the frame (inputs staged once).
template <int NT, int PX, int TY>
__global__ void __launch_bounds__(32 * TY, PX <= 2 ? 1024 / (32 * TY) : 1)
fused_classify_kernel(const PbasArgs a, const GmmArgs g)
{
    __shared__ ClassifySmem<PX, TY> S;
    classify_tile<NT, PX, TY, 3, 3>(a, &g, blockIdx.x * Geo<PX, TY>::TW, blockIdx.y * TY, S, true);
}

// --- several frames in one persistent launch ---------------------------------

// One block of the gradient pre-pass: a 32-pixel-wide strip of kGradStrip
// rows, staged at once (with its 1-pixel halo, edge-clamped, as classify
// stages its tiles) and summed by kGradTY rows of 32 threads.
constexpr int kGradStrip = kGradStripRows, kGradTY = 8;
constexpr int kGradSW = 34, kGradSWP = 36, kGradSH = kGradStrip + 2, kGradCH = kGradSH * kGradSWP;

// Sums of the Sobel magnitudes of the strip at (x0, y0) of frame a, added to
// v[4].  Every thread issues all of its staging loads before it stores any of
// them, so a block waits for one memory round trip, not one per row of loads.
__device__ __forceinline__ void grad_strip(const PbasArgs& a, int x0, int y0, uint8_t* sm, uint32_t (&v)[4])
{
    constexpr int NS = kGradSH * kGradSW, NTH = 32 * kGradTY, NIT = (NS + NTH - 1) / NTH;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const bool mapped = a.Wd != a.W || a.Hd != a.H;
    uint32_t cr[NIT], cg[NIT], cb[NIT], cd[NIT];
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int idx = tid + k * NTH;
        if (idx < NS) {
            const int r = idx / kGradSW, col = idx - r * kGradSW;
            const int gx = min(max(x0 - 1 + col, 0), a.W - 1);
            const int gy = min(max(y0 - 1 + r, 0), a.H - 1);
            const int64_t p = int64_t(gy) * a.W + gx;
            const int64_t pd = mapped ? int64_t(uint32_t(gy * a.Hd) / uint32_t(a.H)) * a.Wd +
                                            int64_t(uint32_t(gx * a.Wd) / uint32_t(a.W))
                                      : p;
            cr[k] = at(a.rgb, 3 * p, 3 * a.P, 2, a.oob);
            cg[k] = at(a.rgb, 3 * p + 1, 3 * a.P, 2, a.oob);
            cb[k] = at(a.rgb, 3 * p + 2, 3 * a.P, 2, a.oob);
            cd[k] = at(a.depth, pd, depth_extent(a), 3, a.oob);
        }
    }
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int idx = tid + k * NTH;
        if (idx < NS) {
            const int r = idx / kGradSW, col = idx - r * kGradSW;
            const int o = r * kGradSWP + col;
            constexpr int n = 4 * kGradCH;
            at(sm, o, n, 1, a.oob) = uint8_t(cr[k]);
            at(sm, kGradCH + o, n, 1, a.oob) = uint8_t(cg[k]);
            at(sm, 2 * kGradCH + o, n, 1, a.oob) = uint8_t(cb[k]);
            at(sm, 3 * kGradCH + o, n, 1, a.oob) = uint8_t(depth_to_u8(cd[k], a.depth_fs, a.depth_m, a.depth_sh));
        }
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    for (int r = threadIdx.y; r < kGradStrip; r += kGradTY) {
        if (x < a.W && y0 + r < a.H) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                v[c] += sobel(sm + c * kGradCH, kGradSWP, r + 1, threadIdx.x + 1, kGradCH, a.oob);
        }
    }
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polls before a wait gives up (each poll sleeps 64 ns and reads L2: well
// over a second in all).  The wait cannot run out: a tile waits only for
// tiles claimed before it, whose blocks are running.
constexpr uint32_t kSeqSpinLimit = 1u << 21;

// Waits until tile (tx, ty) has finished `need` frames of the launch (no-op
// outside the tile grid); on giving up, sets the error word and returns.
__device__ __forceinline__ void seq_wait(const SeqArgs& q, int tx, int ty, int need)
{
    if (tx < 0 || ty < 0 || tx >= q.tiles_x || ty >= q.tiles_y) return;
    const int* f = q.done + ty * q.tiles_x + tx;
    for (uint32_t spin = 0; ld_acquire_gpu(f) < need; ++spin) {
        if (spin >= kSeqSpinLimit || ((spin & 1023u) == 1023u && *(volatile int*)q.err)) {
            atomicExch(q.err, 1);
            return;
        }
        __nanosleep(64);
    }
}

// The arguments of frame t0+i (inputs, masks, frame index, parity planes).
template <int PX>
__device__ __forceinline__ void seq_frame_args(PbasArgs& a, GmmArgs& g, const SeqArgs& q, int i)
{
    const int64_t f = i;
    a.rgb += f * q.rgb_stride;
    a.depth += f * q.depth_stride;
    a.mask += f * q.mask_stride;
    a.t += uint32_t(i);
    const int64_t pl = a.plane;
    a.req_cur = q.req_base + int64_t(a.t & 1u) * pl;
    a.req_prev = q.req_base + int64_t((a.t + 1u) & 1u) * pl;
    if (a.propagate) {
        a.prev = q.prev_base + int64_t(a.t & 1u) * pl;
        a.prev_src = q.prev_base + int64_t((a.t + 1u) & 1u) * pl;
    }
    a.gsum_prev = const_cast<unsigned long long*>(q.gprev) + 4 * f;
    a.gsum_cur = q.gscratch;
    a.gsum_next = q.gscratch + 4;
    if (i > 0) a.apply = 1;
    a.mask_vec = (reinterpret_cast<uintptr_t>(a.mask) % uintptr_t(PX)) == 0 ? 1 : 0;
    g.rgb = a.rgb;
    g.depth = a.depth;
    g.mask += f * q.mask_stride;
}

// GMM (3+3) and PBAS of q.n frames; one block per SM slot, tiles claimed in
// frame-major order.  Bits equal to q.n launches of fused_classify_kernel.
template <int NT, int PX, int TY>
__global__ void __launch_bounds__(32 * TY, PX <= 2 ? 1024 / (32 * TY) : 1)
fused_sequence_kernel(const PbasArgs a0, const GmmArgs g0, const SeqArgs q)
{
    using G = Geo<PX, TY>;
    __shared__ ClassifySmem<PX, TY> S;
    __shared__ int s_it;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int ntiles = q.tiles_x * q.tiles_y;
    const int total = ntiles * q.n;
    for (;;) {
        // s_it is rewritten only after the tile below has passed its own
        // block barriers, so every thread has read it by then
        if (tid == 0) s_it = int(atomicAdd(q.claim, 1u));
        __syncthreads();
        const int it = s_it;
        if (it >= total) break;
        const int i = it / ntiles, j = it - i * ntiles;
        const int tx = j % q.tiles_x, ty = j / q.tiles_x;
        // the 3x3 neighbourhood of frame t0+i-1: nine threads wait, one tile each
        if (i > 0 && tid < 9) seq_wait(q, tx + tid % 3 - 1, ty + tid / 3 - 1, i);
        __syncthreads();
        PbasArgs a = a0;
        GmmArgs g = g0;
        seq_frame_args<PX>(a, g, q, i);
        classify_tile<NT, PX, TY, 3, 3>(a, &g, tx * G::TW, ty * TY, S, true);
        // all of the tile's writes are ordered before the completion word
        __syncthreads();
        if (tid == 0) st_release_gpu(q.done + j, i + 1);
    }
}

// --- many streams, several frames, one persistent launch -------------------

// seq_wait for a tile grid given by pointer and size.
__device__ __forceinline__ void seq_wait_grid(const int* done, int tiles_x, int tiles_y, int tx, int ty,
                                              int need, int* err)
{
    if (tx < 0 || ty < 0 || tx >= tiles_x || ty >= tiles_y) return;
    const int* f = done + ty * tiles_x + tx;
    for (uint32_t spin = 0; ld_acquire_gpu(f) < need; ++spin) {
        if (spin >= kSeqSpinLimit || ((spin & 1023u) == 1023u && *(volatile int*)err)) {
            atomicExch(err, 1);
            return;
        }
        __nanosleep(64);
    }
}

// The arguments of frame t0+i of entry E.
template <int PX>
__device__ __forceinline__ void seq_batch_frame_args(PbasArgs& a, GmmArgs& g, const SeqBatchEntry& E, int i,
                                                     unsigned long long* gscratch)
{
    const int64_t f = i;
    a.rgb += f * E.rgb_stride;
    a.depth += f * E.depth_stride;
    a.mask += f * E.mask_stride;
    a.t += uint32_t(i);
    const int64_t pl = a.plane;
    a.req_cur = E.req_base + int64_t(a.t & 1u) * pl;
    a.req_prev = E.req_base + int64_t((a.t + 1u) & 1u) * pl;
    if (a.propagate) {
        a.prev = E.prev_base + int64_t(a.t & 1u) * pl;
        a.prev_src = E.prev_base + int64_t((a.t + 1u) & 1u) * pl;
    }
    a.gsum_prev = E.gprev + 4 * f;
    a.gsum_cur = gscratch;
    a.gsum_next = gscratch + 4;
    if (i > 0) a.apply = 1;
    a.mask_vec = (reinterpret_cast<uintptr_t>(a.mask) % uintptr_t(PX)) == 0 ? 1 : 0;
    g.rgb = a.rgb;
    g.depth = a.depth;
    g.mask += f * E.mask_stride;
}

// Entry of tile g among entries 0 .. m-1 (tile_off ascending).
__device__ __forceinline__ int seq_batch_entry_of(const SeqBatchTable& T, int g, int m)
{
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.e[mid].tile_off <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int NT, int PX, int TY>
__global__ void __launch_bounds__(32 * TY, PX <= 2 ? 1024 / (32 * TY) : 1)
batch_sequence_kernel(const __grid_constant__ SeqBatchTable T)
{
    using G = Geo<PX, TY>;
    __shared__ ClassifySmem<PX, TY> S;
    __shared__ long long s_it;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const long long total = T.seg_claim0[T.segs];
    for (;;) {
        if (tid == 0) s_it = static_cast<long long>(atomicAdd(T.claim, 1u));
        __syncthreads();
        const long long it = s_it;
        if (it >= total) break;
        int r = 0, hi = T.segs - 1;  // run of slots holding this claim
        while (r < hi) {
            const int mid = (r + hi + 1) >> 1;
            if (T.seg_claim0[mid] <= it) r = mid;
            else hi = mid - 1;
        }
        const long long off = it - T.seg_claim0[r];
        const int i = T.seg_slot0[r] + int(off / T.seg_tiles[r]);
        const int gtile = int(off % T.seg_tiles[r]);
        const int je = seq_batch_entry_of(T, gtile, T.seg_m[r]);
        const SeqBatchEntry& E = T.e[je];
        const int j = gtile - E.tile_off;
        const int tx = j % E.tiles_x, ty = j / E.tiles_x;
        if (i > 0 && tid < 9) seq_wait_grid(E.done, E.tiles_x, E.tiles_y, tx + tid % 3 - 1, ty + tid / 3 - 1, i, T.err);
        __syncthreads();
        PbasArgs a = E.a;
        GmmArgs g = T.g[je];
        seq_batch_frame_args<PX>(a, g, E, i, T.gscratch);
        classify_tile<NT, PX, TY, 3, 3>(a, &g, tx * G::TW, ty * TY, S, true);
        __syncthreads();
        if (tid == 0) st_release_gpu(E.done + j, i + 1);
    }
}

// Zeroes the claim counter, the error word and the completion words; sets
// each entry's gradient sums (frame t0-1 copied, the rest zero for the pre-pass).
__global__ void seq_batch_prepare_kernel(const __grid_constant__ SeqBatchTable T)
{
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, nth = int64_t(gridDim.x) * blockDim.x;
    if (tid == 0) {
        *T.claim = 0u;
        *T.err = 0;
    }
    for (int64_t i = tid; i < T.done_words; i += nth) T.done_all[i] = 0;
    for (int j = 0; j < T.n; ++j) {
        const SeqBatchEntry& E = T.e[j];
        for (int64_t i = tid; i < 4 * int64_t(E.n + 1); i += nth) E.gprev[i] = i < 4 ? E.gsum_src[i] : 0ull;
    }
}

// Gradient sums of every entry's frames: block (x, y) = pre-pass tile x of
// all entries, frame y of its entry.
__global__ void __launch_bounds__(32 * kGradTY) seq_batch_grad_kernel(const __grid_constant__ SeqBatchTable T)
{
    __shared__ __align__(16) uint8_t sm[4 * kGradCH];
    const int gt = int(blockIdx.x), f = int(blockIdx.y);
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.e[mid].gtile_off <= gt) lo = mid;
        else hi = mid - 1;
    }
    const SeqBatchEntry& E = T.e[lo];
    if (f >= E.n) return;  // uniform over the block
    PbasArgs a = E.a;
    a.rgb += int64_t(f) * E.rgb_stride;
    a.depth += int64_t(f) * E.depth_stride;
    const int l = gt - E.gtile_off, gtx = (a.W + 31) / 32;
    uint32_t v[4] = {0, 0, 0, 0};
    grad_strip(a, (l % gtx) * 32, (l / gtx) * kGradStrip, sm, v);
    block_add<kGradTY, 4>(v, [&](int c) { return E.gprev + 4 + 4 * int64_t(f) + c; });
}

// Each entry's last-frame sums where its next per-frame launch reads them,
// and the accumulator of that frame zeroed (one block of 4 * kSeqBatchMax threads).
__global__ void seq_batch_finish_kernel(const __grid_constant__ SeqBatchTable T)
{
    const int j = int(threadIdx.x) / 4, q = int(threadIdx.x) % 4;
    if (j >= T.n) return;
    const SeqBatchEntry& E = T.e[j];
    E.gsum_last[q] = E.gprev[4 * int64_t(E.n) + q];
    E.gsum_zero[q] = 0ull;
}

// Gradient sums of frame blockIdx.z (the Sobel magnitudes classify_tile adds
// to gsum_cur), one 32 x kGradStrip strip per block.
__global__ void __launch_bounds__(32 * kGradTY) grad_sums_kernel(const PbasArgs a0, const SeqArgs q,
                                                                 unsigned long long* out)
{
    __shared__ __align__(16) uint8_t sm[4 * kGradCH];
    PbasArgs a = a0;
    a.rgb += int64_t(blockIdx.z) * q.rgb_stride;
    a.depth += int64_t(blockIdx.z) * q.depth_stride;
    uint32_t v[4] = {0, 0, 0, 0};
    grad_strip(a, blockIdx.x * 32, blockIdx.y * kGradStrip, sm, v);
    block_add<kGradTY, 4>(v, [&](int c) { return out + 4 * int64_t(blockIdx.z) + c; });
}

// Applies the pending neighbour requests of the last frame to the samples
// without classifying (so that an exported state includes them).
template <int NT, int TY>
__global__ void __launch_bounds__(32 * TY) pbas_flush_kernel(const PbasArgs a)
{
    using G = Geo<1, TY>;
    __shared__ uint32_t sreq[G::SH * G::SW];
    const int N = NT > 0 ? NT : a.N;
    const int x0 = blockIdx.x * G::TW, y0 = blockIdx.y * TY;
    stage_requests<1, TY>(a, x0, y0, sreq);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    uint32_t applied[1] = {0};
    if (x < a.W && y < a.H) {
        const int64_t q = int64_t(y) * a.Wp + x;
        const uint32_t mm = request_matches<G::SW>(sreq, threadIdx.y, threadIdx.x + 1, G::SH * G::SW, a.oob);
        if (a.propagate)
            applied[0] = apply_propagated<G::SW>(a, N, sreq, threadIdx.y, threadIdx.x + 1, x, y, mm,
                                                 mm ? at(a.own, q, a.plane, 33, a.oob) : kReqNone4, G::SH * G::SW);
        else
            applied[0] = apply_own_value<G::SW>(a, N, sreq, threadIdx.y, threadIdx.x + 1, x, y, mm,
                                                at(a.prev_src, q, a.plane, 33, a.oob), G::SH * G::SW);
    }
    block_add<TY, 1>(applied, [&](int) { return a.counters + 1; });
}

// One tile of the frame-0 pass of one stream: every slot takes the frame.
template <int NT, int PX, int TY, int KR = 0, int KD = 0>
__device__ __forceinline__ void init_tile(const PbasArgs& a, const GmmArgs* gm, int x0, int y0, uint8_t* sm)
{
    using G = Geo<PX, TY>;
    const int N = NT > 0 ? NT : a.N;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    stage_input<PX, TY>(a, x0, y0, sm);
    if (x0 == 0 && y0 == 0 && tid < 4) a.gsum_next[tid] = 0ull;
    __syncthreads();
    if constexpr (KR > 0) gmm_tile_part<KR, KD, PX, TY>(*gm, a, x0, y0, sm);
    const int lx0 = threadIdx.x * PX, ly = threadIdx.y;
    const int x = x0 + lx0, y = y0 + ly;
    uint32_t gs[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        if (y >= a.H || x + i >= a.W) continue;
        const int col = lx0 + i + 1;
        const int64_t q = int64_t(y) * a.Wp + x + i;
        uint64_t pw = 0ull;
        if (a.propagate) at(a.own, q, a.plane, 34, a.oob) = kReqNone4;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t v = at(sm, c * G::CH + (ly + 1) * G::SWP + col, 4 * G::CH, 35, a.oob);
            const uint32_t g = sobel(sm + c * G::CH, G::SWP, ly + 1, col, G::CH, a.oob);
            gs[c] += g;
            const uint16_t sv = uint16_t(v | (g << 8));
            const int64_t b = sidx(a, N, c, 0, x + i, y);
            for (int k = 0; k < N; ++k) {
                at(a.samp, b + int64_t(k) * kSeg, samp_extent(a), 36, a.oob) = sv;
                at(a.Dq, b + int64_t(k) * kSeg, samp_extent(a), 36, a.oob) = 0;
            }
            at(a.R, int64_t(c) * a.plane + q, rts_extent(a), 37, a.oob) = c < 3 ? a.R_lower_rgb : a.R_lower_d;
            at(a.T, int64_t(c) * a.plane + q, rts_extent(a), 37, a.oob) = a.T_lower;
            at(a.S, int64_t(c) * a.plane + q, rts_extent(a), 37, a.oob) = 0u;
            pw |= uint64_t(sv) << (16 * c);
        }
        at(a.prev, q, a.plane, 38, a.oob) = pw;
        at(a.mask, int64_t(y) * a.W + x + i, a.P, 39, a.oob) = 0;
    }
    block_add<TY, 4>(gs, [&](int q) { return a.gsum_cur + q; });
}

template <int NT, int PX, int TY>
__global__ void __launch_bounds__(32 * TY) pbas_init_kernel(const PbasArgs a)
{
    __shared__ __align__(16) uint8_t sm[4 * Geo<PX, TY>::CH];
    init_tile<NT, PX, TY>(a, nullptr, blockIdx.x * Geo<PX, TY>::TW, blockIdx.y * TY, sm);
}

// Many streams in one launch.  Entry i of the table holds stream i's
// arguments, whether it is at frame 0, its first tile in the launch (prefix
// sum) and its tiles per row; the table is a __grid_constant__ parameter, so
// the arguments are read from the constant bank (one copy per launch, shared
// by every block).  One block per tile, in the order of the streams and of
// their tiles, as the single-stream launch orders them: tiles that share
// sample rows and halo rows run at about the same time (a persistent grid
// that took tiles round-robin ran 23 % slower on one 1280x720 stream).
template <int NT, int PX, int TY, int KR>
__global__ void __launch_bounds__(32 * TY, PX <= 2 ? 1024 / (32 * TY) : 1)
pbas_batch_kernel(const __grid_constant__ PbasBatchTable T)
{
    constexpr int KD = KR;
    __shared__ ClassifySmem<PX, TY> S;
    const int it = int(blockIdx.x);
    if (it >= T.total) return;
    int lo = 0, hi = T.n - 1;  // entry whose tile range holds `it`
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.e[mid].tile_off <= it) lo = mid;
        else hi = mid - 1;
    }
    const PbasBatchEntry& E = T.e[lo];
    const int local = it - E.tile_off, tx = E.tiles_x;
    const int x0 = (local % tx) * Geo<PX, TY>::TW, y0 = (local / tx) * TY;
    if (E.init) init_tile<NT, PX, TY, KR, KD>(E.a, &T.g[lo], x0, y0, S.sm);
    else classify_tile<NT, PX, TY, KR, KD>(E.a, &T.g[lo], x0, y0, S, true);
}

template <int PX, int TY>
dim3 grid_for(const PbasArgs& a)
{
    return dim3(unsigned((a.W + 32 * PX - 1) / (32 * PX)), unsigned((a.H + TY - 1) / TY));
}

// Tile shapes: PX pixels per thread (vector accesses) when W is a multiple of
// PX, TY rows per block; otherwise one pixel per thread, 8 rows, with bounds
// checks on every access.
#define FOS_PBAS_LAUNCHER(NAME, KERNEL)                                                   \
    template <int NT, int PX, int TY>                                                     \
    void NAME##_go(const PbasArgs& a, cudaStream_t s)                                     \
    {                                                                                     \
        KERNEL<NT, PX, TY><<<grid_for<PX, TY>(a), dim3(32, TY), 0, s>>>(a);               \
    }                                                                                     \
    template <int NT>                                                                     \
    bool NAME##_shape(const PbasArgs& a, cudaStream_t s, int px, int ty)                  \
    {                                                                                     \
        if (px == 4 && ty == 4) NAME##_go<NT, 4, 4>(a, s);                                \
        else if (px == 4 && ty == 2) NAME##_go<NT, 4, 2>(a, s);                           \
        else if (px == 4 && ty == 8) NAME##_go<NT, 4, 8>(a, s);                           \
        else if (px == 2 && ty == 4) NAME##_go<NT, 2, 4>(a, s);                           \
        else if (px == 2 && ty == 8) NAME##_go<NT, 2, 8>(a, s);                           \
        else if (px == 1) NAME##_go<NT, 1, 8>(a, s);                                      \
        else return false;                                                                \
        return true;                                                                      \
    }                                                                                     \
    LaunchResult NAME(const PbasArgs& a, cudaStream_t s)                                  \
    {                                                                                     \
        if (a.P == 0) return kLaunchOk;                                                   \
        const int px = (a.px > 1 && a.W % a.px == 0) ? a.px : 1;                          \
        const bool ok = a.N == 20 ? NAME##_shape<20>(a, s, px, a.ty) : NAME##_shape<0>(a, s, px, a.ty); \
        if (!ok) return kLaunchUnsupported;                                               \
        return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;          \
    }

}  // namespace

namespace {
FOS_PBAS_LAUNCHER(init_launch, pbas_init_kernel)
FOS_PBAS_LAUNCHER(classify_launch, pbas_classify_kernel)

template <int NT>
bool fused_shape(const PbasArgs& a, const GmmArgs& g, cudaStream_t s, int px, int ty)
{
#define FOS_F(P, T)                                                                        \
    if (px == P && ty == T) {                                                              \
        fused_classify_kernel<NT, P, T><<<grid_for<P, T>(a), dim3(32, T), 0, s>>>(a, g);   \
        return true;                                                                       \
    }
    FOS_F(2, 8) FOS_F(2, 4) FOS_F(4, 4) FOS_F(4, 8) FOS_F(1, 8)
#undef FOS_F
    return false;
}
}  // namespace

LaunchResult launch_pbas_init(const PbasArgs& a, cudaStream_t s) { return init_launch(a, s); }
LaunchResult launch_pbas_classify(const PbasArgs& a, cudaStream_t s) { return classify_launch(a, s); }

template <int NT, int PX, int TY>
LaunchResult sequence_go(const PbasArgs& a0, const GmmArgs& g0, const SeqArgs& q, cudaStream_t s)
{
    auto k = fused_sequence_kernel<NT, PX, TY>;
    // one block per SM slot (cached per shape); a cooperative launch, so that
    // every block is resident while others wait for it
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * TY, 0) != cudaSuccess)
            return kLaunchCudaError;
    }
    const int64_t total = int64_t(q.tiles_x) * q.tiles_y * q.n;
    const int grid = int(std::min<int64_t>(total, int64_t(per_sm) * sms));
    if (grid < 1) return kLaunchOk;
    PbasArgs a = a0;
    GmmArgs g = g0;
    SeqArgs qq = q;
    void* args[] = {&a, &g, &qq};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(unsigned(grid)), dim3(32, TY), args, 0, s) ==
                   cudaSuccess
               ? kLaunchOk
               : kLaunchCudaError;
}

template <int NT>
LaunchResult sequence_shape(const PbasArgs& a0, const GmmArgs& g0, const SeqArgs& q, cudaStream_t s, int px, int ty)
{
    if (px == 2 && ty == 8) return sequence_go<NT, 2, 8>(a0, g0, q, s);
    if (px == 2 && ty == 4) return sequence_go<NT, 2, 4>(a0, g0, q, s);
    if (px == 1) return sequence_go<NT, 1, 8>(a0, g0, q, s);
    return kLaunchUnsupported;
}

template <int NT, int PX, int TY>
LaunchResult batch_sequence_go(const SeqBatchTable& t, cudaStream_t s)
{
    auto k = batch_sequence_kernel<NT, PX, TY>;
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * TY, 0) != cudaSuccess)
            return kLaunchCudaError;
    }
    const long long total = t.seg_claim0[t.segs];
    const int grid = int(std::min<long long>(total, static_cast<long long>(per_sm) * sms));
    if (grid < 1) return kLaunchOk;
    SeqBatchTable* tp = const_cast<SeqBatchTable*>(&t);
    void* args[] = {tp};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(unsigned(grid)), dim3(32, TY), args, 0, s) ==
                   cudaSuccess
               ? kLaunchOk
               : kLaunchCudaError;
}

template <int NT>
LaunchResult batch_sequence_shape(const SeqBatchTable& t, cudaStream_t s, int px, int ty)
{
    if (px == 2 && ty == 8) return batch_sequence_go<NT, 2, 8>(t, s);
    if (px == 2 && ty == 4) return batch_sequence_go<NT, 2, 4>(t, s);
    if (px == 1 && ty == 8) return batch_sequence_go<NT, 1, 8>(t, s);
    return kLaunchUnsupported;
}

// Tile shape of the sequence launch for a context's options: 2 px x 8 or 4
// rows when the width allows; otherwise 1 px x 8 rows.
static void sequence_tile(const PbasArgs& a, int& px, int& ty)
{
    px = (a.px == 2 && a.W % 2 == 0) ? 2 : 1;
    ty = px == 2 && a.ty == 4 ? 4 : 8;
}

void fused_sequence_tiles(const PbasArgs& a, int& tiles_x, int& tiles_y)
{
    int px, ty;
    sequence_tile(a, px, ty);
    tiles_x = (a.W + 32 * px - 1) / (32 * px);
    tiles_y = (a.H + ty - 1) / ty;
}

LaunchResult launch_fused_sequence(const PbasArgs& a0, const GmmArgs& g0, const SeqArgs& q, cudaStream_t s)
{
    if (a0.P == 0 || q.n == 0) return kLaunchOk;
    int px, ty;
    sequence_tile(a0, px, ty);
    if (q.tiles_x != (a0.W + 32 * px - 1) / (32 * px) || q.tiles_y != (a0.H + ty - 1) / ty) return kLaunchUnsupported;
    return a0.N == 20 ? sequence_shape<20>(a0, g0, q, s, px, ty) : sequence_shape<0>(a0, g0, q, s, px, ty);
}

LaunchResult launch_batch_sequence(const SeqBatchTable& t, int px, int ty, cudaStream_t s)
{
    static_assert(sizeof(SeqBatchTable) <= 32000, "kernel parameter space");
    if (t.n == 0 || t.seg_claim0[t.segs] == 0) return kLaunchOk;
    seq_batch_prepare_kernel<<<64, 256, 0, s>>>(t);
    if (cudaGetLastError() != cudaSuccess) return kLaunchCudaError;
    seq_batch_grad_kernel<<<dim3(unsigned(t.gtiles), unsigned(t.maxn)), dim3(32, kGradTY), 0, s>>>(t);
    if (cudaGetLastError() != cudaSuccess) return kLaunchCudaError;
    const int N = t.e[0].a.N;
    const LaunchResult r = N == 20 ? batch_sequence_shape<20>(t, s, px, ty) : batch_sequence_shape<0>(t, s, px, ty);
    if (r != kLaunchOk) return r;
    seq_batch_finish_kernel<<<1, 4 * kSeqBatchMax, 0, s>>>(t);
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

LaunchResult launch_grad_sums(const PbasArgs& a0, const SeqArgs& q, unsigned long long* out, cudaStream_t s)
{
    if (a0.P == 0 || q.n == 0) return kLaunchOk;
    const dim3 grid(unsigned((a0.W + 31) / 32), unsigned((a0.H + kGradStrip - 1) / kGradStrip), unsigned(q.n));
    grad_sums_kernel<<<grid, dim3(32, kGradTY), 0, s>>>(a0, q, out);
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

LaunchResult launch_fused_classify(const PbasArgs& a, const GmmArgs& g, cudaStream_t s)
{
    if (a.P == 0) return kLaunchOk;
    const int px = (a.px > 1 && a.W % a.px == 0) ? a.px : 1;
    const int ty = px == 1 ? 8 : a.ty;
    const bool ok = a.N == 20 ? fused_shape<20>(a, g, s, px, ty) : fused_shape<0>(a, g, s, px, ty);
    if (!ok) return kLaunchUnsupported;
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

template <int NT, int KR>
bool batch_shape(const PbasBatchTable& t, int blocks, int px, int ty, cudaStream_t s)
{
    if (px == 2 && ty == 8) pbas_batch_kernel<NT, 2, 8, KR><<<blocks, dim3(32, 8), 0, s>>>(t);
    else if (px == 2 && ty == 4) pbas_batch_kernel<NT, 2, 4, KR><<<blocks, dim3(32, 4), 0, s>>>(t);
    else if (px == 4 && ty == 4) pbas_batch_kernel<NT, 4, 4, KR><<<blocks, dim3(32, 4), 0, s>>>(t);
    else if (px == 4 && ty == 8) pbas_batch_kernel<NT, 4, 8, KR><<<blocks, dim3(32, 8), 0, s>>>(t);
    else if (px == 1 && ty == 8) pbas_batch_kernel<NT, 1, 8, KR><<<blocks, dim3(32, 8), 0, s>>>(t);
    else return false;
    return true;
}

LaunchResult launch_pbas_batch(const PbasBatchTable& t, bool fused, int blocks, int N, int px, int ty,
                               cudaStream_t s)
{
    bool ok;
    if (fused) ok = N == 20 ? batch_shape<20, 3>(t, blocks, px, ty, s) : batch_shape<0, 3>(t, blocks, px, ty, s);
    else ok = N == 20 ? batch_shape<20, 0>(t, blocks, px, ty, s) : batch_shape<0, 0>(t, blocks, px, ty, s);
    if (!ok) return kLaunchUnsupported;
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

LaunchResult launch_pbas_flush(const PbasArgs& a, cudaStream_t s)
{
    if (a.P == 0) return kLaunchOk;
    constexpr int TY = 8;
    const dim3 grid = grid_for<1, TY>(a);
    if (a.N == 20) pbas_flush_kernel<20, TY><<<grid, dim3(32, TY), 0, s>>>(a);
    else pbas_flush_kernel<0, TY><<<grid, dim3(32, TY), 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

#undef FOS_PBAS_LAUNCHER

}  // namespace fos
