// pbas_dev.cuh -- device helpers shared by the PBAS kernels (paper Sec. 3.2):
// the tile geometry and input staging (colour, depth converted as in
// Sec. 4.2, 1-pixel halo), the Sobel gradient feature, the pending
// neighbour-request words and how they are applied, the blocked sample
// layout, vector loads and stores, block-wide counter sums, the per-pixel
// random draws and the shared-memory layout of a classify tile.  Every
// operation that enters a result rounds once (explicit _rn intrinsics; the
// including translation units are compiled without contraction).
#pragma once
#include "fos_internal.h"
#include "gmm_dev.cuh"
#include "philox.cuh"

namespace fos {
namespace {

// Neighbour directions N, NE, E, SE, S, SW, W, NW (x to the right, y down).
__host__ __device__ constexpr int dir_dx(int j) { return j == 0 || j == 4 ? 0 : (j < 4 ? 1 : -1); }
__host__ __device__ constexpr int dir_dy(int j) { return j == 2 || j == 6 ? 0 : (j < 2 || j == 7 ? -1 : 1); }

// Depth u16 (mm) -> u8: 0 stays 0 (invalid), the full scale fs maps onto
// 1..255 with round-half-up; the quotient by fs is the context's exact
// multiply-shift (depth_divisor: m, sh).
__device__ __forceinline__ uint32_t depth_to_u8(uint32_t d, uint32_t fs, uint32_t m, int sh)
{
    if (d == 0) return 0;
    const uint32_t q = uint32_t((uint64_t(d * 255u + (fs >> 1)) * m) >> sh);
    return q < 1u ? 1u : (q > 255u ? 255u : q);
}

template <int PX, int TY>
struct Geo {
    static constexpr int TW = 32 * PX;       // tile width (pixels)
    static constexpr int SW = TW + 2;        // staged width with halo
    static constexpr int SH = TY + 2;        // staged height with halo
    static constexpr int SWP = (SW + 3) & ~3;
    static constexpr int CH = SH * SWP;      // bytes per staged channel
};

// Stage the tile plus a 1-pixel halo, edge-clamped, as 4 channel planes
// (R, G, B, depth rescaled to 8 bits; 0 = invalid depth).
template <int PX, int TY>
__device__ __forceinline__ void stage_input(const PbasArgs& a, int x0, int y0, uint8_t* sm)
{
    using G = Geo<PX, TY>;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // depth of another size: the nearest-neighbour source of each colour pixel
    // (products below 2^28 for sizes up to 16384: 32-bit arithmetic)
    const bool mapped = a.Wd != a.W || a.Hd != a.H;
    for (int idx = tid; idx < G::SH * G::SW; idx += 32 * TY) {
        const int r = idx / G::SW, col = idx - r * G::SW;
        const int gx = min(max(x0 - 1 + col, 0), a.W - 1);
        const int gy = min(max(y0 - 1 + r, 0), a.H - 1);
        const int64_t p = int64_t(gy) * a.W + gx;
        const int o = r * G::SWP + col;
        constexpr int n = 4 * G::CH;
        at(sm, o, n, 1, a.oob) = at(a.rgb, 3 * p, 3 * a.P, 2, a.oob);
        at(sm, G::CH + o, n, 1, a.oob) = at(a.rgb, 3 * p + 1, 3 * a.P, 2, a.oob);
        at(sm, 2 * G::CH + o, n, 1, a.oob) = at(a.rgb, 3 * p + 2, 3 * a.P, 2, a.oob);
        const int64_t pd = mapped ? int64_t(uint32_t(gy * a.Hd) / uint32_t(a.H)) * a.Wd +
                                        int64_t(uint32_t(gx * a.Wd) / uint32_t(a.W))
                                  : p;
        at(sm, 3 * G::CH + o, n, 1, a.oob) = uint8_t(depth_to_u8(at(a.depth, pd, depth_extent(a), 3, a.oob), a.depth_fs,
                                                                  a.depth_m, a.depth_sh));
    }
}

// Stage the neighbour-request words of the previous frame with a 1-pixel
// halo; outside the frame there are no requests.
template <int PX, int TY>
__device__ __forceinline__ void stage_requests(const PbasArgs& a, int x0, int y0, uint32_t* sreq)
{
    using G = Geo<PX, TY>;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int idx = tid; idx < G::SH * G::SW; idx += 32 * TY) {
        const int r = idx / G::SW, col = idx - r * G::SW;
        const int gx = x0 - 1 + col, gy = y0 - 1 + r;
        const bool in = gx >= 0 && gx < a.W && gy >= 0 && gy < a.H;
        at(sreq, idx, G::SH * G::SW, 4, a.oob) = in ? at(a.req_prev, int64_t(gy) * a.Wp + gx, a.plane, 5, a.oob) : kReqNone4;
    }
}

// Gradient magnitude: 3x3 Sobel, |gx| + |gy|, >> 3, clamped to 255 (s: one
// staged channel of ch bytes).
__device__ __forceinline__ uint32_t sobel(const uint8_t* s, int swp, int r, int c, int ch = 1 << 30,
                                          OobWord* w = nullptr)
{
    auto px = [&](int i) { return int(at(s, i, ch, 6, w)); };
    const int a00 = px((r - 1) * swp + c - 1), a01 = px((r - 1) * swp + c), a02 = px((r - 1) * swp + c + 1);
    const int a10 = px(r * swp + c - 1), a12 = px(r * swp + c + 1);
    const int a20 = px((r + 1) * swp + c - 1), a21 = px((r + 1) * swp + c), a22 = px((r + 1) * swp + c + 1);
    const int gx = (a02 + 2 * a12 + a22) - (a00 + 2 * a10 + a20);
    const int gy = (a20 + 2 * a21 + a22) - (a00 + 2 * a01 + a02);
    const int m = (abs(gx) + abs(gy)) >> 3;
    return uint32_t(m > 255 ? 255 : m);
}

// Neighbour requests that point at the pixel at staged column `col`, row
// ly+1, as a 32-bit mask: bit 4*j + c is set when the neighbour at -dir(j)
// asked, for channel c, to write into this pixel (its request byte for c is
// (j << 5) | slot; 0x1F means no request).
template <int SW>
__device__ __forceinline__ uint32_t request_matches(const uint32_t* sreq, int ly, int col, int n = 1 << 30,
                                                    OobWord* w = nullptr)
{
    uint32_t mm = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t r = at(sreq, (ly + 1 - dir_dy(j)) * SW + (col - dir_dx(j)), n, 7, w);
        const uint32_t dir_ok = __vcmpeq4(r & 0xE0E0E0E0u, uint32_t(j << 5) * 0x01010101u);
        const uint32_t has = __vcmpne4(r & 0x1F1F1F1Fu, 0x1F1F1F1Fu);
        const uint32_t m = dir_ok & has & 0x08040201u;  // bit c of byte c
        mm |= ((m * 0x01010101u) >> 24) << (4 * j);     // gather the 4 bits
    }
    return mm;
}

// Slot requested by the neighbour at -dir(j) for channel c (a match exists).
template <int SW>
__device__ __forceinline__ int request_slot(const uint32_t* sreq, int ly, int col, int j, int c,
                                            int n = 1 << 30, OobWord* w = nullptr)
{
    const int dy = (j == 2 || j == 6) ? 0 : ((j < 2 || j == 7) ? -1 : 1);
    const int dx = (j == 0 || j == 4) ? 0 : (j < 4 ? 1 : -1);
    return int((at(sreq, (ly + 1 - dy) * SW + (col - dx), n, 8, w) >> (8 * c)) & 31u);
}

// PX pixels of uint16 / float / uint32 planes; PX = 4 uses one vector access.
template <int PX>
__device__ __forceinline__ void ld16(const uint16_t* p, uint32_t (&o)[PX])
{
    if constexpr (PX == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        o[0] = v.x & 0xFFFFu; o[1] = v.x >> 16; o[2] = v.y & 0xFFFFu; o[3] = v.y >> 16;
    } else if constexpr (PX == 2) {
        const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
        o[0] = v & 0xFFFFu; o[1] = v >> 16;
    } else {
        o[0] = *p;
    }
}

template <int PX>
__device__ __forceinline__ void st16(uint16_t* p, const uint32_t (&o)[PX])
{
    if constexpr (PX == 4) *reinterpret_cast<uint2*>(p) = make_uint2(o[0] | (o[1] << 16), o[2] | (o[3] << 16));
    else if constexpr (PX == 2) *reinterpret_cast<uint32_t*>(p) = o[0] | (o[1] << 16);
    else *p = uint16_t(o[0]);
}

// Sample words: slot k of PX pixels as packed (value, gradient) byte pairs.
template <int PX>
struct SWords {
    static constexpr int NW = (PX + 1) / 2;
};

template <int PX>
__device__ __forceinline__ void ldw(const uint16_t* p, uint32_t (&w)[SWords<PX>::NW])
{
    if constexpr (PX == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (PX == 2) {
        w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else {
        w[0] = *p;
    }
}

template <int PX>
__device__ __forceinline__ void ldf(const float* p, float (&o)[PX])
{
    if constexpr (PX == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (PX == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = *p;
    }
}

template <int PX>
__device__ __forceinline__ void stf(float* p, const float (&o)[PX])
{
    if constexpr (PX == 4) *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    else if constexpr (PX == 2) *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    else *p = o[0];
}

template <int PX>
__device__ __forceinline__ void ldu(const uint32_t* p, uint32_t (&o)[PX])
{
    if constexpr (PX == 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (PX == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = *p;
    }
}

template <int PX>
__device__ __forceinline__ void stu(uint32_t* p, const uint32_t (&o)[PX])
{
    if constexpr (PX == 4) *reinterpret_cast<uint4*>(p) = make_uint4(o[0], o[1], o[2], o[3]);
    else if constexpr (PX == 2) *reinterpret_cast<uint2*>(p) = make_uint2(o[0], o[1]);
    else *p = o[0];
}

// Range-checked forms of the plane accesses above: PX elements of `base`
// from element i (extent n, site code for the violation record).
template <int PX>
__device__ __forceinline__ void ldw(const uint16_t* base, int64_t i, int64_t n, int site, OobWord* w,
                                    uint32_t (&o)[SWords<PX>::NW])
{
    if constexpr (PX == 4) {
        const uint2 v = vat<const uint2>(base, i, 4, n, site, w);
        o[0] = v.x; o[1] = v.y;
    } else if constexpr (PX == 2) {
        o[0] = vat<const uint32_t>(base, i, 2, n, site, w);
    } else {
        o[0] = at(base, i, n, site, w);
    }
}

template <int PX, class T, class V2, class V4>
__device__ __forceinline__ void ldv_c(const T* base, int64_t i, int64_t n, int site, OobWord* w, T (&o)[PX])
{
    if constexpr (PX == 4) {
        const V4 v = vat<const V4>(base, i, 4, n, site, w);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (PX == 2) {
        const V2 v = vat<const V2>(base, i, 2, n, site, w);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = at(base, i, n, site, w);
    }
}

template <int PX, class T, class V2, class V4>
__device__ __forceinline__ void stv_c(T* base, int64_t i, int64_t n, int site, OobWord* w, const T (&o)[PX])
{
    if constexpr (PX == 4) {
        V4 v;
        v.x = o[0]; v.y = o[1]; v.z = o[2]; v.w = o[3];
        vat<V4>(base, i, 4, n, site, w) = v;
    } else if constexpr (PX == 2) {
        V2 v;
        v.x = o[0]; v.y = o[1];
        vat<V2>(base, i, 2, n, site, w) = v;
    } else {
        at(base, i, n, site, w) = o[0];
    }
}

template <int PX>
__device__ __forceinline__ void ldf(const float* b, int64_t i, int64_t n, int site, OobWord* w, float (&o)[PX])
{
    ldv_c<PX, float, float2, float4>(b, i, n, site, w, o);
}
template <int PX>
__device__ __forceinline__ void stf(float* b, int64_t i, int64_t n, int site, OobWord* w, const float (&o)[PX])
{
    stv_c<PX, float, float2, float4>(b, i, n, site, w, o);
}
template <int PX>
__device__ __forceinline__ void ldu(const uint32_t* b, int64_t i, int64_t n, int site, OobWord* w,
                                    uint32_t (&o)[PX])
{
    ldv_c<PX, uint32_t, uint2, uint4>(b, i, n, site, w, o);
}
template <int PX>
__device__ __forceinline__ void stu(uint32_t* b, int64_t i, int64_t n, int site, OobWord* w,
                                    const uint32_t (&o)[PX])
{
    stv_c<PX, uint32_t, uint2, uint4>(b, i, n, site, w, o);
}

// Block-wide sums of per-thread counters: v[q] is added to dst(q) with one
// atomicAdd per counter per block (dst maps a counter index to its address).
template <int TY, int NV, class Dst>
__device__ __forceinline__ void block_add(const uint32_t (&v)[NV], Dst dst)
{
    __shared__ uint32_t red[NV][TY];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, v[q]);
        if (threadIdx.x == 0) red[q][threadIdx.y] = s;
    }
    __syncthreads();
    if (threadIdx.y == 0 && threadIdx.x < NV) {
        unsigned long long s = 0;
#pragma unroll
        for (int w = 0; w < TY; ++w) s += red[threadIdx.x][w];
        if (s) atomicAdd(dst(threadIdx.x), s);
    }
}

// Index of sample / D element (c, k) of pixel (x, y) in the blocked layout.
__device__ __forceinline__ int64_t sidx(const PbasArgs& a, int N, int c, int k, int x, int y)
{
    const int64_t seg = int64_t(y) * a.spr + (x >> 7);
    return ((int64_t(c) * a.nseg + seg) * N + k) * kSeg + (x & (kSeg - 1));
}

// Neighbour updates of frame t-1 into pixel (x, y) (staged at row ly + 1,
// column col; mm from request_matches), base method: every asked slot takes
// the pixel's own frame-(t-1) value pw (4 x (value | gradient << 8)); the
// depth slot only if that depth was valid.  Every writer of a slot writes
// the same value, so the order does not matter.  Returns the writes made.
template <int SW>
__device__ __forceinline__ uint32_t apply_own_value(const PbasArgs& a, int N, const uint32_t* sreq, int ly,
                                                    int col, int x, int y, uint32_t mm, uint64_t pw,
                                                    int nreq = 1 << 30)
{
    if (((pw >> 48) & 0xFFu) == 0u) mm &= 0x77777777u;
    uint32_t n = 0;
    while (mm) {
        const int b = __ffs(mm) - 1;
        mm &= mm - 1u;
        const int j = b >> 2, c = b & 3;
        const int k = request_slot<SW>(sreq, ly, col, j, c, nreq, a.oob);
        at(a.samp, sidx(a, N, c, k, x, y), samp_extent(a), 9, a.oob) = uint16_t(pw >> (16 * c));
        ++n;
    }
    return n;
}

// Spatial propagation: an asked slot takes the requester's frame-(t-1) value
// (prev_src at the requester).  A slot the pixel's own update of frame t-1
// wrote (byte c of `own`, 0x1F for none) keeps it; among requests for the
// same slot, the requester at the lowest direction index jy seen from this
// pixel wins (it made request j = jy ^ 4).  Rotating the mask by 16 bits
// turns bit 4j + c into bit 4jy + c; walking it from the top writes the
// winner last.  Returns the writes made.
template <int SW>
__device__ __forceinline__ uint32_t apply_propagated(const PbasArgs& a, int N, const uint32_t* sreq, int ly,
                                                     int col, int x, int y, uint32_t mm, uint32_t own,
                                                     int nreq = 1 << 30)
{
    mm = __byte_perm(mm, 0u, 0x1032);
    uint32_t n = 0;
    while (mm) {
        const int b = 31 - __clz(mm);
        mm &= ~(1u << b);
        const int j = (b >> 2) ^ 4, c = b & 3;
        const int k = request_slot<SW>(sreq, ly, col, j, c, nreq, a.oob);
        if (uint32_t(k) == ((own >> (8 * c)) & 0xFFu)) continue;
        const uint64_t src = at(a.prev_src, int64_t(y - dir_dy(j)) * a.Wp + (x - dir_dx(j)), a.plane, 10, a.oob);
        at(a.samp, sidx(a, N, c, k, x, y), samp_extent(a), 11, a.oob) = uint16_t(src >> (16 * c));
        ++n;
    }
    return n;
}

// Byte c of the own-slot words of PX pixels: the slot of this frame's own
// update in channel c, or 0x1F (slot == nullptr or negative).
template <int PX>
__device__ __forceinline__ void put_own_slots(const PbasArgs& a, int64_t q0, int c, const bool (&inb)[PX],
                                              const int* slot)
{
#pragma unroll
    for (int i = 0; i < PX; ++i)
        if (inb[i])
            at(reinterpret_cast<uint8_t*>(a.own), 4 * (q0 + i) + c, 4 * a.plane, 12, a.oob) =
                uint8_t(slot && slot[i] >= 0 ? slot[i] : 0x1F);
}

struct Draws {
    bool coin1, coin2;
    uint32_t k1, j, k2;
};

// Random draws for pixel p, frame t, channel c: Philox4x32-10 with counter
// (p, t, c, 0) and key (seed, stream_id), its round keys precomputed in a.rk.
// Words 0 and 2 give the two coins (24-bit uniform < prob = fl(1/T), T the
// pixel's learning parameter before this frame's update), word 1 the own
// slot, word 3 the direction (3 bits)
// and the neighbour slot (29 bits).
__device__ __forceinline__ Draws draws(const PbasArgs& a, uint32_t p, uint32_t c, float prob, int N)
{
    Draws d;
    if (a.forced) {  // test draws (see fos_params.forced_rng)
        const uint32_t col = p % uint32_t(a.W), row = p / uint32_t(a.W);
        d.coin1 = d.coin2 = true;
        d.k1 = a.t % uint32_t(N);
        d.k2 = (a.t + 1u) % uint32_t(N);
        if (a.forced == 1) {
            d.j = a.t % 8u;
        } else if (a.forced == 2) {  // east from columns 0, 1 (mod 4), west from 2, 3
            d.j = ((col >> 1) & 1u) == 0u ? 2u : 6u;
        } else {  // north from even columns, south-east from odd; even rows ask for k1
            d.j = (col & 1u) == 0u ? 0u : 3u;
            if ((row & 1u) == 0u) d.k2 = d.k1;
        }
        return d;
    }
    const uint4 u = philox4x32_10_rk(make_uint4(p, a.t, c, 0u), a.rk);
    const float two_m24 = 5.9604644775390625e-8f;
    d.coin1 = __fmul_rn(__uint2float_rn(u.x >> 8), two_m24) < prob;
    d.k1 = __umulhi(u.y, uint32_t(N));
    d.coin2 = __fmul_rn(__uint2float_rn(u.z >> 8), two_m24) < prob;
    d.j = u.w >> 29;
    d.k2 = uint32_t((uint64_t(u.w & 0x1FFFFFFFu) * uint64_t(N)) >> 29);
    return d;
}

// GMM classify + update (Sec. 3.1) of the tile's own pixels, reading the
// colour and the converted depth from the staged tile (fused GMM+PBAS path).
// The model state and the mask are addressed as in the GMM kernels.
template <int KR, int KD, int PX, int TY, bool PAIR = true>
__device__ __forceinline__ void gmm_tile_part(const GmmArgs& g, const PbasArgs& a, int x0, int y0,
                                              const uint8_t* sm)
{
    using G = Geo<PX, TY>;
    const int lx0 = threadIdx.x * PX, ly = threadIdx.y;
    const int x = x0 + lx0, y = y0 + ly;
    if (y >= a.H || x >= a.W) return;
    const int64_t p0 = int64_t(y) * a.W + x;
    const int o = (ly + 1) * G::SWP + lx0 + 1;
    constexpr int n = 4 * G::CH;
    auto st = [&](int i) { return uint32_t(at(sm, i, n, 13, a.oob)); };
    if constexpr (PX == 2 && PAIR) {
        // W is even on this path: both pixels in the frame, 8-byte state accesses
        const uint32_t r[2] = {st(o), st(o + 1)}, gg[2] = {st(G::CH + o), st(G::CH + o + 1)};
        const uint32_t b[2] = {st(2 * G::CH + o), st(2 * G::CH + o + 1)};
        const uint32_t d8[2] = {st(3 * G::CH + o), st(3 * G::CH + o + 1)};
        if (!g.init) {
            const uint32_t m = gmmdev::gmm_pair<KR, KD>(g, p0, r, gg, b, d8);
            if ((reinterpret_cast<uintptr_t>(g.mask) & 1u) == 0) {  // p0 is even
                vat<uint16_t>(g.mask, p0, 2, g.P, 14, g.oob) = uint16_t(m);
            } else {
                at(g.mask, p0, g.P, 14, g.oob) = uint8_t(m);
                at(g.mask, p0 + 1, g.P, 14, g.oob) = uint8_t(m >> 8);
            }
            return;
        }
    }
#pragma unroll 1
    for (int i = 0; i < PX; ++i) {
        if (x + i >= a.W) break;
        at(g.mask, p0 + i, g.P, 14, g.oob) =
            gmmdev::gmm_pixel_lowreg<KR, KD>(g, p0 + i, st(o + i), st(G::CH + o + i), st(2 * G::CH + o + i),
                                             st(3 * G::CH + o + i));
    }
}

// L1 prefetch of the 128-byte line holding p (a hint: no result, no fault
// semantics are relied on; every address passed is inside its buffer).
__device__ __forceinline__ void prefetch_l1(const void* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Prefetch of what channel c of this thread's pixels reads first: its N
// sample slots and R, T, S.  Issued one channel ahead, so the loads of the
// next channel find their lines in L1 (the kernel is latency-bound; deeper
// prefetch evicts lines before use).
template <int NT>
__device__ __forceinline__ void prefetch_channel(const PbasArgs& a, int N, int c, int x, int y, int64_t q0)
{
    const int64_t s0 = sidx(a, N, c, 0, x, y);
#pragma unroll(NT > 0 ? NT : 4)
    for (int k = 0; k < N; ++k) prefetch_l1(&at(a.samp, s0 + int64_t(k) * kSeg, samp_extent(a), 15, a.oob));
    const int64_t pc = int64_t(c) * a.plane + q0;
    prefetch_l1(&at(a.R, pc, rts_extent(a), 15, a.oob));
    prefetch_l1(&at(a.T, pc, rts_extent(a), 15, a.oob));
    prefetch_l1(&at(a.S, pc, rts_extent(a), 15, a.oob));
}

// fl(S / d) for an integer 0 <= S < 2^24 and an integer divisor 1 <= d < 2^23,
// given z = fl(1/d): the quotient from the product, corrected once with the
// exact remainder (both steps fused multiply-adds).  The result is the
// correctly rounded quotient: the remainder r = S - q0 d is exact, the
// corrected value q0 + r z differs from S/d by |r (z - 1/d)| < ulp(S/d) 2^-24,
// while a quotient of two integers that is not a float lies at least
// ulp/(2d) from every rounding midpoint (and is never on one here, since d's
// odd part divides neither side of a midpoint at these magnitudes).  Three
// instructions instead of the general division's twenty.
__device__ __forceinline__ float div_int_const(uint32_t S, float d, float z)
{
    const float y = __uint2float_rn(S);
    const float q0 = __fmul_rn(y, z);
    const float r = __fmaf_rn(-q0, d, y);
    return __fmaf_rn(r, z, q0);
}

// Shared memory of one classify tile.
template <int PX, int TY>
struct ClassifySmem {
    using G = Geo<PX, TY>;
    __align__(16) uint8_t sm[4 * G::CH];  // staged channels with halo
    uint32_t sreq[G::SH * G::SW];         // staged request words with halo
    float wgs[4];
    float rn16;                           // fl(1 / (16 N)) for div_int_const
};

}  // namespace
}  // namespace fos
