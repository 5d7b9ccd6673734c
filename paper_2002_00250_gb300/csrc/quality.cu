// quality.cu -- the quality indicators of the paper's evaluation (Sec. 5):
// confusion counts of foreground masks against ground truth, and PWC, FNR,
// FPR and Si from them.
//
// A byte is foreground when it is non-zero, in the mask and in the ground
// truth alike.  The counting pass reads both arrays once (2 bytes per pixel,
// HBM-bound): 16-byte loads, a per-byte compare (__vcmpne4 gives 0xFF for a
// non-zero byte) and a population count per class, a warp reduction and one
// 64-bit atomic per counter per block.
#include "fos.h"
#include "fos_internal.h"

namespace fos {
namespace {

constexpr int kQThreads = 256;

// Class bits of four bytes: M, G = 0xFF where mask / ground truth is set.
__device__ __forceinline__ void count_word(uint32_t mw, uint32_t gw, uint32_t& tp, uint32_t& tn,
                                           uint32_t& fp, uint32_t& fn)
{
    const uint32_t M = __vcmpne4(mw, 0u), G = __vcmpne4(gw, 0u);
    tp += __popc(M & G);
    tn += __popc(~M & ~G);
    fp += __popc(M & ~G);
    fn += __popc(~M & G);
}

// Counts in units of 8 (each byte contributes 8 set bits) over n bytes:
// the vector body over 16-byte chunks when both pointers are aligned, bytes
// otherwise and for the tail.
__global__ void __launch_bounds__(kQThreads) quality_kernel(const uint8_t* __restrict__ mask,
                                                            const uint8_t* __restrict__ gt, int64_t n,
                                                            int vec, unsigned long long* counts)
{
    uint32_t c[4] = {0, 0, 0, 0};  // set-bit counts of the vector body: tp, tn, fp, fn
    unsigned long long acc[4] = {0, 0, 0, 0};
    const int64_t stride = int64_t(gridDim.x) * kQThreads;
    const int64_t tid = int64_t(blockIdx.x) * kQThreads + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t nv = n / 16;
        const uint4* m4 = reinterpret_cast<const uint4*>(mask);
        const uint4* g4 = reinterpret_cast<const uint4*>(gt);
        int iter = 0;
        for (int64_t i = tid; i < nv; i += stride) {
            const uint4 a = m4[i], b = g4[i];
            count_word(a.x, b.x, c[0], c[1], c[2], c[3]);
            count_word(a.y, b.y, c[0], c[1], c[2], c[3]);
            count_word(a.z, b.z, c[0], c[1], c[2], c[3]);
            count_word(a.w, b.w, c[0], c[1], c[2], c[3]);
            if (++iter == (1 << 20)) {  // 128 bits per chunk: flush long before 32-bit overflow
#pragma unroll
                for (int q = 0; q < 4; ++q) { acc[q] += c[q]; c[q] = 0; }
                iter = 0;
            }
        }
        done = nv * 16;
    }
    for (int64_t i = done + tid; i < n; i += stride) {  // 64-bit counts: any length
        const bool m = mask[i] != 0, g = gt[i] != 0;
        acc[0] += (m && g) ? 8u : 0u;
        acc[1] += (!m && !g) ? 8u : 0u;
        acc[2] += (m && !g) ? 8u : 0u;
        acc[3] += (!m && g) ? 8u : 0u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += c[q];
    __shared__ unsigned long long red[4][kQThreads / 32];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned long long v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long v = 0;
#pragma unroll
        for (int w = 0; w < kQThreads / 32; ++w) v += red[threadIdx.x][w];
        if (v) atomicAdd(counts + threadIdx.x, v / 8ull);
    }
}

}  // namespace
}  // namespace fos

extern "C" {

fos_status fos_quality_counts_device(const uint8_t* d_mask, const uint8_t* d_gt, int64_t n_pixels,
                                     uint64_t* d_counts, void* stream)
{
    using namespace fos;
    set_thread_error("");
    if (n_pixels < 0 || (n_pixels > 0 && (!d_mask || !d_gt)) || !d_counts) {
        set_thread_error("fos_quality_counts_device: NULL pointer or negative size");
        return FOS_ERR_INVALID_ARG;
    }
    if (n_pixels == 0) return FOS_OK;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return FOS_ERR_CUDA;
    }
    const int vec = (reinterpret_cast<uintptr_t>(d_mask) % 16 == 0 && reinterpret_cast<uintptr_t>(d_gt) % 16 == 0) ? 1 : 0;
    // enough blocks to keep every SM streaming, never more than there is work
    const int64_t work = vec ? (n_pixels / 16 + kQThreads - 1) / kQThreads + 1 : (n_pixels + kQThreads - 1) / kQThreads;
    const int blocks = int(work < int64_t(sms) * 8 ? work : int64_t(sms) * 8);
    quality_kernel<<<blocks, kQThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        d_mask, d_gt, n_pixels, vec, reinterpret_cast<unsigned long long*>(d_counts));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return FOS_ERR_CUDA;
    }
    return FOS_OK;
}

void fos_quality_metrics(const uint64_t counts[4], double out[4])
{
    const double tp = double(counts[0]), tn = double(counts[1]), fp = double(counts[2]), fn = double(counts[3]);
    out[0] = 100.0 * (fn + fp) / (tp + fn + fp + tn);  // PWC, percent of wrong classifications
    out[1] = fn / (tp + fn);                            // FNR
    out[2] = fp / (fp + tn);                            // FPR
    out[3] = tp / (tp + fp + fn);                       // Si, similarity
}

}  // extern "C"
