// resample.cu -- depth frame resampled onto the colour grid (Sec. 4.3: the
// sensor's depth resolution can be lower than its colour resolution and the
// paper processes at the colour resolution; it does not say how depth is
// brought there).  Nearest neighbour with floor mapping:
//   out(x, y) = src(floor(x * sw / dw), floor(y * sh / dh)),
// so every output is an input value and the invalid reading 0 is never
// blended into a valid depth.  One thread per output pixel of a row; the
// source row index is uniform per block row.
#include "fos.h"
#include "fos_internal.h"

namespace fos {
namespace {

constexpr int kRsThreads = 256;

__global__ void __launch_bounds__(kRsThreads) depth_resample_kernel(const uint16_t* __restrict__ src, int sw,
                                                                    int sh, uint16_t* __restrict__ dst, int dw,
                                                                    int dh)
{
    const int y = blockIdx.y;
    const int ys = int((int64_t(y) * sh) / dh);
    const uint16_t* row = src + int64_t(ys) * sw;
    uint16_t* out = dst + int64_t(y) * dw;
    for (int x = blockIdx.x * kRsThreads + threadIdx.x; x < dw; x += gridDim.x * kRsThreads)
        out[x] = row[int((int64_t(x) * sw) / dw)];
}

}  // namespace

LaunchResult launch_depth_resample(const uint16_t* src, int sw, int sh, uint16_t* dst, int dw, int dh,
                                   cudaStream_t s)
{
    if (dw <= 0 || dh <= 0) return kLaunchOk;
    const int bx = (dw + kRsThreads - 1) / kRsThreads;
    depth_resample_kernel<<<dim3(unsigned(bx < 64 ? bx : 64), unsigned(dh)), kRsThreads, 0, s>>>(src, sw, sh, dst,
                                                                                                 dw, dh);
    return cudaGetLastError() == cudaSuccess ? kLaunchOk : kLaunchCudaError;
}

}  // namespace fos

extern "C" fos_status fos_depth_resample_device(const uint16_t* d_src, int32_t src_width, int32_t src_height,
                                                uint16_t* d_dst, int32_t dst_width, int32_t dst_height,
                                                void* stream)
{
    using namespace fos;
    set_thread_error("");
    if (!d_src || !d_dst || src_width < 1 || src_height < 1 || dst_width < 1 || dst_height < 1 ||
        src_width > 16384 || src_height > 16384 || dst_width > 16384 || dst_height > 16384) {
        set_thread_error("fos_depth_resample_device: NULL pointer or size outside 1..16384");
        return FOS_ERR_INVALID_ARG;
    }
    if (launch_depth_resample(d_src, src_width, src_height, d_dst, dst_width, dst_height,
                              static_cast<cudaStream_t>(stream)) != kLaunchOk) {
        set_thread_error(cudaGetErrorString(cudaGetLastError()));
        return FOS_ERR_CUDA;
    }
    return FOS_OK;
}
