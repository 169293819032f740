// Projection + bilinear feature gather, the MLP's input assembly for Eq. 1
// and Eq. 2 (Sec. 3.1): x = [Phi(P_xy, g(I)) ..., P_z].
//
// Layout: feature maps are channel-last [H][W][C], so the C channels of one
// texel are one contiguous run; four threads share a point, and each load
// instruction reads four consecutive 16-byte pieces of a texel row per point.
// The 16.8 MB full-size map stays resident in the 129 MB L2 across a frame.
//
// Projection and sampling arithmetic: gather.cuh.
#include <cuda_fp8.h>

#include "gather.cuh"
#include "sm100.cuh"

namespace pifu {
namespace {

__device__ __forceinline__ void store4(float* X, float4 r) {
    *reinterpret_cast<float4*>(X) = r;
}

__device__ __forceinline__ void store4(__nv_bfloat16* X, float4 r) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(r.x, r.y);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(r.z, r.w);
    uint2 v;
    v.x = *reinterpret_cast<const uint32_t*>(&lo);
    v.y = *reinterpret_cast<const uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(X) = v;
}

// kTPP threads per point: thread i of a point takes its row's quads i,
// i + kTPP, i + 2 kTPP, ... (four at a time, their taps' loads all in
// flight), so each load instruction reads kTPP consecutive 16-byte pieces
// of a texel row per point; with BF16 maps whose channels come in groups of
// 8, thread i takes the 8-channel groups i, i + kTPP, ... (two at a time, one
// 16-byte load per tap each), then the row's last quads (depth, padding).
// Every thread computes the point's projection and tap positions, so fewer
// threads per point do less of that and more loads each: at 2^17 points of
// the full-size map, 1 / 2 / 4 / 8 / 16 / 32 threads per point took 175 /
// 86 / 67 / 75 / 95 / 109 us (FP32 map) and 109 / 70 / 50 / 54 / 74 / 90 us
// (BF16 map), against 103 / 66 us with 17 threads of four consecutive quads.
constexpr uint32_t kTPP = 4;

template <typename OutT>
__global__ void __launch_bounds__(256) gather_kernel(PointSrc src, int64_t p0, int64_t m,
                                                     Calib calib, Map map0, Map map1,
                                                     OutT* __restrict__ X, int ldx) {
    // a programmatic dependent of the kernel before it (which may write the
    // point list or the hits it reads); its own dependents may be placed now
    sm100::griddep_wait();
    sm100::griddep_launch_dependents();
    const int nq = ldx >> 2;
    if (src.count) m = min(m, (int64_t)*src.count);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * kTPP;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lp = t / kTPP;
        const int i = (int)(t - lp * kTPP);
        const PointSample ps = sample_point(src, p0 + lp, calib, map0, map1);
        OutT* row = X + lp * ldx;
        const int C0 = ps.map0.C, C1 = ps.map1.C;
        int q_first = i;
        if (ps.map0.dtype == 1 && (C0 & 7) == 0 && (C1 == 0 || (ps.map1.dtype == 1 && (C1 & 7) == 0))) {
            const int no = (C0 + C1) >> 3;
            for (int o0 = i; o0 < no; o0 += 2 * kTPP) {
                float4 v[4];
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (o0 + j * (int)kTPP < no)
                        sample_oct_bf16(ps, 8 * (o0 + j * kTPP), v[2 * j], v[2 * j + 1]);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int o = o0 + j * kTPP;
                    if (o < no) {
                        store4(row + 8 * o, v[2 * j]);
                        store4(row + 8 * o + 4, v[2 * j + 1]);
                    }
                }
            }
            q_first = ((C0 + C1) >> 2) + i;
        }
        for (int q0 = q_first; q0 < nq; q0 += 4 * kTPP) {
            float4 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (q0 + j * (int)kTPP < nq) v[j] = sample_quad(ps, 4 * (q0 + j * kTPP));
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (q0 + j * (int)kTPP < nq) store4(row + 4 * (q0 + j * kTPP), v[j]);
        }
    }
}

// One thread per (point, 4 channels); a device-resident count gets a fixed,
// SM-filling grid that strides over whatever the count turns out to be.
inline unsigned gather_blocks(const PointSrc& src, int64_t total) {
    const int64_t exact = (total + 255) / 256;
    return (unsigned)(src.count ? (exact < 152 * 16 ? exact : 152 * 16) : exact);
}

}  // namespace

cudaError_t launch_gather(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                          const Map& map0, const Map& map1, float* X, int ldx,
                          cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    const int64_t total = m * kTPP;
    return launch_pdl(gather_kernel<float>, dim3(gather_blocks(src, total)), dim3(256), 0, stream,
                      src, p0, m, calib, map0, map1, X, ldx);
}

cudaError_t launch_gather_bf16(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                               const Map& map0, const Map& map1, __nv_bfloat16* X, int ldx,
                               cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    const int64_t total = m * kTPP;
    return launch_pdl(gather_kernel<__nv_bfloat16>, dim3(gather_blocks(src, total)), dim3(256), 0,
                      stream, src, p0, m, calib, map0, map1, X, ldx);
}

}  // namespace pifu
