// Projection + bilinear feature gather, the MLP's input assembly for Eq. 1
// and Eq. 2 (Sec. 3.1): x = [Phi(P_xy, g(I)) ..., P_z].
//
// Layout: feature maps are channel-last [H][W][C], so the C channels of one
// texel are one contiguous run; a thread owns one point and 16 channels and
// issues four 16-byte loads per bilinear tap (two for a BF16 map), and
// consecutive threads of a warp read consecutive pieces of the same texel
// row (coalesced).
// The 16.8 MB full-size map stays resident in the 129 MB L2 across a frame.
//
// Projection and sampling arithmetic: gather.cuh.
#include <cuda_fp8.h>

#include "gather.cuh"

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

// One thread per (point, group of kQPT quads): the projection and the tap
// positions are computed once per group, then the group's 4 kQPT taps are
// independent 16-byte loads; consecutive threads take consecutive groups of
// the same texel rows (64 contiguous bytes each).
constexpr uint32_t kQPT = 4;

template <typename OutT>
__global__ void __launch_bounds__(256) gather_kernel(PointSrc src, int64_t p0, int64_t m,
                                                     Calib calib, Map map0, Map map1,
                                                     OutT* __restrict__ X, int ldx) {
    const uint32_t nq = (uint32_t)ldx >> 2;
    const uint32_t ng = (nq + kQPT - 1) / kQPT;
    if (src.count) m = min(m, (int64_t)*src.count);
    // m ng < 2^32 (at most 2^22 rows of at most 33 groups): 32-bit division
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * ng;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t lp = (uint32_t)t / ng;
        const uint32_t q0 = ((uint32_t)t - lp * ng) * kQPT;
        const PointSample ps = sample_point(src, p0 + lp, calib, map0, map1);
        OutT* row = X + (int64_t)lp * ldx;
#pragma unroll
        for (uint32_t j = 0; j < kQPT; j += 2) {
            const int c = 4 * (int)(q0 + j);
            if (q0 + j + 1 < nq && oct_bf16(ps, c)) {
                // two quads of a BF16 map: 16-byte taps
                float4 lo, hi;
                sample_oct_bf16(ps, c, lo, hi);
                store4(row + c, lo);
                store4(row + c + 4, hi);
            } else {
                if (q0 + j < nq) store4(row + c, sample_quad(ps, c));
                if (q0 + j + 1 < nq) store4(row + c + 4, sample_quad(ps, c + 4));
            }
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
    const int64_t total = m * ((ldx / 4 + kQPT - 1) / kQPT);
    gather_kernel<float><<<gather_blocks(src, total), 256, 0, stream>>>(src, p0, m, calib, map0,
                                                                       map1, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_gather_bf16(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                               const Map& map0, const Map& map1, __nv_bfloat16* X, int ldx,
                               cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    const int64_t total = m * ((ldx / 4 + kQPT - 1) / kQPT);
    gather_kernel<__nv_bfloat16><<<gather_blocks(src, total), 256, 0, stream>>>(src, p0, m, calib,
                                                                               map0, map1, X, ldx);
    return cudaGetLastError();
}

}  // namespace pifu
