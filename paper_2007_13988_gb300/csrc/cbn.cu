// The paper's final occupancy network (Appendix, "Depth Representation",
// Eq. 7, and "Pixel-aligned 3D Lifting", Eq. 8) in FP32: the depth enters as
// its soft one-hot vector Z, the pixel-aligned feature c conditions five
// blocks of conditional batch normalization:
//
//   h_0 = Wz Z + bz;  per block i:
//   a_i = ReLU(gamma_i(c) (h_{i-1} - mu_i) / sqrt(var_i + eps) + beta_i(c)),
//   h_i = W_i a_i + b_i;   O = sigmoid(h_last),
//
// with gamma_i(c) = Gg_i c + gg_i and beta_i(c) = Gb_i c + gb_i.  The running
// statistics are folded on the host into the linear layer before each block
// (n_i = s_i (h_{i-1} - mu_i) = (s_i W) a + s_i (b - mu_i)), and Z has two
// non-zero weights, so the input layer is a linear interpolation of two
// columns of the folded Wz.
//
// One CTA walks 32-point tiles: it gathers the tile's features into shared
// memory (channel-major, so every thread of a GEMM step reads the same
// values), then per block computes the 2K gamma/beta outputs, the ReLU, and
// the K outputs of the next linear layer, and finally the logit with one warp
// per point.  Weights are stored input-major, so a warp's loads of one input
// row are contiguous.  This is the reference arithmetic of the CBN network:
// the plain FP32 form, the re-evaluation of the MIXED form and small batches.
#include <algorithm>

#include "epilogue.cuh"
#include "gather.cuh"

namespace pifu {
namespace {

constexpr int kP = kCbnTile;       // points per tile
constexpr int kLd = kP + 4;        // row stride of the [channel][point] arrays
constexpr int kThreads = 256;
constexpr int kPG = 16;            // points per GEMM work item

// SoftZ of Eq. 7 for depth z: lower index i (<= n_z - 2) and the weight t of
// index i + 1 (Z_i = 1 - t).  P'_z is clamped to [0, 1]; at P'_z = 1 the pair
// (n_z - 2, n_z - 1) with t = 1 gives the same vector as Eq. 7.
__device__ __forceinline__ void soft_z(float z, int n_z, int& i, float& t) {
    const float p = fminf(fmaxf(0.5f * (z + 1.0f), 0.0f), 1.0f);
    const float x = (float)(n_z - 1) * p;
    i = min((int)floorf(x), n_z - 2);
    t = x - (float)i;
}

// out[o][p] = bias[o] + sum_k WT[k][o] in[k][p] for o < n_out, p < kP;
// in / out are [channel][kLd] shared-memory arrays.
__device__ __forceinline__ void tile_gemm(const float* __restrict__ WT,
                                          const float* __restrict__ bias, int n_in, int n_out,
                                          const float* in, float* out) {
    const int items = n_out * (kP / kPG);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int o = it % n_out;
        const int g = it / n_out;
        float acc[kPG];
#pragma unroll
        for (int j = 0; j < kPG; ++j) acc[j] = 0.f;
        const float* ip = in + g * kPG;
        const float* wp = WT + o;
#pragma unroll 4
        for (int k = 0; k < n_in; ++k) {
            const float w = __ldg(wp + (int64_t)k * n_out);
            const float4* a = reinterpret_cast<const float4*>(ip + k * kLd);
#pragma unroll
            for (int q = 0; q < kPG / 4; ++q) {
                const float4 v = a[q];
                acc[4 * q + 0] = fmaf(w, v.x, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(w, v.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(w, v.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(w, v.w, acc[4 * q + 3]);
            }
        }
        const float b = __ldg(bias + o);
        float* op = out + o * kLd + g * kPG;
#pragma unroll
        for (int j = 0; j < kPG; ++j) op[j] = acc[j] + b;
    }
}

__global__ void __launch_bounds__(kThreads) cbn_f32_kernel(CbnF32 net, PointSrc src, int64_t m,
                                                           Calib calib, Map map, Epilogue epi) {
    extern __shared__ __align__(16) float sm[];
    const int C = net.C, K = net.K;
    float* cS = sm;                       // [C][kLd] features
    float* nS = cS + C * kLd;             // [K][kLd] normalized block input
    float* gS = nS + K * kLd;             // [2K][kLd] gamma | beta; a overwrites gamma
    float* tS = gS + 2 * K * kLd;         // [kP] SoftZ weight of the upper index
    int* iS = reinterpret_cast<int*>(tS + kP);   // [kP] SoftZ lower index
    const Map none{nullptr, 0, 0, 0, 0};
    const int nq = C / 4 + 1;             // feature quads + the depth quad
    const int64_t ntiles = (m + kP - 1) / kP;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p0 = tile * kP;
        const int np = (int)(m - p0 < (int64_t)kP ? m - p0 : (int64_t)kP);
        for (int w = threadIdx.x; w < kP * nq; w += blockDim.x) {
            const int p = w % kP;
            const int q = w / kP;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < np) v = gather_quad(src, p0 + p, calib, map, none, 4 * q);
            if (q < C / 4) {
                cS[(4 * q + 0) * kLd + p] = v.x;
                cS[(4 * q + 1) * kLd + p] = v.y;
                cS[(4 * q + 2) * kLd + p] = v.z;
                cS[(4 * q + 3) * kLd + p] = v.w;
            } else {
                int i;
                float t;
                soft_z(v.x, net.n_z, i, t);
                iS[p] = i;
                tS[p] = t;
            }
        }
        __syncthreads();
        // normalized input of block 0: (1 - t) Wz'[:, i] + t Wz'[:, i + 1] + bz'
        for (int w = threadIdx.x; w < K * kP; w += blockDim.x) {
            const int k = w / kP;
            const int p = w % kP;
            const int i = iS[p];
            const float t = tS[p];
            const float lo = __ldg(net.WzT + (int64_t)i * K + k);
            const float hi = __ldg(net.WzT + (int64_t)(i + 1) * K + k);
            nS[k * kLd + p] = fmaf(t, hi, fmaf(1.0f - t, lo, __ldg(net.bz + k)));
        }
        __syncthreads();
        for (int blk = 0; blk < net.nb; ++blk) {
            tile_gemm(net.Gt + (int64_t)blk * C * 2 * K, net.g0 + (int64_t)blk * 2 * K, C, 2 * K,
                      cS, gS);
            __syncthreads();
            for (int w = threadIdx.x; w < K * kP; w += blockDim.x) {
                const int k = w / kP;
                const int p = w % kP;
                const int e = k * kLd + p;
                gS[e] = fmaxf(fmaf(gS[e], nS[e], gS[K * kLd + e]), 0.0f);
            }
            __syncthreads();
            if (blk + 1 < net.nb) {
                tile_gemm(net.WT + (int64_t)blk * K * K, net.bl + (int64_t)blk * K, K, K, gS, nS);
                __syncthreads();
            }
        }
        // logit = wlast . a + blast, one warp per point
        const int warp = threadIdx.x >> 5;
        const int lane = threadIdx.x & 31;
        for (int p = warp; p < np; p += blockDim.x >> 5) {
            float acc = 0.f;
            for (int k = lane; k < K; k += 32) acc = fmaf(__ldg(net.wlast + k), gS[k * kLd + p], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const float t[4] = {acc, 0.f, 0.f, 0.f};
                last_epilogue(epi, p0 + p, 1, t, net.blast);
            }
        }
        __syncthreads();
    }
}

size_t smem_bytes(const CbnF32& net) {
    return (size_t)(net.C + 3 * net.K) * kLd * 4 + 2 * kP * 4;
}

}  // namespace

bool cbn_f32_ok(const CbnF32& net) {
    return net.C % 4 == 0 && net.C >= 4 && net.K >= 1 && net.n_z >= 2 && net.nb >= 1 &&
           smem_bytes(net) <= 227 * 1024;
}

cudaError_t launch_cbn_f32(const CbnF32& net, const PointSrc& src, int64_t m, const Calib& calib,
                           const Map& map, const Epilogue& epi, cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    if (!cbn_f32_ok(net)) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(net);
    cudaError_t e = cudaFuncSetAttribute(cbn_f32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (m + kP - 1) / kP;
    const int per_sm = smem <= 113 * 1024 ? 2 : 1;
    const int64_t grid = std::min<int64_t>(tiles, 152 * per_sm);
    cbn_f32_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(net, src, m, calib, map, epi);
    return cudaGetLastError();
}

}  // namespace pifu
