// The paper's final occupancy network (Appendix, "Depth Representation",
// Eq. 7, and "Pixel-aligned 3D Lifting", Eq. 8) in FP32: the depth enters as
// its soft one-hot vector Z, the pixel-aligned feature c conditions the
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
// Conditional batch normalization acts channel by channel, which sets the
// work split: a cluster of kS CTAs owns a tile of kP points, and CTA r owns
// channels [r Kc, (r + 1) Kc) (Kc = K / kS) in every block.  For its channels
// it computes gamma and beta (a 2 Kc x C slice of the contraction over the
// feature), the normalized input n (its slice of the previous linear layer),
// and a, which it stores into every CTA's copy of the full a through
// distributed shared memory; one cluster barrier per block publishes a, and
// the next linear layer's slice reads all of it.  The tile's features are
// gathered once per cluster (each CTA a slice of the channels, broadcast the
// same way).  Each CTA's weight slice of a block (C x 2 Kc + K x Kc floats,
// contiguous on the host) is loaded into registers during the previous
// block's arithmetic and stored into a shared-memory double buffer, so the
// inner loops read shared memory only.
//
// This is the reference arithmetic of the CBN network: the plain FP32 form,
// the re-evaluation of the MIXED form and small batches, whose latency the
// cluster split keeps low (a tile's arithmetic and weights are spread over
// kS SMs).  The only waits are hardware cluster barriers, which every CTA of
// a cluster reaches the same number of times.
#include <cooperative_groups.h>

#include <algorithm>

#include "epilogue.cuh"
#include "gather.cuh"

namespace cg = cooperative_groups;

namespace pifu {
namespace {

constexpr int kS = kCbnCluster;    // CTAs per cluster
constexpr int kP = 32;             // points per tile
constexpr int kLd = kP + 4;        // row stride of the [channel][point] arrays
constexpr int kThreads = 256;
constexpr int kPG = 4;             // points per GEMM work item
constexpr int kPf = kCbnPrefetch;  // float4 registers of the weight prefetch per thread

// SoftZ of Eq. 7 for depth z: lower index i (<= n_z - 2) and the weight t of
// index i + 1 (Z_i = 1 - t).  P'_z is clamped to [0, 1]; at P'_z = 1 the pair
// (n_z - 2, n_z - 1) with t = 1 gives the same vector as Eq. 7.
__device__ __forceinline__ void soft_z(float z, int n_z, int& i, float& t) {
    const float p = fminf(fmaxf(0.5f * (z + 1.0f), 0.0f), 1.0f);
    const float x = (float)(n_z - 1) * p;
    i = min((int)floorf(x), n_z - 2);
    t = x - (float)i;
}

// out[o][p] = bias[o] + sum_k W[k][o] in[k][p] for o < n_out, p < kP; W is
// [n_in][n_out] and in / out are [channel][kLd], all in shared memory.  A
// warp's work items share their points (broadcast reads) and take
// consecutive outputs (conflict-free weight reads).
__device__ __forceinline__ void tile_gemm(const float* W, const float* __restrict__ bias,
                                          int n_in, int n_out, const float* in, float* out) {
    const int items = n_out * (kP / kPG);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int o = it % n_out;
        const int g = it / n_out;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const float* ip = in + g * kPG;
#pragma unroll 8
        for (int k = 0; k < n_in; ++k) {
            const float w = W[k * n_out + o];
            const float4 v = *reinterpret_cast<const float4*>(ip + k * kLd);
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
            acc.z = fmaf(w, v.z, acc.z);
            acc.w = fmaf(w, v.w, acc.w);
        }
        const float b = __ldg(bias + o);
        float* op = out + o * kLd + g * kPG;
        op[0] = acc.x + b;
        op[1] = acc.y + b;
        op[2] = acc.z + b;
        op[3] = acc.w + b;
    }
}

// Weight slice of block `blk` for CTA r: the gamma/beta part (C x 2Kc), then
// the linear part (K x Kc) unless blk is the last block.
struct Slice {
    const float4* g;
    const float4* w;
    int ng, nw;   // float4 counts
};

__device__ __forceinline__ Slice slice_of(const CbnF32& net, int blk, int r) {
    const int Kc = net.K / kS;
    const int64_t gsz = (int64_t)net.C * 2 * Kc, wsz = (int64_t)net.K * Kc;
    Slice s;
    s.g = reinterpret_cast<const float4*>(net.GS + ((int64_t)blk * kS + r) * gsz);
    s.ng = (int)(gsz / 4);
    const bool lin = blk + 1 < net.nb;
    s.w = lin ? reinterpret_cast<const float4*>(net.WS + ((int64_t)blk * kS + r) * wsz) : nullptr;
    s.nw = lin ? (int)(wsz / 4) : 0;
    return s;
}

__device__ __forceinline__ void prefetch(const Slice& s, float4 (&pf)[kPf]) {
#pragma unroll
    for (int i = 0; i < kPf; ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < s.ng) pf[i] = __ldg(s.g + e);
        else if (e < s.ng + s.nw) pf[i] = __ldg(s.w + (e - s.ng));
    }
}

__device__ __forceinline__ void commit(const Slice& s, const float4 (&pf)[kPf], float* buf) {
    float4* b4 = reinterpret_cast<float4*>(buf);
#pragma unroll
    for (int i = 0; i < kPf; ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < s.ng + s.nw) b4[e] = pf[i];
    }
}

__global__ void __cluster_dims__(kS, 1, 1) __launch_bounds__(kThreads, 1)
    cbn_f32_kernel(CbnF32 net, PointSrc src, int64_t m, Calib calib, Map map, Epilogue epi) {
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int64_t cid = blockIdx.x / kS;
    const int64_t ncl = gridDim.x / kS;
    const int C = net.C, K = net.K, nb = net.nb;
    const int Kc = K / kS, K2c = 2 * Kc;
    const int slice = C * K2c + K * Kc;           // floats of one weight buffer
    extern __shared__ float4 smem4[];
    float* cS = reinterpret_cast<float*>(smem4);   // [C][kLd] features
    float* aS = cS + C * kLd;                      // [2][K][kLd] a of all channels
    float* nS = aS + 2 * K * kLd;                  // [Kc][kLd] normalized input, own channels
    float* gS = nS + Kc * kLd;                     // [2Kc][kLd] gamma | beta, own channels
    float* wS = gS + K2c * kLd;                    // [2][slice] weight double buffer
    float* tS = wS + 2 * slice;                    // [kP] SoftZ weight of the upper index
    int* iS = reinterpret_cast<int*>(tS + kP);     // [kP] SoftZ lower index
    const Map none{nullptr, 0, 0, 0, 0};

    if (src.count) m = min(m, (int64_t)*src.count);
    const int64_t ntiles = (m + kP - 1) / kP;
    float4 pf[kPf];
    {
        const Slice s0 = slice_of(net, 0, r);
        prefetch(s0, pf);
        commit(s0, pf, wS);
    }
    __syncthreads();
    const int qpr = C / 4 / kS;   // feature quads each CTA gathers per point
    int64_t q = 0;                // blocks done by this cluster (buffer parity)
    for (int64_t tile = cid; tile < ntiles; tile += ncl) {
        const int64_t p0 = tile * kP;
        const int np = (int)(m - p0 < (int64_t)kP ? m - p0 : (int64_t)kP);
        // features: CTA r gathers quads [r qpr, (r + 1) qpr) of every point
        // and stores them into every CTA's copy; every CTA takes the depth
        for (int e = threadIdx.x; e < kP * qpr; e += kThreads) {
            const int p = e % kP;
            const int qd = r * qpr + e / kP;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < np) v = gather_quad(src, p0 + p, calib, map, none, 4 * qd);
            float* dst = cS + 4 * qd * kLd + p;
#pragma unroll
            for (int d = 0; d < kS; ++d) {
                float* rd = cl.map_shared_rank(dst, (unsigned)d);
                rd[0] = v.x;
                rd[kLd] = v.y;
                rd[2 * kLd] = v.z;
                rd[3 * kLd] = v.w;
            }
        }
        if (threadIdx.x < kP) {
            const int p = threadIdx.x;
            float z = 0.f;
            if (p < np) z = gather_quad(src, p0 + p, calib, map, none, C).x;
            int i;
            float t;
            soft_z(z, net.n_z, i, t);
            iS[p] = i;
            tS[p] = t;
        }
        cl.sync();
        // normalized input of block 0 for the own channels
        for (int e = threadIdx.x; e < Kc * kP; e += kThreads) {
            const int j = e / kP;
            const int p = e % kP;
            const int k = r * Kc + j;
            const float lo = __ldg(net.WzT + (int64_t)iS[p] * K + k);
            const float hi = __ldg(net.WzT + (int64_t)(iS[p] + 1) * K + k);
            nS[j * kLd + p] = fmaf(tS[p], hi, fmaf(1.0f - tS[p], lo, __ldg(net.bz + k)));
        }
        for (int blk = 0; blk < nb; ++blk, ++q) {
            const float* wb = wS + (q & 1) * slice;
            // the next block's weight slice travels while this block computes
            const bool more = blk + 1 < nb || tile + ncl < ntiles;
            const Slice sn = slice_of(net, blk + 1 < nb ? blk + 1 : 0, r);
            if (more) prefetch(sn, pf);
            __syncthreads();   // nS, the weights of this block
            tile_gemm(wb, net.g0S + ((int64_t)blk * kS + r) * K2c, C, K2c, cS, gS);
            __syncthreads();
            float* aq = aS + (q & 1) * K * kLd;
            for (int e = threadIdx.x; e < Kc * kP; e += kThreads) {
                const int j = e / kP;
                const int p = e % kP;
                const float a = fmaxf(fmaf(gS[j * kLd + p], nS[j * kLd + p], gS[(Kc + j) * kLd + p]),
                                      0.0f);
                float* dst = aq + (r * Kc + j) * kLd + p;
#pragma unroll
                for (int d = 0; d < kS; ++d) *cl.map_shared_rank(dst, (unsigned)d) = a;
            }
            cl.sync();
            if (blk + 1 < nb) {
                tile_gemm(wb + C * K2c, net.blS + ((int64_t)blk * kS + r) * Kc, K, Kc, aq, nS);
            } else {
                // logits: CTA r takes points r, r + kS, ...
                const int lane = threadIdx.x & 31;
                for (int p = r + kS * (threadIdx.x >> 5); p < np; p += kS * (kThreads / 32)) {
                    float acc = 0.f;
                    for (int k = lane; k < K; k += 32) acc = fmaf(__ldg(net.wlast + k), aq[k * kLd + p], acc);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) {
                        const float t[4] = {acc, 0.f, 0.f, 0.f};
                        last_epilogue(epi, p0 + p, 1, t, net.blast);
                    }
                }
            }
            __syncthreads();   // every read of this block's weights is done
            if (more) commit(sn, pf, wS + ((q + 1) & 1) * slice);
        }
    }
}

size_t smem_bytes(const CbnF32& net) {
    const int Kc = net.K / kS;
    const size_t slice = (size_t)net.C * 2 * Kc + (size_t)net.K * Kc;
    return ((size_t)(net.C + 2 * net.K + 3 * Kc) * kLd + 2 * slice + 2 * kP) * 4;
}

int max_clusters(const CbnF32& net) {
    static int cached = -1;
    static size_t cached_smem = 0;
    const size_t smem = smem_bytes(net);
    if (cached >= 0 && cached_smem == smem) return cached;
    if (cudaFuncSetAttribute(cbn_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, cbn_f32_kernel, &cfg) != cudaSuccess) n = 0;
    cached_smem = smem;
    return cached = n;
}

}  // namespace

bool cbn_f32_ok(const CbnF32& net) {
    if (net.C < 4 * kS || net.C % (4 * kS) != 0 || net.K % (4 * kS) != 0 || net.K < 4 * kS ||
        net.n_z < 2 || net.nb < 1)
        return false;
    const int Kc = net.K / kS;
    const int slice = net.C * 2 * Kc + net.K * Kc;
    return slice <= 4 * kPf * kThreads && smem_bytes(net) <= 227 * 1024;
}

cudaError_t cbn_f32_prepare(const CbnF32& net) {
    if (!cbn_f32_ok(net)) return cudaErrorInvalidValue;
    return max_clusters(net) > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t launch_cbn_f32(const CbnF32& net, const PointSrc& src, int64_t m, const Calib& calib,
                           const Map& map, const Epilogue& epi, cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    if (!cbn_f32_ok(net)) return cudaErrorInvalidValue;
    const int ncl = max_clusters(net);
    if (ncl <= 0) return cudaErrorInvalidConfiguration;
    const int64_t tiles = (m + kP - 1) / kP;
    const int64_t grid_cl = src.count ? ncl : std::min<int64_t>(tiles, ncl);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(grid_cl * kS));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem_bytes(net);
    cfg.stream = stream;
    return cudaLaunchKernelEx(&cfg, cbn_f32_kernel, net, src, m, calib, map, epi);
}

}  // namespace pifu
