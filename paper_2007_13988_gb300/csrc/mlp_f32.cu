// Plain FP32 form of the concatenation MLPs f_O and f_T (Sec. 3.1; Appendix,
// "Pixel-aligned 3D Lifting", the "MLP" variant; the colour MLP's 1024-512-
// 256-128-3 widths with skip connections, leaky-ReLU and tanh).
//
// Hidden layers run as a register-blocked SIMT SGEMM with the bias and the
// leaky-ReLU fused into the epilogue.  A skip layer's input [h_{l-1}, x] is
// never materialised: the K loop walks two segments, first h_{l-1}, then x,
// against the matching column ranges of W_l.  The last layer (1 or 3
// outputs) is a warp-per-point dot product fused with the activation and
// with what the caller needs done with the result (store, scatter into a
// localization level with conflict detection, or write pixels).
//
// This is the precision reference on the GPU (FFMA, float32 accumulation);
// the roofline that bounds it is the FP32 SIMT FMA rate.
#include "pifu_internal.h"
#include "epilogue.cuh"

namespace pifu {
namespace {

constexpr int BM = 128, BN = 128, BK = 8;
constexpr int kSmallM = kSplitMaxM;   // batches up to this many points use split-K

__global__ void __launch_bounds__(256) sgemm_bias_lrelu_kernel(
    int M, int N, const float* __restrict__ A1, int lda1, int K1, const float* __restrict__ A2,
    int lda2, int K2, const float* __restrict__ W, int ldw, const float* __restrict__ bias,
    float slope, float* __restrict__ Out, int ldo) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int bm = blockIdx.y * BM;
    const int bn = blockIdx.x * BN;
    const int nk1 = K1 / BK;
    const int nk = nk1 + K2 / BK;

    // global -> shared mapping: 128 rows x 8 k per tile, one float4 per thread
    const int lrow = tid >> 1;
    const int lk = (tid & 1) * 4;
    const int gm = bm + lrow;
    const int gn = bn + lrow;
    const bool m_ok = gm < M;
    const bool n_ok = gn < N;

    float4 ra, rb;
    auto load = [&](int kt) {
        const float* src;
        int kk;
        int lda;
        if (kt < nk1) {
            src = A1; lda = lda1; kk = kt * BK;
        } else {
            src = A2; lda = lda2; kk = (kt - nk1) * BK;
        }
        ra = m_ok ? __ldg(reinterpret_cast<const float4*>(src + (int64_t)gm * lda + kk + lk))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
        rb = n_ok ? __ldg(reinterpret_cast<const float4*>(W + (int64_t)gn * ldw + kt * BK + lk))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto store = [&](int buf) {
        As[buf][lk + 0][lrow] = ra.x; As[buf][lk + 1][lrow] = ra.y;
        As[buf][lk + 2][lrow] = ra.z; As[buf][lk + 3][lrow] = ra.w;
        Bs[buf][lk + 0][lrow] = rb.x; Bs[buf][lk + 1][lrow] = rb.y;
        Bs[buf][lk + 2][lrow] = rb.z; Bs[buf][lk + 3][lrow] = rb.w;
    };

    // compute mapping: 16 x 16 threads, each 8 x 8 outputs in two 4-wide halves
    const int ty = tid >> 4;
    const int tx = tid & 15;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    if (nk > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load(kt + 1);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) store(cur ^ 1);
        __syncthreads();
    }

    // epilogue: bias + leaky-ReLU, float4 stores
#pragma unroll
    for (int hi = 0; hi < 2; ++hi) {
        const int col = bn + hi * 64 + tx * 4;
        if (col >= N) continue;
        const float4 bb = *reinterpret_cast<const float4*>(bias + col);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = bm + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (row >= M) continue;
            float4 o;
            o.x = acc[i][hi * 4 + 0] + bb.x;
            o.y = acc[i][hi * 4 + 1] + bb.y;
            o.z = acc[i][hi * 4 + 2] + bb.z;
            o.w = acc[i][hi * 4 + 3] + bb.w;
            o.x = o.x >= 0.f ? o.x : slope * o.x;
            o.y = o.y >= 0.f ? o.y : slope * o.y;
            o.z = o.z >= 0.f ? o.z : slope * o.z;
            o.w = o.w >= 0.f ? o.w : slope * o.w;
            *reinterpret_cast<float4*>(Out + (int64_t)row * ldo + col) = o;
        }
    }
}

// Small batches (a few points to a few thousand): the 128 x 128 tile above
// leaves most SMs idle, and a CTA's K loop (up to 161 steps of 8) is a
// chain of dependent global loads.  Here a 64-thread CTA computes a 32 x 32
// tile (4 x 4 per thread) over one slice of K (blockIdx.z of gridDim.z) and
// writes its partial sums to its own slice of `part`; a second kernel adds
// the slices in a fixed order (deterministic, no atomics) and applies bias
// and leaky-ReLU.  A batch of M points spreads over (M/32) (N/32) S CTAs.
constexpr int SBM = 32, SBN = 32, SBK = 8;
constexpr int kSplitSteps = 6;    // target K steps per slice (latency-bound: keep short)

__global__ void __launch_bounds__(64) sgemm_small_kernel(
    int M, int N, const float* __restrict__ A1, int lda1, int K1, const float* __restrict__ A2,
    int lda2, int K2, const float* __restrict__ W, int ldw, float* __restrict__ part,
    int steps_per_slice, int S, const unsigned int* __restrict__ m_dev) {
    // M is the capacity (and the slice stride of `part`); a device count
    // narrows the rows actually computed.
    const int Mc = M;
    if (m_dev) M = min(M, (int)*m_dev);
    __shared__ __align__(16) float As[2][SBK][SBM];
    __shared__ __align__(16) float Bs[2][SBK][SBN];
    const int tid = threadIdx.x;
    const int nk1 = K1 / SBK;
    const int tiles_n = (N + SBN - 1) / SBN;
    const int tiles_m = (M + SBM - 1) / SBM;
    const int64_t items = (int64_t)tiles_n * tiles_m * S;
    // one float4 of A and one of W per thread per K step: row tid/2, k (tid&1)*4
    const int lrow = tid >> 1;
    const int lk = (tid & 1) * 4;
    const int ty = tid >> 3;   // rows ty*4 .. +3
    const int tx = tid & 7;    // cols tx*4 .. +3
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int z = (int)(item % S);
        const int64_t tile = item / S;
        const int bn = (int)(tile % tiles_n) * SBN;
        const int bm = (int)(tile / tiles_n) * SBM;
        const int kt0 = z * steps_per_slice;
        const int nk = min(nk1 + K2 / SBK, kt0 + steps_per_slice);
        const int gm = bm + lrow;
        const int gn = bn + lrow;
        float4 ra, rb;
        auto load = [&](int kt) {
            const float* src;
            int kk, lda;
            if (kt < nk1) {
                src = A1; lda = lda1; kk = kt * SBK;
            } else {
                src = A2; lda = lda2; kk = (kt - nk1) * SBK;
            }
            ra = gm < M ? __ldg(reinterpret_cast<const float4*>(src + (int64_t)gm * lda + kk + lk))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
            rb = gn < N ? __ldg(reinterpret_cast<const float4*>(W + (int64_t)gn * ldw + kt * SBK + lk))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto store = [&](int buf) {
            As[buf][lk + 0][lrow] = ra.x; As[buf][lk + 1][lrow] = ra.y;
            As[buf][lk + 2][lrow] = ra.z; As[buf][lk + 3][lrow] = ra.w;
            Bs[buf][lk + 0][lrow] = rb.x; Bs[buf][lk + 1][lrow] = rb.y;
            Bs[buf][lk + 2][lrow] = rb.z; Bs[buf][lk + 3][lrow] = rb.w;
        };
        float acc[4][4] = {};
        if (kt0 < nk) {
            load(kt0);
            store(0);
        }
        __syncthreads();
        for (int kt = kt0; kt < nk; ++kt) {
            const int cur = (kt - kt0) & 1;
            if (kt + 1 < nk) load(kt + 1);
#pragma unroll
            for (int k = 0; k < SBK; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
                const float4 b = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            if (kt + 1 < nk) store(cur ^ 1);
            __syncthreads();
        }
        const int col = bn + tx * 4;
        if (col < N) {
            float* slice = part + (int64_t)z * Mc * N;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = bm + ty * 4 + i;
                if (row >= M) continue;
                *reinterpret_cast<float4*>(slice + (int64_t)row * N + col) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        }
    }
}

// out[m][n] = lrelu(bias[n] + sum over the S slices of part[s][m][n]), four
// columns per thread, slices added in order.  M is the slice stride; a
// device count narrows the rows.
__global__ void __launch_bounds__(256) splitk_finish_kernel(int M, int N, int S,
                                                            const float* __restrict__ part,
                                                            const float* __restrict__ bias,
                                                            float slope, float* __restrict__ Out,
                                                            int ldo,
                                                            const unsigned int* __restrict__ m_dev) {
    const int Mc = M;
    if (m_dev) M = min(M, (int)*m_dev);
    const int nq = N / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)M * nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(q / nq);
        const int col = (int)(q - (int64_t)row * nq) * 4;
        float4 o = *reinterpret_cast<const float4*>(bias + col);
        for (int z = 0; z < S; ++z) {
            const float4 p =
                __ldg(reinterpret_cast<const float4*>(part + ((int64_t)z * Mc + row) * N + col));
            o.x += p.x;
            o.y += p.y;
            o.z += p.z;
            o.w += p.w;
        }
        o.x = o.x >= 0.f ? o.x : slope * o.x;
        o.y = o.y >= 0.f ? o.y : slope * o.y;
        o.z = o.z >= 0.f ? o.z : slope * o.z;
        o.w = o.w >= 0.f ? o.w : slope * o.w;
        *reinterpret_cast<float4*>(Out + (int64_t)row * ldo + col) = o;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// One warp per point (grid-stride over points; a device count narrows M).
template <typename InT>
__global__ void __launch_bounds__(256) last_layer_kernel(
    int64_t p0, int64_t M, int n_out, const InT* __restrict__ A1, int lda1, int K1,
    const InT* __restrict__ A2, int lda2, int K2, const float* __restrict__ W, int ldw,
    const float* __restrict__ bias, Epilogue epi, const unsigned int* __restrict__ m_dev) {
    const int lane = threadIdx.x & 31;
    if (m_dev) M = min(M, (int64_t)*m_dev);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t lp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; lp < M; lp += nwarps) {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        const InT* a1 = A1 + lp * lda1;
        const InT* a2 = A2 + lp * lda2;
        for (int k = lane; k < K1 + K2; k += 32) {
            const float a = (k < K1) ? to_f32(a1[k]) : to_f32(a2[k - K1]);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < n_out) t[j] = fmaf(a, W[(int64_t)j * ldw + k], t[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) t[j] = warp_sum(t[j]);
        if (lane == 0) last_epilogue(epi, p0 + lp, n_out, t, bias);
    }
}

// *out = max(*out, max |p[i]|) as float bits (non-negative floats order like
// their bit patterns).
__global__ void amax_kernel(const float* __restrict__ p, int64_t n, unsigned int* out) {
    float v = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v = fmaxf(v, fabsf(p[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(v));
}

inline unsigned fixed_or_exact(const unsigned int* m_dev, int64_t exact_blocks) {
    return (unsigned)(m_dev ? (exact_blocks < 152 * 16 ? exact_blocks : 152 * 16) : exact_blocks);
}

}  // namespace

int splitk_slices(int K1, int K2) {
    const int steps = (K1 + K2) / SBK;
    return steps <= 0 ? 1 : (steps + kSplitSteps - 1) / kSplitSteps;
}

cudaError_t launch_sgemm_bias_lrelu(int M, int N, const float* A1, int lda1, int K1,
                                    const float* A2, int lda2, int K2, const float* W, int ldw,
                                    const float* bias, float slope, float* Out, int ldo,
                                    cudaStream_t stream, float* part, const unsigned int* m_dev) {
    if (M <= 0) return cudaSuccess;
    if ((M <= kSmallM || m_dev) && part) {
        const int steps = (K1 + K2) / SBK;
        const int S = splitk_slices(K1, K2);
        const int per = (steps + S - 1) / S;
        const int64_t items = (int64_t)((N + SBN - 1) / SBN) * ((M + SBM - 1) / SBM) * S;
        sgemm_small_kernel<<<fixed_or_exact(m_dev, items), 64, 0, stream>>>(
            M, N, A1, lda1, K1, A2, lda2, K2, W, ldw, part, per, S, m_dev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t nthreads = (int64_t)M * (N / 4);
        splitk_finish_kernel<<<fixed_or_exact(m_dev, (nthreads + 255) / 256), 256, 0, stream>>>(
            M, N, S, part, bias, slope, Out, ldo, m_dev);
        return cudaGetLastError();
    }
    if (m_dev) return cudaErrorInvalidValue;   // the big-tile kernel needs a host-known M
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    sgemm_bias_lrelu_kernel<<<grid, 256, 0, stream>>>(M, N, A1, lda1, K1, A2, lda2, K2, W, ldw,
                                                      bias, slope, Out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_last_layer(int64_t p0, int64_t M, int n_out, const float* A1, int lda1, int K1,
                              const float* A2, int lda2, int K2, const float* W, int ldw,
                              const float* bias, const Epilogue& epi, cudaStream_t stream,
                              const unsigned int* m_dev) {
    if (M <= 0) return cudaSuccess;
    const int64_t blocks = (M * 32 + 255) / 256;
    last_layer_kernel<float><<<fixed_or_exact(m_dev, blocks), 256, 0, stream>>>(
        p0, M, n_out, A1, lda1, K1, A2, lda2, K2, W, ldw, bias, epi, m_dev);
    return cudaGetLastError();
}

cudaError_t launch_last_layer_bf16(int64_t p0, int64_t M, int n_out, const __nv_bfloat16* A1,
                                   int lda1, int K1, const __nv_bfloat16* A2, int lda2, int K2,
                                   const float* W, int ldw, const float* bias, const Epilogue& epi,
                                   cudaStream_t stream, const unsigned int* m_dev) {
    if (M <= 0) return cudaSuccess;
    const int64_t blocks = (M * 32 + 255) / 256;
    last_layer_kernel<__nv_bfloat16><<<fixed_or_exact(m_dev, blocks), 256, 0, stream>>>(
        p0, M, n_out, A1, lda1, K1, A2, lda2, K2, W, ldw, bias, epi, m_dev);
    return cudaGetLastError();
}

cudaError_t launch_amax(const float* p, int64_t n, unsigned int* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    amax_kernel<<<(unsigned)blocks, 256, 0, stream>>>(p, n, out);
    return cudaGetLastError();
}

}  // namespace pifu
