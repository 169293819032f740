// Training kernels of the distilled occupancy surrogate (FP32): the forward
// pass of an MLP of the concatenation family without skips, the mean binary
// cross-entropy of its logit against the full network's occupancy (the loss
// the paper trains f_O with, Sec. 3.1), back-propagation, and Adam (the
// optimiser of the paper's texture network, Appendix).
//
// All matrix products are one strided GEMM, C (+)= sum_k A(m, k) B(k, n),
// with arbitrary element strides for A and B, so that forward (X W^T),
// weight gradients (dZ^T H, a reduction over the batch) and activation
// gradients (dZ W) share a kernel.  A 64-thread CTA computes a 32 x 32 tile
// over one slice of the reduction; several slices accumulate with atomicAdd
// into a zeroed C.  The sizes are small (batch 4096, widths <= 264), so the
// kernels are latency- rather than throughput-bound; training is offline.
#include "pifu_internal.h"

namespace pifu {
namespace {

constexpr int GT = 32;   // tile edge
constexpr int GK = 8;    // reduction step

__global__ void __launch_bounds__(64) gemm_strided_kernel(
    int M, int N, int K, const float* __restrict__ A, int64_t a_m, int64_t a_k,
    const float* __restrict__ B, int64_t b_k, int64_t b_n, float* __restrict__ C, int64_t c_m,
    int k_per_slice, int accumulate) {
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * GT;
    const int n0 = blockIdx.x * GT;
    const int k0 = blockIdx.z * k_per_slice;
    const int k1 = min(K, k0 + k_per_slice);
    const int ty = tid >> 3, tx = tid & 7;
    float acc[4][4] = {};
    for (int kb = k0; kb < k1; kb += GK) {
        for (int e = tid; e < GK * GT; e += 64) {
            const int kk = e / GT, r = e % GT;
            const int k = kb + kk;
            As[kk][r] = (m0 + r < M && k < k1) ? A[(int64_t)(m0 + r) * a_m + (int64_t)k * a_k] : 0.f;
            Bs[kk][r] = (n0 + r < N && k < k1) ? B[(int64_t)k * b_k + (int64_t)(n0 + r) * b_n] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float* c = C + (int64_t)m * c_m + n;
            if (accumulate) atomicAdd(c, acc[i][j]);
            else *c = acc[i][j];
        }
    }
}

// H[b][n] = lrelu(Z[b][n] + bias[n]) in place (ld = row stride).
__global__ void bias_lrelu_kernel(int M, int N, float* __restrict__ Z, int ld,
                                  const float* __restrict__ bias, float slope) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int m = (int)(i / N), n = (int)(i % N);
    float z = Z[(int64_t)m * ld + n] + bias[n];
    Z[(int64_t)m * ld + n] = z >= 0.f ? z : slope * z;
}

// g[b] = (sigmoid(t_b + bias) - y_b) / B and loss += softplus(t) - y t
// (per_loss[b] = that sample's loss, if set).
__global__ void bce_grad_kernel(int B, const float* __restrict__ logit, const float* __restrict__ bias,
                                const float* __restrict__ y, float* __restrict__ g,
                                double* __restrict__ loss, float* __restrict__ per_loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        const float t = logit[b] + bias[0];
        const float s = 1.0f / (1.0f + expf(-t));
        g[b] = (s - y[b]) / (float)B;
        // softplus(t) - y t, stable for both signs of t
        const double td = (double)t;
        const double sp = td > 0 ? td + log1p(exp(-td)) : log1p(exp(td));
        l = sp - (double)y[b] * td;
        if (per_loss) per_loss[b] = (float)l;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l / (double)B);
}

// dZ = dH * g'(Z) with g' from the sign of the stored activation H (the
// leaky-ReLU keeps the sign of its input).
__global__ void lrelu_backward_kernel(int64_t n, float* __restrict__ dH,
                                      const float* __restrict__ H, float slope) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (H[i] < 0.f) dH[i] *= slope;
}

__global__ void adam_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- point OHEM (Sec. 3.3, Eq. 6) ----------------------------------------------
//
// Sampling probability proportional to w = 1 / (exp(-L_BCE / alpha) + beta):
// an inclusive FP64 prefix sum of w (blocks of kScanPer elements, then the
// block totals, then their offsets), one splitmix64 uniform per draw from the
// counter seed ^ (step << 32) ^ draw, and an upper-bound search of u * total.

constexpr int kScanThreads = 256;
constexpr int kScanEach = 16;
constexpr int kScanPer = kScanThreads * kScanEach;

__device__ __forceinline__ double warp_incl_scan(double v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Inclusive scan of vals[0 .. n) in one block of kScanThreads threads, each
// owning `each` consecutive values; returns the block total.
template <typename Load, typename Store>
__device__ __forceinline__ double block_scan(int64_t n, int each, Load&& load, Store&& store) {
    __shared__ double warp_tot[kScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t i0 = (int64_t)t * each;
    double run = 0.0;
    for (int k = 0; k < each; ++k)
        if (i0 + k < n) run += load(i0 + k);
    const double incl = warp_incl_scan(run, lane);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    double woff = 0.0, total = 0.0;
    for (int q = 0; q < kScanThreads / 32; ++q) {
        if (q < warp) woff += warp_tot[q];
        total += warp_tot[q];
    }
    double acc = woff + incl - run;   // exclusive prefix of this thread
    for (int k = 0; k < each; ++k)
        if (i0 + k < n) {
            const double v = load(i0 + k);
            acc += v;
            store(i0 + k, acc, v);       // inclusive prefix and the element
        }
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(const float* __restrict__ w,
                                                                   int64_t m, double* __restrict__ cdf,
                                                                   double* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanPer;
    const int64_t n = min((int64_t)kScanPer, m - base);
    const double tot = block_scan(
        n, kScanEach, [&](int64_t i) { return (double)w[base + i]; },
        [&](int64_t i, double incl, double) { cdf[base + i] = incl; });
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive offsets of the block totals, in place (one block).
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(double* __restrict__ sums,
                                                                 int64_t nb) {
    const int each = (int)((nb + kScanThreads - 1) / kScanThreads);
    block_scan(
        nb, each, [&](int64_t i) { return sums[i]; },
        [&](int64_t i, double incl, double v) { sums[i] = incl - v; });   // exclusive
}

__global__ void add_offsets_kernel(double* __restrict__ cdf, int64_t m,
                                   const double* __restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) cdf[i] += offs[i / kScanPer];
}

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void ohem_sample_kernel(const double* __restrict__ cdf, int64_t m, uint64_t seed,
                                   uint32_t step, int B, int* __restrict__ idx) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint64_t z = splitmix64_out(seed ^ ((uint64_t)step << 32) ^ (uint64_t)b);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) * cdf[m - 1];
    int64_t lo = 0, hi = m;   // first i with cdf[i] > u
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    idx[b] = (int)min(lo, m - 1);
}

// xb[b] = x[idx[b]] (rows of ld floats), yb[b] = y[idx[b]].
__global__ void gather_rows_kernel(const float* __restrict__ x, const float* __restrict__ y, int ld,
                                   const int* __restrict__ idx, int B, float* __restrict__ xb,
                                   float* __restrict__ yb) {
    const int nq = ld >> 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * nq) return;
    const int b = (int)(t / nq);
    const int q = (int)(t - (int64_t)b * nq);
    const int64_t r = idx[b];
    reinterpret_cast<float4*>(xb + (int64_t)b * ld)[q] =
        reinterpret_cast<const float4*>(x + r * ld)[q];
    if (q == 0) yb[b] = y[r];
}

// w[idx[b]] = 1 / (exp(-L_b / alpha) + beta), kept in [1e-30, 1e30].
__global__ void ohem_update_kernel(float* __restrict__ w, const int* __restrict__ idx,
                                   const float* __restrict__ loss, int B, float alpha, float beta) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float v = 1.0f / (expf(-loss[b] / alpha) + beta);
    w[idx[b]] = fminf(fmaxf(v, 1e-30f), 1e30f);
}

__global__ void fill_kernel(int64_t n, float* __restrict__ p, float value) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = value;
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_gemm_strided(int M, int N, int K, const float* A, int64_t a_m, int64_t a_k,
                                const float* B, int64_t b_k, int64_t b_n, float* C, int64_t c_m,
                                int k_slices, int accumulate, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (k_slices < 1) k_slices = 1;
    int per = (K + k_slices - 1) / k_slices;
    per = (per + GK - 1) / GK * GK;
    k_slices = (K + per - 1) / per;
    if (k_slices > 1) accumulate = 1;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, k_slices);
    gemm_strided_kernel<<<grid, 64, 0, s>>>(M, N, K, A, a_m, a_k, B, b_k, b_n, C, c_m, per,
                                             accumulate);
    return cudaGetLastError();
}

cudaError_t launch_bias_lrelu(int M, int N, float* Z, int ld, const float* bias, float slope,
                              cudaStream_t s) {
    bias_lrelu_kernel<<<nblk((int64_t)M * N), 256, 0, s>>>(M, N, Z, ld, bias, slope);
    return cudaGetLastError();
}

cudaError_t launch_bce_grad(int B, const float* logit, const float* bias, const float* y, float* g,
                            double* loss, cudaStream_t s, float* per_loss) {
    bce_grad_kernel<<<nblk(B), 256, 0, s>>>(B, logit, bias, y, g, loss, per_loss);
    return cudaGetLastError();
}

cudaError_t launch_lrelu_backward(int64_t n, float* dH, const float* H, float slope,
                                  cudaStream_t s) {
    lrelu_backward_kernel<<<nblk(n), 256, 0, s>>>(n, dH, H, slope);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float* w, const float* g, float* m, float* v, float lr, int t,
                        cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<nblk(n), 256, 0, s>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

int64_t ohem_scan_blocks(int64_t m) { return (m + kScanPer - 1) / kScanPer; }

cudaError_t launch_ohem_sample(const float* w, int64_t m, double* cdf, double* sums,
                               uint64_t seed, uint32_t step, int B, int* idx, cudaStream_t s) {
    const int64_t nb = ohem_scan_blocks(m);
    scan_blocks_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(w, m, cdf, sums);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, nb);
    add_offsets_kernel<<<nblk(m), 256, 0, s>>>(cdf, m, sums);
    ohem_sample_kernel<<<nblk(B), 256, 0, s>>>(cdf, m, seed, step, B, idx);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* x, const float* y, int ld, const int* idx, int B,
                               float* xb, float* yb, cudaStream_t s) {
    gather_rows_kernel<<<nblk((int64_t)B * (ld / 4)), 256, 0, s>>>(x, y, ld, idx, B, xb, yb);
    return cudaGetLastError();
}

cudaError_t launch_ohem_update(float* w, const int* idx, const float* loss, int B, float alpha,
                               float beta, cudaStream_t s) {
    ohem_update_kernel<<<nblk(B), 256, 0, s>>>(w, idx, loss, B, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_fill(int64_t n, float* p, float value, cudaStream_t s) {
    fill_kernel<<<nblk(n), 256, 0, s>>>(n, p, value);
    return cudaGetLastError();
}

}  // namespace pifu
