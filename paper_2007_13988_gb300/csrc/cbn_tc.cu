// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) form of the CBN +
// SoftZ occupancy network (Appendix, Eq. 7 and Eq. 8), the whole network in
// one persistent kernel per 128-point tile:
//
//   block i:  [gamma | beta] = c Gt_i^T            (M 128, N 2K, K C)  MMA
//             a = ReLU((gamma + gg) n + beta + gb)                    epilogue
//             n' = a W'_i^T                         (M 128, N K, K K)  MMA
//   last:     logit = wlast . a + blast                               epilogue
//
// with n the normalized block input (the running statistics are folded into
// W'_i on the host) and n_0 = (1 - t) Wz'[:, i] + t Wz'[:, i + 1] + bz' from
// the point's SoftZ pair (i, t) (Eq. 7 has two non-zero weights).  82% of the
// arithmetic is the gamma/beta contraction over the feature, which one MMA
// per block covers for all of gamma and beta.
//
// Shared memory: the tile's features c (BF16, C/64 K-blocks of 128 x 64,
// loaded once per tile by TMA and read by every block's MMA), the ReLU output
// a written by the epilogue in the same 128-byte-swizzled K-major layout (the
// A operand of the linear layer), and a ring of weight tiles that the TMA
// producer fills ahead of the MMAs (weights do not depend on the tile, so
// their loads overlap the epilogues).  Tensor memory: [0, 2K) the
// gamma/beta accumulator, [2K, 3K) the linear layer's.
//
// Warps: 0 lane 0 TMA producer; 1 TMEM allocation and (lane 0) MMA issue;
// 2 .. 9 epilogue, two per TMEM lane quadrant, each on half of the K
// channels.  A block's epilogue waits for its gamma/beta (and, after block
// 0, the previous linear layer), writes a, and signals; the MMA warp then
// issues the linear layer and the next block's gamma/beta, which overwrite
// accumulators the epilogue has drained.  The last block's two half sums of
// each logit meet through shared memory under an mbarrier.  Every wait is
// bounded; a wait that gives up sets *err and the role stops; before
// returning, the producer waits (bounded) for its own copies in flight and
// the CTA frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "epilogue.cuh"
#include "gather.cuh"
#include "pifu_internal.h"
#include "sm100.cuh"

namespace pifu {
namespace {

using namespace sm100;

constexpr int TM = 128;                // points per tile (MMA M)
constexpr int TK = 64;                 // BF16 elements per 128-byte K-block
constexpr int kStages = 3;
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t KB_BYTES = TM * TK * 2;   // one 128 x 64 BF16 K-block

struct Layout {
    uint32_t a_off, act_off, ring_off, stage_bytes, bar_off, g0_off, bl_off, wl_off, xch_off,
        total;
};

__host__ __device__ inline Layout layout_of(int C, int K, int nb) {
    Layout L{};
    const int nkc = (C + TK - 1) / TK;
    L.a_off = 0;
    L.act_off = L.a_off + nkc * KB_BYTES;
    L.ring_off = L.act_off + (K / TK) * KB_BYTES;
    L.stage_bytes = 2u * K * 128u;
    L.bar_off = L.ring_off + kStages * L.stage_bytes;
    L.g0_off = L.bar_off + 256;
    L.bl_off = L.g0_off + nb * 2 * K * 4;
    L.wl_off = L.bl_off + (nb > 1 ? (nb - 1) : 1) * K * 4;
    L.xch_off = L.wl_off + K * 4;
    L.total = L.xch_off + TM * 4 + 1024;   // + alignment slack of the dynamic base
    return L;
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// 32 consecutive TMEM columns of the warp's lanes into r (two x16 loads).
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t* r) {
    tmem_ld16(taddr, *reinterpret_cast<uint32_t(*)[16]>(r));
    tmem_ld16(taddr + 16, *reinterpret_cast<uint32_t(*)[16]>(r + 16));
}

template <int K>
__global__ void __launch_bounds__(kThreads, 1) cbn_tc_kernel(
    const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmG,
    const __grid_constant__ CUtensorMap tmW, CbnTcArgs p) {
    constexpr int K2 = 2 * K;
    constexpr uint32_t TMEM_COLS = K == 128 ? 512 : 256;
    constexpr uint32_t G_BYTES = K2 * 128;   // one K-block of [gamma; beta] rows
    constexpr uint32_t W_BYTES = K * 128;    // one K-block of the linear layer
    constexpr int HALF = K / 2;              // channels per epilogue warp
    const int C = p.C, nb = p.nb;
    const int nkc = (C + TK - 1) / TK;
    const Layout L = layout_of(C, K, nb);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sA = base + L.a_off;
    uint8_t* sAct = base + L.act_off;
    uint8_t* sRing = base + L.ring_off;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + L.bar_off);
    uint64_t* empty = full + kStages;
    uint64_t* a_full = empty + kStages;    // tile features loaded
    uint64_t* a_empty = a_full + 1;        // last gamma/beta MMA of the tile done
    uint64_t* g_full = a_empty + 1;        // gamma/beta accumulator ready
    uint64_t* h_full = g_full + 1;         // linear-layer accumulator ready
    uint64_t* epi_done = h_full + 1;       // a written, accumulators drained (8 warps)
    uint64_t* xch_full = epi_done + 1;     // half sums of the logits published (4 warps)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(xch_full + 1);
    float* sg0 = reinterpret_cast<float*>(base + L.g0_off);
    float* sbl = reinterpret_cast<float*>(base + L.bl_off);
    float* swl = reinterpret_cast<float*>(base + L.wl_off);
    float* sxch = reinterpret_cast<float*>(base + L.xch_off);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        mbar_init(g_full, 1);
        mbar_init(h_full, 1);
        mbar_init(epi_done, kEpiWarps);
        mbar_init(xch_full, kEpiWarps / 2);
        fence_mbar_init();
        prefetch_tmap(&tmX);
        prefetch_tmap(&tmG);
        if (nb > 1) prefetch_tmap(&tmW);
    }
    for (int c = threadIdx.x; c < nb * K2; c += blockDim.x) sg0[c] = p.g0[c];
    for (int c = threadIdx.x; c < (nb - 1) * K; c += blockDim.x) sbl[c] = p.bl[c];
    for (int c = threadIdx.x; c < K; c += blockDim.x) swl[c] = p.wlast[c];
    if (warp == 1) tmem_alloc(tslot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tm_g = tmem;
    const uint32_t tm_h = tmem + K2;
    const int M = p.m_dev ? min(p.M, (int)*p.m_dev) : p.M;   // a device-resident count
    const int n_tiles = (M + TM - 1) / TM;

    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;      // ring loads issued
            uint32_t it = 0;     // tiles begun
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++it) {
                if (it > 0 && !mbar_wait(a_empty, (it - 1) & 1u, kWaitLimit)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(a_full, nkc * KB_BYTES);
                for (int kb = 0; kb < nkc; ++kb)
                    tma_load_2d(sA + kb * KB_BYTES, &tmX, kb * TK, t * TM, a_full);
                for (int blk = 0; blk < nb && ok; ++blk) {
                    const int nk = nkc + (blk + 1 < nb ? K / TK : 0);
                    for (int kb = 0; kb < nk; ++kb, ++g) {
                        const uint32_t s = g % kStages, u = g / kStages;
                        if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1u, kWaitLimit)) {
                            ok = false;
                            break;
                        }
                        uint8_t* dst = sRing + s * L.stage_bytes;
                        if (kb < nkc) {
                            mbar_arrive_expect_tx(&full[s], G_BYTES);
                            tma_load_2d(dst, &tmG, kb * TK, blk * K2, &full[s]);
                        } else {
                            mbar_arrive_expect_tx(&full[s], W_BYTES);
                            tma_load_2d(dst, &tmW, (kb - nkc) * TK, blk * K, &full[s]);
                        }
                    }
                }
            }
            // copies still in flight land before the CTA goes away
            for (uint32_t s = 0; s < kStages && s < g; ++s) {
                const uint32_t last = (g - 1 - s) / kStages * kStages + s;   // last use of stage s
                mbar_wait(&full[s], (last / kStages) & 1u, kWaitLimit);
            }
            if (it > 0) mbar_wait(a_full, (it - 1) & 1u, kWaitLimit);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idG = idesc_bf16_f32(TM, K2);
            constexpr uint32_t idH = idesc_bf16_f32(TM, K);
            uint32_t g = 0, e = 0, it = 0, ng = 0, nh = 0;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++it) {
                if (!mbar_wait(a_full, it & 1u, kWaitLimit)) {
                    ok = false;
                    break;
                }
                for (int blk = 0; blk < nb && ok; ++blk) {
                    // the epilogue has drained the gamma/beta accumulator
                    if (ng > 0) {
                        if (!mbar_wait(epi_done, e & 1u, kWaitLimit)) {
                            ok = false;
                            break;
                        }
                        ++e;
                        tc_fence_after();
                        if (blk > 0) {
                            // linear layer of the previous block on its a
                            for (int kb = 0; kb < K / TK; ++kb, ++g) {
                                const uint32_t s = g % kStages, u = g / kStages;
                                if (!mbar_wait(&full[s], u & 1u, kWaitLimit)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint32_t a0 = smem_u32(sAct + kb * KB_BYTES);
                                const uint32_t b0 = smem_u32(sRing + s * L.stage_bytes);
#pragma unroll
                                for (int k = 0; k < 4; ++k)
                                    mma_bf16(tm_h, desc_k_sw128(a0 + k * 32),
                                             desc_k_sw128(b0 + k * 32), idH, (kb | k) != 0);
                                mma_commit(&empty[s]);
                            }
                            mma_commit(h_full);
                            ++nh;
                            if (!ok) break;
                        }
                    }
                    for (int kb = 0; kb < nkc; ++kb, ++g) {
                        const uint32_t s = g % kStages, u = g / kStages;
                        if (!mbar_wait(&full[s], u & 1u, kWaitLimit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sA + kb * KB_BYTES);
                        const uint32_t b0 = smem_u32(sRing + s * L.stage_bytes);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_bf16(tm_g, desc_k_sw128(a0 + k * 32), desc_k_sw128(b0 + k * 32),
                                     idG, (kb | k) != 0);
                        mma_commit(&empty[s]);
                    }
                    if (blk + 1 == nb) mma_commit(a_empty);
                    mma_commit(g_full);   // also after an error, so the epilogue is released
                    ++ng;
                }
            }
            (void)nh;
        }
    } else {
        const int q = warp & 3;
        const int hf = (warp - 2) >> 2;
        const int c_lo = hf * HALF;
        const int rt = q * 32 + lane;                       // row within the tile
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        uint32_t ig = 0, ih = 0, ix = 0;
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const int row = t * TM + rt;
            const bool live = row < M;
            int zi = 0;
            float zt = 0.f;
            if (live) {
                const float z = p.zbuf[row];
                const float pz = fminf(fmaxf(0.5f * (z + 1.0f), 0.0f), 1.0f);
                const float x = (float)(p.n_z - 1) * pz;
                zi = min((int)floorf(x), p.n_z - 2);
                zt = x - (float)zi;
            }
            float logit = 0.f;
            for (int blk = 0; blk < nb && ok; ++blk) {
                if (!__all_sync(0xffffffffu, mbar_wait(g_full, ig & 1u, kWaitLimit))) {
                    ok = false;
                    break;
                }
                ++ig;
                if (blk > 0) {
                    if (!__all_sync(0xffffffffu, mbar_wait(h_full, ih & 1u, kWaitLimit))) {
                        ok = false;
                        break;
                    }
                    ++ih;
                }
                tc_fence_after();
                const float* g0 = sg0 + blk * K2;
                const float* bl = sbl + (blk > 0 ? (blk - 1) * K : 0);
                const bool last = blk + 1 == nb;
#pragma unroll 1
                for (int c0 = c_lo; c0 < c_lo + HALF; c0 += 32) {
                    uint32_t rg[32], rb[32], rh[32];
                    ld32(tm_g + lane_off + c0, rg);
                    ld32(tm_g + lane_off + K + c0, rb);
                    if (blk > 0) ld32(tm_h + lane_off + c0, rh);
                    tmem_ld_wait();
                    float a[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = c0 + j;
                        float n;
                        if (blk > 0) {
                            n = __uint_as_float(rh[j]) + bl[c];
                        } else {
                            const float lo = __ldg(p.WzT + (int64_t)zi * K + c);
                            const float hi = __ldg(p.WzT + (int64_t)(zi + 1) * K + c);
                            n = fmaf(zt, hi, fmaf(1.0f - zt, lo, __ldg(p.bz + c)));
                        }
                        const float gm = __uint_as_float(rg[j]) + g0[c];
                        const float bt = __uint_as_float(rb[j]) + g0[K + c];
                        a[j] = fmaxf(fmaf(gm, n, bt), 0.0f);
                    }
                    if (last) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) logit = fmaf(swl[c0 + j], a[j], logit);
                    } else {
                        // BF16 a at (row rt, channel c) of the swizzled K-major operand
                        uint8_t* kbp = sAct + (c0 / TK) * KB_BYTES + rt * 128;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int chunk = ((c0 % TK) / 8 + v) ^ (rt & 7);
                            uint4 w;
                            w.x = pack2(a[8 * v + 0], a[8 * v + 1]);
                            w.y = pack2(a[8 * v + 2], a[8 * v + 3]);
                            w.z = pack2(a[8 * v + 4], a[8 * v + 5]);
                            w.w = pack2(a[8 * v + 6], a[8 * v + 7]);
                            *reinterpret_cast<uint4*>(kbp + chunk * 16) = w;
                        }
                    }
                }
                if (!last) fence_async_smem();   // a is read by the next MMA
                tc_fence_before();
                __syncwarp();
                if (last) {
                    // the two halves of each logit meet in shared memory
                    if (hf == 1) {
                        sxch[rt] = logit;
                        __syncwarp();
                        if (lane == 0) mbar_arrive(xch_full);
                    } else {
                        const bool seen = __all_sync(
                            0xffffffffu, mbar_wait(xch_full, ix & 1u, kWaitLimit));
                        if (!seen) ok = false;
                        if (seen && live) {
                            const float tt[4] = {logit + sxch[rt], 0.f, 0.f, 0.f};
                            last_epilogue(p.epi, p.p0 + row, 1, tt, p.blast);
                        }
                        __syncwarp();
                    }
                    ++ix;
                }
                if (lane == 0) mbar_arrive(epi_done);
            }
        }
    }
    if (!ok) atomicOr(p.err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// SoftZ depth and BF16 feature rows of points p0 .. p0 + m - 1: row r of X
// holds the C channels of point p0 + r; z[r] its projected depth (FP32).
// One thread per (point, 4 quads): the projection and taps once per group.
__global__ void __launch_bounds__(256) cbn_gather_kernel(PointSrc src, int64_t p0, int64_t m,
                                                         Calib calib, Map map,
                                                         __nv_bfloat16* __restrict__ X, int C,
                                                         float* __restrict__ z) {
    const uint32_t nq = (uint32_t)C / 4 + 1;          // feature quads + the depth quad
    const uint32_t ng = (nq + 3) / 4;
    if (src.count) m = min(m, (int64_t)*src.count);
    const int64_t total = m * ng;   // < 2^32: at most 2^22 rows of at most 257 groups
    const Map none{nullptr, 0, 0, 0, 0};
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)w / ng;
        const uint32_t q0 = ((uint32_t)w - r * ng) * 4;
        const PointSample ps = sample_point(src, p0 + r, calib, map, none);
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t qd = q0 + j;
            if (qd >= nq) break;
            const float4 v = sample_quad(ps, 4 * (int)qd);
            if (qd < (uint32_t)C / 4) {
                uint2 pk;
                pk.x = pack2(v.x, v.y);
                pk.y = pack2(v.z, v.w);
                *reinterpret_cast<uint2*>(X + (int64_t)r * C + 4 * qd) = pk;
            } else {
                z[r] = v.x;
            }
        }
    }
}

// Per device and width: the dynamic shared-memory size the kernel attribute
// allows so far (raised when a larger network needs more).
uint32_t g_attr[2][64] = {};

int g_sms[64] = {};

template <int K>
cudaError_t prepare_k(int C, int nb, int* sms_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const Layout L = layout_of(C, K, nb);
    const int idx = K == 128 ? 1 : 0;
    if (!(dev >= 0 && dev < 64 && g_attr[idx][dev] >= L.total)) {
        e = cudaFuncSetAttribute(cbn_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.total);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) g_attr[idx][dev] = L.total;
    }
    if (dev >= 0 && dev < 64 && g_sms[dev] > 0) {
        *sms_out = g_sms[dev];
        return cudaSuccess;
    }
    e = cudaDeviceGetAttribute(sms_out, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_sms[dev] = *sms_out;
    return e;
}

template <int K>
cudaError_t launch_k(const CbnTcMaps& mp, const CbnTcArgs& a, cudaStream_t s) {
    int sms = 0;
    cudaError_t e = prepare_k<K>(a.C, a.nb, &sms);
    if (e != cudaSuccess) return e;
    const Layout L = layout_of(a.C, K, a.nb);
    const int tiles = (a.M + TM - 1) / TM;
    const int grid = tiles < sms ? tiles : sms;
    cbn_tc_kernel<K><<<grid, kThreads, L.total, s>>>(*mp.tmX, *mp.tmG, *mp.tmW, a);
    return cudaGetLastError();
}

}  // namespace

bool cbn_tc_ok(int C, int K, int nb) {
    return (K == 64 || K == 128) && C % TK == 0 && C >= TK && nb >= 1 && nb <= 8 &&
           layout_of(C, K, nb).total <= 227 * 1024;
}

cudaError_t launch_cbn_gather(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                              const Map& map, __nv_bfloat16* X, int C, float* z,
                              cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    const int64_t total = m * ((C / 4 + 1 + 3) / 4);
    // a device-resident count gets a fixed, SM-filling grid that strides
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    cbn_gather_kernel<<<(unsigned)blocks, 256, 0, stream>>>(src, p0, m, calib, map, X, C, z);
    return cudaGetLastError();
}

cudaError_t cbn_tc_prepare(int C, int K, int nb) {
    if (!cbn_tc_ok(C, K, nb)) return cudaErrorInvalidValue;
    int sms = 0;
    return K == 128 ? prepare_k<128>(C, nb, &sms) : prepare_k<64>(C, nb, &sms);
}

cudaError_t launch_cbn_tc(const CbnTcMaps& mp, const CbnTcArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    if (!cbn_tc_ok(a.C, a.K, a.nb)) return cudaErrorInvalidValue;
    return a.K == 128 ? launch_k<128>(mp, a, s) : launch_k<64>(mp, a, s);
}

}  // namespace pifu
