// Tensor-core (tcgen05) form of one hidden MLP layer: BF16 or E4M3
// operands, FP32 accumulation in tensor memory (Sec. 3.1's concatenation
// MLP, the "MLP" variant of Table A1: 2.36 MFLOP per point at full size, a
// dense contraction over a batch of points).
//
//   out[M][N] = lrelu( s[n] ([H | X][M][K] * W[N][K]^T) + b )
//
// BF16 modes: s = 1, BF16 operands, BF16 or E4M3 out (the latter multiplied
// by the next layer's inverse activation scale).  Mixed modes (the FP8 form's
// later layers): H in E4M3 against E4M3 weights (kind::f8f6f4), both stored
// divided by their scales (per tensor for H, per output channel for W), then
// X in BF16 against BF16 weights divided by the same two scales (kind::f16),
// all into one FP32 accumulator that s[n] multiplies back; BF16 or E4M3 out.
// One K-block is 128 bytes of a row in every mode: 64 BF16 or 128 E4M3
// values.
//
// The skip concatenation [h_{l-1}, x] is fused as two K segments: the TMA
// producer fetches A tiles from the H tensor map for the first nk1 K-blocks
// and from the X tensor map for the remaining nk2, against the matching
// columns of W (whose x part is zero-padded to a whole K-block).
//
// Persistent, warp-specialised kernel: one CTA per SM walks the 128 x BN
// output tiles (tile t covers rows 128 (t / (N/BN)), columns BN (t % (N/BN)),
// so the CTAs working at one moment share A rows through L2).  10 warps:
//   warp 0 lane 0   TMA producer: A (128 x 64) and W (BN x 64) tiles into a
//                   ring of 128B-swizzled shared-memory buffers, 4 stages
//                   deep for BN = 256, 6 for 128, 8 for 64 (the same 192 KB);
//   warp 1          allocates 2 x BN TMEM columns; lane 0 issues 4 x
//                   tcgen05.mma (K = 16) per stage into the accumulator of
//                   the current tile (two accumulators, used alternately),
//                   tcgen05.commit releases the stage and, after the last
//                   K-block, hands the accumulator to the epilogue;
//   warps 2 .. 9    epilogue, two warps per TMEM lane quadrant (the tile's
//                   rows 32 (warp % 4) ..), each taking half of the columns:
//                   tcgen05.ld 64 columns per wait, bias (staged in shared
//                   memory once per CTA) + leaky-ReLU, BF16 stores, then
//                   give the accumulator back -- overlapping the next
//                   tile's main loop.
// Every mbarrier wait is bounded; a wait that gives up sets *err, the role
// stops, and the CTA still releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "epilogue.cuh"
#include "pifu_internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"

namespace pifu {
namespace {

using namespace sm100;

constexpr int TBM = 128;
constexpr int TBK = 64;
constexpr int TSTAGES = 4;
constexpr uint32_t kWaitLimit = 1u << 20;   // polls; legitimate waits are microseconds

constexpr int kMaxN = 1024;   // widest layer whose bias is staged in shared memory
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;

constexpr int kFuseFloats = 4 * 256 + 2 * 4 * TBM + 16;   // last-layer W, exchange, flags
constexpr int kStageRowBytes = 64;                          // store staging: 64 B per row
constexpr int kStageBytes = kEpiWarps * 32 * kStageRowBytes; // 32 rows per epilogue warp

// Ring depth of a tile width: narrower W tiles make smaller stages, so the
// same 192 KB holds more of them (BN 256: 4, 128: 6, 64: 8) and more operand
// bytes stay in flight per MMA cycle.
__host__ __device__ constexpr int tc_stages(int BN) {
    return TSTAGES * (TBM * TBK * 2 + 256 * TBK * 2) / (TBM * TBK * 2 + BN * TBK * 2);
}

__host__ __device__ constexpr uint32_t tc_smem_bytes(int BN) {
    // operand ring + 1024-byte alignment slack + barriers + staged bias and
    // column scales + fused last layer + output staging
    return (uint32_t)tc_stages(BN) * (TBM * TBK * 2 + BN * TBK * 2) + 1024 + 256 + 2 * kMaxN * 4 +
           kFuseFloats * 4 + kStageBytes + 1024;   // + alignment of the staging area
}
static_assert(tc_stages(256) == 4 && tc_stages(128) == 6 && tc_stages(64) == 8, "ring depths");
static_assert(2 * tc_stages(64) * 8 + 4 * 8 + 4 <= 256, "barriers fit in front of the bias");
static_assert(tc_smem_bytes(256) <= 227 * 1024, "shared memory of the widest tile");

// Four consecutive floats of shared memory (16-byte aligned) in one load.
__device__ __forceinline__ float4 lds4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
}

// Four values rounded to E4M3 (saturating), first value in the lowest byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

template <int BN, bool FUSE, int MODE>
__global__ void __launch_bounds__(kThreads, 1) tc_linear_kernel(
    const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2,
    const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmO, int use_tmo,
    int nk1, int nk2, int klast, int M, int N, const float* __restrict__ bias, float slope,
    void* __restrict__ out_raw, int ldo, unsigned int* __restrict__ err,
    const unsigned int* __restrict__ m_dev, FuseLast fl, const float* __restrict__ colscale,
    float out_scale) {
    static_assert(!(FUSE && MODE != TC_BF16), "the fused last layer reads BF16 activations");
    constexpr bool MIX = MODE == TC_MIX_E4M3 || MODE == TC_MIX_BF16;
    constexpr bool OUT8 = MODE == TC_BF16_E4M3 || MODE == TC_MIX_E4M3;
    // elements per 128-byte K-block: A1 (E4M3 in the mixed modes), A2 (BF16),
    // W (a byte matrix in the mixed modes)
    constexpr int E1 = MIX ? 2 * TBK : TBK;
    constexpr int E2 = TBK;
    constexpr int EW = MIX ? 2 * TBK : TBK;
    constexpr uint32_t A_BYTES = TBM * TBK * 2;
    constexpr uint32_t B_BYTES = BN * TBK * 2;
    constexpr uint32_t TMEM_COLS = 2 * BN;   // two accumulators; 128, 256 or 512
    constexpr int NST = tc_stages(BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sA = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sB = sA + NST * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + NST * B_BYTES);
    uint64_t* empty = full + NST;
    uint64_t* accf = empty + NST;   // [2] accumulator ready for the epilogue
    uint64_t* acce = accf + 2;          // [2] accumulator drained by the epilogue
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
    float* sbias = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(full) + 256);
    float* scol = sbias + kMaxN;             // E4M3 modes: accumulator scale per column
    float* sW5 = scol + kMaxN;               // fused last layer: [4][BN]
    float* sxch = sW5 + 4 * 256;             // [2 buffers][4 outputs][128 rows] partial sums
    volatile uint32_t* sflag = reinterpret_cast<volatile uint32_t*>(sxch + 2 * 4 * TBM);  // [2][4]
    // per-warp store staging, 1024-byte aligned: its XOR pattern is the
    // 64-byte swizzle, so a TMA store (tmO) can take it as it is
    uint4* sstage = reinterpret_cast<uint4*>(
        (reinterpret_cast<uintptr_t>(sxch + 2 * 4 * TBM) + 64 + 1023) & ~static_cast<uintptr_t>(1023));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nk = nk1 + nk2;
    const int n_tn = N / BN;

    // Prologue: everything here depends only on the weights, so with a
    // programmatic dependent launch it overlaps the previous kernel's tail.
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps);   // one arrival per epilogue warp
        }
        fence_mbar_init();
        if (nk1 > 0) prefetch_tmap(&tmA1);
        prefetch_tmap(&tmA2);
        prefetch_tmap(&tmW);
    }
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        sbias[c] = bias[c];
        scol[c] = MIX ? colscale[c] : 1.f;
    }
    if (FUSE) {
        for (int c = threadIdx.x; c < fl.n_out * BN; c += blockDim.x)
            sW5[c] = fl.W[(int64_t)(c / BN) * fl.ldw + (c % BN)];
        if (threadIdx.x < 8) sflag[threadIdx.x] = 0u;
    }
    if (warp == 1) tmem_alloc(tslot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    // the activations and the device-resident row count come from earlier kernels
    griddep_wait();
    if (m_dev) M = min(M, (int)*m_dev);
    const int n_tiles = ((M + TBM - 1) / TBM) * n_tn;

    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            uint32_t g = 0;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int m0 = (t / n_tn) * TBM;
                const int n0 = (t % n_tn) * BN;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % NST;
                    const uint32_t u = g / NST;
                    if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1u, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                    if (kb < nk1)
                        tma_load_2d(sA + s * A_BYTES, &tmA1, kb * E1, m0, &full[s]);
                    else
                        tma_load_2d(sA + s * A_BYTES, &tmA2, (kb - nk1) * E2, m0, &full[s]);
                    tma_load_2d(sB + s * B_BYTES, &tmW, kb * EW, n0, &full[s]);
                }
            }
            // every load of this CTA is issued: the next layer's CTAs may be
            // placed (and run their prologue) as SMs free up
            griddep_launch_dependents();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            constexpr uint32_t idesc16 = idesc_bf16_f32(TBM, BN);
            constexpr uint32_t idesc8 = idesc_e4m3_f32(TBM, BN);
            uint32_t g = 0, i = 0;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++i) {
                const uint32_t b = i & 1u, j = i >> 1;
                if (j > 0 && !mbar_wait(&acce[b], (j - 1) & 1u, kWaitLimit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + b * BN;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % NST;
                    const uint32_t u = g / NST;
                    if (!mbar_wait(&full[s], u & 1u, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * A_BYTES);
                    const uint32_t b0 = smem_u32(sB + s * B_BYTES);
                    // 4 MMAs of 32 bytes of K each (16 BF16 or 32 E4M3 values);
                    // the last K-block stops after its last real column
                    const bool f8 = MIX && kb < nk1;
                    const int ksteps = kb == nk - 1 ? klast : 4;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k >= ksteps) break;
                        if (f8)
                            mma_e4m3(d, desc_k_sw128(a0 + k * 32), desc_k_sw128(b0 + k * 32),
                                     idesc8, (kb | k) != 0 ? 1u : 0u);
                        else
                            mma_bf16(d, desc_k_sw128(a0 + k * 32), desc_k_sw128(b0 + k * 32),
                                     idesc16, (kb | k) != 0 ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&accf[b]);   // also after an error, so the epilogue is released
            }
        }
    } else {
        // epilogue warps 2..9: TMEM lane quadrant q holds tile rows 32 q .. 32 q + 31;
        // warps 2-5 take columns [0, BN/2), warps 6-9 columns [BN/2, BN)
        constexpr int HALF = BN / 2;
        const int q = warp & 3;
        const int cbase = ((warp - 2) >> 2) * HALF;
        uint32_t i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            const uint32_t b = i & 1u, j = i >> 1;
            const int m0 = (t / n_tn) * TBM;
            const int n0 = (t % n_tn) * BN;
            // warp-uniform: tcgen05.ld below is a .sync.aligned warp instruction
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], j & 1u, kWaitLimit))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int row = m0 + q * 32 + lane;
            const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + b * BN;
            const float* bb = sbias + n0;
            const float* sc = scol + n0;
            const int half = (warp - 2) >> 2;
            float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + HALF; c0 += 64) {
                uint32_t r[64];
                if (HALF >= 64) {
                    tmem_ld64(tl + (uint32_t)c0, r);
                } else {
                    uint32_t(&r0)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[0]);
                    uint32_t(&r1)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[16]);
                    tmem_ld16(tl + (uint32_t)c0, r0);
                    tmem_ld16(tl + (uint32_t)c0 + 16, r1);
                    tmem_ld_wait();
                }
                constexpr int NC = HALF >= 64 ? 64 : HALF;
                if (FUSE) {
                    // h rounded to BF16 (as the unfused path stores it), dotted
                    // with the last layer's rows; shared-memory operands in
                    // 16-byte loads (the same values, in the same order)
#pragma unroll
                    for (int c4 = 0; c4 < NC; c4 += 4) {
                        const float4 b4 = lds4(bb + c0 + c4);
                        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
                        float h[4];
#pragma unroll
                        for (int t4 = 0; t4 < 4; ++t4) {
                            float a = __uint_as_float(r[c4 + t4]) + bv[t4];
                            a = a >= 0.f ? a : slope * a;
                            h[t4] = __bfloat162float(__float2bfloat16_rn(a));
                        }
#pragma unroll
                        for (int jo = 0; jo < 4; ++jo)
                            if (jo < fl.n_out) {
                                const float4 w4 = lds4(sW5 + jo * BN + c0 + c4);
                                part[jo] = fmaf(h[0], w4.x, part[jo]);
                                part[jo] = fmaf(h[1], w4.y, part[jo]);
                                part[jo] = fmaf(h[2], w4.z, part[jo]);
                                part[jo] = fmaf(h[3], w4.w, part[jo]);
                            }
                    }
                } else if (OUT8) {
                    // 64 E4M3 values = 64 bytes of the row: one staged pass
                    uint4 pk4[4];
#pragma unroll
                    for (int v = 0; v < NC / 16; ++v) {
                        uint32_t pk[4];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int cq = v * 16 + 4 * jj;
                            const float4 b4 = lds4(bb + c0 + cq);
                            const float4 s4 = lds4(sc + c0 + cq);
                            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
                            const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
                            float e[4];
#pragma unroll
                            for (int t4 = 0; t4 < 4; ++t4) {
                                float a = fmaf(__uint_as_float(r[cq + t4]), sv[t4], bv[t4]);
                                a = a >= 0.f ? a : slope * a;
                                e[t4] = a * out_scale;
                            }
                            pk[jj] = pack_e4m3x4(e[0], e[1], e[2], e[3]);
                        }
                        pk4[v] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                    if (NC == 64)
                        store_rows64(sstage + (warp - 2) * 32 * 4, pk4, lane,
                                     static_cast<uint8_t*>(out_raw) + n0 + c0, ldo, m0 + q * 32, M);
                    else if (row < M)
#pragma unroll
                        for (int v = 0; v < NC / 16; ++v)
                            reinterpret_cast<uint4*>(static_cast<uint8_t*>(out_raw) +
                                                     (int64_t)row * ldo + n0 + c0)[v] = pk4[v];
                } else {
                    // 64 BF16 values = 128 bytes of the row: two staged passes of 64 bytes
#pragma unroll
                    for (int hb = 0; hb < NC / 32; ++hb) {
                        uint4 pk4[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            // the 8 columns' bias (and scales) in two 16-byte loads
                            const int c8 = hb * 32 + v * 8;
                            const float4 b4a = lds4(bb + c0 + c8);
                            const float4 b4b = lds4(bb + c0 + c8 + 4);
                            const float bv[8] = {b4a.x, b4a.y, b4a.z, b4a.w,
                                                 b4b.x, b4b.y, b4b.z, b4b.w};
                            float sv[8];
                            if (MIX) {
                                const float4 s4a = lds4(sc + c0 + c8);
                                const float4 s4b = lds4(sc + c0 + c8 + 4);
                                sv[0] = s4a.x; sv[1] = s4a.y; sv[2] = s4a.z; sv[3] = s4a.w;
                                sv[4] = s4b.x; sv[5] = s4b.y; sv[6] = s4b.z; sv[7] = s4b.w;
                            }
                            uint32_t pk[4];
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int cc = c8 + 2 * jj;
                                float a, c;
                                if (!MIX) {
                                    a = __uint_as_float(r[cc]) + bv[2 * jj];
                                    c = __uint_as_float(r[cc + 1]) + bv[2 * jj + 1];
                                } else {
                                    a = fmaf(__uint_as_float(r[cc]), sv[2 * jj], bv[2 * jj]);
                                    c = fmaf(__uint_as_float(r[cc + 1]), sv[2 * jj + 1],
                                             bv[2 * jj + 1]);
                                }
                                a = a >= 0.f ? a : slope * a;
                                c = c >= 0.f ? c : slope * c;
                                pk[jj] = pack_bf16x2(a, c);
                            }
                            pk4[v] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                        uint4* st = sstage + (warp - 2) * 32 * 4;
                        if (use_tmo) {
                            // the TMA engine writes the warp's 32 x 32 box (rows past the
                            // tensor are dropped; rows past M are scratch of this pass)
                            if (lane == 0) bulk_wait_read();   // the previous box was read
                            __syncwarp();
                            const int sw = (lane >> 1) & 3;
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) st[lane * 4 + (jj ^ sw)] = pk4[jj];
                            fence_async_shared();
                            __syncwarp();
                            if (lane == 0) {
                                tma_store_2d(&tmO, n0 + c0 + 32 * hb, m0 + q * 32, st);
                                bulk_commit();
                            }
                        } else {
                            store_rows64(st, pk4, lane,
                                         reinterpret_cast<uint8_t*>(
                                             static_cast<__nv_bfloat16*>(out_raw) + n0 + c0 +
                                             32 * hb),
                                         (int64_t)ldo * 2, m0 + q * 32, M);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (!FUSE || half == 1) {
                if (lane == 0) mbar_arrive(&acce[b]);
            }
            if (FUSE) {
                // the column-half-1 warp of this lane quadrant publishes its
                // partial sums; the half-0 warp adds them and finishes the row
                float* xb = sxch + b * 4 * TBM;
                const int rit = q * 32 + lane;
                volatile uint32_t* flag = sflag + b * 4 + q;
                if (half == 1) {
#pragma unroll
                    for (int jo = 0; jo < 4; ++jo)
                        if (jo < fl.n_out) xb[jo * TBM + rit] = part[jo];
                    __threadfence_block();
                    __syncwarp();
                    if (lane == 0) *flag = i + 1u;
                } else {
                    bool seen = true;
                    if (lane == 0) {
                        seen = false;
                        for (uint32_t it = 0; it < kWaitLimit; ++it)
                            if (*flag == i + 1u) {
                                seen = true;
                                break;
                            }
                    }
                    seen = __shfl_sync(0xffffffffu, seen ? 1 : 0, 0) != 0;
                    __threadfence_block();
                    if (!seen) ok = false;
                    if (seen && row < M) {
                        float tt[4];
#pragma unroll
                        for (int jo = 0; jo < 4; ++jo)
                            tt[jo] = jo < fl.n_out ? part[jo] + xb[jo * TBM + rit] : 0.f;
                        last_epilogue(fl.epi, fl.p0 + row, fl.n_out, tt, fl.bias);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[b]);   // after reading the exchange
                    if (!seen) break;
                }
            }
        }
    }
    if (use_tmo && warp >= 2 && lane == 0) bulk_wait();   // the output is written
    if (!ok) atomicOr(err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ---- CTA-pair form ------------------------------------------------------------
//
// The same layer (BF16 operands and output, no fused last layer) on pairs of
// CTAs (clusters of 2) issuing cta_group::2 MMAs of M = 256, N = 256.  A pair
// walks 256 x 256 output tiles.  CTA r of the pair loads A rows m0 + 128 r
// and W rows n0 + 128 r of each K-block into its own shared memory, so a
// stage holds 32 KB per CTA instead of 48 KB for the same MMA work per SM:
// the ring is PS stages deep (more MMA work in flight per byte of shared
// memory) and each SM fetches a third less operand data from L2.
//   * Both CTAs' TMA loads complete on the even CTA's `full` barrier, whose
//     producer announces both CTAs' bytes.
//   * The even CTA's lane 0 of warp 1 issues the MMAs; its commits arrive on
//     the `empty` and `accf` barriers of both CTAs (multicast).
//   * Each CTA's epilogue drains its own 128 rows x 256 columns of tensor
//     memory and arrives on the even CTA's `acce` barrier.
// Every wait is bounded as in tc_linear_kernel; before the CTAs leave, the
// producers wait for the last releases of their stages and the pair meets at
// a cluster barrier, so no arrival is still on its way to a CTA that exited.
constexpr int kPairBN = 256;

__host__ __device__ constexpr uint32_t tc_pair_smem_bytes(int PS, int SB) {
    // operand ring + alignment slack + barriers + staged bias + output staging
    return (uint32_t)PS * (TBM * TBK * 2 + (kPairBN / 2) * TBK * 2) + 1024 + 256 + kMaxN * 4 +
           (uint32_t)SB * kStageBytes + 1024;
}

template <int PS, int SB>
__global__ void __launch_bounds__(kThreads, 1) tc_pair_kernel(
    const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2,
    const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmO, int use_tmo,
    int nk1, int nk2, int klast, int M, int N, const float* __restrict__ bias, float slope,
    __nv_bfloat16* __restrict__ out, int ldo, unsigned int* __restrict__ err,
    const unsigned int* __restrict__ m_dev) {
    constexpr int BN = kPairBN;
    constexpr uint32_t A_BYTES = TBM * TBK * 2;          // this CTA's 128 rows
    constexpr uint32_t B_BYTES = (BN / 2) * TBK * 2;     // this CTA's half of the columns
    constexpr uint32_t TMEM_COLS = 2 * BN;               // two accumulators of 256 columns
    static_assert((2 * PS + 4) * 8 + 4 <= 256, "barriers fit in front of the bias");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sA = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sB = sA + PS * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + PS * B_BYTES);
    uint64_t* empty = full + PS;
    uint64_t* accf = empty + PS;   // [2] accumulator ready (both CTAs)
    uint64_t* acce = accf + 2;     // [2] accumulator drained (counted in the even CTA)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
    float* sbias = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(full) + 256);
    uint4* sstage = reinterpret_cast<uint4*>(
        (reinterpret_cast<uintptr_t>(sbias + kMaxN) + 1023) & ~static_cast<uintptr_t>(1023));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();   // 0: issues the MMAs
    const int nk = nk1 + nk2;
    const int n_tn = N / BN;
    const int pair = blockIdx.x >> 1;
    const int n_pairs = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 2 * kEpiWarps);   // every epilogue warp of both CTAs
        }
        fence_mbar_init();
        if (nk1 > 0) prefetch_tmap(&tmA1);
        prefetch_tmap(&tmA2);
        prefetch_tmap(&tmW);
    }
    for (int c = threadIdx.x; c < N; c += blockDim.x) sbias[c] = bias[c];
    // both CTAs' barriers exist before either CTA signals the other's, and
    // both CTAs run before the pair allocates tensor memory
    cluster_sync();
    if (warp == 1) tmem_alloc_pair(tslot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    griddep_wait();
    if (m_dev) M = min(M, (int)*m_dev);
    const int n_tiles = ((M + 2 * TBM - 1) / (2 * TBM)) * n_tn;

    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            // TMA producer of this CTA's halves; the bytes of both count on the
            // even CTA's full barrier
            uint32_t g = 0;
            for (int t = pair; t < n_tiles && ok; t += n_pairs) {
                const int m0 = (t / n_tn) * 2 * TBM + (int)rank * TBM;
                const int n0 = (t % n_tn) * BN + (int)rank * (BN / 2);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % PS;
                    const uint32_t u = g / PS;
                    if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1u, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * (A_BYTES + B_BYTES));
                    const uint32_t fb = mapa_shared(smem_u32(&full[s]), 0);
                    if (kb < nk1)
                        tma_load_2d_pair(sA + s * A_BYTES, &tmA1, kb * TBK, m0, fb);
                    else
                        tma_load_2d_pair(sA + s * A_BYTES, &tmA2, (kb - nk1) * TBK, m0, fb);
                    tma_load_2d_pair(sB + s * B_BYTES, &tmW, kb * TBK, n0, fb);
                }
            }
            // the last release of every stage used has arrived here
            if (ok) {
                for (uint32_t s = 0; s < (uint32_t)PS && s < g; ++s) {
                    const uint32_t uses = (g - s + PS - 1) / PS;
                    if (!mbar_wait(&empty[s], (uses - 1) & 1u, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // MMA issuer of the pair
            constexpr uint32_t idesc = idesc_bf16_f32(2 * TBM, BN);
            uint32_t g = 0, i = 0;
            for (int t = pair; t < n_tiles && ok; t += n_pairs, ++i) {
                const uint32_t b = i & 1u, j = i >> 1;
                if (j > 0 && !mbar_wait_cluster(&acce[b], (j - 1) & 1u, kWaitLimit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + b * BN;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % PS;
                    const uint32_t u = g / PS;
                    if (!mbar_wait(&full[s], u & 1u, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * A_BYTES);
                    const uint32_t b0 = smem_u32(sB + s * B_BYTES);
                    const int ksteps = kb == nk - 1 ? klast : 4;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k >= ksteps) break;
                        mma_bf16_pair(d, desc_k_sw128(a0 + k * 32), desc_k_sw128(b0 + k * 32),
                                      idesc, (kb | k) != 0 ? 1u : 0u);
                    }
                    mma_commit_pair(&empty[s], (uint16_t)3);
                }
                mma_commit_pair(&accf[b], (uint16_t)3);   // also after an error
            }
        }
    } else {
        // epilogue warps 2..9 of each CTA: its rows 32 (warp % 4) .. + 31 of
        // the pair tile's half, warps 2-5 columns [0, 128), warps 6-9 [128, 256)
        constexpr int HALF = BN / 2;
        const int q = warp & 3;
        const int cbase = ((warp - 2) >> 2) * HALF;
        const uint32_t acce0 = mapa_shared(smem_u32(&acce[0]), 0);
        uint4* stw = sstage + (warp - 2) * SB * 32 * 4;   // this warp's SB staging boxes
        uint32_t i = 0, nbox = 0;
        for (int t = pair; t < n_tiles; t += n_pairs, ++i) {
            const uint32_t b = i & 1u, j = i >> 1;
            const int m0 = (t / n_tn) * 2 * TBM + (int)rank * TBM;
            const int n0 = (t % n_tn) * BN;
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], j & 1u, kWaitLimit))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + b * BN;
            const float* bb = sbias + n0;
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + HALF; c0 += 64) {
                uint32_t r[64];
                tmem_ld64(tl + (uint32_t)c0, r);
#pragma unroll
                for (int hb = 0; hb < 2; ++hb) {
                    uint4 pk4[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        uint32_t pk[4];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int cc = hb * 32 + v * 8 + 2 * jj;
                            float a = __uint_as_float(r[cc]) + bb[c0 + cc];
                            float c = __uint_as_float(r[cc + 1]) + bb[c0 + cc + 1];
                            a = a >= 0.f ? a : slope * a;
                            c = c >= 0.f ? c : slope * c;
                            pk[jj] = pack_bf16x2(a, c);
                        }
                        pk4[v] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                    uint4* st = stw + (nbox % SB) * 32 * 4;
                    ++nbox;
                    if (use_tmo) {
                        // at most SB - 1 of this warp's earlier boxes may still be read
                        if (lane == 0) bulk_wait_read_n<SB - 1>();
                        __syncwarp();
                        const int sw = (lane >> 1) & 3;
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) st[lane * 4 + (jj ^ sw)] = pk4[jj];
                        fence_async_shared();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_2d(&tmO, n0 + c0 + 32 * hb, m0 + q * 32, st);
                            bulk_commit();
                        }
                    } else {
                        store_rows64(st, pk4, lane,
                                     reinterpret_cast<uint8_t*>(out + n0 + c0 + 32 * hb),
                                     (int64_t)ldo * 2, m0 + q * 32, M);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acce0 + b * 8u);
        }
    }
    if (use_tmo && warp >= 2 && lane == 0) bulk_wait();
    if (!ok) atomicOr(err, 1u);
    tc_fence_before();
    __syncwarp();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) tmem_dealloc_pair(tmem, TMEM_COLS);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Per device: kernel attributes set (index by BN: 64, 128, 256) and SM count.
bool g_attr_set[3][64] = {};
int g_n_sm[64] = {};

constexpr int bn_index(int BN) { return BN == 64 ? 0 : (BN == 128 ? 1 : 2); }

template <int BN>
cudaError_t ensure_attr(int dev) {
    if (dev >= 0 && dev < 64 && g_attr_set[bn_index(BN)][dev]) return cudaSuccess;
    const int bytes = (int)tc_smem_bytes(BN);
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(tc_linear_kernel<BN, false, TC_BF16>, at, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tc_linear_kernel<BN, true, TC_BF16>, at, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_linear_kernel<BN, false, TC_BF16_E4M3>, at, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_linear_kernel<BN, false, TC_MIX_E4M3>, at, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_linear_kernel<BN, false, TC_MIX_BF16>, at, bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_attr_set[bn_index(BN)][dev] = true;
    return e;
}

cudaError_t sm_count(int dev, int* out) {
    if (dev >= 0 && dev < 64 && g_n_sm[dev] > 0) {
        *out = g_n_sm[dev];
        return cudaSuccess;
    }
    const cudaError_t e = cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_n_sm[dev] = *out;
    return e;
}

template <int BN>
cudaError_t launch_bn(const TcLayerArgs& a, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = ensure_attr<BN>(dev);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = sm_count(dev, &sms);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)(a.N / BN) * ((a.M + TBM - 1) / TBM);
    const int grid = (int)(tiles < sms ? tiles : sms);
    const uint32_t smem = tc_smem_bytes(BN);
    if (a.mode != TC_BF16 && a.fuse) return cudaErrorInvalidValue;
    if ((a.mode == TC_MIX_E4M3 || a.mode == TC_MIX_BF16) && !a.colscale)
        return cudaErrorInvalidValue;
    // programmatic dependent launch: the prologue overlaps the previous kernel
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const float* noscale = nullptr;
    const int kl = a.klast >= 1 && a.klast <= 4 ? a.klast : 4;
    // the TMA-store epilogue needs the output map (BF16 output, not fused)
    const int use_tmo = a.tmO ? 1 : 0;
    const CUtensorMap& tmO = a.tmO ? *a.tmO : *a.tmW;
    if (a.fuse) {
        if (a.N != BN || a.fuse->n_out < 1 || a.fuse->n_out > 4) return cudaErrorInvalidValue;
        return cudaLaunchKernelEx(&cfg, tc_linear_kernel<BN, true, TC_BF16>, *a.tmA1, *a.tmA2,
                                  *a.tmW, tmO, 0, a.nk1, a.nk2, kl, a.M, a.N, a.bias, a.slope, a.out,
                                  a.ldo, a.err, a.m_dev, *a.fuse, noscale, 1.f);
    }
    if (a.mode == TC_BF16_E4M3)
        return cudaLaunchKernelEx(&cfg, tc_linear_kernel<BN, false, TC_BF16_E4M3>, *a.tmA1,
                                  *a.tmA2, *a.tmW, tmO, 0, a.nk1, a.nk2, kl, a.M, a.N, a.bias,
                                  a.slope, a.out, a.ldo, a.err, a.m_dev, FuseLast{}, noscale,
                                  a.out_scale);
    if (a.mode == TC_MIX_E4M3)
        return cudaLaunchKernelEx(&cfg, tc_linear_kernel<BN, false, TC_MIX_E4M3>, *a.tmA1,
                                  *a.tmA2, *a.tmW, tmO, 0, a.nk1, a.nk2, kl, a.M, a.N, a.bias,
                                  a.slope, a.out, a.ldo, a.err, a.m_dev, FuseLast{}, a.colscale,
                                  a.out_scale);
    if (a.mode == TC_MIX_BF16)
        return cudaLaunchKernelEx(&cfg, tc_linear_kernel<BN, false, TC_MIX_BF16>, *a.tmA1,
                                  *a.tmA2, *a.tmW, tmO, use_tmo, a.nk1, a.nk2, kl, a.M, a.N, a.bias,
                                  a.slope, a.out, a.ldo, a.err, a.m_dev, FuseLast{}, a.colscale,
                                  1.f);
    return cudaLaunchKernelEx(&cfg, tc_linear_kernel<BN, false, TC_BF16>, *a.tmA1, *a.tmA2,
                              *a.tmW, tmO, use_tmo, a.nk1, a.nk2, kl, a.M, a.N, a.bias, a.slope,
                              a.out, a.ldo, a.err, a.m_dev, FuseLast{}, noscale, 1.f);
}

// CTA-pair form: ring depth and output staging boxes per epilogue warp.
constexpr int kPairStages = 6;
constexpr int kPairStageBufs = 1;
static_assert(tc_pair_smem_bytes(kPairStages, kPairStageBufs) <= 227 * 1024,
              "shared memory of the CTA-pair form");

// Co-resident clusters of 2 per device (0: not known yet); finding them also
// sets the kernel's shared-memory attribute.
template <int PS, int SB>
cudaError_t pair_clusters(int dev, int* out) {
    static int g_pair_clusters[64] = {};
    if (dev >= 0 && dev < 64 && g_pair_clusters[dev] > 0) {
        *out = g_pair_clusters[dev];
        return cudaSuccess;
    }
    const uint32_t smem = tc_pair_smem_bytes(PS, SB);
    cudaError_t e = cudaFuncSetAttribute(tc_pair_kernel<PS, SB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, tc_pair_kernel<PS, SB>, &cfg);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) g_pair_clusters[dev] = n;
    *out = n;
    return cudaSuccess;
}

template <int PS, int SB>
cudaError_t launch_pair_cfg(const TcLayerArgs& a, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int ncl = 0;
    e = pair_clusters<PS, SB>(dev, &ncl);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)(a.N / kPairBN) * ((a.M + 2 * TBM - 1) / (2 * TBM));
    const int clusters = (int)(tiles < ncl ? tiles : ncl);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(2 * clusters));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = tc_pair_smem_bytes(PS, SB);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    const int use_tmo = a.tmO ? 1 : 0;
    const CUtensorMap& tmO = a.tmO ? *a.tmO : *a.tmW;
    const int kl = a.klast >= 1 && a.klast <= 4 ? a.klast : 4;
    return cudaLaunchKernelEx(&cfg, tc_pair_kernel<PS, SB>, *a.tmA1, *a.tmA2, *a.tmW, tmO, use_tmo,
                              a.nk1, a.nk2, kl, a.M, a.N, a.bias, a.slope,
                              static_cast<__nv_bfloat16*>(a.out), a.ldo, a.err, a.m_dev);
}

cudaError_t launch_pair(const TcLayerArgs& a, cudaStream_t s) {
    // BF16 in and out, 256-column pair tiles, no fused last layer
    if (a.BN != kPairBN || a.mode != TC_BF16 || a.fuse || a.N % kPairBN != 0)
        return cudaErrorInvalidValue;
    return launch_pair_cfg<kPairStages, kPairStageBufs>(a, s);
}

}  // namespace

namespace {

bool encode_2d(void* map, CUtensorMapDataType dtype, const void* base, uint64_t cols,
               uint64_t rows, uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows,
               CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {row_stride_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(static_cast<CUtensorMap*>(map), dtype, 2,
                                const_cast<void*>(base), dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_encode_2d_bf16(void* map, const void* base, uint64_t cols, uint64_t rows,
                       uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, cols, rows, row_stride_bytes,
                     box_cols, box_rows);
}

bool tc_encode_2d_bf16_out(void* map, const void* base, uint64_t cols, uint64_t rows,
                           uint64_t row_stride_bytes) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, cols, rows, row_stride_bytes, 32,
                     32, CU_TENSOR_MAP_SWIZZLE_64B);
}

bool tc_encode_2d_u8(void* map, const void* base, uint64_t cols, uint64_t rows,
                     uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, base, cols, rows, row_stride_bytes,
                     box_cols, box_rows);
}

cudaError_t tc_prepare() {
    int dev = 0, sms = 0, ncl = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = ensure_attr<64>(dev);
    if (e == cudaSuccess) e = ensure_attr<128>(dev);
    if (e == cudaSuccess) e = ensure_attr<256>(dev);
    if (e == cudaSuccess) e = sm_count(dev, &sms);
    if (e == cudaSuccess) e = pair_clusters<kPairStages, kPairStageBufs>(dev, &ncl);
    return e;
}

cudaError_t launch_tc_linear(const TcLayerArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    if (a.N > kMaxN) return cudaErrorInvalidValue;
    if (a.pair) return launch_pair(a, s);
    switch (a.BN) {
        case 256: return launch_bn<256>(a, s);
        case 128: return launch_bn<128>(a, s);
        case 64: return launch_bn<64>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pifu
