// Tensor-core (tcgen05) form of one hidden MLP layer: BF16 operands, FP32
// accumulation in tensor memory (Sec. 3.1's concatenation MLP, the "MLP"
// variant of Table A1: 2.36 MFLOP per point at full size, a dense
// contraction over a batch of points).
//
//   out[M][N] = lrelu( [H | X][M][K] * W[N][K]^T + b )        (BF16 out)
//
// The skip concatenation [h_{l-1}, x] is fused as two K segments: the TMA
// producer fetches A tiles from the H tensor map for the first nk1 K-blocks
// and from the X tensor map for the remaining nk2, against the matching
// columns of W (whose x part is zero-padded to a whole K-block).
//
// One CTA computes a 128 x BN tile with 4 warps:
//   warp 0 lane 0  TMA producer: A (128 x 64) and W (BN x 64) tiles into a
//                  4-stage ring of 128B-swizzled shared-memory buffers;
//   warp 1 lane 0  MMA issuer: 4 x tcgen05.mma (K = 16 each) per stage into
//                  one TMEM accumulator of BN columns, tcgen05.commit frees
//                  the stage;
//   all 4 warps    epilogue: tcgen05.ld of their 32 TMEM lanes (= rows),
//                  bias + leaky-ReLU, BF16 stores.
// Every mbarrier wait is bounded; a wait that gives up sets *err and the CTA
// still releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "pifu_internal.h"
#include "sm100.cuh"

namespace pifu {
namespace {

using namespace sm100;

constexpr int TBM = 128;
constexpr int TBK = 64;
constexpr int TSTAGES = 4;
constexpr uint32_t kWaitLimit = 1u << 20;   // polls; legitimate waits are microseconds

__host__ __device__ constexpr uint32_t tc_smem_bytes(int BN) {
    return (uint32_t)TSTAGES * (TBM * TBK * 2 + BN * TBK * 2) + 1024 + 256;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <int BN>
__global__ void __launch_bounds__(128, 1) tc_linear_kernel(
    const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2,
    const __grid_constant__ CUtensorMap tmW, int nk1, int nk2, int M,
    const float* __restrict__ bias, float slope, __nv_bfloat16* __restrict__ out, int ldo,
    unsigned int* __restrict__ err) {
    constexpr uint32_t A_BYTES = TBM * TBK * 2;
    constexpr uint32_t B_BYTES = BN * TBK * 2;
    constexpr uint32_t TMEM_COLS = BN;   // 64, 128 or 256: a power of two >= 32
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sA = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sB = sA + TSTAGES * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + TSTAGES * B_BYTES);
    uint64_t* empty = full + TSTAGES;
    uint64_t* accf = empty + TSTAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TBM;
    const int n0 = blockIdx.x * BN;
    const int nk = nk1 + nk2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        fence_mbar_init();
        if (nk1 > 0) prefetch_tmap(&tmA1);
        prefetch_tmap(&tmA2);
        prefetch_tmap(&tmW);
    }
    if (warp == 0) tmem_alloc(tslot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TSTAGES;
            const uint32_t u = (uint32_t)(kb / TSTAGES);
            if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1u, kWaitLimit)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
            if (kb < nk1)
                tma_load_2d(sA + s * A_BYTES, &tmA1, kb * TBK, m0, &full[s]);
            else
                tma_load_2d(sA + s * A_BYTES, &tmA2, (kb - nk1) * TBK, m0, &full[s]);
            tma_load_2d(sB + s * B_BYTES, &tmW, kb * TBK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16_f32(TBM, BN);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TSTAGES;
            const uint32_t u = (uint32_t)(kb / TSTAGES);
            if (!mbar_wait(&full[s], u & 1u, kWaitLimit)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * A_BYTES);
            const uint32_t b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int k = 0; k < TBK / 16; ++k)
                mma_bf16(tmem, desc_k_sw128(a0 + k * 32), desc_k_sw128(b0 + k * 32), idesc,
                         (kb | k) != 0 ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        mma_commit(accf);   // also after an error, so the epilogue is released
    }
    __syncwarp();

    // epilogue: TMEM lanes 32 warp .. 32 warp + 31 hold rows m0 + 32 warp + lane
    // warp-uniform decision: tcgen05.ld below is a .sync.aligned warp instruction
    const bool acc_ready = __all_sync(0xffffffffu, mbar_wait(accf, 0, kWaitLimit));
    tc_fence_after();
    if (acc_ready) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tl + (uint32_t)c0, r);
            tmem_ld_wait();
            if (row < M) {
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float a = __uint_as_float(r[2 * j]) + __ldg(bias + n0 + c0 + 2 * j);
                    float b = __uint_as_float(r[2 * j + 1]) + __ldg(bias + n0 + c0 + 2 * j + 1);
                    a = a >= 0.f ? a : slope * a;
                    b = b >= 0.f ? b : slope * b;
                    pk[j] = pack_bf16x2(a, b);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + (int64_t)row * ldo + n0 + c0);
                dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
    } else {
        ok = false;
    }
    if (!ok) atomicOr(err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

template <int BN>
cudaError_t launch_bn(const TcLayerArgs& a, cudaStream_t s) {
    static bool attr_set[64] = {};   // per device ordinal
    const uint32_t smem = tc_smem_bytes(BN);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(tc_linear_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid(a.N / BN, (unsigned)((a.M + TBM - 1) / TBM));
    tc_linear_kernel<BN><<<grid, 128, smem, s>>>(*a.tmA1, *a.tmA2, *a.tmW, a.nk1, a.nk2, a.M,
                                                 a.bias, a.slope, a.out, a.ldo, a.err);
    return cudaGetLastError();
}

}  // namespace

bool tc_encode_2d_bf16(void* map, const void* base, uint64_t cols, uint64_t rows,
                       uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows) {
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
    const CUresult r = g_encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                const_cast<void*>(base), dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_tc_linear(const TcLayerArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    switch (a.BN) {
        case 256: return launch_bn<256>(a, s);
        case 128: return launch_bn<128>(a, s);
        case 64: return launch_bn<64>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pifu
