// Device helpers shared by the tensor-core layer kernels (mlp_tc.cu,
// mlp_chain.cu): TMEM reads, BF16 packing and the staged row stores of the
// epilogues.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "sm100.cuh"

namespace pifu {

// Store a warp's 32 rows x 64 bytes (lane l holds row l's four 16-byte
// pieces v[0..3]) to dst(row) + 16 j: through the warp's shared-memory
// staging area so that each global store instruction writes 8 rows x 64
// contiguous bytes (full 32-byte sectors) instead of 32 rows x 16 bytes.
// Pieces are XOR-swizzled by row so both the write and the read-back take the
// minimum number of shared-memory wavefronts.  Rows with !live skip the store.
__device__ __forceinline__ void store_rows64(uint4* stage, const uint4 (&v)[4], int lane,
                                             uint8_t* row_base, int64_t row_stride, int row0,
                                             int M) {
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) stage[lane * 4 + (j ^ sw)] = v[j];
    __syncwarp();
    const int j = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = (lane >> 2) + 8 * i;
        const uint4 x = stage[r * 4 + (j ^ ((r >> 1) & 3))];
        if (row0 + r < M)
            *reinterpret_cast<uint4*>(row_base + (int64_t)(row0 + r) * row_stride + 16 * j) = x;
    }
    __syncwarp();
}

// 64 consecutive TMEM columns of the warp's 32 lanes: four x16 loads, one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
    uint32_t(&r0)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[0]);
    uint32_t(&r1)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[16]);
    uint32_t(&r2)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[32]);
    uint32_t(&r3)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[48]);
    sm100::tmem_ld16(taddr, r0);
    sm100::tmem_ld16(taddr + 16, r1);
    sm100::tmem_ld16(taddr + 32, r2);
    sm100::tmem_ld16(taddr + 48, r3);
    sm100::tmem_ld_wait();
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

}  // namespace pifu
