// All hidden layers of one tensor-core batch (BF16 operands, FP32
// accumulation, Sec. 3.1's concatenation MLP) in ONE persistent launch.
//
// The per-layer form (mlp_tc.cu) finishes layer l on every row before layer
// l + 1 starts.  Each launch then ends in a partly filled wave, and at the
// finest level the 1024-wide activations of all rows (170 MB at 83 K points)
// pass through DRAM between the two layers.  Here one grid of one CTA per SM
// walks the tiles of all layers in a fixed order in which rows move through
// the layers in groups:
//
//   step s: layer L-1 on row group s - lag (L-1), ..., layer 1 on group
//           s - lag, layer 0 on group s    (a group: `group` 128-row blocks)
//
// so the activations a layer reads were written `lag` steps earlier and are
// still in L2, and the tiles of one layer fill the tail of another.  CTAs
// take the next tile of that order from a global counter when their TMA
// producer is ready for it (tiles of different layers take different times,
// so a fixed assignment would leave CTAs idle).  A tile of
// layer l >= 1 reads all columns of layer l-1 on its rows, which other CTAs
// may produce: every epilogue warp counts its finished part of a tile in
// dep[l][row block] (release), and the TMA producer waits for the full count
// of layer l-1 on its row block (acquire) before loading that operand.
//
// Deadlock freedom: tiles are handed out in increasing order, only to CTAs
// that are running, and a tile waits only on tiles with a smaller index,
// which were handed out before it to running CTAs.  The smallest tile any CTA
// is waiting on therefore has all its inputs finished, so some CTA always
// moves; the CTAs need not be resident all at once.  A tile's count is
// published when its own stores are done, never later, so no wait goes from
// a tile to a larger one.  Every wait is bounded anyway; one that gives up
// sets *err and the CTA stops.  The counters start at zero (set when the
// buffer is made) and the last CTA to finish zeroes them again.
//
// The producer passes each tile index to the MMA warp and the epilogue warps
// through an 8-slot queue in shared memory (full/empty mbarriers).
//
// Inside a CTA the roles are those of tc_linear_kernel: warp 0 lane 0 the TMA
// producer (4-stage ring of 128 x 64 A and BN x 64 W tiles), warp 1 the TMEM
// allocation and the MMA issuer (two accumulators of 256 columns), warps 2-9
// the epilogue (bias, leaky-ReLU, BF16 stores staged through shared memory,
// or the last layer fused into the last hidden layer's epilogue).
#include <cuda.h>
#include <cuda_bf16.h>

#include "epilogue.cuh"
#include "pifu_internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"
#include "chain_order.cuh"

namespace pifu {
namespace {

using namespace sm100;

constexpr int CBM = 128;
constexpr int CBK = 64;
constexpr int CSTAGES = 4;
constexpr int kCEpi = 8;
constexpr int kCThreads = 64 + 32 * kCEpi + 32;   // + the signal warp
constexpr uint32_t kCWait = 1u << 20;       // mbarrier polls
constexpr uint32_t kDepWait = 1u << 22;     // dependency polls (32 ns apart at least)
constexpr int kAccCols = 256;               // one accumulator: the widest tile
constexpr uint32_t kABytes = CBM * CBK * 2;
constexpr uint32_t kBBytes = kAccCols * CBK * 2;
constexpr int kFuseFloats = 4 * 256 + 2 * 4 * CBM + 16;   // last-layer W, exchange, flags
constexpr int kStageBytes = kCEpi * 32 * 64;

constexpr uint32_t chain_smem_bytes() {
    // ring + alignment slack + barriers + biases + fused last layer + staging
    return (uint32_t)CSTAGES * (kABytes + kBBytes) + 1024 + 512 + kChainBiasFloats * 4 +
           kFuseFloats * 4 + kStageBytes + 1024;
}
static_assert(chain_smem_bytes() <= 227 * 1024, "shared memory of the chain kernel");
static_assert(kChainMaxLayers <= kChainOrderMaxLayers, "tile order of every chain");

constexpr int kTQ = 8;   // tile queue slots (the producer runs at most 6 tiles ahead)

__device__ __forceinline__ bool wait_dep(const unsigned int* p, unsigned int target) {
    for (uint32_t it = 0; it < kDepWait; ++it) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return true;
        __nanosleep(32);
    }
    return false;
}

// Generic-proxy accesses before this point are ordered before later
// async-proxy (TMA) accesses of global memory.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__global__ void __launch_bounds__(kCThreads, 1) tc_chain_kernel(const __grid_constant__ ChainArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sA = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sB = sA + CSTAGES * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + CSTAGES * kBBytes);
    uint64_t* empty = full + CSTAGES;
    uint64_t* accf = empty + CSTAGES;
    uint64_t* acce = accf + 2;
    uint64_t* tq_full = acce + 2;        // [kTQ] tile index published
    uint64_t* tq_empty = tq_full + kTQ;  // [kTQ] read by the MMA, epilogue and signal warps
    uint64_t* tdone = tq_empty + kTQ;    // [2] every epilogue warp stored its part of the tile
    volatile int* stq = reinterpret_cast<volatile int*>(tdone + 2);   // [kTQ]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tdone + 2) + kTQ;
    float* sbias = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(full) + 512);
    float* sW5 = sbias + kChainBiasFloats;   // fused last layer: [n_out][BN of its layer]
    float* sxch = sW5 + 4 * 256;             // [2 buffers][4 outputs][128 rows]
    volatile uint32_t* sflag = reinterpret_cast<volatile uint32_t*>(sxch + 2 * 4 * CBM);
    uint4* sstage = reinterpret_cast<uint4*>(
        (reinterpret_cast<uintptr_t>(sxch + 2 * 4 * CBM) + 64 + 1023) & ~static_cast<uintptr_t>(1023));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nl = a.nl;
    const bool fused = a.fl.n_out > 0;
    const int lf = nl - 1;   // the layer carrying the last layer when fused

    if (threadIdx.x == 0) {
        for (int s = 0; s < CSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kCEpi);
        }
        for (int j = 0; j < kTQ; ++j) {
            mbar_init(&tq_full[j], 1);
            mbar_init(&tq_empty[j], 2 + kCEpi);
        }
        for (int b = 0; b < 2; ++b) mbar_init(&tdone[b], kCEpi);
        fence_mbar_init();
        for (int l = 0; l < nl; ++l) {
            if (a.L[l].nk1 > 0) prefetch_tmap(&a.L[l].tmA1);
            prefetch_tmap(&a.L[l].tmA2);
            prefetch_tmap(&a.L[l].tmW);
        }
    }
    for (int l = 0; l < nl; ++l)
        for (int c = threadIdx.x; c < a.L[l].N; c += blockDim.x)
            sbias[a.boff[l] + c] = a.L[l].bias[c];
    if (fused) {
        const int bn = a.L[lf].BN;
        for (int c = threadIdx.x; c < a.fl.n_out * bn; c += blockDim.x)
            sW5[c] = a.fl.W[(int64_t)(c / bn) * a.fl.ldw + (c % bn)];
        if (threadIdx.x < 8) sflag[threadIdx.x] = 0u;
    }
    if (warp == 1) tmem_alloc(tslot, 2 * kAccCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    griddep_wait();
    int M = a.M;
    if (a.m_dev) M = min(M, (int)*a.m_dev);
    const int n_mb = (M + CBM - 1) / CBM;
    const int n_g = (n_mb + a.group - 1) / a.group;

    ChainShape shape{};
    shape.nl = nl;
    shape.lag = a.lag;
    shape.group = a.group;
    long long total = 0;
    for (int l = 0; l < nl; ++l) {
        shape.ntn[l] = a.L[l].N / a.L[l].BN;
        total += (long long)n_mb * shape.ntn[l];
    }

    bool ok = true;
    // each role walks the same increasing tile indices with its own cursor
    ChainPos p = chain_begin(shape, n_mb, n_g);
    if (n_g > 0) chain_advance(shape, n_mb, n_g, p, 0);
    long long at = 0;
    auto seek = [&](long long t) {
        chain_advance(shape, n_mb, n_g, p, t - at);
        at = t;
        return chain_decode(shape, p);
    };

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: takes the next tile, publishes it, loads it
            // the next index is taken one tile ahead, so the atomic's latency
            // overlaps the current tile's loads (a taken tile still waits
            // only on smaller ones)
            uint32_t g = 0;
            unsigned int nxt = atomicAdd(a.next_tile, 1u);
            for (uint32_t i = 0; ok; ++i) {
                const uint32_t qj = i % kTQ, qu = i / kTQ;
                if (qu > 0 && !mbar_wait(&tq_empty[qj], (qu - 1) & 1u, kCWait)) {
                    ok = false;
                    break;
                }
                const long long tix = (long long)nxt;
                const int enc = tix < total ? (int)tix : -1;
                stq[qj] = enc;
                mbar_arrive(&tq_full[qj]);
                if (enc < 0) break;
                nxt = atomicAdd(a.next_tile, 1u);
                const ChainTile t = seek(enc);
                const ChainLayer& Ly = a.L[t.l];
                if (t.l > 0 && Ly.nk1 > 0) {
                    // every column of layer l-1 on this row block is stored
                    const ChainLayer& Lp = a.L[t.l - 1];
                    if (!wait_dep(a.dep + (t.l - 1) * a.max_mb + t.mb,
                                  (unsigned)(Lp.N / Lp.BN * kCEpi))) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async_global();
                }
                const int m0 = t.mb * CBM;
                const int n0 = t.nt * Ly.BN;
                const int nk = Ly.nk1 + Ly.nk2;
                const uint32_t bytes = kABytes + (uint32_t)Ly.BN * CBK * 2;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % CSTAGES;
                    const uint32_t u = g / CSTAGES;
                    if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1u, kCWait)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], bytes);
                    if (kb < Ly.nk1)
                        tma_load_2d(sA + s * kABytes, &Ly.tmA1, kb * CBK, m0, &full[s]);
                    else
                        tma_load_2d(sA + s * kABytes, &Ly.tmA2, (kb - Ly.nk1) * CBK, m0, &full[s]);
                    tma_load_2d(sB + s * kBBytes, &Ly.tmW, kb * CBK, n0, &full[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            uint32_t g = 0;
            for (uint32_t i = 0; ok; ++i) {
                const uint32_t qj = i % kTQ, qu = i / kTQ;
                if (!mbar_wait(&tq_full[qj], qu & 1u, kCWait)) {
                    ok = false;
                    break;
                }
                const int enc = stq[qj];
                mbar_arrive(&tq_empty[qj]);
                if (enc < 0) break;
                const ChainTile t = seek(enc);
                const ChainLayer& Ly = a.L[t.l];
                const uint32_t idesc = idesc_bf16_f32(CBM, Ly.BN);
                const uint32_t b = i & 1u, j = i >> 1;
                if (j > 0 && !mbar_wait(&acce[b], (j - 1) & 1u, kCWait)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + b * kAccCols;
                const int nk = Ly.nk1 + Ly.nk2;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % CSTAGES;
                    const uint32_t u = g / CSTAGES;
                    if (!mbar_wait(&full[s], u & 1u, kCWait)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kABytes);
                    const uint32_t b0 = smem_u32(sB + s * kBBytes);
                    // the last K-block stops after its last real column
                    const int ksteps = kb == nk - 1 ? Ly.klast : 4;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k >= ksteps) break;
                        mma_bf16(d, desc_k_sw128(a0 + k * 32), desc_k_sw128(b0 + k * 32), idesc,
                                 (kb | k) != 0 ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&accf[b]);   // also after an error, so the epilogue is released
            }
        }
    } else if (warp == 2 + kCEpi) {
        if (lane == 0) {
            // signal warp: once every epilogue warp has stored its part of a
            // tile (CTA-scope acquire), one GPU-scope fence and one count of
            // all of them for the CTAs that read it
            for (uint32_t i = 0; ok; ++i) {
                const uint32_t qj = i % kTQ, qu = i / kTQ;
                if (!mbar_wait(&tq_full[qj], qu & 1u, kCWait)) {
                    ok = false;
                    break;
                }
                const int enc = stq[qj];
                mbar_arrive(&tq_empty[qj]);
                if (enc < 0) break;
                const ChainTile t = seek(enc);
                const uint32_t b = i & 1u, j = i >> 1;
                if (!mbar_wait(&tdone[b], j & 1u, kCWait)) {
                    ok = false;
                    break;
                }
                if (!(fused && t.l == lf)) {
                    __threadfence();
                    atomicAdd(a.dep + t.l * a.max_mb + t.mb, (unsigned)kCEpi);
                }
            }
        }
    } else {
        // epilogue: TMEM lane quadrant q = warp % 4 holds rows 32 q .. + 31;
        // warps 2-5 take the tile's first half of the columns, 6-9 the second
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        uint4* st = sstage + (warp - 2) * 32 * 4;
        for (uint32_t i = 0;; ++i) {
            const uint32_t qj = i % kTQ, qu = i / kTQ;
            if (!__all_sync(0xffffffffu, mbar_wait(&tq_full[qj], qu & 1u, kCWait))) {
                ok = false;
                break;
            }
            const int enc = stq[qj];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tq_empty[qj]);
            if (enc < 0) break;
            const ChainTile t = seek(enc);
            const ChainLayer& Ly = a.L[t.l];
            const uint32_t b = i & 1u, j = i >> 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], j & 1u, kCWait))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int BN = Ly.BN;
            const int HALF = BN / 2;
            const int cbase = half * HALF;
            const int m0 = t.mb * CBM;
            const int n0 = t.nt * BN;
            const int row = m0 + q * 32 + lane;
            const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + b * kAccCols;
            const float* bb = sbias + a.boff[t.l] + n0;
            const bool fuse_here = fused && t.l == lf;
            float part[4] = {0.f, 0.f, 0.f, 0.f};
            // 64 columns per TMEM wait (32 when the half tile is narrower)
            const int CW = HALF >= 64 ? 64 : 32;
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + HALF; c0 += CW) {
                uint32_t r[64];
                if (CW == 64) {
                    tmem_ld64(tl + (uint32_t)c0, r);
                } else {
                    uint32_t(&r0)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[0]);
                    uint32_t(&r1)[16] = *reinterpret_cast<uint32_t(*)[16]>(&r[16]);
                    tmem_ld16(tl + (uint32_t)c0, r0);
                    tmem_ld16(tl + (uint32_t)c0 + 16, r1);
                    tmem_ld_wait();
                }
                if (fuse_here) {
                    // h rounded to BF16 (as a stored activation), dotted with
                    // the last layer's rows
#pragma unroll
                    for (int cc = 0; cc < 64; ++cc) {
                        if (cc >= CW) break;
                        float v = __uint_as_float(r[cc]) + bb[c0 + cc];
                        v = v >= 0.f ? v : a.slope * v;
                        v = __bfloat162float(__float2bfloat16_rn(v));
#pragma unroll
                        for (int jo = 0; jo < 4; ++jo)
                            if (jo < a.fl.n_out) part[jo] = fmaf(v, sW5[jo * BN + c0 + cc], part[jo]);
                    }
                } else {
                    // 32 BF16 values = 64 bytes of each row per staged store
#pragma unroll
                    for (int hb = 0; hb < 2; ++hb) {
                        if (hb * 32 >= CW) break;
                        uint4 pk4[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            uint32_t pk[4];
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int cc = hb * 32 + v * 8 + 2 * jj;
                                float x = __uint_as_float(r[cc]) + bb[c0 + cc];
                                float y = __uint_as_float(r[cc + 1]) + bb[c0 + cc + 1];
                                x = x >= 0.f ? x : a.slope * x;
                                y = y >= 0.f ? y : a.slope * y;
                                pk[jj] = pack_bf16x2(x, y);
                            }
                            pk4[v] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                        store_rows64(st, pk4, lane,
                                     reinterpret_cast<uint8_t*>(Ly.out + n0 + c0 + 32 * hb),
                                     (int64_t)Ly.ldo * 2, m0 + q * 32, M);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (!fuse_here) {
                // this warp's part of the tile is stored (the signal warp
                // publishes it) and its accumulator is free
                if (lane == 0) {
                    mbar_arrive(&tdone[b]);
                    mbar_arrive(&acce[b]);
                }
                continue;
            }
            // fused last layer: the column-half-1 warp of this lane quadrant
            // publishes its partial sums, the half-0 warp adds them and
            // finishes the row
            if (half == 1 && lane == 0) mbar_arrive(&acce[b]);
            float* xb = sxch + b * 4 * CBM;
            const int rit = q * 32 + lane;
            volatile uint32_t* flag = sflag + b * 4 + q;
            if (half == 1) {
#pragma unroll
                for (int jo = 0; jo < 4; ++jo)
                    if (jo < a.fl.n_out) xb[jo * CBM + rit] = part[jo];
                __threadfence_block();
                __syncwarp();
                if (lane == 0) {
                    *flag = i + 1u;
                    mbar_arrive(&tdone[b]);
                }
            } else {
                bool seen = true;
                if (lane == 0) {
                    seen = false;
                    for (uint32_t it = 0; it < kCWait; ++it)
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
                        tt[jo] = jo < a.fl.n_out ? part[jo] + xb[jo * CBM + rit] : 0.f;
                    last_epilogue(a.fl.epi, a.fl.p0 + row, a.fl.n_out, tt, a.fl.bias);
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&acce[b]);   // after reading the exchange
                    mbar_arrive(&tdone[b]);
                }
                if (!seen) break;
            }
        }
    }
    if (!ok) atomicOr(a.err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, 2 * kAccCols);
    // The last CTA to finish sets every counter back to zero for the next
    // launch (all others have made their last count before counting out).
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(a.done, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int l = 0; l < nl; ++l)
            for (int i = threadIdx.x; i < n_mb; i += blockDim.x) a.dep[l * a.max_mb + i] = 0u;
        if (threadIdx.x == 0) {
            *a.next_tile = 0u;
            *a.done = 0u;
        }
    }
}

int g_chain_attr[64] = {};   // per device: 1 once the shared-memory attribute is set
int g_chain_sms[64] = {};

}  // namespace

cudaError_t chain_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && g_chain_attr[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(tc_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chain_smem_bytes());
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_chain_kernel, kCThreads,
                                                      chain_smem_bytes());
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) {
        g_chain_attr[dev] = 1;
        g_chain_sms[dev] = sms;   // one CTA per SM
    }
    return cudaSuccess;
}

int chain_grid() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return g_chain_sms[dev];
}

cudaError_t launch_tc_chain(const ChainArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    if (a.nl < 1 || a.nl > kChainMaxLayers || a.group < 1 || a.lag < 1)
        return cudaErrorInvalidValue;
    cudaError_t e = chain_prepare();
    if (e != cudaSuccess) return e;
    const int grid = chain_grid();
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (a.next_tile != a.dep + (size_t)a.nl * a.max_mb || a.done != a.next_tile + 1)
        return cudaErrorInvalidValue;
    // Only running CTAs take tiles, and a tile waits only on tiles taken
    // before it, so the CTAs need not all be resident at once: a plain launch,
    // whose prologue may overlap the previous kernel (programmatic dependent
    // launch; the counters are read only after griddepcontrol.wait).
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = chain_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_chain_kernel, a);
}

}  // namespace pifu
