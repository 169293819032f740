// FP32-accurate MLP on the tensor cores, for the small batches of the MIXED
// forms: the re-evaluation of occupancies that the BF16 pass put near Sec.
// 3.2's decision threshold 0.5, and batches too small for a BF16 pass plus a
// re-check.  These batches hold a few to a few thousand points; in FP32 FFMA
// they are latency-bound on a few SMs.
//
// Arithmetic (the split-TF32 method of Ootomo and Yokota, 2022, restated):
// each FP32 value v is held as two TF32 values, hi = tf32(v) and
// lo = tf32(v - hi), so v = hi + lo to about 2^-22 |v|; a product a b is
// formed as a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo is below
// 2^-22 |a b|), three kind::tf32 tcgen05 MMAs into one FP32 accumulator.  The
// result is within a few FP32 roundings of the FP32 network's.
//
// Layout: a layer's weights are [N][2 KP] FP32 rows, hi values in columns
// [0, KP) and lo values in [KP, 2 KP), KP = KH + KX (the h part, then the x
// part zero-padded to whole 32-value K-blocks); activations the same way,
// [rows][2 K].
//
// One cooperative launch runs the whole network: the gather of the input
// rows' planes by every thread, then the hidden layers one after the other,
// a grid-wide barrier between phases (a CTA's TMA producer waits, bounded,
// until every CTA has finished the phase its loads read).
//
// Swapped operands: the MMA's A operand is 128 neurons of W and its B
// operand up to 128 points, so a batch of 20 points costs MMAs of N = 32, not
// 128-row tiles.  A work unit is (128 points, 128 neurons, a range of
// K-blocks).  When a layer has fewer (point, neuron) tiles than the grid has
// CTAs, the K-blocks of each tile are split over several units (one per CTA
// then); each unit writes its partial tile, counts itself in at the tile's
// counter, waits (bounded) until all splits have, and finishes its share of
// the tile's columns: the partials summed in split order (the same sums
// whichever CTA takes a column), the bias, the leaky ReLU, and the hi/lo
// planes written -- or, in the last hidden layer, the one-output last layer
// in FP32 and the network's epilogue.  Without a split the unit finishes from
// tensor memory.
//
// Warp-specialised, one CTA per SM: warp 0 lane 0 loads W and point tiles by
// TMA into a 3-stage ring (64 KB a stage: hi and lo of both operands), warp 1
// lane 0 issues the MMAs into one of two TMEM accumulators, warps 2-9 (two
// per TMEM lane quadrant, one neuron per thread) run the epilogue of one unit
// while the next unit's MMAs run.  Every wait is bounded; a wait that gives
// up sets *err and the roles stop.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "epilogue.cuh"
#include "gather.cuh"
#include "pifu_internal.h"
#include "sm100.cuh"

namespace pifu {
namespace {

using namespace sm100;

constexpr int XP = kX3Tile;                         // points per unit (MMA N <= 128)
constexpr int XK = 32;                              // FP32 values per 128-byte K-block
constexpr int XNST = 3;                             // ring stages
constexpr uint32_t W_PLANE = 128 * 128;             // 128 neuron rows x 128 bytes
constexpr uint32_t P_PLANE = XP * 128;              // 128 point rows x 128 bytes
constexpr uint32_t P_BOX = 32 * 128;                // one 32-row TMA box of points
constexpr uint32_t STAGE_BYTES = 2 * W_PLANE + 2 * P_PLANE;
constexpr int kThreads = 320;                       // 2 role warps + 8 epilogue warps
constexpr uint32_t kTmemCols = 2 * XP;              // two accumulators
constexpr uint32_t kWaitLimit = 1u << 20;           // polls; legitimate waits are microseconds
constexpr uint32_t kTestWaitLimit = 1u << 12;
constexpr int kMaxSplits = 8;
constexpr uint32_t kSmemBytes = XNST * STAGE_BYTES + 1024 + 256 + 4 * XP * 4;
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(XP == 128, "one TMEM lane per neuron, 128 columns per accumulator");

// The unit decomposition of one layer, the same in every CTA.
struct Units {
    int count, n_tiles, pairs, splits, units, nk;
};

__device__ __forceinline__ Units units_of(const X3NetLayer& L, int count) {
    Units u;
    u.count = count;
    u.n_tiles = L.N / 128;
    u.pairs = ((count + XP - 1) / XP) * u.n_tiles;
    u.nk = L.nk1 + L.nk2;
    const int G = (int)gridDim.x;
    u.splits = 1;
    // split the K-blocks (at least two per split, at most kMaxSplits) while
    // tiles are fewer than CTAs; then units = pairs x splits <= G <= kX3MaxUnits
    if (u.pairs > 0 && u.pairs < G)
        u.splits = max(1, min(min(G / u.pairs, u.nk / 2), kMaxSplits));
    u.units = u.pairs * u.splits;
    return u;
}

// Unit `t`: its tile (consecutive units share the points, so the CTAs working
// at one moment read the same point rows through L2) and K range.
struct Unit {
    int pair, split, n0, p0, pcount, pn, kb0, kb1;
};

__device__ __forceinline__ Unit unit_of(const Units& us, int t) {
    Unit w;
    w.pair = t / us.splits;
    w.split = t - w.pair * us.splits;
    w.n0 = (w.pair % us.n_tiles) * 128;
    w.p0 = (w.pair / us.n_tiles) * XP;
    w.pcount = min(XP, us.count - w.p0);
    w.pn = (w.pcount + 31) / 32;
    w.kb0 = (int)((long long)w.split * us.nk / us.splits);
    w.kb1 = (int)((long long)(w.split + 1) * us.nk / us.splits);
    return w;
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Global word read with acquire semantics at GPU scope.
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* a) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// Orders this thread's view of global memory after an acquire before its
// later asynchronous-proxy (TMA) reads.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Finishes column c (point p0 + c of the unit) of this thread's neuron n from
// its accumulated sum a: bias, leaky ReLU, then the hi/lo planes of the
// output, or (FUSE) the point's contribution to the one-output last layer,
// summed over the warp's 32 neurons into sred[q][c].  c is warp-uniform.
template <bool FUSE>
__device__ __forceinline__ void finish_one(float a, int c, bool live, const Unit& w, float* out,
                                           int N, float slope, int n, float bn, float w5, int q,
                                           int lane, float* sred) {
    float h = a + bn;
    h = h >= 0.f ? h : slope * h;
    if (!FUSE) {
        if (live) {
            const float hi = tf32_round(h);
            const float lo = tf32_round(h - hi);
            float* row = out + (int64_t)(w.p0 + c) * (2 * N);
            __stcg(row + n, hi);
            __stcg(row + N + n, lo);
        }
    } else {
        const float t = warp_sum(h * w5);
        if (lane == 0) sred[q * XP + c] = t;
    }
}

// Shared-memory state of a CTA.
struct Smem {
    uint8_t* ring;
    uint64_t* full;
    uint64_t* empty;
    uint64_t* accf;               // [2] accumulator ready for the epilogue
    uint64_t* acce;               // [2] accumulator drained by the epilogue
    volatile uint32_t* sflag;     // [0] accumulator ready, [1] all splits of the tile in
    float* sred;                  // [4][XP] the last layer's quadrant sums
};

// The grid barrier's words: [p] the CTAs that have finished phase p (0: the
// gather, 1 + l: hidden layer l), one counter per phase, so that a CTA with
// no work in the later phases, which passes them at once, cannot count for an
// earlier one; [kX3MaxLayers + 1] the CTAs that have left the kernel.
__device__ __forceinline__ unsigned int* grid_bar(const X3NetArgs& a) {
    return a.ctr + 2 * kX3MaxUnits;
}

// The gather phase: hi and lo planes of the input rows of points p0 ..
// p0 + count - 1, one (point, channel quad) per item, items dealt round-robin
// over the CTAs (a batch of a few points still spreads over the whole GPU
// instead of queueing on the first CTA's threads).
__device__ __forceinline__ void gather_rows(const X3NetArgs& a, int count) {
    const uint32_t nq = (uint32_t)a.KX >> 2;
    const int64_t total = (int64_t)count * nq;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)threadIdx.x * gridDim.x + blockIdx.x; t < total; t += stride) {
        const uint32_t lp = (uint32_t)(t / nq);
        const uint32_t qd = (uint32_t)t - lp * nq;
        const PointSample ps = sample_point(a.src, a.p0 + lp, a.calib, a.map0, a.map1);
        const float4 v = sample_quad(ps, 4 * (int)qd);
        float4 hi, lo;
        hi.x = tf32_round(v.x);
        hi.y = tf32_round(v.y);
        hi.z = tf32_round(v.z);
        hi.w = tf32_round(v.w);
        lo.x = tf32_round(v.x - hi.x);
        lo.y = tf32_round(v.y - hi.y);
        lo.z = tf32_round(v.z - hi.z);
        lo.w = tf32_round(v.w - hi.w);
        float* row = a.X + (int64_t)lp * 2 * a.KX;
        *reinterpret_cast<float4*>(row + 4 * qd) = hi;
        *reinterpret_cast<float4*>(row + a.KX + 4 * qd) = lo;
    }
}

// TMA producer (one thread): per layer, once every CTA has finished the phase
// the layer reads, per unit and K-block W hi and lo (128 rows) and the
// unit's point rows in 32-row boxes, hi and lo.
__device__ bool produce(const X3NetArgs& a, const Smem& sm, int count) {
    const int G = (int)gridDim.x;
    const unsigned int* gb = grid_bar(a);
    uint32_t g = 0;
    for (int l = 0; l < a.nl; ++l) {
        const X3NetLayer& L = a.L[l];
        // every CTA has finished phase l (the gather, or hidden layer l - 1)
        uint32_t it = 0;
        while (ld_acquire(gb + l) < (unsigned int)G && ++it < kWaitLimit) {
        }
        if (it >= kWaitLimit) return false;
        fence_proxy_async_global();
        const Units us = units_of(L, count);
        for (int t = blockIdx.x; t < us.units; t += G) {
            const Unit w = unit_of(us, t);
            for (int kb = w.kb0; kb < w.kb1; ++kb, ++g) {
                const uint32_t s = g % XNST;
                const uint32_t u = g / XNST;
                if (u > 0 && !mbar_wait(&sm.empty[s], (u - 1) & 1u, kWaitLimit)) return false;
                uint8_t* st = sm.ring + s * STAGE_BYTES;
                mbar_arrive_expect_tx(&sm.full[s], 2 * W_PLANE + 2 * (uint32_t)w.pn * P_BOX);
                tma_load_2d(st, &L.tmW, kb * XK, w.n0, &sm.full[s]);
                tma_load_2d(st + W_PLANE, &L.tmW, L.KP + kb * XK, w.n0, &sm.full[s]);
                const bool from_h = kb < L.nk1;
                const CUtensorMap* mb = from_h ? &L.tmH : &a.tmX;
                const int x = from_h ? kb * XK : (kb - L.nk1) * XK;
                const int xl = x + (from_h ? L.KH : L.KX);
                for (int j = 0; j < w.pn; ++j) {
                    tma_load_2d(st + 2 * W_PLANE + j * P_BOX, mb, x, w.p0 + 32 * j, &sm.full[s]);
                    tma_load_2d(st + 2 * W_PLANE + P_PLANE + j * P_BOX, mb, xl, w.p0 + 32 * j,
                                &sm.full[s]);
                }
            }
        }
    }
    return true;
}

// MMA issuer (one thread): per K-block 4 steps of K = 8, three products each,
// into the unit's accumulator.
__device__ bool issue(const X3NetArgs& a, const Smem& sm, uint32_t tmem, int count) {
    const int G = (int)gridDim.x;
    uint32_t g = 0, i = 0;
    for (int l = 0; l < a.nl; ++l) {
        const Units us = units_of(a.L[l], count);
        for (int t = blockIdx.x; t < us.units; t += G, ++i) {
            const Unit w = unit_of(us, t);
            const uint32_t b = i & 1u, j = i >> 1;
            if (j > 0 && !mbar_wait(&sm.acce[b], (j - 1) & 1u, kWaitLimit)) return false;
            tc_fence_after();
            const uint32_t d = tmem + b * XP;
            const uint32_t idesc = idesc_tf32_f32(128, 32 * w.pn);
            bool ok = true;
            for (int kb = w.kb0; kb < w.kb1; ++kb, ++g) {
                const uint32_t s = g % XNST;
                const uint32_t u = g / XNST;
                if (!mbar_wait(&sm.full[s], u & 1u, kWaitLimit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ah = smem_u32(sm.ring + s * STAGE_BYTES);
                const uint32_t al = ah + W_PLANE;
                const uint32_t bh = ah + 2 * W_PLANE;
                const uint32_t bl = bh + P_PLANE;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t acc = (kb != w.kb0 || k != 0) ? 1u : 0u;
                    mma_tf32(d, desc_k_sw128(ah + k * 32), desc_k_sw128(bh + k * 32), idesc, acc);
                    mma_tf32(d, desc_k_sw128(ah + k * 32), desc_k_sw128(bl + k * 32), idesc, 1u);
                    mma_tf32(d, desc_k_sw128(al + k * 32), desc_k_sw128(bh + k * 32), idesc, 1u);
                }
                mma_commit(&sm.empty[s]);
            }
            mma_commit(&sm.accf[b]);   // also after an error, so the epilogue is released
            if (!ok) return false;
        }
    }
    return true;
}

// The epilogue of one unit (warps 2-9).  TMEM lane quadrant q = neurons
// 32 q .. 32 q + 31, one neuron per thread; the quadrant's two warps (half 0:
// warps 2-5, half 1: warps 6-9) take alternate groups of columns.  It runs
// once or twice per CTA and layer, from a cold instruction cache, and a TMEM
// load takes hundreds of cycles: 16 columns per load, the next group's load
// in flight while this one is finished, one short loop per path.
template <bool FUSE>
__device__ bool epi_unit(const X3NetArgs& a, const X3NetLayer& L, const Units& us, const Unit& w,
                         int t, uint32_t i, const Smem& sm, uint32_t tmem, int warp, int lane) {
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int nl = q * 32 + lane;
    const int et = (int)threadIdx.x - 64;   // 0 .. 255
    const uint32_t b = i & 1u, j = i >> 1;
    // one thread waits, the eight warps take its answer (they stay together
    // at the named barriers)
    if (et == 0) sm.sflag[0] = mbar_wait(&sm.accf[b], j & 1u, kWaitLimit) ? 1u : 0u;
    epi_bar();
    if (sm.sflag[0] == 0u) return false;
    tc_fence_after();
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + b * XP;
    const int n = w.n0 + nl;
    const float bn = L.bias[n];
    const float w5 = FUSE ? a.fl.W[nl] : 0.f;   // the last layer's weight of this neuron
    const bool direct = us.splits == 1;
    float* dst = a.part + (int64_t)t * XP * 128;   // this split's partial tile [c][nl]
    {
        const int ng = (w.pcount + 15) >> 4;   // 16-column groups: g = half, half + 2, ..
        uint32_t ra[16], rb[16];
        int g = half;
        if (g < ng) tmem_ld16(tl + (uint32_t)(16 * g), ra);
        tmem_ld_wait();
        if (direct) {
            while (g < ng) {
                const int gn = g + 2;
                if (gn < ng) tmem_ld16(tl + (uint32_t)(16 * gn), rb);
#pragma unroll
                for (int cc = 0; cc < 16; ++cc)
                    finish_one<FUSE>(__uint_as_float(ra[cc]), 16 * g + cc, 16 * g + cc < w.pcount,
                                     w, L.out, L.N, a.slope, n, bn, w5, q, lane, sm.sred);
                tmem_ld_wait();
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) ra[cc] = rb[cc];
                g = gn;
            }
        } else {
            while (g < ng) {
                const int gn = g + 2;
                if (gn < ng) tmem_ld16(tl + (uint32_t)(16 * gn), rb);
#pragma unroll
                for (int cc = 0; cc < 16; ++cc)
                    if (16 * g + cc < w.pcount)
                        __stcg(dst + (16 * g + cc) * 128 + nl, __uint_as_float(ra[cc]));
                tmem_ld_wait();
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) ra[cc] = rb[cc];
                g = gn;
            }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.acce[b]);
    }
    int cs = 0, ce = w.pcount;   // the columns this unit finishes
    if (!direct) {
        // every split of the tile finishes its own share of the columns, once
        // all the tile's partial tiles are written (one unit per CTA here, all
        // CTAs resident: the wait ends)
        __threadfence();
        epi_bar();
        if (et == 0) {
            atomicAdd(&a.ctr[w.pair], 1u);
            // wait_extra > 0 (a test): an arrival that never comes, and a
            // shorter limit
            const unsigned int need = (unsigned)us.splits + a.wait_extra;
            const uint32_t lim = a.wait_extra ? kTestWaitLimit : kWaitLimit;
            uint32_t it = 0;
            while (ld_acquire(&a.ctr[w.pair]) < need && ++it < lim) {
            }
            sm.sflag[1] = it < lim ? 1u : 0u;
        }
        epi_bar();
        if (sm.sflag[1] == 0u) return false;
        __threadfence();
        cs = (int)((long long)w.split * w.pcount / us.splits);
        ce = (int)((long long)(w.split + 1) * w.pcount / us.splits);
        const float* src = a.part + (int64_t)w.pair * us.splits * XP * 128 + nl;
        // four columns at a time (alternate fours per half), every split's value
        // loaded before the sums, which run in split order; loads from clamped
        // (valid) addresses, masked afterwards, so that no branch stands
        // between them
        for (int c = cs + 4 * half; c < ce; c += 8) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            float t2[kMaxSplits][4];
#pragma unroll
            for (int s2 = 0; s2 < kMaxSplits; ++s2)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int sc = s2 < us.splits ? s2 : 0;
                    const int cj = min(c + jj, ce - 1);
                    const float x = __ldcg(src + ((int64_t)sc * XP + cj) * 128);
                    t2[s2][jj] = (s2 < us.splits && c + jj < ce) ? x : 0.f;
                }
#pragma unroll
            for (int s2 = 0; s2 < kMaxSplits; ++s2)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) v[jj] += t2[s2][jj];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (c + jj < ce)
                    finish_one<FUSE>(v[jj], c + jj, true, w, L.out, L.N, a.slope, n, bn, w5, q,
                                     lane, sm.sred);
        }
        // the last split out resets the tile's counters for the next layer
        epi_bar();
        if (et == 0) {
            const unsigned int prev = atomicAdd(&a.ctr[kX3MaxUnits + w.pair], 1u);
            if (prev + 1u == (unsigned)us.splits) {
                a.ctr[w.pair] = 0u;
                a.ctr[kX3MaxUnits + w.pair] = 0u;
            }
        }
    }
    if (FUSE) {
        // the last layer: the four quadrants' sums per point, in order
        epi_bar();
        if (et >= cs && et < ce) {
            float tt[4] = {0.f, 0.f, 0.f, 0.f};
            for (int qq = 0; qq < 4; ++qq) tt[0] += sm.sred[qq * XP + et];
            last_epilogue(a.fl.epi, a.fl.p0 + w.p0 + et, 1, tt, a.fl.bias);
        }
    }
    epi_bar();   // sflag and sred are free for the next unit
    return true;
}

// The epilogue warps over all layers; after its last unit of a layer the CTA
// counts itself in at the grid barrier.
__device__ bool epilogue(const X3NetArgs& a, const Smem& sm, uint32_t tmem, int count, int warp,
                         int lane) {
    const int G = (int)gridDim.x;
    const int et = (int)threadIdx.x - 64;
    unsigned int* gb = grid_bar(a);
    uint32_t i = 0;
    for (int l = 0; l < a.nl; ++l) {
        const X3NetLayer& L = a.L[l];
        const bool last = l + 1 == a.nl;
        const Units us = units_of(L, count);
        for (int t = blockIdx.x; t < us.units; t += G, ++i) {
            const Unit w = unit_of(us, t);
            const bool ok = last ? epi_unit<true>(a, L, us, w, t, i, sm, tmem, warp, lane)
                                 : epi_unit<false>(a, L, us, w, t, i, sm, tmem, warp, lane);
            if (!ok) return false;
        }
        // the layer's generic stores are read by other CTAs' TMA loads: a
        // proxy fence by each writing thread, then the release
        fence_proxy_async_global();
        __threadfence();
        epi_bar();
        if (et == 0) atomicAdd(gb + 1 + l, 1u);
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 1) x3_net_kernel(const __grid_constant__ X3NetArgs a) {
    extern __shared__ uint8_t smem_raw[];
    Smem sm;
    sm.ring = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    sm.full = reinterpret_cast<uint64_t*>(sm.ring + XNST * STAGE_BYTES);
    sm.empty = sm.full + XNST;
    sm.accf = sm.empty + XNST;
    sm.acce = sm.accf + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm.acce + 2);
    sm.sflag = tslot + 1;
    sm.sred = reinterpret_cast<float*>(sm.ring + XNST * STAGE_BYTES + 256);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < XNST; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm.accf[b], 1);
            mbar_init(&sm.acce[b], 8);   // one arrival per epilogue warp
        }
        fence_mbar_init();
        prefetch_tmap(&a.tmX);
        for (int l = 0; l < a.nl; ++l) {
            prefetch_tmap(&a.L[l].tmW);
            if (a.L[l].nk1 > 0) prefetch_tmap(&a.L[l].tmH);
        }
    }
    if (warp == 1) tmem_alloc(tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    int count = a.M;
    if (a.m_dev) count = min(count, (int)*a.m_dev);
    count = max(count, 0);

    // phase 0: the input rows' planes, by every thread of the grid
    gather_rows(a, count);
    fence_proxy_async_global();   // the planes are read by TMA (the async proxy)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(grid_bar(a), 1u);

    bool ok = true;
    if (warp == 0) {
        if (lane == 0) ok = produce(a, sm, count);
    } else if (warp == 1) {
        if (lane == 0) ok = issue(a, sm, tmem, count);
    } else {
        ok = epilogue(a, sm, tmem, count, warp, lane);
    }
    if (!ok) atomicOr(a.err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
    if (threadIdx.x == 0) {
        // every CTA has passed every phase once it leaves: the last one out
        // zeroes the grid barrier for the next launch
        unsigned int* gb = grid_bar(a);
        const unsigned int prev = atomicAdd(gb + kX3MaxLayers + 1, 1u);
        if (prev + 1u == gridDim.x)
            for (int k = 0; k <= kX3MaxLayers + 1; ++k) gb[k] = 0u;
    }
}

bool g_attr_set[64] = {};
int g_n_sm[64] = {};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// One CTA per SM must fit (the cooperative launch needs the whole grid resident).
cudaError_t ensure_attr(int dev, int* sms) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(x3_net_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        int per_sm = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, x3_net_kernel, kThreads,
                                                              kSmemBytes);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorCooperativeLaunchTooLarge;
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&g_n_sm[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_attr_set[dev] = true;
    }
    *sms = g_n_sm[dev];
    return cudaSuccess;
}

}  // namespace

bool x3_encode_2d(void* map, const void* base, uint64_t cols, uint64_t rows,
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
    return g_encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t x3_prepare() {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = ensure_attr(dev, &sms);
    return e;
}

cudaError_t launch_x3_net(const X3NetArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    if (a.nl < 1 || a.nl > kX3MaxLayers || a.KX <= 0 || a.KX % XK != 0 || !a.X || !a.part ||
        !a.ctr || !a.err || a.fl.n_out != 1 || !a.fl.W || a.L[a.nl - 1].N != 128)
        return cudaErrorInvalidValue;
    for (int l = 0; l < a.nl; ++l) {
        const X3NetLayer& L = a.L[l];
        if (L.N <= 0 || L.N % 128 != 0 || L.KH % XK != 0 || L.KX % XK != 0 ||
            L.KP != L.KH + L.KX || L.nk1 * XK != L.KH || L.nk2 * XK != L.KX ||
            L.nk1 + L.nk2 < 1 || (L.nk2 > 0 && L.KX != a.KX) || !L.bias ||
            (l + 1 < a.nl && !L.out) || (l == 0 && L.nk1 != 0) ||
            (l > 0 && L.KH != a.L[l - 1].N))
            return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = ensure_attr(dev, &sms);
    if (e != cudaSuccess) return e;
    // one CTA per SM (the ring takes 192 KB), all resident (the grid barrier);
    // at most kX3MaxUnits, which bounds the split-K partial tiles
    const int grid = sms < kX3MaxUnits ? sms : kX3MaxUnits;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, x3_net_kernel, a);
}

}  // namespace pifu
