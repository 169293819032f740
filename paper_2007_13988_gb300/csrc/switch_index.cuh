// Which body of the graph's switch nodes a device-resident batch takes, as
// plain functions that compile for the device and for the host (the CPU
// tests check the routing on this same code).
//
// A batch of the MIXED forms' FP32-accurate passes (a re-check queue, or a
// conflict round of at most `threshold` points) has up to three kinds of
// body: the fused cluster network at each usable cluster size (plan.n
// bodies, indices 0 .. plan.n-1), then the split-TF32 network (x3_hi > 0),
// then the whole-GPU network (grid_hi > 0).  A conflict round's switch has
// one body more, the tensor-core pass for batches above `threshold`.  An
// index past the last body runs nothing.
#pragma once

#if defined(__CUDACC__)
#define PIFU_HD __host__ __device__ __forceinline__
#else
#define PIFU_HD inline
#endif

namespace pifu {

constexpr int kFusedTilePoints = 16;   // points per cluster tile of the fused network

// The cluster sizes the fused kernel can use for a network, with the number
// of clusters of each size that fit on the device at once and the latency of
// one tile relative to 8-CTA clusters.
struct FusedPlan {
    int n = 0;
    int cl[4] = {};
    int ncl[4] = {};
    float lat[4] = {};
};

// Index in `p` of the size with the fewest latency-weighted rounds for
// `tiles` tiles; ties go to the larger clusters (lower latency).
PIFU_HD int fused_pick(const FusedPlan& p, long long tiles) {
    int best = 0;
    float best_cost = 3.0e38f;
    for (int i = 0; i < p.n; ++i) {
        const long long rounds = (tiles + p.ncl[i] - 1) / p.ncl[i];
        const float cost = (float)rounds * p.lat[i];
        if (cost < best_cost * 0.999f) {
            best_cost = cost;
            best = i;
        }
    }
    return best;
}

// The re-check switch's body for a queue of c points: the whole-GPU network
// up to grid_hi points, else split TF32 for x3_lo < c <= x3_hi, else the
// cluster size fused_pick chooses; nothing for an empty queue.
PIFU_HD unsigned int fused_index(const FusedPlan& plan, unsigned int c, unsigned int x3_lo,
                                 unsigned int x3_hi, unsigned int grid_hi) {
    const unsigned int x3_idx = (unsigned)plan.n;
    const unsigned int grid_idx = x3_idx + (x3_hi > 0u ? 1u : 0u);
    if (c == 0u) return grid_idx + (grid_hi > 0u ? 1u : 0u);
    if (c <= grid_hi) return grid_idx;
    if (c > x3_lo && c <= x3_hi) return x3_idx;
    return (unsigned)fused_pick(plan, ((long long)c + kFusedTilePoints - 1) / kFusedTilePoints);
}

// A conflict round's (or small batch's) switch of nt + 1 bodies: c points,
// 1 <= c <= threshold, take an FP32 body (body 0 when single, else
// fused_index for min(c, cap)); c > threshold takes body nt (the
// tensor-core pass); an empty batch nothing.
PIFU_HD unsigned int batch_index(const FusedPlan& plan, unsigned int c, unsigned int cap,
                                 unsigned int threshold, int nt, bool single, unsigned int x3_lo,
                                 unsigned int x3_hi, unsigned int grid_hi) {
    if (c == 0u) return (unsigned)nt + 1u;
    if (c > threshold) return (unsigned)nt;
    if (single) return 0u;
    return fused_index(plan, c < cap ? c : cap, x3_lo, x3_hi, grid_hi);
}

}  // namespace pifu
