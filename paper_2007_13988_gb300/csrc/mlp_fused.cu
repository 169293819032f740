// The whole network in FP32 (Eq. 1 / Eq. 2: gather, hidden layers with the
// input re-concatenated where the network has skips, last layer and its
// activation) for a small point batch in ONE launch.  This is the
// re-evaluation of the mixed-precision forms and the FP32 pass of batches too
// small to fill the GPU, where the chain gather -> one GEMM per layer -> last
// layer would be ten dependent launches of a few microseconds of work each.
//
// Work split: a cluster of CL CTAs owns a tile of kFP points, CL = 16, 8, 4
// or 2 (16 is a non-portable size).  Larger clusters split each layer's
// neurons finer, so one tile finishes sooner; smaller ones fit more clusters
// on the GPU at once (2-CTA clusters: 76 tiles per round instead of 15), so a
// batch of many tiles takes fewer rounds.  The host picks the size with the
// fewest latency-weighted rounds (fused_pick; in a graph, a switch node set
// on the device from the batch size picks among launches of each).  Every CTA
// assembles the tile's input rows itself (projection + bilinear sample, the
// same device code as the gather kernel), then for each hidden layer computes
// its 1/CL share of the output neurons for all kFP points and stores that
// slice into every CTA's copy of the layer output through distributed shared
// memory; one cluster barrier per layer publishes it.  The weights are read
// once per tile per cluster (each CTA reads its own rows), from L2.
//
// Inside a CTA, thread t owns two neurons (g and g + S/2 of the CTA's S) and
// one of KS interleaved K-splits; it keeps kFP x 2 accumulators, reads each
// weight quad once (16-byte load) and the input quads of the kFP points from
// shared memory (the same address across the warp: broadcast).  The K-split
// partial sums meet in shared memory, in a fixed order (deterministic).
//
// Shape rules (checked on the host, fused_ok): hidden widths n_out with
// n_out / CL a power of two in [8, 512]; K1, K2, ldw multiples of 4; at
// most 4 outputs in the last layer; 16-byte aligned weights and biases.
//
// No waits other than the hardware cluster barrier, which every CTA of a
// cluster reaches the same number of times (all CTAs of a cluster walk the
// same tiles and layers).
#include <cooperative_groups.h>

#include <algorithm>

#include "epilogue.cuh"
#include "gather.cuh"
#include "sm100.cuh"

namespace cg = cooperative_groups;

namespace pifu {
namespace {

constexpr int kFP = kFusedTilePoints;   // points per cluster tile (16)
constexpr int kCL = 8;      // CTAs per cluster for a device-resident batch size
constexpr int kFT = 256;    // threads per CTA
constexpr int kNW = kFT / 32;
constexpr int kNJ = 8;      // neurons per warp task
constexpr int kAcc = kFP * kNJ;
constexpr int kMaxLdx = 528;
constexpr int kMaxHidden = 1024;
constexpr int kMaxLast = 4096;   // floats of the last layer's weights kept in shared memory

// K-split partial sums: max(kFP * S, kNW * kNJ * kFP) floats, S <= kMaxHidden / CL
template <int CL>
__host__ __device__ constexpr int red_floats() {
    return kFP * (kMaxHidden / CL) > kNW * kNJ * kFP ? kFP * (kMaxHidden / CL) : kNW * kNJ * kFP;
}
template <int CL>
__host__ __device__ constexpr size_t smem_bytes() {
    return (size_t)(kFP * kMaxLdx + 2 * kFP * kMaxHidden + red_floats<CL>() + kMaxLast) * 4;
}
static_assert(smem_bytes<2>() <= 227 * 1024, "shared memory of the 2-CTA form");

__device__ __forceinline__ float lrelu(float v, float s) { return v >= 0.f ? v : s * v; }

__device__ __forceinline__ float warp_sum32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float4 lds4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
}

__device__ __forceinline__ void load_wq(float4 (&w)[kNJ], const float* __restrict__ wrow,
                                        int ldw, int kq, int Kq) {
#pragma unroll
    for (int j = 0; j < kNJ; ++j)
        w[j] = kq < Kq ? ld4(wrow + (int64_t)j * ldw + 4 * kq) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// One hidden layer of the tile: this CTA's S = n_out / CL neurons, stored
// into every CTA's `out` ([kFP][n_out]), then a cluster barrier.
//
// A warp task is kNJ consecutive neurons over one of KW interleaved K-splits;
// lane l takes the K quads l, l + 32 KW, ... so that the 32 lanes read 512
// contiguous bytes of each weight row (coalesced) and 32 consecutive input
// quads of each point (conflict-free).  The next quad's weights are loaded
// before the current quad's arithmetic.  The kFP x kNJ accumulators are then
// summed over the lanes by recursive halving (each step exchanges half of the
// values), which leaves lane l the sums of point l/2, neurons 4 (l & 1) ..
// + 3; K-splits meet in shared memory in a fixed order.
template <int CL>
__device__ __forceinline__ void fused_layer(const FusedLayer& Ly, float slope,
                                            const float* __restrict__ in,
                                            const float* __restrict__ xs, int ldx, int d_in,
                                            float* out, float* __restrict__ red, unsigned rank,
                                            cg::cluster_group& cl) {
    const int S = Ly.n_out / CL;
    const int groups = S / kNJ;
    const int KW = groups >= kNW ? 1 : kNW / groups;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // whole quads of real columns; the x segment's last d_in % 4 columns
    // (quad Kq) are added one by one, and its padding to ldx not at all
    const int Kq = (Ly.K1 + (Ly.K2 > 0 ? (d_in & ~3) : 0)) >> 2;
    const int tail = Ly.K2 > 0 ? (d_in & 3) : 0;
    const int pitch = kFP * S;
    for (int task = warp; task < groups * KW; task += kNW) {
        const int g = task % groups;
        const int ksw = task / groups;
        const float* __restrict__ wrow = Ly.W + (int64_t)((int)rank * S + g * kNJ) * Ly.ldw;
        float acc[kAcc];
#pragma unroll
        for (int i = 0; i < kAcc; ++i) acc[i] = 0.f;
        int kq = lane + 32 * ksw;
        float4 w[kNJ];
        load_wq(w, wrow, Ly.ldw, kq, Kq);
        for (; kq < Kq; kq += 32 * KW) {
            float4 wn[kNJ];
            load_wq(wn, wrow, Ly.ldw, kq + 32 * KW, Kq);
            const int k = 4 * kq;
            const bool from_h = k < Ly.K1;
            const float* base = from_h ? in + k : xs + (k - Ly.K1);
            const int ld = from_h ? Ly.K1 : ldx;
#pragma unroll
            for (int p = 0; p < kFP; ++p) {
                const float4 x = lds4(base + p * ld);
#pragma unroll
                for (int j = 0; j < kNJ; ++j)
                    acc[p * kNJ + j] = fmaf(x.w, w[j].w, fmaf(x.z, w[j].z,
                                       fmaf(x.y, w[j].y, fmaf(x.x, w[j].x, acc[p * kNJ + j]))));
            }
#pragma unroll
            for (int j = 0; j < kNJ; ++j) w[j] = wn[j];
        }
        if (tail && lane == (Kq & 31) && ksw == (Kq >> 5) % KW) {
            // the lane whose turn quad Kq is (the order of the 4-wide loop)
            const int k = 4 * Kq;
            for (int e = 0; e < tail; ++e) {
                float wv[kNJ];
#pragma unroll
                for (int j = 0; j < kNJ; ++j) wv[j] = __ldg(wrow + (int64_t)j * Ly.ldw + k + e);
#pragma unroll
                for (int p = 0; p < kFP; ++p) {
                    const float x = xs[p * ldx + (k - Ly.K1) + e];
#pragma unroll
                    for (int j = 0; j < kNJ; ++j) acc[p * kNJ + j] = fmaf(x, wv[j], acc[p * kNJ + j]);
                }
            }
        }
        // sum over the lanes: value v = p * kNJ + j ends in lane v / 4
#pragma unroll
        for (int h = kAcc / 2, off = 16; h >= 4; h >>= 1, off >>= 1) {
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float send = upper ? acc[i] : acc[i + h];
                const float keep = upper ? acc[i + h] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
        const int p = lane >> 1;
        *reinterpret_cast<float4*>(red + ksw * pitch + p * S + g * kNJ + 4 * (lane & 1)) =
            make_float4(acc[0], acc[1], acc[2], acc[3]);
    }
    __syncthreads();
    const int S4 = S >> 2;
    for (int o = threadIdx.x; o < kFP * S4; o += kFT) {
        const int p = o / S4;
        const int j = (o - p * S4) * 4;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < KW; ++q) {
            const float4 r = lds4(red + q * pitch + p * S + j);
            s.x += r.x;
            s.y += r.y;
            s.z += r.z;
            s.w += r.w;
        }
        const float4 b = ld4(Ly.b + (int)rank * S + j);
        s.x = lrelu(s.x + b.x, slope);
        s.y = lrelu(s.y + b.y, slope);
        s.z = lrelu(s.z + b.z, slope);
        s.w = lrelu(s.w + b.w, slope);
        float* dst = out + p * Ly.n_out + (int)rank * S + j;
#pragma unroll
        for (int r = 0; r < CL; ++r)
            *reinterpret_cast<float4*>(cl.map_shared_rank(dst, (unsigned)r)) = s;
    }
    cl.sync();
}

// Launched with a cluster dimension of CL (launch attribute).
template <int CL>
__global__ void __launch_bounds__(kFT, 1)
    mlp_fused_kernel(FusedNet net, PointSrc src, int64_t p0, int64_t m, Calib calib, Map map0,
                     Map map1, Epilogue epi) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    const int64_t cid = blockIdx.x / CL;
    const int64_t ncl = gridDim.x / CL;
    extern __shared__ float4 smem4[];
    float* xs = reinterpret_cast<float*>(smem4);   // [kFP][ldx]
    float* hb0 = xs + kFP * net.ldx;               // [kFP][<= max_hidden]
    float* hb1 = hb0 + kFP * net.max_hidden;
    float* red = hb1 + kFP * net.max_hidden;       // [red_floats<CL>()]
    float* wl = red + red_floats<CL>();            // last layer's weights [n_out][ldw]
    const FusedLayer& Ll = net.L[net.nl - 1];
    for (int e = threadIdx.x; e < Ll.n_out * Ll.ldw; e += kFT) wl[e] = Ll.W[e];
    __syncthreads();
    if (src.count) m = min(m, (int64_t)*src.count);
    const int nq = net.ldx >> 2;
    const int64_t ntiles = (m + kFP - 1) / kFP;
    constexpr int kPerRank = kFP / CL;   // points each CTA gathers
    for (int64_t tile = cid; tile < ntiles; tile += ncl) {
        const int64_t t0 = tile * kFP;
        const int np = (int)(m - t0 < kFP ? m - t0 : kFP);
        // input rows: CTA `rank` assembles points rank, rank + CL, ... and
        // stores them into every CTA's copy
        for (int e = threadIdx.x; e < kPerRank * nq; e += kFT) {
            const int i = e / nq;
            const int c = (e - i * nq) * 4;
            const int p = (int)rank + CL * i;
            const float4 r = p < np ? gather_quad(src, p0 + t0 + p, calib, map0, map1, c)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            float* dst = xs + p * net.ldx + c;
#pragma unroll
            for (int q = 0; q < CL; ++q)
                *reinterpret_cast<float4*>(cl.map_shared_rank(dst, (unsigned)q)) = r;
        }
        cl.sync();
        const float* in = nullptr;
        for (int l = 0; l + 1 < net.nl; ++l) {
            float* out = (l & 1) ? hb1 : hb0;
            fused_layer<CL>(net.L[l], net.slope, in, xs, net.ldx, net.d_in, out, red, rank, cl);
            in = out;
        }
        // last layer and epilogue: CTA `rank` takes points rank, rank + CL, ...
        {
            const int K = Ll.K1 + Ll.K2;
            const int lane = threadIdx.x & 31;
            const int w = threadIdx.x >> 5;
            const int p = (int)rank + CL * w;
            if (w < kPerRank && p < np) {
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                for (int k = lane; k < K; k += 32) {
                    const float a = k < Ll.K1 ? in[p * Ll.K1 + k] : xs[p * net.ldx + (k - Ll.K1)];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (j < Ll.n_out) acc[j] = fmaf(a, wl[j * Ll.ldw + k], acc[j]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = warp_sum32(acc[j]);
                if (lane == 0) last_epilogue(epi, p0 + t0 + p, Ll.n_out, acc, Ll.b);
            }
        }
        cl.sync();   // buffers are reused by the next tile
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int CL>
int max_clusters() {
    static int cached = -1;
    if (cached >= 0) return cached;
    if (cudaFuncSetAttribute(mlp_fused_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<CL>()) != cudaSuccess)
        return cached = 0;
    if (CL > 8 && cudaFuncSetAttribute(mlp_fused_kernel<CL>,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed,
                                       1) != cudaSuccess) {
        (void)cudaGetLastError();
        return cached = 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kFT);
    cfg.dynamicSmemBytes = smem_bytes<CL>();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, mlp_fused_kernel<CL>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
    }
    return cached = n;
}

template <int CL>
cudaError_t launch_cl(const FusedNet& net, const PointSrc& src, int64_t p0, int64_t m,
                      const Calib& calib, const Map& map0, const Map& map1, const Epilogue& epi,
                      int64_t grid_cl, cudaStream_t stream) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(grid_cl * CL));
    cfg.blockDim = dim3(kFT);
    cfg.dynamicSmemBytes = smem_bytes<CL>();
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mlp_fused_kernel<CL>, net, src, p0, m, calib, map0, map1, epi);
}

// Every hidden width splits into CL slices of a power-of-two number (at least
// kNJ) of neurons.
bool cl_ok(const FusedNet& n, int CL) {
    for (int l = 0; l + 1 < n.nl; ++l) {
        const int S = n.L[l].n_out / CL;
        if (n.L[l].n_out % CL || S < kNJ || (S & (S - 1))) return false;
    }
    return true;
}

}  // namespace

bool fused_ok(const FusedNet& n) {
    if (n.nl < 1 || n.nl > kFusedMaxLayers || n.ldx % 4 || n.ldx > kMaxLdx ||
        n.max_hidden > kMaxHidden || n.max_hidden % 4)
        return false;
    for (int l = 0; l < n.nl; ++l) {
        const FusedLayer& L = n.L[l];
        if (L.K1 % 4 || L.K2 % 4 || L.ldw % 4 || L.ldw < L.K1 + L.K2 || !L.W || !L.b)
            return false;
        if (L.K2 != 0 && L.K2 != n.ldx) return false;
        if (l > 0 && L.K1 != n.L[l - 1].n_out) return false;
        if (l == 0 && L.K1 != 0) return false;
        if (!aligned16(L.W) || !aligned16(L.b)) return false;
        if (l + 1 < n.nl) {
            const int S = L.n_out / kCL;
            if (L.n_out % kCL || S < kNJ || S > 256 || (S & (S - 1)) || L.n_out > n.max_hidden)
                return false;
        } else if (L.n_out < 1 || L.n_out > 4 || L.n_out * L.ldw > kMaxLast) {
            return false;
        }
    }
    return true;
}

namespace {

// Latency of one tile relative to 8-CTA clusters (full-size f_O, GB300: one
// round of 16-, 8-, 4- and 2-CTA clusters took 32, 36, 60 and 106 us).
constexpr int kClSizes[4] = {16, 8, 4, 2};
constexpr float kClLatency[4] = {0.88f, 1.f, 1.67f, 2.94f};

int clusters_of(int CL) {
    switch (CL) {
        case 16: return max_clusters<16>();
        case 8: return max_clusters<8>();
        case 4: return max_clusters<4>();
        case 2: return max_clusters<2>();
        default: return 0;
    }
}

// fused_pick, fused_index and batch_index: switch_index.cuh.
__global__ void fused_switch_kernel(cudaGraphConditionalHandle h, FusedPlan plan,
                                    const unsigned int* count, unsigned int cap, unsigned int x3_lo,
                                    unsigned int x3_hi, unsigned int grid_hi,
                                    unsigned long long* stat, unsigned int stat_cap,
                                    unsigned int* err) {
    sm100::griddep_wait();   // a programmatic dependent of the pass that fills the queue
    const unsigned int v = *count;
    if (stat) {
        *stat += v;
        if (v > stat_cap) atomicOr(err, kErrCapacity);
    }
    cudaGraphSetConditional(h, fused_index(plan, min(v, cap), x3_lo, x3_hi, grid_hi));
}

// One batch of the MIXED forms in the graph as one SWITCH: bodies 0 .. nt-1
// evaluate a batch of 1 .. threshold points in FP32 (single: body 0 alone,
// else fused_switch_kernel's choice among them), body nt takes a larger
// batch to the tensor cores, and an empty batch runs no body.  has_rs: the
// batch is a conflict round, whose size is first moved from the frontier
// count, with round_start_kernel's statistics and zeroing.
__global__ void batch_switch_kernel(cudaGraphConditionalHandle h, FusedPlan plan,
                                    unsigned int* count, unsigned int cap,
                                    unsigned int threshold, int nt, int single,
                                    unsigned int x3_lo, unsigned int x3_hi, unsigned int grid_hi,
                                    RoundStart rs, int has_rs, unsigned int* zero) {
    if (zero) *zero = 0u;
    unsigned int c;
    if (has_rs) {
        c = *rs.next;
        *count = c;
        *rs.next = 0u;
        *rs.evals += c;
        if (c > rs.cap) atomicOr(rs.err, kErrCapacity);
        *rs.zero = 0u;
    } else {
        c = *count;
    }
    cudaGraphSetConditional(h, batch_index(plan, c, cap, threshold, nt, single != 0, x3_lo, x3_hi,
                                           grid_hi));
}

}  // namespace

FusedPlan fused_plan(const FusedNet& net) {
    FusedPlan p;
    for (int i = 0; i < 4; ++i) {
        const int CL = kClSizes[i];
        const int n = cl_ok(net, CL) ? clusters_of(CL) : 0;
        if (n <= 0) continue;
        p.cl[p.n] = CL;
        p.ncl[p.n] = n;
        p.lat[p.n] = kClLatency[i];
        ++p.n;
    }
    return p;
}

cudaError_t launch_fused_switch(cudaGraphConditionalHandle h, const FusedPlan& plan,
                                const unsigned int* count, unsigned int cap, cudaStream_t stream,
                                unsigned int x3_lo, unsigned int x3_hi, unsigned int grid_hi,
                                unsigned long long* stat, unsigned int stat_cap,
                                unsigned int* err) {
    return launch_pdl(fused_switch_kernel, dim3(1), dim3(1), 0, stream, h, plan, count, cap, x3_lo,
                      x3_hi, grid_hi, stat, stat_cap, err);
}

cudaError_t launch_batch_switch(cudaGraphConditionalHandle h, const FusedPlan& plan,
                                unsigned int* count, unsigned int cap, unsigned int threshold,
                                int nt, bool single, unsigned int x3_lo, unsigned int x3_hi,
                                unsigned int grid_hi, const RoundStart* rs, unsigned int* zero,
                                cudaStream_t stream) {
    batch_switch_kernel<<<1, 1, 0, stream>>>(h, plan, count, cap, threshold, nt, single ? 1 : 0,
                                             x3_lo, x3_hi, grid_hi, rs ? *rs : RoundStart{},
                                             rs ? 1 : 0, zero);
    return cudaGetLastError();
}

cudaError_t launch_mlp_fused(const FusedNet& net, const PointSrc& src, int64_t p0, int64_t m,
                             const Calib& calib, const Map& map0, const Map& map1,
                             const Epilogue& epi, cudaStream_t stream, int cl) {
    if (m <= 0) return cudaSuccess;
    const int64_t tiles = (m + kFP - 1) / kFP;
    if (cl == 0) {
        if (src.count) {
            cl = kCL;
        } else {
            const FusedPlan p = fused_plan(net);
            if (p.n == 0) return cudaErrorInvalidConfiguration;
            cl = p.cl[fused_pick(p, tiles)];
        }
    }
    const int ncl = cl_ok(net, cl) ? clusters_of(cl) : 0;
    if (ncl <= 0) return cudaErrorInvalidConfiguration;
    // a device-resident count gets every co-resident cluster (persistent loop)
    const int64_t grid_cl = src.count ? ncl : std::min<int64_t>(tiles, ncl);
    cudaError_t e = cudaErrorInvalidValue;
    switch (cl) {
        case 16: e = launch_cl<16>(net, src, p0, m, calib, map0, map1, epi, grid_cl, stream); break;
        case 8: e = launch_cl<8>(net, src, p0, m, calib, map0, map1, epi, grid_cl, stream); break;
        case 4: e = launch_cl<4>(net, src, p0, m, calib, map0, map1, epi, grid_cl, stream); break;
        case 2: e = launch_cl<2>(net, src, p0, m, calib, map0, map1, epi, grid_cl, stream); break;
        default: break;
    }
    return e;
}

}  // namespace pifu
