// The whole network in FP32 (Eq. 1 / Eq. 2: the input rows, the hidden layers
// with the input re-concatenated where the network has skips, the last layer
// and its activation) for a batch of up to a few dozen points (at most 128
// for the 257-1024-512-256-128-1 network), in ONE cooperative launch over
// every SM.  These are the FP32-accurate passes of the MIXED forms: the
// re-evaluation of occupancies that the BF16 pass put near Sec. 3.2's
// threshold, and the conflict rounds' small batches.  On a few SMs such a
// pass is bound by streaming the FP32 weights (4.7 MB for that network) and
// by those SMs' FFMA rate; spread over the whole GPU, each SM holds a small
// slice of every layer and what is left is the sequence of layers.
//
// Work split: the batch's m points form P point groups of Pt = ceil(m / P)
// points, every hidden layer's neurons Q = G / P neuron groups (G CTAs, one
// per SM); CTA c < P Q takes point group c % P and neuron group c / P.  P is
// chosen from m, the same way in every CTA, among the splits whose shared
// memory fits, by a cost model of the bytes a CTA stages after each barrier
// and the FFMAs it runs.
//
// Per CTA: the input rows of its points (projection and bilinear sample, the
// gather's device code) into shared memory; per hidden layer, its neurons'
// weight rows by one bulk copy, issued before the barrier that precedes the
// layer (weights do not depend on it), and after that barrier the previous
// layer's rows of its points, loaded from L2 by every thread; the (point,
// neuron) tile in FP32 FFMA from shared memory; bias and leaky ReLU; the tile
// stored to global memory; then one thread releases the CTA's stores and
// counts the CTA in at the layer's grid barrier.  The last
// hidden layer's tile stays in the CTA: its contribution to the last layer
// (at most 4 outputs) is written as one partial sum per (point, neuron
// group), and the CTA that arrives last at its point group's counter sums the
// partials in neuron-group order, adds the last layer's x segment and runs
// the network's epilogue (nobody waits there: the last arrival does it).
//
// Inside a CTA a warp task is a 4-point x 4-neuron register tile over one of
// KS interleaved K-splits (KS > 1 while tasks are fewer than warps): lane l
// reads K quads l, l + 32 KS, ... of the 4 input rows and the 4 weight rows
// (16-byte shared loads, consecutive across the warp), the 16 sums are
// reduced over the lanes by recursive halving, and the K-splits meet in
// shared memory.  Every sum is taken in a fixed order, so results do not
// depend on timing.
//
// Waits: the grid barrier (polls of a global counter) and the bulk copies'
// mbarriers, all bounded.  A wait that gives up sets kErrTimeout; the CTA
// then waits (bounded) for its own copies in flight and leaves, and the host
// zeroes the counters when it reads the error.
#include "epilogue.cuh"
#include "gather.cuh"
#include "pifu_internal.h"
#include "sm100.cuh"

namespace pifu {
namespace {

using namespace sm100;

constexpr int kGT = 512;                     // threads per CTA
constexpr int kGW = kGT / 32;                // warps per CTA
constexpr int RP = 4;                        // points per register tile
constexpr int RN = 4;                        // neurons per register tile
constexpr uint32_t kGridSmem = 227 * 1024;   // dynamic shared memory per CTA (the most an SM gives one)
constexpr uint32_t kHdr = 64;                // mbarriers and split before the float regions
constexpr uint32_t kWaitLimit = 1u << 20;    // polls; legitimate waits are microseconds
constexpr uint32_t kTestWaitLimit = 1u << 12;

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int up_to(int v, int r) { return (v + r - 1) / r * r; }

// Rows of a neuron group of a layer of N neurons split over Q groups (the
// widest group), rounded up to the register tile.
__host__ __device__ __forceinline__ int group_rows(int N, int Q) {
    return up_to((N + Q - 1) / Q, RN);
}

// Neurons [n0, n1) of group g of Q.
__host__ __device__ __forceinline__ void group_range(int N, int Q, int g, int& n0, int& n1) {
    n0 = (int)((long long)g * N / Q);
    n1 = (int)((long long)(g + 1) * N / Q);
}

struct Split {
    int P, Q, Pt;
};

// Float offsets of the shared-memory regions for point groups of Pt points
// and Q neuron groups: input rows, previous-layer rows, this layer's weight
// rows, the last layer's weights, biases (this layer's, then the last
// layer's), K-split sums, the last hidden layer's tile.
struct Layout {
    int xs, hs, ws, wl, bs, bl, red, hb, total;
};

__host__ __device__ inline Layout layout_of(const FusedNet& n, int Pt, int Q) {
    const int Ptr = up_to(Pt, RP);
    int k1 = 0, w = 0, red = 0, nb = 0;
    for (int l = 0; l + 1 < n.nl; ++l) {
        const FusedLayer& L = n.L[l];
        const int nr = group_rows(L.n_out, Q);
        if (l > 0) k1 = imax(k1, L.K1);
        w = imax(w, nr * L.ldw);
        nb = imax(nb, nr);
        const int tasks = (Ptr / RP) * (nr / RN);
        red = imax(red, imax(tasks, kGW) * RP * RN);
    }
    const FusedLayer& Lo = n.L[n.nl - 1];
    Layout s;
    s.xs = 0;
    s.hs = s.xs + Ptr * n.ldx;
    s.ws = s.hs + Ptr * k1;
    s.wl = s.ws + w;
    s.bs = s.wl + up_to(Lo.n_out * Lo.ldw, 4);
    s.bl = s.bs + up_to(nb, 4);
    s.red = s.bl + 4;
    s.hb = s.red + red;
    s.total = s.hb + Ptr * group_rows(n.L[n.nl - 2].n_out, Q);
    return s;
}

__host__ __device__ inline bool fits(const FusedNet& n, int Pt, int Q) {
    return kHdr + 4u * (uint32_t)layout_of(n, Pt, Q).total <= kGridSmem;
}

// The estimated time of splitting m points over G CTAs into P point groups,
// if that split fits: per hidden layer, the bytes a CTA stages after the
// barrier (its points' previous-layer rows, about 150 B/ns per SM from L2)
// and its FFMAs (about 100 per ns per SM); for the input rows, 16 B of taps
// per channel and point.
__host__ __device__ inline bool split_cost(const FusedNet& n, int m, int G, int P, float& cost) {
    const int Pt = (m + P - 1) / P;
    const int Q = G / P;
    if (Q < 1 || !fits(n, Pt, Q)) return false;
    const float Ptr = (float)up_to(Pt, RP);
    cost = Ptr * (float)n.ldx * (16.0f / 150.0f);
    for (int l = 0; l + 1 < n.nl; ++l) {
        const FusedLayer& L = n.L[l];
        cost += Ptr * (float)L.K1 * (4.0f / 150.0f) +
                Ptr * (float)group_rows(L.n_out, Q) * (float)L.ldw * 0.01f;
    }
    return true;
}

__host__ __device__ inline int max_groups(int m, int G) { return imin(imin(m, G), kGridMaxGroups); }

// The split of lowest estimated time (ties: fewer groups); P = 0: none fits.
__host__ inline Split split_of(const FusedNet& n, int m, int G) {
    Split best{0, 0, 0};
    float best_cost = 3.0e38f;
    for (int P = 1; P <= max_groups(m, G); ++P) {
        float c;
        if (split_cost(n, m, G, P, c) && c < best_cost) {
            best_cost = c;
            best = Split{P, G / P, (m + P - 1) / P};
        }
    }
    return best;
}

// Shared-memory header.
struct Hdr {
    uint64_t mbW;        // weight rows of the current layer (and, first, the last layer's)
    int P, Q, Pt;
    unsigned int flag;   // a wait gave up
    unsigned int fin;    // this CTA finishes its point group
};
static_assert(sizeof(Hdr) <= kHdr, "header");

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* a) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// *a += v with release semantics at GPU scope (the CTA's earlier stores,
// ordered before this thread by a CTA barrier, become visible first).
__device__ __forceinline__ void red_release(unsigned int* a, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* a, unsigned int v) {
    unsigned int r;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(a), "r"(v)
                 : "memory");
    return r;
}

// Polls *w until it reaches `need`, at most `limit` times.
__device__ __forceinline__ bool grid_wait(const unsigned int* w, unsigned int need,
                                          uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (ld_acquire(w) >= need) return true;
    return false;
}

__device__ __forceinline__ float lrelu(float v, float s) { return v >= 0.f ? v : s * v; }

__device__ __forceinline__ float4 lds4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The (point, neuron) tile of one hidden layer: rows [0, Pr) of the inputs
// (Hs: the previous layer's K1 columns, Xs: the ldx input columns) against
// rows [0, Nr) of Ws ([Nr][ldw], the h columns then the x columns), sums
// into red[KS][Pr][Nr].  Rows past the CTA's points or neurons hold stale
// values; their sums are never read.
__device__ __forceinline__ void tile_sums(const float* Hs, const float* Xs, const float* Ws,
                                          float* red, int K1, int K2, int ldx, int ldw, int Pr,
                                          int Nr, int& KS) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int tp = Pr / RP;
    const int tasks = tp * (Nr / RN);
    KS = tasks >= kGW ? 1 : kGW / tasks;
    const int Kq = (K1 + K2) >> 2;
    const int K1q = K1 >> 2;
    for (int task = warp; task < tasks * KS; task += kGW) {
        const int t = task % tasks;
        const int ks = task / tasks;
        const int pb = (t % tp) * RP;
        const int nb = (t / tp) * RN;
        float acc[RP * RN];
#pragma unroll
        for (int i = 0; i < RP * RN; ++i) acc[i] = 0.f;
        for (int kq = ks * 32 + lane; kq < Kq; kq += 32 * KS) {
            const bool fh = kq < K1q;
            const float* xb = fh ? Hs + 4 * kq : Xs + 4 * (kq - K1q);
            const int ld = fh ? K1 : ldx;
            float4 x[RP], w[RN];
#pragma unroll
            for (int i = 0; i < RP; ++i) x[i] = lds4(xb + (pb + i) * ld);
#pragma unroll
            for (int j = 0; j < RN; ++j) w[j] = lds4(Ws + (nb + j) * ldw + 4 * kq);
#pragma unroll
            for (int i = 0; i < RP; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j)
                    acc[i * RN + j] = fmaf(x[i].w, w[j].w, fmaf(x[i].z, w[j].z,
                                      fmaf(x[i].y, w[j].y, fmaf(x[i].x, w[j].x, acc[i * RN + j]))));
        }
        // sum over the lanes by recursive halving: value v = i RN + j ends in
        // lanes 2v and 2v + 1
#pragma unroll
        for (int h = RP * RN / 2, off = 16; h >= 1; h >>= 1, off >>= 1) {
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float send = upper ? acc[i] : acc[i + h];
                const float keep = upper ? acc[i + h] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
        if ((lane & 1) == 0) {
            const int v = lane >> 1;
            red[(ks * Pr + pb + v / RN) * Nr + nb + v % RN] = acc[0];
        }
    }
}

__global__ void __launch_bounds__(kGT, 1) mlp_grid_kernel(const __grid_constant__ GridArgs a) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    Hdr& hd = *reinterpret_cast<Hdr*>(smem_raw);
    float* sm = reinterpret_cast<float*>(smem_raw + kHdr);
    const FusedNet& net = a.net;
    int m = a.M;
    if (a.m_dev) m = imin(m, (int)*a.m_dev);
    if (m <= 0) return;   // the same in every CTA: no counter is touched
    const int G = (int)gridDim.x;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (warp == 0) {
        // split_of with the candidates spread over the lanes
        float best_c = 3.0e38f;
        int best_p = 0;
        for (int P = lane + 1; P <= max_groups(m, G); P += 32) {
            float c;
            if (split_cost(net, m, G, P, c) && c < best_c) {
                best_c = c;
                best_p = P;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oc = __shfl_xor_sync(0xffffffffu, best_c, o);
            const int op = __shfl_xor_sync(0xffffffffu, best_p, o);
            if (oc < best_c || (oc == best_c && op < best_p)) {
                best_c = oc;
                best_p = op;
            }
        }
        if (lane == 0) {
            hd.P = best_p;
            hd.Q = best_p ? G / best_p : 0;
            hd.Pt = best_p ? (m + best_p - 1) / best_p : 0;
            hd.flag = 0u;
            hd.fin = 0u;
            mbar_init(&hd.mbW, 1);
            fence_mbar_init();
        }
    }
    __syncthreads();
    const int P = hd.P, Q = hd.Q, Pt = hd.Pt;
    if (P == 0) {   // more points than fit: the host never launches that
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    const Layout ly = layout_of(net, Pt, Q);
    float* Xs = sm + ly.xs;
    float* Hs = sm + ly.hs;
    float* Ws = sm + ly.ws;
    float* Wl = sm + ly.wl;
    float* bs = sm + ly.bs;
    float* bl = sm + ly.bl;
    float* red = sm + ly.red;
    float* hb = sm + ly.hb;
    const int c = (int)blockIdx.x;
    const int pg = c % P;
    const int qg = c / P;
    const int pbeg = pg * Pt;
    const int pcnt = c < P * Q ? imax(0, imin(Pt, m - pbeg)) : 0;
    const bool work = pcnt > 0;
    const int Pr = up_to(pcnt, RP);
    const int nh = net.nl - 1;   // hidden layers
    const FusedLayer& Lo = net.L[nh];
    unsigned int* gb = a.ctr;                          // barrier counter per hidden layer
    unsigned int* pgc = a.ctr + kFusedMaxLayers + 1;   // last-layer arrivals per point group
    const uint32_t lim = a.wait_extra ? kTestWaitLimit : kWaitLimit;
    const unsigned int need = (unsigned int)G + a.wait_extra;
    // The test hook issues each layer's weight rows after its barrier, so
    // that the wait it starves has no copy in flight.
    const bool early = a.wait_extra == 0u;

    // this CTA's weight rows of layer l (with the last layer's, for l = 0);
    // thread 0, uniform condition
    auto issue_w = [&](int l) {
        const FusedLayer& L = net.L[l];
        int n0, n1;
        group_range(L.n_out, Q, qg, n0, n1);
        const uint32_t bw = (uint32_t)(n1 - n0) * (uint32_t)L.ldw * 4u;
        const uint32_t bo = l == 0 ? (uint32_t)(Lo.n_out * Lo.ldw) * 4u : 0u;
        fence_async_shared();
        mbar_arrive_expect_tx(&hd.mbW, bw + bo);
        if (bw) bulk_load_1d(Ws, L.W + (int64_t)n0 * L.ldw, bw, &hd.mbW);
        if (bo) bulk_load_1d(Wl, Lo.W, bo, &hd.mbW);
    };
    auto needs_w = [&](int l) {
        if (!work) return false;
        int n0, n1;
        group_range(net.L[l].n_out, Q, qg, n0, n1);
        return l == 0 || n1 > n0;
    };

    bool w_out = false;   // a weight copy in flight (uniform)
    uint32_t wph = 0;     // completed phases of mbW
    bool ok = true;
    if (needs_w(0)) {
        if (threadIdx.x == 0) issue_w(0);
        w_out = true;
    }
    if (work) {
        if (warp == kGW - 1 && lane < Lo.n_out) bl[lane] = Lo.b[lane];
        // the input rows of this CTA's points, four items per thread in flight
        const int nq = net.ldx >> 2;
        const int total = pcnt * nq;
        for (int e0 = threadIdx.x; e0 < total; e0 += 4 * kGT) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * kGT;
                if (e < total) {
                    const int p = e / nq;
                    v[u] = gather_quad(a.src, a.p0 + pbeg + p, a.calib, a.map0, a.map1,
                                       4 * (e - p * nq));
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * kGT;
                if (e < total) {
                    const int p = e / nq;
                    *reinterpret_cast<float4*>(Xs + p * net.ldx + 4 * (e - p * nq)) = v[u];
                }
            }
        }
    }

    for (int l = 0; l < nh; ++l) {
        const FusedLayer& L = net.L[l];
        const bool last_hidden = l + 1 == nh;
        int n0, n1;
        group_range(L.n_out, Q, qg, n0, n1);
        const int nt = n1 - n0;
        const bool act = work && nt > 0;
        if (act && warp == kGW - 1)   // not warp 0, whose thread 0 polls the barrier
            for (int t = lane; t < nt; t += 32) bs[t] = L.b[n0 + t];
        if (l > 0 && act) {
            // every CTA has stored its share of layer l - 1: load this CTA's
            // rows of it (L2 only: other SMs wrote them)
            if (threadIdx.x == 0) {
                if (!grid_wait(gb + l - 1, need, lim)) hd.flag = 1u;
                else if (!early) issue_w(l);
            }
            __syncthreads();
            if (hd.flag) {
                ok = false;
                break;
            }
            if (!early) w_out = true;
            const float4* src = reinterpret_cast<const float4*>(a.H[(l - 1) & 1] +
                                                               (int64_t)pbeg * L.K1);
            float4* dst = reinterpret_cast<float4*>(Hs);
            const int nq = (pcnt * L.K1) >> 2;
            for (int e0 = threadIdx.x; e0 < nq; e0 += 8 * kGT) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e0 + u * kGT < nq) v[u] = __ldcg(src + e0 + u * kGT);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e0 + u * kGT < nq) dst[e0 + u * kGT] = v[u];
            }
        }
        const int Nr = up_to(nt, RN);
        int KS = 1;
        if (act || (l == 0 && work)) {
            if (!mbar_wait(&hd.mbW, wph & 1u, lim)) hd.flag = 1u;
            __syncthreads();
            if (hd.flag) {
                ok = false;
                break;
            }
            ++wph;
            w_out = false;
        }
        if (act) {
            tile_sums(Hs, Xs, Ws, red, L.K1, L.K2, net.ldx, L.ldw, Pr, Nr, KS);
            __syncthreads();
            // bias, leaky ReLU; K-splits summed in split order
            float* out = last_hidden ? hb : a.H[l & 1];
            for (int o = threadIdx.x; o < pcnt * nt; o += kGT) {
                const int p = o / nt;
                const int n = o - p * nt;
                float s = red[p * Nr + n];
                for (int k = 1; k < KS; ++k) s += red[(k * Pr + p) * Nr + n];
                s = lrelu(s + bs[n], net.slope);
                if (last_hidden) out[p * Nr + n] = s;
                else out[(int64_t)(pbeg + p) * L.n_out + n0 + n] = s;
            }
        }
        if (!last_hidden) {
            // the release of the CTA's stores (ordered before it by the CTA
            // barrier), then the arrival
            __syncthreads();
            const bool next = early && needs_w(l + 1);
            if (threadIdx.x == 0) {
                red_release(gb + l, 1u);
                if (next) issue_w(l + 1);   // Ws is free: every warp is past this layer's tile
            }
            if (next) w_out = true;
            continue;
        }
        if (!work) break;
        // the last layer: this neuron group's share of each point's sums
        __syncthreads();
        for (int o = threadIdx.x; o < pcnt * Lo.n_out; o += kGT) {
            const int p = o / Lo.n_out;
            const int j = o - p * Lo.n_out;
            float s = 0.f;
            for (int n = 0; n < nt; ++n) s = fmaf(Wl[j * Lo.ldw + n0 + n], hb[p * Nr + n], s);
            a.part[((int64_t)(pbeg + p) * kGridMaxCtas + qg) * 4 + j] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // releases this CTA's partials, acquires the earlier arrivals'
            const unsigned int prev = atom_add_acq_rel(pgc + pg, 1u);
            hd.fin = prev + 1u == (unsigned int)Q ? 1u : 0u;
            if (hd.fin) pgc[pg] = 0u;   // every neuron group is in
        }
        __syncthreads();
        if (hd.fin) {
            // per point (one warp): the partials in neuron-group order
            // (lane-strided, then a fixed shuffle tree), plus the x segment
            for (int p = warp; p < pcnt; p += kGW) {
                float t[4] = {0.f, 0.f, 0.f, 0.f};
                for (int j = 0; j < Lo.n_out; ++j) {
                    float s = 0.f;
                    for (int q = lane; q < Q; q += 32)
                        s += __ldcg(a.part + ((int64_t)(pbeg + p) * kGridMaxCtas + q) * 4 + j);
                    for (int k = lane; k < Lo.K2; k += 32)
                        s = fmaf(Xs[p * net.ldx + k], Wl[j * Lo.ldw + Lo.K1 + k], s);
                    t[j] = warp_sum(s);
                }
                if (lane == 0) last_epilogue(a.epi, a.p0 + pbeg + p, Lo.n_out, t, bl);
            }
        }
    }
    // leave: a wait that gave up is reported, this CTA's copies in flight
    // are waited for (bounded), and the last CTA out zeroes the barrier
    if (!ok && threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
    if (w_out) (void)mbar_wait(&hd.mbW, wph & 1u, lim);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(gb + kFusedMaxLayers, 1u);
        if (prev + 1u == (unsigned int)G)
            for (int k = 0; k <= kFusedMaxLayers; ++k) gb[k] = 0u;
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool g_ready[64] = {};
int g_ctas[64] = {};

// The grid of the current device: one CTA per SM (the cooperative launch
// needs every CTA resident), at most kGridMaxCtas.
cudaError_t grid_ctas(int* ctas) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_ready[dev]) {
        e = cudaFuncSetAttribute(mlp_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kGridSmem));
        int per_sm = 0, sms = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_grid_kernel, kGT,
                                                              kGridSmem);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorCooperativeLaunchTooLarge;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_ctas[dev] = sms < kGridMaxCtas ? sms : kGridMaxCtas;
        g_ready[dev] = true;
    }
    *ctas = g_ctas[dev];
    return cudaSuccess;
}

}  // namespace

bool grid_ok(const FusedNet& n) {
    if (n.nl < 2 || n.nl > kFusedMaxLayers || n.ldx <= 0 || n.ldx % 4) return false;
    for (int l = 0; l < n.nl; ++l) {
        const FusedLayer& L = n.L[l];
        if (!L.W || !L.b || !aligned16(L.W) || L.ldw % 4 || L.K1 % 4 || L.K2 % 4 ||
            L.ldw < L.K1 + L.K2 || L.n_out < 1)
            return false;
        if (l == 0 ? (L.K1 != 0 || L.K2 != n.ldx) : (L.K1 != n.L[l - 1].n_out)) return false;
        if (L.K2 != 0 && L.K2 != n.ldx) return false;
        if (l + 1 < n.nl ? L.n_out % 4 != 0 : L.n_out > 4) return false;
    }
    return true;
}

int grid_max_rows(const FusedNet& n) {
    int G = 0;
    if (!grid_ok(n) || grid_ctas(&G) != cudaSuccess || G < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    for (int m = kGridMaxRows; m >= 1; --m)
        if (split_of(n, m, G).P > 0) return m;
    return 0;
}

cudaError_t launch_mlp_grid(const GridArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    if (a.M > kGridMaxRows || !grid_ok(a.net) || !a.part || !a.ctr || !a.err ||
        (a.net.nl > 2 && (!a.H[0] || !a.H[1])))
        return cudaErrorInvalidValue;
    int G = 0;
    const cudaError_t e = grid_ctas(&G);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kGT);
    cfg.dynamicSmemBytes = kGridSmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mlp_grid_kernel, a);
}

}  // namespace pifu
