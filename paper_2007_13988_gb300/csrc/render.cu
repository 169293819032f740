// Ray first crossing of the mesh-free render (Sec. 3.2, "Mesh-free
// Rendering"): the volume is aligned with the target view, x/y with the
// pixel axes and z with the rays, higher z nearer to the observer.
//
// One thread per pixel walks its ray from the observer (depth node N, z = +1)
// backwards.  A sample is the bilinear (x, y) interpolation of the four node
// columns around the pixel centre; a node's value is the network's occupancy
// where the node was evaluated and its binarized 0/1 value elsewhere.  The
// first sample >= 0.5 is the surface: the depth is the linear 0.5 crossing
// between it and the previous sample (the two nodes "interpolated by the
// predicted occupancy").  Empty space costs four bit tests per sample (the
// evaluated and binarized bitsets of two node rows), so a miss reads only
// bitsets.  Hits are appended (warp-aggregated) to a list of surface points
// for the colour MLP; misses get the background of Eq. 3.
#include <math.h>

#include <algorithm>

#include "pifu_internal.h"
#include "sm100.cuh"

namespace pifu {
namespace {

// The set bits of word w of eval | bin raise the column tops (and bottoms).
__device__ __forceinline__ void column_top_word(int N, int row_words, const uint32_t* __restrict__ eval,
                                                const uint32_t* __restrict__ bin, int* top,
                                                int* bot, int64_t w) {
    const int n1 = N + 1;
    uint32_t bits = __ldg(eval + w) | __ldg(bin + w);
    if (!bits) return;
    const int wx = (int)(w % row_words);
    const int64_t row = w / row_words;   // k (N+1) + j
    const int j = (int)(row % n1);
    const int k = (int)(row / n1);
    int* t = top + (int64_t)j * n1 + wx * 32;
    int* u = bot ? bot + (int64_t)j * n1 + wx * 32 : nullptr;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        atomicMax(t + b, k);
        if (u) atomicMax(u + b, N - k);
    }
}

// Highest depth-node index k (z index, 0..N) at which node column (i, j) has
// any evaluated or inside node: one thread per bitset word (k, j, word), one
// atomicMax per set bit into top[j][i], which starts at -1 (empty column).
// With `bot`, also N - (lowest such k) into bot[j][i] (also from -1): the
// last ray sample index from the observer at which the column is non-empty.
__global__ void __launch_bounds__(256) column_top_kernel(int N, int row_words,
                                                         const uint32_t* __restrict__ eval,
                                                         const uint32_t* __restrict__ bin,
                                                         int* __restrict__ top, int* __restrict__ bot,
                                                         int64_t slot_words, int64_t slot_top,
                                                         unsigned int* __restrict__ hits) {
    sm100::griddep_launch_dependents();   // the rays wait for this grid
    // the hit list's length, appended to by render_rays_kernel after this launch
    if (hits && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *hits = 0u;
    const int n1 = N + 1;
    {
        const int64_t f = blockIdx.y;   // frame of a lockstep batch
        eval += f * slot_words;
        bin += f * slot_words;
        top += f * slot_top;
        if (bot) bot += f * slot_top;
    }
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= (int64_t)n1 * n1 * row_words) return;
    column_top_word(N, row_words, eval, bin, top, bot, w);
}

// bits ix and ix+1 of a bitset row as bits 0 and 1 (ix + 1 <= N is in the row)
__device__ __forceinline__ uint32_t two_bits(const uint32_t* __restrict__ rowp, int ix) {
    uint32_t v = __ldg(rowp + (ix >> 5)) >> (ix & 31);
    if ((ix & 31) == 31) v |= __ldg(rowp + (ix >> 5) + 1) << 1;
    return v & 3u;
}

// Fine node coordinate of a pixel centre along one axis: (2i+1) N / (2 R) as
// an integer part and an exact fraction (for power-of-two N and R).
__device__ __forceinline__ void pixel_node(int i, int R, int N, int& i0, float& w) {
    const long long num = (long long)(2 * i + 1) * N;
    const long long den = 2LL * R;
    long long q = num / den;
    long long r = num - q * den;
    if (q >= N) {  // cannot happen for i < R; keeps i0 + 1 <= N regardless
        q = N - 1;
        r = den;
    }
    i0 = (int)q;
    w = (float)r / (float)den;
}

// The first crossing of pixel pix's ray through one frame's volume (the
// arrays of `a`): true on a hit, with its depth zs; (px, py) is the pixel
// centre in NDC.
__device__ __forceinline__ bool ray_crossing(const RenderArgs& a, int64_t pix, float& zs,
                                             float& px, float& py) {
    bool hit = false;
    zs = 0.f;
    const int i = (int)(pix % a.width);
    const int j = (int)(pix / a.width);
    int ix0, iy0;
    float wx, wy;
    pixel_node(i, a.width, a.N, ix0, wx);
    pixel_node(j, a.height, a.N, iy0, wy);
    px = __fmaf_rn((float)(2 * i + 1), 1.0f / (float)a.width, -1.0f);
    py = __fmaf_rn((float)(2 * j + 1), 1.0f / (float)a.height, -1.0f);
    const int n1 = a.N + 1;
    const int rw = a.row_words;
    const float w00 = (1.f - wx) * (1.f - wy), w10 = wx * (1.f - wy);
    const float w01 = (1.f - wx) * wy, w11 = wx * wy;
    const float h = 2.0f / (float)a.N;
    // samples nearer the observer than every node of the four columns are 0
    const int64_t c0 = (int64_t)iy0 * n1 + ix0;
    const int ktop = max(max(a.top[c0], a.top[c0 + 1]), max(a.top[c0 + n1], a.top[c0 + n1 + 1]));
    const int kstart = ktop < 0 ? a.N + 1 : a.N - ktop;
    // and the samples farther than every node of the four columns are 0
    const int* bt = a.top + (int64_t)n1 * n1;
    const int kend = max(max(bt[c0], bt[c0 + 1]), max(bt[c0 + n1], bt[c0 + n1 + 1]));
    float vprev = 0.f;
    for (int k = kstart; k <= kend; ++k) {
        const int iz = a.N - k;
        const int64_t row0 = (int64_t)iz * n1 + iy0;
        const int64_t row1 = row0 + 1;
        const uint32_t e0 = two_bits(a.eval + row0 * rw, ix0);
        const uint32_t e1 = two_bits(a.eval + row1 * rw, ix0);
        const uint32_t b0 = two_bits(a.bin + row0 * rw, ix0);
        const uint32_t b1 = two_bits(a.bin + row1 * rw, ix0);
        float v = 0.f;
        if (e0 | e1 | b0 | b1) {
            const float v00 = (e0 & 1u) ? a.values[row0 * n1 + ix0] : (float)(b0 & 1u);
            const float v10 = (e0 & 2u) ? a.values[row0 * n1 + ix0 + 1] : (float)(b0 >> 1);
            const float v01 = (e1 & 1u) ? a.values[row1 * n1 + ix0] : (float)(b1 & 1u);
            const float v11 = (e1 & 2u) ? a.values[row1 * n1 + ix0 + 1] : (float)(b1 >> 1);
            v = fmaf(w11, v11, fmaf(w01, v01, fmaf(w10, v10, w00 * v00)));
        }
        if (v >= kHalf) {
            hit = true;
            if (k == 0) {
                zs = 1.0f;
            } else {
                const float t = (kHalf - vprev) / (v - vprev);
                const float zprev = __fmaf_rn(-(float)(k - 1), h, 1.0f);
                zs = zprev - t * h;
            }
            break;
        }
        vprev = v;
    }
    return hit;
}

// Writes a pixel's depth, mask and (on a miss) background colour, and
// appends its hit with key `hit_key` (warp-aggregated; the whole warp calls).
__device__ __forceinline__ void ray_outputs(const RenderArgs& a, int64_t pix, bool valid, bool hit,
                                            float zs, float px, float py, int hit_key) {
    const int lane = threadIdx.x & 31;
    if (valid) {
        if (a.depth) a.depth[pix] = hit ? zs : __int_as_float(0x7fc00000);
        if (a.mask) a.mask[pix] = hit ? 1 : 0;
        if (a.rgb && !hit) {
            a.rgb[pix * 3 + 0] = a.bg[0];
            a.rgb[pix * 3 + 1] = a.bg[1];
            a.rgb[pix * 3 + 2] = a.bg[2];
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    if (ballot == 0u) return;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(a.hit_count, (unsigned)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) {
        const unsigned pos = base + __popc(ballot & ((1u << lane) - 1u));
        a.hit_xyz[3 * (int64_t)pos + 0] = px;
        a.hit_xyz[3 * (int64_t)pos + 1] = py;
        a.hit_xyz[3 * (int64_t)pos + 2] = zs;
        a.hit_pix[pos] = hit_key;
    }
}

__global__ void __launch_bounds__(256) render_rays_kernel(RenderArgs a) {
    // a programmatic dependent of the column table; the colour gather after
    // it waits for this grid
    sm100::griddep_wait();
    sm100::griddep_launch_dependents();
    const int64_t npix = (int64_t)a.width * a.height;
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t frame = blockIdx.y;   // frame of a lockstep batch (0: one frame)
    if (frame > 0) {
        a.values += frame * a.slot_nodes;
        a.eval += frame * a.slot_words;
        a.bin += frame * a.slot_words;
        a.top += frame * 2 * (int64_t)(a.N + 1) * (a.N + 1);
        if (a.depth) a.depth += frame * npix;
        if (a.mask) a.mask += frame * npix;
        if (a.rgb) a.rgb += frame * npix * 3;
    }
    bool hit = false;
    float zs = 0.f, px = 0.f, py = 0.f;
    const bool valid = pix < npix;
    if (valid) hit = ray_crossing(a, pix, zs, px, py);
    ray_outputs(a, pix, valid, hit, zs, px, py, (int)(frame * npix + pix));
}

// ---- frame stream: the render of the slots whose finest level converged ----
//
// Grid y = slot; only slots whose round op is RENDER do anything.

// Column tops and bottoms back to -1 (empty), in [2][(N+1)^2] ints.
__global__ void __launch_bounds__(256) stream_top_reset_kernel(const SlotView* __restrict__ sv) {
    const SlotView v = sv[blockIdx.y];
    if (v.op != SLOT_RENDER) return;
    const int64_t n = 2 * (int64_t)(v.N + 1) * (v.N + 1);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        v.top[q] = -1;
}

// Column tops and bottoms of the slot's volume, and the copy of its
// binarized finest level into the frame's place of bits_out.
__global__ void __launch_bounds__(256) stream_column_top_kernel(const SlotView* __restrict__ sv) {
    const SlotView v = sv[blockIdx.y];
    if (v.op != SLOT_RENDER) return;
    const int n1 = v.N + 1;
    const int rw = row_words_of(v.N);
    const int64_t total = words_of(v.N);
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (int64_t)gridDim.x * blockDim.x) {
        column_top_word(v.N, rw, v.eval, v.bin, v.top, v.top + (int64_t)n1 * n1, w);
        if (v.bits_out) v.bits_out[w] = v.bin[w];
    }
}

// Rays of the slot's frame: its depth, mask and background into the frame's
// outputs, its hits appended with keys frame * width * height + pixel.
__global__ void __launch_bounds__(256) stream_rays_kernel(const SlotView* __restrict__ sv,
                                                          RenderArgs a) {
    const SlotView v = sv[blockIdx.y];
    if (v.op != SLOT_RENDER) return;
    a.N = v.N;
    a.row_words = row_words_of(v.N);
    a.values = v.values;
    a.eval = v.eval;
    a.bin = v.bin;
    a.top = v.top;
    a.depth = v.depth;
    a.rgb = v.rgb;
    a.mask = v.mask;
    const int64_t npix = (int64_t)a.width * a.height;
    // whole warps iterate together (the hit append is warp-aggregated)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npix;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = base + threadIdx.x;
        bool hit = false;
        float zs = 0.f, px = 0.f, py = 0.f;
        const bool valid = pix < npix;
        if (valid) hit = ray_crossing(a, pix, zs, px, py);
        ray_outputs(a, pix, valid, hit, zs, px, py, (int)((int64_t)v.frame * npix + pix));
    }
}

}  // namespace

cudaError_t launch_render_rays(const RenderArgs& a, cudaStream_t stream) {
    const int64_t npix = (int64_t)a.width * a.height;
    if (npix <= 0) return cudaSuccess;
    const int64_t n1 = a.N + 1;
    const int slots = a.slots > 1 ? a.slots : 1;
    if (slots > 65535 || (int64_t)slots * npix > 2147483647LL) return cudaErrorInvalidValue;
    // per frame: top [(N+1)^2] then bottom [(N+1)^2], both from -1
    cudaError_t e =
        cudaMemsetAsync(a.top, 0xff, (size_t)(2 * n1 * n1 * slots) * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const int64_t nt = n1 * n1 * a.row_words;
    column_top_kernel<<<dim3((unsigned)((nt + 255) / 256), (unsigned)slots), 256, 0, stream>>>(
        a.N, a.row_words, a.eval, a.bin, a.top, a.top + n1 * n1, a.slot_words, 2 * n1 * n1,
        a.hit_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pdl(render_rays_kernel, dim3((unsigned)((npix + 255) / 256), (unsigned)slots),
                      dim3(256), 0, stream, a);
}

cudaError_t launch_stream_render(const SlotView* sv, int slots, int N_fine, const RenderArgs& a,
                                 cudaStream_t stream) {
    const int64_t npix = (int64_t)a.width * a.height;
    if (slots < 1 || slots > 65535 || npix <= 0) return cudaErrorInvalidValue;
    const int64_t n1 = N_fine + 1;
    const unsigned gt = (unsigned)std::min<int64_t>((2 * n1 * n1 + 255) / 256, 152 * 2);
    stream_top_reset_kernel<<<dim3(gt, (unsigned)slots), 256, 0, stream>>>(sv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned gw = (unsigned)std::min<int64_t>((words_of(N_fine) + 255) / 256, 152 * 2);
    stream_column_top_kernel<<<dim3(gw, (unsigned)slots), 256, 0, stream>>>(sv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned gp = (unsigned)std::min<int64_t>((npix + 255) / 256, 152 * 4);
    stream_rays_kernel<<<dim3(gp, (unsigned)slots), 256, 0, stream>>>(sv, a);
    return cudaGetLastError();
}

}  // namespace pifu

// ---- view-culled final level (Sec. 3.2) ----------------------------------------

namespace pifu {
namespace {

// The binarized localized level along one pixel column: the bilinear (x, y)
// weights of the four node columns around the pixel centre, and the column
// value at a coarse depth node counted from the observer.  Exact in float for
// power-of-two sizes (dyadic weights, sums of at most four of them).
struct CullColumn {
    const uint32_t* bin;
    int Nc, rw, ix0, iy0;
    float w00, w10, w01, w11;

    __device__ __forceinline__ float coarse(int kc) const {
        const int iz = Nc - kc;
        const int64_t row0 = (int64_t)iz * (Nc + 1) + iy0;
        const uint32_t b0 = two_bits(bin + row0 * rw, ix0);
        const uint32_t b1 = two_bits(bin + (row0 + 1) * rw, ix0);
        return w00 * (float)(b0 & 1u) + w10 * (float)(b0 >> 1) + w01 * (float)(b1 & 1u) +
               w11 * (float)(b1 >> 1);
    }
};

__device__ __forceinline__ CullColumn cull_column(const CullArgs& a, int i, int j) {
    CullColumn c;
    c.bin = a.bin;
    c.Nc = a.Nc;
    c.rw = a.row_words;
    float wx, wy;
    pixel_node(i, a.width, a.Nc, c.ix0, wx);
    pixel_node(j, a.height, a.Nc, c.iy0, wy);
    c.w00 = (1.f - wx) * (1.f - wy);
    c.w10 = wx * (1.f - wy);
    c.w01 = (1.f - wx) * wy;
    c.w11 = wx * wy;
    return c;
}

// Walks the fine depth nodes k = 0 .. 2 Nc of a column in order, with the
// tentative value T_k (coarse node k/2, or the mean of its two neighbours for
// odd k), stopping after the first T = 1 (the nodes behind it are shadow
// nodes).  visit(k, T) is called for every non-shadow node.  Returns the
// number of nodes walked.
template <typename F>
__device__ __forceinline__ void walk_column(const CullColumn& c, int kc_start, F&& visit) {
    float prev = 0.f;   // coarse nodes before kc_start are empty (value 0)
    for (int kc = kc_start; kc <= c.Nc; ++kc) {
        const float v = c.coarse(kc);
        if (kc > 0) {
            const float t = 0.5f * (prev + v);
            if (!visit(2 * kc - 1, t)) return;
        }
        if (!visit(2 * kc, v)) return;
        prev = v;
    }
}

__device__ __forceinline__ int cull_start(const CullArgs& a, const int* top, const CullColumn& c) {
    const int n1 = a.Nc + 1;
    const int64_t c0 = (int64_t)c.iy0 * n1 + c.ix0;
    const int ktop = max(max(top[c0], top[c0 + 1]), max(top[c0 + n1], top[c0 + n1 + 1]));
    return ktop < 0 ? -1 : a.Nc - ktop;   // first coarse depth node (from the observer) that may be set
}

__global__ void __launch_bounds__(256) cull_select_kernel(CullArgs a) {
    const int* __restrict__ top = a.top;
    const int64_t npix = (int64_t)a.width * a.height;
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t n1f = 2 * (int64_t)a.Nc + 1;
    int n = 0;
    CullColumn c{};
    int ks = -1;
    if (pix < npix) {
        c = cull_column(a, (int)(pix % a.width), (int)(pix / a.width));
        ks = cull_start(a, top, c);
        if (ks >= 0)
            walk_column(c, ks, [&](int, float t) {
                if (t >= 1.f) return false;
                if (t > 0.f) ++n;
                return true;
            });
    }
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int warp_total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int base = 0u;
    if (lane == 31 && warp_total > 0) base = atomicAdd(a.count, (unsigned int)warp_total);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (n) {
        unsigned int pos = base + (unsigned int)(incl - n);
        if (pos + (unsigned int)n > a.cap) {
            atomicOr(a.err, kErrCapacity);   // the list would overflow: drop this column
            return;
        }
        walk_column(c, ks, [&](int k, float t) {
            if (t >= 1.f) return false;
            if (t > 0.f) a.list[pos++] = (int)(pix * n1f + k);
            return true;
        });
    }
}

__global__ void __launch_bounds__(256) cull_final_kernel(CullArgs a) {
    const int* __restrict__ top = a.top;
    const int64_t npix = (int64_t)a.width * a.height;
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t n1f = 2 * (int64_t)a.Nc + 1;
    bool hit = false;
    float zs = 0.f, px = 0.f, py = 0.f;
    if (pix < npix) {
        const int i = (int)(pix % a.width);
        const int j = (int)(pix / a.width);
        px = __fmaf_rn((float)(2 * i + 1), 1.0f / (float)a.width, -1.0f);
        py = __fmaf_rn((float)(2 * j + 1), 1.0f / (float)a.height, -1.0f);
        const CullColumn c = cull_column(a, i, j);
        const int ks = cull_start(a, top, c);
        if (ks >= 0) {
            const float h = 1.0f / (float)a.Nc;   // fine node spacing 2 / (2 Nc)
            const float* vals = a.values + pix * n1f;
            float vprev = 0.f;
            walk_column(c, ks, [&](int k, float t) {
                const float v = (t > 0.f && t < 1.f) ? vals[k] : t;   // evaluated candidates
                if (v >= kHalf) {
                    hit = true;
                    if (k == 0) {
                        zs = 1.0f;
                    } else {
                        const float u = (kHalf - vprev) / (v - vprev);
                        const float zprev = __fmaf_rn(-(float)(k - 1), h, 1.0f);
                        zs = zprev - u * h;
                    }
                    return false;
                }
                vprev = v;
                return true;
            });
        }
        if (a.depth) a.depth[pix] = hit ? zs : __int_as_float(0x7fc00000);
        if (a.mask) a.mask[pix] = hit ? 1 : 0;
        if (a.rgb && !hit) {
            a.rgb[pix * 3 + 0] = a.bg[0];
            a.rgb[pix * 3 + 1] = a.bg[1];
            a.rgb[pix * 3 + 2] = a.bg[2];
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    if (ballot == 0u) return;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(a.hit_count, (unsigned)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) {
        const unsigned pos = base + __popc(ballot & ((1u << lane) - 1u));
        a.hit_xyz[3 * (int64_t)pos + 0] = px;
        a.hit_xyz[3 * (int64_t)pos + 1] = py;
        a.hit_xyz[3 * (int64_t)pos + 2] = zs;
        a.hit_pix[pos] = (int)pix;
    }
}

}  // namespace

cudaError_t launch_cull_select(const CullArgs& a, cudaStream_t stream) {
    const int64_t npix = (int64_t)a.width * a.height;
    if (npix <= 0) return cudaSuccess;
    if (a.width != a.height || a.Nc < 1 || (2 * (int64_t)a.Nc + 1) * npix > 2147483647LL)
        return cudaErrorInvalidValue;
    // highest set depth node of every column of the localized level (bin only)
    const int64_t n1 = a.Nc + 1;
    cudaError_t e = cudaMemsetAsync(a.top, 0xff, (size_t)(n1 * n1) * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const int64_t nt = n1 * n1 * a.row_words;
    column_top_kernel<<<dim3((unsigned)((nt + 255) / 256), 1u), 256, 0, stream>>>(
        a.Nc, a.row_words, a.bin, a.bin, a.top, nullptr, 0, 0, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cull_select_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cull_final(const CullArgs& a, cudaStream_t stream) {
    const int64_t npix = (int64_t)a.width * a.height;
    if (npix <= 0) return cudaSuccess;
    cull_final_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace pifu
