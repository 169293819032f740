// Bookkeeping kernels of the coarse-to-fine surface localization (Sec. 3.2,
// "Octree-based Robust Surface Localization").
//
// Every per-node set of a level (tentative binarized value, boundary
// candidates, evaluated, conflicts, binarized result) is a bitset with one
// padded 32-bit-word row per (k, j) node row: bit i of row (k, j) lives in
// word (k (N+1) + j) * row_words + (i >> 5).  One thread owns one word, so
// all set operations are word-wide, the 26-neighbourhood dilation is an OR of
// nine shifted rows, and the list of nodes to evaluate is built by a
// warp-aggregated prefix sum of popcounts (one atomic per warp).  At 256^3 a
// bitset is 2.4 MB; the whole level's bookkeeping touches ~15 MB, against
// hundreds of MFLOP per evaluated point of MLP work.
//
// Several frames in lockstep: blockIdx.y is the frame; its bitsets start
// `fslot` words (coarse: `cslot`) further, and the node keys it appends are
// frame * slot_nodes + node, into one list for all frames.
#include <algorithm>

#include "pifu_internal.h"
#include "sm100.cuh"

namespace pifu {
namespace {

__device__ __forceinline__ uint32_t valid_mask(int N, int wx) {
    // bits of word wx that hold nodes i <= N
    const int first = wx * 32;
    const int n_valid = min(32, N + 1 - first);
    return n_valid >= 32 ? 0xffffffffu : ((1u << n_valid) - 1u);
}

// 64 bits of a coarse row starting at coarse x = 16 wx (bits beyond the row
// are zero because padding bits are kept zero).
__device__ __forceinline__ uint64_t coarse_segment(const uint32_t* row, int row_words, int wx) {
    const int q = wx >> 1;
    const uint64_t lo = q < row_words ? row[q] : 0u;
    const uint64_t hi = q + 1 < row_words ? row[q + 1] : 0u;
    return (lo | (hi << 32)) >> ((wx & 1) * 16);
}

// Bits 0..15 of x moved to the even bits 0, 2, .., 30.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// Tentative value of a fine node = tri-linear interpolation of the binarized
// coarse level = mean of its 1, 2, 4 or 8 coarse corners (a fine index i sits
// on coarse node i/2 when even, between (i-1)/2 and (i+1)/2 when odd).
// cand: 0 < mean < 1.  tent: mean >= 1/2.  For bitset word w of an N-cell
// level (w below words_of(N)).
__device__ __forceinline__ void classify_word(const uint32_t* __restrict__ coarse, int N, int64_t w,
                                              uint32_t& c_word, uint32_t& t_word) {
    const int n1 = N + 1;
    const int rw = row_words_of(N);
    const int Nc = N / 2;
    const int rwc = row_words_of(Nc);
    const int wx = (int)(w % rw);
    const int64_t rowid = w / rw;
    const int j = (int)(rowid % n1);
    const int k = (int)(rowid / n1);
    const int kc0 = k >> 1, kc1 = (k + 1) >> 1;
    const int jc0 = j >> 1, jc1 = (j + 1) >> 1;
    const int nz = (k & 1) ? 2 : 1;
    const int ny = (j & 1) ? 2 : 1;
    uint64_t seg[4];
    int nrows = 0;
    for (int a = 0; a < nz; ++a)
        for (int b = 0; b < ny; ++b) {
            const int kc = a ? kc1 : kc0;
            const int jc = b ? jc1 : jc0;
            seg[nrows++] = coarse_segment(coarse + ((int64_t)kc * (Nc + 1) + jc) * rwc, rwc, wx);
        }
    // Bit-parallel over the word's 32 fine nodes: fine bit 2c (even x) sits
    // on coarse bit c, fine bit 2c+1 (odd x) between coarse bits c and c+1.
    // Per coarse row r: X_r = the first corner of every fine bit, Y_r = the
    // second corner of the odd ones (0 at even bits).
    constexpr uint32_t EV = 0x55555555u, OD = 0xAAAAAAAAu;
    uint32_t any = 0u, all = 0xffffffffu;
    uint32_t b0 = 0u, b1 = 0u, b2 = 0u, b3 = 0u;   // bit-sliced corner count
    auto add = [&](uint32_t v) {
        uint32_t c = v, t;
        t = b0 & c; b0 ^= c; c = t;
        t = b1 & c; b1 ^= c; c = t;
        t = b2 & c; b2 ^= c; c = t;
        b3 ^= c;
    };
    for (int r = 0; r < nrows; ++r) {
        const uint32_t e = spread16((uint32_t)seg[r] & 0xffffu);          // bit 2c = coarse c
        const uint32_t e1 = spread16((uint32_t)(seg[r] >> 1) & 0xffffu);  // bit 2c = coarse c+1
        const uint32_t X = e | (e << 1);                                  // even: c; odd: c
        const uint32_t Y = (e1 << 1) & OD;                                // odd: c+1
        any |= X | Y;
        all &= X & (Y | EV);
        add(X);
        add(Y);
    }
    // corners per fine bit: nrows (even x) or 2 nrows (odd x); tent: 2 cnt >= corners
    const uint32_t ge1 = b0 | b1 | b2 | b3;
    const uint32_t ge2 = b1 | b2 | b3;
    const uint32_t ge4 = b2 | b3;
    const uint32_t t_even = nrows == 4 ? ge2 : ge1;                      // cnt >= ceil(nrows / 2)
    const uint32_t t_odd = nrows == 1 ? ge1 : (nrows == 2 ? ge2 : ge4);   // cnt >= nrows
    const uint32_t vm = valid_mask(N, wx);
    c_word = any & ~all & vm;
    t_word = ((t_even & EV) | (t_odd & OD)) & vm;
}

// cands (optional, one frame): += the number of candidate bits; zero
// (optional): set to 0 (the list count the selection after it appends to).
__global__ void __launch_bounds__(256) classify_kernel(const uint32_t* __restrict__ coarse, int N,
                                                       uint32_t* __restrict__ cand,
                                                       uint32_t* __restrict__ tent,
                                                       uint32_t* __restrict__ bin,
                                                       uint32_t* __restrict__ eval,
                                                       uint32_t* __restrict__ conf0,
                                                       int64_t cslot, int64_t fslot,
                                                       unsigned long long* __restrict__ cands,
                                                       unsigned int* __restrict__ zero) {
    sm100::griddep_launch_dependents();   // the selection waits for this grid
    {
        const int64_t f = blockIdx.y;
        coarse += f * cslot;
        cand += f * fslot;
        tent += f * fslot;
        bin += f * fslot;
        eval += f * fslot;
        conf0 += f * fslot;
    }
    if (zero && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *zero = 0u;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t c_word = 0u;
    if (w < words_of(N)) {
        uint32_t t_word;
        classify_word(coarse, N, w, c_word, t_word);
        cand[w] = c_word;
        tent[w] = t_word;
        bin[w] = t_word;
        eval[w] = 0u;
        conf0[w] = 0u;
    }
    if (cands) {
        unsigned int n = __popc(c_word);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        if ((threadIdx.x & 31) == 0 && n) atomicAdd(cands, (unsigned long long)n);
    }
}

// The conflict loop's decision (loop_control_kernel's) taken by the last CTA
// of the kernel that wrote the frontier count, instead of a launch of its
// own.  Every thread of the kernel calls it once, at its end.
__device__ __forceinline__ void loop_tail(const LoopTail& t, const unsigned int* count) {
    if (!t.done) return;
    __syncthreads();
    if (threadIdx.x != 0) return;
    __threadfence();
    const unsigned int ctas = gridDim.x * gridDim.y;
    if (atomicAdd(t.done, 1u) + 1u != ctas) return;
    __threadfence();
    const unsigned int c = *reinterpret_cast<const volatile unsigned int*>(count);
    bool go = c > 0u;
    if (go && c > t.cap) {
        atomicOr(t.err, kErrCapacity);
        go = false;
    }
    if (go && t.count_round) {
        const unsigned int r = *t.rounds + 1u;
        *t.rounds = r;
        if ((int)r > t.max_rounds) {
            atomicOr(t.err, kErrNotConverged);
            go = false;
        }
    }
    *t.done = 0u;
    cudaGraphSetConditional(t.h, go ? 1u : 0u);
}

__global__ void __launch_bounds__(256) dense_setup_kernel(int N, uint32_t* __restrict__ cand,
                                                          uint32_t* __restrict__ tent,
                                                          uint32_t* __restrict__ bin,
                                                          uint32_t* __restrict__ eval,
                                                          uint32_t* __restrict__ conf0,
                                                          int64_t fslot, ZeroSpans z) {
    sm100::griddep_launch_dependents();   // the gather after it waits for this grid
    if (blockIdx.x == 0 && blockIdx.y == 0)
        for (int q = 0; q < ZeroSpans::kMax; ++q)
            for (uint32_t i = threadIdx.x; i < z.words[q]; i += blockDim.x) z.p[q][i] = 0u;
    const int n1 = N + 1;
    const int rw = row_words_of(N);
    const int64_t total = (int64_t)n1 * n1 * rw;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + blockIdx.y * fslot;
    if (w - (int64_t)blockIdx.y * fslot >= total) return;
    cand[w] = 0u;
    tent[w] = 0u;
    bin[w] = 0u;
    conf0[w] = 0u;
    eval[w] = valid_mask(N, (int)((w - (int64_t)blockIdx.y * fslot) % rw));
}

// Word w of dilate26(src), restricted to the grid: the OR of the nine node
// rows around it, each with its bits shifted by -1, 0 and +1.
__device__ __forceinline__ uint32_t dilate_word(const uint32_t* __restrict__ src, int N, int64_t w) {
    const int n1 = N + 1;
    const int rw = row_words_of(N);
    const int wx = (int)(w % rw);
    const int64_t row = w / rw;
    const int j = (int)(row % n1);
    const int k = (int)(row / n1);
    uint32_t acc = 0u;
    for (int dk = -1; dk <= 1; ++dk) {
        const int kk = k + dk;
        if (kk < 0 || kk > N) continue;
        for (int dj = -1; dj <= 1; ++dj) {
            const int jj = j + dj;
            if (jj < 0 || jj > N) continue;
            const uint32_t* r = src + ((int64_t)kk * n1 + jj) * rw;
            const uint32_t c = r[wx];
            const uint32_t l = wx > 0 ? r[wx - 1] : 0u;
            const uint32_t h = wx + 1 < rw ? r[wx + 1] : 0u;
            acc |= c | (c << 1) | (c >> 1) | (l >> 31) | (h << 31);
        }
    }
    return acc & valid_mask(N, wx);
}

// sel = dilate26(src) & ~eval, restricted to the grid; eval |= sel; compact.
// radius 0: sel = src & ~eval (no dilation; the binarized-octree baseline).
__global__ void __launch_bounds__(256) dilate_select_kernel(const uint32_t* __restrict__ src,
                                                            uint32_t* __restrict__ eval,
                                                            uint32_t* __restrict__ clear, int N,
                                                            int* __restrict__ list,
                                                            unsigned int* __restrict__ count,
                                                            int64_t fslot, int64_t slot_nodes,
                                                            int radius, LoopTail tail) {
    sm100::griddep_wait();   // a programmatic dependent of the level's classify
    {
        const int64_t f = blockIdx.y;
        src += f * fslot;
        eval += f * fslot;
        if (clear) clear += f * fslot;
    }
    const int n1 = N + 1;
    const int rw = row_words_of(N);
    const int64_t total = (int64_t)n1 * n1 * rw;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t sel = 0u;
    int64_t row = 0;
    int wx = 0;
    if (w < total) {
        wx = (int)(w % rw);
        row = w / rw;
        const uint32_t acc = radius ? dilate_word(src, N, w) : src[w] & valid_mask(N, wx);
        const uint32_t e = eval[w];
        sel = acc & ~e;
        if (sel) eval[w] = e | sel;
        if (clear) clear[w] = 0u;
    }
    // warp-aggregated compaction of the selected node indices
    const int n = __popc(sel);
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int warp_total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int base = 0u;
    if (lane == 31 && warp_total > 0) base = atomicAdd(count, (unsigned int)warp_total);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (n) {
        int pos = (int)base + incl - n;
        const int64_t node0 = row * n1 + (int64_t)wx * 32 + (int64_t)blockIdx.y * slot_nodes;
        uint32_t s = sel;
        while (s) {
            const int b = __ffs(s) - 1;
            s &= s - 1u;
            list[pos++] = (int)(node0 + b);
        }
    }
    loop_tail(tail, count);
}

// Threshold subdivision, the second octree baseline of Fig. 3: every fine
// node takes the mean of the continuous coarse values at its 1, 2, 4 or 8
// coarse corners (their tri-linear interpolation) and is selected for
// evaluation when the largest absolute deviation of those values from the
// mean exceeds `thr`.  One warp per bitset word, lane b on node 32 wx + b:
// the value store is coalesced and the word's bits come from ballots.
// coarse: the dense (N/2 + 1)^3 values of the coarser level.
__global__ void __launch_bounds__(256) threshold_select_kernel(
    const float* __restrict__ coarse, int N, float thr, float* __restrict__ values,
    uint32_t* __restrict__ tent, uint32_t* __restrict__ bin, uint32_t* __restrict__ eval,
    uint32_t* __restrict__ conf0, int* __restrict__ list, unsigned int* __restrict__ count) {
    const int n1 = N + 1;
    const int rw = row_words_of(N);
    const int nc1 = N / 2 + 1;
    const int64_t total = (int64_t)n1 * n1 * rw;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= total) return;                  // whole warps only (blockDim % 32 == 0)
    const int wx = (int)(w % rw);
    const int64_t row = w / rw;
    const int j = (int)(row % n1);
    const int k = (int)(row / n1);
    const int i = wx * 32 + lane;
    const bool valid = i <= N;
    float mean = 0.f, dev = 0.f;
    if (valid) {
        const int kc[2] = {k >> 1, (k + 1) >> 1};
        const int jc[2] = {j >> 1, (j + 1) >> 1};
        const int ic[2] = {i >> 1, (i + 1) >> 1};
        const int nz = 1 + (k & 1), ny = 1 + (j & 1), nx = 1 + (i & 1);
        float c[8];
        int n = 0;
        float sum = 0.f;
        for (int a = 0; a < nz; ++a)
            for (int b = 0; b < ny; ++b)
                for (int d = 0; d < nx; ++d) {
                    c[n] = coarse[((int64_t)kc[a] * nc1 + jc[b]) * nc1 + ic[d]];
                    sum += c[n++];
                }
        mean = sum / (float)n;               // n is 1, 2, 4 or 8: an exact scaling
        for (int m = 0; m < n; ++m) dev = fmaxf(dev, fabsf(c[m] - mean));
        values[row * n1 + i] = mean;
    }
    const bool sel = valid && dev > thr;
    const uint32_t sbits = __ballot_sync(0xffffffffu, sel);
    const uint32_t tbits = __ballot_sync(0xffffffffu, valid && mean >= kHalf);
    if (lane == 0) {
        tent[w] = tbits;
        bin[w] = tbits;
        eval[w] = sbits;
        conf0[w] = 0u;
    }
    if (sbits) {
        unsigned int base = 0u;
        if (lane == 0) base = atomicAdd(count, (unsigned int)__popc(sbits));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (sel) list[base + __popc(sbits & ((1u << lane) - 1u))] = (int)(row * n1 + i);
    }
}

__global__ void __launch_bounds__(256) popcount_kernel(const uint32_t* __restrict__ bits,
                                                       int64_t words,
                                                       unsigned long long* __restrict__ count,
                                                       int64_t fslot) {
    bits += (int64_t)blockIdx.y * fslot;   // frame blockIdx.y into count[blockIdx.y]
    count += blockIdx.y;
    unsigned long long local = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x)
        local += __popc(bits[w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// Graph form: decides whether the conflict loop runs (another) round.  The
// frontier `count` must be non-empty and fit the batch capacity; a round
// beyond max_rounds ends the loop with the not-converged error bit.
__global__ void loop_control_kernel(cudaGraphConditionalHandle h, const unsigned int* count,
                                    unsigned int cap, unsigned int* rounds, int count_round,
                                    int max_rounds, unsigned int* err) {
    const unsigned int c = *count;
    bool go = c > 0u;
    if (go && c > cap) {
        atomicOr(err, kErrCapacity);
        go = false;
    }
    if (go && count_round) {
        const unsigned int r = *rounds + 1u;
        *rounds = r;
        if ((int)r > max_rounds) {
            atomicOr(err, kErrNotConverged);
            go = false;
        }
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// One thread per (conflict, neighbour) pair; warp-aggregated append.
// Frame stream (sv set): a key's slot gives the level and the evaluated
// bitset, and slot_count[slot] counts the keys appended for it.
__global__ void __launch_bounds__(256) expand_conflicts_kernel(
    const int* __restrict__ clist, const unsigned int* __restrict__ ccount, unsigned int max_c,
    int N0, uint32_t* __restrict__ eval0, int64_t key_div, int64_t slot_words,
    int* __restrict__ list, unsigned int* __restrict__ count, unsigned int cap,
    unsigned int* __restrict__ err, const SlotView* __restrict__ sv,
    unsigned int* __restrict__ slot_count, int* __restrict__ list_f,
    unsigned int* __restrict__ count_f, LoopTail tail) {
    const unsigned int nc = min(*ccount, max_c);
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)nc * 26;
    // whole warps iterate together (ballots below)
    for (int64_t base_t = (int64_t)blockIdx.x * blockDim.x; base_t < total;
         base_t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base_t + threadIdx.x;
        bool fresh = false;
        bool to_f = false;   // frame stream: a key of a slot at its finest level
        int64_t nkey = 0;
        if (t < total) {
            const int64_t c = t / 26;
            int nb = (int)(t - c * 26);
            nb += nb >= 13 ? 1 : 0;                // skip the centre of the 3x3x3 block
            const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
            int64_t key = clist[c];
            int64_t f = 0;
            if (key_div) {
                f = key / key_div;
                key -= f * key_div;
            }
            int N = N0;
            uint32_t* eval = eval0 + f * slot_words;
            if (sv) {
                N = sv[f].N;
                eval = sv[f].eval;
                to_f = list_f != nullptr && sv[f].finest != 0;
            }
            const int n1 = N + 1;
            const int rw = row_words_of(N);
            const int64_t row = key / n1;           // k (N+1) + j
            const int i = (int)(key - row * n1) + dx;
            const int j = (int)(row % n1) + dy;
            const int k = (int)(row / n1) + dz;
            if (i >= 0 && i <= N && j >= 0 && j <= N && k >= 0 && k <= N) {
                const int64_t r2 = (int64_t)k * n1 + j;
                uint32_t* wptr = eval + r2 * rw + (i >> 5);
                const uint32_t bit = 1u << (i & 31);
                if (!(*wptr & bit)) {
                    const uint32_t old = atomicOr(wptr, bit);
                    fresh = !(old & bit);
                }
                nkey = f * (key_div ? key_div : 0) + r2 * n1 + i;
                if (fresh && slot_count) atomicAdd(slot_count + f, 1u);
            }
        }
        // two warp-aggregated appends: the first list, and the second one
        // (frame stream: keys of slots at their finest level)
#pragma unroll
        for (int which = 0; which < 2; ++which) {
            const bool mine = fresh && (to_f == (which == 1));
            const unsigned ballot = __ballot_sync(0xffffffffu, mine);
            if (ballot == 0u) continue;
            unsigned int* cnt = which ? count_f : count;
            int* lst = which ? list_f : list;
            unsigned int b = 0u;
            if (lane == 0) b = atomicAdd(cnt, (unsigned int)__popc(ballot));
            b = __shfl_sync(0xffffffffu, b, 0);
            if (mine) {
                const unsigned int pos = b + __popc(ballot & ((1u << lane) - 1u));
                if (pos < cap) lst[pos] = (int)nkey;
                else atomicOr(err, kErrCapacity);
            }
        }
    }
    loop_tail(tail, count);
}

// ---- frame stream: the set-up and selection of every slot in one launch each ----
//
// Grid (x: enough blocks for the finest level's words, striding; y: slot).
// A slot whose round op is START gets level 0 set up (every node evaluated,
// nothing else set); ADVANCE runs the classify step from its coarser level.

__global__ void __launch_bounds__(256) stream_setup_kernel(const SlotView* __restrict__ sv) {
    const SlotView v = sv[blockIdx.y];
    if (v.op != SLOT_START && v.op != SLOT_ADVANCE) return;
    const int N = v.N;
    const int rw = row_words_of(N);
    const int64_t total = words_of(N);
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c_word = 0u, t_word = 0u, e_word = 0u;
        if (v.op == SLOT_START)
            e_word = valid_mask(N, (int)(w % rw));
        else
            classify_word(v.coarse, N, w, c_word, t_word);
        v.cand[w] = c_word;
        v.tent[w] = t_word;
        v.bin[w] = t_word;
        v.eval[w] = e_word;
        v.conf[w] = 0u;
    }
}

// Queues the nodes a slot evaluates first in its new level, as keys
// slot * slot_nodes + node appended at *count (beyond cap the error word gets
// kErrCapacity): START every node of level 0; ADVANCE the 26-ring of the
// boundary candidates (dilate26(cand) & ~eval, then eval |= it), whose number
// goes to cands[slot].  pend[slot] += the keys queued for the slot.
__global__ void __launch_bounds__(256) stream_select_kernel(
    const SlotView* __restrict__ sv, int64_t slot_nodes, int* __restrict__ list,
    unsigned int* __restrict__ count, unsigned int cap, unsigned int* __restrict__ err,
    unsigned int* __restrict__ pend, unsigned long long* __restrict__ cands,
    int* __restrict__ list_f, unsigned int* __restrict__ count_f) {
    const int slot = blockIdx.y;
    const SlotView v = sv[slot];
    if (v.op != SLOT_START && v.op != SLOT_ADVANCE) return;
    if (list_f && v.finest) {   // the finest level's keys go to the second list
        list = list_f;
        count = count_f;
    }
    const int N = v.N;
    const int n1 = N + 1;
    const int rw = row_words_of(N);
    const int64_t total = words_of(N);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long ncand = 0;
    // whole warps iterate together (shuffles below)
    for (int64_t base_w = (int64_t)blockIdx.x * blockDim.x; base_w < total; base_w += stride) {
        const int64_t w = base_w + threadIdx.x;
        uint32_t sel = 0u;
        int64_t node0 = 0;
        if (w < total) {
            const int wx = (int)(w % rw);
            node0 = (w / rw) * n1 + (int64_t)wx * 32;
            if (v.op == SLOT_START) {
                sel = valid_mask(N, wx);   // level-0 set-up marked them evaluated
            } else {
                ncand += __popc(v.cand[w]);
                const uint32_t e = v.eval[w];
                sel = dilate_word(v.cand, N, w) & ~e;
                if (sel) v.eval[w] = e | sel;
            }
        }
        const int n = __popc(sel);
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int warp_total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned int base = 0u;
        if (lane == 31 && warp_total > 0) {
            base = atomicAdd(count, (unsigned int)warp_total);
            atomicAdd(pend + slot, (unsigned int)warp_total);
        }
        base = __shfl_sync(0xffffffffu, base, 31);
        if (n) {
            unsigned int pos = base + (unsigned int)(incl - n);
            const int64_t key0 = node0 + (int64_t)slot * slot_nodes;
            uint32_t s = sel;
            while (s) {
                const int b = __ffs(s) - 1;
                s &= s - 1u;
                if (pos < cap) list[pos] = (int)(key0 + b);
                else atomicOr(err, kErrCapacity);
                ++pos;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
    if (lane == 0 && ncand) atomicAdd(cands + slot, ncand);
}

// *dst += *src, flagging a capacity error when *src exceeds cap.
__global__ void accumulate_kernel(unsigned long long* dst, const unsigned int* src,
                                  unsigned int cap, unsigned int* err) {
    const unsigned int v = *src;
    *dst += v;
    if (v > cap) atomicOr(err, kErrCapacity);
}

// An enqueued frame's error word ORed into a word that only the host clears
// (the asynchronous frame call: the next frame's graph zeroes its own word).
__global__ void latch_err_kernel(const unsigned int* err, unsigned int* sticky) {
    const unsigned int e = *err;
    if (e) atomicOr(sticky, e);
}

// The start of a conflict round in the graph: the round's size moved from
// the frontier count to the batch count, accumulate_kernel's statistics and
// *zero = 0, in one launch (batch_switch_kernel does the same for a batch
// that also picks its branch).
__global__ void round_start_kernel(unsigned int* count, unsigned long long* evals,
                                   unsigned int cap, unsigned int* err, unsigned int* zero,
                                   unsigned int* next) {
    const unsigned int c = *next;
    *count = c;
    *next = 0u;
    *evals += c;
    if (c > cap) atomicOr(err, kErrCapacity);
    *zero = 0u;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_classify(const uint32_t* coarse_bin, int N, uint32_t* cand, uint32_t* tent,
                            uint32_t* bin, uint32_t* eval, uint32_t* conf0, cudaStream_t stream,
                            int slots, int64_t cslot, int64_t fslot, unsigned long long* cands,
                            unsigned int* zero) {
    if (slots < 1 || slots > 65535 || (cands && slots != 1)) return cudaErrorInvalidValue;
    classify_kernel<<<dim3(blocks_for(words_of(N)), (unsigned)slots), 256, 0, stream>>>(
        coarse_bin, N, cand, tent, bin, eval, conf0, cslot, fslot, cands, zero);
    return cudaGetLastError();
}

cudaError_t launch_dense_setup(int N, uint32_t* cand, uint32_t* tent, uint32_t* bin,
                               uint32_t* eval, uint32_t* conf0, cudaStream_t stream, int slots,
                               int64_t fslot, const ZeroSpans* zero) {
    if (slots < 1 || slots > 65535) return cudaErrorInvalidValue;
    dense_setup_kernel<<<dim3(blocks_for(words_of(N)), (unsigned)slots), 256, 0, stream>>>(
        N, cand, tent, bin, eval, conf0, fslot, zero ? *zero : ZeroSpans{});
    return cudaGetLastError();
}

cudaError_t launch_dilate_select(const uint32_t* src, uint32_t* eval, uint32_t* clear, int N,
                                 int* list, unsigned int* count, cudaStream_t stream, int slots,
                                 int64_t fslot, int64_t slot_nodes, const LoopTail* tail) {
    if (slots < 1 || slots > 65535) return cudaErrorInvalidValue;
    return launch_pdl(dilate_select_kernel, dim3(blocks_for(words_of(N)), (unsigned)slots),
                      dim3(256), 0, stream, src, eval, clear, N, list, count, fslot, slot_nodes, 1,
                      tail ? *tail : LoopTail{});
}

cudaError_t launch_select(const uint32_t* src, uint32_t* eval, int N, int* list,
                          unsigned int* count, cudaStream_t stream) {
    return launch_pdl(dilate_select_kernel, dim3(blocks_for(words_of(N))), dim3(256), 0, stream,
                      src, eval, static_cast<uint32_t*>(nullptr), N, list, count, (int64_t)0,
                      (int64_t)0, 0, LoopTail{});
}

cudaError_t launch_threshold_select(const float* coarse, int N, float thr, float* values,
                                    uint32_t* tent, uint32_t* bin, uint32_t* eval,
                                    uint32_t* conf0, int* list, unsigned int* count,
                                    cudaStream_t stream) {
    const int64_t threads = words_of(N) * 32;
    threshold_select_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(
        coarse, N, thr, values, tent, bin, eval, conf0, list, count);
    return cudaGetLastError();
}

cudaError_t launch_loop_control(cudaGraphConditionalHandle h, const unsigned int* count,
                                unsigned int cap, unsigned int* rounds, int count_round,
                                int max_rounds, unsigned int* err, cudaStream_t stream) {
    loop_control_kernel<<<1, 1, 0, stream>>>(h, count, cap, rounds, count_round, max_rounds, err);
    return cudaGetLastError();
}

cudaError_t launch_expand_conflicts(const int* clist, const unsigned int* ccount,
                                    unsigned int max_c, int N, uint32_t* eval, int64_t key_div,
                                    int64_t slot_words, int* list, unsigned int* count,
                                    unsigned int cap, unsigned int* err, cudaStream_t stream,
                                    const SlotView* sv, unsigned int* slot_count, int* list_f,
                                    unsigned int* count_f, const LoopTail* tail) {
    if (max_c == 0) return tail ? cudaErrorInvalidValue : cudaSuccess;
    const int64_t total = (int64_t)max_c * 26;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 8);
    expand_conflicts_kernel<<<(unsigned)blocks, 256, 0, stream>>>(
        clist, ccount, max_c, N, eval, key_div, slot_words, list, count, cap, err, sv,
        slot_count, list_f, count_f, tail ? *tail : LoopTail{});
    return cudaGetLastError();
}

cudaError_t launch_stream_setup(const SlotView* sv, int slots, int N_fine, cudaStream_t stream) {
    if (slots < 1 || slots > 65535) return cudaErrorInvalidValue;
    const unsigned gx = (unsigned)std::min<int64_t>(blocks_for(words_of(N_fine)), 152 * 2);
    stream_setup_kernel<<<dim3(gx, (unsigned)slots), 256, 0, stream>>>(sv);
    return cudaGetLastError();
}

cudaError_t launch_stream_select(const SlotView* sv, int slots, int N_fine, int64_t slot_nodes,
                                 int* list, unsigned int* count, unsigned int cap,
                                 unsigned int* err, unsigned int* pend,
                                 unsigned long long* cands, cudaStream_t stream, int* list_f,
                                 unsigned int* count_f) {
    if (slots < 1 || slots > 65535) return cudaErrorInvalidValue;
    const unsigned gx = (unsigned)std::min<int64_t>(blocks_for(words_of(N_fine)), 152 * 2);
    stream_select_kernel<<<dim3(gx, (unsigned)slots), 256, 0, stream>>>(
        sv, slot_nodes, list, count, cap, err, pend, cands, list_f, count_f);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(unsigned long long* dst, const unsigned int* src, unsigned int cap,
                              unsigned int* err, cudaStream_t stream) {
    accumulate_kernel<<<1, 1, 0, stream>>>(dst, src, cap, err);
    return cudaGetLastError();
}

cudaError_t launch_latch_err(const unsigned int* err, unsigned int* sticky, cudaStream_t stream) {
    latch_err_kernel<<<1, 1, 0, stream>>>(err, sticky);
    return cudaGetLastError();
}

cudaError_t launch_round_start(unsigned int* count, const RoundStart& rs, cudaStream_t stream) {
    round_start_kernel<<<1, 1, 0, stream>>>(count, rs.evals, rs.cap, rs.err, rs.zero, rs.next);
    return cudaGetLastError();
}

cudaError_t launch_popcount(const uint32_t* bits, int64_t words, unsigned long long* count,
                            cudaStream_t stream, int slots, int64_t fslot) {
    if (slots < 1 || slots > 65535) return cudaErrorInvalidValue;
    const unsigned gx = slots > 1 ? 152u : 152u * 4u;
    popcount_kernel<<<dim3(gx, (unsigned)slots), 256, 0, stream>>>(bits, words, count, fslot);
    return cudaGetLastError();
}

}  // namespace pifu
