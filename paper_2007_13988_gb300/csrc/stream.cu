// Scheduler kernel of the frame stream (the work-queue form of the batched
// frames, not in the paper): between two rounds it takes every slot one
// scheduling step further (stream_sched.cuh) and writes the views the next
// round's kernels read (SlotView), including the frame-dependent pointers of a
// slot that takes a frame from the queue.
#include "pifu_internal.h"

namespace pifu {
namespace {

__device__ __forceinline__ unsigned long long device_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void stream_sched_kernel(StreamArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long now = device_clock_ns();
    StreamCtl* ctl = a.ctl;
    if (a.init) {
        ctl->next_frame = 0u;
        ctl->rounds = 0u;
        ctl->rechecked = 0ull;
        ctl->fallback = 0ull;
        ctl->t_start = now;
        ctl->render_rounds = 0u;
        ctl->colour_passes = 0u;
        for (int s = 0; s < a.S; ++s) {
            a.st[s] = StreamSlot{-1, 0, 0, 0};
            a.sv[s].op = SLOT_IDLE;
            a.pend_eval[s] = 0u;
            a.pend_next[s] = 0u;
            a.cands[s] = 0ull;
        }
    } else {
        ctl->rounds += 1u;
    }
    bool not_converged = ctl->rounds > a.max_total_rounds;
    bool busy = false;
    bool rendered = false;
    unsigned int next = ctl->next_frame;
    for (int s = 0; s < a.S; ++s) {
        StreamSlot t = a.st[s];
        SlotView& v = a.sv[s];
        const int op = v.op;
        rendered = rendered || op == SLOT_RENDER;
        const int nop = stream_step(t, op, a.pend_eval[s], a.pend_next[s], a.cands[s], a.L,
                                    a.max_rounds, a.fs, &next, (unsigned)a.F, now, s,
                                    &not_converged);
        a.pend_eval[s] = a.pend_next[s];
        a.pend_next[s] = 0u;
        a.cands[s] = 0ull;
        if (nop == SLOT_START) {
            a.slot_maps0[s] = a.frame_maps0[t.frame];
            if (a.frame_maps1) a.slot_maps1[s] = a.frame_maps1[t.frame];
            a.slot_calibs[s] = a.frame_calibs[t.frame];
        }
        const int64_t sw = (int64_t)s * a.slot_words;
        v.op = nop;
        v.frame = t.frame;
        v.level = t.level;
        v.N = a.n0 << t.level;
        v.first_level = t.level == 0 ? 1 : 0;
        v.finest = t.level == a.L - 1 ? 1 : 0;
        v.bin = (t.cur ? a.bin1 : a.bin0) + sw;
        v.coarse = (t.cur ? a.bin0 : a.bin1) + sw;
        v.cand = a.cand + sw;
        v.tent = a.tent + sw;
        v.eval = a.eval + sw;
        v.conf = a.conf + sw;
        v.values = a.values + (int64_t)s * a.slot_nodes;
        v.top = a.top + (int64_t)s * a.slot_top;
        const int64_t f = t.frame;
        const bool has = f >= 0;
        v.depth = has && a.depth ? a.depth + f * a.npix : nullptr;
        v.rgb = has && a.rgb ? a.rgb + f * a.npix * 3 : nullptr;
        v.mask = has && a.mask ? a.mask + f * a.npix : nullptr;
        v.bits_out = has && a.bits_out ? a.bits_out + f * a.out_words : nullptr;
        a.st[s] = t;
        busy = busy || nop != SLOT_IDLE;
    }
    ctl->next_frame = next;
    if (rendered) ctl->render_rounds += 1u;
    if (not_converged) atomicOr(a.err, kErrNotConverged);
    const unsigned int err = *a.err;
    ctl->err = err;
    const bool go = busy && err == 0u;
    cudaGraphSetConditional(a.h, go ? 1u : 0u);
}

__global__ void set_if_kernel(cudaGraphConditionalHandle h, const unsigned int* count) {
    cudaGraphSetConditional(h, *count > 0u ? 1u : 0u);
}

__global__ void colour_cond_kernel(cudaGraphConditionalHandle h, const unsigned int* hits,
                                   const SlotView* sv, int S, int64_t npix, unsigned int cap,
                                   unsigned int* passes) {
    int renders = 0;
    for (int s = 0; s < S; ++s) renders += sv[s].op == SLOT_RENDER ? 1 : 0;
    const bool go = (int64_t)*hits + (int64_t)renders * npix > (int64_t)cap;
    if (go) *passes += 1u;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

}  // namespace

cudaError_t launch_stream_sched(const StreamArgs& a, cudaStream_t stream) {
    stream_sched_kernel<<<1, 32, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_set_if(cudaGraphConditionalHandle h, const unsigned int* count,
                          cudaStream_t stream) {
    set_if_kernel<<<1, 1, 0, stream>>>(h, count);
    return cudaGetLastError();
}

cudaError_t launch_colour_cond(cudaGraphConditionalHandle h, const unsigned int* hits,
                               const SlotView* sv, int S, int64_t npix, unsigned int cap,
                               unsigned int* passes, cudaStream_t stream) {
    colour_cond_kernel<<<1, 1, 0, stream>>>(h, hits, sv, S, npix, cap, passes);
    return cudaGetLastError();
}

}  // namespace pifu
