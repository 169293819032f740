// The scheduling step of the frame stream (the work-queue form of the batched
// frames), for the device (the scheduler kernel) and the host (a CPU test of
// its invariants).  Not in the paper: the paper processes each frame on its
// own; here frames of a queue flow through a fixed set of slots, and every
// round of the stream advances each slot by one step of the method of
// Sec. 3.2 for the frame it holds:
//
//   START    the frame's level 0: every node queued for evaluation;
//   ADVANCE  its level converged (empty frontier): the next level's set-up
//            (binarize, interpolate, candidates) and first selection
//            (the candidates' 26-ring);
//   EVAL     a conflict round: the unevaluated 26-neighbours of the last
//            evaluation's conflicts are queued already (non-empty frontier);
//   RENDER   its finest level converged: ray first crossing and colour;
//            the slot is free for the next frame of the queue afterwards.
//
// So each frame takes exactly the steps, and the conflict rounds, it takes
// alone, whatever the other slots hold; a frame that needs few rounds leaves
// its slot to the next frame instead of waiting for the slowest one.
#pragma once

#if defined(__CUDACC__)
#define PIFU_STREAM_HD __host__ __device__ __forceinline__
#else
#define PIFU_STREAM_HD inline
#endif

namespace pifu {

constexpr int kStreamMaxLevels = 8;

// What one round of the frame stream does for one of its slots.
enum SlotOp : int {
    SLOT_IDLE = 0,     // no frame
    SLOT_START = 1,    // a frame just taken from the queue: level-0 set-up, all its nodes queued
    SLOT_ADVANCE = 2,  // its level converged: the next level's set-up and selection
    SLOT_EVAL = 3,     // a conflict round of its level: the frontier is queued already
    SLOT_RENDER = 4,   // its finest level converged: ray first crossing and colour
};

// Persistent state of one slot.
struct StreamSlot {
    int frame;   // the frame it holds (-1: idle)
    int level;   // level index of that frame
    int cur;     // which of the two binarized bitsets holds the level
    int pad;
};

// Per-frame results of the stream.
struct StreamFrameStats {
    unsigned long long evals[kStreamMaxLevels];   // nodes evaluated per level
    unsigned long long cands[kStreamMaxLevels];   // boundary candidates per level
    unsigned int rounds[kStreamMaxLevels];        // conflict rounds per level
    unsigned long long t_admit;                   // device clock (ns) at admission
    unsigned long long t_done;                    // and after its render
    int slot;
    int done;
};

// One scheduling step of slot `t` after a round in which it did `op`.
// evaluated: the keys of the slot evaluated in that round; frontier: the
// keys its conflict expansion queued for the next round; cands: the boundary
// candidates its selection counted.  fs: the per-frame results; *next: the
// next frame of the queue (F frames).  Returns the slot's op for the next
// round and updates t, fs and *next.  *not_converged is set when a level
// needs more than max_rounds conflict rounds.
PIFU_STREAM_HD int stream_step(StreamSlot& t, int op, unsigned int evaluated, unsigned int frontier,
                               unsigned long long cands, int num_levels, int max_rounds,
                               StreamFrameStats* fs, unsigned int* next, unsigned int F,
                               unsigned long long now, int slot, bool* not_converged) {
    // account the round that ended
    if (t.frame >= 0) {
        StreamFrameStats& f = fs[t.frame];
        if (op == SLOT_START || op == SLOT_ADVANCE || op == SLOT_EVAL)
            f.evals[t.level] += evaluated;
        if (op == SLOT_ADVANCE) f.cands[t.level] += cands;
        if (op == SLOT_RENDER) {
            f.t_done = now;
            f.done = 1;
            t.frame = -1;
        }
    }
    // the next step of the frame it holds
    int nop = SLOT_IDLE;
    if (t.frame >= 0) {
        if (frontier > 0u) {
            nop = SLOT_EVAL;   // a conflict round
            StreamFrameStats& f = fs[t.frame];
            f.rounds[t.level] += 1u;
            if ((int)f.rounds[t.level] > max_rounds) *not_converged = true;
        } else if (t.level + 1 < num_levels) {
            nop = SLOT_ADVANCE;
            t.level += 1;
            t.cur ^= 1;
        } else {
            nop = SLOT_RENDER;
        }
    } else if (*next < F) {
        // a free slot takes the next frame of the queue
        t.frame = (int)(*next);
        *next += 1u;
        t.level = 0;
        t.cur = 0;
        StreamFrameStats& f = fs[t.frame];
        for (int l = 0; l < kStreamMaxLevels; ++l) {
            f.evals[l] = 0;
            f.cands[l] = 0;
            f.rounds[l] = 0;
        }
        f.t_admit = now;
        f.t_done = 0;
        f.slot = slot;
        f.done = 0;
        nop = SLOT_START;
    }
    return nop;
}

}  // namespace pifu
