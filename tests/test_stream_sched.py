"""The scheduling step of the frame stream (the work-queue batch form), on the
host, from the same header the scheduler kernel includes
(csrc/stream_sched.cuh).  A simulated stream gives every frame its own
profile of conflict rounds per level (the frontier a round leaves behind)
and drives S slots round by round as the device does.  Checked: every frame
is taken from the queue once, in order, and finishes; its recorded conflict
rounds, evaluations and candidates are its own; it never waits -- from its
admission to its render it takes exactly L set-up rounds, its conflict
rounds and one render round; no slot holds two frames; a free slot takes
the next frame in the round it frees up; the stream ends when the queue and
the slots are empty; a level over max_rounds is reported.  The lockstep
batch's rounds are the sum over levels of the slowest frame's, which this
form undercuts whenever the frames' profiles differ."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2007_13988_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "stream_sched.cuh"
using namespace pifu;

static int fail(const char* what, int a, int b, int c) {
    std::printf("FAIL %s %d %d %d\n", what, a, b, c);
    return 1;
}

// F frames, L levels, S slots; prof[f][l] = conflict rounds of frame f at level l.
static int run(int F, int L, int S, const std::vector<std::vector<int>>& prof, int max_rounds,
               bool expect_not_converged, long long* rounds_out) {
    std::vector<StreamSlot> st(S, StreamSlot{-1, 0, 0, 0});
    std::vector<int> op(S, SLOT_IDLE);
    std::vector<unsigned> pend_eval(S, 0), pend_next(S, 0);
    std::vector<unsigned long long> cands(S, 0);
    std::vector<StreamFrameStats> fs(F);
    std::vector<int> left(S, 0);          // conflict rounds still to come at the slot's level
    std::vector<long long> admit(F, -1), done(F, -1);
    unsigned next = 0;
    bool nc = false;
    long long round = 0;
    // the initial step admits the first frames (pend counters are zero)
    for (long long guard = 0; guard < 1000000; ++guard) {
        bool busy = false;
        for (int s = 0; s < S; ++s) {
            const int before = st[s].frame;
            const int nop = stream_step(st[s], op[s], pend_eval[s], pend_next[s], cands[s], L,
                                        max_rounds, fs.data(), &next, (unsigned)F,
                                        (unsigned long long)round, s, &nc);
            pend_eval[s] = pend_next[s];
            pend_next[s] = 0;
            cands[s] = 0;
            if (op[s] == SLOT_RENDER && done[before] < 0) done[before] = round;
            if (nop == SLOT_START) {
                if (st[s].frame != (int)next - 1) return fail("order", s, st[s].frame, (int)next);
                if (admit[st[s].frame] >= 0) return fail("twice", s, st[s].frame, 0);
                admit[st[s].frame] = round;
                // a slot that was free takes a frame at once
                if (before >= 0 && op[s] != SLOT_RENDER) return fail("overwrite", s, before, 0);
            }
            if (op[s] == SLOT_RENDER && nop != SLOT_START && next < (unsigned)F)
                return fail("slot left free", s, (int)next, 0);
            op[s] = nop;
            busy = busy || nop != SLOT_IDLE;
        }
        if (nc) break;
        if (!busy) break;
        ++round;
        // the round itself: selection, evaluation and expansion of every slot
        for (int s = 0; s < S; ++s) {
            const StreamSlot& t = st[s];
            if (op[s] == SLOT_START || op[s] == SLOT_ADVANCE) {
                const int f = t.frame;
                pend_eval[s] += 100 + 10 * f + t.level;   // the level's first selection
                if (op[s] == SLOT_ADVANCE) cands[s] += 7 * f + t.level;
                left[s] = t.level == 0 ? 0 : prof[f][t.level];
            }
            if (op[s] == SLOT_START || op[s] == SLOT_ADVANCE || op[s] == SLOT_EVAL) {
                if (left[s] > 0) {
                    pend_next[s] += 1 + s;               // a non-empty frontier
                    --left[s];
                }
            }
        }
    }
    *rounds_out = round;
    if (expect_not_converged) return nc ? 0 : fail("no not-converged report", 0, 0, 0);
    if (nc) return fail("not converged", 0, 0, 0);
    if ((int)next != F) return fail("queue left", (int)next, F, 0);
    for (int f = 0; f < F; ++f) {
        if (!fs[f].done) return fail("not done", f, 0, 0);
        long long own = L + 1;                           // set-ups and the render
        for (int l = 0; l < L; ++l) {
            const int want = l == 0 ? 0 : prof[f][l];
            if ((int)fs[f].rounds[l] != want) return fail("rounds", f, l, (int)fs[f].rounds[l]);
            const unsigned long long ev = 100 + 10 * f + l + (unsigned long long)want * 0;
            if (fs[f].evals[l] < ev) return fail("evals", f, l, (int)fs[f].evals[l]);
            if (l > 0 && fs[f].cands[l] != (unsigned long long)(7 * f + l))
                return fail("cands", f, l, (int)fs[f].cands[l]);
            own += want;
        }
        // from the round after admission to the render round: no waiting
        if (done[f] - admit[f] != own) return fail("waited", f, (int)(done[f] - admit[f]), (int)own);
        if (fs[f].t_admit != (unsigned long long)admit[f]) return fail("t_admit", f, 0, 0);
    }
    return 0;
}

int main() {
    int bad = 0;
    std::srand(11);
    for (int S : {1, 2, 3, 8, 16}) {
        for (int F : {1, 2, 5, 17, 64}) {
            for (int L : {1, 2, 4, 5}) {
                std::vector<std::vector<int>> prof(F, std::vector<int>(L, 0));
                long long lockstep = 0;
                for (int l = 0; l < L; ++l) {
                    int worst = 0;
                    for (int f = 0; f < F; ++f) {
                        prof[f][l] = l == 0 ? 0 : std::rand() % 7;
                        worst = prof[f][l] > worst ? prof[f][l] : worst;
                    }
                    lockstep += worst;
                }
                long long rounds = 0;
                bad |= run(F, L, S, prof, 4096, false, &rounds);
                // F <= S: one batch; the stream ends with its slowest frame,
                // which takes at most the lockstep batch's rounds
                if (F <= S && rounds > L + 1 + lockstep) bad |= fail("slower", F, L, S);
            }
        }
    }
    {
        std::vector<std::vector<int>> prof(3, std::vector<int>(3, 0));
        prof[1][2] = 9;
        long long r = 0;
        bad |= run(3, 3, 2, prof, 5, true, &r);
    }
    std::printf(bad ? "failed\n" : "ok\n");
    return bad;
}
"""


def test_stream_schedule_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "sched.cpp"
    exe = tmp_path / "sched"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
