"""Routing of a device-resident batch to the graph's switch bodies, on the
host, from the same header the kernels include (csrc/switch_index.cuh):

- the cluster-size pick has the fewest latency-weighted rounds (brute force
  over the plan), ties to the earlier (larger) cluster size;
- the re-check switch sends a queue of at most grid_hi points to the
  whole-GPU body, one of x3_lo < c <= x3_hi to the split-TF32 body, the rest
  to the picked cluster body, and an empty queue past every body;
- a conflict round's switch sends an empty batch past every body, a batch
  above the threshold to the tensor-core body, and every other batch to an
  FP32 body (body 0 when there is one form), never out of range."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2007_13988_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "switch_index.cuh"
using namespace pifu;

static int bad = 0;
#define CHECK(cond, a, b) do { if (!(cond)) { std::printf("FAIL %s %lld %lld\n", #cond, \
    (long long)(a), (long long)(b)); bad = 1; } } while (0)

static FusedPlan plan_of(int n) {
    // cluster sizes 16, 8, 4, 2 as the device offers them: more clusters of
    // the smaller sizes fit at once, each with a longer tile latency
    const int ncl[4] = {9, 18, 38, 76};
    const float lat[4] = {0.7f, 1.0f, 1.6f, 2.8f};
    FusedPlan p;
    for (int i = 0; i < n; ++i) {
        p.cl[i] = 16 >> i;
        p.ncl[i] = ncl[i];
        p.lat[i] = lat[i];
    }
    p.n = n;
    return p;
}

int main() {
    // the pick: fewest latency-weighted rounds, first on ties (0.1% band)
    for (int n = 1; n <= 4; ++n) {
        const FusedPlan p = plan_of(n);
        for (long long tiles = 1; tiles <= 2000; ++tiles) {
            const int got = fused_pick(p, tiles);
            CHECK(got >= 0 && got < n, tiles, got);
            float best = 3.0e38f;
            for (int i = 0; i < n; ++i) {
                const float c = (float)((tiles + p.ncl[i] - 1) / p.ncl[i]) * p.lat[i];
                if (c < best) best = c;
            }
            const float gc = (float)((tiles + p.ncl[got] - 1) / p.ncl[got]) * p.lat[got];
            CHECK(gc <= best * 1.001f, tiles, got);
            for (int i = 0; i < got; ++i) {
                const float c = (float)((tiles + p.ncl[i] - 1) / p.ncl[i]) * p.lat[i];
                CHECK(!(c <= best * 1.0f), tiles, i);   // an earlier size at the optimum wins
            }
        }
    }
    // the re-check switch: bodies [clusters..., x3?, grid?]
    for (int n = 1; n <= 4; ++n) {
        const FusedPlan p = plan_of(n);
        for (int x3 = 0; x3 <= 1; ++x3) {
            for (int g = 0; g <= 1; ++g) {
                const unsigned x3_lo = x3 ? 192u : 0u, x3_hi = x3 ? 32768u : 0u;
                const unsigned grid_hi = g ? 64u : 0u;
                const unsigned nb = (unsigned)n + (unsigned)x3 + (unsigned)g;
                CHECK(fused_index(p, 0u, x3_lo, x3_hi, grid_hi) >= nb, n, nb);
                for (unsigned c = 1; c <= 40000; c += (c < 600 ? 1u : 97u)) {
                    const unsigned i = fused_index(p, c, x3_lo, x3_hi, grid_hi);
                    CHECK(i < nb, c, i);
                    if (g && c <= grid_hi) CHECK(i == (unsigned)n + (unsigned)x3, c, i);
                    else if (x3 && c > x3_lo && c <= x3_hi) CHECK(i == (unsigned)n, c, i);
                    else CHECK(i == (unsigned)fused_pick(p, (c + kFusedTilePoints - 1) /
                                                              kFusedTilePoints), c, i);
                }
            }
        }
    }
    // a conflict round's switch: nt FP32 bodies, then the tensor-core body
    for (int n = 0; n <= 4; ++n) {
        const FusedPlan p = plan_of(n);
        const bool single = n <= 1;
        const int nt = single ? 1 : n + 2;   // with x3 and the whole-GPU body
        const unsigned cap = 1u << 20, thr = 256u;
        CHECK(batch_index(p, 0u, cap, thr, nt, single, 192u, 32768u, 64u) == (unsigned)nt + 1u, n, 0);
        for (unsigned c = 1; c <= 5000; ++c) {
            const unsigned i = batch_index(p, c, cap, thr, nt, single, 192u, 32768u, 64u);
            if (c > thr) CHECK(i == (unsigned)nt, c, i);
            else if (single) CHECK(i == 0u, c, i);
            else CHECK(i < (unsigned)nt && i == fused_index(p, c, 192u, 32768u, 64u), c, i);
        }
        // the queue length is clamped to the capacity the bodies were sized for
        if (!single) CHECK(batch_index(p, 200u, 100u, thr, nt, single, 192u, 32768u, 64u) ==
                           fused_index(p, 100u, 192u, 32768u, 64u), n, 100);
    }
    std::printf(bad ? "failed\n" : "ok\n");
    return bad;
}
"""


def test_switch_routing(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "route.cpp"
    exe = tmp_path / "route"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr
