"""The tile order of the chained tensor-core schedule, on the host, from the
same header the kernel includes (csrc/chain_order.cuh): every tile of every
layer appears once; every tile of layer l >= 1 comes after all the tiles of
layer l-1 on its row block (the property the kernel's deadlock freedom rests
on: a tile waits only on tiles handed out before it); and a jump of k tiles
lands where k single steps do (the kernel's cursors jump)."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2007_13988_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>
#include <vector>
#include "chain_order.cuh"
using namespace pifu;

static int fail(const char* what, int a, int b, int c) {
    std::printf("FAIL %s %d %d %d\n", what, a, b, c);
    return 1;
}

static int check(int nl, int lag, int group, const int* ntn, int n_mb) {
    ChainShape c{};
    c.nl = nl;
    c.lag = lag;
    c.group = group;
    long long total = 0;
    for (int l = 0; l < nl; ++l) {
        c.ntn[l] = ntn[l];
        total += (long long)n_mb * ntn[l];
    }
    const int n_g = (n_mb + group - 1) / group;
    // single steps
    std::vector<ChainTile> seq;
    ChainPos p = chain_begin(c, n_mb, n_g);
    bool have = n_g > 0 && chain_advance(c, n_mb, n_g, p, 0);
    while (have) {
        seq.push_back(chain_decode(c, p));
        have = chain_advance(c, n_mb, n_g, p, 1);
    }
    if ((long long)seq.size() != total) return fail("count", (int)seq.size(), (int)total, nl);
    std::map<std::tuple<int, int, int>, long long> index;
    for (long long t = 0; t < (long long)seq.size(); ++t) {
        const ChainTile& x = seq[t];
        if (x.l < 0 || x.l >= nl || x.mb < 0 || x.mb >= n_mb || x.nt < 0 || x.nt >= ntn[x.l])
            return fail("range", x.l, x.mb, x.nt);
        if (!index.emplace(std::make_tuple(x.l, x.mb, x.nt), t).second)
            return fail("twice", x.l, x.mb, x.nt);
    }
    // dependencies come first
    for (long long t = 0; t < (long long)seq.size(); ++t) {
        const ChainTile& x = seq[t];
        if (x.l == 0) continue;
        for (int nt = 0; nt < ntn[x.l - 1]; ++nt)
            if (index.at(std::make_tuple(x.l - 1, x.mb, nt)) >= t)
                return fail("order", x.l, x.mb, nt);
    }
    // jumps equal single steps
    std::srand(7);
    for (int trial = 0; trial < 200 && total > 0; ++trial) {
        const long long a = std::rand() % total;
        const long long k = std::rand() % (total - a + 3);
        ChainPos q = chain_begin(c, n_mb, n_g);
        chain_advance(c, n_mb, n_g, q, 0);
        chain_advance(c, n_mb, n_g, q, a);
        const bool ok = chain_advance(c, n_mb, n_g, q, k);
        if (a + k < total) {
            const ChainTile y = chain_decode(c, q);
            const ChainTile& z = seq[a + k];
            if (!ok || y.l != z.l || y.mb != z.mb || y.nt != z.nt) return fail("jump", (int)a, (int)k, 0);
        } else if (ok) {
            return fail("past end", (int)a, (int)k, 0);
        }
    }
    return 0;
}

int main() {
    const int fo[4] = {4, 2, 1, 1};   // f_O: 1024, 512, 256, 128 wide with BN 256, 256, 256, 128
    const int odd[4] = {3, 1, 2, 5};
    const int one[1] = {2};
    int bad = 0;
    for (int n_mb : {0, 1, 2, 5, 19, 20, 39, 281, 651}) {
        for (int lag : {1, 2, 4}) {
            for (int group : {1, 7, 19}) {
                bad |= check(4, lag, group, fo, n_mb);
                bad |= check(4, lag, group, odd, n_mb);
                bad |= check(2, lag, group, fo, n_mb);
                bad |= check(1, lag, group, one, n_mb);
            }
        }
    }
    std::printf(bad ? "failed\n" : "ok\n");
    return bad;
}
"""


def test_chain_tile_order_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "order.cpp"
    exe = tmp_path / "order"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
