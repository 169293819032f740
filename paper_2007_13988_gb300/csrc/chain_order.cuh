// Tile order of the chained tensor-core schedule (mlp_chain.cu), as plain
// functions that compile for the device and for the host (the CPU tests
// check its invariants on this same code).
//
// Step s holds, for layer slots j = 0 .. nl-1 (layer l = nl-1-j), the tiles
// of layer l on row group gi = s - lag * l (a group: `group` 128-row blocks,
// the last one ragged), row block major, column tile minor.  A tile of layer
// l >= 1 reads every column tile of layer l-1 on its row block; those sit in
// step s - lag (lag >= 1), so they come earlier in the order.
#pragma once

#if defined(__CUDACC__)
#define PIFU_HD __host__ __device__ __forceinline__
#else
#define PIFU_HD inline
#endif

namespace pifu {

constexpr int kChainOrderMaxLayers = 8;

struct ChainShape {
    int nl;                              // hidden layers in the chain
    int lag;                             // steps between consecutive layers on a group
    int group;                           // 128-row blocks per row group
    int ntn[kChainOrderMaxLayers];       // column tiles of each layer (N / BN)
};

// Position in the order: step s, layer slot j, tile pos of the segment (s, j)
// whose length is len.
struct ChainPos {
    int s, j, pos, len;
};

struct ChainTile {
    int l, mb, nt;
};

PIFU_HD int chain_seg_len(const ChainShape& c, int n_mb, int n_g, int s, int j) {
    const int l = c.nl - 1 - j;
    const int gi = s - c.lag * l;
    if (gi < 0 || gi >= n_g) return 0;
    const int mb0 = gi * c.group;
    const int nmb = c.group < n_mb - mb0 ? c.group : n_mb - mb0;
    return nmb * c.ntn[l];
}

// The position of the first tile (len 0 when there is none).
PIFU_HD ChainPos chain_begin(const ChainShape& c, int n_mb, int n_g) {
    ChainPos p{0, 0, 0, n_g > 0 ? chain_seg_len(c, n_mb, n_g, 0, 0) : 0};
    return p;
}

// Moves k >= 0 tiles forward; false past the last tile.
PIFU_HD bool chain_advance(const ChainShape& c, int n_mb, int n_g, ChainPos& p, long long k) {
    const int n_steps = n_g + c.lag * (c.nl - 1);
    while (p.s < n_steps) {
        if ((long long)p.pos + k < (long long)p.len) {
            p.pos += (int)k;
            return true;
        }
        k -= p.len - p.pos;
        if (++p.j == c.nl) {
            p.j = 0;
            ++p.s;
        }
        p.pos = 0;
        p.len = p.s < n_steps ? chain_seg_len(c, n_mb, n_g, p.s, p.j) : 0;
    }
    return false;
}

PIFU_HD ChainTile chain_decode(const ChainShape& c, const ChainPos& p) {
    ChainTile t;
    t.l = c.nl - 1 - p.j;
    const int ntn = c.ntn[t.l];
    t.mb = (p.s - c.lag * t.l) * c.group + p.pos / ntn;
    t.nt = p.pos % ntn;
    return t;
}

}  // namespace pifu
