// Internal declarations shared by the translation units of libpifu.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "stream_sched.cuh"
#include "switch_index.cuh"

#include <utility>

namespace pifu {

// A launch as a programmatic dependent of the kernel before it on the stream
// (the launch may be placed before that kernel has finished; the kernel must
// call griddepcontrol.wait before touching anything the earlier kernel
// writes or reads).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr float kHalf = 0.5f;

// Bits of the context's device error word.
constexpr unsigned int kErrTimeout = 1u;       // a bounded device wait gave up
constexpr unsigned int kErrNotConverged = 2u;  // graph form: conflict loop over max_rounds
constexpr unsigned int kErrCapacity = 4u;      // graph form: a device count over its capacity

// 3x4 calibration passed by value to kernels.
struct Calib {
    float c[12];
};

// A feature map as the kernels see it.
struct Map {
    const void* data;
    int H, W, C;
    int dtype;  // 0 f32, 1 bf16
};

// ---- frame stream (work-queue form): slot ops and the scheduling step ---------

// One slot of the frame stream as the kernels of a round see it (written by
// the scheduler kernel between rounds).  Its arrays are the slot's, sized for
// the finest level; the current level uses their first words.
struct SlotView {
    int op;                  // SlotOp of this round
    int frame;               // the stream frame the slot holds (-1: none)
    int level;               // level index
    int N;                   // cells per axis of the level
    int first_level;         // 1 at level 0: no tentative values, no conflicts
    int finest;              // 1 at the last level
    const uint32_t* coarse;  // SLOT_ADVANCE: the binarized coarser level
    uint32_t* cand;
    uint32_t* tent;
    uint32_t* bin;
    uint32_t* eval;
    uint32_t* conf;
    float* values;           // dense store of the level's occupancies
    int* top;                // render scratch [2][(N+1)^2]
    float* depth;            // the frame's outputs (each may be null)
    float* rgb;
    uint8_t* mask;
    uint32_t* bits_out;      // optional copy of the frame's binarized finest level
};

// Where the points of an MLP batch come from.
enum PointMode : int {
    PTS_XYZ = 0,     // float32 [m][3] positions
    PTS_LIST = 1,    // int32 node indices of a level with N cells per axis
    PTS_DENSE = 2,   // node index = base + point number
    PTS_XYZ_IDX = 3, // positions xyz[list[p]] (a subset of a position array)
    PTS_COLUMN = 4,  // view-culled final level: key list[p] = pixel (N+1) + k, the point
                     // at pixel (i, j) of a width x width image and depth node k of N cells
};

struct PointSrc {
    int mode;
    const float* xyz;   // PTS_XYZ
    const int* list;    // PTS_LIST
    int64_t base;       // PTS_DENSE first node index
    int N;              // grid modes: cells per axis
    // Device-resident batch size: when set, a launch sized for m points
    // processes min(*count, m) of them (graph form, no host read of counts).
    const unsigned int* count;
    // Several frames in one batch (lockstep form), when maps0 is set: a
    // point's key is list[p] (PTS_LIST), base + p (PTS_DENSE) or keys[p]
    // (PTS_XYZ); its frame is key / slot_div, whose maps and calibration
    // replace the launch's, and in the grid modes its node is key % slot_div.
    const Map* maps0;
    const Map* maps1;     // may be null
    const Calib* calibs;
    const int* keys;      // PTS_XYZ
    int64_t slot_div;
    int width;            // PTS_COLUMN: pixels per image side
    // Frame stream: the grid modes' key / slot_div is a slot, whose level
    // resolution replaces N.
    const SlotView* sv;
};

// What the last MLP layer does with its output.
enum EpilogueMode : int {
    EPI_STORE = 0,   // out[p * n_out + c] = act(t)   (p = pix[p] when pix is set)
    EPI_LEVEL = 1,   // scatter occupancy into a level (values, bits, conflicts)
    EPI_PIXELS = 2,  // out[pix[p] * 3 + c] = act(t)
    EPI_COLUMN = 3,  // out[key] = occupancy, key = list[p] (view-culled final level)
};

enum OutAct : int { ACT_SIGMOID = 0, ACT_TANH01 = 1 };

struct LevelBits {
    float* values;          // dense [(N+1)^3]
    const uint32_t* tent;   // tentative binarized values (read-only during a level)
    uint32_t* bin;          // working binarized values
    uint32_t* conf;         // conflicts found by this evaluation
    int N;
    int row_words;
    int first_level;        // 1: no tentative values, no conflicts
    // Several frames (lockstep form): a node key is frame * key_div + node,
    // and frame f's arrays start f slot_nodes values / f slot_words words
    // further.
    int64_t key_div;        // 0: one frame
    int64_t slot_nodes;
    int64_t slot_words;
    // Optional: the keys of the conflicts found are also appended here (the
    // sparse expansion of the next conflict round reads them).
    int* clist;
    unsigned int* ccount;
    unsigned int ccap;      // beyond it the error word gets kErrCapacity
    unsigned int* err;
    // Frame stream: key / key_div is a slot whose arrays, resolution and
    // first-level flag replace the ones above.
    const SlotView* sv;
};

struct Epilogue {
    int mode;
    int act;
    float* out;             // EPI_STORE / EPI_PIXELS
    const int* pix;         // EPI_PIXELS pixel index per point
    const int* list;        // EPI_LEVEL node index per point (null: dense from base)
    int64_t base;           // EPI_LEVEL dense base
    LevelBits lv;
    // Mixed precision: occupancies within `margin` of 0.5 are not committed;
    // their node index (EPI_LEVEL) or point number (EPI_STORE) is appended to
    // recheck[] for re-evaluation in FP32.  Null recheck: commit everything.
    int* recheck;
    unsigned int* recheck_count;
    float margin;
};

// --- gather.cu -------------------------------------------------------------
// X[p][0 .. ldx) = [Phi(map0), Phi(map1) (if C1 > 0), z_in, 0 ...] for the
// points p in [p0, p0 + m).
cudaError_t launch_gather(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                          const Map& map0, const Map& map1, float* X, int ldx,
                          cudaStream_t stream);

// *out = max(*out, max_i |p[i]|) with *out holding float bits.
cudaError_t launch_amax(const float* p, int64_t n, unsigned int* out, cudaStream_t stream);
// Same rows in BF16 (the tensor-core MLP's A operand); ldx a multiple of 8.
cudaError_t launch_gather_bf16(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                               const Map& map0, const Map& map1, __nv_bfloat16* X, int ldx,
                               cudaStream_t stream);

// --- mlp_f32.cu ------------------------------------------------------------
// Out[M][N] = lrelu(A1[M][K1] W[:, :K1]^T + A2[M][K2] W[:, K1:]^T + b);
// K1, K2 multiples of 8; N a multiple of 4; ld* multiples of 4.  Batches of
// at most kSplitMaxM points use split-K over `part`, a scratch array of
// splitk_slices(K1, K2) * M * N floats (null: always the big-tile kernel).
constexpr int kSplitMaxM = 2048;
int splitk_slices(int K1, int K2);
// m_dev (optional): device-resident row count, at most M; then M is only
// the capacity (the slice stride of part) and the split-K kernels are used.
cudaError_t launch_sgemm_bias_lrelu(int M, int N, const float* A1, int lda1, int K1,
                                    const float* A2, int lda2, int K2, const float* W, int ldw,
                                    const float* bias, float slope, float* Out, int ldo,
                                    cudaStream_t stream, float* part,
                                    const unsigned int* m_dev = nullptr);

// Last layer (n_out <= 4 outputs) plus activation and epilogue, one warp per point.
cudaError_t launch_last_layer(int64_t p0, int64_t M, int n_out, const float* A1, int lda1, int K1,
                              const float* A2, int lda2, int K2, const float* W, int ldw,
                              const float* bias, const Epilogue& epi, cudaStream_t stream,
                              const unsigned int* m_dev = nullptr);

// Last layer reading BF16 activations (A1 = h, A2 = x rows), FP32 weights.
cudaError_t launch_last_layer_bf16(int64_t p0, int64_t M, int n_out, const __nv_bfloat16* A1,
                                   int lda1, int K1, const __nv_bfloat16* A2, int lda2, int K2,
                                   const float* W, int ldw, const float* bias, const Epilogue& epi,
                                   cudaStream_t stream, const unsigned int* m_dev = nullptr);

// --- mlp_tc.cu -------------------------------------------------------------
// One hidden layer on the tensor cores (tcgen05, BF16 in, FP32 accumulate):
// out[M][N] = lrelu([A1 | A2] W^T + b) in BF16.  A1 (nk1 K-blocks of 64)
// and A2 (nk2 K-blocks) are 2-D tensor maps over BF16 rows, W a tensor map
// over [N][64 (nk1 + nk2)] BF16; box 64 x 128 for A, 64 x BN for W, all
// with the 128-byte swizzle.  N a multiple of BN (64, 128 or 256).
// The last layer fused into the epilogue of the last hidden tensor-core layer
// (possible when one tile spans the hidden width and the last layer reads
// only h): out = epilogue(W h + b) per row, h rounded to BF16 as stored.
struct FuseLast {
    const float* W;     // [n_out][ldw] FP32
    int ldw;
    const float* bias;
    int n_out;          // <= 4
    int64_t p0;         // point number of the batch's first row
    Epilogue epi;
};

// Operand and output types of one tensor-core layer.
enum TcMode : int {
    TC_BF16 = 0,       // BF16 A and W, BF16 out
    TC_BF16_E4M3 = 1,  // BF16 A and W, E4M3 out (multiplied by out_scale first)
    // Mixed layers: the A1 segment (the previous layer's output) in E4M3
    // against E4M3 weights (kind::f8f6f4), then the A2 segment (the input
    // rows x) in BF16 against BF16 weights (kind::f16), both into the same
    // FP32 accumulator, which the epilogue multiplies by colscale[n].  W is a
    // byte matrix: per row the E4M3 part (nk1 x 128 bytes), then the BF16
    // part (nk2 x 64 values), each 128-byte K-block one TMA box.
    TC_MIX_E4M3 = 2,   // E4M3 out (multiplied by out_scale first)
    TC_MIX_BF16 = 3,   // BF16 out
};
struct TcLayerArgs {
    const CUtensorMap* tmA1;
    const CUtensorMap* tmA2;
    const CUtensorMap* tmW;
    const CUtensorMap* tmO;       // optional: BF16 output [rows][N], box 32 x 32, 64-byte
                                  // swizzle (the epilogue then stores with TMA)
    int nk1, nk2, M, N, BN;       // nk1, nk2: 128-byte K-blocks of the two A segments
    int klast;                    // MMA steps (16 BF16 values each) of the last K-block
                                  // that hold real columns, 1..4 (0: all 4); the rest of
                                  // that block is zero padding in both operands
    int pair;                     // 1: CTA-pair form (BN = 256, TC_BF16, no fuse); tmW's
                                  // box is then 128 rows (each CTA loads half of a tile's W)
    const float* bias;
    float slope;
    void* out;                    // [M][ldo] of the mode's output type
    int ldo;
    unsigned int* err;
    const unsigned int* m_dev;   // optional device-resident row count (<= M)
    const FuseLast* fuse;        // optional: last layer fused (requires N == BN, TC_BF16)
    int mode;                    // TcMode
    const float* colscale;       // E4M3 modes: accumulator scale per output column
    float out_scale;             // E4M3 outputs: multiplied by this before rounding
};
cudaError_t launch_tc_linear(const TcLayerArgs& a, cudaStream_t stream);
// Set the tensor-core kernels' attributes on the current device (before a
// stream capture: launches inside a capture then make no attribute calls).
cudaError_t tc_prepare();

// --- mlp_x3.cu ---------------------------------------------------------------
// FP32-accurate hidden layers on the tensor cores for small batches: each
// FP32 value v is held as two TF32 values, hi = tf32(v) and
// lo = tf32(v - hi), and each product as a_hi b_hi + a_hi b_lo + a_lo b_hi.
//
// v rounded to TF32 (10 explicit mantissa bits, ties away from zero): the
// 13 low bits of the FP32 encoding cleared after adding half of their range
// (sign-magnitude, so the same for both signs).  Finite v only.
__host__ __device__ __forceinline__ float tf32_round(float v) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
#else
    uint32_t u;
    memcpy(&u, &v, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
#endif
}

constexpr int kX3MaxUnits = 256;   // work units of one launch that hold split-K partials
constexpr int kX3Tile = 128;       // points and neurons per work unit

// The whole network over a batch in one cooperative launch: the gather into
// the input-row planes, then every hidden layer over [H | X] (split planes: a
// row of K values is stored as 2 K floats, the hi values then the lo values),
//   h_l[p][n] = lrelu(b[n] + sum_k W[n][k] [h_{l-1} | x][p][k]),
// written back as hi/lo planes [rows][2 N], the last hidden layer (N = 128)
// handed to the one-output last layer (FP32) and its epilogue.  A grid-wide
// barrier (bounded waits) separates the phases.
constexpr int kX3MaxLayers = 4;
constexpr int kX3CtrWords = 2 * kX3MaxUnits + kX3MaxLayers + 2;
struct X3NetLayer {
    CUtensorMap tmW;             // [N][2 KP] FP32, box 32 x 128, 128-byte swizzle
    CUtensorMap tmH;             // [rows][2 KH] previous layer's planes, box 32 x 32 (l >= 1)
    int nk1, nk2;                // 32-value K-blocks from H, then from X
    int KH, KX, KP;              // lo-plane column offsets (KP = KH + KX)
    int N;                       // neurons, a multiple of 128
    const float* bias;
    float* out;                  // [rows][2 N] (unused by the last hidden layer)
};
struct X3NetArgs {
    X3NetLayer L[kX3MaxLayers];
    CUtensorMap tmX;             // [rows][2 KX] input-row planes, box 32 x 32
    int nl;                      // hidden layers
    int M;                       // points (a capacity with m_dev)
    const unsigned int* m_dev;   // optional device-resident point count (<= M)
    float slope;
    // gather: points p0 .. p0 + count - 1 of src into X
    PointSrc src;
    int64_t p0;
    Calib calib;
    Map map0, map1;
    float* X;
    int KX;
    FuseLast fl;                 // the last layer (n_out = 1) and its epilogue
    float* part;                 // [kX3MaxUnits][128][128] split-K partial tiles
    unsigned int* ctr;           // [2][kX3MaxUnits] arrivals and departures per tile, then
                                 // [kX3MaxLayers + 2] grid barrier counters per phase and
                                 // CTA departures (kX3CtrWords); all zero at launch and
                                 // zero again at exit
    unsigned int* err;
    unsigned int wait_extra;     // test hook (0): the split-K arrival wait needs this many
                                 // arrivals more than there are, so it runs out
};
// One cooperative launch (every CTA resident: one per SM).
cudaError_t launch_x3_net(const X3NetArgs& a, cudaStream_t stream);
cudaError_t x3_prepare();
// Tensor map of an FP32 matrix [rows][cols] (row stride in bytes), box
// box_cols x box_rows, 128-byte swizzle.
bool x3_encode_2d(void* map, const void* base, uint64_t cols, uint64_t rows,
                  uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows);

// --- mlp_chain.cu ------------------------------------------------------------
// All hidden layers of one BF16 batch in one persistent launch (rows move
// through the layers in groups; per-row-block counters order a layer after
// the one it reads).
constexpr int kChainMaxLayers = 4;
constexpr int kChainBiasFloats = 2048;   // sum of the hidden widths
struct ChainLayer {
    CUtensorMap tmA1;       // layer l-1's output [rows][K1] (l >= 1, nk1 > 0)
    CUtensorMap tmA2;       // the input rows x [rows][ldx]
    CUtensorMap tmW;        // [N][Kw] BF16, box BN x 64
    int nk1, nk2, N, BN;    // 128-byte K-blocks of the two segments; BN | N, BN <= 256
    int klast;              // as in TcLayerArgs
    const float* bias;      // [N]
    __nv_bfloat16* out;     // [rows][ldo] (unused by a layer carrying the fused last layer)
    int ldo;
};
struct ChainArgs {
    ChainLayer L[kChainMaxLayers];
    int boff[kChainMaxLayers];   // offsets of the layers' biases in shared memory
    int nl;
    int M;                       // rows (capacity when m_dev is given)
    const unsigned int* m_dev;   // optional device-resident row count (<= M)
    unsigned int* err;
    unsigned int* dep;           // [nl][max_mb] tile-part counters, zero at launch
    unsigned int* next_tile;     // = dep + nl * max_mb: the tile counter
    unsigned int* done;          // = next_tile + 1: CTAs finished (the last one zeroes all)
    int max_mb;                  // >= ceil(M / 128)
    int group;                   // 128-row blocks per row group
    int lag;                     // steps between a layer and the next on one row group
    float slope;
    FuseLast fl;                 // fl.n_out > 0: the last layer rides in layer nl-1
};
// Sets the kernel's attributes on the current device (call before a capture).
cudaError_t chain_prepare();
// CTAs of one chained launch (one per SM; 0 before chain_prepare).
int chain_grid();
// Launches one CTA per SM (programmatic dependent launch); the counters must
// be zero, and are zero again when the kernel ends.
cudaError_t launch_tc_chain(const ChainArgs& a, cudaStream_t stream);

// Encode a 2-D BF16 tensor map (128-byte swizzle, zero fill out of bounds).
bool tc_encode_2d_bf16(void* map, const void* base, uint64_t cols, uint64_t rows,
                       uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows);
// A layer's BF16 output as the epilogue's TMA stores see it: box 32 x 32,
// 64-byte swizzle.
bool tc_encode_2d_bf16_out(void* map, const void* base, uint64_t cols, uint64_t rows,
                           uint64_t row_stride_bytes);
// The same for 8-bit elements (E4M3 stored as bytes).
bool tc_encode_2d_u8(void* map, const void* base, uint64_t cols, uint64_t rows,
                     uint64_t row_stride_bytes, uint32_t box_cols, uint32_t box_rows);

// --- train.cu --------------------------------------------------------------
// C[m][n] (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m a_m + k a_k],
// B(k, n) = B[k b_k + n b_n], C row stride c_m; the reduction is split into
// k_slices slices accumulated with atomicAdd (C must then start at zero).
cudaError_t launch_gemm_strided(int M, int N, int K, const float* A, int64_t a_m, int64_t a_k,
                                const float* B, int64_t b_k, int64_t b_n, float* C, int64_t c_m,
                                int k_slices, int accumulate, cudaStream_t s);
cudaError_t launch_bias_lrelu(int M, int N, float* Z, int ld, const float* bias, float slope,
                              cudaStream_t s);
// g[b] = (sigmoid(logit[b] + bias) - y[b]) / B; *loss += mean BCE;
// per_loss[b] = sample b's BCE (if non-null).
cudaError_t launch_bce_grad(int B, const float* logit, const float* bias, const float* y, float* g,
                            double* loss, cudaStream_t s, float* per_loss = nullptr);
// Point OHEM: B indices drawn with probability proportional to w[0 .. m)
// (cdf: m doubles, sums: ohem_scan_blocks(m) doubles of scratch).
int64_t ohem_scan_blocks(int64_t m);
cudaError_t launch_ohem_sample(const float* w, int64_t m, double* cdf, double* sums,
                               uint64_t seed, uint32_t step, int B, int* idx, cudaStream_t s);
cudaError_t launch_gather_rows(const float* x, const float* y, int ld, const int* idx, int B,
                               float* xb, float* yb, cudaStream_t s);
// w[idx[b]] = 1 / (exp(-loss[b] / alpha) + beta) (Eq. 6).
cudaError_t launch_ohem_update(float* w, const int* idx, const float* loss, int B, float alpha,
                               float beta, cudaStream_t s);
cudaError_t launch_lrelu_backward(int64_t n, float* dH, const float* H, float slope,
                                  cudaStream_t s);
cudaError_t launch_adam(int64_t n, float* w, const float* g, float* m, float* v, float lr, int t,
                        cudaStream_t s);
cudaError_t launch_fill(int64_t n, float* p, float value, cudaStream_t s);

// --- localize.cu -----------------------------------------------------------
__host__ __device__ inline int row_words_of(int N) { return (N + 1 + 31) / 32; }
__host__ __device__ inline int64_t words_of(int N) {
    return (int64_t)(N + 1) * (N + 1) * row_words_of(N);
}

// Level set-up from the binarized coarse level (N/2 cells): tentative bits,
// candidate bits; clears eval, conf0 and the working bits (= tentative).
// Several frames: `slots` of them, bitsets cslot (coarse) / fslot (fine)
// words apart.
// One frame: cands (optional) += the candidates' count, zero (optional) = 0.
cudaError_t launch_classify(const uint32_t* coarse_bin, int N, uint32_t* cand, uint32_t* tent,
                            uint32_t* bin, uint32_t* eval, uint32_t* conf0, cudaStream_t stream,
                            int slots = 1, int64_t cslot = 0, int64_t fslot = 0,
                            unsigned long long* cands = nullptr, unsigned int* zero = nullptr);

// Graph form: the conflict loop's decision (launch_loop_control's, on the
// kernel's own list count) taken by the last CTA of the kernel that builds
// the frontier.  done: a CTA counter, zero between launches.  done = null:
// no decision.
struct LoopTail {
    cudaGraphConditionalHandle h;
    unsigned int* done;
    unsigned int cap;
    unsigned int* rounds;
    int count_round;
    int max_rounds;
    unsigned int* err;
};

// Up to kMax device spans of 32-bit words that a kernel zeroes on the way
// (in the graph forms, in place of memset nodes before it).
struct ZeroSpans {
    static constexpr int kMax = 3;
    unsigned int* p[kMax];
    uint32_t words[kMax];
};
// Level-0 set-up: everything empty except eval = all nodes; the spans of
// `zero` (optional) are zeroed too.
cudaError_t launch_dense_setup(int N, uint32_t* cand, uint32_t* tent, uint32_t* bin,
                               uint32_t* eval, uint32_t* conf0, cudaStream_t stream,
                               int slots = 1, int64_t fslot = 0,
                               const ZeroSpans* zero = nullptr);

// sel = dilate26(src) & ~eval; eval |= sel; clear[w] = 0 (if non-null);
// append the node indices of sel to list at *count.
// Several frames: one list for all, keys frame * slot_nodes + node.
cudaError_t launch_dilate_select(const uint32_t* src, uint32_t* eval, uint32_t* clear, int N,
                                 int* list, unsigned int* count, cudaStream_t stream,
                                 int slots = 1, int64_t fslot = 0, int64_t slot_nodes = 0,
                                 const LoopTail* tail = nullptr);

// src & ~eval (no dilation); eval |= it; append the node indices to list.
cudaError_t launch_select(const uint32_t* src, uint32_t* eval, int N, int* list,
                          unsigned int* count, cudaStream_t stream);

// Threshold subdivision (octree baseline of Fig. 3) of an N-cell level from
// the dense continuous values of the N/2-cell level: values = the tri-linear
// interpolation of the coarse values; tent = bin = (values >= 1/2);
// eval = the nodes whose coarse corners deviate from their mean by more
// than thr, also appended to list at *count; conf0 cleared.
cudaError_t launch_threshold_select(const float* coarse, int N, float thr, float* values,
                                    uint32_t* tent, uint32_t* bin, uint32_t* eval,
                                    uint32_t* conf0, int* list, unsigned int* count,
                                    cudaStream_t stream);

// Graph form: set the conditional handle to (*count > 0) within capacity
// and round limits (count_round: this decision starts a conflict round).
cudaError_t launch_loop_control(cudaGraphConditionalHandle h, const unsigned int* count,
                                unsigned int cap, unsigned int* rounds, int count_round,
                                int max_rounds, unsigned int* err, cudaStream_t stream);
// Sparse conflict expansion (Sec. 3.2's conflict rounds): for every key in
// clist[0 .. *ccount) (frame * key_div + node of an N-cell level), every
// 26-neighbour inside the grid whose evaluated bit was clear gets it set and
// is appended to list at *count (at most cap; beyond it kErrCapacity).  The
// same set as dilate26(conflicts) & ~evaluated, in work proportional to the
// conflicts.  Launched for up to max_c conflicts (a device-resident count).
// Frame stream: sv gives every key's slot level and evaluated bitset (N and
// eval are then unused) and slot_count[slot] counts the keys appended; with
// list_f, the keys of slots at their finest level go to list_f at *count_f
// instead (each list at most cap).
cudaError_t launch_expand_conflicts(const int* clist, const unsigned int* ccount,
                                    unsigned int max_c, int N, uint32_t* eval, int64_t key_div,
                                    int64_t slot_words, int* list, unsigned int* count,
                                    unsigned int cap, unsigned int* err, cudaStream_t stream,
                                    const SlotView* sv = nullptr,
                                    unsigned int* slot_count = nullptr, int* list_f = nullptr,
                                    unsigned int* count_f = nullptr,
                                    const LoopTail* tail = nullptr);

// Frame stream: everything the scheduler kernel reads and writes.
struct StreamCtl {
    unsigned int next_frame;          // the queue's next frame
    unsigned int rounds;              // rounds run
    unsigned long long rechecked;     // MIXED: evaluations redone in FP32, all frames
    unsigned long long fallback;      // surrogate: evaluations redone by f_O, all frames
    unsigned long long t_start;       // device clock (ns) of the first admission
    unsigned int render_rounds;       // rounds in which a slot rendered
    unsigned int err;                 // the error word when the loop stopped
    unsigned int colour_passes;       // deferred colour passes inside the loop
};
struct StreamArgs {
    SlotView* sv;                     // [S] this round's views (written here)
    StreamSlot* st;                   // [S] persistent slot state
    StreamFrameStats* fs;             // [F]
    StreamCtl* ctl;
    unsigned int* pend_eval;          // [S] keys of the slot in the round's evaluation
    unsigned int* pend_next;          // [S] keys its conflict expansion queued
    unsigned long long* cands;        // [S] candidates its selection counted
    int S, F, L, n0, max_rounds;
    unsigned int max_total_rounds;    // beyond it: kErrNotConverged
    // the slots' arrays: slot s at s * slot_words / slot_nodes / slot_top
    uint32_t* cand;
    uint32_t* tent;
    uint32_t* bin0;
    uint32_t* bin1;
    uint32_t* eval;
    uint32_t* conf;
    float* values;
    int* top;
    int64_t slot_words, slot_nodes, slot_top;
    // the frames' inputs (copied to a slot's entries when it takes a frame)
    const Map* frame_maps0;
    const Map* frame_maps1;           // may be null
    const Calib* frame_calibs;
    Map* slot_maps0;
    Map* slot_maps1;
    Calib* slot_calibs;
    // the frames' outputs, frame f at f * npix pixels / f * out_words words
    float* depth;
    float* rgb;
    uint8_t* mask;
    uint32_t* bits_out;
    int64_t npix, out_words;
    unsigned int* err;
    cudaGraphConditionalHandle h;     // the loop's condition: another round
    int init;                         // 1: reset the stream and admit its first frames
};
// One thread: every slot's scheduling step (stream_step), the views of the
// next round, and the loop condition (another round while a slot holds a
// frame or the queue holds one, and no error is latched).
cudaError_t launch_stream_sched(const StreamArgs& a, cudaStream_t stream);
// h = (*count > 0).
cudaError_t launch_set_if(cudaGraphConditionalHandle h, const unsigned int* count,
                          cudaStream_t stream);
// Frame stream: h = (*hits + npix x the slots rendering this round > cap),
// i.e. the hit list could not take this round's renders; *passes += h.
cudaError_t launch_colour_cond(cudaGraphConditionalHandle h, const unsigned int* hits,
                               const SlotView* sv, int S, int64_t npix, unsigned int cap,
                               unsigned int* passes, cudaStream_t stream);

// Frame stream: the level set-up (op START: level 0 with every node
// evaluated; op ADVANCE: the classify step) of every slot whose round op asks
// for one, and the first selection of those slots' level (START: every node;
// ADVANCE: the candidates' 26-ring), appended as keys slot * slot_nodes +
// node at *count (at most cap; beyond it kErrCapacity); pend[slot] += keys
// queued, cands[slot] += boundary candidates.  With list_f, a slot at its
// finest level appends to list_f at *count_f instead.  N_fine sizes the grid.
cudaError_t launch_stream_setup(const SlotView* sv, int slots, int N_fine, cudaStream_t stream);
cudaError_t launch_stream_select(const SlotView* sv, int slots, int N_fine, int64_t slot_nodes,
                                 int* list, unsigned int* count, unsigned int cap,
                                 unsigned int* err, unsigned int* pend,
                                 unsigned long long* cands, cudaStream_t stream,
                                 int* list_f = nullptr, unsigned int* count_f = nullptr);

// *dst += *src; capacity error bit if *src > cap.
cudaError_t launch_accumulate(unsigned long long* dst, const unsigned int* src, unsigned int cap,
                              unsigned int* err, cudaStream_t stream);
// *sticky |= *err (one thread): an enqueued frame's error kept for the host.
cudaError_t launch_latch_err(const unsigned int* err, unsigned int* sticky, cudaStream_t stream);
// A conflict round's start in one launch: the round's size c = *next (the
// frontier count the previous selection or expansion appended to) becomes
// *count, the batch size its passes read, and *next = 0 for the next
// expansion; *evals += c (capacity error bit if above cap), *zero = 0.
struct RoundStart {
    unsigned long long* evals;
    unsigned int cap;
    unsigned int* err;
    unsigned int* zero;
    unsigned int* next;
};
cudaError_t launch_round_start(unsigned int* count, const RoundStart& rs, cudaStream_t stream);

// Population count of a bitset (for statistics) added into *count.
// Several frames: count[f] += popcount of frame f's bitset.
cudaError_t launch_popcount(const uint32_t* bits, int64_t words, unsigned long long* count,
                            cudaStream_t stream, int slots = 1, int64_t fslot = 0);

// --- mlp_fused.cu ----------------------------------------------------------
// The whole network in FP32 for a small (or device-sized) batch in one
// launch: clusters of 8 CTAs, one 16-point tile per cluster at a time.
constexpr int kFusedMaxLayers = 8;
struct FusedLayer {
    const float* W;   // [n_out][ldw]: K1 columns on h_{l-1}, then K2 on x
    const float* b;
    int n_out, K1, K2, ldw;
};
struct FusedNet {
    FusedLayer L[kFusedMaxLayers];
    int nl, ldx, max_hidden;
    int d_in;         // input row width before the padding to ldx
    float slope;
};
// Whether the network's shape fits the fused kernel.
bool fused_ok(const FusedNet& n);
// The cluster sizes the fused kernel can use for a network (FusedPlan,
// switch_index.cuh).
FusedPlan fused_plan(const FusedNet& n);
// Points p0 .. p0 + m - 1 of `src` (src.count: a device-resident m, at most
// m).  cl = 0: the cluster size of fewest latency-weighted rounds for a
// host-known m, 8-CTA clusters for a device-resident one; else that size
// (one of the plan's).
cudaError_t launch_mlp_fused(const FusedNet& net, const PointSrc& src, int64_t p0, int64_t m,
                             const Calib& calib, const Map& map0, const Map& map1,
                             const Epilogue& epi, cudaStream_t stream, int cl = 0);
// Graph form: sets the switch `h` to the index (in `plan`) of the cluster
// size the device-resident batch size c = min(*count, cap) calls for; to
// plan.n when x3_lo < c <= x3_hi (the split-TF32 body, if the switch has
// one: x3_hi > 0); to a value past every body (no branch) when c is 0.
// stat (optional): *stat += *count, capacity error bit in *err when *count
// exceeds stat_cap (launch_accumulate's work, in the same launch).
cudaError_t launch_fused_switch(cudaGraphConditionalHandle h, const FusedPlan& plan,
                                const unsigned int* count, unsigned int cap, cudaStream_t stream,
                                unsigned int x3_lo = 0, unsigned int x3_hi = 0,
                                unsigned int grid_hi = 0, unsigned long long* stat = nullptr,
                                unsigned int stat_cap = 0, unsigned int* err = nullptr);
// Graph form, one evaluation batch of the MIXED forms as one switch `h` of
// nt + 1 bodies: a device-resident batch of c points, 1 <= c <= threshold,
// selects an FP32 body (body 0 when single, else launch_fused_switch's index
// for min(c, cap)); c > threshold selects body nt (the tensor-core pass);
// c = 0 none.  rs (optional): the batch is a conflict round; c is first
// moved from *rs->next into *count with round_start's statistics.  *zero = 0
// (optional: the tensor-core body's re-check queue length).
cudaError_t launch_batch_switch(cudaGraphConditionalHandle h, const FusedPlan& plan,
                                unsigned int* count, unsigned int cap, unsigned int threshold,
                                int nt, bool single, unsigned int x3_lo, unsigned int x3_hi,
                                unsigned int grid_hi, const RoundStart* rs, unsigned int* zero,
                                cudaStream_t stream);

// --- mlp_grid.cu -----------------------------------------------------------
// The whole network in FP32 for a batch of at most kGridMaxRows points in one
// cooperative launch over every SM: each hidden layer's neurons split over
// the CTAs, a bounded grid barrier between layers (mlp_grid.cu).
constexpr int kGridMaxRows = 256;    // points per launch
constexpr int kGridMaxCtas = 256;    // CTAs per launch (one per SM)
constexpr int kGridMaxGroups = 64;   // point groups per launch
// [kFusedMaxLayers] grid barrier counters (one per hidden layer), [1] CTA
// departures, [kGridMaxGroups] last-layer arrivals per point group
constexpr int kGridCtrWords = kFusedMaxLayers + 1 + kGridMaxGroups;
struct GridArgs {
    FusedNet net;
    PointSrc src;                // points p0 .. p0 + min(M, *m_dev) - 1
    int64_t p0;
    int M;                       // <= kGridMaxRows
    const unsigned int* m_dev;   // device-resident batch size, or null
    Calib calib;
    Map map0, map1;
    Epilogue epi;
    float* H[2];                 // [kGridMaxRows][max_hidden] hidden activations, ping-pong
    float* part;                 // [kGridMaxRows][kGridMaxCtas][4] last-layer partial sums
    unsigned int* ctr;           // kGridCtrWords, zero at launch and again at exit
    unsigned int* err;           // device error word (kErrTimeout, kErrCapacity)
    unsigned int wait_extra;     // test hook (0): the grid barrier needs this many more arrivals
};
// Whether the network's shape fits the kernel (hidden widths and ldw
// multiples of 4, 16-byte aligned weights, at most 4 outputs, >= 1 hidden layer).
bool grid_ok(const FusedNet& n);
// The largest batch one launch takes for this network on the current device
// (0: the network does not fit or the device cannot hold the grid).
int grid_max_rows(const FusedNet& n);
cudaError_t launch_mlp_grid(const GridArgs& a, cudaStream_t stream);

// --- cbn.cu --------------------------------------------------------------
// The CBN + SoftZ occupancy network (Appendix, Eq. 7 and Eq. 8) in FP32, with
// each block's running statistics folded into the linear layer before it.
// Clusters of kCbnCluster CTAs; CTA r of a cluster owns channels
// [r Kc, (r + 1) Kc), Kc = K / kCbnCluster, and its weight slices are
// contiguous.
constexpr int kCbnCluster = 8;
constexpr int kCbnPrefetch = 12;   // float4 per thread: a slice holds <= 12 x 256 float4
struct CbnF32 {
    const float* WzT;    // [n_z][K]: s_0 Wz, transposed
    const float* bz;     // [K]: s_0 (bz - mu_0)
    const float* GS;     // nb x kCbnCluster x [C][2Kc]: gamma then beta columns of the slice
    const float* g0S;    // nb x kCbnCluster x [2Kc]: gg then gb of the slice
    const float* WS;     // (nb - 1) x kCbnCluster x [K][Kc]: s_{i+1} W_i, the slice's outputs
    const float* blS;    // (nb - 1) x kCbnCluster x [Kc]: s_{i+1} (b_i - mu_{i+1})
    const float* wlast;  // [K]
    const float* blast;  // [4] (one value, padded)
    int C, n_z, K, nb;
};
bool cbn_f32_ok(const CbnF32& net);
// Kernel attributes and the co-resident cluster count, set on the current
// device (before a stream capture).
cudaError_t cbn_f32_prepare(const CbnF32& net);
// Occupancy logits of points 0 .. m - 1 of `src` (src.count: a device-resident
// m) through the level / store epilogue; the feature is map's bilinear
// sample, the depth its projection.
cudaError_t launch_cbn_f32(const CbnF32& net, const PointSrc& src, int64_t m, const Calib& calib,
                           const Map& map, const Epilogue& epi, cudaStream_t stream);

// --- cbn_tc.cu -------------------------------------------------------------
// The CBN + SoftZ network on tcgen05 tensor cores (BF16 operands, FP32
// accumulation): one persistent kernel runs all blocks per 128-point tile.
struct CbnTcArgs {
    const float* zbuf;    // [M] projected depth of each row (FP32)
    const float* WzT;     // FP32 folded input layer, as CbnF32
    const float* bz;
    const float* g0;      // nb x [2K]: [gg; gb]
    const float* bl;      // (nb - 1) x [K]
    const float* wlast;   // [K]
    const float* blast;   // [4]
    int C, n_z, K, nb;
    int M;                // rows of this pass (with m_dev: the capacity)
    const unsigned int* m_dev;   // optional device-resident row count (<= M)
    int64_t p0;           // point number of row 0 (for the epilogue)
    unsigned int* err;    // device error word
    Epilogue epi;
};
struct CbnTcMaps {
    const CUtensorMap* tmX;   // BF16 feature rows [rows][C], box 64 x 128
    const CUtensorMap* tmG;   // BF16 [nb 2K][C] = [Gg; Gb] per block, box 64 x 2K
    const CUtensorMap* tmW;   // BF16 [(nb - 1) K][K] folded linear layers, box 64 x K
};
bool cbn_tc_ok(int C, int K, int nb);
// Kernel attributes on the current device (before a stream capture).
cudaError_t cbn_tc_prepare(int C, int K, int nb);
// X[r][0 .. C) = BF16 feature of point p0 + r, z[r] = its projected depth
// (src.count: a device-resident m).
cudaError_t launch_cbn_gather(const PointSrc& src, int64_t p0, int64_t m, const Calib& calib,
                              const Map& map, __nv_bfloat16* X, int C, float* z,
                              cudaStream_t stream);
cudaError_t launch_cbn_tc(const CbnTcMaps& maps, const CbnTcArgs& args, cudaStream_t stream);

// --- render.cu -------------------------------------------------------------
struct RenderArgs {
    int width, height;
    int N, row_words;
    const float* values;
    const uint32_t* eval;
    const uint32_t* bin;
    float bg[3];
    float* depth;         // may be null
    float* rgb;           // may be null
    uint8_t* mask;        // may be null
    float* hit_xyz;       // [width*height][3] surface points of hits
    int* hit_pix;         // pixel index per hit
    unsigned int* hit_count;   // zeroed by the launch (before any hit is appended)
    int* top;             // [2][(N+1)^2] scratch per frame: highest non-empty depth node
                          // per column, then N - the lowest
    // Several frames (lockstep form): frame f's volume starts f slot_nodes
    // values / f slot_words words further, its outputs f width*height pixels
    // further, and its hits carry pixel keys f width*height + pixel.
    int slots;            // 0 or 1: one frame
    int64_t slot_nodes, slot_words;
};
cudaError_t launch_render_rays(const RenderArgs& a, cudaStream_t stream);
// Frame stream: the render of every slot whose round op is RENDER, from the
// slot's arrays into its frame's outputs (SlotView); a supplies the image
// size, the background and the hit list, whose keys are frame * width *
// height + pixel.  N_fine sizes the grid.
cudaError_t launch_stream_render(const SlotView* sv, int slots, int N_fine, const RenderArgs& a,
                                 cudaStream_t stream);

// View-culled final level (Sec. 3.2): the render's pixel columns at the N_f =
// 2 N_c depth nodes of the level after the last localized one (N_c cells,
// binarized bits `bin`).  Per pixel the binarized level is upsampled
// tri-linearly along the column (tentative T); nodes behind the nearest
// T = 1 node are shadow nodes; the non-shadow nodes with 0 < T < 1 are the
// candidates.
struct CullArgs {
    int width, height;     // square images only: width == height
    int Nc, row_words;     // the localized level
    const uint32_t* bin;
    int* list;             // candidates' keys pixel (N_f + 1) + k
    unsigned int* count;   // appended at *count
    unsigned int cap;      // list capacity: beyond it the error word gets kErrCapacity
    unsigned int* err;
    const float* values;   // [width*height][N_f + 1]: the candidates' occupancies
    float bg[3];
    float* depth;          // may be null
    float* rgb;            // may be null
    uint8_t* mask;         // may be null
    float* hit_xyz;
    int* hit_pix;
    unsigned int* hit_count;
    int* top;              // [(Nc+1)^2] scratch: highest set depth node per column
};
// Candidates of every pixel into list (warp-aggregated).
cudaError_t launch_cull_select(const CullArgs& a, cudaStream_t stream);
// Second argmax over T and the evaluated candidates, the crossing, outputs
// and the hit list for the colour MLP.
cudaError_t launch_cull_final(const CullArgs& a, cudaStream_t stream);

}  // namespace pifu
