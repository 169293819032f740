// Host-side internals of libpifu shared by its translation units: the
// context, the device forms of the networks, workspaces, and the helpers
// the entry points are built from.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pifu.h"
#include "pifu_internal.h"

#include <cuda_fp8.h>

namespace pifu_host {

using namespace pifu;


constexpr int kMaxLevels = 8;
constexpr int kMaxFine = 512;
constexpr int64_t kChunk = 65536;    // points per FP32 MLP pass (bounds its activation workspace)
constexpr int64_t kChunkTC = 1 << 20; // points per tensor-core MLP pass (a whole 512^3 level list)
constexpr int64_t kTcRowsMax = 1 << 22; // device-sized batches of a lockstep frame batch
constexpr int kMaxBatch = 64;           // frames of a lockstep batch
constexpr int64_t kRecheckCap = 8192; // graph form: FP32 re-checks per batch (split-K path)
constexpr int64_t kFusedMaxM = 2048;   // host-sized FP32 batches up to this size: fused kernel
constexpr int64_t kTinyBatch = 256; // mixed precision: batches this small run in FP32
constexpr int64_t kX3Rows = 16384;   // points per pass of the split-TF32 network (its workspace rows)
constexpr int64_t kGridPreferRows = 64;  // FP32 passes of at most this many points (and
                                         // at most DevNet::grid_rows) run the whole-GPU
                                         // network, where its latency is the lowest
constexpr int64_t kX3MinRows = 192;  // FP32 passes of more points run it (fewer: the one-launch
                                     // SIMT network, whose latency is lower there)

struct DevLayer {
    int n_out = 0;
    int K1 = 0;     // columns reading h_{l-1}
    int K2 = 0;     // columns reading x (padded to the gather's row width), 0 if none
    int ldw = 0;    // K1 + K2
    int fan_in = 0; // unpadded fan-in (algorithmic K)
    float* W = nullptr;
    float* b = nullptr;
};

// BF16 tensor-core form of a hidden layer: W as [n_out][Kw] BF16 with the x
// segment zero-padded to whole 64-column K-blocks, and its tensor maps.
struct TcLayer {
    __nv_bfloat16* W = nullptr;
    int Kw = 0, nk1 = 0, nk2 = 0, BN = 0;
    int klast = 4;        // the 16-value MMA steps of the last K-block that reach a real column
    bool pair = false;    // CTA-pair form (BN = 256; tmW's box is then 128 rows)
    CUtensorMap tmW{};
    CUtensorMap tmA1{};   // the previous layer's BF16 output (l >= 1)
    CUtensorMap tmO{};    // this layer's BF16 output, for the epilogue's TMA stores
    bool tmO_ok = false;
};

// FP8 form of one of f_O's leading wide hidden layers.  Layer 0 keeps the
// BF16 operands of the tensor-core form and rounds its output to E4M3
// (multiplied by out_scale = 1 / s of the next layer's input).  A later layer
// reads that E4M3 output against E4M3 weights W_h / s_w[n] (s_w[n]: the
// per-output-channel absolute maximum / 448) and the BF16 input rows against
// BF16 weights W_x / (s_a s_w[n]), into one FP32 accumulator that the
// epilogue multiplies by colscale[n] = s_w[n] s_a (s_a: the per-tensor scale
// of its E4M3 input).
struct Fp8Layer {
    bool bf16_in = false;        // layer 0: W and tmW are over the BF16 weights
    uint8_t* W = nullptr;        // later layers: [n_out][Kw] bytes, E4M3 h part then BF16 x part
    const void* Wmap = nullptr;  // the weights tmW covers
    float* colscale = nullptr;   // [n_out] (later layers)
    int Kw = 0, nk1 = 0, nk2 = 0, BN = 0;   // Kw: row width in the map's elements
    int klast = 4;                          // as in TcLayer
    float out_scale = 1.f;       // E4M3 output: 1 / s of the next layer's input
    CUtensorMap tmW{};
    CUtensorMap tmA1{};          // the previous layer's E4M3 output (layer >= 1)
};

// Split-TF32 form of a hidden layer (mlp_x3.cu): W as [n_out][2 KP] FP32,
// hi values then lo values, KP = KH + KX (the h part, then the x part
// zero-padded to 32 values), and its tensor maps.
struct X3Layer {
    float* W = nullptr;
    int KH = 0, KX = 0, KP = 0;
    CUtensorMap tmW{};
    CUtensorMap tmH{};   // the previous layer's output planes (l >= 1)
};

struct DevNet {
    int kind = 0;       // 0 occupancy (sigmoid), 1 colour (tanh01)
    int d_in = 0;
    int ldx = 0;        // gather row width: d_in rounded up to 8
    int ldx_tc = 0;     // BF16 tensor-core input row width: d_in rounded up to 64 (whole
                        // K-blocks, the padding zero), so no TMA box reads past a row
    float slope = 0.01f;
    int max_hidden = 0;
    std::vector<DevLayer> layers;
    bool tc_ok = false;             // shapes allow the tensor-core form
    std::vector<TcLayer> tc;        // hidden layers only
    // chained form (all hidden layers in one launch): shapes and buffers
    // allow it; chain_tmA1[l] reads layer l-1's output in its chain buffer
    bool chain_ok = false;
    std::vector<CUtensorMap> chain_tmA1;
    CUtensorMap tmX{};              // BF16 gather rows as the A operand
    // FP8 form (pifu_calibrate_fp8): the first f8.size() hidden layers
    bool f8_ok = false;
    std::vector<Fp8Layer> f8;
    float s_x = 0.f;                // per-tensor scale of the input rows (reported)
    uint64_t f8_version = 0;        // bumped by every calibration
    // split-TF32 form (the MIXED forms' FP32-accurate passes): hidden widths
    // multiples of 128, the last hidden one 128 wide, a one-output last layer
    // reading only it
    bool x3_ok = false;
    std::vector<X3Layer> x3;
    int x3_KX = 0;                  // x part of a plane row: d_in rounded up to 32
    CUtensorMap tmX3{};             // the input-row planes [kX3Rows][2 x3_KX]
    // whole-GPU FP32 form of small passes (mlp_grid.cu): the largest batch
    // one launch takes (0: not usable), set by ensure_x3
    int grid_rows = 0;
};

constexpr int kNetCbn = 2;   // DevNet.kind of the CBN + SoftZ occupancy network

// Device copy of the CBN + SoftZ occupancy network (statistics folded).
struct CbnDev {
    bool ready = false;
    std::vector<float*> bufs;   // every allocation, freed together
    CbnF32 f32{};
    const float* g0 = nullptr;   // nb x [2K] (tensor-core epilogue)
    const float* bl = nullptr;   // (nb - 1) x [K]
    // tensor-core form
    bool tc_ok = false;
    __nv_bfloat16* Gbf = nullptr;   // [nb 2K][C]
    __nv_bfloat16* Wbf = nullptr;   // [(nb - 1) K][K] (or a dummy row block when nb = 1)
    CUtensorMap tmG{}, tmW{}, tmX{};
};

inline bool prec_f8(int p) { return p == PIFU_PREC_FP8 || p == PIFU_PREC_FP8_MIXED; }
inline bool prec_mixed(int p) { return p == PIFU_PREC_MIXED || p == PIFU_PREC_FP8_MIXED; }
inline bool prec_valid(int p) { return p >= PIFU_PREC_FP32 && p <= PIFU_PREC_FP8; }

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// The fused FP32 kernel's view of a network (nl = 0 if it has too many layers).
inline FusedNet fused_of(const DevNet& n) {
    FusedNet f{};
    if (n.layers.size() > (size_t)kFusedMaxLayers) return f;
    f.nl = (int)n.layers.size();
    f.ldx = n.ldx;
    f.d_in = n.d_in;
    f.max_hidden = round_up(std::max(n.max_hidden, 8), 4);
    f.slope = n.slope;
    for (int l = 0; l < f.nl; ++l) {
        const DevLayer& L = n.layers[(size_t)l];
        f.L[l] = FusedLayer{L.W, L.b, L.n_out, L.K1, L.K2, L.ldw};
    }
    return f;
}

// Everything a captured frame graph depends on; a call with the same key
// relaunches the graph, any difference recaptures it.
struct FrameKey {
    const void* occ;
    const void* col;
    int oH, oW, oC, cH, cW, cC;
    float calib[12];
    int n0, num_levels, precision, max_rounds;
    float margin;
    int use_surrogate;
    float sur_margin;
    uint64_t sur_version;          // f_S's tensor-core weights are rebuilt on change
    uint64_t f8_version;           // f_O's E4M3 weights are rebuilt by calibration
    int width, height, cam_precision, final_level;
    float bg[3];
    float* depth;
    float* rgb;
    uint8_t* mask;
};

// Device-side counters of a graph frame, copied to the host once at its end.
struct GraphStats {
    unsigned long long culled;   // view-culled final level: candidates evaluated
    unsigned long long evals[8];
    unsigned long long cands[8];
    unsigned long long rechecked[8];
    unsigned long long fallback[8];
    unsigned int rounds[8];
    unsigned int err;
    unsigned int pad;
};

// Launch counters (always on) and CUDA-event timing (when enabled) per
// kernel class.
struct Profiler {
    bool on = false;
    pifu_kernel_stats k[PIFU_K_COUNT] = {};
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // Brackets one launch: call begin before, end after.
    cudaEvent_t begin(cudaStream_t s) {
        if (!on) return nullptr;
        cudaEvent_t a = get();
        cudaEventRecord(a, s);
        return a;
    }
    void end(int cls, cudaEvent_t a, cudaStream_t s, double flops, double bytes) {
        k[cls].launches += 1;
        k[cls].flops += flops;
        k[cls].bytes += bytes;
        if (!on || !a) return;
        cudaEvent_t b = get();
        cudaEventRecord(b, s);
        pending.push_back({cls, a, b});
    }
    cudaError_t resolve() {
        cudaError_t err = cudaSuccess;
        for (auto& p : pending) {
            float ms = 0.f;
            cudaError_t e = cudaEventSynchronize(p.b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
            if (e != cudaSuccess) err = e;
            k[p.cls].ms += ms;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        return err;
    }
    void reset() {
        resolve();
        for (auto& x : k) x = pifu_kernel_stats{};
    }
    ~Profiler() {
        for (auto& p : pending) {
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};


// Device-side counters of a lockstep batch, copied to the host once at its end.
struct BatchStats {
    unsigned long long evals[8][kMaxBatch];   // per level and frame: evaluated nodes
    unsigned long long cands[8][kMaxBatch];   // per level and frame: boundary candidates
    unsigned long long keys[8];               // per level: keys evaluated, all frames
    unsigned long long rechecked[8];
    unsigned long long fallback[8];
    unsigned int rounds[8];
    unsigned int err;
    unsigned int pad;
};

// Everything a captured batch graph depends on besides the map pointers and
// calibrations (read on the device).
struct BatchKey {
    int B;
    int oH, oW, oC, odt, cH, cW, cC, cdt;
    int n0, num_levels, precision, max_rounds;
    float margin;
    int use_surrogate;
    float sur_margin;
    uint64_t sur_version;
    uint64_t f8_version;
    int width, height;
    float bg[3];
    float* depth;
    float* rgb;
    uint8_t* mask;
};

// Per-frame level state of a lockstep batch: B slots of the finest level's
// size, so one slot stride serves every level.
struct BatchWs {
    int B = 0, N = 0;                  // allocated for B slots, finest N
    int64_t slot_words = 0, slot_nodes = 0, cap = 0, npix = 0;
    uint32_t* cand = nullptr;
    uint32_t* tent = nullptr;
    uint32_t* bin[2] = {nullptr, nullptr};
    uint32_t* eval = nullptr;
    uint32_t* conf = nullptr;
    float* values = nullptr;
    int* list = nullptr;               // [cap] keys frame * slot_nodes + node
    int* recheck = nullptr;            // [cap]
    int* squeue = nullptr;             // [cap]
    int* col_top = nullptr;            // [B][2][(N+1)^2]: column top, then bottom
    float* hit_xyz = nullptr;          // [B npix][3]
    int* hit_pix = nullptr;            // [B npix]
    Map* d_maps0 = nullptr;            // [kMaxBatch] device
    Map* d_maps1 = nullptr;
    Calib* d_calibs = nullptr;
    Map* h_maps0 = nullptr;            // pinned staging
    Map* h_maps1 = nullptr;
    Calib* h_calibs = nullptr;
    BatchStats* d_stats = nullptr;
    BatchStats* h_stats = nullptr;     // pinned
    bool g_valid = false;
    BatchKey key{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_fixed = 0;
    int64_t launches_body[8] = {};
};

}  // namespace pifu_host

using namespace pifu;
using namespace pifu_host;

namespace pifu_host {

// Everything a captured stream graph depends on besides the frames' map
// pointers and calibrations (read on the device).
struct StreamKey {
    int F, S;
    int oH, oW, oC, odt, cH, cW, cC, cdt;
    int n0, num_levels, precision, max_rounds;
    float margin;
    int use_surrogate;
    float sur_margin;
    uint64_t sur_version;
    uint64_t f8_version;
    int width, height;
    float bg[3];
    float* depth;
    float* rgb;
    uint8_t* mask;
    uint32_t* bits_out;
};

// Work-queue stream of frames (pifu_stream): S slots of the finest level's
// size, the frames' inputs and results, and the graph.
struct StreamWs {
    int S = 0, N = 0, F = 0;           // allocated for S slots, finest N, F frames
    int64_t npix = 0;
    int64_t slot_words = 0, slot_nodes = 0, slot_top = 0, cap = 0;
    uint32_t* cand = nullptr;
    uint32_t* tent = nullptr;
    uint32_t* bin[2] = {nullptr, nullptr};
    uint32_t* eval = nullptr;
    uint32_t* conf = nullptr;
    float* values = nullptr;
    int* top = nullptr;
    int* list = nullptr;               // [cap] keys slot * slot_nodes + node
    int* recheck = nullptr;            // [cap]
    int* squeue = nullptr;             // [cap]
    float* hit_xyz = nullptr;          // [S npix][3]
    int* hit_pix = nullptr;            // [S npix] keys frame * npix + pixel
    unsigned int* d_hits = nullptr;
    SlotView* sv = nullptr;            // [S]
    StreamSlot* st = nullptr;          // [S]
    unsigned int* pend = nullptr;      // [2 S]: keys in the round's evaluation, keys queued next
    unsigned long long* cands = nullptr;   // [S]
    Map* slot_maps0 = nullptr;         // [S]
    Map* slot_maps1 = nullptr;
    Calib* slot_calibs = nullptr;
    Map* frame_maps0 = nullptr;        // [F] device
    Map* frame_maps1 = nullptr;
    Calib* frame_calibs = nullptr;
    Map* h_maps0 = nullptr;            // [F] pinned staging
    Map* h_maps1 = nullptr;
    Calib* h_calibs = nullptr;
    StreamFrameStats* d_fs = nullptr;  // [F]
    StreamFrameStats* h_fs = nullptr;  // pinned
    StreamCtl* d_ctl = nullptr;
    StreamCtl* h_ctl = nullptr;        // pinned
    bool g_valid = false;
    StreamKey key{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_fixed = 0;
    int64_t launches_body = 0;
    int64_t launches_colour = 0;
};

}  // namespace pifu_host

struct pifu_ctx {
    int device = 0;
    DevNet net[2];
    CbnDev cbn;           // net[0].kind == kNetCbn: the occupancy network
    std::string last_error;
    // MLP activation workspace (FP32 and BF16 forms)
    float* X = nullptr;
    float* HA = nullptr;
    float* HB = nullptr;
    int64_t X_cap = 0, H_cap = 0;   // elements
    __nv_bfloat16* Xb = nullptr;
    __nv_bfloat16* Hb[2] = {nullptr, nullptr};
    unsigned int* chain_dep = nullptr;   // [kChainMaxLayers][tc_rows / 128] tile-part counters,
                                         // the tile counter and the finished-CTA counter
    bool chain_on = false;               // pifu_set_schedule
    int64_t tc_rows = 0;            // rows of Xb, Hb[] (grown on demand up to kChunkTC)
    // split-TF32 passes: input-row planes, two output-plane buffers, split-K
    // partial tiles and their arrival counters (allocated on first use)
    float* X3 = nullptr;
    float* H3[2] = {nullptr, nullptr};
    float* x3_part = nullptr;
    unsigned int* x3_ctr = nullptr;
    bool x3_ready = false;
    // whole-GPU FP32 passes: hidden activations, last-layer partial sums,
    // barrier counters (allocated with the split-TF32 buffers)
    float* grid_H[2] = {nullptr, nullptr};
    float* grid_part = nullptr;
    unsigned int* grid_ctr = nullptr;
    int recheck_form = 0;             // pifu_set_recheck
    unsigned int x3_starve = 0;       // pifu_test_starve_wait
    float* part = nullptr;            // split-K partial sums of small FP32 batches
    int64_t part_cap = 0;
    // level workspace, sized for ws_N
    int ws_N = 0;
    uint32_t* cand = nullptr;
    uint32_t* tent = nullptr;
    uint32_t* bin[2] = {nullptr, nullptr};
    uint32_t* eval = nullptr;
    uint32_t* conf[2] = {nullptr, nullptr};
    float* values = nullptr;
    int* list = nullptr;
    int* recheck = nullptr;                   // mixed precision: points to redo in FP32
    int64_t recheck_cap = 0;
    unsigned int* d_recheck = nullptr;        // its length (device)
    unsigned int* h_recheck = nullptr;        // pinned copy
    unsigned int* d_count = nullptr;          // [0] list length, [1] device error word
    unsigned int* h_count = nullptr;          // pinned [2]
    unsigned long long* d_pop = nullptr;      // [kMaxLevels]
    unsigned long long* h_pop = nullptr;      // pinned [kMaxLevels]
    // render workspace
    float* hit_xyz = nullptr;
    int* hit_pix = nullptr;
    int64_t hit_cap = 0;
    int* col_top = nullptr;       // render: per node column, highest and lowest non-empty depth
    // view-culled final level: candidate keys and their occupancies
    int* cull_list = nullptr;
    float* cull_values = nullptr;
    float* prev_values = nullptr;         // threshold subdivision: the coarser level's values
    int64_t prev_cap = 0;
    int64_t cull_cap = 0, cull_vals_cap = 0;
    int vol_prec = 0;             // arithmetic of the last localization
    float vol_margin = 0.f;
    // last localized volume
    bool have_volume = false;
    int vol_N = 0;
    int vol_bin = 0;
    pifu_volume stats{};
    Profiler prof;
    // learned surrogate f_S (d_in -> h1 -> h2 -> 1), FP32 master parameters
    struct {
        bool ready = false;
        int h1 = 0, h2 = 0;
        int64_t n = 0;                 // parameters in the padded device layout
        int64_t off_w[3] = {}, off_b[3] = {};
        float* params = nullptr;       // [W1 h1 x ldx | b1 | W2 h2 x h1 | b2 | W3 1 x h2 | b3]
        float* grads = nullptr;
        float* adam_m = nullptr;
        float* adam_v = nullptr;
        int step = 0;
        int batch_cap = 0;
        uint64_t version = 0;          // bumped whenever the BF16 form is rebuilt
        float *H1 = nullptr, *H2 = nullptr, *logit = nullptr, *g = nullptr, *dH1 = nullptr,
              *dH2 = nullptr, *ones = nullptr;
        double* d_loss = nullptr;
        double* h_loss = nullptr;      // pinned
        // point OHEM (Eq. 6): per-tuple weights and the sampled batch
        int64_t ohem_m = 0;
        float* ohem_w = nullptr;
        double* ohem_cdf = nullptr;
        double* ohem_sums = nullptr;
        int ohem_B = 0;
        float* xb = nullptr;
        float* yb = nullptr;
        int* ib = nullptr;
        float* per_loss = nullptr;
    } sur;
    DevNet snet;                       // f_S as the MLP runners see it
    int* squeue = nullptr;             // surrogate fall-back queue (node indices)
    unsigned int* d_squeue = nullptr;
    unsigned int* h_squeue = nullptr;  // pinned
    // graph form (pifu_frame)
    bool g_valid = false;
    FrameKey gkey{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;    // capture of the frame
    cudaStream_t cap_stream2 = nullptr;   // capture of the loop bodies
    cudaStream_t cap_stream3 = nullptr;   // capture of conditional branches
    cudaStream_t cap_stream4 = nullptr;   // capture of the FP32 cluster-size switch's bodies
    int* clist = nullptr;                 // graph form: conflicts of a round (keys)
    unsigned int* d_ccount = nullptr;
    int64_t clist_cap = 0;
    GraphStats* d_gstats = nullptr;
    GraphStats* h_gstats = nullptr;       // pinned
    unsigned int* d_tail = nullptr;       // graph form: the loop tails' CTA counters [2]
    unsigned int* d_count2 = nullptr;     // graph form: the frontier count (in d_tail's block)
    int64_t g_launches_fixed = 0;         // kernel launches outside the loops
    int64_t g_launches_body[8] = {};      // kernel launches per loop iteration
    // asynchronous frames (pifu_frame_async / pifu_frame_wait)
    unsigned int* d_sticky = nullptr;     // the enqueued frames' errors, ORed; host-cleared
    int64_t async_frames = 0;             // enqueued since the last wait
    FrameKey async_key{};                 // the last enqueued frame's arguments
    // lockstep frame batches (pifu_frames)
    BatchWs batch;
    // work-queue stream of frames (pifu_stream)
    StreamWs stream;
};

namespace pifu_host {


// Every captured graph (frame, lockstep batch, stream) holds the addresses
// of the workspaces it was captured with: a workspace that moves makes them
// invalid, and the next call recaptures.
inline void invalidate_graphs(pifu_ctx* ctx) {
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    ctx->stream.g_valid = false;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline int fail_cuda(pifu_ctx* ctx, cudaError_t e) {
    if (ctx) ctx->last_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PIFU_ERR_OOM : PIFU_ERR_CUDA;
}

#define CK(expr)                                      \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_); \
    } while (0)

template <typename T>
cudaError_t dev_alloc(T** p, int64_t n) {
    *p = nullptr;
    if (n <= 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), (size_t)n * sizeof(T));
}

template <typename T>
void dev_free(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

inline bool map_ok(const pifu_fmap* m) {
    if (!m || !m->data) return false;
    if (m->H < 1 || m->W < 1 || m->C < 4 || m->C % 4 != 0) return false;
    if (m->H > 65536 || m->W > 65536) return false;
    if ((reinterpret_cast<uintptr_t>(m->data) & 15u) != 0) return false;
    return m->dtype == PIFU_F32 || m->dtype == PIFU_BF16;
}

inline Map to_map(const pifu_fmap* m) {
    Map r{};
    if (m) {
        r.data = m->data;
        r.H = m->H;
        r.W = m->W;
        r.C = m->C;
        r.dtype = m->dtype;
    }
    return r;
}

inline Calib to_calib(const float* c) {
    Calib r;
    std::memcpy(r.c, c, sizeof(r.c));
    return r;
}

inline bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// ---- weight blob ------------------------------------------------------------

struct Reader {
    const uint8_t* p;
    size_t n, off = 0;
    bool get(void* dst, size_t bytes) {
        if (off + bytes > n || off + bytes < off) return false;
        std::memcpy(dst, p + off, bytes);
        off += bytes;
        return true;
    }
    bool u32(uint32_t& v) { return get(&v, 4); }
    bool f32(float& v) { return get(&v, 4); }
};

// Host copy of one parsed net: per layer the repacked weights
// [n_out][K1 | x padded to ldx] and the bias padded to a multiple of 4.
struct HostNet {
    DevNet shape;
    std::vector<std::vector<float>> W, b;
};

// Host copy of the CBN + SoftZ occupancy network with every block's running
// statistics folded into the linear layer before it: with
// s_i = 1 / sqrt(var_i + eps), block i's normalized input is
// s_i (W a + b - mu_i) = (s_i W) a + s_i (b - mu_i).
struct HostCbn {
    int C = 0, n_z = 0, K = 0, nb = 0;
    std::vector<float> WzT, bz, Gt, g0, WT, bl, wlast, blast;
    std::vector<float> GS, g0S, WS, blS;   // the FP32 kernel's per-CTA slices
};

// ---- declarations of the helpers defined in the other units --------------------

int parse_net(Reader& rd, HostNet& hn, int want_kind);
int parse_cbn(Reader& rd, HostCbn& h);
int upload_cbn(pifu_ctx* ctx, const HostCbn& h);
void free_cbn(CbnDev& d);
int upload_net(pifu_ctx* ctx, const HostNet& hn, DevNet& net);
void free_f8(DevNet& net);
void free_net(DevNet& net);
int ensure_mlp_ws(pifu_ctx* ctx);
__nv_bfloat16* chain_out(pifu_ctx* ctx, const DevNet& net, int l);
int encode_act_maps(pifu_ctx* ctx, DevNet& net);
int encode_all_act_maps(pifu_ctx* ctx);
int ensure_tc_rows(pifu_ctx* ctx, int64_t rows);
int build_tc(pifu_ctx* ctx, const HostNet& hn, DevNet& net);
int build_x3(pifu_ctx* ctx, const HostNet& hn, DevNet& net);
int ensure_x3(pifu_ctx* ctx);
// The FP32-accurate pass of the MIXED forms (re-checks, tiny batches): the
// split-TF32 network when the context's re-check form is the tensor cores and
// the net allows it (m points, or a device-sized batch of at most m), else
// the FP32 SIMT network.
bool x3_usable(const pifu_ctx* ctx, const DevNet& net);
// Passes of more points than this run the split-TF32 network (when usable).
int64_t x3_min_rows(const pifu_ctx* ctx);
int run_mlp_x3(pifu_ctx* ctx, const DevNet& net, const PointSrc& src_in, int64_t m,
               const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
               cudaStream_t s, const unsigned int* m_dev);
int run_recheck(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                cudaStream_t s);
// Passes of at most this many points run the whole-GPU FP32 network
// (mlp_grid.cu) in the default re-check form; 0: not usable.
int64_t grid_rows(const pifu_ctx* ctx, const DevNet& net);
int run_mlp_grid(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                 const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                 cudaStream_t s, const unsigned int* m_dev);
uint8_t e4m3_byte(float v);
int build_fp8(pifu_ctx* ctx, DevNet& net, int F, const std::vector<float>& s_h);
int calibrate_fp8(pifu_ctx* ctx, const Map& map, const Calib& cal, int n0, cudaStream_t s);
int ensure_level_ws(pifu_ctx* ctx, int N);
int ensure_prev_values(pifu_ctx* ctx, int64_t n);
int ensure_hit_ws(pifu_ctx* ctx, int64_t npix);
int run_cbn_tc(pifu_ctx* ctx, const PointSrc& src, int64_t m, const Map& map, const Calib& calib,
               const Epilogue& epi, cudaStream_t s, const unsigned int* m_dev);
bool chain_usable(const pifu_ctx* ctx, const DevNet& net);
int run_mlp_tc(pifu_ctx* ctx, const DevNet& net, const PointSrc& src_in, int64_t m,
               const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
               cudaStream_t s, const unsigned int* m_dev = nullptr, bool f8 = false);
int run_cbn_tc(pifu_ctx* ctx, const PointSrc& src_in, int64_t m, const Map& map,
               const Calib& calib, const Epilogue& epi, cudaStream_t s,
               const unsigned int* m_dev);
int run_mlp(pifu_ctx* ctx, const DevNet& net, const PointSrc& src_in, int64_t m, const Map& map0,
            const Map& map1, const Calib& calib, const Epilogue& epi, cudaStream_t s,
            int precision = PIFU_PREC_FP32, const unsigned int* m_dev = nullptr,
            int fused_cl = 0);
int read_recheck(pifu_ctx* ctx, cudaStream_t s, unsigned int* out);
int run_mlp_mixed(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                  const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                  float margin, cudaStream_t s, int64_t* rechecked, bool f8 = false);
int eval_level_batch(pifu_ctx* ctx, const PointSrc& src, int64_t n, const Map& map,
                     const Calib& cal, const Epilogue& epi, int prec, float margin, bool surrogate,
                     float sur_margin, cudaStream_t s, int64_t* rechecked, int64_t* fallback);
int ensure_cull_ws(pifu_ctx* ctx, int64_t npix, int Nc);
int eval_batch(pifu_ctx* ctx, const PointSrc& src, int64_t n, const Map& map, const Calib& cal,
               const Epilogue& epi, int prec, float margin, cudaStream_t s);
int ensure_clist(pifu_ctx* ctx, int64_t cap);
int ohem_ensure(pifu_ctx* ctx, int64_t m, int B, bool reset);
int decode_err(unsigned int e);
// After a device error word was read: clears it and puts back what a kernel
// that stopped early may have left behind (the split-TF32 tile counters), so
// the context stays usable.
int reset_after_error(pifu_ctx* ctx, cudaStream_t s);
int read_count(pifu_ctx* ctx, cudaStream_t s, unsigned int* out);
uint64_t splitmix64(uint64_t& x);
void sur_free(pifu_ctx* ctx);
void sur_bind(pifu_ctx* ctx);
int sur_build_tc(pifu_ctx* ctx);
int sur_init(pifu_ctx* ctx, int h1, int h2, uint64_t seed);
int sur_batch_ws(pifu_ctx* ctx, int B);
int sur_grad(pifu_ctx* ctx, const float* x, const float* y, int B, cudaStream_t s,
             float* per_loss = nullptr);
int64_t sur_unpadded_count(const pifu_ctx* ctx);
void sur_pack(const pifu_ctx* ctx, const std::vector<float>& padded, float* out);
void sur_unpack(const pifu_ctx* ctx, const float* in, std::vector<float>& padded);
int g_add_cond(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h,
               cudaGraphConditionalNodeType type, cudaGraph_t* body);
int g_add_switch(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, int n,
                 cudaGraph_t* bodies);
int64_t launches_now(const pifu_ctx* ctx);
// stat (optional): *stat += the queue length, capacity error above stat_cap.
int g_recheck(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t cap,
              const Map& map, const Calib& cal, const Epilogue& epi, cudaStream_t s,
              const unsigned int* m_dev, unsigned long long* stat = nullptr,
              unsigned int stat_cap = 0);
// recheck_zeroed: a launch before this batch zeroed the re-check queue length.
int g_eval(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t cap,
           const unsigned int* m_dev, const Map& map, const Calib& cal, const Epilogue& epi,
           int prec, float margin, unsigned long long* rechecked, cudaStream_t s,
           bool sur = false, float sur_margin = 0.f, unsigned long long* fallback = nullptr,
           int64_t qcap_in = 0, const RoundStart* rs = nullptr, bool recheck_zeroed = false);
int g_add_while(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body);
int g_enqueue_frame(pifu_ctx* ctx, const FrameKey& k, const Map& occ, const Map& col,
                    const Calib& cal);
void g_destroy(pifu_ctx* ctx);
int g_build(pifu_ctx* ctx, const FrameKey& k, const Map& occ, const Map& col, const Calib& cal);
void batch_free(pifu_ctx* ctx);
int64_t batch_cap(int B);
int batch_ensure(pifu_ctx* ctx, int B, int N, int64_t npix);
int g_enqueue_batch(pifu_ctx* ctx, const BatchKey& k);
int b_build(pifu_ctx* ctx, const BatchKey& k);
bool encode_w(bool fp8, CUtensorMap* tmW, void* Wdev, int Kw, int n_out, int code);
int tune_layer(pifu_ctx* ctx, const TcLayerArgs& base, int n_out, bool fp8, bool allow_pair,
               CUtensorMap* tmW, void* Wdev, int Kw, int* code, cudaStream_t s, double* best_ms);
int autotune(pifu_ctx* ctx, int64_t rows, cudaStream_t s, int32_t* bn_out, double* ms_out,
             int n_max, int* n_done);
int set_tiles(pifu_ctx* ctx, const int32_t* codes, int n);
void stream_free(pifu_ctx* ctx);

}  // namespace pifu_host
