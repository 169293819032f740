// C ABI of libpifu: weight-blob parsing, device memory, and the host side of
// the coarse-to-fine localization loop and of the render (include/pifu.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pifu.h"
#include "pifu_internal.h"

#include <cuda_fp8.h>

using namespace pifu;

namespace {

constexpr int kMaxLevels = 8;
constexpr int kMaxFine = 512;
constexpr int64_t kChunk = 65536;    // points per FP32 MLP pass (bounds its activation workspace)
constexpr int64_t kChunkTC = 1 << 20; // points per tensor-core MLP pass (a whole 512^3 level list)
constexpr int64_t kTcRowsMax = 1 << 22; // device-sized batches of a lockstep frame batch
constexpr int kMaxBatch = 64;           // frames of a lockstep batch
constexpr int64_t kRecheckCap = 8192; // graph form: FP32 re-checks per batch (split-K path)
constexpr int64_t kFusedMaxM = 2048;   // host-sized FP32 batches up to this size: fused kernel
constexpr int64_t kTinyBatch = 256; // mixed precision: batches this small run in FP32

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
    bool pair = false;    // CTA-pair form (BN = 256; tmW's box is then 128 rows)
    CUtensorMap tmW{};
    CUtensorMap tmA1{};   // the previous layer's BF16 output (l >= 1)
    CUtensorMap tmO{};    // this layer's BF16 output, for the epilogue's TMA stores
    bool tmO_ok = false;
};

// E4M3 form of one of f_O's leading wide hidden layers: W divided by a
// per-output-channel scale s_w[n] (the x columns first multiplied by
// s_x / s_a), the accumulator multiplied back by colscale[n] = s_w[n] s_a.
struct Fp8Layer {
    uint8_t* W = nullptr;        // [n_out][Kw] E4M3 bytes, x segment zero-padded
    float* colscale = nullptr;   // [n_out]
    int Kw = 0, nk1 = 0, nk2 = 0, BN = 0;
    float out_scale = 1.f;       // E4M3 output: 1 / s of the next layer's input
    CUtensorMap tmW{};
    CUtensorMap tmA1{};          // the previous layer's E4M3 output (layer >= 1)
};

struct DevNet {
    int kind = 0;       // 0 occupancy (sigmoid), 1 colour (tanh01)
    int d_in = 0;
    int ldx = 0;        // gather row width: d_in rounded up to 8
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
    float s_x = 0.f;                // per-tensor scale of the input rows
    uint64_t f8_version = 0;        // bumped by every calibration
    CUtensorMap tmX8{};             // E4M3 gather rows as the A operand
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

bool prec_f8(int p) { return p == PIFU_PREC_FP8 || p == PIFU_PREC_FP8_MIXED; }
bool prec_mixed(int p) { return p == PIFU_PREC_MIXED || p == PIFU_PREC_FP8_MIXED; }
bool prec_valid(int p) { return p >= PIFU_PREC_FP32 && p <= PIFU_PREC_FP8; }

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// The fused FP32 kernel's view of a network (nl = 0 if it has too many layers).
FusedNet fused_of(const DevNet& n) {
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

}  // namespace

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
    int64_t tc_rows = 0;            // rows of Xb, Hb[], X8 (grown on demand up to kChunkTC)
    uint8_t* X8 = nullptr;          // [tc_rows][ldx8] E4M3 gather rows (FP8 forms):
    int ldx8 = 0;                   //   x_hi at [0, kx8), x_lo at [kx8, 2 kx8)
    int kx8 = 0;
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
    int64_t g_launches_fixed = 0;         // kernel launches outside the loops
    int64_t g_launches_body[8] = {};      // kernel launches per loop iteration
    // lockstep frame batches (pifu_frames)
    BatchWs batch;
};

namespace {

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

int fail_cuda(pifu_ctx* ctx, cudaError_t e) {
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

int parse_net(Reader& rd, HostNet& hn, int want_kind) {
    uint32_t kind, d_in, n_layers, skip_mask;
    float slope;
    if (!rd.u32(kind) || !rd.u32(d_in) || !rd.u32(n_layers) || !rd.f32(slope)) return PIFU_ERR_FORMAT;
    if ((int)kind != want_kind || d_in == 0 || d_in > 4096 || n_layers == 0 || n_layers > 16)
        return PIFU_ERR_FORMAT;
    std::vector<uint32_t> widths(n_layers);
    for (auto& w : widths)
        if (!rd.u32(w) || w == 0 || w > 8192) return PIFU_ERR_FORMAT;
    if (!rd.u32(skip_mask)) return PIFU_ERR_FORMAT;
    const uint32_t n_out = widths[n_layers - 1];
    if ((kind == 0 && n_out != 1) || (kind == 1 && n_out != 3)) return PIFU_ERR_FORMAT;
    for (uint32_t l = 0; l + 1 < n_layers; ++l)
        if (widths[l] % 8 != 0) return PIFU_ERR_UNSUPPORTED;
    DevNet& net = hn.shape;
    net.kind = (int)kind;
    net.d_in = (int)d_in;
    net.ldx = round_up((int)d_in, 8);
    net.slope = slope;
    net.layers.assign(n_layers, DevLayer{});
    net.max_hidden = 0;
    hn.W.assign(n_layers, {});
    hn.b.assign(n_layers, {});
    for (uint32_t l = 0; l < n_layers; ++l) {
        const bool skip = (l > 0) && ((skip_mask >> l) & 1u);
        const int prev = l == 0 ? 0 : (int)widths[l - 1];
        const int fan_in = (l == 0 ? (int)d_in : prev) + (skip ? (int)d_in : 0);
        DevLayer& L = net.layers[l];
        L.n_out = (int)widths[l];
        L.K1 = l == 0 ? 0 : prev;
        L.K2 = (l == 0 || skip) ? net.ldx : 0;
        L.ldw = L.K1 + L.K2;
        L.fan_in = fan_in;
        if (l + 1 < n_layers) net.max_hidden = std::max(net.max_hidden, L.n_out);
        std::vector<float> w((size_t)L.n_out * fan_in), b(L.n_out);
        if (!rd.get(w.data(), w.size() * 4) || !rd.get(b.data(), b.size() * 4)) return PIFU_ERR_FORMAT;
        std::vector<float>& wp = hn.W[l];
        wp.assign((size_t)L.n_out * L.ldw, 0.f);
        for (int o = 0; o < L.n_out; ++o) {
            const float* src = w.data() + (size_t)o * fan_in;
            float* dst = wp.data() + (size_t)o * L.ldw;
            if (l == 0) {
                std::memcpy(dst, src, d_in * 4);
            } else {
                std::memcpy(dst, src, prev * 4);
                if (skip) std::memcpy(dst + L.K1, src + prev, d_in * 4);
            }
        }
        hn.b[l].assign(round_up(L.n_out, 4), 0.f);
        std::memcpy(hn.b[l].data(), b.data(), L.n_out * 4);
    }
    return PIFU_OK;
}

// Host copy of the CBN + SoftZ occupancy network with every block's running
// statistics folded into the linear layer before it: with
// s_i = 1 / sqrt(var_i + eps), block i's normalized input is
// s_i (W a + b - mu_i) = (s_i W) a + s_i (b - mu_i).
struct HostCbn {
    int C = 0, n_z = 0, K = 0, nb = 0;
    std::vector<float> WzT, bz, Gt, g0, WT, bl, wlast, blast;
    std::vector<float> GS, g0S, WS, blS;   // the FP32 kernel's per-CTA slices
};

int parse_cbn(Reader& rd, HostCbn& h) {
    uint32_t kind, C, n_z, K, nb;
    float eps;
    if (!rd.u32(kind) || !rd.u32(C) || !rd.u32(n_z) || !rd.u32(K) || !rd.u32(nb) || !rd.f32(eps))
        return PIFU_ERR_FORMAT;
    if (kind != (uint32_t)kNetCbn || C == 0 || C > 4096 || n_z < 2 || n_z > 4096 || K == 0 ||
        K > 1024 || nb == 0 || nb > 8 || !(eps >= 0.f && eps < 1.f))
        return PIFU_ERR_FORMAT;
    if (C % 8 != 0 || K % 8 != 0) return PIFU_ERR_UNSUPPORTED;
    auto vec = [&rd](std::vector<float>& v, size_t n) {
        v.resize(n);
        return rd.get(v.data(), n * 4);
    };
    std::vector<float> Wz, bz;
    if (!vec(Wz, (size_t)K * n_z) || !vec(bz, K)) return PIFU_ERR_FORMAT;
    std::vector<std::vector<float>> Gg(nb), gg(nb), Gb(nb), gb(nb), mu(nb), var(nb), W(nb), b(nb);
    for (uint32_t i = 0; i < nb; ++i) {
        const size_t kout = i + 1 < nb ? K : 1;
        if (!vec(Gg[i], (size_t)K * C) || !vec(gg[i], K) || !vec(Gb[i], (size_t)K * C) ||
            !vec(gb[i], K) || !vec(mu[i], K) || !vec(var[i], K) || !vec(W[i], kout * K) ||
            !vec(b[i], kout))
            return PIFU_ERR_FORMAT;
        for (float v : var[i])
            if (!(v + eps > 0.f) || !std::isfinite(v)) return PIFU_ERR_FORMAT;
    }
    std::vector<std::vector<double>> sc(nb, std::vector<double>(K));
    for (uint32_t i = 0; i < nb; ++i)
        for (uint32_t k = 0; k < K; ++k) sc[i][k] = 1.0 / std::sqrt((double)var[i][k] + (double)eps);
    h.C = (int)C;
    h.n_z = (int)n_z;
    h.K = (int)K;
    h.nb = (int)nb;
    h.WzT.assign((size_t)n_z * K, 0.f);
    h.bz.assign(K, 0.f);
    for (uint32_t k = 0; k < K; ++k) {
        for (uint32_t j = 0; j < n_z; ++j)
            h.WzT[(size_t)j * K + k] = (float)(sc[0][k] * Wz[(size_t)k * n_z + j]);
        h.bz[k] = (float)(sc[0][k] * ((double)bz[k] - mu[0][k]));
    }
    const size_t K2 = 2 * (size_t)K;
    h.Gt.assign(nb * C * K2, 0.f);
    h.g0.assign(nb * K2, 0.f);
    for (uint32_t i = 0; i < nb; ++i)
        for (size_t o = 0; o < K2; ++o) {
            const bool gam = o < K;
            const std::vector<float>& G = gam ? Gg[i] : Gb[i];
            const size_t row = gam ? o : o - K;
            for (uint32_t c = 0; c < C; ++c) h.Gt[(i * C + c) * K2 + o] = G[row * C + c];
            h.g0[i * K2 + o] = gam ? gg[i][row] : gb[i][row];
        }
    h.WT.assign((size_t)(nb - 1) * K * K, 0.f);
    h.bl.assign((size_t)(nb - 1) * K, 0.f);
    for (uint32_t i = 0; i + 1 < nb; ++i)
        for (uint32_t o = 0; o < K; ++o) {
            const double s1 = sc[i + 1][o];
            for (uint32_t k = 0; k < K; ++k)
                h.WT[((size_t)i * K + k) * K + o] = (float)(s1 * W[i][(size_t)o * K + k]);
            h.bl[(size_t)i * K + o] = (float)(s1 * ((double)b[i][o] - mu[i + 1][o]));
        }
    h.wlast = W[nb - 1];
    h.blast = {b[nb - 1][0], 0.f, 0.f, 0.f};
    // slices of the cluster kernel: CTA r owns channels [r Kc, (r + 1) Kc)
    if (K % kCbnCluster == 0) {
        const size_t S = kCbnCluster, Kc = K / S, K2c = 2 * Kc;
        h.GS.assign(nb * S * C * K2c, 0.f);
        h.g0S.assign(nb * S * K2c, 0.f);
        for (size_t i = 0; i < nb; ++i)
            for (size_t r = 0; r < S; ++r)
                for (size_t j = 0; j < K2c; ++j) {
                    const size_t o = j < Kc ? r * Kc + j : K + r * Kc + (j - Kc);
                    for (size_t c = 0; c < C; ++c)
                        h.GS[((i * S + r) * C + c) * K2c + j] = h.Gt[(i * C + c) * K2 + o];
                    h.g0S[(i * S + r) * K2c + j] = h.g0[i * K2 + o];
                }
        h.WS.assign((nb - 1) * S * K * Kc, 0.f);
        h.blS.assign((nb - 1) * S * Kc, 0.f);
        for (size_t i = 0; i + 1 < nb; ++i)
            for (size_t r = 0; r < S; ++r)
                for (size_t j = 0; j < Kc; ++j) {
                    const size_t o = r * Kc + j;
                    for (size_t k = 0; k < K; ++k)
                        h.WS[((i * S + r) * K + k) * Kc + j] = h.WT[(i * K + k) * K + o];
                    h.blS[(i * S + r) * Kc + j] = h.bl[i * K + o];
                }
    }
    return PIFU_OK;
}

int upload_cbn(pifu_ctx* ctx, const HostCbn& h) {
    CbnDev& d = ctx->cbn;
    auto up = [&d](const std::vector<float>& v, const float** dst) -> cudaError_t {
        float* p = nullptr;
        cudaError_t e = dev_alloc(&p, (int64_t)std::max<size_t>(v.size(), 1));
        if (e != cudaSuccess) return e;
        d.bufs.push_back(p);
        *dst = p;
        return v.empty() ? cudaSuccess
                         : cudaMemcpy(p, v.data(), v.size() * 4, cudaMemcpyHostToDevice);
    };
    CbnF32& f = d.f32;
    CK(up(h.WzT, &f.WzT));
    CK(up(h.bz, &f.bz));
    CK(up(h.GS, &f.GS));
    CK(up(h.g0S, &f.g0S));
    CK(up(h.WS, &f.WS));
    CK(up(h.blS, &f.blS));
    CK(up(h.wlast, &f.wlast));
    CK(up(h.blast, &f.blast));
    CK(up(h.g0, &d.g0));
    CK(up(h.bl, &d.bl));
    f.C = h.C;
    f.n_z = h.n_z;
    f.K = h.K;
    f.nb = h.nb;
    if (!cbn_f32_ok(f)) return PIFU_ERR_UNSUPPORTED;
    if (cbn_tc_ok(h.C, h.K, h.nb)) {
        // BF16 weights in the MMA's K-major B layout: rows are outputs
        const size_t K2 = 2 * (size_t)h.K;
        std::vector<__nv_bfloat16> G((size_t)h.nb * K2 * h.C);
        for (int i = 0; i < h.nb; ++i)
            for (size_t o = 0; o < K2; ++o)
                for (int c = 0; c < h.C; ++c)
                    G[((size_t)i * K2 + o) * h.C + c] =
                        __float2bfloat16_rn(h.Gt[((size_t)i * h.C + c) * K2 + o]);
        const int nw = std::max(h.nb - 1, 1);
        std::vector<__nv_bfloat16> W((size_t)nw * h.K * h.K, __float2bfloat16_rn(0.f));
        for (int i = 0; i + 1 < h.nb; ++i)
            for (int o = 0; o < h.K; ++o)
                for (int k = 0; k < h.K; ++k)
                    W[((size_t)i * h.K + o) * h.K + k] =
                        __float2bfloat16_rn(h.WT[((size_t)i * h.K + k) * h.K + o]);
        CK(dev_alloc(&d.Gbf, (int64_t)G.size()));
        CK(dev_alloc(&d.Wbf, (int64_t)W.size()));
        CK(cudaMemcpy(d.Gbf, G.data(), G.size() * 2, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d.Wbf, W.data(), W.size() * 2, cudaMemcpyHostToDevice));
        if (!tc_encode_2d_bf16(&d.tmG, d.Gbf, (uint64_t)h.C, (uint64_t)h.nb * K2,
                               (uint64_t)h.C * 2, 64, (uint32_t)K2) ||
            !tc_encode_2d_bf16(&d.tmW, d.Wbf, (uint64_t)h.K, (uint64_t)nw * h.K,
                               (uint64_t)h.K * 2, 64, (uint32_t)h.K))
            return PIFU_ERR_CUDA;
        d.tc_ok = true;
    }
    // the occupancy slot's shape: the depth is one input scalar as for the
    // concatenation network; no layers of its own
    DevNet& net = ctx->net[0];
    net = DevNet{};
    net.kind = kNetCbn;
    net.d_in = h.C + 1;
    net.ldx = round_up(h.C + 1, 8);
    net.max_hidden = h.K;
    net.tc_ok = d.tc_ok;
    d.ready = true;
    return PIFU_OK;
}

void free_cbn(CbnDev& d) {
    for (float* p : d.bufs) dev_free(p);
    d.bufs.clear();
    dev_free(d.Gbf);
    dev_free(d.Wbf);
    d.tc_ok = false;
    d.f32 = CbnF32{};
    d.g0 = d.bl = nullptr;
    d.ready = false;
}

int upload_net(pifu_ctx* ctx, const HostNet& hn, DevNet& net) {
    net = hn.shape;
    for (auto& L : net.layers) L.W = L.b = nullptr;
    for (size_t l = 0; l < net.layers.size(); ++l) {
        DevLayer& L = net.layers[l];
        CK(dev_alloc(&L.W, (int64_t)hn.W[l].size()));
        CK(dev_alloc(&L.b, (int64_t)hn.b[l].size()));
        CK(cudaMemcpy(L.W, hn.W[l].data(), hn.W[l].size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(L.b, hn.b[l].data(), hn.b[l].size() * 4, cudaMemcpyHostToDevice));
    }
    return PIFU_OK;
}

void free_f8(DevNet& net) {
    for (auto& Q : net.f8) {
        dev_free(Q.W);
        dev_free(Q.colscale);
    }
    net.f8.clear();
    net.f8_ok = false;
}

void free_net(DevNet& net) {
    for (auto& L : net.layers) {
        dev_free(L.W);
        dev_free(L.b);
    }
    for (auto& T : net.tc) dev_free(T.W);
    free_f8(net);
    net.layers.clear();
    net.tc.clear();
}

// ---- workspaces -------------------------------------------------------------

int ensure_mlp_ws(pifu_ctx* ctx) {
    int64_t need_x = 0, need_h = 0;
    for (const DevNet& n : ctx->net) {
        need_x = std::max<int64_t>(need_x, n.ldx);
        need_h = std::max<int64_t>(need_h, std::max(n.max_hidden, 8));
    }
    if (need_x > ctx->X_cap) {   // per-point widths; FP32 rows are kChunk points
        dev_free(ctx->X);
        CK(dev_alloc(&ctx->X, need_x * kChunk));
        ctx->X_cap = need_x;
    }
    if (need_h > ctx->H_cap) {
        dev_free(ctx->HA);
        dev_free(ctx->HB);
        CK(dev_alloc(&ctx->HA, need_h * kChunk));
        CK(dev_alloc(&ctx->HB, need_h * kChunk));
        ctx->H_cap = need_h;
    }
    // split-K partial sums: host-sized batches up to kSplitMaxM, device-sized
    // re-check batches up to kRecheckCap
    int64_t need_p = 0;
    for (const DevNet& n : ctx->net)
        for (const DevLayer& L : n.layers)
            need_p = std::max<int64_t>(need_p, (int64_t)splitk_slices(L.K1, L.K2) *
                                                   std::max<int64_t>(kSplitMaxM, kRecheckCap) *
                                                   L.n_out);
    if (need_p > ctx->part_cap) {
        dev_free(ctx->part);
        CK(dev_alloc(&ctx->part, need_p));
        ctx->part_cap = need_p;
    }
    return PIFU_OK;
}

// Tensor-core form of a net: BF16 weights and the tensor maps over them and
// over the BF16 workspaces (which must already exist).  Nets whose hidden
// widths are not multiples of 64 keep tc_ok = false.
// TMA maps of a network's activation operands (gather rows, previous layer
// outputs) over the current tensor-core workspaces of tc_rows rows.
// Output buffer of hidden layer l in the chained form: [tc_rows][n_out_l].
__nv_bfloat16* chain_out(pifu_ctx* ctx, const DevNet& net, int l) {
    if (l == 0) return ctx->Hb[0];
    int64_t off = 0;
    for (int k = 1; k < l; ++k) off += net.layers[k].n_out;
    return ctx->Hb[1] + off * ctx->tc_rows;
}

int encode_act_maps(pifu_ctx* ctx, DevNet& net) {
    if (!net.tc_ok || ctx->tc_rows == 0 || net.kind == kNetCbn) return PIFU_OK;
    const uint64_t rows = (uint64_t)ctx->tc_rows;
    if (!tc_encode_2d_bf16(&net.tmX, ctx->Xb, (uint64_t)net.d_in, rows, (uint64_t)net.ldx * 2, 64,
                           128))
        return PIFU_ERR_CUDA;
    for (size_t l = 1; l < net.tc.size(); ++l) {
        const DevLayer& Ly = net.layers[l];
        if (!tc_encode_2d_bf16(&net.tc[l].tmA1, ctx->Hb[(l - 1) % 2], (uint64_t)Ly.K1, rows,
                               (uint64_t)Ly.K1 * 2, 64, 128))
            return PIFU_ERR_CUDA;
    }
    for (size_t l = 0; l < net.tc.size(); ++l) {
        const DevLayer& Ly = net.layers[l];
        net.tc[l].tmO_ok = tc_encode_2d_bf16_out(&net.tc[l].tmO, ctx->Hb[l % 2],
                                                 (uint64_t)Ly.n_out, rows,
                                                 (uint64_t)Ly.n_out * 2);
        if (!net.tc[l].tmO_ok) return PIFU_ERR_CUDA;
    }
    // chained form: layer 0 writes Hb[0], layers 1 .. nl-2 write consecutive
    // column blocks of Hb[1] (the last hidden layer carries the fused last
    // layer and writes nothing)
    {
        const int nl = (int)net.tc.size();
        int64_t hcap = 8;
        for (const DevNet& n : ctx->net) hcap = std::max<int64_t>(hcap, std::max(n.max_hidden, 8));
        int sum_n = 0, sum_mid = 0;
        for (int l = 0; l < nl; ++l) sum_n += net.layers[l].n_out;
        for (int l = 1; l + 1 < nl; ++l) sum_mid += net.layers[l].n_out;
        net.chain_ok = nl >= 1 && nl <= kChainMaxLayers && sum_n <= kChainBiasFloats &&
                       net.layers[0].n_out <= hcap && sum_mid <= hcap;
        net.chain_tmA1.assign((size_t)std::max(nl, 1), CUtensorMap{});
        for (int l = 1; net.chain_ok && l < nl; ++l) {
            const int K1 = net.layers[l].K1;
            if (!tc_encode_2d_bf16(&net.chain_tmA1[l], chain_out(ctx, net, l - 1), (uint64_t)K1,
                                   rows, (uint64_t)K1 * 2, 64, 128))
                return PIFU_ERR_CUDA;
        }
    }
    if (net.f8_ok) {
        if (!tc_encode_2d_u8(&net.tmX8, ctx->X8, (uint64_t)ctx->ldx8, rows, (uint64_t)ctx->ldx8,
                             128, 128))
            return PIFU_ERR_CUDA;
        for (size_t l = 1; l < net.f8.size(); ++l) {
            const DevLayer& Ly = net.layers[l];
            if (!tc_encode_2d_u8(&net.f8[l].tmA1, ctx->Hb[(l - 1) % 2], (uint64_t)Ly.K1, rows,
                                 (uint64_t)Ly.K1, 128, 128))
                return PIFU_ERR_CUDA;
        }
    }
    return PIFU_OK;
}

int encode_all_act_maps(pifu_ctx* ctx);

// Grow the tensor-core workspaces to at least `rows` points (powers of two
// from 65,536 up to kChunkTC).  Growing frees the old buffers (cudaFree waits
// for the device) and invalidates a captured frame graph, which holds maps
// of them; the graph form reserves kChunkTC rows before it captures.
int ensure_tc_rows(pifu_ctx* ctx, int64_t rows) {
    if (rows <= ctx->tc_rows) return PIFU_OK;
    if (rows > kTcRowsMax) return PIFU_ERR_ARG;
    int64_t cap = 65536;
    while (cap < rows) cap *= 2;
    cap = std::min<int64_t>(cap, kTcRowsMax);
    int64_t need_x = 0, need_h = 0;
    for (const DevNet& n : ctx->net) {
        need_x = std::max<int64_t>(need_x, n.ldx);
        need_h = std::max<int64_t>(need_h, std::max(n.max_hidden, 8));
    }
    ctx->g_valid = false;
    dev_free(ctx->Xb);
    dev_free(ctx->Hb[0]);
    dev_free(ctx->Hb[1]);
    dev_free(ctx->X8);
    dev_free(ctx->chain_dep);
    ctx->tc_rows = 0;
    CK(dev_alloc(&ctx->chain_dep, (int64_t)kChainMaxLayers * (cap / 128) + 2));
    CK(cudaMemset(ctx->chain_dep, 0, sizeof(unsigned int) * ((size_t)kChainMaxLayers * (cap / 128) + 2)));
    CK(dev_alloc(&ctx->Xb, need_x * cap));
    CK(dev_alloc(&ctx->Hb[0], need_h * cap));
    CK(dev_alloc(&ctx->Hb[1], need_h * cap));
    if (ctx->ldx8 > 0) {
        CK(dev_alloc(&ctx->X8, (int64_t)ctx->ldx8 * cap));
        CK(cudaMemset(ctx->X8, 0, (size_t)ctx->ldx8 * cap));
    }
    ctx->tc_rows = cap;
    return encode_all_act_maps(ctx);
}

int build_tc(pifu_ctx* ctx, const HostNet& hn, DevNet& net) {
    const int L = (int)net.layers.size();
    net.tc_ok = false;
    net.tc.assign(L > 1 ? L - 1 : 0, TcLayer{});
    for (int l = 0; l + 1 < L; ++l)
        if (net.layers[l].n_out % 64 != 0) return PIFU_OK;
    const int k2pad = round_up(net.d_in, 64);
    for (int l = 0; l + 1 < L; ++l) {
        const DevLayer& Ly = net.layers[l];
        TcLayer& T = net.tc[l];
        const bool has_x = Ly.K2 > 0;
        T.nk1 = Ly.K1 / 64;
        T.nk2 = has_x ? k2pad / 64 : 0;
        T.Kw = Ly.K1 + (has_x ? k2pad : 0);
        // single-CTA tiles by default (pifu_autotune / pifu_set_tiles may
        // choose the CTA-pair form)
        T.BN = Ly.n_out % 256 == 0 ? 256 : (Ly.n_out % 128 == 0 ? 128 : 64);
        T.pair = false;
        std::vector<__nv_bfloat16> wb((size_t)Ly.n_out * T.Kw, __float2bfloat16(0.f));
        const std::vector<float>& wf = hn.W[l];   // [n_out][K1 | ldx]
        for (int o = 0; o < Ly.n_out; ++o) {
            for (int k = 0; k < Ly.K1; ++k)
                wb[(size_t)o * T.Kw + k] = __float2bfloat16(wf[(size_t)o * Ly.ldw + k]);
            if (has_x)
                for (int k = 0; k < net.d_in; ++k)
                    wb[(size_t)o * T.Kw + Ly.K1 + k] =
                        __float2bfloat16(wf[(size_t)o * Ly.ldw + Ly.K1 + k]);
        }
        CK(dev_alloc(&T.W, (int64_t)wb.size()));
        CK(cudaMemcpy(T.W, wb.data(), wb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
        if (!tc_encode_2d_bf16(&T.tmW, T.W, (uint64_t)T.Kw, (uint64_t)Ly.n_out, (uint64_t)T.Kw * 2,
                               64, (uint32_t)(T.pair ? T.BN / 2 : T.BN)))
            return PIFU_ERR_CUDA;
    }
    net.tc_ok = true;
    return encode_act_maps(ctx, net);
}

// ---- FP8 form of f_O ----------------------------------------------------------

uint8_t e4m3_byte(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// The E4M3 layers 0 .. F-1 of `net` from its FP32 weights (read back from the
// device) and the activation scales: net.s_x for the input rows, s_h[l] for
// h_l (the output of layer l, l < F-1).  The input rows enter as two E4M3
// terms (x / s_x ~ hi + lo / 16), so a layer's x columns appear twice: once
// against hi and once, divided by 16, against lo.
int build_fp8(pifu_ctx* ctx, DevNet& net, int F, const std::vector<float>& s_h) {
    free_f8(net);
    const int kx8 = ctx->kx8;
    const int nk2 = 2 * kx8 / 128;
    net.f8.assign((size_t)F, Fp8Layer{});
    for (int l = 0; l < F; ++l) {
        const DevLayer& Ly = net.layers[(size_t)l];
        Fp8Layer& Q = net.f8[(size_t)l];
        const bool has_x = Ly.K2 > 0;
        Q.nk1 = Ly.K1 / 128;
        Q.nk2 = has_x ? nk2 : 0;
        Q.Kw = Ly.K1 + (has_x ? 2 * kx8 : 0);
        Q.BN = net.tc[(size_t)l].BN;
        const float s_a = l == 0 ? net.s_x : s_h[(size_t)l - 1];
        const float xf = has_x ? net.s_x / s_a : 0.f;   // x columns in units of s_a
        std::vector<float> wf((size_t)Ly.n_out * Ly.ldw);
        CK(cudaMemcpy(wf.data(), Ly.W, wf.size() * 4, cudaMemcpyDeviceToHost));
        std::vector<uint8_t> w8((size_t)Ly.n_out * Q.Kw, 0);
        std::vector<float> cs((size_t)Ly.n_out);
        for (int o = 0; o < Ly.n_out; ++o) {
            const float* row = &wf[(size_t)o * Ly.ldw];
            float amax = 0.f;
            for (int k = 0; k < Ly.K1; ++k) amax = std::max(amax, std::fabs(row[k]));
            if (has_x)
                for (int k = 0; k < net.d_in; ++k)
                    amax = std::max(amax, std::fabs(row[Ly.K1 + k] * xf));
            const float sw = amax > 0.f ? amax / 448.f : 1.f;
            uint8_t* dst = &w8[(size_t)o * Q.Kw];
            for (int k = 0; k < Ly.K1; ++k) dst[k] = e4m3_byte(row[k] / sw);
            if (has_x)
                for (int k = 0; k < net.d_in; ++k) {
                    dst[Ly.K1 + k] = e4m3_byte(row[Ly.K1 + k] * xf / sw);
                    dst[Ly.K1 + kx8 + k] = e4m3_byte(row[Ly.K1 + k] * xf / (16.f * sw));
                }
            cs[(size_t)o] = sw * s_a;
        }
        CK(dev_alloc(&Q.W, (int64_t)w8.size()));
        CK(dev_alloc(&Q.colscale, (int64_t)cs.size()));
        CK(cudaMemcpy(Q.W, w8.data(), w8.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(Q.colscale, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice));
        if (!tc_encode_2d_u8(&Q.tmW, Q.W, (uint64_t)Q.Kw, (uint64_t)Ly.n_out, (uint64_t)Q.Kw, 128,
                             (uint32_t)Q.BN))
            return PIFU_ERR_CUDA;
        Q.out_scale = l + 1 < F ? 1.f / s_h[(size_t)l] : 1.f;
    }
    net.f8_ok = true;
    ++net.f8_version;
    return encode_act_maps(ctx, net);
}

// Activation scales from FP32 evaluations of the input rows and of h_0 ..
// h_{F-2} at the (n0+1)^3 nodes of the dense grid, then build_fp8.
int calibrate_fp8(pifu_ctx* ctx, const Map& map, const Calib& cal, int n0, cudaStream_t s) {
    DevNet& net = ctx->net[0];
    if (!net.tc_ok) return PIFU_ERR_UNSUPPORTED;
    const int L = (int)net.layers.size();
    int F = 0;   // the leading hidden layers with >= 512 outputs
    while (F + 1 < L && net.layers[(size_t)F].n_out >= 512 &&
           net.layers[(size_t)F].n_out % 128 == 0 && net.layers[(size_t)F].K1 % 128 == 0)
        ++F;
    if (F == 0) return PIFU_ERR_UNSUPPORTED;
    // [x_hi | x_lo], each padded to whole 128-byte K-blocks; the padding
    // stays zero (the gather writes only the first ldx bytes of each half)
    const int kx8 = round_up(std::max(net.d_in, net.ldx), 128);
    int st0 = ensure_tc_rows(ctx, 1);
    if (st0 != PIFU_OK) return st0;
    if (!ctx->X8 || ctx->ldx8 != 2 * kx8) {
        dev_free(ctx->X8);
        ctx->ldx8 = ctx->kx8 = 0;
        CK(dev_alloc(&ctx->X8, (int64_t)2 * kx8 * ctx->tc_rows));
        CK(cudaMemset(ctx->X8, 0, (size_t)2 * kx8 * ctx->tc_rows));
        ctx->ldx8 = 2 * kx8;
        ctx->kx8 = kx8;
    }
    unsigned int* d_amax = nullptr;
    CK(cudaMalloc(&d_amax, sizeof(unsigned int) * (size_t)F));
    cudaError_t e = cudaMemsetAsync(d_amax, 0, sizeof(unsigned int) * (size_t)F, s);
    const int64_t nodes = (int64_t)(n0 + 1) * (n0 + 1) * (n0 + 1);
    PointSrc src{PTS_DENSE, nullptr, nullptr, 0, n0, nullptr};
    for (int64_t p0 = 0; p0 < nodes && e == cudaSuccess; p0 += kChunk) {
        const int64_t mc = std::min<int64_t>(kChunk, nodes - p0);
        e = launch_gather(src, p0, mc, cal, map, Map{}, ctx->X, net.ldx, s);
        if (e == cudaSuccess) e = launch_amax(ctx->X, mc * net.ldx, d_amax, s);
        const float* h = nullptr;
        int hw = 0;
        for (int l = 0; l + 1 < F && e == cudaSuccess; ++l) {
            const DevLayer& Ly = net.layers[(size_t)l];
            float* out = (l % 2 == 0) ? ctx->HA : ctx->HB;
            e = launch_sgemm_bias_lrelu((int)mc, Ly.n_out, h, hw, Ly.K1, ctx->X, net.ldx, Ly.K2,
                                        Ly.W, Ly.ldw, Ly.b, net.slope, out, Ly.n_out, s, nullptr,
                                        nullptr);
            if (e == cudaSuccess) e = launch_amax(out, mc * Ly.n_out, d_amax + 1 + l, s);
            h = out;
            hw = Ly.n_out;
        }
    }
    std::vector<unsigned int> bits((size_t)F, 0u);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bits.data(), d_amax, sizeof(unsigned int) * (size_t)F,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_amax);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    auto scale = [](unsigned int b) {
        float a;
        std::memcpy(&a, &b, 4);
        return a > 0.f && std::isfinite(a) ? a / 448.f : 1.f;
    };
    net.s_x = scale(bits[0]);
    std::vector<float> s_h;
    for (int l = 0; l + 1 < F; ++l) s_h.push_back(scale(bits[(size_t)l + 1]));
    const int st = build_fp8(ctx, net, F, s_h);
    if (st != PIFU_OK) free_f8(net);
    return st;
}

int ensure_level_ws(pifu_ctx* ctx, int N) {
    if (N <= ctx->ws_N) return PIFU_OK;
    uint32_t** bitsets[] = {&ctx->cand, &ctx->tent, &ctx->bin[0], &ctx->bin[1],
                            &ctx->eval, &ctx->conf[0], &ctx->conf[1]};
    for (auto b : bitsets) dev_free(*b);
    dev_free(ctx->values);
    dev_free(ctx->list);
    ctx->ws_N = 0;
    ctx->have_volume = false;
    const int64_t words = words_of(N);
    const int64_t nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
    for (auto b : bitsets) {
        CK(dev_alloc(b, words));
        CK(cudaMemset(*b, 0, (size_t)words * 4));
    }
    CK(dev_alloc(&ctx->values, nodes));
    CK(dev_alloc(&ctx->list, nodes));
    dev_free(ctx->col_top);
    CK(dev_alloc(&ctx->col_top, 2 * (int64_t)(N + 1) * (N + 1)));
    if (nodes > ctx->recheck_cap) {
        dev_free(ctx->recheck);
        dev_free(ctx->squeue);
        ctx->recheck_cap = 0;
        CK(dev_alloc(&ctx->recheck, nodes));
        CK(dev_alloc(&ctx->squeue, nodes));
        ctx->recheck_cap = nodes;
    }
    ctx->ws_N = N;
    return PIFU_OK;
}

int ensure_prev_values(pifu_ctx* ctx, int64_t n) {
    if (n <= ctx->prev_cap) return PIFU_OK;
    dev_free(ctx->prev_values);
    ctx->prev_cap = 0;
    CK(dev_alloc(&ctx->prev_values, n));
    ctx->prev_cap = n;
    return PIFU_OK;
}

int ensure_hit_ws(pifu_ctx* ctx, int64_t npix) {
    if (npix <= ctx->hit_cap) return PIFU_OK;
    dev_free(ctx->hit_xyz);
    dev_free(ctx->hit_pix);
    ctx->hit_cap = 0;
    CK(dev_alloc(&ctx->hit_xyz, 3 * npix));
    CK(dev_alloc(&ctx->hit_pix, npix));
    ctx->hit_cap = npix;
    return PIFU_OK;
}

// ---- argument checks ----------------------------------------------------------

bool map_ok(const pifu_fmap* m) {
    if (!m || !m->data) return false;
    if (m->H < 1 || m->W < 1 || m->C < 4 || m->C % 4 != 0) return false;
    if (m->H > 65536 || m->W > 65536) return false;
    if ((reinterpret_cast<uintptr_t>(m->data) & 15u) != 0) return false;
    return m->dtype == PIFU_F32 || m->dtype == PIFU_BF16;
}

Map to_map(const pifu_fmap* m) {
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

Calib to_calib(const float* c) {
    Calib r;
    std::memcpy(r.c, c, sizeof(r.c));
    return r;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// ---- the MLP over a point batch ---------------------------------------------------

// m_dev (optional): the batch size is device-resident, at most m <= kChunkTC
// (graph form); m is then only the capacity the launches are sized for.
int run_cbn_tc(pifu_ctx* ctx, const PointSrc& src, int64_t m, const Map& map, const Calib& calib,
               const Epilogue& epi, cudaStream_t s, const unsigned int* m_dev);
// The chained form applies to this network now: its shapes and buffers
// allow it, it is switched on, and no layer uses the CTA-pair form.
bool chain_usable(const pifu_ctx* ctx, const DevNet& net) {
    if (!ctx->chain_on || !net.chain_ok || net.kind == kNetCbn) return false;
    for (const TcLayer& T : net.tc)
        if (T.pair || T.BN > 256) return false;
    return true;
}

int run_mlp_tc(pifu_ctx* ctx, const DevNet& net, const PointSrc& src_in, int64_t m,
               const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
               cudaStream_t s, const unsigned int* m_dev = nullptr, bool f8 = false) {
    if (net.kind == kNetCbn) {
        if (f8) return PIFU_ERR_UNSUPPORTED;
        return run_cbn_tc(ctx, src_in, m, map0, calib, epi, s, m_dev);
    }
    if (!net.tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (f8 && !net.f8_ok) return PIFU_ERR_STATE;
    const int F = f8 ? (int)net.f8.size() : 0;   // leading E4M3 layers
    // a device-resident count is a total: such a batch is one pass (the
    // graph forms reserve its rows before capture); host-sized batches go in
    // chunks of kChunkTC
    const int64_t chunk = m_dev ? std::max<int64_t>(m, 1) : kChunkTC;
    {
        const int st = ensure_tc_rows(ctx, std::min<int64_t>(m, chunk));
        if (st != PIFU_OK) return st;
    }
    if (m_dev && m > kTcRowsMax) return PIFU_ERR_ARG;
    PointSrc src = src_in;
    src.count = m_dev;
    const int L = (int)net.layers.size();
    Profiler& pr = ctx->prof;
    for (int64_t p0 = 0; p0 < m; p0 += chunk) {
        const int64_t mc = std::min<int64_t>(chunk, m - p0);
        cudaEvent_t ev = pr.begin(s);
        if (F > 0)
            CK(launch_gather_dual(src, p0, mc, calib, map0, map1, ctx->Xb, net.ldx, ctx->X8,
                                  ctx->ldx8, ctx->kx8, 1.f / net.s_x, s));
        else
            CK(launch_gather_bf16(src, p0, mc, calib, map0, map1, ctx->Xb, net.ldx, s));
        pr.end(PIFU_K_GATHER, ev, s, 0.0,
               (double)mc * (4.0 * 4.0 * (map0.C + map1.C) + (F > 0 ? 3.0 : 2.0) * net.ldx));
        // the last layer rides in the last hidden layer's epilogue when that
        // layer is one tile wide and the last layer reads only its output
        const DevLayer& Ll = net.layers[L - 1];
        const bool fuse = L > 1 && Ll.K2 == 0 && Ll.n_out <= 4 && !net.tc[L - 2].pair &&
                          net.tc[L - 2].BN == net.layers[L - 2].n_out;
        FuseLast fl{};
        if (fuse) {
            fl.W = Ll.W;
            fl.ldw = Ll.ldw;
            fl.bias = Ll.b;
            fl.n_out = Ll.n_out;
            fl.p0 = p0;
            fl.epi = epi;
        }
        if (F == 0 && fuse && chain_usable(ctx, net)) {
            // all hidden layers (and the fused last layer) in one launch
            ChainArgs ca{};
            double flops = 2.0 * mc * Ll.fan_in * Ll.n_out, bytes = 0.0;
            int sum_tiles = 0, boff = 0;
            ca.nl = L - 1;
            for (int l = 0; l + 1 < L; ++l) {
                const DevLayer& Ly = net.layers[l];
                const TcLayer& T = net.tc[l];
                ChainLayer& C = ca.L[l];
                C.tmA1 = l > 0 ? net.chain_tmA1[l] : net.tmX;
                C.tmA2 = net.tmX;
                C.tmW = T.tmW;
                C.nk1 = T.nk1;
                C.nk2 = T.nk2;
                C.N = Ly.n_out;
                C.BN = T.BN;
                C.bias = Ly.b;
                C.out = l + 2 < L ? chain_out(ctx, net, l) : nullptr;
                C.ldo = Ly.n_out;
                ca.boff[l] = boff;
                boff += Ly.n_out;
                sum_tiles += Ly.n_out / T.BN;
                flops += 2.0 * mc * Ly.fan_in * Ly.n_out;
                bytes += 2.0 * ((double)mc * (Ly.fan_in + Ly.n_out) + (double)Ly.n_out * Ly.fan_in);
            }
            CK(chain_prepare());
            ca.M = (int)mc;
            ca.m_dev = m_dev;
            ca.err = ctx->d_count + 1;
            ca.dep = ctx->chain_dep;
            ca.max_mb = (int)(ctx->tc_rows / 128);
            ca.next_tile = ca.dep + (size_t)ca.nl * ca.max_mb;
            ca.done = ca.next_tile + 1;
            ca.lag = 4;
            // a row group: about one wave of tiles over all layers
            ca.group = std::max(1, chain_grid() / std::max(1, sum_tiles));
            ca.slope = net.slope;
            ca.fl = fl;
            ev = pr.begin(s);
            CK(launch_tc_chain(ca, s));
            pr.end(PIFU_K_MLP_HIDDEN, ev, s, flops, bytes);
            continue;
        }
        for (int l = 0; l + 1 < L; ++l) {
            const DevLayer& Ly = net.layers[l];
            const TcLayer& T = net.tc[l];
            TcLayerArgs a{};
            a.tmA1 = l > 0 ? &T.tmA1 : &net.tmX;
            a.tmA2 = &net.tmX;
            a.tmW = &T.tmW;
            a.tmO = T.tmO_ok ? &T.tmO : nullptr;
            a.nk1 = T.nk1;
            a.nk2 = T.nk2;
            a.M = (int)mc;
            a.N = Ly.n_out;
            a.BN = T.BN;
            a.pair = T.pair ? 1 : 0;
            a.bias = Ly.b;
            a.slope = net.slope;
            a.out = ctx->Hb[l % 2];
            a.ldo = Ly.n_out;
            a.err = ctx->d_count + 1;
            a.m_dev = m_dev;
            a.fuse = (fuse && l == L - 2) ? &fl : nullptr;
            a.mode = TC_BF16;
            if (l < F) {
                // E4M3 operands; the last E4M3 layer hands BF16 to the next one
                const Fp8Layer& Q = net.f8[(size_t)l];
                a.tmA1 = l > 0 ? &Q.tmA1 : &net.tmX8;
                a.tmA2 = &net.tmX8;
                a.tmW = &Q.tmW;
                a.nk1 = Q.nk1;
                a.nk2 = Q.nk2;
                a.BN = Q.BN;
                a.pair = 0;
                a.mode = l + 1 < F ? TC_E4M3_E4M3 : TC_E4M3_BF16;
                a.colscale = Q.colscale;
                a.out_scale = Q.out_scale;
                if (a.fuse) return PIFU_ERR_UNSUPPORTED;
            }
            double flops = 2.0 * mc * Ly.fan_in * Ly.n_out;
            if (a.fuse) flops += 2.0 * mc * Ll.fan_in * Ll.n_out;
            ev = pr.begin(s);
            CK(launch_tc_linear(a, s));
            pr.end(PIFU_K_MLP_HIDDEN, ev, s, flops,
                   2.0 * ((double)mc * (Ly.fan_in + Ly.n_out) + (double)Ly.n_out * Ly.fan_in));
        }
        if (!fuse) {
            const __nv_bfloat16* h = L > 1 ? ctx->Hb[(L - 2) % 2] : nullptr;
            const int hw = L > 1 ? net.layers[L - 2].n_out : 0;
            ev = pr.begin(s);
            CK(launch_last_layer_bf16(p0, mc, Ll.n_out, h, hw, Ll.K1, ctx->Xb, net.ldx, Ll.K2,
                                      Ll.W, Ll.ldw, Ll.b, epi, s, m_dev));
            pr.end(PIFU_K_MLP_LAST, ev, s, 2.0 * mc * Ll.fan_in * Ll.n_out,
                   2.0 * (double)mc * (Ll.fan_in + Ll.n_out));
        }
    }
    return PIFU_OK;
}

// The CBN + SoftZ network on the tensor cores over a host-sized batch, in
// passes of at most kChunkTC points: gather (BF16 features, FP32 depth), then
// the whole network in one launch.
int run_cbn_tc(pifu_ctx* ctx, const PointSrc& src_in, int64_t m, const Map& map,
               const Calib& calib, const Epilogue& epi, cudaStream_t s,
               const unsigned int* m_dev) {
    CbnDev& d = ctx->cbn;
    if (!d.tc_ok) return PIFU_ERR_UNSUPPORTED;
    const CbnF32& f = d.f32;
    // a device-resident count is one pass of capacity m (the graph forms
    // reserve its rows before capture)
    const int64_t chunk = m_dev ? std::max<int64_t>(m, 1) : kChunkTC;
    if (m_dev && m > kTcRowsMax) return PIFU_ERR_ARG;
    {
        const int st = ensure_tc_rows(ctx, std::min<int64_t>(m, chunk));
        if (st != PIFU_OK) return st;
    }
    PointSrc src = src_in;
    src.count = m_dev;
    float* zbuf = reinterpret_cast<float*>(ctx->Hb[0]);
    const CbnTcMaps maps{&d.tmX, &d.tmG, &d.tmW};
    Profiler& pr = ctx->prof;
    const double flops_pt = 2.0 * ((double)f.n_z * f.K + 2.0 * f.nb * f.C * f.K +
                                   (double)(f.nb - 1) * f.K * f.K + f.K);
    for (int64_t p0 = 0; p0 < m; p0 += chunk) {
        const int64_t mc = std::min<int64_t>(chunk, m - p0);
        cudaEvent_t ev = pr.begin(s);
        CK(launch_cbn_gather(src, p0, mc, calib, map, ctx->Xb, f.C, zbuf, s));
        pr.end(PIFU_K_GATHER, ev, s, 0.0, (double)mc * (4.0 * 4.0 * map.C + 2.0 * f.C + 4.0));
        CbnTcArgs a{};
        a.zbuf = zbuf;
        a.WzT = f.WzT;
        a.bz = f.bz;
        a.g0 = d.g0;
        a.bl = d.bl;
        a.wlast = f.wlast;
        a.blast = f.blast;
        a.C = f.C;
        a.n_z = f.n_z;
        a.K = f.K;
        a.nb = f.nb;
        a.M = (int)mc;
        a.m_dev = m_dev;
        a.p0 = p0;
        a.err = ctx->d_count + 1;
        a.epi = epi;
        ev = pr.begin(s);
        CK(launch_cbn_tc(maps, a, s));
        pr.end(PIFU_K_CBN_TC, ev, s, flops_pt * (double)mc,
               2.0 * (double)mc * f.C + 2.0 * f.nb * (2.0 * f.C * f.K + (double)f.K * f.K));
    }
    return PIFU_OK;
}

int run_mlp(pifu_ctx* ctx, const DevNet& net, const PointSrc& src_in, int64_t m, const Map& map0,
            const Map& map1, const Calib& calib, const Epilogue& epi, cudaStream_t s,
            int precision = PIFU_PREC_FP32, const unsigned int* m_dev = nullptr,
            int fused_cl = 0) {
    if (net.kind == kNetCbn) {
        if (precision != PIFU_PREC_FP32)
            return run_mlp_tc(ctx, net, src_in, m, map0, map1, calib, epi, s, m_dev,
                              precision == PIFU_PREC_FP8);
        PointSrc srcc = src_in;
        srcc.count = m_dev;   // a device-resident count: persistent clusters
        const CbnF32& f = ctx->cbn.f32;
        const double flops = 2.0 * (double)m *
                             ((double)f.n_z * f.K + 2.0 * f.nb * f.C * f.K +
                              (double)(f.nb - 1) * f.K * f.K + f.K);
        const double wbytes = 4.0 * ((double)f.n_z * f.K + f.nb * (2.0 * f.C * f.K + f.K * f.K));
        cudaEvent_t ev = ctx->prof.begin(s);
        CK(launch_cbn_f32(f, srcc, m, calib, map0, epi, s));
        ctx->prof.end(PIFU_K_MLP_F32, ev, s, flops, wbytes + (double)m * 4.0 * (4.0 * map0.C + 1));
        return PIFU_OK;
    }
    if (precision == PIFU_PREC_BF16 || precision == PIFU_PREC_FP8)
        return run_mlp_tc(ctx, net, src_in, m, map0, map1, calib, epi, s, m_dev,
                          precision == PIFU_PREC_FP8);
    PointSrc src = src_in;
    src.count = m_dev;
    const int L = (int)net.layers.size();
    Profiler& pr = ctx->prof;
    const FusedNet fz = fused_of(net);
    if ((m_dev || m <= kFusedMaxM) && fused_ok(fz)) {
        // the whole network in one launch (gather included)
        double flops = 0.0, wbytes = 0.0;
        for (const DevLayer& Ly : net.layers) {
            flops += 2.0 * (double)m * Ly.fan_in * Ly.n_out;
            wbytes += 4.0 * (double)Ly.n_out * (Ly.fan_in + 1);
        }
        cudaEvent_t ev = pr.begin(s);
        CK(launch_mlp_fused(fz, src, 0, m, calib, map0, map1, epi, s, fused_cl));
        pr.end(PIFU_K_MLP_F32, ev, s, flops,
               wbytes + (double)m * 4.0 * (4.0 * (map0.C + map1.C) + net.layers[L - 1].n_out));
        return PIFU_OK;
    }
    // a device-resident batch size uses the split-K kernels, sized for m <= kRecheckCap
    if (m_dev && m > kRecheckCap) return PIFU_ERR_ARG;
    for (int64_t p0 = 0; p0 < m; p0 += kChunk) {
        const int64_t mc = std::min<int64_t>(kChunk, m - p0);
        // gather: 4 taps x C channels read (L2), one padded row written
        cudaEvent_t ev = pr.begin(s);
        CK(launch_gather(src, p0, mc, calib, map0, map1, ctx->X, net.ldx, s));
        pr.end(PIFU_K_GATHER, ev, s, 0.0,
               (double)mc * (4.0 * (map0.C + map1.C) + net.ldx) * 4.0);
        const float* h = nullptr;
        int hw = 0;
        for (int l = 0; l + 1 < L; ++l) {
            const DevLayer& Ly = net.layers[l];
            float* out = (l % 2 == 0) ? ctx->HA : ctx->HB;
            ev = pr.begin(s);
            CK(launch_sgemm_bias_lrelu((int)mc, Ly.n_out, h, hw, Ly.K1, ctx->X, net.ldx, Ly.K2, Ly.W,
                                       Ly.ldw, Ly.b, net.slope, out, Ly.n_out, s, ctx->part,
                                       m_dev));
            pr.end(PIFU_K_MLP_F32, ev, s, 2.0 * mc * Ly.fan_in * Ly.n_out,
                   4.0 * ((double)mc * (Ly.fan_in + Ly.n_out) + (double)Ly.n_out * (Ly.fan_in + 1)));
            h = out;
            hw = Ly.n_out;
        }
        const DevLayer& Ll = net.layers[L - 1];
        ev = pr.begin(s);
        CK(launch_last_layer(p0, mc, Ll.n_out, h, hw, Ll.K1, ctx->X, net.ldx, Ll.K2, Ll.W, Ll.ldw,
                             Ll.b, epi, s, m_dev));
        pr.end(PIFU_K_MLP_LAST, ev, s, 2.0 * mc * Ll.fan_in * Ll.n_out,
               4.0 * (double)mc * (Ll.fan_in + Ll.n_out));
    }
    return PIFU_OK;
}

// Mixed precision over one batch: the tensor-core BF16 pass commits every
// occupancy farther than `margin` from 0.5 and queues the others (node
// indices for a level, point numbers otherwise) on ctx->recheck; the queued
// ones are then evaluated again in FP32 and committed.  One host read of the
// queue length per batch.  *rechecked += the queue length.
int read_recheck(pifu_ctx* ctx, cudaStream_t s, unsigned int* out);

int run_mlp_mixed(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                  const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                  float margin, cudaStream_t s, int64_t* rechecked, bool f8 = false) {
    if (m > ctx->recheck_cap) return PIFU_ERR_ARG;
    // A tiny batch costs less in FP32 outright than in BF16 plus a re-check
    // pass (both are latency-bound there); FP32 is the re-check's arithmetic.
    if (m <= kTinyBatch) return run_mlp(ctx, net, src, m, map0, map1, calib, epi, s, PIFU_PREC_FP32);
    CK(cudaMemsetAsync(ctx->d_recheck, 0, sizeof(unsigned int), s));
    Epilogue e1 = epi;
    e1.recheck = ctx->recheck;
    e1.recheck_count = ctx->d_recheck;
    e1.margin = margin;
    int st = run_mlp_tc(ctx, net, src, m, map0, map1, calib, e1, s, nullptr, f8);
    if (st != PIFU_OK) return st;
    unsigned int n = 0;
    st = read_recheck(ctx, s, &n);
    if (st != PIFU_OK) return st;
    if (rechecked) *rechecked += n;
    if (n == 0) return PIFU_OK;
    PointSrc s2 = src;
    Epilogue e2 = epi;
    if (epi.mode == EPI_LEVEL || epi.mode == EPI_COLUMN) {
        // the queue holds keys of the same kind as the batch's
        s2.mode = epi.mode == EPI_COLUMN ? PTS_COLUMN : PTS_LIST;
        s2.list = ctx->recheck;
        e2.list = ctx->recheck;
    } else {
        // EPI_STORE over positions: point numbers index the batch's arrays
        s2.mode = PTS_XYZ_IDX;
        s2.list = ctx->recheck;
        e2.pix = ctx->recheck;
    }
    return run_mlp(ctx, net, s2, n, map0, map1, calib, e2, s, PIFU_PREC_FP32);
}

int read_recheck(pifu_ctx* ctx, cudaStream_t s, unsigned int* out) {
    CK(cudaMemcpyAsync(ctx->h_recheck, ctx->d_recheck, sizeof(unsigned int),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = *ctx->h_recheck;
    return PIFU_OK;
}

// One evaluation batch of a level: the plain/BF16/MIXED network, or, at a
// coarse level with the surrogate on, f_S first and f_O for the occupancies
// f_S puts within `sur_margin` of 0.5 (one host read of that queue).
int eval_level_batch(pifu_ctx* ctx, const PointSrc& src, int64_t n, const Map& map,
                     const Calib& cal, const Epilogue& epi, int prec, float margin, bool surrogate,
                     float sur_margin, cudaStream_t s, int64_t* rechecked, int64_t* fallback) {
    const DevNet& fo = ctx->net[0];
    if (!surrogate) {
        return prec_mixed(prec)
                   ? run_mlp_mixed(ctx, fo, src, n, map, Map{}, cal, epi, margin, s, rechecked,
                                   prec == PIFU_PREC_FP8_MIXED)
                   : run_mlp(ctx, fo, src, n, map, Map{}, cal, epi, s, prec);
    }
    if (n > ctx->recheck_cap) return PIFU_ERR_ARG;
    CK(cudaMemsetAsync(ctx->d_squeue, 0, sizeof(unsigned int), s));
    Epilogue es = epi;
    es.recheck = ctx->squeue;
    es.recheck_count = ctx->d_squeue;
    es.margin = sur_margin;
    int st = run_mlp(ctx, ctx->snet, src, n, map, Map{}, cal, es, s,
                     prec == PIFU_PREC_FP32 || !ctx->snet.tc_ok ? PIFU_PREC_FP32 : PIFU_PREC_BF16);
    if (st != PIFU_OK) return st;
    CK(cudaMemcpyAsync(ctx->h_squeue, ctx->d_squeue, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const unsigned int nf = *ctx->h_squeue;
    if (fallback) *fallback += nf;
    if (nf == 0) return PIFU_OK;
    PointSrc sf{PTS_LIST, nullptr, ctx->squeue, 0, src.N, nullptr};
    Epilogue ef = epi;
    ef.list = ctx->squeue;
    return eval_level_batch(ctx, sf, nf, map, cal, ef, prec, margin, false, 0.f, s, rechecked,
                            nullptr);
}

// View-culled final level workspaces: candidate keys (16 per pixel) and the
// dense per-(pixel, depth node) occupancy store (touched only at candidates).
int ensure_cull_ws(pifu_ctx* ctx, int64_t npix, int Nc) {
    const int64_t cap = npix * 16;
    const int64_t vals = npix * (2 * (int64_t)Nc + 1);
    if (cap > ctx->cull_cap) {
        dev_free(ctx->cull_list);
        ctx->cull_cap = 0;
        CK(dev_alloc(&ctx->cull_list, cap));
        ctx->cull_cap = cap;
    }
    if (vals > ctx->cull_vals_cap) {
        dev_free(ctx->cull_values);
        ctx->cull_vals_cap = 0;
        CK(dev_alloc(&ctx->cull_values, vals));
        ctx->cull_vals_cap = vals;
    }
    return PIFU_OK;
}

// One host-sized evaluation batch in the given arithmetic (FP32, the tensor-
// core forms, or those with the FP32 re-check).
int eval_batch(pifu_ctx* ctx, const PointSrc& src, int64_t n, const Map& map, const Calib& cal,
               const Epilogue& epi, int prec, float margin, cudaStream_t s) {
    const DevNet& fo = ctx->net[0];
    if (prec_mixed(prec))
        return run_mlp_mixed(ctx, fo, src, n, map, Map{}, cal, epi, margin, s, nullptr,
                             prec == PIFU_PREC_FP8_MIXED);
    return run_mlp(ctx, fo, src, n, map, Map{}, cal, epi, s, prec);
}

// Conflict list of the graph forms' rounds (keys), at least `cap` entries.
int ensure_clist(pifu_ctx* ctx, int64_t cap) {
    if (!ctx->d_ccount) CK(dev_alloc(&ctx->d_ccount, 1));
    if (cap > ctx->clist_cap) {
        dev_free(ctx->clist);
        ctx->clist_cap = 0;
        CK(dev_alloc(&ctx->clist, cap));
        ctx->clist_cap = cap;
    }
    return PIFU_OK;
}

// Point OHEM state for m tuples (weights 1) and a sampled batch of B rows.
int ohem_ensure(pifu_ctx* ctx, int64_t m, int B, bool reset) {
    auto& S = ctx->sur;
    if (m != S.ohem_m) {
        dev_free(S.ohem_w);
        dev_free(S.ohem_cdf);
        dev_free(S.ohem_sums);
        S.ohem_m = 0;
        CK(dev_alloc(&S.ohem_w, m));
        CK(dev_alloc(&S.ohem_cdf, m));
        CK(dev_alloc(&S.ohem_sums, ohem_scan_blocks(m)));
        S.ohem_m = m;
        reset = true;
    }
    if (reset) CK(launch_fill(m, S.ohem_w, 1.0f, nullptr));
    if (B > S.ohem_B) {
        dev_free(S.xb);
        dev_free(S.yb);
        dev_free(S.ib);
        dev_free(S.per_loss);
        S.ohem_B = 0;
        CK(dev_alloc(&S.xb, (int64_t)B * ctx->snet.ldx));
        CK(dev_alloc(&S.yb, B));
        CK(dev_alloc(&S.ib, B));
        CK(dev_alloc(&S.per_loss, B));
        S.ohem_B = B;
    }
    return PIFU_OK;
}

int decode_err(unsigned int e) {
    if (e & kErrCapacity) return PIFU_ERR_CAPACITY;
    if (e & kErrNotConverged) return PIFU_ERR_NOT_CONVERGED;
    return PIFU_ERR_TIMEOUT;
}

// Reads the list length and the device error word (set by a bounded wait
// that gave up); a set error word is cleared and reported as a timeout.
int read_count(pifu_ctx* ctx, cudaStream_t s, unsigned int* out) {
    CK(cudaMemcpyAsync(ctx->h_count, ctx->d_count, 2 * sizeof(unsigned int),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = ctx->h_count[0];
    if (ctx->h_count[1] != 0u) {
        const unsigned int e = ctx->h_count[1];
        CK(cudaMemsetAsync(ctx->d_count + 1, 0, sizeof(unsigned int), s));
        return decode_err(e);
    }
    return PIFU_OK;
}

}  // namespace

namespace {

// ---- learned surrogate f_S ---------------------------------------------------
//
// Not in the paper: a small MLP of the same family, distilled from f_O on
// (features, depth, occupancy) tuples that f_O itself produces, and used at
// the coarse levels where only the side of 0.5 matters.  Occupancies it puts
// within a margin of 0.5 fall back to f_O.  Training runs entirely in the
// library's kernels (train.cu): FP32 forward, mean BCE, back-propagation,
// Adam.

uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void sur_free(pifu_ctx* ctx) {
    auto& S = ctx->sur;
    dev_free(S.params);
    dev_free(S.grads);
    dev_free(S.adam_m);
    dev_free(S.adam_v);
    dev_free(S.H1);
    dev_free(S.H2);
    dev_free(S.logit);
    dev_free(S.g);
    dev_free(S.dH1);
    dev_free(S.dH2);
    dev_free(S.ones);
    dev_free(S.d_loss);
    if (S.h_loss) cudaFreeHost(S.h_loss);
    S.h_loss = nullptr;
    for (auto& T : ctx->snet.tc) dev_free(T.W);
    ctx->snet.tc.clear();
    ctx->snet.layers.clear();
    ctx->snet.tc_ok = false;
    S.ready = false;
    S.batch_cap = 0;
    dev_free(S.ohem_w);
    dev_free(S.ohem_cdf);
    dev_free(S.ohem_sums);
    dev_free(S.xb);
    dev_free(S.yb);
    dev_free(S.ib);
    dev_free(S.per_loss);
    S.ohem_m = 0;
    S.ohem_B = 0;
}

// The FP32 runner's view of f_S (weights inside the flat parameter buffer).
void sur_bind(pifu_ctx* ctx) {
    auto& S = ctx->sur;
    const DevNet& fo = ctx->net[0];
    DevNet& n = ctx->snet;
    n.kind = 0;
    n.d_in = fo.d_in;
    n.ldx = fo.ldx;
    n.slope = fo.slope;
    n.max_hidden = std::max(S.h1, S.h2);
    n.layers.assign(3, DevLayer{});
    const int widths[3] = {S.h1, S.h2, 1};
    for (int l = 0; l < 3; ++l) {
        DevLayer& L = n.layers[l];
        L.n_out = widths[l];
        L.K1 = l == 0 ? 0 : widths[l - 1];
        L.K2 = l == 0 ? fo.ldx : 0;
        L.ldw = L.K1 + L.K2;
        L.fan_in = l == 0 ? fo.d_in : widths[l - 1];
        L.W = S.params + S.off_w[l];
        L.b = S.params + S.off_b[l];
    }
}

// Rebuild the BF16 tensor-core form of f_S from its current parameters.
int sur_build_tc(pifu_ctx* ctx) {
    auto& S = ctx->sur;
    DevNet& n = ctx->snet;
    ++S.version;
    for (auto& T : n.tc) dev_free(T.W);
    n.tc.clear();
    std::vector<float> p((size_t)S.n);
    CK(cudaMemcpy(p.data(), S.params, (size_t)S.n * 4, cudaMemcpyDeviceToHost));
    HostNet hn;
    hn.shape = n;
    hn.W.resize(3);
    hn.b.resize(3);
    for (int l = 0; l < 3; ++l) {
        const DevLayer& L = n.layers[l];
        hn.W[l].assign(p.begin() + S.off_w[l], p.begin() + S.off_w[l] + (int64_t)L.n_out * L.ldw);
        hn.b[l].assign(p.begin() + S.off_b[l], p.begin() + S.off_b[l] + round_up(L.n_out, 4));
    }
    return build_tc(ctx, hn, n);
}

int encode_all_act_maps(pifu_ctx* ctx) {
    for (DevNet& n : ctx->net) {
        const int st = encode_act_maps(ctx, n);
        if (st != PIFU_OK) return st;
    }
    CbnDev& cb = ctx->cbn;
    if (cb.tc_ok && ctx->tc_rows > 0 &&
        !tc_encode_2d_bf16(&cb.tmX, ctx->Xb, (uint64_t)cb.f32.C, (uint64_t)ctx->tc_rows,
                           (uint64_t)cb.f32.C * 2, 64, 128))
        return PIFU_ERR_CUDA;
    return ctx->sur.ready ? encode_act_maps(ctx, ctx->snet) : PIFU_OK;
}

int sur_init(pifu_ctx* ctx, int h1, int h2, uint64_t seed) {
    sur_free(ctx);
    auto& S = ctx->sur;
    const DevNet& fo = ctx->net[0];
    S.h1 = h1;
    S.h2 = h2;
    const int ldx = fo.ldx;
    const int64_t sizes_w[3] = {(int64_t)h1 * ldx, (int64_t)h2 * h1, (int64_t)h2};
    const int64_t sizes_b[3] = {round_up(h1, 4), round_up(h2, 4), 4};
    int64_t off = 0;
    for (int l = 0; l < 3; ++l) {
        S.off_w[l] = off;
        off += sizes_w[l];
        S.off_b[l] = off;
        off += sizes_b[l];
    }
    S.n = off;
    // Kaiming-uniform weights (leaky-ReLU gain) from a splitmix64 stream,
    // zero biases; padding columns stay zero.
    std::vector<float> p((size_t)off, 0.f);
    uint64_t st = seed;
    const int fan[3] = {fo.d_in, h1, h2};
    const int rows[3] = {h1, h2, 1};
    const int ld[3] = {ldx, h1, h2};
    for (int l = 0; l < 3; ++l) {
        const double bound = std::sqrt(6.0 / fan[l]) / (l == 2 ? std::sqrt(2.0) : 1.0);
        for (int r = 0; r < rows[l]; ++r)
            for (int k = 0; k < fan[l]; ++k) {
                const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
                p[(size_t)(S.off_w[l] + (int64_t)r * ld[l] + k)] = (float)((2.0 * u - 1.0) * bound);
            }
    }
    CK(dev_alloc(&S.params, off));
    CK(dev_alloc(&S.grads, off));
    CK(dev_alloc(&S.adam_m, off));
    CK(dev_alloc(&S.adam_v, off));
    CK(cudaMemcpy(S.params, p.data(), (size_t)off * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(S.adam_m, 0, (size_t)off * 4));
    CK(cudaMemset(S.adam_v, 0, (size_t)off * 4));
    CK(dev_alloc(&S.d_loss, 1));
    CK(cudaHostAlloc(&S.h_loss, sizeof(double), cudaHostAllocDefault));
    S.step = 0;
    S.ready = true;
    sur_bind(ctx);
    return sur_build_tc(ctx);
}

int sur_batch_ws(pifu_ctx* ctx, int B) {
    auto& S = ctx->sur;
    if (B <= S.batch_cap) return PIFU_OK;
    float** bufs[] = {&S.H1, &S.H2, &S.logit, &S.g, &S.dH1, &S.dH2, &S.ones};
    for (auto b : bufs) dev_free(*b);
    S.batch_cap = 0;
    CK(dev_alloc(&S.H1, (int64_t)B * S.h1));
    CK(dev_alloc(&S.dH1, (int64_t)B * S.h1));
    CK(dev_alloc(&S.H2, (int64_t)B * S.h2));
    CK(dev_alloc(&S.dH2, (int64_t)B * S.h2));
    CK(dev_alloc(&S.logit, B));
    CK(dev_alloc(&S.g, B));
    CK(dev_alloc(&S.ones, B));
    CK(launch_fill(B, S.ones, 1.f, 0));
    CK(cudaDeviceSynchronize());
    S.batch_cap = B;
    return PIFU_OK;
}

// Forward + backward of f_S on one batch (rows x: [B][ldx], targets y):
// gradients into S.grads, mean BCE added to *S.d_loss.
int sur_grad(pifu_ctx* ctx, const float* x, const float* y, int B, cudaStream_t s,
             float* per_loss = nullptr) {
    auto& S = ctx->sur;
    const int ldx = ctx->snet.ldx;
    const float slope = ctx->snet.slope;
    float* P = S.params;
    float* G = S.grads;
    const int h1 = S.h1, h2 = S.h2;
    const int red = std::max(1, B / 256);   // reduction slices over the batch
    // forward
    CK(launch_gemm_strided(B, h1, ldx, x, ldx, 1, P + S.off_w[0], 1, ldx, S.H1, h1, 1, 0, s));
    CK(launch_bias_lrelu(B, h1, S.H1, h1, P + S.off_b[0], slope, s));
    CK(launch_gemm_strided(B, h2, h1, S.H1, h1, 1, P + S.off_w[1], 1, h1, S.H2, h2, 1, 0, s));
    CK(launch_bias_lrelu(B, h2, S.H2, h2, P + S.off_b[1], slope, s));
    CK(launch_gemm_strided(B, 1, h2, S.H2, h2, 1, P + S.off_w[2], 1, h2, S.logit, 1, 1, 0, s));
    CK(launch_bce_grad(B, S.logit, P + S.off_b[2], y, S.g, S.d_loss, s, per_loss));
    // backward
    CK(cudaMemsetAsync(G, 0, (size_t)S.n * 4, s));
    // layer 3: dW3 = g^T H2, db3 = sum g, dH2 = g W3
    CK(launch_gemm_strided(1, h2, B, S.g, 0, 1, S.H2, h2, 1, G + S.off_w[2], h2, red, 1, s));
    CK(launch_gemm_strided(1, 1, B, S.g, 0, 1, S.ones, 1, 0, G + S.off_b[2], 1, red, 1, s));
    CK(launch_gemm_strided(B, h2, 1, S.g, 1, 0, P + S.off_w[2], 0, 1, S.dH2, h2, 1, 0, s));
    CK(launch_lrelu_backward((int64_t)B * h2, S.dH2, S.H2, slope, s));
    // layer 2: dW2 = dZ2^T H1, db2 = column sums, dH1 = dZ2 W2
    CK(launch_gemm_strided(h2, h1, B, S.dH2, 1, h2, S.H1, h1, 1, G + S.off_w[1], h1, red, 1, s));
    CK(launch_gemm_strided(h2, 1, B, S.dH2, 1, h2, S.ones, 1, 0, G + S.off_b[1], 1, red, 1, s));
    CK(launch_gemm_strided(B, h1, h2, S.dH2, h2, 1, P + S.off_w[1], h1, 1, S.dH1, h1, 1, 0, s));
    CK(launch_lrelu_backward((int64_t)B * h1, S.dH1, S.H1, slope, s));
    // layer 1: dW1 = dZ1^T X (padding columns of X are 0, so are theirs), db1
    CK(launch_gemm_strided(h1, ldx, B, S.dH1, 1, h1, x, ldx, 1, G + S.off_w[0], ldx, red, 1, s));
    CK(launch_gemm_strided(h1, 1, B, S.dH1, 1, h1, S.ones, 1, 0, G + S.off_b[0], 1, red, 1, s));
    return PIFU_OK;
}

// Unpadded parameter layout (the blob's order): per layer W[n_out][fan_in], b.
int64_t sur_unpadded_count(const pifu_ctx* ctx) {
    const auto& S = ctx->sur;
    const int fi = ctx->snet.d_in;
    return (int64_t)S.h1 * fi + S.h1 + (int64_t)S.h2 * S.h1 + S.h2 + S.h2 + 1;
}

void sur_pack(const pifu_ctx* ctx, const std::vector<float>& padded, float* out) {
    const auto& S = ctx->sur;
    const DevNet& n = ctx->snet;
    int64_t o = 0;
    for (int l = 0; l < 3; ++l) {
        const DevLayer& L = n.layers[l];
        for (int r = 0; r < L.n_out; ++r)
            for (int k = 0; k < L.fan_in; ++k) out[o++] = padded[(size_t)(S.off_w[l] + (int64_t)r * L.ldw + k)];
        for (int r = 0; r < L.n_out; ++r) out[o++] = padded[(size_t)(S.off_b[l] + r)];
    }
}

void sur_unpack(const pifu_ctx* ctx, const float* in, std::vector<float>& padded) {
    const auto& S = ctx->sur;
    const DevNet& n = ctx->snet;
    padded.assign((size_t)S.n, 0.f);
    int64_t o = 0;
    for (int l = 0; l < 3; ++l) {
        const DevLayer& L = n.layers[l];
        for (int r = 0; r < L.n_out; ++r)
            for (int k = 0; k < L.fan_in; ++k) padded[(size_t)(S.off_w[l] + (int64_t)r * L.ldw + k)] = in[o++];
        for (int r = 0; r < L.n_out; ++r) padded[(size_t)(S.off_b[l] + r)] = in[o++];
    }
}

// ---- graph form: one CUDA graph per frame ------------------------------------
//
// pifu_frame captures localization + render once per argument set and then
// relaunches the graph.  Batch sizes never come back to the host: the MLP
// launches are sized for a capacity and read the true size from the
// device counter the previous kernel wrote, and each level's conflict loop is
// a conditional WHILE node whose body ends with a kernel that sets the
// condition from the new frontier's size.  The host synchronises once, at the
// end of the frame, to read the counters and the error word.

int g_add_cond(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h,
               cudaGraphConditionalNodeType type, cudaGraph_t* body);

int g_add_switch(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, int n,
                 cudaGraph_t* bodies);
int64_t launches_now(const pifu_ctx* ctx);

// The FP32 pass over a device-sized queue in the graph.  With the fused
// kernel, a switch node set on the device from the queue length launches it
// with the cluster size that length calls for (few points: large clusters,
// the lowest latency per tile; many: small clusters, more tiles per round).
int g_recheck(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t cap,
              const Map& map, const Calib& cal, const Epilogue& epi, cudaStream_t s,
              const unsigned int* m_dev) {
    const FusedNet fz = fused_of(net);
    const bool sw = net.kind != kNetCbn && ctx->cap_stream4 && s != ctx->cap_stream4 &&
                    fused_ok(fz);
    const FusedPlan plan = sw ? fused_plan(fz) : FusedPlan{};
    if (plan.n <= 1)
        return run_mlp(ctx, net, src, cap, map, Map{}, cal, epi, s, PIFU_PREC_FP32, m_dev);
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
    CK(launch_fused_switch(h, plan, m_dev, (unsigned)cap, s));
    cudaGraph_t bodies[4] = {};
    int st = g_add_switch(ctx, s, h, plan.n, bodies);
    if (st != PIFU_OK) return st;
    cudaStream_t s4 = ctx->cap_stream4;
    const int64_t before = launches_now(ctx);
    for (int i = 0; i < plan.n; ++i) {
        CK(cudaStreamBeginCaptureToGraph(s4, bodies[i], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        st = run_mlp(ctx, net, src, cap, map, Map{}, cal, epi, s4, PIFU_PREC_FP32, m_dev,
                     plan.cl[i]);
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(s4, &out);
        if (st != PIFU_OK) return st;
        if (ee != cudaSuccess) return fail_cuda(ctx, ee);
    }
    // one body runs per replay: count its launches once
    const int64_t per_body = (launches_now(ctx) - before) / plan.n;
    ctx->prof.k[PIFU_K_MLP_F32].launches -= (launches_now(ctx) - before) - per_body;
    return PIFU_OK;
}

// One evaluation batch in the graph: BF16 on the tensor cores, and for MIXED
// the FP32 re-evaluation of the queued near-0.5 occupancies (device-sized).
// With `sur`, f_S runs first and f_O takes the occupancies f_S put within
// `sur_margin` of 0.5 (a device-sized queue; *fallback += its length).
int g_eval(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t cap,
           const unsigned int* m_dev, const Map& map, const Calib& cal, const Epilogue& epi,
           int prec, float margin, unsigned long long* rechecked, cudaStream_t s,
           bool sur = false, float sur_margin = 0.f, unsigned long long* fallback = nullptr) {
    if (sur) {
        CK(cudaMemsetAsync(ctx->d_squeue, 0, sizeof(unsigned int), s));
        Epilogue es = epi;
        es.recheck = ctx->squeue;
        es.recheck_count = ctx->d_squeue;
        es.margin = sur_margin;
        int st = run_mlp_tc(ctx, ctx->snet, src, cap, map, Map{}, cal, es, s, m_dev);
        if (st != PIFU_OK) return st;
        // a queue longer than one device-sized batch latches a capacity error
        const int64_t qcap = std::min<int64_t>(cap, kTcRowsMax);
        CK(launch_accumulate(fallback, ctx->d_squeue, (unsigned)qcap, ctx->d_count + 1, s));
        PointSrc sf = src;   // keeps the frames' maps of a lockstep batch
        sf.mode = PTS_LIST;
        sf.list = ctx->squeue;
        sf.base = 0;
        sf.count = nullptr;
        Epilogue ef = epi;
        ef.list = ctx->squeue;
        return g_eval(ctx, net, sf, qcap, ctx->d_squeue, map, cal, ef, prec, margin, rechecked, s);
    }
    if (prec == PIFU_PREC_BF16 || prec == PIFU_PREC_FP8)
        return run_mlp_tc(ctx, net, src, cap, map, Map{}, cal, epi, s, m_dev,
                          prec == PIFU_PREC_FP8);
    if (m_dev && ctx->cap_stream3 && s != ctx->cap_stream3) {
        // A device-sized batch of at most kTinyBatch points goes straight to
        // FP32 (one fused launch), as in the host-driven form; the tensor-core
        // pass and its re-check run above that.  Two IF nodes, set on the device.
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle hs, hl;
        CK(cudaGraphConditionalHandleCreate(&hs, cg, 0, 0));
        CK(cudaGraphConditionalHandleCreate(&hl, cg, 0, 0));
        CK(launch_branch(hs, hl, m_dev, (unsigned)kTinyBatch, s));
        cudaStream_t s3 = ctx->cap_stream3;
        for (int br = 0; br < 2; ++br) {
            cudaGraph_t body = nullptr;
            int st = g_add_cond(ctx, s, br == 0 ? hs : hl, cudaGraphCondTypeIf, &body);
            if (st != PIFU_OK) return st;
            CK(cudaStreamBeginCaptureToGraph(s3, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
            if (br == 0)
                st = g_recheck(ctx, net, src, cap, map, cal, epi, s3, m_dev);
            else
                st = g_eval(ctx, net, src, cap, m_dev, map, cal, epi, prec, margin, rechecked, s3);
            cudaGraph_t out = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(s3, &out);
            if (st != PIFU_OK) return st;
            if (ee != cudaSuccess) return fail_cuda(ctx, ee);
        }
        return PIFU_OK;
    }
    CK(cudaMemsetAsync(ctx->d_recheck, 0, sizeof(unsigned int), s));
    Epilogue e1 = epi;
    e1.recheck = ctx->recheck;
    e1.recheck_count = ctx->d_recheck;
    e1.margin = margin;
    int st = run_mlp_tc(ctx, net, src, cap, map, Map{}, cal, e1, s, m_dev,
                        prec == PIFU_PREC_FP8_MIXED);
    if (st != PIFU_OK) return st;
    PointSrc s2 = src;   // keeps the frames' maps of a lockstep batch
    s2.mode = src.mode == PTS_COLUMN ? PTS_COLUMN : PTS_LIST;   // the queue holds keys
    s2.list = ctx->recheck;
    s2.base = 0;
    s2.count = nullptr;
    Epilogue e2 = epi;
    e2.list = ctx->recheck;
    // the fused kernel takes any queue length (at most the batch's); the
    // split-K path has a fixed capacity
    const int64_t rcap = (net.kind == kNetCbn || fused_ok(fused_of(net))) ? cap : kRecheckCap;
    st = g_recheck(ctx, net, s2, rcap, map, cal, e2, s, ctx->d_recheck);
    if (st != PIFU_OK) return st;
    CK(launch_accumulate(rechecked, ctx->d_recheck, (unsigned)rcap, ctx->d_count + 1, s));
    return PIFU_OK;
}

// Appends a WHILE node to the capture of `s` (after everything captured so
// far) and returns its body graph; the condition is set by the kernel that
// was captured last (launch_loop_control).
int g_add_cond(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h,
               cudaGraphConditionalNodeType type, cudaGraph_t* body);

int g_add_while(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    return g_add_cond(ctx, s, h, cudaGraphCondTypeWhile, body);
}

// Appends a conditional node of `type` to the capture of `s` (after
// everything captured so far) and returns its body graph.
int g_add_cond(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h,
               cudaGraphConditionalNodeType type, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, &edata, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return PIFU_ERR_STATE;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, edata, ndeps, &np));
    *body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return PIFU_OK;
}

// Appends a SWITCH node with n bodies to the capture of `s`; the condition
// is set by the kernel that was captured last (launch_fused_switch).
int g_add_switch(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, int n,
                 cudaGraph_t* bodies) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, &edata, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return PIFU_ERR_STATE;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeSwitch;
    np.conditional.size = (unsigned)n;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, edata, ndeps, &np));
    for (int i = 0; i < n; ++i) bodies[i] = np.conditional.phGraph_out[i];
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return PIFU_OK;
}

int64_t launches_now(const pifu_ctx* ctx) {
    int64_t n = 0;
    for (const auto& k : ctx->prof.k) n += k.launches;
    return n;
}

// The frame, captured on ctx->cap_stream (loop bodies on cap_stream2).
int g_enqueue_frame(pifu_ctx* ctx, const FrameKey& k, const Map& occ, const Map& col,
                    const Calib& cal) {
    cudaStream_t s = ctx->cap_stream;
    cudaStream_t sb = ctx->cap_stream2;
    GraphStats* gs = ctx->d_gstats;
    unsigned int* err = ctx->d_count + 1;
    const DevNet& net = ctx->net[0];
    int st = PIFU_OK;
    CK(cudaMemsetAsync(gs, 0, sizeof(GraphStats), s));
    CK(cudaMemsetAsync(err, 0, sizeof(unsigned int), s));
    // level 0: every node
    int N = k.n0, cur = 0;
    CK(launch_dense_setup(N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval, ctx->conf[0], s));
    {
        const int64_t nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
        PointSrc src{PTS_DENSE, nullptr, nullptr, 0, N, nullptr};
        Epilogue epi{};
        epi.mode = EPI_LEVEL;
        epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[0], N, row_words_of(N), 1};
        st = g_eval(ctx, net, src, nodes, nullptr, occ, cal, epi, k.precision, k.margin,
                    &gs->rechecked[0], s, k.use_surrogate && k.num_levels > 1, k.sur_margin,
                    &gs->fallback[0]);
        if (st != PIFU_OK) return st;
    }
    for (int l = 1; l < k.num_levels; ++l) {
        const int prev = cur;
        cur ^= 1;
        N *= 2;
        CK(launch_classify(ctx->bin[prev], N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval,
                           ctx->conf[0], s));
        CK(launch_popcount(ctx->cand, words_of(N), &gs->cands[l], s));
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
        CK(launch_dilate_select(ctx->cand, ctx->eval, nullptr, N, ctx->list, ctx->d_count, s));
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
        CK(launch_loop_control(h, ctx->d_count, (unsigned)kChunkTC, &gs->rounds[l], 0, k.max_rounds,
                               err, s));
        cudaGraph_t body = nullptr;
        st = g_add_while(ctx, s, h, &body);
        if (st != PIFU_OK) return st;
        // loop body: evaluate the list, then the unevaluated ring of its conflicts
        const int64_t before = launches_now(ctx);
        CK(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        {
            const int rw = row_words_of(N);
            PointSrc src{PTS_LIST, nullptr, ctx->list, 0, N, nullptr};
            Epilogue epi{};
            epi.mode = EPI_LEVEL;
            epi.list = ctx->list;
            epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[0], N, rw, 0};
            // the round's conflicts as a list: the next frontier is their
            // unevaluated 26-neighbours, found in work proportional to them
            epi.lv.clist = ctx->clist;
            epi.lv.ccount = ctx->d_ccount;
            epi.lv.ccap = (unsigned)ctx->clist_cap;
            epi.lv.err = err;
            st = launch_accumulate(&gs->evals[l], ctx->d_count, (unsigned)kChunkTC, err, sb) == cudaSuccess
                     ? PIFU_OK : PIFU_ERR_CUDA;
            if (st == PIFU_OK &&
                cudaMemsetAsync(ctx->d_ccount, 0, sizeof(unsigned int), sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            if (st == PIFU_OK)
                st = g_eval(ctx, net, src, kChunkTC, ctx->d_count, occ, cal, epi, k.precision,
                            k.margin, &gs->rechecked[l], sb,
                            k.use_surrogate && l < k.num_levels - 1, k.sur_margin,
                            &gs->fallback[l]);
            if (st == PIFU_OK && cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            if (st == PIFU_OK &&
                launch_expand_conflicts(ctx->clist, ctx->d_ccount, (unsigned)kChunkTC, N, ctx->eval,
                                        0, 0, ctx->list, ctx->d_count, (unsigned)kChunkTC, err,
                                        sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            if (st == PIFU_OK && launch_loop_control(h, ctx->d_count, (unsigned)kChunkTC,
                                                     &gs->rounds[l], 1, k.max_rounds, err,
                                                     sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
        }
        cudaGraph_t body_out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(sb, &body_out);
        if (st != PIFU_OK) return st;
        if (ee != cudaSuccess) return fail_cuda(ctx, ee);
        ctx->g_launches_body[l] = launches_now(ctx) - before;
    }
    if (k.final_level) {
        // the view-culled final level at 2 N depth nodes, then colour
        CullArgs c{};
        c.width = k.width;
        c.height = k.height;
        c.Nc = N;
        c.row_words = row_words_of(N);
        c.bin = ctx->bin[cur];
        c.list = ctx->cull_list;
        c.count = ctx->d_count;
        c.cap = (unsigned)std::min<int64_t>(ctx->cull_cap, kChunkTC);
        c.err = err;
        c.values = ctx->cull_values;
        for (int q = 0; q < 3; ++q) c.bg[q] = k.bg[q];
        c.depth = k.depth;
        c.rgb = k.rgb;
        c.mask = k.mask;
        c.hit_xyz = ctx->hit_xyz;
        c.hit_pix = ctx->hit_pix;
        c.hit_count = ctx->d_count;
        c.top = ctx->col_top;
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
        CK(launch_cull_select(c, s));
        CK(launch_accumulate(&gs->culled, ctx->d_count, c.cap, err, s));
        PointSrc src{PTS_COLUMN, nullptr, ctx->cull_list, 0, 2 * N, nullptr};
        src.width = k.width;
        Epilogue epi{};
        epi.mode = EPI_COLUMN;
        epi.out = ctx->cull_values;
        epi.list = ctx->cull_list;
        const int lf = std::min(k.num_levels, kMaxLevels - 1);
        st = g_eval(ctx, net, src, (int64_t)c.cap, ctx->d_count, occ, cal, epi, k.precision,
                    k.margin, &gs->rechecked[lf], s);
        if (st != PIFU_OK) return st;
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
        CK(launch_cull_final(c, s));
        ctx->prof.k[PIFU_K_RENDER].launches += 3;
        if (k.rgb) {
            const int64_t npix = (int64_t)k.width * k.height;
            PointSrc hs{PTS_XYZ, ctx->hit_xyz, nullptr, 0, 0, nullptr};
            Epilogue he{};
            he.mode = EPI_PIXELS;
            he.act = ACT_TANH01;
            he.out = k.rgb;
            he.pix = ctx->hit_pix;
            const Map m0 = col.C > 0 ? col : occ;
            const Map m1 = col.C > 0 ? occ : Map{};
            st = run_mlp_tc(ctx, ctx->net[1], hs, npix, m0, m1, cal, he, s, ctx->d_count);
            if (st != PIFU_OK) return st;
        }
        CK(cudaMemcpyAsync(&gs->err, err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->h_gstats, gs, sizeof(GraphStats), cudaMemcpyDeviceToHost, s));
        return PIFU_OK;
    }
    // render: first-occupied depth per column, rays, colour at the hits
    RenderArgs a{};
    a.width = k.width;
    a.height = k.height;
    a.N = N;
    a.row_words = row_words_of(N);
    a.values = ctx->values;
    a.eval = ctx->eval;
    a.bin = ctx->bin[cur];
    for (int c = 0; c < 3; ++c) a.bg[c] = k.bg[c];
    a.depth = k.depth;
    a.rgb = k.rgb;
    a.mask = k.mask;
    a.hit_xyz = ctx->hit_xyz;
    a.hit_pix = ctx->hit_pix;
    a.hit_count = ctx->d_count;
    a.top = ctx->col_top;
    CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
    CK(launch_render_rays(a, s));
    ctx->prof.k[PIFU_K_RENDER].launches += 2;
    if (k.rgb) {
        const int64_t npix = (int64_t)k.width * k.height;
        PointSrc src{PTS_XYZ, ctx->hit_xyz, nullptr, 0, 0, nullptr};
        Epilogue epi{};
        epi.mode = EPI_PIXELS;
        epi.act = ACT_TANH01;
        epi.out = k.rgb;
        epi.pix = ctx->hit_pix;
        const Map m0 = col.C > 0 ? col : occ;
        const Map m1 = col.C > 0 ? occ : Map{};
        st = run_mlp_tc(ctx, ctx->net[1], src, npix, m0, m1, cal, epi, s, ctx->d_count);
        if (st != PIFU_OK) return st;
    }
    CK(cudaMemcpyAsync(&gs->err, err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ctx->h_gstats, gs, sizeof(GraphStats), cudaMemcpyDeviceToHost, s));
    return PIFU_OK;
}

void g_destroy(pifu_ctx* ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->g_valid = false;
}

int g_build(pifu_ctx* ctx, const FrameKey& k, const Map& occ, const Map& col, const Calib& cal) {
    g_destroy(ctx);
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (!ctx->cap_stream2) CK(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
    if (!ctx->cap_stream3) CK(cudaStreamCreateWithFlags(&ctx->cap_stream3, cudaStreamNonBlocking));
    if (!ctx->cap_stream4) CK(cudaStreamCreateWithFlags(&ctx->cap_stream4, cudaStreamNonBlocking));
    if (!ctx->d_gstats) CK(dev_alloc(&ctx->d_gstats, 1));
    {
        const int st = ensure_clist(ctx, kChunkTC);
        if (st != PIFU_OK) return st;
    }
    if (!ctx->h_gstats) CK(cudaHostAlloc(&ctx->h_gstats, sizeof(GraphStats), cudaHostAllocDefault));
    CK(tc_prepare());
    CK(chain_prepare());
    if (ctx->net[0].kind == kNetCbn) {
        const CbnF32& f = ctx->cbn.f32;
        CK(cbn_f32_prepare(f));
        if (ctx->cbn.tc_ok) CK(cbn_tc_prepare(f.C, f.K, f.nb));
    }
    {
        // device-sized batches: the workspaces must hold a whole capacity
        const int st = ensure_tc_rows(ctx, kChunkTC);
        if (st != PIFU_OK) return st;
    }
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;   // no timing events inside a graph
    const int64_t before = launches_now(ctx);
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int st = g_enqueue_frame(ctx, k, occ, col, cal);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->prof.on = prof_on;
    int64_t body = 0;
    for (int l = 1; l < k.num_levels; ++l) body += ctx->g_launches_body[l];
    ctx->g_launches_fixed = launches_now(ctx) - before - body;
    for (auto& x : ctx->prof.k) x.launches = 0;   // capture is not execution
    if (st != PIFU_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ee != cudaSuccess) return fail_cuda(ctx, ee);
    ctx->graph = g;
    const cudaError_t ie = cudaGraphInstantiate(&ctx->gexec, g, 0);
    if (ie != cudaSuccess) {
        g_destroy(ctx);
        return fail_cuda(ctx, ie);
    }
    ctx->gkey = k;
    ctx->g_valid = true;
    return PIFU_OK;
}

// ---- lockstep batch of frames (pifu_frames) -----------------------------------
//
// B independent frames advance through the levels together: a level's set-up,
// dilation and compaction run over all B frames' bitsets (grid.y = frame), and
// every evaluation batch is one device-sized list of keys frame * slot_nodes +
// node for all frames -- the work queue that one persistent tensor-core
// launch per layer drains.  The conflict loop of a level runs while any frame
// has a frontier.  Map pointers and calibrations are device arrays, written
// before each launch, so a captured graph serves every batch of the same
// shape.

void batch_free(pifu_ctx* ctx) {
    BatchWs& b = ctx->batch;
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
    b.g_valid = false;
    uint32_t** bits[] = {&b.cand, &b.tent, &b.bin[0], &b.bin[1], &b.eval, &b.conf};
    for (auto p : bits) dev_free(*p);
    dev_free(b.values);
    dev_free(b.list);
    dev_free(b.recheck);
    dev_free(b.squeue);
    dev_free(b.col_top);
    dev_free(b.hit_xyz);
    dev_free(b.hit_pix);
    b.B = b.N = 0;
    b.slot_words = b.slot_nodes = b.cap = b.npix = 0;
}

// Capacity of one device-sized batch for B frames: B x 2^18 keys rounded up
// to a power of two, between 2^20 and kTcRowsMax.
int64_t batch_cap(int B) {
    int64_t c = 1 << 20;
    while (c < (int64_t)B * (1 << 18) && c < kTcRowsMax) c *= 2;
    return c;
}

int batch_ensure(pifu_ctx* ctx, int B, int N, int64_t npix) {
    BatchWs& b = ctx->batch;
    if (!b.d_maps0) {
        CK(dev_alloc(&b.d_maps0, kMaxBatch));
        CK(dev_alloc(&b.d_maps1, kMaxBatch));
        CK(dev_alloc(&b.d_calibs, kMaxBatch));
        CK(cudaHostAlloc(&b.h_maps0, sizeof(Map) * kMaxBatch, cudaHostAllocDefault));
        CK(cudaHostAlloc(&b.h_maps1, sizeof(Map) * kMaxBatch, cudaHostAllocDefault));
        CK(cudaHostAlloc(&b.h_calibs, sizeof(Calib) * kMaxBatch, cudaHostAllocDefault));
        CK(dev_alloc(&b.d_stats, 1));
        CK(cudaHostAlloc(&b.h_stats, sizeof(BatchStats), cudaHostAllocDefault));
    }
    if (b.B >= B && b.N == N && b.npix >= npix) return PIFU_OK;
    const int Bn = std::max(B, b.B);
    const int64_t np = std::max(npix, b.npix);
    Map* keep[3] = {b.d_maps0, b.d_maps1, nullptr};
    (void)keep;
    batch_free(ctx);
    const int64_t words = words_of(N);
    const int64_t nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
    if ((int64_t)Bn * nodes > 2147483647LL) return PIFU_ERR_ARG;   // int32 keys
    uint32_t** bits[] = {&b.cand, &b.tent, &b.bin[0], &b.bin[1], &b.eval, &b.conf};
    for (auto p : bits) {
        CK(dev_alloc(p, words * Bn));
        CK(cudaMemset(*p, 0, (size_t)(words * Bn) * 4));
    }
    const int64_t cap = batch_cap(Bn);
    CK(dev_alloc(&b.values, nodes * Bn));
    CK(dev_alloc(&b.list, cap));
    CK(dev_alloc(&b.recheck, cap));
    CK(dev_alloc(&b.squeue, cap));
    CK(dev_alloc(&b.col_top, 2 * (int64_t)(N + 1) * (N + 1) * Bn));
    CK(dev_alloc(&b.hit_xyz, 3 * np * Bn));
    CK(dev_alloc(&b.hit_pix, np * Bn));
    b.B = Bn;
    b.N = N;
    b.npix = np;
    b.slot_words = words;
    b.slot_nodes = nodes;
    b.cap = cap;
    return PIFU_OK;
}

// The batch's frame pipeline, captured on ctx->cap_stream (loop bodies on
// cap_stream2).  g_eval's queues are pointed at the batch's for the capture.
int g_enqueue_batch(pifu_ctx* ctx, const BatchKey& k) {
    BatchWs& bw = ctx->batch;
    cudaStream_t s = ctx->cap_stream;
    cudaStream_t sb = ctx->cap_stream2;
    BatchStats* gs = bw.d_stats;
    unsigned int* err = ctx->d_count + 1;
    const DevNet& net = ctx->net[0];
    const int B = k.B;
    const int64_t cap = bw.cap;
    const int64_t fs = bw.slot_words, sn = bw.slot_nodes;
    int st = PIFU_OK;
    CK(cudaMemsetAsync(gs, 0, sizeof(BatchStats), s));
    CK(cudaMemsetAsync(err, 0, sizeof(unsigned int), s));
    int N = k.n0, cur = 0;
    CK(launch_dense_setup(N, bw.cand, bw.tent, bw.bin[cur], bw.eval, bw.conf, s, B, fs));
    const bool sur = k.use_surrogate != 0;
    {
        const int64_t nodes0 = (int64_t)(N + 1) * (N + 1) * (N + 1);
        PointSrc src{PTS_DENSE, nullptr, nullptr, 0, N, nullptr};
        src.maps0 = bw.d_maps0;
        src.calibs = bw.d_calibs;
        src.slot_div = nodes0;
        Epilogue epi{};
        epi.mode = EPI_LEVEL;
        epi.lv = LevelBits{bw.values, bw.tent, bw.bin[cur], bw.conf, N, row_words_of(N), 1,
                           nodes0, sn, fs};
        if (B * nodes0 > cap) return PIFU_ERR_CAPACITY;
        st = g_eval(ctx, net, src, B * nodes0, nullptr, Map{}, Calib{}, epi, k.precision, k.margin,
                    &gs->rechecked[0], s, sur && k.num_levels > 1, k.sur_margin,
                    &gs->fallback[0]);
        if (st != PIFU_OK) return st;
    }
    for (int l = 1; l < k.num_levels; ++l) {
        const int prev = cur;
        cur ^= 1;
        N *= 2;
        CK(launch_classify(bw.bin[prev], N, bw.cand, bw.tent, bw.bin[cur], bw.eval, bw.conf, s, B,
                           fs, fs));
        CK(launch_popcount(bw.cand, words_of(N), &gs->cands[l][0], s, B, fs));
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
        CK(launch_dilate_select(bw.cand, bw.eval, nullptr, N, bw.list, ctx->d_count, s, B, fs, sn));
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
        CK(launch_loop_control(h, ctx->d_count, (unsigned)cap, &gs->rounds[l], 0, k.max_rounds,
                               err, s));
        cudaGraph_t body = nullptr;
        st = g_add_while(ctx, s, h, &body);
        if (st != PIFU_OK) return st;
        const int64_t before = launches_now(ctx);
        CK(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        {
            const int rw = row_words_of(N);
            PointSrc src{PTS_LIST, nullptr, bw.list, 0, N, nullptr};
            src.maps0 = bw.d_maps0;
            src.calibs = bw.d_calibs;
            src.slot_div = sn;
            Epilogue epi{};
            epi.mode = EPI_LEVEL;
            epi.list = bw.list;
            epi.lv = LevelBits{bw.values, bw.tent, bw.bin[cur], bw.conf, N, rw, 0, sn, sn, fs};
            epi.lv.clist = ctx->clist;
            epi.lv.ccount = ctx->d_ccount;
            epi.lv.ccap = (unsigned)ctx->clist_cap;
            epi.lv.err = err;
            st = launch_accumulate(&gs->keys[l], ctx->d_count, (unsigned)cap, err, sb) == cudaSuccess
                     ? PIFU_OK : PIFU_ERR_CUDA;
            if (st == PIFU_OK &&
                cudaMemsetAsync(ctx->d_ccount, 0, sizeof(unsigned int), sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            if (st == PIFU_OK)
                st = g_eval(ctx, net, src, cap, ctx->d_count, Map{}, Calib{}, epi, k.precision,
                            k.margin, &gs->rechecked[l], sb, sur && l < k.num_levels - 1,
                            k.sur_margin, &gs->fallback[l]);
            if (st == PIFU_OK && cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            if (st == PIFU_OK &&
                launch_expand_conflicts(ctx->clist, ctx->d_ccount, (unsigned)cap, N, bw.eval, sn,
                                        fs, bw.list, ctx->d_count, (unsigned)cap, err,
                                        sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            if (st == PIFU_OK && launch_loop_control(h, ctx->d_count, (unsigned)cap,
                                                     &gs->rounds[l], 1, k.max_rounds, err,
                                                     sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
        }
        cudaGraph_t body_out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(sb, &body_out);
        if (st != PIFU_OK) return st;
        if (ee != cudaSuccess) return fail_cuda(ctx, ee);
        bw.launches_body[l] = launches_now(ctx) - before;
        CK(launch_popcount(bw.eval, words_of(N), &gs->evals[l][0], s, B, fs));
    }
    // render all frames, then the colour MLP over all their hits
    const int64_t npix = (int64_t)k.width * k.height;
    RenderArgs a{};
    a.width = k.width;
    a.height = k.height;
    a.N = N;
    a.row_words = row_words_of(N);
    a.values = bw.values;
    a.eval = bw.eval;
    a.bin = bw.bin[cur];
    for (int c = 0; c < 3; ++c) a.bg[c] = k.bg[c];
    a.depth = k.depth;
    a.rgb = k.rgb;
    a.mask = k.mask;
    a.hit_xyz = bw.hit_xyz;
    a.hit_pix = bw.hit_pix;
    a.hit_count = ctx->d_count;
    a.top = bw.col_top;
    a.slots = B;
    a.slot_nodes = sn;
    a.slot_words = fs;
    CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
    CK(launch_render_rays(a, s));
    ctx->prof.k[PIFU_K_RENDER].launches += 2;
    if (k.rgb) {
        PointSrc src{PTS_XYZ, bw.hit_xyz, nullptr, 0, 0, nullptr};
        const bool col = k.cC > 0;
        src.maps0 = col ? bw.d_maps1 : bw.d_maps0;   // colour maps first (Eq. 2)
        src.maps1 = col ? bw.d_maps0 : nullptr;
        src.calibs = bw.d_calibs;
        src.keys = bw.hit_pix;
        src.slot_div = npix;
        Epilogue epi{};
        epi.mode = EPI_PIXELS;
        epi.act = ACT_TANH01;
        epi.out = k.rgb;
        epi.pix = bw.hit_pix;
        if (B * npix > kTcRowsMax) return PIFU_ERR_CAPACITY;
        st = run_mlp_tc(ctx, ctx->net[1], src, B * npix, Map{}, Map{}, Calib{}, epi, s,
                        ctx->d_count);
        if (st != PIFU_OK) return st;
    }
    CK(cudaMemcpyAsync(&gs->err, err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(bw.h_stats, gs, sizeof(BatchStats), cudaMemcpyDeviceToHost, s));
    return PIFU_OK;
}

int b_build(pifu_ctx* ctx, const BatchKey& k) {
    BatchWs& bw = ctx->batch;
    if (bw.exec) cudaGraphExecDestroy(bw.exec);
    if (bw.graph) cudaGraphDestroy(bw.graph);
    bw.exec = nullptr;
    bw.graph = nullptr;
    bw.g_valid = false;
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (!ctx->cap_stream2) CK(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
    if (!ctx->cap_stream3) CK(cudaStreamCreateWithFlags(&ctx->cap_stream3, cudaStreamNonBlocking));
    if (!ctx->cap_stream4) CK(cudaStreamCreateWithFlags(&ctx->cap_stream4, cudaStreamNonBlocking));
    {
        const int st = ensure_clist(ctx, bw.cap);
        if (st != PIFU_OK) return st;
    }
    CK(tc_prepare());
    CK(chain_prepare());
    if (ctx->net[0].kind == kNetCbn) {
        const CbnF32& f = ctx->cbn.f32;
        CK(cbn_f32_prepare(f));
        if (ctx->cbn.tc_ok) CK(cbn_tc_prepare(f.C, f.K, f.nb));
    }
    {
        const int st = ensure_tc_rows(ctx, std::max<int64_t>(bw.cap, (int64_t)k.B * k.width * k.height));
        if (st != PIFU_OK) return st;
    }
    // g_eval's queues are the context's; point them at the batch's for the capture
    int* keep_recheck = ctx->recheck;
    int* keep_squeue = ctx->squeue;
    ctx->recheck = bw.recheck;
    ctx->squeue = bw.squeue;
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;
    const int64_t before = launches_now(ctx);
    int st = PIFU_OK;
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (ee == cudaSuccess) {
        st = g_enqueue_batch(ctx, k);
        ee = cudaStreamEndCapture(ctx->cap_stream, &g);
    }
    ctx->recheck = keep_recheck;
    ctx->squeue = keep_squeue;
    ctx->prof.on = prof_on;
    int64_t body = 0;
    for (int l = 1; l < k.num_levels; ++l) body += bw.launches_body[l];
    bw.launches_fixed = launches_now(ctx) - before - body;
    for (auto& x : ctx->prof.k) x.launches = 0;   // capture is not execution
    if (st != PIFU_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ee != cudaSuccess) return fail_cuda(ctx, ee);
    bw.graph = g;
    const cudaError_t ie = cudaGraphInstantiate(&bw.exec, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        bw.graph = nullptr;
        return fail_cuda(ctx, ie);
    }
    bw.key = k;
    bw.g_valid = true;
    return PIFU_OK;
}

// ---- tile autotuner --------------------------------------------------------------
//
// Picks, per tensor-core hidden layer, the output tile width BN (64, 128 or
// 256 columns of the 128-row tile) that runs fastest on a batch of `rows`
// points, by timing each candidate with CUDA events.  The last hidden layer
// keeps BN = its width when the last layer is fused into its epilogue.  The
// chosen tile changes the weight tensor map's box, so captured graphs are
// invalidated.

// Tile codes: 64, 128, 256 = BN of the single-CTA 128 x BN tile; kPairCode =
// the CTA-pair form (two CTAs on a 256 x 256 tile, BF16 layers only).
constexpr int kPairCode = 512;

bool encode_w(bool fp8, CUtensorMap* tmW, void* Wdev, int Kw, int n_out, int code) {
    const uint32_t box = (uint32_t)(code == kPairCode ? 128 : code);
    return fp8 ? tc_encode_2d_u8(tmW, Wdev, (uint64_t)Kw, (uint64_t)n_out, (uint64_t)Kw, 128, box)
               : tc_encode_2d_bf16(tmW, Wdev, (uint64_t)Kw, (uint64_t)n_out, (uint64_t)Kw * 2, 64,
                                   box);
}

int tune_layer(pifu_ctx* ctx, const TcLayerArgs& base, int n_out, bool fp8, bool allow_pair,
               CUtensorMap* tmW, void* Wdev, int Kw, int* code, cudaStream_t s, double* best_ms) {
    const int cands[4] = {64, 128, 256, kPairCode};
    int best = *code;
    double best_t = 1e30;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int st = PIFU_OK;
    for (int c : cands) {
        const bool pair = c == kPairCode;
        if (st != PIFU_OK || (pair ? !allow_pair || n_out % 256 != 0 : n_out % c != 0)) continue;
        if (!encode_w(fp8, tmW, Wdev, Kw, n_out, c)) {
            st = PIFU_ERR_CUDA;
            break;
        }
        TcLayerArgs a = base;
        a.BN = pair ? 256 : c;
        a.pair = pair ? 1 : 0;
        a.tmW = tmW;
        float ms = 0.f;
        cudaError_t e = launch_tc_linear(a, s);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_tc_linear(a, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = fail_cuda(ctx, e);
            break;
        }
        if (ms < best_t) {
            best_t = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PIFU_OK) return st;
    *best_ms = best_t / 3.0;
    *code = best;
    return encode_w(fp8, tmW, Wdev, Kw, n_out, best) ? PIFU_OK : PIFU_ERR_CUDA;
}

int autotune(pifu_ctx* ctx, int64_t rows, cudaStream_t s, int32_t* bn_out, double* ms_out,
             int n_max, int* n_done) {
    int st = ensure_tc_rows(ctx, rows);
    if (st != PIFU_OK) return st;
    CK(tc_prepare());
    CK(chain_prepare());
    int n = 0;
    auto record = [&](int bn, double ms) {
        if (n < n_max) {
            if (bn_out) bn_out[n] = bn;
            if (ms_out) ms_out[n] = ms;
        }
        ++n;
    };
    for (int which = 0; which < 2; ++which) {
        DevNet& net = ctx->net[which];
        if (!net.tc_ok) continue;
        const int L = (int)net.layers.size();
        for (int l = 0; l + 1 < L; ++l) {
            const DevLayer& Ly = net.layers[(size_t)l];
            const bool fused_last = l == L - 2 && net.layers[(size_t)L - 1].K2 == 0 &&
                                    net.layers[(size_t)L - 1].n_out <= 4;
            TcLayerArgs a{};
            a.M = (int)rows;
            a.N = Ly.n_out;
            a.bias = Ly.b;
            a.slope = net.slope;
            a.out = ctx->Hb[l % 2];
            a.ldo = Ly.n_out;
            a.err = ctx->d_count + 1;
            a.mode = TC_BF16;
            const bool f8 = net.f8_ok && l < (int)net.f8.size();
            if (f8) {
                Fp8Layer& Q = net.f8[(size_t)l];
                a.tmA1 = l > 0 ? &Q.tmA1 : &net.tmX8;
                a.tmA2 = &net.tmX8;
                a.nk1 = Q.nk1;
                a.nk2 = Q.nk2;
                a.mode = l + 1 < (int)net.f8.size() ? TC_E4M3_E4M3 : TC_E4M3_BF16;
                a.colscale = Q.colscale;
                a.out_scale = Q.out_scale;
                double ms = 0.0;
                st = tune_layer(ctx, a, Ly.n_out, true, false, &Q.tmW, Q.W, Q.Kw, &Q.BN, s, &ms);
                if (st != PIFU_OK) return st;
                record(Q.BN, ms);
            }
            TcLayer& T = net.tc[(size_t)l];
            if (fused_last) {
                record(T.BN, 0.0);   // kept: the fused last layer needs BN = n_out
                continue;
            }
            a.tmA1 = l > 0 ? &T.tmA1 : &net.tmX;
            a.tmA2 = &net.tmX;
            a.nk1 = T.nk1;
            a.nk2 = T.nk2;
            a.mode = TC_BF16;
            a.colscale = nullptr;
            a.out_scale = 1.f;
            double ms = 0.0;
            int code = T.pair ? kPairCode : T.BN;
            st = tune_layer(ctx, a, Ly.n_out, false, true, &T.tmW, T.W, T.Kw, &code, s, &ms);
            if (st != PIFU_OK) return st;
            T.pair = code == kPairCode;
            T.BN = T.pair ? 256 : code;
            record(code, ms);
        }
    }
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    if (n_done) *n_done = n;
    return PIFU_OK;
}

// The tuned layers in pifu_autotune's order; visit(q, t, n_out, fused_last)
// gets the E4M3 form (q != nullptr) or the BF16 form (t != nullptr).
template <typename F>
void for_each_tuned_layer(pifu_ctx* ctx, F&& visit) {
    for (int which = 0; which < 2; ++which) {
        DevNet& net = ctx->net[which];
        if (!net.tc_ok) continue;
        const int L = (int)net.layers.size();
        for (int l = 0; l + 1 < L; ++l) {
            const int n_out = net.layers[(size_t)l].n_out;
            const bool fused_last = l == L - 2 && net.layers[(size_t)L - 1].K2 == 0 &&
                                    net.layers[(size_t)L - 1].n_out <= 4;
            if (net.f8_ok && l < (int)net.f8.size())
                visit(&net.f8[(size_t)l], (TcLayer*)nullptr, n_out, false);
            visit((Fp8Layer*)nullptr, &net.tc[(size_t)l], n_out, fused_last);
        }
    }
}

int set_tiles(pifu_ctx* ctx, const int32_t* codes, int n) {
    // validate everything first, so that a refused call changes nothing
    int i = 0;
    bool valid = true;
    for_each_tuned_layer(ctx, [&](Fp8Layer* q, TcLayer* t, int n_out, bool fused_last) {
        if (i >= n) {
            valid = false;
            ++i;
            return;
        }
        const int c = codes[i++];
        if (q)
            valid = valid && (c == 64 || c == 128 || c == 256) && n_out % c == 0;
        else if (fused_last)
            valid = valid && c == (t->pair ? kPairCode : t->BN);
        else if (c == kPairCode)
            valid = valid && n_out % 256 == 0;
        else
            valid = valid && (c == 64 || c == 128 || c == 256) && n_out % c == 0;
    });
    if (!valid || i != n) return PIFU_ERR_ARG;
    i = 0;
    bool ok = true;
    for_each_tuned_layer(ctx, [&](Fp8Layer* q, TcLayer* t, int n_out, bool) {
        const int c = codes[i++];
        if (q) {
            q->BN = c;
            ok = ok && encode_w(true, &q->tmW, q->W, q->Kw, n_out, c);
        } else {
            t->pair = c == kPairCode;
            t->BN = t->pair ? 256 : c;
            ok = ok && encode_w(false, &t->tmW, t->W, t->Kw, n_out, c);
        }
    });
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    return ok ? PIFU_OK : PIFU_ERR_CUDA;
}

}  // namespace

// ============================================================================
extern "C" {

const char* pifu_status_string(int status) {
    switch (status) {
        case PIFU_OK: return "ok";
        case PIFU_ERR_ARG: return "invalid argument";
        case PIFU_ERR_FORMAT: return "malformed weight blob";
        case PIFU_ERR_CUDA: return "CUDA error";
        case PIFU_ERR_OOM: return "out of device memory";
        case PIFU_ERR_NOT_CONVERGED: return "conflict loop did not converge within max_rounds";
        case PIFU_ERR_TIMEOUT: return "bounded device wait timed out";
        case PIFU_ERR_STATE: return "call order violated";
        case PIFU_ERR_UNSUPPORTED: return "unsupported configuration";
        case PIFU_ERR_CAPACITY: return "a device-side count exceeded a fixed capacity of the graph form";
        default: return "unknown status";
    }
}

const char* pifu_last_error(const pifu_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : "";
}

int pifu_create(const void* weight_blob, size_t bytes, pifu_ctx** out) {
    if (!out) return PIFU_ERR_ARG;
    *out = nullptr;
    if (!weight_blob) return PIFU_ERR_ARG;
    // Parse and validate the whole blob on the host before touching CUDA.
    Reader rd{static_cast<const uint8_t*>(weight_blob), bytes};
    char magic[4];
    uint32_t version, n_nets;
    if (!rd.get(magic, 4) || std::memcmp(magic, "PIFU", 4) != 0) return PIFU_ERR_FORMAT;
    if (!rd.u32(version) || version != 1 || !rd.u32(n_nets) || n_nets != 2) return PIFU_ERR_FORMAT;
    HostNet hn[2];
    HostCbn hc;
    uint32_t kind0 = 0;
    if (rd.off + 4 <= rd.n) std::memcpy(&kind0, rd.p + rd.off, 4);
    const bool cbn = kind0 == (uint32_t)kNetCbn;
    int st = cbn ? parse_cbn(rd, hc) : parse_net(rd, hn[0], 0);
    if (st == PIFU_OK) st = parse_net(rd, hn[1], 1);
    if (st == PIFU_OK && rd.off != rd.n) st = PIFU_ERR_FORMAT;
    if (st != PIFU_OK) return st;
    pifu_ctx* ctx = new pifu_ctx();
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return PIFU_ERR_CUDA;
    }
    st = cbn ? upload_cbn(ctx, hc) : upload_net(ctx, hn[0], ctx->net[0]);
    if (st == PIFU_OK) st = upload_net(ctx, hn[1], ctx->net[1]);
    if (st == PIFU_OK) st = ensure_mlp_ws(ctx);
    if (st == PIFU_OK && !cbn) st = build_tc(ctx, hn[0], ctx->net[0]);
    if (st == PIFU_OK) st = build_tc(ctx, hn[1], ctx->net[1]);
    if (st == PIFU_OK) {
        cudaError_t e = cudaMalloc(&ctx->d_count, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(ctx->d_count, 0, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_pop, kMaxLevels * sizeof(unsigned long long));
        if (e == cudaSuccess)
            e = cudaHostAlloc(&ctx->h_count, 2 * sizeof(unsigned int), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_recheck, sizeof(unsigned int));
        if (e == cudaSuccess)
            e = cudaHostAlloc(&ctx->h_recheck, sizeof(unsigned int), cudaHostAllocDefault);
        if (e == cudaSuccess) e = dev_alloc(&ctx->recheck, kChunk);
        if (e == cudaSuccess) e = dev_alloc(&ctx->squeue, kChunk);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_squeue, sizeof(unsigned int));
        if (e == cudaSuccess)
            e = cudaHostAlloc(&ctx->h_squeue, sizeof(unsigned int), cudaHostAllocDefault);
        if (e == cudaSuccess) ctx->recheck_cap = kChunk;
        if (e == cudaSuccess)
            e = cudaHostAlloc(&ctx->h_pop, kMaxLevels * sizeof(unsigned long long), cudaHostAllocDefault);
        if (e != cudaSuccess) st = fail_cuda(ctx, e);
    }
    if (st != PIFU_OK) {
        pifu_destroy(ctx);
        return st;
    }
    *out = ctx;
    return PIFU_OK;
}

void pifu_destroy(pifu_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    batch_free(ctx);
    {
        BatchWs& bw = ctx->batch;
        dev_free(bw.d_maps0);
        dev_free(bw.d_maps1);
        dev_free(bw.d_calibs);
        dev_free(bw.d_stats);
        if (bw.h_maps0) cudaFreeHost(bw.h_maps0);
        if (bw.h_maps1) cudaFreeHost(bw.h_maps1);
        if (bw.h_calibs) cudaFreeHost(bw.h_calibs);
        if (bw.h_stats) cudaFreeHost(bw.h_stats);
    }
    free_net(ctx->net[0]);
    free_cbn(ctx->cbn);
    free_net(ctx->net[1]);
    dev_free(ctx->X);
    dev_free(ctx->HA);
    dev_free(ctx->HB);
    dev_free(ctx->Xb);
    dev_free(ctx->Hb[0]);
    dev_free(ctx->Hb[1]);
    dev_free(ctx->X8);
    dev_free(ctx->chain_dep);
    dev_free(ctx->part);
    uint32_t** bitsets[] = {&ctx->cand, &ctx->tent, &ctx->bin[0], &ctx->bin[1],
                            &ctx->eval, &ctx->conf[0], &ctx->conf[1]};
    for (auto b : bitsets) dev_free(*b);
    dev_free(ctx->values);
    dev_free(ctx->prev_values);
    dev_free(ctx->list);
    dev_free(ctx->recheck);
    dev_free(ctx->d_recheck);
    if (ctx->h_recheck) cudaFreeHost(ctx->h_recheck);
    dev_free(ctx->d_count);
    dev_free(ctx->d_pop);
    dev_free(ctx->hit_xyz);
    dev_free(ctx->hit_pix);
    dev_free(ctx->col_top);
    g_destroy(ctx);
    sur_free(ctx);
    dev_free(ctx->squeue);
    dev_free(ctx->d_squeue);
    if (ctx->h_squeue) cudaFreeHost(ctx->h_squeue);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
    if (ctx->cap_stream3) cudaStreamDestroy(ctx->cap_stream3);
    if (ctx->cap_stream4) cudaStreamDestroy(ctx->cap_stream4);
    dev_free(ctx->clist);
    dev_free(ctx->d_ccount);
    dev_free(ctx->d_gstats);
    if (ctx->h_gstats) cudaFreeHost(ctx->h_gstats);
    if (ctx->h_count) cudaFreeHost(ctx->h_count);
    if (ctx->h_pop) cudaFreeHost(ctx->h_pop);
    delete ctx;
}

int pifu_query(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
               const float* pts_dev, int64_t m, float* occ_dev, void* stream) {
    return pifu_query_ex(ctx, occ_map, calib, pts_dev, m, occ_dev, PIFU_PREC_FP32, 0.f, stream);
}

int pifu_query_ex(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                  const float* pts_dev, int64_t m, float* occ_dev, int precision, float margin,
                  void* stream) {
    if (!ctx || !calib || m < 0) return PIFU_ERR_ARG;
    if (!prec_valid(precision)) return PIFU_ERR_UNSUPPORTED;
    if (ctx->net[0].kind == kNetCbn && prec_f8(precision)) return PIFU_ERR_UNSUPPORTED;
    if (prec_mixed(precision) && !(margin >= 0.f && margin <= 0.5f)) return PIFU_ERR_ARG;
    if (m == 0) return PIFU_OK;
    if (!pts_dev || !occ_dev || !map_ok(occ_map)) return PIFU_ERR_ARG;
    if (ctx->net[0].d_in != occ_map->C + 1) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PointSrc src{PTS_XYZ, pts_dev, nullptr, 0, 0};
    Epilogue epi{};
    epi.mode = EPI_STORE;
    epi.act = ACT_SIGMOID;
    epi.out = occ_dev;
    if (precision != PIFU_PREC_FP32 && !ctx->net[0].tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (prec_f8(precision) && !ctx->net[0].f8_ok) return PIFU_ERR_STATE;
    if (!prec_mixed(precision))
        return run_mlp(ctx, ctx->net[0], src, m, to_map(occ_map), Map{}, to_calib(calib), epi, s,
                       precision);
    // mixed: batches of at most one workspace chunk, each BF16 then FP32 for
    // the occupancies near 0.5 (synchronises the stream once per batch)
    for (int64_t p0 = 0; p0 < m; p0 += kChunk) {
        const int64_t mc = std::min<int64_t>(kChunk, m - p0);
        PointSrc sb{PTS_XYZ, pts_dev + 3 * p0, nullptr, 0, 0};
        Epilogue eb = epi;
        eb.out = occ_dev + p0;
        const int st = run_mlp_mixed(ctx, ctx->net[0], sb, mc, to_map(occ_map), Map{},
                                     to_calib(calib), eb, margin, s, nullptr,
                                     precision == PIFU_PREC_FP8_MIXED);
        if (st != PIFU_OK) return st;
    }
    return PIFU_OK;
}

int pifu_query_colour(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
                      const float calib[12], const float* pts_dev, int64_t m, float* rgb_dev,
                      void* stream) {
    if (!ctx || !calib || m < 0) return PIFU_ERR_ARG;
    if (m == 0) return PIFU_OK;
    if (!pts_dev || !rgb_dev || !map_ok(occ_map) || (col_map && !map_ok(col_map))) return PIFU_ERR_ARG;
    const int c_t = col_map ? col_map->C : 0;
    if (ctx->net[1].d_in != c_t + occ_map->C + 1) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PointSrc src{PTS_XYZ, pts_dev, nullptr, 0, 0};
    Epilogue epi{};
    epi.mode = EPI_STORE;
    epi.act = ACT_TANH01;
    epi.out = rgb_dev;
    const Map m0 = col_map ? to_map(col_map) : to_map(occ_map);
    const Map m1 = col_map ? to_map(occ_map) : Map{};
    return run_mlp(ctx, ctx->net[1], src, m, m0, m1, to_calib(calib), epi, s);
}

int pifu_localize(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                  const pifu_levels* lv, void* stream, pifu_volume* out) {
    if (!ctx || !calib || !lv || !map_ok(occ_map)) return PIFU_ERR_ARG;
    if (!is_pow2(lv->n0) || lv->n0 < 2 || lv->num_levels < 1 || lv->num_levels > kMaxLevels)
        return PIFU_ERR_ARG;
    const int64_t n_fine = (int64_t)lv->n0 << (lv->num_levels - 1);
    if (n_fine > kMaxFine) return PIFU_ERR_ARG;
    if (!prec_valid(lv->precision)) return PIFU_ERR_UNSUPPORTED;
    if (lv->precision != PIFU_PREC_FP32 && !ctx->net[0].tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (prec_f8(lv->precision) && !ctx->net[0].f8_ok) return PIFU_ERR_STATE;
    if (prec_mixed(lv->precision) && !(lv->margin >= 0.f && lv->margin <= 0.5f))
        return PIFU_ERR_ARG;
    const int prec = lv->precision;
    const bool use_sur = lv->use_surrogate != 0;
    if (use_sur && (!ctx->sur.ready || !(lv->surrogate_margin >= 0.f && lv->surrogate_margin <= 0.5f)))
        return use_sur && !ctx->sur.ready ? PIFU_ERR_STATE : PIFU_ERR_ARG;
    if (ctx->net[0].d_in != occ_map->C + 1) return PIFU_ERR_ARG;
    const int subdiv = lv->subdivision;
    if (subdiv < PIFU_SUBDIV_METHOD || subdiv > PIFU_SUBDIV_THRESHOLD) return PIFU_ERR_ARG;
    if (subdiv == PIFU_SUBDIV_THRESHOLD && !(lv->threshold >= 0.f && lv->threshold <= 1.f))
        return PIFU_ERR_ARG;
    if (subdiv != PIFU_SUBDIV_METHOD && use_sur) return PIFU_ERR_UNSUPPORTED;
    if (ctx->net[0].kind == kNetCbn && (use_sur || prec_f8(prec))) return PIFU_ERR_UNSUPPORTED;
    const int max_rounds = lv->max_rounds > 0 ? lv->max_rounds : 4096;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ctx->have_volume = false;
    int st = ensure_level_ws(ctx, (int)n_fine);
    if (st != PIFU_OK) return st;

    pifu_volume vs{};
    vs.num_levels = lv->num_levels;
    const Map map = to_map(occ_map);
    const Calib cal = to_calib(calib);
    CK(cudaMemsetAsync(ctx->d_pop, 0, kMaxLevels * sizeof(unsigned long long), s));

    // level 0: dense evaluation of every node
    int N = lv->n0;
    int cur = 0;
    {
        cudaEvent_t ev = ctx->prof.begin(s);
        CK(launch_dense_setup(N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval, ctx->conf[0], s));
        ctx->prof.end(PIFU_K_LEVEL, ev, s, 0.0, 5.0 * 4.0 * words_of(N));
    }
    {
        const int64_t nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
        PointSrc src{PTS_DENSE, nullptr, nullptr, 0, N};
        Epilogue epi{};
        epi.mode = EPI_LEVEL;
        epi.list = nullptr;
        epi.base = 0;
        epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[0], N, row_words_of(N), 1};
        st = eval_level_batch(ctx, src, nodes, map, cal, epi, prec, lv->margin,
                              use_sur && lv->num_levels > 1, lv->surrogate_margin, s,
                              &vs.rechecked_per_level[0], &vs.fallback_per_level[0]);
        if (st != PIFU_OK) return st;
        vs.evals_per_level[0] = nodes;
        vs.n_eval = nodes;
    }
    // finer levels
    for (int l = 1; l < lv->num_levels; ++l) {
        const int prev = cur;
        cur ^= 1;
        N *= 2;
        const int rw = row_words_of(N);
        const double wbytes = 4.0 * words_of(N);
        cudaEvent_t ev;
        if (subdiv == PIFU_SUBDIV_THRESHOLD) {
            // the coarser level's continuous values, read while this level's
            // are written
            const int64_t nc = (int64_t)(N / 2 + 1) * (N / 2 + 1) * (N / 2 + 1);
            st = ensure_prev_values(ctx, nc);
            if (st != PIFU_OK) return st;
            CK(cudaMemcpyAsync(ctx->prev_values, ctx->values, (size_t)nc * 4,
                               cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
            ev = ctx->prof.begin(s);
            CK(launch_threshold_select(ctx->prev_values, N, lv->threshold, ctx->values, ctx->tent,
                                       ctx->bin[cur], ctx->eval, ctx->conf[0], ctx->list,
                                       ctx->d_count, s));
            ctx->prof.end(PIFU_K_SELECT, ev, s, 0.0,
                          4.0 * nc + 4.0 * (double)(N + 1) * (N + 1) * (N + 1) + 4.0 * wbytes);
            CK(launch_popcount(ctx->eval, words_of(N), ctx->d_pop + l, s));
        } else {
            ev = ctx->prof.begin(s);
            CK(launch_classify(ctx->bin[prev], N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval,
                               ctx->conf[0], s));
            ctx->prof.end(PIFU_K_LEVEL, ev, s, 0.0, 4.0 * words_of(N / 2) + 5.0 * wbytes);
            ev = ctx->prof.begin(s);
            CK(launch_popcount(ctx->cand, words_of(N), ctx->d_pop + l, s));
            ctx->prof.end(PIFU_K_LEVEL, ev, s, 0.0, wbytes);
            CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
            ev = ctx->prof.begin(s);
            if (subdiv == PIFU_SUBDIV_BINARIZED)   // the candidates alone
                CK(launch_select(ctx->cand, ctx->eval, N, ctx->list, ctx->d_count, s));
            else                                   // boundary candidates and their 1-ring
                CK(launch_dilate_select(ctx->cand, ctx->eval, ctx->conf[1], N, ctx->list,
                                        ctx->d_count, s));
            ctx->prof.end(PIFU_K_SELECT, ev, s, 0.0, 4.0 * wbytes);
        }
        unsigned int n = 0;
        st = read_count(ctx, s, &n);
        if (st != PIFU_OK) return st;
        ctx->prof.k[PIFU_K_SELECT].bytes += 4.0 * n;   // the list it wrote
        if (subdiv != PIFU_SUBDIV_METHOD) {
            // octree baselines: one pass, no conflict rounds
            if (n > 0) {
                PointSrc src{PTS_LIST, nullptr, ctx->list, 0, N};
                Epilogue epi{};
                epi.mode = EPI_LEVEL;
                epi.list = ctx->list;
                epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[0], N, rw, 0};
                st = eval_level_batch(ctx, src, n, map, cal, epi, prec, lv->margin, false, 0.f, s,
                                      &vs.rechecked_per_level[l], &vs.fallback_per_level[l]);
                if (st != PIFU_OK) return st;
            }
            vs.evals_per_level[l] = n;
            vs.n_eval += n;
            continue;
        }
        int64_t level_evals = 0;
        int q = 0;     // conflicts of the next evaluation go to conf[q]
        int rounds = 0;
        PointSrc src{PTS_LIST, nullptr, ctx->list, 0, N};
        Epilogue epi{};
        epi.mode = EPI_LEVEL;
        epi.list = ctx->list;
        while (n > 0) {
            epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[q], N, rw, 0};
            st = eval_level_batch(ctx, src, n, map, cal, epi, prec, lv->margin,
                                  use_sur && l < lv->num_levels - 1, lv->surrogate_margin, s,
                                  &vs.rechecked_per_level[l], &vs.fallback_per_level[l]);
            if (st != PIFU_OK) return st;
            level_evals += n;
            // unevaluated 1-ring of this evaluation's conflicts
            CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
            ev = ctx->prof.begin(s);
            CK(launch_dilate_select(ctx->conf[q], ctx->eval, ctx->conf[1 - q], N, ctx->list,
                                    ctx->d_count, s));
            ctx->prof.end(PIFU_K_SELECT, ev, s, 0.0, 4.0 * wbytes);
            st = read_count(ctx, s, &n);
            if (st != PIFU_OK) return st;
            ctx->prof.k[PIFU_K_SELECT].bytes += 4.0 * n;
            if (n > 0) {
                if (rounds >= max_rounds) return PIFU_ERR_NOT_CONVERGED;
                ++rounds;
            }
            q = 1 - q;
        }
        vs.evals_per_level[l] = level_evals;
        vs.conflict_rounds[l] = rounds;
        vs.n_eval += level_evals;
    }
    CK(cudaMemcpyAsync(ctx->h_pop, ctx->d_pop, kMaxLevels * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    {
        unsigned int dummy;
        st = read_count(ctx, s, &dummy);   // synchronises and checks the error word
        if (st != PIFU_OK) return st;
    }
    for (int l = 1; l < lv->num_levels; ++l) vs.candidates_per_level[l] = (int64_t)ctx->h_pop[l];
    vs.n = N;
    vs.row_words = row_words_of(N);
    vs.occ_bits_dev = ctx->bin[cur];
    vs.eval_bits_dev = ctx->eval;
    vs.values_dev = ctx->values;
    ctx->stats = vs;
    ctx->have_volume = true;
    ctx->vol_N = N;
    ctx->vol_bin = cur;
    ctx->vol_prec = prec;
    ctx->vol_margin = lv->margin;
    if (out) *out = vs;
    return PIFU_OK;
}

int pifu_render(pifu_ctx* ctx, const pifu_camera* cam, const pifu_fmap* occ_map,
                const pifu_fmap* col_map, const float calib[12], void* stream, float* depth_dev,
                float* rgb_dev, uint8_t* mask_dev) {
    if (!ctx || !cam || !calib) return PIFU_ERR_ARG;
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return PIFU_ERR_ARG;
    if (!ctx->have_volume) return PIFU_ERR_STATE;
    if (cam->precision != PIFU_PREC_FP32 && cam->precision != PIFU_PREC_BF16)
        return PIFU_ERR_UNSUPPORTED;
    if (rgb_dev && cam->precision == PIFU_PREC_BF16 && !ctx->net[1].tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (rgb_dev) {
        if (!map_ok(occ_map) || (col_map && !map_ok(col_map))) return PIFU_ERR_ARG;
        const int c_t = col_map ? col_map->C : 0;
        if (ctx->net[1].d_in != c_t + occ_map->C + 1) return PIFU_ERR_ARG;
    }
    if (cam->final_level != 0 &&
        (cam->final_level != 1 || cam->width != cam->height || !is_pow2(cam->width) ||
         !map_ok(occ_map) || ctx->net[0].d_in != occ_map->C + 1))
        return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npix = (int64_t)cam->width * cam->height;
    int st = ensure_hit_ws(ctx, npix);
    if (st != PIFU_OK) return st;
    unsigned int n = 0;
    if (cam->final_level) {
        // view-culled final level (Sec. 3.2) at 2 N depth nodes of the pixel columns
        const int Nc = ctx->vol_N;
        st = ensure_cull_ws(ctx, npix, Nc);
        if (st != PIFU_OK) return st;
        CullArgs c{};
        c.width = cam->width;
        c.height = cam->height;
        c.Nc = Nc;
        c.row_words = row_words_of(Nc);
        c.bin = ctx->bin[ctx->vol_bin];
        c.list = ctx->cull_list;
        c.count = ctx->d_count;
        c.cap = (unsigned)ctx->cull_cap;
        c.err = ctx->d_count + 1;
        c.values = ctx->cull_values;
        for (int q = 0; q < 3; ++q) c.bg[q] = cam->background[q];
        c.depth = depth_dev;
        c.rgb = rgb_dev;
        c.mask = mask_dev;
        c.hit_xyz = ctx->hit_xyz;
        c.hit_pix = ctx->hit_pix;
        c.hit_count = ctx->d_count;
        c.top = ctx->col_top;
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
        cudaEvent_t ev = ctx->prof.begin(s);
        CK(launch_cull_select(c, s));
        ctx->prof.end(PIFU_K_SELECT, ev, s, 0.0, 4.0 * words_of(Nc) + 4.0 * npix);
        unsigned int nc = 0;
        st = read_count(ctx, s, &nc);
        if (st != PIFU_OK) return st;
        if (nc > 0) {
            PointSrc src{PTS_COLUMN, nullptr, ctx->cull_list, 0, 2 * Nc, nullptr};
            src.width = cam->width;
            Epilogue epi{};
            epi.mode = EPI_COLUMN;
            epi.out = ctx->cull_values;
            epi.list = ctx->cull_list;
            st = eval_batch(ctx, src, nc, to_map(occ_map), to_calib(calib), epi, ctx->vol_prec,
                            ctx->vol_margin, s);
            if (st != PIFU_OK) return st;
        }
        if (ctx->stats.num_levels < kMaxLevels)
            ctx->stats.evals_per_level[ctx->stats.num_levels] = nc;
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
        ev = ctx->prof.begin(s);
        CK(launch_cull_final(c, s));
        ctx->prof.end(PIFU_K_RENDER, ev, s, 0.0, 4.0 * words_of(Nc) + 4.0 * nc + 17.0 * npix);
        st = read_count(ctx, s, &n);
        if (st != PIFU_OK) return st;
        ctx->prof.k[PIFU_K_RENDER].bytes += 16.0 * n;   // the hit list
        if (!rgb_dev || n == 0) return PIFU_OK;
        PointSrc hs{PTS_XYZ, ctx->hit_xyz, nullptr, 0, 0};
        Epilogue he{};
        he.mode = EPI_PIXELS;
        he.act = ACT_TANH01;
        he.out = rgb_dev;
        he.pix = ctx->hit_pix;
        const Map m0 = col_map ? to_map(col_map) : to_map(occ_map);
        const Map m1 = col_map ? to_map(occ_map) : Map{};
        return run_mlp(ctx, ctx->net[1], hs, n, m0, m1, to_calib(calib), he, s, cam->precision);
    }
    RenderArgs a{};
    a.width = cam->width;
    a.height = cam->height;
    a.N = ctx->vol_N;
    a.row_words = row_words_of(ctx->vol_N);
    a.values = ctx->values;
    a.eval = ctx->eval;
    a.bin = ctx->bin[ctx->vol_bin];
    for (int c = 0; c < 3; ++c) a.bg[c] = cam->background[c];
    a.depth = depth_dev;
    a.rgb = rgb_dev;
    a.mask = mask_dev;
    a.hit_xyz = ctx->hit_xyz;
    a.hit_pix = ctx->hit_pix;
    a.hit_count = ctx->d_count;
    a.top = ctx->col_top;
    CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
    cudaEvent_t ev = ctx->prof.begin(s);
    CK(launch_render_rays(a, s));
    {
        // the volume once (two bitsets + the evaluated values) and the outputs
        const double vol_bytes = 2.0 * 4.0 * words_of(ctx->vol_N) +
                                 4.0 * (double)ctx->stats.evals_per_level[ctx->stats.num_levels - 1];
        const double out_bytes =
            (double)npix * ((depth_dev ? 4 : 0) + (rgb_dev ? 12 : 0) + (mask_dev ? 1 : 0));
        ctx->prof.end(PIFU_K_RENDER, ev, s, 0.0, vol_bytes + out_bytes);
    }
    st = read_count(ctx, s, &n);
    if (st != PIFU_OK) return st;
    ctx->prof.k[PIFU_K_RENDER].bytes += 16.0 * n;   // the hit list
    if (!rgb_dev) return PIFU_OK;
    if (n == 0) return PIFU_OK;
    PointSrc src{PTS_XYZ, ctx->hit_xyz, nullptr, 0, 0};
    Epilogue epi{};
    epi.mode = EPI_PIXELS;
    epi.act = ACT_TANH01;
    epi.out = rgb_dev;
    epi.pix = ctx->hit_pix;
    const Map m0 = col_map ? to_map(col_map) : to_map(occ_map);
    const Map m1 = col_map ? to_map(occ_map) : Map{};
    return run_mlp(ctx, ctx->net[1], src, n, m0, m1, to_calib(calib), epi, s, cam->precision);
}

int pifu_frame(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
               const float calib[12], const pifu_levels* lv, const pifu_camera* cam, void* stream,
               float* depth_dev, float* rgb_dev, uint8_t* mask_dev, pifu_volume* out) {
    if (!ctx || !calib || !lv || !cam || !map_ok(occ_map) || (col_map && !map_ok(col_map)))
        return PIFU_ERR_ARG;
    if (!is_pow2(lv->n0) || lv->n0 < 2 || lv->num_levels < 1 || lv->num_levels > kMaxLevels)
        return PIFU_ERR_ARG;
    const int64_t n_fine = (int64_t)lv->n0 << (lv->num_levels - 1);
    if (n_fine > kMaxFine) return PIFU_ERR_ARG;
    if (cam->width < 1 || cam->height < 1) return PIFU_ERR_ARG;
    if ((int64_t)cam->width * cam->height > kChunkTC) return PIFU_ERR_CAPACITY;
    if (cam->final_level != 0 &&
        (cam->final_level != 1 || cam->width != cam->height || !is_pow2(cam->width)))
        return PIFU_ERR_ARG;
    if (!prec_valid(lv->precision) || lv->precision == PIFU_PREC_FP32) return PIFU_ERR_UNSUPPORTED;
    if (lv->subdivision != PIFU_SUBDIV_METHOD) return PIFU_ERR_UNSUPPORTED;
    if (ctx->net[0].kind == kNetCbn && (prec_f8(lv->precision) || lv->use_surrogate))
        return PIFU_ERR_UNSUPPORTED;
    if (prec_f8(lv->precision) && !ctx->net[0].f8_ok) return PIFU_ERR_STATE;
    if (prec_mixed(lv->precision) && !(lv->margin >= 0.f && lv->margin <= 0.5f))
        return PIFU_ERR_ARG;
    if (lv->use_surrogate) {
        if (!ctx->sur.ready || !ctx->snet.tc_ok) return PIFU_ERR_STATE;
        if (!(lv->surrogate_margin >= 0.f && lv->surrogate_margin <= 0.5f)) return PIFU_ERR_ARG;
    }
    if (ctx->net[0].d_in != occ_map->C + 1) return PIFU_ERR_ARG;
    if (!ctx->net[0].tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (rgb_dev) {
        const int c_t = col_map ? col_map->C : 0;
        if (ctx->net[1].d_in != c_t + occ_map->C + 1) return PIFU_ERR_ARG;
        if (!ctx->net[1].tc_ok) return PIFU_ERR_UNSUPPORTED;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FrameKey k;
    std::memset(&k, 0, sizeof(k));   // padding too: keys are compared bytewise
    k.occ = occ_map->data;
    k.oH = occ_map->H;
    k.oW = occ_map->W;
    k.oC = occ_map->C;
    if (col_map) {
        k.col = col_map->data;
        k.cH = col_map->H;
        k.cW = col_map->W;
        k.cC = col_map->C;
    }
    std::memcpy(k.calib, calib, sizeof(k.calib));
    k.n0 = lv->n0;
    k.num_levels = lv->num_levels;
    k.precision = lv->precision;
    k.max_rounds = lv->max_rounds > 0 ? lv->max_rounds : 4096;
    k.margin = prec_mixed(lv->precision) ? lv->margin : 0.f;
    k.f8_version = prec_f8(lv->precision) ? ctx->net[0].f8_version : 0;
    if (lv->use_surrogate) {
        k.use_surrogate = 1;
        k.sur_margin = lv->surrogate_margin;
        k.sur_version = ctx->sur.version;
    }
    k.width = cam->width;
    k.height = cam->height;
    k.cam_precision = cam->precision;
    k.final_level = cam->final_level;
    for (int c = 0; c < 3; ++c) k.bg[c] = cam->background[c];
    k.depth = depth_dev;
    k.rgb = rgb_dev;
    k.mask = mask_dev;
    int st = ensure_level_ws(ctx, (int)n_fine);
    if (st != PIFU_OK) return st;
    st = ensure_hit_ws(ctx, (int64_t)cam->width * cam->height);
    if (st != PIFU_OK) return st;
    if (cam->final_level) {
        st = ensure_cull_ws(ctx, (int64_t)cam->width * cam->height, (int)n_fine);
        if (st != PIFU_OK) return st;
    }
    if (!ctx->g_valid || std::memcmp(&k, &ctx->gkey, sizeof(k)) != 0) {
        st = g_build(ctx, k, to_map(occ_map), to_map(col_map), to_calib(calib));
        if (st != PIFU_OK) return st;
    }
    ctx->have_volume = false;
    CK(cudaGraphLaunch(ctx->gexec, s));
    CK(cudaStreamSynchronize(s));
    const GraphStats& gs = *ctx->h_gstats;
    pifu_volume vs{};
    vs.num_levels = lv->num_levels;
    vs.evals_per_level[0] = (int64_t)(lv->n0 + 1) * (lv->n0 + 1) * (lv->n0 + 1);
    vs.n_eval = vs.evals_per_level[0];
    int64_t launches = ctx->g_launches_fixed;
    for (int l = 0; l < lv->num_levels; ++l) {
        if (l > 0) {
            vs.evals_per_level[l] = (int64_t)gs.evals[l];
            vs.n_eval += (int64_t)gs.evals[l];
            vs.candidates_per_level[l] = (int64_t)gs.cands[l];
            vs.conflict_rounds[l] = (int32_t)gs.rounds[l];
            launches += ctx->g_launches_body[l] * (int64_t)(gs.rounds[l] + 1);
        }
        vs.rechecked_per_level[l] = (int64_t)gs.rechecked[l];
        vs.fallback_per_level[l] = (int64_t)gs.fallback[l];
    }
    ctx->prof.k[PIFU_K_MLP_HIDDEN].launches += launches;   // graph: counted in one class
    const int cur = (lv->num_levels - 1) & 1;
    vs.n = (int32_t)n_fine;
    vs.row_words = row_words_of((int)n_fine);
    vs.occ_bits_dev = ctx->bin[cur];
    vs.eval_bits_dev = ctx->eval;
    vs.values_dev = ctx->values;
    if (cam->final_level && lv->num_levels < kMaxLevels)
        vs.evals_per_level[lv->num_levels] = (int64_t)gs.culled;   // the culled final level
    if (out) *out = vs;
    if (gs.err) return decode_err(gs.err);
    ctx->stats = vs;
    ctx->have_volume = true;
    ctx->vol_N = (int)n_fine;
    ctx->vol_bin = cur;
    ctx->vol_prec = lv->precision;
    ctx->vol_margin = lv->margin;
    return PIFU_OK;
}

int pifu_calibrate_fp8(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12], int n0,
                       void* stream) {
    if (!ctx || !calib || !map_ok(occ_map) || n0 < 1 || n0 > 256) return PIFU_ERR_ARG;
    if (ctx->net[0].d_in != occ_map->C + 1) return PIFU_ERR_ARG;
    if (ctx->net[0].kind == kNetCbn) return PIFU_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    ctx->g_valid = false;   // a captured frame holds the previous scales
    return calibrate_fp8(ctx, to_map(occ_map), to_calib(calib), n0,
                         static_cast<cudaStream_t>(stream));
}

int pifu_frames(pifu_ctx* ctx, int B, const pifu_fmap* occ_maps, const pifu_fmap* col_maps,
                const float* calibs, const pifu_levels* lv, const pifu_camera* cam, void* stream,
                float* depth_dev, float* rgb_dev, uint8_t* mask_dev, pifu_volume* out) {
    if (!ctx || B < 1 || B > kMaxBatch || !occ_maps || !calibs || !lv || !cam)
        return PIFU_ERR_ARG;
    const pifu_fmap& o0 = occ_maps[0];
    for (int f = 0; f < B; ++f) {
        const pifu_fmap& o = occ_maps[f];
        if (!map_ok(&o) || o.H != o0.H || o.W != o0.W || o.C != o0.C || o.dtype != o0.dtype)
            return PIFU_ERR_ARG;
        if (col_maps) {
            const pifu_fmap& c = col_maps[f];
            if (!map_ok(&c) || c.H != col_maps[0].H || c.W != col_maps[0].W ||
                c.C != col_maps[0].C || c.dtype != col_maps[0].dtype)
                return PIFU_ERR_ARG;
        }
    }
    if (!is_pow2(lv->n0) || lv->n0 < 2 || lv->num_levels < 1 || lv->num_levels > kMaxLevels)
        return PIFU_ERR_ARG;
    const int64_t n_fine = (int64_t)lv->n0 << (lv->num_levels - 1);
    if (n_fine > kMaxFine) return PIFU_ERR_ARG;
    if (cam->width < 1 || cam->height < 1) return PIFU_ERR_ARG;
    if (cam->final_level) return PIFU_ERR_UNSUPPORTED;   // lockstep batches ray-march the volume
    const int64_t npix = (int64_t)cam->width * cam->height;
    if ((int64_t)B * npix > kTcRowsMax) return PIFU_ERR_CAPACITY;
    if (!prec_valid(lv->precision) || lv->precision == PIFU_PREC_FP32) return PIFU_ERR_UNSUPPORTED;
    if (lv->subdivision != PIFU_SUBDIV_METHOD) return PIFU_ERR_UNSUPPORTED;
    if (ctx->net[0].kind == kNetCbn && (prec_f8(lv->precision) || lv->use_surrogate))
        return PIFU_ERR_UNSUPPORTED;
    if (prec_f8(lv->precision) && !ctx->net[0].f8_ok) return PIFU_ERR_STATE;
    if (prec_mixed(lv->precision) && !(lv->margin >= 0.f && lv->margin <= 0.5f))
        return PIFU_ERR_ARG;
    if (lv->use_surrogate) {
        if (!ctx->sur.ready || !ctx->snet.tc_ok) return PIFU_ERR_STATE;
        if (!(lv->surrogate_margin >= 0.f && lv->surrogate_margin <= 0.5f)) return PIFU_ERR_ARG;
    }
    if (ctx->net[0].d_in != o0.C + 1) return PIFU_ERR_ARG;
    if (!ctx->net[0].tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (rgb_dev) {
        const int c_t = col_maps ? col_maps[0].C : 0;
        if (ctx->net[1].d_in != c_t + o0.C + 1) return PIFU_ERR_ARG;
        if (!ctx->net[1].tc_ok) return PIFU_ERR_UNSUPPORTED;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = batch_ensure(ctx, B, (int)n_fine, npix);
    if (st != PIFU_OK) return st;
    BatchWs& bw = ctx->batch;
    BatchKey k;
    std::memset(&k, 0, sizeof(k));   // padding too: keys are compared bytewise
    k.B = B;
    k.oH = o0.H;
    k.oW = o0.W;
    k.oC = o0.C;
    k.odt = o0.dtype;
    if (col_maps) {
        k.cH = col_maps[0].H;
        k.cW = col_maps[0].W;
        k.cC = col_maps[0].C;
        k.cdt = col_maps[0].dtype;
    }
    k.n0 = lv->n0;
    k.num_levels = lv->num_levels;
    k.precision = lv->precision;
    k.max_rounds = lv->max_rounds > 0 ? lv->max_rounds : 4096;
    k.margin = prec_mixed(lv->precision) ? lv->margin : 0.f;
    if (lv->use_surrogate) {
        k.use_surrogate = 1;
        k.sur_margin = lv->surrogate_margin;
        k.sur_version = ctx->sur.version;
    }
    k.f8_version = prec_f8(lv->precision) ? ctx->net[0].f8_version : 0;
    k.width = cam->width;
    k.height = cam->height;
    for (int c = 0; c < 3; ++c) k.bg[c] = cam->background[c];
    k.depth = depth_dev;
    k.rgb = rgb_dev;
    k.mask = mask_dev;
    if (!bw.g_valid || std::memcmp(&k, &bw.key, sizeof(k)) != 0) {
        st = b_build(ctx, k);
        if (st != PIFU_OK) return st;
    }
    // this batch's maps and calibrations, read by the graph's kernels
    for (int f = 0; f < B; ++f) {
        bw.h_maps0[f] = to_map(&occ_maps[f]);
        bw.h_maps1[f] = col_maps ? to_map(&col_maps[f]) : Map{};
        bw.h_calibs[f] = to_calib(calibs + 12 * f);
    }
    CK(cudaMemcpyAsync(bw.d_maps0, bw.h_maps0, sizeof(Map) * B, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bw.d_maps1, bw.h_maps1, sizeof(Map) * B, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(bw.d_calibs, bw.h_calibs, sizeof(Calib) * B, cudaMemcpyHostToDevice, s));
    ctx->have_volume = false;
    CK(cudaGraphLaunch(bw.exec, s));
    CK(cudaStreamSynchronize(s));
    const BatchStats& gs = *bw.h_stats;
    const int64_t nodes0 = (int64_t)(lv->n0 + 1) * (lv->n0 + 1) * (lv->n0 + 1);
    int64_t launches = bw.launches_fixed;
    for (int l = 1; l < lv->num_levels; ++l) launches += bw.launches_body[l] * (int64_t)(gs.rounds[l] + 1);
    ctx->prof.k[PIFU_K_MLP_HIDDEN].launches += launches;   // graph: counted in one class
    const int cur = (lv->num_levels - 1) & 1;
    for (int f = 0; f < B && out; ++f) {
        pifu_volume vs{};
        vs.num_levels = lv->num_levels;
        vs.n = (int32_t)n_fine;
        vs.row_words = row_words_of((int)n_fine);
        vs.occ_bits_dev = bw.bin[cur] + f * bw.slot_words;
        vs.eval_bits_dev = bw.eval + f * bw.slot_words;
        vs.values_dev = bw.values + f * bw.slot_nodes;
        vs.evals_per_level[0] = nodes0;
        vs.n_eval = nodes0;
        for (int l = 0; l < lv->num_levels; ++l) {
            if (l > 0) {
                vs.evals_per_level[l] = (int64_t)gs.evals[l][f];
                vs.n_eval += (int64_t)gs.evals[l][f];
                vs.candidates_per_level[l] = (int64_t)gs.cands[l][f];
                vs.conflict_rounds[l] = (int32_t)gs.rounds[l];
            }
            vs.rechecked_per_level[l] = (int64_t)gs.rechecked[l];
            vs.fallback_per_level[l] = (int64_t)gs.fallback[l];
        }
        out[f] = vs;
    }
    if (gs.err) return decode_err(gs.err);
    return PIFU_OK;
}

int pifu_autotune(pifu_ctx* ctx, int64_t rows, void* stream, int32_t* bn_out, double* ms_out,
                  int n_max, int* n_layers) {
    if (!ctx || rows < 128 || rows > kTcRowsMax || n_max < 0) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    return autotune(ctx, rows, static_cast<cudaStream_t>(stream), bn_out, ms_out, n_max, n_layers);
}

int pifu_set_schedule(pifu_ctx* ctx, int schedule) {
    if (!ctx || (schedule != PIFU_SCHED_CHAINED && schedule != PIFU_SCHED_PER_LAYER))
        return PIFU_ERR_ARG;
    ctx->chain_on = schedule == PIFU_SCHED_CHAINED;
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    return PIFU_OK;
}

int pifu_set_tiles(pifu_ctx* ctx, const int32_t* codes, int n) {
    if (!ctx || n < 0 || (n > 0 && !codes)) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    return set_tiles(ctx, codes, n);
}

int pifu_surrogate_init(pifu_ctx* ctx, int h1, int h2, uint64_t seed) {
    if (!ctx || h1 < 64 || h2 < 64 || h1 % 64 || h2 % 64 || h1 > 1024 || h2 > 1024)
        return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    return sur_init(ctx, h1, h2, seed);
}

int pifu_surrogate_samples(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                           const float* pts_dev, int64_t m, float* x_dev, float* o_dev,
                           void* stream) {
    if (!ctx || !calib || m < 0 || !map_ok(occ_map)) return PIFU_ERR_ARG;
    if (m == 0) return PIFU_OK;
    if (!pts_dev || !x_dev || !o_dev) return PIFU_ERR_ARG;
    if (ctx->net[0].d_in != occ_map->C + 1) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Map map = to_map(occ_map);
    const Calib cal = to_calib(calib);
    PointSrc src{PTS_XYZ, pts_dev, nullptr, 0, 0, nullptr};
    // the rows f_S reads: [Phi(g_O), z, 0 ...] with the row width of f_O
    for (int64_t p0 = 0; p0 < m; p0 += kChunk) {
        const int64_t mc = std::min<int64_t>(kChunk, m - p0);
        CK(launch_gather(src, p0, mc, cal, map, Map{}, x_dev + p0 * ctx->net[0].ldx,
                         ctx->net[0].ldx, s));
    }
    // the targets: f_O's occupancy in FP32
    Epilogue epi{};
    epi.mode = EPI_STORE;
    epi.act = ACT_SIGMOID;
    epi.out = o_dev;
    return run_mlp(ctx, ctx->net[0], src, m, map, Map{}, cal, epi, s, PIFU_PREC_FP32);
}

int pifu_surrogate_query(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                         const float* pts_dev, int64_t m, float* occ_dev, int precision,
                         void* stream) {
    if (!ctx || !calib || m < 0 || !map_ok(occ_map)) return PIFU_ERR_ARG;
    if (!ctx->sur.ready) return PIFU_ERR_STATE;
    if (m == 0) return PIFU_OK;
    if (!pts_dev || !occ_dev) return PIFU_ERR_ARG;
    if (precision != PIFU_PREC_FP32 && precision != PIFU_PREC_BF16) return PIFU_ERR_UNSUPPORTED;
    if (precision == PIFU_PREC_BF16 && !ctx->snet.tc_ok) return PIFU_ERR_UNSUPPORTED;
    if (ctx->snet.d_in != occ_map->C + 1) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    PointSrc src{PTS_XYZ, pts_dev, nullptr, 0, 0, nullptr};
    Epilogue epi{};
    epi.mode = EPI_STORE;
    epi.act = ACT_SIGMOID;
    epi.out = occ_dev;
    return run_mlp(ctx, ctx->snet, src, m, to_map(occ_map), Map{}, to_calib(calib), epi,
                   static_cast<cudaStream_t>(stream), precision);
}

int pifu_surrogate_grad(pifu_ctx* ctx, const float* x_dev, const float* y_dev, int64_t B,
                        float* grad_host, double* loss_host, void* stream) {
    if (!ctx || !x_dev || !y_dev || B < 1 || B > (1 << 20)) return PIFU_ERR_ARG;
    if (!ctx->sur.ready) return PIFU_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = sur_batch_ws(ctx, (int)B);
    if (st != PIFU_OK) return st;
    CK(cudaMemsetAsync(ctx->sur.d_loss, 0, sizeof(double), s));
    st = sur_grad(ctx, x_dev, y_dev, (int)B, s);
    if (st != PIFU_OK) return st;
    CK(cudaMemcpyAsync(ctx->sur.h_loss, ctx->sur.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    std::vector<float> gp((size_t)ctx->sur.n);
    CK(cudaMemcpyAsync(gp.data(), ctx->sur.grads, (size_t)ctx->sur.n * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (grad_host) sur_pack(ctx, gp, grad_host);
    if (loss_host) *loss_host = *ctx->sur.h_loss;
    return PIFU_OK;
}

int pifu_surrogate_train(pifu_ctx* ctx, const float* x_dev, const float* y_dev, int64_t m,
                         int batch, int steps, float lr, double* loss_host, void* stream) {
    if (!ctx || !x_dev || !y_dev || m < 1 || batch < 1 || batch > (1 << 20) || steps < 0 ||
        !(lr > 0.f))
        return PIFU_ERR_ARG;
    if (!ctx->sur.ready) return PIFU_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto& S = ctx->sur;
    const int B = (int)std::min<int64_t>(batch, m);
    int st = sur_batch_ws(ctx, B);
    if (st != PIFU_OK) return st;
    const int64_t nb = m / B;   // whole batches; the samples are already in random order
    double first = 0.0;
    for (int it = 0; it < steps; ++it) {
        const int64_t b0 = (int64_t)(it % nb) * B;
        CK(cudaMemsetAsync(S.d_loss, 0, sizeof(double), s));
        st = sur_grad(ctx, x_dev + b0 * ctx->snet.ldx, y_dev + b0, B, s);
        if (st != PIFU_OK) return st;
        CK(launch_adam(S.n, S.params, S.grads, S.adam_m, S.adam_v, lr, ++S.step, s));
        if (it == 0) {
            CK(cudaMemcpyAsync(S.h_loss, S.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            first = *S.h_loss;
        }
    }
    CK(cudaMemcpyAsync(S.h_loss, S.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (loss_host) {
        loss_host[0] = first;
        loss_host[1] = *S.h_loss;
    }
    return sur_build_tc(ctx);   // inference form follows the new parameters
}

int pifu_surrogate_ohem_init(pifu_ctx* ctx, int64_t m) {
    if (!ctx || m < 1 || m > ((int64_t)1 << 31) - 1) return PIFU_ERR_ARG;
    if (!ctx->sur.ready) return PIFU_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    int st = ohem_ensure(ctx, m, 1, true);
    if (st != PIFU_OK) return st;
    CK(cudaDeviceSynchronize());
    return PIFU_OK;
}

int pifu_surrogate_ohem_weights(pifu_ctx* ctx, float* host, int64_t n, int set) {
    if (!ctx || !host) return PIFU_ERR_ARG;
    auto& S = ctx->sur;
    if (!S.ohem_w) return PIFU_ERR_STATE;
    if (n != S.ohem_m) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    CK(cudaMemcpy(set ? (void*)S.ohem_w : (void*)host, set ? (const void*)host : (const void*)S.ohem_w,
                  (size_t)n * 4, set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost));
    return PIFU_OK;
}

int pifu_surrogate_ohem_sample(pifu_ctx* ctx, uint64_t seed, int step, int B, int* idx_dev,
                               void* stream) {
    if (!ctx || !idx_dev || B < 1 || step < 0) return PIFU_ERR_ARG;
    auto& S = ctx->sur;
    if (!S.ohem_w) return PIFU_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_ohem_sample(S.ohem_w, S.ohem_m, S.ohem_cdf, S.ohem_sums, seed, (uint32_t)step, B,
                          idx_dev, s));
    CK(cudaStreamSynchronize(s));
    return PIFU_OK;
}

int pifu_surrogate_train_ohem(pifu_ctx* ctx, const float* x_dev, const float* y_dev, int64_t m,
                              int batch, int steps, float lr, float alpha, float beta,
                              uint64_t seed, double* loss_host, void* stream) {
    if (!ctx || !x_dev || !y_dev || m < 1 || batch < 1 || batch > (1 << 20) || steps < 0 ||
        !(lr > 0.f) || !(alpha > 0.f) || !(beta >= 0.f))
        return PIFU_ERR_ARG;
    auto& S = ctx->sur;
    if (!S.ready) return PIFU_ERR_STATE;
    if (S.ohem_m != m) return PIFU_ERR_STATE;   // pifu_surrogate_ohem_init(m) first
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int B = batch;
    int st = sur_batch_ws(ctx, B);
    if (st == PIFU_OK) st = ohem_ensure(ctx, m, B, false);
    if (st != PIFU_OK) return st;
    const int ldx = ctx->snet.ldx;
    double first = 0.0;
    for (int it = 0; it < steps; ++it) {
        // draw the batch by the current weights, train on it, re-weight it
        CK(launch_ohem_sample(S.ohem_w, m, S.ohem_cdf, S.ohem_sums, seed, (uint32_t)it, B, S.ib,
                              s));
        CK(launch_gather_rows(x_dev, y_dev, ldx, S.ib, B, S.xb, S.yb, s));
        CK(cudaMemsetAsync(S.d_loss, 0, sizeof(double), s));
        st = sur_grad(ctx, S.xb, S.yb, B, s, S.per_loss);
        if (st != PIFU_OK) return st;
        CK(launch_ohem_update(S.ohem_w, S.ib, S.per_loss, B, alpha, beta, s));
        CK(launch_adam(S.n, S.params, S.grads, S.adam_m, S.adam_v, lr, ++S.step, s));
        if (it == 0) {
            CK(cudaMemcpyAsync(S.h_loss, S.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            first = *S.h_loss;
        }
    }
    CK(cudaMemcpyAsync(S.h_loss, S.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (loss_host) {
        loss_host[0] = first;
        loss_host[1] = *S.h_loss;
    }
    return sur_build_tc(ctx);
}

int pifu_surrogate_params(pifu_ctx* ctx, float* host, int64_t n, int set) {
    if (!ctx) return PIFU_ERR_ARG;
    if (!ctx->sur.ready) return PIFU_ERR_STATE;
    if (!host || n != sur_unpadded_count(ctx)) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    std::vector<float> p;
    if (set) {
        sur_unpack(ctx, host, p);
        CK(cudaMemcpy(ctx->sur.params, p.data(), (size_t)ctx->sur.n * 4, cudaMemcpyHostToDevice));
        return sur_build_tc(ctx);
    }
    p.resize((size_t)ctx->sur.n);
    CK(cudaMemcpy(p.data(), ctx->sur.params, (size_t)ctx->sur.n * 4, cudaMemcpyDeviceToHost));
    sur_pack(ctx, p, host);
    return PIFU_OK;
}

int pifu_profile(pifu_ctx* ctx, int enable) {
    if (!ctx) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    ctx->prof.reset();
    ctx->prof.on = enable != 0;
    return PIFU_OK;
}

int pifu_profile_read(pifu_ctx* ctx, pifu_kernel_stats* out) {
    if (!ctx || !out) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = ctx->prof.resolve();
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    for (int i = 0; i < PIFU_K_COUNT; ++i) out[i] = ctx->prof.k[i];
    return PIFU_OK;
}

int pifu_sync_stats(pifu_ctx* ctx, pifu_volume* out) {
    if (!ctx || !out) return PIFU_ERR_ARG;
    if (!ctx->have_volume) return PIFU_ERR_STATE;
    *out = ctx->stats;
    return PIFU_OK;
}

}  // extern "C"
