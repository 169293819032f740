// The work-queue stream of frames (pifu_stream; not in the paper, whose
// frames are processed one by one): F frames go through S slots in one CUDA
// graph whose loop runs rounds on the device until the queue is drained.
//
// One round:
//   1. set-up and first selection of the slots that start a frame or advance
//      to their next level (one launch each, grid.y = slot);
//   2. one evaluation pass over the round's key list -- every slot's keys at
//      once, whatever level each slot is at: the gather and one persistent
//      tensor-core launch per layer (with the MIXED forms' FP32 re-check and
//      the surrogate's fall-back, as in the other graph forms);
//   3. the sparse conflict expansion, which queues the next round's keys of
//      the slots whose level is not converged;
//   4. the render of the slots whose finest level converged, and the colour
//      MLP over their hits (a conditional node: only rounds with hits);
//   5. the scheduler kernel, which takes every slot one step further
//      (stream_sched.cuh), hands free slots the next frames of the queue,
//      and sets the loop condition.
// So a frame runs exactly its own steps and conflict rounds; a frame with
// few rounds hands its slot to the next frame while the others iterate.
#include "host.h"

namespace pifu_host {

constexpr int kStreamMaxSlots = 16;
constexpr int kStreamMaxFrames = 4096;

void stream_free(pifu_ctx* ctx) {
    StreamWs& w = ctx->stream;
    if (w.exec) cudaGraphExecDestroy(w.exec);
    if (w.graph) cudaGraphDestroy(w.graph);
    w.exec = nullptr;
    w.graph = nullptr;
    w.g_valid = false;
    uint32_t** bits[] = {&w.cand, &w.tent, &w.bin[0], &w.bin[1], &w.eval, &w.conf};
    for (auto p : bits) dev_free(*p);
    dev_free(w.values);
    dev_free(w.top);
    dev_free(w.list);
    dev_free(w.recheck);
    dev_free(w.squeue);
    dev_free(w.hit_xyz);
    dev_free(w.hit_pix);
    dev_free(w.d_hits);
    dev_free(w.sv);
    dev_free(w.st);
    dev_free(w.pend);
    dev_free(w.cands);
    dev_free(w.slot_maps0);
    dev_free(w.slot_maps1);
    dev_free(w.slot_calibs);
    dev_free(w.frame_maps0);
    dev_free(w.frame_maps1);
    dev_free(w.frame_calibs);
    dev_free(w.d_fs);
    dev_free(w.d_ctl);
    if (w.h_maps0) cudaFreeHost(w.h_maps0);
    if (w.h_maps1) cudaFreeHost(w.h_maps1);
    if (w.h_calibs) cudaFreeHost(w.h_calibs);
    if (w.h_fs) cudaFreeHost(w.h_fs);
    if (w.h_ctl) cudaFreeHost(w.h_ctl);
    w.h_maps0 = w.h_maps1 = nullptr;
    w.h_calibs = nullptr;
    w.h_fs = nullptr;
    w.h_ctl = nullptr;
    w.S = w.N = w.F = 0;
    w.npix = w.slot_words = w.slot_nodes = w.slot_top = w.cap = 0;
}

// Key-list capacity of one round: S x 2^18 keys rounded up to a power of two
// (between 2^20 and kTcRowsMax), and at least the hits of S renders.
int64_t stream_cap(int S, int64_t npix) {
    int64_t c = batch_cap(S);
    while (c < (int64_t)S * npix && c < kTcRowsMax) c *= 2;
    return c;
}

int stream_ensure(pifu_ctx* ctx, int S, int N, int F, int64_t npix) {
    StreamWs& w = ctx->stream;
    if (w.S >= S && w.N == N && w.F >= F && w.npix >= npix) return PIFU_OK;
    const int Sn = std::max(S, w.S);
    const int Fn = std::max(F, w.F);
    const int64_t np = std::max(npix, w.npix);
    stream_free(ctx);
    invalidate_graphs(ctx);
    const int64_t words = words_of(N);
    const int64_t nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
    if ((int64_t)Sn * nodes > 2147483647LL) return PIFU_ERR_ARG;   // int32 keys
    uint32_t** bits[] = {&w.cand, &w.tent, &w.bin[0], &w.bin[1], &w.eval, &w.conf};
    for (auto p : bits) {
        CK(dev_alloc(p, words * Sn));
        CK(cudaMemset(*p, 0, (size_t)(words * Sn) * 4));
    }
    const int64_t cap = stream_cap(Sn, np);
    const int64_t top = 2 * (int64_t)(N + 1) * (N + 1);
    CK(dev_alloc(&w.values, nodes * Sn));
    CK(dev_alloc(&w.top, top * Sn));
    CK(dev_alloc(&w.list, cap));
    CK(dev_alloc(&w.recheck, 2 * cap));   // a surrogate round's f_O pass takes up to 2 cap
    // the surrogate's f_O queue: the finest-level keys, then f_S's fall-backs
    CK(dev_alloc(&w.squeue, 2 * cap));
    CK(dev_alloc(&w.hit_xyz, 3 * np * Sn));
    CK(dev_alloc(&w.hit_pix, np * Sn));
    CK(dev_alloc(&w.d_hits, 1));
    CK(dev_alloc(&w.sv, Sn));
    CK(cudaMemset(w.sv, 0, sizeof(SlotView) * (size_t)Sn));
    CK(dev_alloc(&w.st, Sn));
    CK(dev_alloc(&w.pend, 2 * (int64_t)Sn));
    CK(dev_alloc(&w.cands, Sn));
    CK(dev_alloc(&w.slot_maps0, Sn));
    CK(dev_alloc(&w.slot_maps1, Sn));
    CK(dev_alloc(&w.slot_calibs, Sn));
    CK(dev_alloc(&w.frame_maps0, Fn));
    CK(dev_alloc(&w.frame_maps1, Fn));
    CK(dev_alloc(&w.frame_calibs, Fn));
    CK(dev_alloc(&w.d_fs, Fn));
    CK(dev_alloc(&w.d_ctl, 1));
    CK(cudaHostAlloc(&w.h_maps0, sizeof(Map) * (size_t)Fn, cudaHostAllocDefault));
    CK(cudaHostAlloc(&w.h_maps1, sizeof(Map) * (size_t)Fn, cudaHostAllocDefault));
    CK(cudaHostAlloc(&w.h_calibs, sizeof(Calib) * (size_t)Fn, cudaHostAllocDefault));
    CK(cudaHostAlloc(&w.h_fs, sizeof(StreamFrameStats) * (size_t)Fn, cudaHostAllocDefault));
    CK(cudaHostAlloc(&w.h_ctl, sizeof(StreamCtl), cudaHostAllocDefault));
    w.S = Sn;
    w.N = N;
    w.F = Fn;
    w.npix = np;
    w.slot_words = words;
    w.slot_nodes = nodes;
    w.slot_top = top;
    w.cap = cap;
    return PIFU_OK;
}

// The stream's graph, captured on ctx->cap_stream (the loop body on
// cap_stream2).  g_eval's queues are pointed at the stream's for the capture.
int g_enqueue_stream(pifu_ctx* ctx, const StreamKey& k) {
    StreamWs& w = ctx->stream;
    cudaStream_t s = ctx->cap_stream;
    cudaStream_t sb = ctx->cap_stream2;
    unsigned int* err = ctx->d_count + 1;
    const DevNet& net = ctx->net[0];
    const int S = k.S;
    const int N_fine = k.n0 << (k.num_levels - 1);
    const int64_t cap = w.cap;
    const int64_t npix = (int64_t)k.width * k.height;
    int st = PIFU_OK;
    CK(cudaMemsetAsync(err, 0, sizeof(unsigned int), s));
    CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
    CK(cudaMemsetAsync(ctx->d_ccount, 0, sizeof(unsigned int), s));
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
    StreamArgs a{};
    a.sv = w.sv;
    a.st = w.st;
    a.fs = w.d_fs;
    a.ctl = w.d_ctl;
    a.pend_eval = w.pend;
    a.pend_next = w.pend + S;
    a.cands = w.cands;
    a.S = S;
    a.F = k.F;
    a.L = k.num_levels;
    a.n0 = k.n0;
    a.max_rounds = k.max_rounds;
    // a frame takes at most L set-ups, L x max_rounds conflict rounds and a
    // render; the queue adds one round per slot at most
    a.max_total_rounds = (unsigned)std::min<int64_t>(
        4000000000LL, (int64_t)k.F * (k.num_levels * ((int64_t)k.max_rounds + 1) + 2) + S + 8);
    a.cand = w.cand;
    a.tent = w.tent;
    a.bin0 = w.bin[0];
    a.bin1 = w.bin[1];
    a.eval = w.eval;
    a.conf = w.conf;
    a.values = w.values;
    a.top = w.top;
    a.slot_words = w.slot_words;
    a.slot_nodes = w.slot_nodes;
    a.slot_top = w.slot_top;
    a.frame_maps0 = w.frame_maps0;
    a.frame_maps1 = k.cC > 0 ? w.frame_maps1 : nullptr;
    a.frame_calibs = w.frame_calibs;
    a.slot_maps0 = w.slot_maps0;
    a.slot_maps1 = w.slot_maps1;
    a.slot_calibs = w.slot_calibs;
    a.depth = k.depth;
    a.rgb = k.rgb;
    a.mask = k.mask;
    a.bits_out = k.bits_out;
    a.npix = npix;
    a.out_words = words_of(N_fine);
    a.err = err;
    a.h = h;
    a.init = 1;
    CK(cudaMemsetAsync(w.d_hits, 0, sizeof(unsigned int), s));
    CK(cudaMemsetAsync(ctx->d_squeue, 0, sizeof(unsigned int), s));
    // the hit list holds the hits of every render since the last colour pass
    const int64_t hcap = std::min<int64_t>((int64_t)w.S * w.npix, cap);
    // the colour MLP over the hit list, then the list emptied
    auto colour_pass = [&](cudaStream_t cs) -> int {
        PointSrc hs{PTS_XYZ, w.hit_xyz, nullptr, 0, 0, nullptr};
        const bool col = k.cC > 0;
        hs.maps0 = col ? w.frame_maps1 : w.frame_maps0;   // colour maps first (Eq. 2)
        hs.maps1 = col ? w.frame_maps0 : nullptr;
        hs.calibs = w.frame_calibs;
        hs.keys = w.hit_pix;
        hs.slot_div = npix;
        Epilogue he{};
        he.mode = EPI_PIXELS;
        he.act = ACT_TANH01;
        he.out = k.rgb;
        he.pix = w.hit_pix;
        int r = run_mlp_tc(ctx, ctx->net[1], hs, hcap, Map{}, Map{}, Calib{}, he, cs, w.d_hits);
        if (r == PIFU_OK && cudaMemsetAsync(w.d_hits, 0, sizeof(unsigned int), cs) != cudaSuccess)
            r = PIFU_ERR_CUDA;
        return r;
    };
    CK(launch_stream_sched(a, s));   // admits the first frames, sets the condition
    cudaGraph_t body = nullptr;
    st = g_add_while(ctx, s, h, &body);
    if (st != PIFU_OK) return st;
    const int64_t before = launches_now(ctx);
    CK(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    {
        // With the surrogate, the keys of slots at their finest level go
        // straight to f_O's queue (that level always runs f_O); f_S runs on
        // the coarse levels' keys and appends its fall-backs after them.
        const bool sur = k.use_surrogate != 0;
        int* list_f = sur ? w.squeue : nullptr;
        unsigned int* count_f = sur ? ctx->d_squeue : nullptr;
        // 1. set-up and first selection of the starting and advancing slots
        if (launch_stream_setup(w.sv, S, N_fine, sb) != cudaSuccess ||
            launch_stream_select(w.sv, S, N_fine, w.slot_nodes, w.list, ctx->d_count,
                                 (unsigned)cap, err, a.pend_eval, w.cands, sb, list_f,
                                 count_f) != cudaSuccess)
            st = PIFU_ERR_CUDA;
        ctx->prof.k[PIFU_K_LEVEL].launches += 1;
        ctx->prof.k[PIFU_K_SELECT].launches += 1;
        // 2. one evaluation pass over every slot's keys
        PointSrc src{PTS_LIST, nullptr, w.list, 0, N_fine, nullptr};
        src.maps0 = w.slot_maps0;
        src.calibs = w.slot_calibs;
        src.slot_div = w.slot_nodes;
        src.sv = w.sv;
        Epilogue epi{};
        epi.mode = EPI_LEVEL;
        epi.list = w.list;
        epi.lv = LevelBits{w.values, w.tent, w.bin[0], w.conf, N_fine, row_words_of(N_fine), 0,
                           w.slot_nodes, w.slot_nodes, w.slot_words};
        epi.lv.clist = ctx->clist;
        epi.lv.ccount = ctx->d_ccount;
        epi.lv.ccap = (unsigned)ctx->clist_cap;
        epi.lv.err = err;
        epi.lv.sv = w.sv;
        if (st == PIFU_OK &&
            cudaMemsetAsync(ctx->d_ccount, 0, sizeof(unsigned int), sb) != cudaSuccess)
            st = PIFU_ERR_CUDA;
        if (st == PIFU_OK)
            st = g_eval(ctx, net, src, cap, ctx->d_count, Map{}, Calib{}, epi, k.precision,
                        k.margin, &w.d_ctl->rechecked, sb, sur, k.sur_margin,
                        &w.d_ctl->fallback, sur ? std::min<int64_t>(2 * cap, kTcRowsMax) : 0);
        if (st == PIFU_OK && sur &&
            cudaMemsetAsync(ctx->d_squeue, 0, sizeof(unsigned int), sb) != cudaSuccess)
            st = PIFU_ERR_CUDA;
        // 3. the next round's keys: the unevaluated ring of this round's conflicts
        if (st == PIFU_OK && cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), sb) != cudaSuccess)
            st = PIFU_ERR_CUDA;
        if (st == PIFU_OK &&
            launch_expand_conflicts(ctx->clist, ctx->d_ccount, (unsigned)ctx->clist_cap, N_fine,
                                    w.eval, w.slot_nodes, w.slot_words, w.list, ctx->d_count,
                                    (unsigned)cap, err, sb, w.sv, a.pend_next, list_f,
                                    count_f) != cudaSuccess)
            st = PIFU_ERR_CUDA;
        ctx->prof.k[PIFU_K_SELECT].launches += 1;
        // 4. colour of the hits gathered so far, when the hit list could not
        //    take this round's renders; then the render of the converged slots.
        //    The colour pass is deferred so that it runs on many frames' hits
        //    at once (the rest run after the loop).
        RenderArgs ra{};
        ra.width = k.width;
        ra.height = k.height;
        for (int c = 0; c < 3; ++c) ra.bg[c] = k.bg[c];
        ra.hit_xyz = w.hit_xyz;
        ra.hit_pix = w.hit_pix;
        ra.hit_count = w.d_hits;
        if (st == PIFU_OK && k.rgb) {
            cudaStreamCaptureStatus cs2;
            cudaGraph_t cgb = nullptr;
            cudaGraphConditionalHandle hc;
            if (cudaStreamGetCaptureInfo(sb, &cs2, nullptr, &cgb, nullptr, nullptr, nullptr) !=
                    cudaSuccess ||
                cudaGraphConditionalHandleCreate(&hc, cgb, 0, 0) != cudaSuccess ||
                launch_colour_cond(hc, w.d_hits, w.sv, S, npix, (unsigned)hcap, &w.d_ctl->colour_passes,
                                   sb) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            cudaGraph_t cbody = nullptr;
            if (st == PIFU_OK) st = g_add_cond(ctx, sb, hc, cudaGraphCondTypeIf, &cbody);
            cudaStream_t s3 = ctx->cap_stream3;
            if (st == PIFU_OK &&
                cudaStreamBeginCaptureToGraph(s3, cbody, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                st = PIFU_ERR_CUDA;
            const int64_t before_colour = launches_now(ctx);
            if (st == PIFU_OK) {
                st = colour_pass(s3);
                cudaGraph_t out = nullptr;
                const cudaError_t ee = cudaStreamEndCapture(s3, &out);
                if (st == PIFU_OK && ee != cudaSuccess) st = PIFU_ERR_CUDA;
            }
            w.launches_colour = launches_now(ctx) - before_colour;
        } else if (st == PIFU_OK &&
                   cudaMemsetAsync(w.d_hits, 0, sizeof(unsigned int), sb) != cudaSuccess) {
            st = PIFU_ERR_CUDA;   // no colour: the hit list starts empty every round
        }
        if (st == PIFU_OK && launch_stream_render(w.sv, S, N_fine, ra, sb) != cudaSuccess)
            st = PIFU_ERR_CUDA;
        ctx->prof.k[PIFU_K_RENDER].launches += 3;
        // 5. every slot one step further; the loop condition
        a.init = 0;
        if (st == PIFU_OK && launch_stream_sched(a, sb) != cudaSuccess) st = PIFU_ERR_CUDA;
    }
    cudaGraph_t body_out = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(sb, &body_out);
    if (st != PIFU_OK) return st;
    if (ee != cudaSuccess) return fail_cuda(ctx, ee);
    w.launches_body = launches_now(ctx) - before - w.launches_colour;
    if (k.rgb) {
        // the colour of the hits the loop left
        st = colour_pass(s);
        if (st != PIFU_OK) return st;
    }
    CK(cudaMemcpyAsync(w.h_ctl, w.d_ctl, sizeof(StreamCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(w.h_fs, w.d_fs, sizeof(StreamFrameStats) * (size_t)k.F,
                       cudaMemcpyDeviceToHost, s));
    return PIFU_OK;
}

int s_build(pifu_ctx* ctx, const StreamKey& k) {
    StreamWs& w = ctx->stream;
    if (w.exec) cudaGraphExecDestroy(w.exec);
    if (w.graph) cudaGraphDestroy(w.graph);
    w.exec = nullptr;
    w.graph = nullptr;
    w.g_valid = false;
    w.launches_colour = 0;
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (!ctx->cap_stream2) CK(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
    if (!ctx->cap_stream3) CK(cudaStreamCreateWithFlags(&ctx->cap_stream3, cudaStreamNonBlocking));
    if (!ctx->cap_stream4) CK(cudaStreamCreateWithFlags(&ctx->cap_stream4, cudaStreamNonBlocking));
    {
        const int st = ensure_clist(ctx, 2 * w.cap);
        if (st != PIFU_OK) return st;
    }
    CK(tc_prepare());
    CK(chain_prepare());
    {
        // the surrogate's f_O pass takes up to twice a round's list (its
        // finest-level keys and the fall-backs)
        const int64_t rows = k.use_surrogate ? std::min<int64_t>(2 * w.cap, kTcRowsMax) : w.cap;
        int st = ensure_tc_rows(ctx, rows);
        if (st == PIFU_OK && (k.precision == PIFU_PREC_MIXED || k.precision == PIFU_PREC_FP8_MIXED))
            st = ensure_x3(ctx);
        if (st != PIFU_OK) return st;
    }
    // g_eval's queues are the context's; point them at the stream's for the capture
    int* keep_recheck = ctx->recheck;
    int* keep_squeue = ctx->squeue;
    ctx->recheck = w.recheck;
    ctx->squeue = w.squeue;
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;
    const int64_t before = launches_now(ctx);
    int st = PIFU_OK;
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (ee == cudaSuccess) {
        st = g_enqueue_stream(ctx, k);
        ee = cudaStreamEndCapture(ctx->cap_stream, &g);
    }
    ctx->recheck = keep_recheck;
    ctx->squeue = keep_squeue;
    ctx->prof.on = prof_on;
    w.launches_fixed = launches_now(ctx) - before - w.launches_body - w.launches_colour;
    for (auto& x : ctx->prof.k) x.launches = 0;   // capture is not execution
    if (st != PIFU_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ee != cudaSuccess) return fail_cuda(ctx, ee);
    w.graph = g;
    const cudaError_t ie = cudaGraphInstantiate(&w.exec, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        w.graph = nullptr;
        return fail_cuda(ctx, ie);
    }
    w.key = k;
    w.g_valid = true;
    return PIFU_OK;
}

}  // namespace pifu_host

using namespace pifu_host;

extern "C" {

int pifu_stream(pifu_ctx* ctx, int F, const pifu_fmap* occ_maps, const pifu_fmap* col_maps,
                const float* calibs, int slots, const pifu_levels* lv, const pifu_camera* cam,
                void* stream, float* depth_dev, float* rgb_dev, uint8_t* mask_dev,
                uint32_t* occ_bits_dev, pifu_volume* out, pifu_frame_time* times) {
    if (!ctx || F < 1 || F > kStreamMaxFrames || slots < 1 || slots > kStreamMaxSlots ||
        !occ_maps || !calibs || !lv || !cam)
        return PIFU_ERR_ARG;
    const pifu_fmap& o0 = occ_maps[0];
    for (int f = 0; f < F; ++f) {
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
    if (cam->final_level) return PIFU_ERR_UNSUPPORTED;   // the stream ray-marches the volume
    const int64_t npix = (int64_t)cam->width * cam->height;
    if ((int64_t)slots * npix > kTcRowsMax || (int64_t)F * npix > 2147483647LL)
        return PIFU_ERR_CAPACITY;
    if (!prec_valid(lv->precision) || lv->precision == PIFU_PREC_FP32) return PIFU_ERR_UNSUPPORTED;
    if (lv->subdivision != PIFU_SUBDIV_METHOD) return PIFU_ERR_UNSUPPORTED;
    if (ctx->net[0].kind == kNetCbn) return PIFU_ERR_UNSUPPORTED;
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
    int st = stream_ensure(ctx, slots, (int)n_fine, F, npix);
    if (st != PIFU_OK) return st;
    StreamWs& w = ctx->stream;
    StreamKey k;
    std::memset(&k, 0, sizeof(k));   // padding too: keys are compared bytewise
    k.F = F;
    k.S = slots;
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
    k.bits_out = occ_bits_dev;
    if (!w.g_valid || std::memcmp(&k, &w.key, sizeof(k)) != 0) {
        st = s_build(ctx, k);
        if (st != PIFU_OK) return st;
    }
    // this call's maps and calibrations, read by the graph's kernels
    for (int f = 0; f < F; ++f) {
        w.h_maps0[f] = to_map(&occ_maps[f]);
        w.h_maps1[f] = col_maps ? to_map(&col_maps[f]) : Map{};
        w.h_calibs[f] = to_calib(calibs + 12 * f);
    }
    CK(cudaMemcpyAsync(w.frame_maps0, w.h_maps0, sizeof(Map) * F, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.frame_maps1, w.h_maps1, sizeof(Map) * F, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.frame_calibs, w.h_calibs, sizeof(Calib) * F, cudaMemcpyHostToDevice, s));
    ctx->have_volume = false;
    CK(cudaGraphLaunch(w.exec, s));
    CK(cudaStreamSynchronize(s));
    const StreamCtl& ctl = *w.h_ctl;
    // graph: counted in one class; the deferred colour pass runs when it fired
    ctx->prof.k[PIFU_K_MLP_HIDDEN].launches += w.launches_fixed +
                                              w.launches_body * (int64_t)ctl.rounds +
                                              w.launches_colour * (int64_t)ctl.colour_passes;
    // the last frame each slot held keeps its volume there
    std::vector<int> last(slots, -1);
    for (int f = 0; f < F; ++f) {
        const int sl = w.h_fs[f].slot;
        if (sl >= 0 && sl < slots && (last[sl] < 0 || w.h_fs[f].t_admit >= w.h_fs[last[sl]].t_admit))
            last[sl] = f;
    }
    const int cur = (lv->num_levels - 1) & 1;   // the finest level's binarized bitset
    // f_O's queue also took every finest-level key: the fall-backs are the rest
    int64_t fallback = (int64_t)ctl.fallback;
    if (lv->use_surrogate)
        for (int f = 0; f < F; ++f) fallback -= (int64_t)w.h_fs[f].evals[lv->num_levels - 1];
    for (int f = 0; f < F; ++f) {
        const StreamFrameStats& fs = w.h_fs[f];
        if (out) {
            pifu_volume vs{};
            vs.num_levels = lv->num_levels;
            vs.n = (int32_t)n_fine;
            vs.row_words = row_words_of((int)n_fine);
            const int sl = fs.slot;
            if (sl >= 0 && sl < slots && last[sl] == f) {
                vs.occ_bits_dev = w.bin[cur] + (int64_t)sl * w.slot_words;
                vs.eval_bits_dev = w.eval + (int64_t)sl * w.slot_words;
                vs.values_dev = w.values + (int64_t)sl * w.slot_nodes;
            }
            for (int l = 0; l < lv->num_levels; ++l) {
                vs.evals_per_level[l] = (int64_t)fs.evals[l];
                vs.n_eval += (int64_t)fs.evals[l];
                vs.candidates_per_level[l] = (int64_t)fs.cands[l];
                vs.conflict_rounds[l] = (int32_t)fs.rounds[l];
            }
            vs.rechecked_per_level[0] = (int64_t)ctl.rechecked;
            vs.fallback_per_level[0] = fallback;
            out[f] = vs;
        }
        if (times) {
            times[f].admit_ms = (float)((double)(fs.t_admit - ctl.t_start) * 1e-6);
            times[f].done_ms = (float)((double)(fs.t_done - ctl.t_start) * 1e-6);
            times[f].slot = fs.slot;
            times[f].stream_rounds = (int32_t)ctl.rounds;
        }
    }
    if (ctl.err) {
        CK(cudaMemsetAsync(ctx->d_count + 1, 0, sizeof(unsigned int), s));
        const int st = reset_after_error(ctx, s);
        return st != PIFU_OK ? st : decode_err(ctl.err);
    }
    for (int f = 0; f < F; ++f)
        if (!w.h_fs[f].done) return PIFU_ERR_NOT_CONVERGED;
    return PIFU_OK;
}

}  // extern "C"
