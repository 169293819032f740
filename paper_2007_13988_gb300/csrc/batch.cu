// Lockstep batches of frames (pifu_frames).
#include "host.h"

namespace pifu_host {

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
        int st = ensure_tc_rows(ctx, std::max<int64_t>(bw.cap, (int64_t)k.B * k.width * k.height));
        if (st == PIFU_OK && (k.precision == PIFU_PREC_MIXED || k.precision == PIFU_PREC_FP8_MIXED))
            st = ensure_x3(ctx);
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


}  // namespace pifu_host

using namespace pifu_host;

extern "C" {

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
    if (gs.err) {
        const int st = reset_after_error(ctx, s);
        return st != PIFU_OK ? st : decode_err(gs.err);
    }
    return PIFU_OK;
}

}  // extern "C"
