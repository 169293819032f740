// The frame as one CUDA graph (pifu_frame): device-sized batches, conditional nodes for the conflict loops and the FP32 re-checks.
#include "host.h"

namespace pifu_host {

int g_add_cond(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h,
               cudaGraphConditionalNodeType type, cudaGraph_t* body);

int g_add_switch(pifu_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, int n,
                 cudaGraph_t* bodies);
int64_t launches_now(const pifu_ctx* ctx);

// The FP32 pass over a device-sized queue in the graph.  With the fused
// kernel, a switch node set on the device from the queue length launches it
// with the cluster size that length calls for (few points: large clusters,
// the lowest latency per tile; many: small clusters, more tiles per round);
// in the default re-check form a queue of at most grid_rows points runs the
// whole-GPU FP32 network instead, and, when the split-TF32 network is usable
// (x3_usable), a queue of more than x3_min_rows and at most kX3Rows points
// runs that network (one more body each of the same switch).  An empty queue
// launches nothing.
// The FP32 forms a device-sized batch of at most `cap` points may take:
// the plan's cluster sizes, then the split-TF32 network (x3), then the
// whole-GPU network (ghi > 0: batches of at most ghi points); single: one
// form only (the cluster network at its default size), so no switch.
struct Fp32Forms {
    FusedPlan plan;
    int64_t x3_lo = 0, ghi = 0;
    bool x3 = false, single = true;
    int n = 1;   // bodies of the switch
};

Fp32Forms fp32_forms(pifu_ctx* ctx, const DevNet& net, int64_t cap) {
    Fp32Forms f;
    const FusedNet fz = fused_of(net);
    const bool sw = net.kind != kNetCbn && ctx->cap_stream4 && fused_ok(fz);
    if (sw) f.plan = fused_plan(fz);
    f.x3_lo = x3_min_rows(ctx);
    f.x3 = sw && f.plan.n >= 1 && x3_usable(ctx, net) && cap > f.x3_lo;
    f.ghi = sw && f.plan.n >= 1 ? std::min<int64_t>(grid_rows(ctx, net), cap) : 0;
    f.single = f.plan.n <= 1 && !f.x3 && f.ghi <= 0;
    f.n = f.single ? 1 : f.plan.n + (f.x3 ? 1 : 0) + (f.ghi > 0 ? 1 : 0);
    return f;
}

// Body i of a switch over fp32_forms(ctx, net, cap), captured on s.
int fp32_form_body(pifu_ctx* ctx, const DevNet& net, const Fp32Forms& f, int i,
                   const PointSrc& src, int64_t cap, const Map& map, const Calib& cal,
                   const Epilogue& epi, cudaStream_t s, const unsigned int* m_dev) {
    if (f.single)
        return run_mlp(ctx, net, src, cap, map, Map{}, cal, epi, s, PIFU_PREC_FP32, m_dev);
    if (i < f.plan.n)
        return run_mlp(ctx, net, src, cap, map, Map{}, cal, epi, s, PIFU_PREC_FP32, m_dev,
                       f.plan.cl[i]);
    if (f.x3 && i == f.plan.n)
        return run_mlp_x3(ctx, net, src, std::min<int64_t>(cap, kX3Rows), map, Map{}, cal, epi, s,
                          m_dev);
    return run_mlp_grid(ctx, net, src, f.ghi, map, Map{}, cal, epi, s, m_dev);
}

int g_recheck(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t cap,
              const Map& map, const Calib& cal, const Epilogue& epi, cudaStream_t s,
              const unsigned int* m_dev, unsigned long long* stat, unsigned int stat_cap) {
    Fp32Forms f = fp32_forms(ctx, net, cap);
    if (s == ctx->cap_stream4) f = Fp32Forms{};   // inside a switch body: one form, no switch
    if (f.single) {
        if (stat) CK(launch_accumulate(stat, m_dev, stat_cap, ctx->d_count + 1, s));
        return run_mlp(ctx, net, src, cap, map, Map{}, cal, epi, s, PIFU_PREC_FP32, m_dev);
    }
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
    CK(launch_fused_switch(h, f.plan, m_dev, (unsigned)cap, s, f.x3 ? (unsigned)f.x3_lo : 0u,
                           f.x3 ? (unsigned)kX3Rows : 0u, f.ghi > 0 ? (unsigned)f.ghi : 0u, stat,
                           stat_cap, ctx->d_count + 1));
    const int nb = f.n;
    cudaGraph_t bodies[6] = {};
    int st = g_add_switch(ctx, s, h, nb, bodies);
    if (st != PIFU_OK) return st;
    cudaStream_t s4 = ctx->cap_stream4;
    const int64_t before = launches_now(ctx);
    for (int i = 0; i < nb; ++i) {
        CK(cudaStreamBeginCaptureToGraph(s4, bodies[i], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        st = fp32_form_body(ctx, net, f, i, src, cap, map, cal, epi, s4, m_dev);
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(s4, &out);
        if (st != PIFU_OK) return st;
        if (ee != cudaSuccess) return fail_cuda(ctx, ee);
    }
    // one body, one launch, runs per replay
    ctx->prof.k[PIFU_K_MLP_F32].launches -= (launches_now(ctx) - before) - 1;
    return PIFU_OK;
}

// One evaluation batch in the graph: BF16 on the tensor cores, and for MIXED
// the FP32 re-evaluation of the queued near-0.5 occupancies (device-sized).
// With `sur`, f_S runs first and f_O takes the occupancies f_S put within
// `sur_margin` of 0.5 (a device-sized queue; *fallback += its length).
// rs (a conflict round's start, m_dev its batch size): the round's statistics
// and the zeroing of its conflict count, merged into the launch that sets
// the tiny/large branch where the batch takes that branch, else launched
// before the batch.
int g_eval(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t cap,
           const unsigned int* m_dev, const Map& map, const Calib& cal, const Epilogue& epi,
           int prec, float margin, unsigned long long* rechecked, cudaStream_t s,
           bool sur, float sur_margin, unsigned long long* fallback, int64_t qcap_in,
           const RoundStart* rs, bool recheck_zeroed) {
    const bool branch = !sur && prec != PIFU_PREC_BF16 && prec != PIFU_PREC_FP8 && m_dev &&
                        ctx->cap_stream3 && s != ctx->cap_stream3;
    if (rs && !branch)
        CK(launch_round_start(const_cast<unsigned int*>(m_dev), *rs, s));
    if (sur) {
        // qcap_in > 0: the f_O queue already holds keys (the frame stream's
        // finest-level keys), f_S's fall-backs are appended after them
        if (qcap_in <= 0) CK(cudaMemsetAsync(ctx->d_squeue, 0, sizeof(unsigned int), s));
        Epilogue es = epi;
        es.recheck = ctx->squeue;
        es.recheck_count = ctx->d_squeue;
        es.margin = sur_margin;
        int st = run_mlp_tc(ctx, ctx->snet, src, cap, map, Map{}, cal, es, s, m_dev);
        if (st != PIFU_OK) return st;
        // a queue longer than one device-sized batch latches a capacity error
        const int64_t qcap = std::min<int64_t>(qcap_in > 0 ? qcap_in : cap, kTcRowsMax);
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
    if (branch) {
        // A device-sized batch of at most kTinyBatch points goes straight to
        // FP32, as in the host-driven form; the tensor-core pass and its
        // re-check run above that.  One SWITCH, set on the device (with a
        // conflict round's start in the same launch): its first bodies are
        // g_recheck's FP32 forms for the small batch, its last the
        // tensor-core pass; an empty batch runs none.
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
        cudaStream_t s3 = ctx->cap_stream3;
        // the FP32 forms g_recheck would switch between for this capacity
        const Fp32Forms f = fp32_forms(ctx, net, cap);
        const int nt = f.n;
        CK(launch_batch_switch(h, f.plan, const_cast<unsigned int*>(m_dev), (unsigned)cap,
                               (unsigned)kTinyBatch, nt, f.single, f.x3 ? (unsigned)f.x3_lo : 0u,
                               f.x3 ? (unsigned)kX3Rows : 0u, f.ghi > 0 ? (unsigned)f.ghi : 0u, rs,
                               ctx->d_recheck, s));
        cudaGraph_t bodies[8] = {};
        int st = g_add_switch(ctx, s, h, nt + 1, bodies);
        if (st != PIFU_OK) return st;
        const int64_t before = launches_now(ctx);
        int64_t small = 0;
        for (int i = 0; i <= nt; ++i) {
            CK(cudaStreamBeginCaptureToGraph(s3, bodies[i], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
            if (i == nt)
                st = g_eval(ctx, net, src, cap, m_dev, map, cal, epi, prec, margin, rechecked, s3,
                            false, 0.f, nullptr, 0, nullptr, true);
            else
                st = fp32_form_body(ctx, net, f, i, src, cap, map, cal, epi, s3, m_dev);
            cudaGraph_t out = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(s3, &out);
            if (st != PIFU_OK) return st;
            if (ee != cudaSuccess) return fail_cuda(ctx, ee);
            if (i + 1 == nt) small = launches_now(ctx) - before;
        }
        // one small body, one launch, runs per replay (the large body's
        // launches stay counted, as the branch that does the work)
        ctx->prof.k[PIFU_K_MLP_F32].launches -= small - 1;
        return PIFU_OK;
    }
    if (!recheck_zeroed) CK(cudaMemsetAsync(ctx->d_recheck, 0, sizeof(unsigned int), s));
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
    // the re-check count joins the statistics in the launch that picks its form
    return g_recheck(ctx, net, s2, rcap, map, cal, e2, s, ctx->d_recheck, rechecked,
                     (unsigned)rcap);
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
    // level 0: every node; the set-up launch also zeroes the frame's
    // statistics, its error word and the re-check queue length
    int N = k.n0, cur = 0;
    static_assert(sizeof(GraphStats) % 4 == 0, "statistics zeroed as words");
    const ZeroSpans zs{{reinterpret_cast<unsigned int*>(gs), err, ctx->d_recheck},
                       {(uint32_t)(sizeof(GraphStats) / 4), 1u, 1u}};
    CK(launch_dense_setup(N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval, ctx->conf[0], s, 1,
                          0, &zs));
    {
        const int64_t nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
        PointSrc src{PTS_DENSE, nullptr, nullptr, 0, N, nullptr};
        Epilogue epi{};
        epi.mode = EPI_LEVEL;
        epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[0], N, row_words_of(N), 1};
        st = g_eval(ctx, net, src, nodes, nullptr, occ, cal, epi, k.precision, k.margin,
                    &gs->rechecked[0], s, k.use_surrogate && k.num_levels > 1, k.sur_margin,
                    &gs->fallback[0], 0, nullptr, true);
        if (st != PIFU_OK) return st;
    }
    for (int l = 1; l < k.num_levels; ++l) {
        const int prev = cur;
        cur ^= 1;
        N *= 2;
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
        // the level's set-up (candidate count and the list count's zeroing in
        // the same launch), then its first selection, whose last CTA decides
        // whether the loop runs
        // (the frontier counts in d_count2: each round's start moves it to
        // d_count, the size its passes read)
        CK(launch_classify(ctx->bin[prev], N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval,
                           ctx->conf[0], s, 1, 0, 0, &gs->cands[l], ctx->d_count2));
        const LoopTail first{h, ctx->d_tail, (unsigned)kChunkTC, &gs->rounds[l], 0, k.max_rounds,
                             err};
        CK(launch_dilate_select(ctx->cand, ctx->eval, nullptr, N, ctx->list, ctx->d_count2, s, 1,
                                0, 0, &first));
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
            // the round's statistics and the zeroing of its conflict count
            // ride in the launch that picks the batch's branch; the expansion's
            // last CTA decides whether another round runs
            const RoundStart rs{&gs->evals[l], (unsigned)kChunkTC, err, ctx->d_ccount,
                                ctx->d_count2};
            st = g_eval(ctx, net, src, kChunkTC, ctx->d_count, occ, cal, epi, k.precision,
                        k.margin, &gs->rechecked[l], sb, k.use_surrogate && l < k.num_levels - 1,
                        k.sur_margin, &gs->fallback[l], 0, &rs);
            const LoopTail next{h, ctx->d_tail + 1, (unsigned)kChunkTC, &gs->rounds[l], 1,
                                k.max_rounds, err};
            if (st == PIFU_OK &&
                launch_expand_conflicts(ctx->clist, ctx->d_ccount, (unsigned)kChunkTC, N, ctx->eval,
                                        0, 0, ctx->list, ctx->d_count2, (unsigned)kChunkTC, err,
                                        sb, nullptr, nullptr, nullptr, nullptr, &next) != cudaSuccess)
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
    if (!ctx->d_tail) {
        // the loop tails' CTA counters [2], then the frontier count
        CK(dev_alloc(&ctx->d_tail, 3));
        CK(cudaMemset(ctx->d_tail, 0, 3 * sizeof(unsigned int)));
        ctx->d_count2 = ctx->d_tail + 2;
    }
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
        int st = ensure_tc_rows(ctx, kChunkTC);
        auto mixed = [](int p) { return p == PIFU_PREC_MIXED || p == PIFU_PREC_FP8_MIXED; };
        if (st == PIFU_OK && (mixed(k.precision) || mixed(k.cam_precision))) st = ensure_x3(ctx);
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


// The validation, the graph (captured when the argument set is new) and its
// launch on `stream` of pifu_frame and pifu_frame_async; *kout: the frame's
// key.  Nothing is enqueued when an argument or a host-known capacity is
// refused.
int frame_enqueue(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
                  const float calib[12], const pifu_levels* lv, const pifu_camera* cam,
                  void* stream, float* depth_dev, float* rgb_dev, uint8_t* mask_dev,
                  FrameKey* kout) {
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
        // frames in flight use the workspaces and the graph being replaced
        if (ctx->async_frames > 0) CK(cudaStreamSynchronize(s));
        st = g_build(ctx, k, to_map(occ_map), to_map(col_map), to_calib(calib));
        if (st != PIFU_OK) return st;
    }
    ctx->have_volume = false;
    CK(cudaGraphLaunch(ctx->gexec, s));
    *kout = k;
    return PIFU_OK;
}

// The volume and counters of the last frame launched with key k (its
// counters in ctx->h_gstats, the graph's last copy), after the stream has
// been synchronised; `frames` frames ran (launch accounting); err: their
// error word (nonzero: the device counters are reset and the error decoded).
int frame_readout(pifu_ctx* ctx, const FrameKey& k, int64_t frames, unsigned int err,
                  cudaStream_t s, pifu_volume* out) {
    const GraphStats& gs = *ctx->h_gstats;
    pifu_volume vs{};
    vs.num_levels = k.num_levels;
    vs.evals_per_level[0] = (int64_t)(k.n0 + 1) * (k.n0 + 1) * (k.n0 + 1);
    vs.n_eval = vs.evals_per_level[0];
    int64_t launches = ctx->g_launches_fixed;
    for (int l = 0; l < k.num_levels; ++l) {
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
    ctx->prof.k[PIFU_K_MLP_HIDDEN].launches += launches * frames;   // graph: counted in one class
    const int cur = (k.num_levels - 1) & 1;
    const int64_t n_fine = (int64_t)k.n0 << (k.num_levels - 1);
    vs.n = (int32_t)n_fine;
    vs.row_words = row_words_of((int)n_fine);
    vs.occ_bits_dev = ctx->bin[cur];
    vs.eval_bits_dev = ctx->eval;
    vs.values_dev = ctx->values;
    if (k.final_level && k.num_levels < kMaxLevels)
        vs.evals_per_level[k.num_levels] = (int64_t)gs.culled;   // the culled final level
    if (out) *out = vs;
    if (err) {
        const int st = reset_after_error(ctx, s);
        return st != PIFU_OK ? st : decode_err(err);
    }
    ctx->stats = vs;
    ctx->have_volume = true;
    ctx->vol_N = (int)n_fine;
    ctx->vol_bin = cur;
    ctx->vol_prec = k.precision;
    ctx->vol_margin = k.margin;
    return PIFU_OK;
}


}  // namespace pifu_host

using namespace pifu_host;

extern "C" {

int pifu_frame(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
               const float calib[12], const pifu_levels* lv, const pifu_camera* cam, void* stream,
               float* depth_dev, float* rgb_dev, uint8_t* mask_dev, pifu_volume* out) {
    if (ctx && ctx->async_frames > 0) return PIFU_ERR_STATE;   // pifu_frame_wait first
    FrameKey k;
    int st = frame_enqueue(ctx, occ_map, col_map, calib, lv, cam, stream, depth_dev, rgb_dev,
                           mask_dev, &k);
    if (st != PIFU_OK) return st;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(s));
    return frame_readout(ctx, k, 1, ctx->h_gstats->err, s, out);
}

int pifu_frame_async(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
                     const float calib[12], const pifu_levels* lv, const pifu_camera* cam,
                     void* stream, float* depth_dev, float* rgb_dev, uint8_t* mask_dev) {
    if (!ctx) return PIFU_ERR_ARG;
    {
        DeviceGuard g(ctx->device);
        if (!g.ok) return PIFU_ERR_CUDA;
        if (!ctx->d_sticky) {
            CK(dev_alloc(&ctx->d_sticky, 1));
            CK(cudaMemset(ctx->d_sticky, 0, sizeof(unsigned int)));
        }
    }
    FrameKey k;
    const int st = frame_enqueue(ctx, occ_map, col_map, calib, lv, cam, stream, depth_dev, rgb_dev,
                                 mask_dev, &k);
    if (st != PIFU_OK) return st;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    CK(launch_latch_err(ctx->d_count + 1, ctx->d_sticky, static_cast<cudaStream_t>(stream)));
    ctx->prof.k[PIFU_K_MLP_HIDDEN].launches += 1;   // counted with the graph's launches
    ctx->async_key = k;
    ++ctx->async_frames;
    return PIFU_OK;
}

int pifu_frame_wait(pifu_ctx* ctx, void* stream, pifu_volume* out) {
    if (!ctx) return PIFU_ERR_ARG;
    if (ctx->async_frames <= 0) return PIFU_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(s));
    unsigned int sticky = 0;
    CK(cudaMemcpy(&sticky, ctx->d_sticky, sizeof(sticky), cudaMemcpyDeviceToHost));
    if (sticky) CK(cudaMemset(ctx->d_sticky, 0, sizeof(unsigned int)));
    const int64_t n = ctx->async_frames;
    ctx->async_frames = 0;
    return frame_readout(ctx, ctx->async_key, n, sticky, s, out);
}

}  // extern "C"
