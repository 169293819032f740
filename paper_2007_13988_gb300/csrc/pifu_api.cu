// C ABI of libpifu: context creation and destruction, queries, the host-driven
// localization loop and render, FP8 calibration and the profiler (include/pifu.h).
#include "host.h"

using namespace pifu_host;

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
    if (st == PIFU_OK && !cbn) st = build_x3(ctx, hn[0], ctx->net[0]);
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
    // frames from pifu_frame_async may still run on the context's buffers
    if (ctx->async_frames > 0) (void)cudaDeviceSynchronize();
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
    dev_free(ctx->chain_dep);
    dev_free(ctx->part);
    dev_free(ctx->X3);
    dev_free(ctx->H3[0]);
    dev_free(ctx->H3[1]);
    dev_free(ctx->x3_part);
    dev_free(ctx->x3_ctr);
    dev_free(ctx->grid_H[0]);
    dev_free(ctx->grid_H[1]);
    dev_free(ctx->grid_part);
    dev_free(ctx->grid_ctr);
    dev_free(ctx->d_tail);
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
    dev_free(ctx->d_sticky);
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
    if (st == PIFU_OK && subdiv == PIFU_SUBDIV_METHOD) st = ensure_clist(ctx, kChunkTC);
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
            // the level's set-up; the candidates are counted in the same launch
            ev = ctx->prof.begin(s);
            CK(launch_classify(ctx->bin[prev], N, ctx->cand, ctx->tent, ctx->bin[cur], ctx->eval,
                               ctx->conf[0], s, 1, 0, 0, ctx->d_pop + l, nullptr));
            ctx->prof.end(PIFU_K_LEVEL, ev, s, 0.0, 4.0 * words_of(N / 2) + 5.0 * wbytes);
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
        const int64_t level_nodes = (int64_t)(N + 1) * (N + 1) * (N + 1);
        while (n > 0) {
            // The round's conflicts also go to a key list when it can hold
            // them all (at most n): the next frontier, their unevaluated
            // 26-neighbours, is then found in work proportional to them.
            // Otherwise the conflict bitset conf[q] is dilated over the whole
            // grid (stale bits of earlier list rounds add nothing: their
            // neighbours are evaluated).
            const bool sparse = (int64_t)n <= ctx->clist_cap;
            epi.lv = LevelBits{ctx->values, ctx->tent, ctx->bin[cur], ctx->conf[q], N, rw, 0};
            if (sparse) {
                epi.lv.clist = ctx->clist;
                epi.lv.ccount = ctx->d_ccount;
                epi.lv.ccap = (unsigned)ctx->clist_cap;
                epi.lv.err = ctx->d_count + 1;
                CK(cudaMemsetAsync(ctx->d_ccount, 0, sizeof(unsigned int), s));
            }
            st = eval_level_batch(ctx, src, n, map, cal, epi, prec, lv->margin,
                                  use_sur && l < lv->num_levels - 1, lv->surrogate_margin, s,
                                  &vs.rechecked_per_level[l], &vs.fallback_per_level[l]);
            if (st != PIFU_OK) return st;
            level_evals += n;
            // unevaluated 1-ring of this evaluation's conflicts
            CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned int), s));
            ev = ctx->prof.begin(s);
            if (sparse)
                CK(launch_expand_conflicts(ctx->clist, ctx->d_ccount, n, N, ctx->eval, 0, 0,
                                           ctx->list, ctx->d_count, (unsigned)level_nodes,
                                           ctx->d_count + 1, s));
            else
                CK(launch_dilate_select(ctx->conf[q], ctx->eval, ctx->conf[1 - q], N, ctx->list,
                                        ctx->d_count, s));
            // the list expansion reads a few bytes per conflict, counted
            // with the list it writes (below)
            ctx->prof.end(PIFU_K_SELECT, ev, s, 0.0, sparse ? 0.0 : 4.0 * wbytes);
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
