// The MLP over a point batch: FP32, tensor-core and mixed-precision passes, and one evaluation batch of a localization level.
#include "host.h"

namespace pifu_host {

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
               cudaStream_t s, const unsigned int* m_dev, bool f8) {
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
        CK(launch_gather_bf16(src, p0, mc, calib, map0, map1, ctx->Xb, net.ldx_tc, s));
        pr.end(PIFU_K_GATHER, ev, s, 0.0,
               (double)mc * (4.0 * 4.0 * (map0.C + map1.C) + 2.0 * net.ldx_tc));
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
                C.klast = T.klast;
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
            a.klast = T.klast;
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
                // the FP8 form (Fp8Layer): layer 0 BF16 in, E4M3 out; later
                // layers E4M3 h and BF16 x into one accumulator, E4M3 out but
                // for the last, which hands BF16 to the next layer
                const Fp8Layer& Q = net.f8[(size_t)l];
                a.tmA1 = l > 0 ? &Q.tmA1 : &net.tmX;
                a.tmA2 = &net.tmX;
                a.tmW = &Q.tmW;
                a.nk1 = Q.nk1;
                a.nk2 = Q.nk2;
                a.klast = Q.klast;
                a.BN = Q.BN;
                a.pair = 0;
                a.mode = l == 0 ? TC_BF16_E4M3 : (l + 1 < F ? TC_MIX_E4M3 : TC_MIX_BF16);
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
            CK(launch_last_layer_bf16(p0, mc, Ll.n_out, h, hw, Ll.K1, ctx->Xb, net.ldx_tc, Ll.K2,
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
            int precision, const unsigned int* m_dev,
            int fused_cl) {
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

// ---- the FP32-accurate pass on the tensor cores (split TF32, mlp_x3.cu) -------

bool x3_usable(const pifu_ctx* ctx, const DevNet& net) {
    return net.x3_ok && ctx->x3_ready && ctx->recheck_form != PIFU_RECHECK_SIMT;
}

int64_t x3_min_rows(const pifu_ctx* ctx) {
    return ctx->recheck_form == PIFU_RECHECK_TENSOR_ALL ? 0 : kX3MinRows;
}

// The whole network (gather into hi/lo planes, every hidden layer, the last
// layer and the epilogue) in one cooperative launch per pass of at most
// kX3Rows points (a device-sized batch is one pass of at most m <= kX3Rows).
int run_mlp_x3(pifu_ctx* ctx, const DevNet& net, const PointSrc& src_in, int64_t m,
               const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
               cudaStream_t s, const unsigned int* m_dev) {
    if (!x3_usable(ctx, net)) return PIFU_ERR_UNSUPPORTED;
    if (m_dev && m > kX3Rows) return PIFU_ERR_ARG;
    const int L = (int)net.layers.size();
    if (L - 1 > kX3MaxLayers) return PIFU_ERR_UNSUPPORTED;
    const DevLayer& Ll = net.layers[(size_t)L - 1];
    Profiler& pr = ctx->prof;
    for (int64_t p0 = 0; p0 < m; p0 += kX3Rows) {
        const int64_t mc = std::min<int64_t>(kX3Rows, m - p0);
        X3NetArgs a{};
        double flops = 2.0 * mc * Ll.fan_in * Ll.n_out, bytes = 0.0;
        for (int l = 0; l + 1 < L; ++l) {
            const DevLayer& Ly = net.layers[(size_t)l];
            const X3Layer& X = net.x3[(size_t)l];
            X3NetLayer& A = a.L[l];
            A.tmW = X.tmW;
            if (l > 0) A.tmH = X.tmH;
            A.nk1 = X.KH / 32;
            A.nk2 = X.KX / 32;
            A.KH = X.KH;
            A.KX = X.KX;
            A.KP = X.KP;
            A.N = Ly.n_out;
            A.bias = Ly.b;
            A.out = l + 2 < L ? ctx->H3[l % 2] : nullptr;
            flops += 3.0 * 2.0 * mc * Ly.fan_in * Ly.n_out;
            bytes += 8.0 * ((double)mc * (X.KP + Ly.n_out) + (double)Ly.n_out * X.KP);
        }
        a.tmX = net.tmX3;
        a.nl = L - 1;
        a.M = (int)mc;
        a.m_dev = m_dev;
        a.slope = net.slope;
        a.src = src_in;
        a.src.count = nullptr;   // the count is m_dev, read by the kernel
        a.p0 = p0;
        a.calib = calib;
        a.map0 = map0;
        a.map1 = map1;
        a.X = ctx->X3;
        a.KX = net.x3_KX;
        a.fl.W = Ll.W;
        a.fl.ldw = Ll.ldw;
        a.fl.bias = Ll.b;
        a.fl.n_out = Ll.n_out;
        a.fl.p0 = p0;
        a.fl.epi = epi;
        a.part = ctx->x3_part;
        a.ctr = ctx->x3_ctr;
        a.err = ctx->d_count + 1;
        a.wait_extra = ctx->x3_starve;
        cudaEvent_t ev = pr.begin(s);
        CK(launch_x3_net(a, s));
        pr.end(PIFU_K_MLP_F32, ev, s, flops,
               bytes + (double)mc * (4.0 * 4.0 * (map0.C + map1.C) + 8.0 * net.x3_KX));
    }
    return PIFU_OK;
}

// ---- the FP32 pass over the whole GPU (mlp_grid.cu) -------------------------------

int64_t grid_rows(const pifu_ctx* ctx, const DevNet& net) {
    if (ctx->recheck_form != PIFU_RECHECK_TENSOR || !ctx->grid_ctr) return 0;
    return std::min<int64_t>(net.grid_rows, kGridPreferRows);
}

// The whole network (input rows, every hidden layer, the last layer and the
// epilogue) in one cooperative launch of one CTA per SM, for m <= grid_rows
// points (a device-sized batch: at most m of them).
int run_mlp_grid(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                 const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                 cudaStream_t s, const unsigned int* m_dev) {
    if (m <= 0) return PIFU_OK;
    if (m > net.grid_rows || !ctx->grid_ctr) return PIFU_ERR_UNSUPPORTED;
    GridArgs a{};
    a.net = fused_of(net);
    a.src = src;
    a.src.count = nullptr;   // the count is m_dev, read by the kernel
    a.p0 = 0;
    a.M = (int)m;
    a.m_dev = m_dev;
    a.calib = calib;
    a.map0 = map0;
    a.map1 = map1;
    a.epi = epi;
    a.H[0] = ctx->grid_H[0];
    a.H[1] = ctx->grid_H[1];
    a.part = ctx->grid_part;
    a.ctr = ctx->grid_ctr;
    a.err = ctx->d_count + 1;
    a.wait_extra = ctx->x3_starve;
    double flops = 0.0, wbytes = 0.0;
    for (const DevLayer& Ly : net.layers) {
        flops += 2.0 * (double)m * Ly.fan_in * Ly.n_out;
        wbytes += 4.0 * (double)Ly.n_out * (Ly.fan_in + 1);
    }
    cudaEvent_t ev = ctx->prof.begin(s);
    CK(launch_mlp_grid(a, s));
    ctx->prof.end(PIFU_K_MLP_F32, ev, s, flops,
                  wbytes + (double)m * 4.0 * (4.0 * (map0.C + map1.C) + net.layers.back().n_out));
    return PIFU_OK;
}

int run_recheck(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                cudaStream_t s) {
    if (m <= grid_rows(ctx, net))
        return run_mlp_grid(ctx, net, src, m, map0, map1, calib, epi, s, nullptr);
    if (m > x3_min_rows(ctx) && x3_usable(ctx, net))
        return run_mlp_x3(ctx, net, src, m, map0, map1, calib, epi, s, nullptr);
    return run_mlp(ctx, net, src, m, map0, map1, calib, epi, s, PIFU_PREC_FP32);
}

// Mixed precision over one batch: the tensor-core BF16 pass commits every
// occupancy farther than `margin` from 0.5 and queues the others (node
// indices for a level, point numbers otherwise) on ctx->recheck; the queued
// ones are then evaluated again in FP32 and committed.  One host read of the
// queue length per batch.  *rechecked += the queue length.
int read_recheck(pifu_ctx* ctx, cudaStream_t s, unsigned int* out);

int run_mlp_mixed(pifu_ctx* ctx, const DevNet& net, const PointSrc& src, int64_t m,
                  const Map& map0, const Map& map1, const Calib& calib, const Epilogue& epi,
                  float margin, cudaStream_t s, int64_t* rechecked, bool f8) {
    if (m > ctx->recheck_cap) return PIFU_ERR_ARG;
    {
        const int st = ensure_x3(ctx);
        if (st != PIFU_OK) return st;
    }
    // A tiny batch costs less in FP32 outright than in BF16 plus a re-check
    // pass (both are latency-bound there); FP32 is the re-check's arithmetic.
    if (m <= kTinyBatch) return run_recheck(ctx, net, src, m, map0, map1, calib, epi, s);
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
    return run_recheck(ctx, net, s2, n, map0, map1, calib, e2, s);
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
        invalidate_graphs(ctx);
        dev_free(ctx->cull_list);
        ctx->cull_cap = 0;
        CK(dev_alloc(&ctx->cull_list, cap));
        ctx->cull_cap = cap;
    }
    if (vals > ctx->cull_vals_cap) {
        invalidate_graphs(ctx);
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
        invalidate_graphs(ctx);
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
        const int st = reset_after_error(ctx, s);
        return st != PIFU_OK ? st : decode_err(e);
    }
    return PIFU_OK;
}

int reset_after_error(pifu_ctx* ctx, cudaStream_t s) {
    CK(cudaMemsetAsync(ctx->d_count + 1, 0, sizeof(unsigned int), s));
    if (ctx->x3_ctr)
        CK(cudaMemsetAsync(ctx->x3_ctr, 0, sizeof(unsigned int) * kX3CtrWords, s));
    if (ctx->grid_ctr)
        CK(cudaMemsetAsync(ctx->grid_ctr, 0, sizeof(unsigned int) * kGridCtrWords, s));
    if (ctx->d_tail) CK(cudaMemsetAsync(ctx->d_tail, 0, 2 * sizeof(unsigned int), s));
    return PIFU_OK;
}


}  // namespace pifu_host
