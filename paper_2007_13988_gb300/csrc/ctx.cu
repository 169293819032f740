// Weight-blob parsing, upload of the networks and the context's device workspaces.
#include "host.h"

namespace pifu_host {

// ---- weight blob ------------------------------------------------------------

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
    net.ldx_tc = round_up((int)d_in, 64);
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
    net.ldx_tc = round_up(h.C + 1, 64);
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
    for (auto& X : net.x3) dev_free(X.W);
    free_f8(net);
    net.layers.clear();
    net.tc.clear();
    net.x3.clear();
    net.x3_ok = false;
}

// ---- workspaces -------------------------------------------------------------

int ensure_mlp_ws(pifu_ctx* ctx) {
    int64_t need_x = 0, need_h = 0;
    for (const DevNet& n : ctx->net) {
        need_x = std::max<int64_t>(need_x, n.ldx);
        need_h = std::max<int64_t>(need_h, std::max(n.max_hidden, 8));
    }
    if (need_x > ctx->X_cap) {   // per-point widths; FP32 rows are kChunk points
        invalidate_graphs(ctx);
        dev_free(ctx->X);
        CK(dev_alloc(&ctx->X, need_x * kChunk));
        ctx->X_cap = need_x;
    }
    if (need_h > ctx->H_cap) {
        invalidate_graphs(ctx);
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
        invalidate_graphs(ctx);
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
    if (!tc_encode_2d_bf16(&net.tmX, ctx->Xb, (uint64_t)net.ldx_tc, rows,
                           (uint64_t)net.ldx_tc * 2, 64, 128))
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
        need_x = std::max<int64_t>(need_x, std::max(n.ldx, n.ldx_tc));
        need_h = std::max<int64_t>(need_h, std::max(n.max_hidden, 8));
    }
    invalidate_graphs(ctx);
    dev_free(ctx->Xb);
    dev_free(ctx->Hb[0]);
    dev_free(ctx->Hb[1]);
    dev_free(ctx->chain_dep);
    ctx->tc_rows = 0;
    CK(dev_alloc(&ctx->chain_dep, (int64_t)kChainMaxLayers * (cap / 128) + 2));
    CK(cudaMemset(ctx->chain_dep, 0, sizeof(unsigned int) * ((size_t)kChainMaxLayers * (cap / 128) + 2)));
    CK(dev_alloc(&ctx->Xb, need_x * cap));
    CK(dev_alloc(&ctx->Hb[0], need_h * cap));
    CK(dev_alloc(&ctx->Hb[1], need_h * cap));
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
        // the last K-block's MMA steps past d_in (zeros on both sides) are skipped
        T.klast = has_x ? (net.d_in - 64 * (T.nk2 - 1) + 15) / 16 : 4;
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

// ---- split-TF32 form (FP32-accurate passes on the tensor cores) -------------

// Weights of the split-TF32 layers: per hidden layer [n_out][2 KP], the TF32
// value hi = tf32(w) of every weight in columns [0, KP) and lo = tf32(w - hi)
// in [KP, 2 KP), the h part first, then the x part zero-padded to KX.  Nets
// of other shapes (hidden widths not multiples of 128, a last hidden layer
// other than 128 wide, a last layer of more than one output or reading x)
// keep x3_ok = false: their FP32 passes use the SIMT kernels.
int build_x3(pifu_ctx* ctx, const HostNet& hn, DevNet& net) {
    (void)ctx;
    net.x3_ok = false;
    const int L = (int)net.layers.size();
    if (net.kind == kNetCbn || L < 2) return PIFU_OK;
    for (int l = 0; l + 1 < L; ++l) {
        const DevLayer& Ly = net.layers[(size_t)l];
        if (Ly.n_out % kX3Tile != 0 || (l == 0) != (Ly.K1 == 0)) return PIFU_OK;
    }
    const DevLayer& Ll = net.layers[(size_t)L - 1];
    if (net.layers[(size_t)L - 2].n_out != kX3Tile || Ll.K2 != 0 || Ll.n_out != 1) return PIFU_OK;
    const int KX = round_up(net.d_in, 32);
    net.x3.assign((size_t)L - 1, X3Layer{});
    for (int l = 0; l + 1 < L; ++l) {
        const DevLayer& Ly = net.layers[(size_t)l];
        X3Layer& X = net.x3[(size_t)l];
        X.KH = Ly.K1;
        X.KX = Ly.K2 > 0 ? KX : 0;
        X.KP = X.KH + X.KX;
        if (X.KP == 0) return PIFU_OK;
        const size_t row = 2 * (size_t)X.KP;
        std::vector<float> w((size_t)Ly.n_out * row, 0.f);
        const std::vector<float>& wf = hn.W[(size_t)l];   // [n_out][K1 | ldx]
        for (int o = 0; o < Ly.n_out; ++o) {
            auto put = [&](int k, float v) {
                const float hi = tf32_round(v);
                w[(size_t)o * row + (size_t)k] = hi;
                w[(size_t)o * row + (size_t)X.KP + (size_t)k] = tf32_round(v - hi);
            };
            for (int k = 0; k < Ly.K1; ++k) put(k, wf[(size_t)o * Ly.ldw + k]);
            if (Ly.K2 > 0)
                for (int k = 0; k < net.d_in; ++k) put(X.KH + k, wf[(size_t)o * Ly.ldw + Ly.K1 + k]);
        }
        CK(dev_alloc(&X.W, (int64_t)w.size()));
        CK(cudaMemcpy(X.W, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice));
        if (!x3_encode_2d(&X.tmW, X.W, row, (uint64_t)Ly.n_out, row * 4, 32, 128))
            return PIFU_ERR_CUDA;
    }
    net.x3_KX = KX;
    net.x3_ok = true;
    return PIFU_OK;
}

// The split-TF32 workspaces (kX3Rows points) and the tensor maps over them,
// once per context.  Called before any capture (a graph holds the maps).
// The whole-GPU FP32 network's buffers, and each concatenation network's
// largest batch for it.
int ensure_grid(pifu_ctx* ctx) {
    if (ctx->grid_ctr) return PIFU_OK;
    int64_t h = 0;
    for (DevNet& n : ctx->net) {
        n.grid_rows = n.kind == kNetCbn ? 0 : grid_max_rows(fused_of(n));
        if (n.grid_rows > 0) h = std::max<int64_t>(h, n.max_hidden);
    }
    if (h == 0) return PIFU_OK;
    CK(dev_alloc(&ctx->grid_H[0], kGridMaxRows * h));
    CK(dev_alloc(&ctx->grid_H[1], kGridMaxRows * h));
    CK(dev_alloc(&ctx->grid_part, (int64_t)kGridMaxRows * kGridMaxCtas * 4));
    CK(dev_alloc(&ctx->grid_ctr, (int64_t)kGridCtrWords));
    CK(cudaMemset(ctx->grid_ctr, 0, sizeof(unsigned int) * kGridCtrWords));
    return PIFU_OK;
}

// The FP32-accurate passes' workspaces: the whole-GPU FP32 network's and the
// split-TF32 network's.
int ensure_x3(pifu_ctx* ctx) {
    const int st = ensure_grid(ctx);
    if (st != PIFU_OK) return st;
    if (ctx->x3_ready) return PIFU_OK;
    int64_t kx = 0, h = 0;
    for (const DevNet& n : ctx->net) {
        if (!n.x3_ok) continue;
        kx = std::max<int64_t>(kx, n.x3_KX);
        for (size_t l = 0; l + 1 < n.layers.size(); ++l) h = std::max<int64_t>(h, n.layers[l].n_out);
    }
    if (kx == 0) return PIFU_OK;
    CK(x3_prepare());
    CK(dev_alloc(&ctx->X3, kX3Rows * 2 * kx));
    CK(dev_alloc(&ctx->H3[0], kX3Rows * 2 * h));
    CK(dev_alloc(&ctx->H3[1], kX3Rows * 2 * h));
    CK(dev_alloc(&ctx->x3_part, (int64_t)kX3MaxUnits * kX3Tile * kX3Tile));
    // tile counters [2][kX3MaxUnits], then the grid barrier's words
    CK(dev_alloc(&ctx->x3_ctr, (int64_t)kX3CtrWords));
    CK(cudaMemset(ctx->x3_ctr, 0, sizeof(unsigned int) * kX3CtrWords));
    for (DevNet& n : ctx->net) {
        if (!n.x3_ok) continue;
        const uint64_t rx = 2 * (uint64_t)n.x3_KX;
        if (!x3_encode_2d(&n.tmX3, ctx->X3, rx, (uint64_t)kX3Rows, rx * 4, 32, 32))
            return PIFU_ERR_CUDA;
        for (size_t l = 1; l < n.x3.size(); ++l) {
            const uint64_t rh = 2 * (uint64_t)n.x3[l].KH;
            if (!x3_encode_2d(&n.x3[l].tmH, ctx->H3[(l - 1) % 2], rh, (uint64_t)kX3Rows, rh * 4, 32,
                              32))
                return PIFU_ERR_CUDA;
        }
    }
    ctx->x3_ready = true;
    return PIFU_OK;
}

// ---- FP8 form of f_O ----------------------------------------------------------

uint8_t e4m3_byte(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// The FP8 layers 0 .. F-1 of `net` (F >= 2; Fp8Layer), from its FP32 and
// BF16 weights and the activation scales s_h[l] of h_l, l < F-1.
int build_fp8(pifu_ctx* ctx, DevNet& net, int F, const std::vector<float>& s_h) {
    free_f8(net);
    net.f8.assign((size_t)F, Fp8Layer{});
    for (int l = 0; l < F; ++l) {
        const DevLayer& Ly = net.layers[(size_t)l];
        const TcLayer& T = net.tc[(size_t)l];
        Fp8Layer& Q = net.f8[(size_t)l];
        Q.BN = T.BN;
        Q.out_scale = l + 1 < F ? 1.f / s_h[(size_t)l] : 1.f;
        Q.nk2 = T.nk2;
        Q.klast = T.klast;
        if (l == 0) {
            // the BF16 operands of the tensor-core form, its own tile map
            Q.bf16_in = true;
            Q.nk1 = T.nk1;
            Q.Kw = T.Kw;
            Q.Wmap = T.W;
            if (!tc_encode_2d_bf16(&Q.tmW, T.W, (uint64_t)T.Kw, (uint64_t)Ly.n_out,
                                   (uint64_t)T.Kw * 2, 64, (uint32_t)Q.BN))
                return PIFU_ERR_CUDA;
            continue;
        }
        const bool has_x = Ly.K2 > 0;
        Q.nk1 = Ly.K1 / 128;
        Q.Kw = Ly.K1 + Q.nk2 * 128;   // bytes
        const float s_a = s_h[(size_t)l - 1];
        std::vector<float> wf((size_t)Ly.n_out * Ly.ldw);
        CK(cudaMemcpy(wf.data(), Ly.W, wf.size() * 4, cudaMemcpyDeviceToHost));
        std::vector<uint8_t> w8((size_t)Ly.n_out * Q.Kw, 0);
        std::vector<float> cs((size_t)Ly.n_out);
        for (int o = 0; o < Ly.n_out; ++o) {
            const float* row = &wf[(size_t)o * Ly.ldw];
            float amax = 0.f;
            for (int k = 0; k < Ly.K1; ++k) amax = std::max(amax, std::fabs(row[k]));
            const float sw = amax > 0.f ? amax / 448.f : 1.f;
            uint8_t* dst = &w8[(size_t)o * Q.Kw];
            for (int k = 0; k < Ly.K1; ++k) dst[k] = e4m3_byte(row[k] / sw);
            if (has_x)
                for (int k = 0; k < net.d_in; ++k) {
                    const __nv_bfloat16 v = __float2bfloat16(row[Ly.K1 + k] / (s_a * sw));
                    std::memcpy(dst + Ly.K1 + 2 * k, &v, 2);
                }
            cs[(size_t)o] = sw * s_a;
        }
        CK(dev_alloc(&Q.W, (int64_t)w8.size()));
        CK(dev_alloc(&Q.colscale, (int64_t)cs.size()));
        CK(cudaMemcpy(Q.W, w8.data(), w8.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(Q.colscale, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice));
        Q.Wmap = Q.W;
        if (!tc_encode_2d_u8(&Q.tmW, Q.W, (uint64_t)Q.Kw, (uint64_t)Ly.n_out, (uint64_t)Q.Kw, 128,
                             (uint32_t)Q.BN))
            return PIFU_ERR_CUDA;
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
    if (F < 2) return PIFU_ERR_UNSUPPORTED;   // a first layer and one that reads it in E4M3
    int st0 = ensure_tc_rows(ctx, 1);
    if (st0 != PIFU_OK) return st0;
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
    invalidate_graphs(ctx);
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
    invalidate_graphs(ctx);
    dev_free(ctx->prev_values);
    ctx->prev_cap = 0;
    CK(dev_alloc(&ctx->prev_values, n));
    ctx->prev_cap = n;
    return PIFU_OK;
}

int ensure_hit_ws(pifu_ctx* ctx, int64_t npix) {
    if (npix <= ctx->hit_cap) return PIFU_OK;
    invalidate_graphs(ctx);
    dev_free(ctx->hit_xyz);
    dev_free(ctx->hit_pix);
    ctx->hit_cap = 0;
    CK(dev_alloc(&ctx->hit_xyz, 3 * npix));
    CK(dev_alloc(&ctx->hit_pix, npix));
    ctx->hit_cap = npix;
    return PIFU_OK;
}

// ---- argument checks ----------------------------------------------------------


}  // namespace pifu_host
