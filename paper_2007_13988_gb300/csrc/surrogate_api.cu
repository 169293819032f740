// The learned surrogate f_S (not in the paper): its parameters, training and point OHEM, and their C entry points.
#include "host.h"

namespace pifu_host {


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
    n.ldx_tc = fo.ldx_tc;
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
             float* per_loss) {
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


}  // namespace pifu_host

using namespace pifu_host;

extern "C" {

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

}  // extern "C"
