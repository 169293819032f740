// Tile autotuner, tile codes and the layer schedule.
#include "host.h"

namespace pifu_host {

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
                const int F = (int)net.f8.size();
                a.tmA1 = l > 0 ? &Q.tmA1 : &net.tmX;
                a.tmA2 = &net.tmX;
                a.nk1 = Q.nk1;
                a.nk2 = Q.nk2;
                a.klast = Q.klast;
                a.mode = l == 0 ? TC_BF16_E4M3 : (l + 1 < F ? TC_MIX_E4M3 : TC_MIX_BF16);
                a.colscale = Q.colscale;
                a.out_scale = Q.out_scale;
                double ms = 0.0;
                st = tune_layer(ctx, a, Ly.n_out, !Q.bf16_in, false, &Q.tmW,
                                const_cast<void*>(Q.Wmap), Q.Kw, &Q.BN, s, &ms);
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
            a.klast = T.klast;
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
    ctx->stream.g_valid = false;
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
            ok = ok && encode_w(!q->bf16_in, &q->tmW, const_cast<void*>(q->Wmap), q->Kw, n_out,
                                c);
        } else {
            t->pair = c == kPairCode;
            t->BN = t->pair ? 256 : c;
            ok = ok && encode_w(false, &t->tmW, t->W, t->Kw, n_out, c);
        }
    });
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    ctx->stream.g_valid = false;
    return ok ? PIFU_OK : PIFU_ERR_CUDA;
}


}  // namespace pifu_host

using namespace pifu_host;

extern "C" {

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
    ctx->stream.g_valid = false;
    return PIFU_OK;
}

int pifu_set_recheck(pifu_ctx* ctx, int form) {
    if (!ctx || (form != PIFU_RECHECK_TENSOR && form != PIFU_RECHECK_SIMT &&
                 form != PIFU_RECHECK_TENSOR_ALL))
        return PIFU_ERR_ARG;
    ctx->recheck_form = form;
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    ctx->stream.g_valid = false;
    return PIFU_OK;
}

int pifu_test_starve_wait(pifu_ctx* ctx, int starve) {
    if (!ctx || (starve != 0 && starve != 1)) return PIFU_ERR_ARG;
    ctx->x3_starve = (unsigned int)starve;
    ctx->g_valid = false;
    ctx->batch.g_valid = false;
    ctx->stream.g_valid = false;
    return PIFU_OK;
}

int pifu_set_tiles(pifu_ctx* ctx, const int32_t* codes, int n) {
    if (!ctx || n < 0 || (n > 0 && !codes)) return PIFU_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PIFU_ERR_CUDA;
    return set_tiles(ctx, codes, n);
}

}  // extern "C"
