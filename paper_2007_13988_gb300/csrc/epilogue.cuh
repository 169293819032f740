// The last MLP layer's activation and the destinations of its result,
// shared by the FP32 last-layer kernel and the tensor-core kernel that fuses
// the last layer into its epilogue.
#pragma once

#include "pifu_internal.h"

namespace pifu {

__device__ __forceinline__ float apply_act(int act, float t) {
    if (act == ACT_SIGMOID) return 1.0f / (1.0f + expf(-t));
    return 0.5f * (tanhf(t) + 1.0f);
}


// The epilogue of one point: activation and where the result goes (for
// EPI_LEVEL the occupancy, its binarized bit and the conflict test of
// Sec. 3.2; with a re-check queue, occupancies near 0.5 are queued instead).
__device__ __forceinline__ void last_epilogue(const Epilogue& epi, int64_t p, int n_out,
                                              const float (&t)[4], const float* __restrict__ bias) {
    if (epi.recheck) {
        // mixed precision: defer occupancies close to the decision threshold
        const float o = apply_act(ACT_SIGMOID, t[0] + bias[0]);
        if (fabsf(o - kHalf) < epi.margin) {
            const unsigned pos = atomicAdd(epi.recheck_count, 1u);
            epi.recheck[pos] = (epi.mode == EPI_LEVEL || epi.mode == EPI_COLUMN)
                                   ? (epi.list ? epi.list[p] : (int)(epi.base + p))
                                   : (epi.pix ? epi.pix[p] : (int)p);
            return;
        }
    }
    if (epi.mode == EPI_STORE) {
        const int64_t q = epi.pix ? (int64_t)epi.pix[p] : p;
        for (int j = 0; j < n_out; ++j) epi.out[q * n_out + j] = apply_act(epi.act, t[j] + bias[j]);
    } else if (epi.mode == EPI_COLUMN) {
        epi.out[epi.list ? (int64_t)epi.list[p] : epi.base + p] =
            apply_act(ACT_SIGMOID, t[0] + bias[0]);
    } else if (epi.mode == EPI_PIXELS) {
        const int64_t pix = epi.pix[p];
        for (int j = 0; j < n_out; ++j) epi.out[pix * 3 + j] = apply_act(epi.act, t[j] + bias[j]);
    } else {
        // Occupancy scattered into a localization level (Sec. 3.2): store the
        // value, set the binarized bit, and flag a conflict when the
        // binarized prediction differs from the binarized interpolation.
        const float o = apply_act(ACT_SIGMOID, t[0] + bias[0]);
        int64_t idx = epi.list ? (int64_t)epi.list[p] : epi.base + p;
        const int key = (int)idx;
        const LevelBits& lv = epi.lv;
        float* values = lv.values;
        const uint32_t* tent = lv.tent;
        uint32_t* bin = lv.bin;
        uint32_t* conf = lv.conf;
        int N = lv.N, row_words = lv.row_words, first_level = lv.first_level;
        if (lv.key_div) {   // several frames: key = frame * key_div + node
            const int64_t f = idx / lv.key_div;
            idx -= f * lv.key_div;
            if (lv.sv) {    // frame stream: the slot's arrays and level
                const SlotView& v = lv.sv[f];
                values = v.values;
                tent = v.tent;
                bin = v.bin;
                conf = v.conf;
                N = v.N;
                row_words = row_words_of(N);
                first_level = v.first_level;
            } else {
                values += f * lv.slot_nodes;
                tent += f * lv.slot_words;
                bin += f * lv.slot_words;
                conf += f * lv.slot_words;
            }
        }
        values[idx] = o;
        const int64_t n1 = N + 1;
        const int64_t row = idx / n1;            // k (N+1) + j
        const int i = (int)(idx - row * n1);
        const int64_t w = row * row_words + (i >> 5);
        const uint32_t bit = 1u << (i & 31);
        const bool ob = o >= kHalf;
        if (first_level) {
            if (ob) atomicOr(&bin[w], bit);
        } else {
            const bool tb = (tent[w] & bit) != 0u;
            if (ob != tb) {
                atomicOr(&conf[w], bit);
                if (ob) atomicOr(&bin[w], bit);
                else atomicAnd(&bin[w], ~bit);
                if (lv.clist) {
                    const unsigned int pos = atomicAdd(lv.ccount, 1u);
                    if (pos < lv.ccap) lv.clist[pos] = key;
                    else atomicOr(lv.err, kErrCapacity);
                }
            }
        }
    }
}

}  // namespace pifu
