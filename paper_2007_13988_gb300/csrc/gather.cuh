// Device-side projection and bilinear sampling of the MLP input row
// (Eq. 1 / Eq. 2, Sec. 3.1), shared by the gather kernels and the fused FP32
// MLP kernel so that both assemble bit-identical rows.
//
// Precision: the texel coordinate s = u W/2 + (W-1)/2 has magnitude up to
// W, so computing it in float32 and taking s - floor(s) would leave the
// bilinear weight with an absolute error of ~ulp(W) (4e-6 at W = 128), which
// a steep occupancy logit turns into a visible occupancy error.  Instead the
// projection u = C [P, 1] is evaluated as an unevaluated float-float sum
// (error-free products and sums) and the weight is formed directly as
// fma(u_hi, W/2, (W-1)/2 - floor(s)) + u_lo W/2, whose only rounding is at
// the weight's own magnitude (< 1).
#pragma once

#include "pifu_internal.h"

namespace pifu {

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// c0 x + c1 y + c2 z + c3 as hi + lo (|lo| <= ulp(hi) / 2 up to O(eps^2)).
__device__ __forceinline__ void affine_ff(const float* c, float x, float y, float z,
                                          float& hi, float& lo) {
    float s = c[3], err = 0.f, p, e, t;
    two_prod(c[0], x, p, e); two_sum(s, p, s, t); err = __fadd_rn(err, __fadd_rn(e, t));
    two_prod(c[1], y, p, e); two_sum(s, p, s, t); err = __fadd_rn(err, __fadd_rn(e, t));
    two_prod(c[2], z, p, e); two_sum(s, p, s, t); err = __fadd_rn(err, __fadd_rn(e, t));
    hi = __fadd_rn(s, err);
    lo = __fsub_rn(err, __fsub_rn(hi, s));
}

// Texel coordinate s = u W/2 + (W-1)/2 of u = hi + lo: integer part i0 and
// fractional weight a (accurate to ~1e-7 absolute; may leave [0, 1) by that
// much when s is within rounding of an integer, which keeps the sample
// continuous).
__device__ __forceinline__ void texel_coord(float hi, float lo, int W, int& i0, float& a) {
    const float hw = 0.5f * (float)W;
    const float off = hw - 0.5f;
    const float sl = __fmul_rn(lo, hw);
    const float s = __fmaf_rn(hi, hw, off);
    const float fl = floorf(__fadd_rn(s, sl));
    a = __fadd_rn(__fmaf_rn(hi, hw, __fsub_rn(off, fl)), sl);
    i0 = (int)fmaxf(fminf(fl, (float)W + 1.f), -2.f);   // NaN -> W + 1 (clamped below)
}

__device__ __forceinline__ float4 ld4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

// Position of point p; returns its frame (0 unless the source spans frames).
// Node indices and keys are below 2^31 (int32 lists; (N + 1)^3 <= 513^3), so
// they are decoded with 32-bit unsigned divisions.
__device__ __forceinline__ int point_xyz(const PointSrc& src, int64_t p, float& x, float& y,
                                         float& z) {
    if (src.mode == PTS_XYZ || src.mode == PTS_XYZ_IDX) {
        const int64_t q = src.mode == PTS_XYZ ? p : (int64_t)src.list[p];
        x = src.xyz[3 * q + 0];
        y = src.xyz[3 * q + 1];
        z = src.xyz[3 * q + 2];
        return src.maps0 ? (int)((uint32_t)src.keys[p] / (uint32_t)src.slot_div) : 0;
    }
    if (src.mode == PTS_COLUMN) {
        // key = pixel (N + 1) + k; pixel centre (2i+1)/width - 1, depth 1 - 2k/N
        const uint32_t key = (uint32_t)src.list[p];
        const uint32_t n1 = (uint32_t)src.N + 1u;
        const uint32_t pix = key / n1;
        const int k = (int)(key - pix * n1);
        const uint32_t wd = (uint32_t)src.width;
        const int j = (int)(pix / wd);
        const int i = (int)(pix - (uint32_t)j * wd);
        const float inv = 1.0f / (float)src.width;   // exact for power-of-two widths
        x = __fmaf_rn((float)(2 * i + 1), inv, -1.0f);
        y = __fmaf_rn((float)(2 * j + 1), inv, -1.0f);
        z = __fmaf_rn(-(float)k, 2.0f / (float)src.N, 1.0f);
        return 0;
    }
    uint32_t idx = (src.mode == PTS_LIST) ? (uint32_t)src.list[p] : (uint32_t)(src.base + p);
    int f = 0;
    int N = src.N;
    if (src.maps0) {
        const uint32_t sd = (uint32_t)src.slot_div;
        f = (int)(idx / sd);
        idx -= (uint32_t)f * sd;
        if (src.sv) N = src.sv[f].N;   // frame stream: the slot's level
    }
    const uint32_t n1 = (uint32_t)N + 1u;
    const uint32_t row = idx / n1;             // k (N + 1) + j
    const int i = (int)(idx - row * n1);
    const uint32_t kk = row / n1;
    const int j = (int)(row - kk * n1);
    const int k = (int)kk;
    const float h = 2.0f / (float)N;   // exact for power-of-two N
    x = __fmaf_rn((float)i, h, -1.0f);
    y = __fmaf_rn((float)j, h, -1.0f);
    z = __fmaf_rn((float)k, h, -1.0f);
    return f;
}

// Four consecutive channels of a texel as floats (FP32 or BF16 storage).
__device__ __forceinline__ float4 tap4(const Map& mp, int64_t e) {
    if (mp.dtype == 1) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(mp.data) + e));
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                           __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    }
    return ld4(static_cast<const float*>(mp.data) + e);
}

// Eight consecutive channels of a BF16 texel as floats: one 16-byte load
// (e a multiple of 8, the map 16-byte aligned).
__device__ __forceinline__ void tap8_bf16(const Map& mp, int64_t e, float4& lo, float4& hi) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(mp.data) + e));
    lo = make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                     __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    hi = make_float4(__uint_as_float(v.z << 16), __uint_as_float(v.z & 0xffff0000u),
                     __uint_as_float(v.w << 16), __uint_as_float(v.w & 0xffff0000u));
}

// A point's projection, the frame's maps and the four bilinear taps of
// each map: everything its channels share.
struct PointSample {
    Map map0, map1;
    float zh, zl;                  // projected depth as hi + lo
    int64_t e0[4], e1[4];          // tap element offsets (channel 0) in map0 / map1
    float w0[4], w1[4];            // bilinear weights w00, w10, w01, w11 of each map
};

__device__ __forceinline__ void taps_of(const Map& mp, float uh, float ul, float vh, float vl,
                                        int64_t (&e)[4], float (&w)[4]) {
    int i0, j0;
    float a, b;
    texel_coord(uh, ul, mp.W, i0, a);
    texel_coord(vh, vl, mp.H, j0, b);
    const int i1 = min(max(i0 + 1, 0), mp.W - 1);
    const int j1 = min(max(j0 + 1, 0), mp.H - 1);
    i0 = min(max(i0, 0), mp.W - 1);
    j0 = min(max(j0, 0), mp.H - 1);
    e[0] = ((int64_t)j0 * mp.W + i0) * mp.C;
    e[1] = ((int64_t)j0 * mp.W + i1) * mp.C;
    e[2] = ((int64_t)j1 * mp.W + i0) * mp.C;
    e[3] = ((int64_t)j1 * mp.W + i1) * mp.C;
    w[0] = (1.f - a) * (1.f - b);
    w[1] = a * (1.f - b);
    w[2] = (1.f - a) * b;
    w[3] = a * b;
}

__device__ __forceinline__ PointSample sample_point(const PointSrc& src, int64_t p,
                                                    const Calib& calib_in, const Map& map0_in,
                                                    const Map& map1_in) {
    PointSample ps;
    float x, y, z;
    const int f = point_xyz(src, p, x, y, z);
    const bool multi = src.maps0 != nullptr;
    // by value: a reference that may name the kernel's parameter would put
    // the parameter in local memory
    const Calib calib = multi ? src.calibs[f] : calib_in;
    ps.map0 = multi ? src.maps0[f] : map0_in;
    ps.map1 = multi ? (src.maps1 ? src.maps1[f] : Map{nullptr, 0, 0, 0, 0}) : map1_in;
    float uh, ul, vh, vl;
    affine_ff(calib.c + 0, x, y, z, uh, ul);
    affine_ff(calib.c + 4, x, y, z, vh, vl);
    affine_ff(calib.c + 8, x, y, z, ps.zh, ps.zl);
    if (ps.map0.C > 0) taps_of(ps.map0, uh, ul, vh, vl, ps.e0, ps.w0);
    if (ps.map1.C > 0) taps_of(ps.map1, uh, ul, vh, vl, ps.e1, ps.w1);
    return ps;
}

// Channels c..c+3 of the sampled point's MLP input row: the bilinear sample
// of map0 (channels [0, C0)) or map1 ([C0, C0 + C1)), then the projected
// depth at C0 + C1, then zero padding.
__device__ __forceinline__ float4 sample_quad(const PointSample& ps, int c) {
    const int C0 = ps.map0.C, C1 = ps.map1.C;
    if (c >= C0 + C1) return make_float4(c == C0 + C1 ? __fadd_rn(ps.zh, ps.zl) : 0.f, 0.f, 0.f, 0.f);
    // selections by value (constant indices keep the arrays in registers)
    const bool first = c < C0;
    const Map& mp = first ? ps.map0 : ps.map1;
    const int64_t cc = first ? c : c - C0;
    const float4 f00 = tap4(mp, (first ? ps.e0[0] : ps.e1[0]) + cc);
    const float4 f10 = tap4(mp, (first ? ps.e0[1] : ps.e1[1]) + cc);
    const float4 f01 = tap4(mp, (first ? ps.e0[2] : ps.e1[2]) + cc);
    const float4 f11 = tap4(mp, (first ? ps.e0[3] : ps.e1[3]) + cc);
    const float w00 = first ? ps.w0[0] : ps.w1[0], w10 = first ? ps.w0[1] : ps.w1[1];
    const float w01 = first ? ps.w0[2] : ps.w1[2], w11 = first ? ps.w0[3] : ps.w1[3];
    float4 r;
    r.x = fmaf(w11, f11.x, fmaf(w01, f01.x, fmaf(w10, f10.x, w00 * f00.x)));
    r.y = fmaf(w11, f11.y, fmaf(w01, f01.y, fmaf(w10, f10.y, w00 * f00.y)));
    r.z = fmaf(w11, f11.z, fmaf(w01, f01.z, fmaf(w10, f10.z, w00 * f00.z)));
    r.w = fmaf(w11, f11.w, fmaf(w01, f01.w, fmaf(w10, f10.w, w00 * f00.w)));
    return r;
}

// Whether channels c..c+7 of the sampled point's row lie in one BF16 map at
// a multiple of 8 of its channels (then sample_oct_bf16 reads them with one
// 16-byte load per tap).
__device__ __forceinline__ bool oct_bf16(const PointSample& ps, int c) {
    const int C0 = ps.map0.C, C1 = ps.map1.C;
    if (c + 8 <= C0) return ps.map0.dtype == 1 && (C0 & 7) == 0 && (c & 7) == 0;
    return c >= C0 && c + 8 <= C0 + C1 && ps.map1.dtype == 1 && (C1 & 7) == 0 &&
           ((c - C0) & 7) == 0;
}

// Channels c..c+7 of the sampled point's row when oct_bf16(ps, c): the
// same bilinear arithmetic as sample_quad, per channel.
__device__ __forceinline__ void sample_oct_bf16(const PointSample& ps, int c, float4& lo,
                                                float4& hi) {
    const bool first = c < ps.map0.C;
    const Map& mp = first ? ps.map0 : ps.map1;
    const int64_t cc = first ? c : c - ps.map0.C;
    float4 a[4], b[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) tap8_bf16(mp, (first ? ps.e0[t] : ps.e1[t]) + cc, a[t], b[t]);
    const float w00 = first ? ps.w0[0] : ps.w1[0], w10 = first ? ps.w0[1] : ps.w1[1];
    const float w01 = first ? ps.w0[2] : ps.w1[2], w11 = first ? ps.w0[3] : ps.w1[3];
    lo.x = fmaf(w11, a[3].x, fmaf(w01, a[2].x, fmaf(w10, a[1].x, w00 * a[0].x)));
    lo.y = fmaf(w11, a[3].y, fmaf(w01, a[2].y, fmaf(w10, a[1].y, w00 * a[0].y)));
    lo.z = fmaf(w11, a[3].z, fmaf(w01, a[2].z, fmaf(w10, a[1].z, w00 * a[0].z)));
    lo.w = fmaf(w11, a[3].w, fmaf(w01, a[2].w, fmaf(w10, a[1].w, w00 * a[0].w)));
    hi.x = fmaf(w11, b[3].x, fmaf(w01, b[2].x, fmaf(w10, b[1].x, w00 * b[0].x)));
    hi.y = fmaf(w11, b[3].y, fmaf(w01, b[2].y, fmaf(w10, b[1].y, w00 * b[0].y)));
    hi.z = fmaf(w11, b[3].z, fmaf(w01, b[2].z, fmaf(w10, b[1].z, w00 * b[0].z)));
    hi.w = fmaf(w11, b[3].w, fmaf(w01, b[2].w, fmaf(w10, b[1].w, w00 * b[0].w)));
}

// Channels c..c+3 of the MLP input row of point p (one quad on its own,
// the same arithmetic as sample_point + sample_quad; written out so that
// only the map holding channel c is touched, which keeps the register count
// of the kernels that inline it next to their hot loops).
__device__ __forceinline__ float4 gather_quad(const PointSrc& src, int64_t p, const Calib& calib_in,
                                              const Map& map0_in, const Map& map1_in, int c) {
    float x, y, z;
    const int f = point_xyz(src, p, x, y, z);
    const bool multi = src.maps0 != nullptr;
    const Calib& calib = multi ? src.calibs[f] : calib_in;
    const Map map0 = multi ? src.maps0[f] : map0_in;
    const Map map1 = multi ? (src.maps1 ? src.maps1[f] : Map{nullptr, 0, 0, 0, 0}) : map1_in;
    float uh, ul, vh, vl, zh, zl;
    affine_ff(calib.c + 0, x, y, z, uh, ul);
    affine_ff(calib.c + 4, x, y, z, vh, vl);
    affine_ff(calib.c + 8, x, y, z, zh, zl);

    float4 r;
    const int C0 = map0.C, C1 = map1.C;
    if (c < C0 + C1) {
        const Map& mp = (c < C0) ? map0 : map1;
        const int cc = (c < C0) ? c : c - C0;
        int i0, j0;
        float a, b;
        texel_coord(uh, ul, mp.W, i0, a);
        texel_coord(vh, vl, mp.H, j0, b);
        const int i1 = min(max(i0 + 1, 0), mp.W - 1);
        const int j1 = min(max(j0 + 1, 0), mp.H - 1);
        i0 = min(max(i0, 0), mp.W - 1);
        j0 = min(max(j0, 0), mp.H - 1);
        const float4 f00 = tap4(mp, ((int64_t)j0 * mp.W + i0) * mp.C + cc);
        const float4 f10 = tap4(mp, ((int64_t)j0 * mp.W + i1) * mp.C + cc);
        const float4 f01 = tap4(mp, ((int64_t)j1 * mp.W + i0) * mp.C + cc);
        const float4 f11 = tap4(mp, ((int64_t)j1 * mp.W + i1) * mp.C + cc);
        const float w00 = (1.f - a) * (1.f - b), w10 = a * (1.f - b);
        const float w01 = (1.f - a) * b, w11 = a * b;
        r.x = fmaf(w11, f11.x, fmaf(w01, f01.x, fmaf(w10, f10.x, w00 * f00.x)));
        r.y = fmaf(w11, f11.y, fmaf(w01, f01.y, fmaf(w10, f10.y, w00 * f00.y)));
        r.z = fmaf(w11, f11.z, fmaf(w01, f01.z, fmaf(w10, f10.z, w00 * f00.z)));
        r.w = fmaf(w11, f11.w, fmaf(w01, f01.w, fmaf(w10, f10.w, w00 * f00.w)));
    } else {
        r = make_float4(c == C0 + C1 ? __fadd_rn(zh, zl) : 0.f, 0.f, 0.f, 0.f);
    }
    return r;
}

}  // namespace pifu
