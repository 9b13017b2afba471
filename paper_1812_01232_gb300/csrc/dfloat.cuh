// Double-float arithmetic (a value carried as an unevaluated FP32 sum hi + lo)
// from the error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and
// the FMA-based exact product.  Used for per-component geometry of a cube
// (differences, rotations, unit directions) so that the bound kernel needs no
// FP64 arithmetic: FP64 runs at ~1/64 of the FP32 rate on this GPU.
#pragma once

#include <cuda_runtime.h>

namespace gosma {

struct df {
    float h, l;
};

// s + e = a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// s + e = a + b exactly, provided |a| >= |b| or a == 0.
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}

// p + e = a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = a * b;
    return {p, fmaf(a, b, -p)};
}

// (a - b) for double-floats, relative error ~2^-44.
__device__ __forceinline__ df df_sub(df a, df b) {
    df s = two_sum(a.h, -b.h);
    s.l += a.l - b.l;
    return fast_two_sum(s.h, s.l);
}

// |x|^2 of a 3-vector of double-floats.
__device__ __forceinline__ df df_norm2(df x, df y, df z) {
    df px = two_prod(x.h, x.h), py = two_prod(y.h, y.h), pz = two_prod(z.h, z.h);
    float ex = fmaf(2.f * x.h, x.l, px.l), ey = fmaf(2.f * y.h, y.l, py.l), ez = fmaf(2.f * z.h, z.l, pz.l);
    df s = two_sum(px.h, py.h);
    df t = two_sum(s.h, pz.h);
    float e = s.l + t.l + (ex + ey + ez);
    return fast_two_sum(t.h, e);
}

// 1/sqrt(d) for a double-float d > 0: FP32 rsqrt plus one Newton step
// r1 = r0 (1 + (1 - d r0^2) / 2) carried in double-float.
__device__ __forceinline__ df df_rsqrt(df d, float r0) {
    df q = two_prod(r0, r0);
    df hh = two_prod(d.h, q.h);
    float hl = hh.l + fmaf(d.h, q.l, d.l * q.h);
    float one_minus = (1.f - hh.h) - hl;  // 1 - hh.h is exact (hh.h is within a factor 2 of 1)
    return fast_two_sum(r0, 0.5f * r0 * one_minus);
}

// a * b for double-floats (second-order terms dropped).
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.h, b.h);
    p.l += fmaf(a.h, b.l, a.l * b.h);
    return fast_two_sum(p.h, p.l);
}

// Dot product of three double-float pairs sum_k a_k b_k.
__device__ __forceinline__ df df_dot3(df a0, df b0, df a1, df b1, df a2, df b2) {
    df p0 = two_prod(a0.h, b0.h), p1 = two_prod(a1.h, b1.h), p2 = two_prod(a2.h, b2.h);
    float e0 = fmaf(a0.h, b0.l, fmaf(a0.l, b0.h, p0.l));
    float e1 = fmaf(a1.h, b1.l, fmaf(a1.l, b1.h, p1.l));
    float e2 = fmaf(a2.h, b2.l, fmaf(a2.l, b2.h, p2.l));
    df s = two_sum(p0.h, p1.h);
    df t = two_sum(s.h, p2.h);
    return fast_two_sum(t.h, s.l + t.l + (e0 + e1 + e2));
}

// a + b for double-floats.
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return fast_two_sum(s.h, s.l);
}

// (s + c) * w for an unevaluated sum s + c (|c| <= u|s|) and an FP32 w: the
// leading product is exact, the rest is second order.
__device__ __forceinline__ df df_scale(float s, float c, float w) {
    df p = two_prod(s, w);
    p.l = fmaf(c, w, p.l);
    return fast_two_sum(p.h, p.l);
}

// a / b for double-floats (b != 0): an FP32 quotient and one correction
// from the exact remainder, relative error ~2^-44.
__device__ __forceinline__ df df_div(df a, df b) {
    const float q0 = a.h / b.h;
    const df p = two_prod(q0, b.h);
    const float r = ((a.h - p.h) - p.l + a.l) - q0 * b.l;  // a - q0 b; a.h - p.h is exact
    return fast_two_sum(q0, r / b.h);
}

// sin and cos of a double-float 0 <= t <= 8, to ~2^-46 absolute (Cody and
// Waite's reduction by k pi/2 with pi/2 in three floats, the first two of
// 20 bits so that k times them is exact; then the Taylor series of sin and
// cos on |x| <= pi/4, the terms from x^11 and x^10 on in FP32, the leading
// five in double-float).
__device__ inline void df_sincos(df t, df &s, df &c) {
    const float P1 = 0x1.921fcp+0f, P2 = -0x1.5777ap-21f, P3 = -0x1.73dcb4p-43f;
    const float k = rintf(t.h * 0x1.45f306p-1f);  // nearest multiple of pi/2
    const df a = two_sum(t.h - k * P1, t.l);       // t.h - k P1 is exact
    const df b = two_sum(a.h, -k * P2);
    const df x = fast_two_sum(b.h, (a.l + b.l) - k * P3);
    const df z = df_mul(x, x);
    // sin x / x = sum (-1)^n z^n / (2n + 1)!, cos x = sum (-1)^n z^n / (2n)!
    float ts = 0x1.71b8fp-66f, tc = -0x1.0ce396p-70f;
    ts = fmaf(ts, z.h, -0x1.2f49b4p-57f);
    ts = fmaf(ts, z.h, 0x1.952c78p-49f);
    ts = fmaf(ts, z.h, -0x1.ae7f3ep-41f);
    ts = fmaf(ts, z.h, 0x1.612462p-33f);
    ts = fmaf(ts, z.h, -0x1.ae6456p-26f);
    tc = fmaf(tc, z.h, 0x1.e542bap-62f);
    tc = fmaf(tc, z.h, -0x1.682786p-53f);
    tc = fmaf(tc, z.h, 0x1.ae7f3ep-45f);
    tc = fmaf(tc, z.h, -0x1.93974ap-37f);
    tc = fmaf(tc, z.h, 0x1.1eed8ep-29f);
    tc = fmaf(tc, z.h, -0x1.27e4fcp-22f);
    const df cs[5] = {{1.f, 0.f},
                      {-0x1.555556p-3f, 0x1.555556p-28f},
                      {0x1.111112p-7f, -0x1.dddddep-32f},
                      {-0x1.a01a02p-13f, 0x1.7f97fap-39f},
                      {0x1.71de3ap-19f, 0x1.55b1ccp-45f}};
    const df cc[5] = {{1.f, 0.f},
                      {-0.5f, 0.f},
                      {0x1.555556p-5f, -0x1.555556p-30f},
                      {-0x1.6c16c2p-10f, 0x1.27d27ep-35f},
                      {0x1.a01a02p-16f, -0x1.7f97fap-42f}};
    df ps = {ts, 0.f}, pc = {tc, 0.f};
#pragma unroll
    for (int n = 4; n >= 0; --n) {
        ps = df_add(df_mul(ps, z), cs[n]);
        pc = df_add(df_mul(pc, z), cc[n]);
    }
    const df sx = df_mul(x, ps);
    const int q = (int)k & 3;
    const df nsx = {-sx.h, -sx.l}, npc = {-pc.h, -pc.l};
    s = q == 0 ? sx : q == 1 ? pc : q == 2 ? nsx : npc;
    c = q == 0 ? pc : q == 1 ? nsx : q == 2 ? npc : sx;
}

__host__ __device__ inline void split_double(double x, float &h, float &l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

}  // namespace gosma
