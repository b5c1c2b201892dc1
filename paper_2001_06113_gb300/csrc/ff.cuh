// Double-float ("ff") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, giving a 48-bit significand from the
// FP32 pipes.  Used for the mode state u^, W and the one-step phase p_0 in
// mixed precision: GB300 issues FP32 FMAs at ~58x its FP64 rate.
//
// Building blocks (error-free transformations, Knuth/Dekker, FMA form):
//   two_sum(a, b):  s = fl(a + b), e = (a + b) - s exactly
//   two_prod(a, b): p = fl(a b),   e = fma(a, b, -p) = a b - p exactly
// A complex ff value is a float4 (re_hi, im_hi, re_lo, im_lo).
#pragma once
#include <cuda_runtime.h>

namespace tdse {

struct ffr { float hi, lo; };

__device__ __forceinline__ ffr ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ ffr ff_quick(float a, float b) {   // requires |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
// a + b (the "sloppy" sum: error bounded relative to |a| + |b|)
__device__ __forceinline__ ffr ff_add(ffr a, ffr b) {
    ffr s = ff_two_sum(a.hi, b.hi);
    return ff_quick(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ffr ff_add_f(ffr a, float b) {
    ffr s = ff_two_sum(a.hi, b);
    return ff_quick(s.hi, s.lo + a.lo);
}
// a*c - b*d and a*d + b*c with one renormalisation each
__device__ __forceinline__ ffr ff_dot2(ffr a, ffr c, ffr b, ffr d, float sgn) {
    const float p1 = a.hi * c.hi;
    const float e1 = fmaf(a.hi, c.hi, -p1);
    const float p2 = sgn * b.hi * d.hi;
    const float e2 = fmaf(sgn * b.hi, d.hi, -p2);
    ffr s = ff_two_sum(p1, p2);
    float lo = s.lo + (e1 + e2);
    lo = fmaf(a.hi, c.lo, lo);
    lo = fmaf(a.lo, c.hi, lo);
    lo = fmaf(sgn * b.hi, d.lo, lo);
    lo = fmaf(sgn * b.lo, d.hi, lo);
    return ff_quick(s.hi, lo);
}

// complex ff packed as float4 (re_hi, im_hi, re_lo, im_lo)
__device__ __forceinline__ ffr ff_re(float4 z) { return {z.x, z.z}; }
__device__ __forceinline__ ffr ff_im(float4 z) { return {z.y, z.w}; }
__device__ __forceinline__ float4 ff_pack(ffr re, ffr im) { return make_float4(re.hi, im.hi, re.lo, im.lo); }

__device__ __forceinline__ float4 ffc_mul(float4 x, float4 y) {
    const ffr a = ff_re(x), b = ff_im(x), c = ff_re(y), d = ff_im(y);
    return ff_pack(ff_dot2(a, c, b, d, -1.f), ff_dot2(a, d, b, c, 1.f));
}
// x + (re, im) with FP32 increments
__device__ __forceinline__ float4 ffc_add_f(float4 x, float re, float im) {
    return ff_pack(ff_add_f(ff_re(x), re), ff_add_f(ff_im(x), im));
}
__device__ __forceinline__ double2 ffc_to_d(float4 z) {
    return make_double2((double)z.x + (double)z.z, (double)z.y + (double)z.w);
}
__device__ __forceinline__ float4 d_to_ffc(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}

}  // namespace tdse
