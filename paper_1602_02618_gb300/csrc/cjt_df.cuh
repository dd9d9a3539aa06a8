// Double-float arithmetic: a real number held as the unevaluated sum h + l of two
// floats with |l| <= ulp(h)/2 (about 48 significant bits), computed on the FP32 pipe.
//
// On GB300 the FP32 pipe issues about 70 times more operations per clock than the
// FP64 pipe, so the transforms and the stored-recurrence products run in this
// representation in the CJT_DFLOAT form: each double-float operation costs 4 to 20
// float operations but keeps the rounding error within a small multiple of 2^-48.
//
// Building blocks (published error-free transformations):
//   two-sum      s + e = a + b exactly                     (Knuth, TAOCP vol. 2, 4.2.2)
//   fast-two-sum s + e = a + b exactly when |a| >= |b|     (Dekker 1971)
//   two-product  p + e = a * b exactly, e = fma(a, b, -p)
// Addition is the "sloppy" double-float sum (two-sum of the high parts, low parts
// added, one fast renormalisation): its error is bounded by a small multiple of
// 2^-48 (|a| + |b|), which is the bound a transform's error analysis needs.
// Products are rounded explicitly (__fmul_rn) so that the compiler cannot fuse
// them into a neighbouring addition.
#pragma once

#include <cuda_runtime.h>

struct __align__(8) dfs {    // real double-float
    float h, l;
};
struct __align__(16) dfc {   // complex double-float
    float rh, rl, ih, il;
};

__device__ __forceinline__ dfs df_make(float h, float l) { dfs r; r.h = h; r.l = l; return r; }

// nearest double-float to v (exact for |v| within float range; 48-bit rounding)
__device__ __forceinline__ dfs df_from(double v) {
    const float h = __double2float_rn(v);
    return df_make(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double df_to(dfs a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ dfs df_fast_renorm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return df_make(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfs df_add(dfs a, dfs b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return df_fast_renorm(s, e);
}
__device__ __forceinline__ dfs df_neg(dfs a) { return df_make(-a.h, -a.l); }
__device__ __forceinline__ dfs df_sub(dfs a, dfs b) { return df_add(a, df_neg(b)); }

// a + b without the final renormalisation: (s, e) with s + e = a + b up to the rounding
// of a.l + b.l, e possibly above ulp(s)/2.  For intermediate sums that feed another
// addition straight away (which renormalises); its error bound is the same multiple of
// 2^-48 (|a| + |b|).
__device__ __forceinline__ dfs df_add_nr(dfs a, dfs b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return df_make(s, e);
}

// a * b
__device__ __forceinline__ dfs df_mul(dfs a, dfs b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_fast_renorm(p, e);
}

// a * b - c * d, both products and their difference carried exactly to first order
__device__ __forceinline__ dfs df_mms(dfs a, dfs b, dfs c, dfs d) {
    const float p1 = __fmul_rn(a.h, b.h);
    const float e1 = fmaf(a.h, b.h, -p1);
    const float p2 = __fmul_rn(c.h, d.h);
    const float e2 = fmaf(c.h, d.h, -p2);
    const float s = __fsub_rn(p1, p2);
    const float bb = __fsub_rn(s, p1);
    const float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(-p2, bb));
    float t = fmaf(a.h, b.l, e1);
    t = fmaf(a.l, b.h, t);
    t = fmaf(-c.h, d.l, t);
    t = fmaf(-c.l, d.h, t);
    t = __fadd_rn(__fsub_rn(t, e2), es);
    return df_fast_renorm(s, t);
}

// acc + a * b (renormalised)
__device__ __forceinline__ dfs df_mac(dfs acc, dfs a, dfs b) { return df_add(acc, df_mul(a, b)); }

// complex
__device__ __forceinline__ dfc dfc_make(dfs re, dfs im) { dfc r; r.rh = re.h; r.rl = re.l; r.ih = im.h; r.il = im.l; return r; }
__device__ __forceinline__ dfs dfc_re(dfc a) { return df_make(a.rh, a.rl); }
__device__ __forceinline__ dfs dfc_im(dfc a) { return df_make(a.ih, a.il); }
__device__ __forceinline__ dfc dfc_zero() { dfc r; r.rh = r.rl = r.ih = r.il = 0.0f; return r; }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return dfc_make(df_add(dfc_re(a), dfc_re(b)), df_add(dfc_im(a), dfc_im(b))); }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return dfc_make(df_sub(dfc_re(a), dfc_re(b)), df_sub(dfc_im(a), dfc_im(b))); }
__device__ __forceinline__ dfc dfc_add_nr(dfc a, dfc b) { return dfc_make(df_add_nr(dfc_re(a), dfc_re(b)), df_add_nr(dfc_im(a), dfc_im(b))); }
__device__ __forceinline__ dfc dfc_sub_nr(dfc a, dfc b) {
    return dfc_make(df_add_nr(dfc_re(a), df_neg(dfc_re(b))), df_add_nr(dfc_im(a), df_neg(dfc_im(b))));
}
// a * w
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc w) {
    const dfs ar = dfc_re(a), ai = dfc_im(a), wr = dfc_re(w), wi = dfc_im(w);
    return dfc_make(df_mms(ar, wr, ai, wi), df_mms(ar, wi, df_neg(ai), wr));
}
// a * (-i)
__device__ __forceinline__ dfc dfc_mul_mi(dfc a) { dfc r; r.rh = a.ih; r.rl = a.il; r.ih = -a.rh; r.il = -a.rl; return r; }
__device__ __forceinline__ dfc dfc_conj(dfc a) { a.ih = -a.ih; a.il = -a.il; return a; }
// a * s for s a power of two (exact)
__device__ __forceinline__ dfc dfc_scale_pow2(dfc a, float s) { a.rh *= s; a.rl *= s; a.ih *= s; a.il *= s; return a; }
