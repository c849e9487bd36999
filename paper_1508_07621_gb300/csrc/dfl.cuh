// Double-float arithmetic (each value an unevaluated sum hi + lo of two FP32 numbers, about 48
// significant bits): Dekker's splitting, Knuth's two-sum and the two-product by FMA, with every
// operation explicitly rounded so that the compiler cannot contract or reorder it.  Shared by the
// tiled tridiagonal chain and the small-N dense resident chain (FQ_DF32).
#pragma once

#include <cuda_runtime.h>

namespace {

// double-float value hi + lo, |lo| <= ulp(hi) / 2
struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl dfl_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dfl_value(dfl a) { return (double)a.h + (double)a.l; }

// a * b + c in double-float: exact two-product of the high parts (FMA), the cross terms, a
// two-sum with c's high part, and a final fast renormalisation.  Every step uses an explicitly
// rounded operation, so the compiler cannot contract or reorder it.
__device__ __forceinline__ dfl dfl_fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.h, b.h);
  float pe = __fmaf_rn(a.h, b.h, -p);
  pe = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, pe));
  const float s = __fadd_rn(p, c.h);
  const float bb = __fsub_rn(s, p);
  float se = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.h, bb));
  se = __fadd_rn(se, __fadd_rn(pe, c.l));
  const float h = __fadd_rn(s, se);
  return {h, __fsub_rn(se, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl dfl_neg(dfl a) { return {-a.h, -a.l}; }

// A complex double-float value packed for FP32x2 arithmetic: h = (re.hi, im.hi), l = (re.lo, im.lo).
// A real operator entry acts on the real and imaginary parts alike, so every double-float FMA of
// the step runs on both components at once with packed FFMA2 / FADD2 / FMUL2.
struct dflc {
  float2 h, l;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// a * x + c for a real double-float a and complex double-float x, c
__device__ __forceinline__ dflc dflc_fma(dfl a, dflc x, dflc c) {
  const float2 ah = make_float2(a.h, a.h), al = make_float2(a.l, a.l);
  const float2 p = __fmul2_rn(ah, x.h);
  float2 pe = __ffma2_rn(ah, x.h, neg2(p));
  pe = __ffma2_rn(ah, x.l, __ffma2_rn(al, x.h, pe));
  const float2 sm = __fadd2_rn(p, c.h);
  const float2 bb = __fadd2_rn(sm, neg2(p));
  float2 se = __fadd2_rn(__fadd2_rn(p, neg2(__fadd2_rn(sm, neg2(bb)))), __fadd2_rn(c.h, neg2(bb)));
  se = __fadd2_rn(se, __fadd2_rn(pe, c.l));
  const float2 h = __fadd2_rn(sm, se);
  return {h, __fadd2_rn(se, neg2(__fadd2_rn(h, neg2(sm))))};
}

// i cc * v + c: (-cc v_im, cc v_re) + c, one component at a time
__device__ __forceinline__ dflc dflc_ifma(dfl cc, dflc v, dflc c) {
  const dfl r = dfl_fma(dfl_neg(cc), dfl{v.h.y, v.l.y}, dfl{c.h.x, c.l.x});
  const dfl i = dfl_fma(cc, dfl{v.h.x, v.l.x}, dfl{c.h.y, c.l.y});
  return {make_float2(r.h, i.h), make_float2(r.l, i.l)};
}

__device__ __forceinline__ dflc dflc_neg(dflc a) { return {neg2(a.h), neg2(a.l)}; }


// a + c for complex double-float values (the product by 1 is exact)
__device__ __forceinline__ dflc dflc_add(dflc a, dflc c) { return dflc_fma(dfl{1.f, 0.f}, a, c); }

// i a x + c for a real double-float a and complex x, c, packed: i x = (-x_im, x_re)
__device__ __forceinline__ dflc dflc_ifma2(dfl a, dflc x, dflc c) {
  const dflc ix = {make_float2(-x.h.y, x.h.x), make_float2(-x.l.y, x.l.x)};
  return dflc_fma(a, ix, c);
}

}  // namespace
