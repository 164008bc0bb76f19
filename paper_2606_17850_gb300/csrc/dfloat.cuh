// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  Built from the
// error-free transformations of Knuth (TwoSum, TAOCP vol. 2, 4.2.2), Dekker
// (Fast2Sum, Numer. Math. 18, 1971) and the FMA form of TwoProduct.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so the FP64 refinement
// residual of the mixed path (about 20 FP64 operations per cell) is ALU-bound; in
// double-float the same residual costs about 165 FP32 operations per cell (with
// the unnormalised forms below).  The residual needs ~1e-12 relative accuracy on each
// face flux (the fluxes through a cell cancel down to its power), which
// double-float provides and FP32 does not.
#pragma once

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) {
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

// Dekker Fast2Sum (requires |a| >= |b| or a == 0): s + e == a + b exactly.
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

// TwoProduct with FMA: p + e == a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return df_make(p, e);
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}

// double-float times an FP32 number
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, e);
}

// Unnormalised ("lazy") forms for chains of operations whose result is rounded to
// FP32 at the end: the sum keeps TwoSum's exact high part and adds the low parts
// without the final Fast2Sum, the product keeps TwoProduct's exact high part and
// the two cross terms.  The low part may then exceed ulp(hi)/2, but the absolute
// error of a chain stays of the order 2^-47 times its largest operand, the same
// order as the normalised forms' (the low parts of double-float inputs already
// carry that much rounding).
__device__ __forceinline__ df ldf_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return df_make(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df ldf_sub(df a, df b) { return ldf_add(a, df_neg(b)); }

__device__ __forceinline__ df ldf_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.hi, b.hi, -p)));
  return df_make(p, e);
}

// FP64 <-> double-float (used once per solve at the boundary, not in the loops)
__host__ __device__ __forceinline__ void df_split(double v, float* h, float* l) {
  const float a = (float)v;
  *h = a;
  *l = (float)(v - (double)a);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
