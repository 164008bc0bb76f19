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

// Two double-float values per operation (lanes x and y), on Blackwell's paired FP32
// instructions: every helper below performs, lane by lane, the same round-to-nearest
// operations in the same order as its one-value form above, so each lane's result is
// bit-identical to it.  A difference x - y is the fused multiply-add y * (-1) + x
// (exact product, one rounding: the same as the subtraction).
struct df2 {
  float2 hi, lo;
};

__device__ __forceinline__ df2 df2_make(float2 h, float2 l) {
  df2 r;
  r.hi = h;
  r.lo = l;
  return r;
}
__device__ __forceinline__ df2 df2_of(df a, df b) {
  return df2_make(make_float2(a.hi, b.hi), make_float2(a.lo, b.lo));
}
__device__ __forceinline__ float2 f2_sub(float2 x, float2 y) {
  return __ffma2_rn(y, make_float2(-1.f, -1.f), x);
}

// df_sub: TwoSum of (a.hi, -b.hi), low parts, Fast2Sum
__device__ __forceinline__ df2 df2_sub(df2 a, df2 b) {
  const float2 s = f2_sub(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);                           // s - a   (= (-b) rounded part)
  const float2 e0 = f2_sub(f2_sub(a.hi, f2_sub(s, bb)), __fadd2_rn(b.hi, bb));  // (a - (s - bb)) + (-b - bb)
  const float2 e = __fadd2_rn(e0, f2_sub(a.lo, b.lo));
  const float2 h = __fadd2_rn(s, e);
  return df2_make(h, f2_sub(e, f2_sub(h, s)));
}

// ldf_add: TwoSum of the high parts, the low parts added without renormalising
__device__ __forceinline__ df2 ldf2_add(df2 a, df2 b) {
  const float2 s = __fadd2_rn(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);
  const float2 e0 = __fadd2_rn(f2_sub(a.hi, f2_sub(s, bb)), f2_sub(b.hi, bb));
  return df2_make(s, __fadd2_rn(e0, __fadd2_rn(a.lo, b.lo)));
}

// ldf_sub: ldf_add of (a, -b)
__device__ __forceinline__ df2 ldf2_sub(df2 a, df2 b) {
  const float2 s = f2_sub(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);
  const float2 e0 = f2_sub(f2_sub(a.hi, f2_sub(s, bb)), __fadd2_rn(b.hi, bb));
  return df2_make(s, __fadd2_rn(e0, f2_sub(a.lo, b.lo)));
}

// ldf_mul: exact high product and the two cross terms
__device__ __forceinline__ df2 ldf2_mul(df2 a, df2 b) {
  const float2 p = __fmul2_rn(a.hi, b.hi);
  const float2 np = __fmul2_rn(p, make_float2(-1.f, -1.f));
  const float2 e = __ffma2_rn(a.lo, b.hi, __ffma2_rn(a.hi, b.lo, __ffma2_rn(a.hi, b.hi, np)));
  return df2_make(p, e);
}

// FP64 <-> double-float (used once per solve at the boundary, not in the loops)
__host__ __device__ __forceinline__ void df_split(double v, float* h, float* l) {
  const float a = (float)v;
  *h = a;
  *l = (float)(v - (double)a);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
