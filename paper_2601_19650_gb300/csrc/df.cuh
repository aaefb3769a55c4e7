// Double-float arithmetic shared by the FP32-based stages of the mixed path (the
// tridiagonal reductions and the back transformation): a value is h + l, two FP32
// numbers, ~2^-46 relative per operation.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace cbc {

// ---- double-float arithmetic (value = h + l, two FP32 numbers, ~2^-46 relative) -----
// On this part FP32 issues ~64x faster than FP64, so the mixed path keeps the rows of
// the tridiagonal reduction as double-float pairs and runs its two O(m^2)-per-column
// loops (p = A v and the rank-2 update) in FP32 with error-free transformations
// (TwoProduct by fma, TwoSum; Dekker and Knuth).  The rounded intrinsics keep the
// compiler from contracting them.
struct df1 {
  float h, l;
};
struct dfz {
  df1 re, im;
};
template <typename T>
struct dfof;
template <>
struct dfof<double> {
  using type = df1;
};
template <>
struct dfof<zdbl> {
  using type = dfz;
};
__device__ __forceinline__ df1 df_make(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ df1 df_neg(df1 a) { return {-a.h, -a.l}; }
// c + a b
__device__ __forceinline__ df1 df_fma(df1 a, df1 b, df1 c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float s = __fadd_rn(c.h, p);
  const float bb = __fsub_rn(s, c.h);
  float t = __fadd_rn(__fsub_rn(c.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  t = __fadd_rn(t, __fadd_rn(c.l, e));
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ df1 to_df(double x) { return df_make(x); }
__device__ __forceinline__ dfz to_df(zdbl x) { return {df_make(x.re), df_make(x.im)}; }
__device__ __forceinline__ double from_df(df1 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ zdbl from_df(dfz a) { return {from_df(a.re), from_df(a.im)}; }
__device__ __forceinline__ df1 dff(df1 a, df1 b, df1 c) { return df_fma(a, b, c); }
__device__ __forceinline__ dfz dff(dfz a, dfz b, dfz c) {  // c + a b, complex
  return {df_fma(df_neg(a.im), b.im, df_fma(a.re, b.re, c.re)),
          df_fma(a.im, b.re, df_fma(a.re, b.im, c.im))};
}
__device__ __forceinline__ df1 dfconj(df1 a) { return a; }
__device__ __forceinline__ dfz dfconj(dfz a) { return {a.re, df_neg(a.im)}; }

// a + b (TwoSum of the high parts, the low parts and the rounding error added, then
// renormalised)
__device__ __forceinline__ df1 df_add(df1 a, df1 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  t = __fadd_rn(t, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfz df_add(dfz a, dfz b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfz df_neg(dfz a) { return {df_neg(a.re), df_neg(a.im)}; }
__device__ __forceinline__ df1 df_shfl_xor(df1 a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}
__device__ __forceinline__ dfz df_shfl_xor(dfz a, int o) {
  return {df_shfl_xor(a.re, o), df_shfl_xor(a.im, o)};
}
__device__ __forceinline__ df1 df_shfl_idx(df1 a, int src) {
  return {__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src)};
}
__device__ __forceinline__ dfz df_shfl_idx(dfz a, int src) {
  return {df_shfl_idx(a.re, src), df_shfl_idx(a.im, src)};
}
// |a|^2 as a real double-float
__device__ __forceinline__ df1 df_abs2(df1 a) { return df_fma(a, a, df1{0.f, 0.f}); }
__device__ __forceinline__ df1 df_abs2(dfz a) {
  return df_fma(a.im, a.im, df_fma(a.re, a.re, df1{0.f, 0.f}));
}

}  // namespace cbc
