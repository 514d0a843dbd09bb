// Double-float arithmetic on the FP32 pipes for reductions that need more
// than single precision: a value is the unevaluated sum h + l of two floats
// (about 48 significant bits), added with error-free transformations (Knuth's
// two-sum, FMA-based two-product).  GB300 runs FP64 at a small fraction of its
// FP32 rate, and these sums sit in every iteration of the persistent
// coarsest-level solvers; the order of every sum is fixed, so results stay
// reproducible bit for bit.
#pragma once
#include <cuda_runtime.h>

namespace mg {

struct df {
  float h, l;
};
__device__ __forceinline__ df df_of(float x) { return df{x, 0.f}; }
__device__ __forceinline__ df df_norm(float s, float e) {   // s + e with |e| small: renormalise
  const float h = s + e;
  return df{h, e - (h - s)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb) + (a.l + b.l);
  return df_norm(s, e);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p) + (a.h * b.l + a.l * b.h);
  return df_norm(p, e);
}
// a / b (b > 0) by one correction of the float quotient
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = a.h / b.h;
  const df r = df_add(a, df_neg(df_mul(df_of(q1), b)));
  return df_norm(q1, r.h / b.h);
}
// sqrt(a), a >= 0, by one Newton correction of sqrtf
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.h > 0.f)) return df_of(0.f);
  const float s = sqrtf(a.h);
  const df r = df_add(a, df_neg(df_mul(df_of(s), df_of(s))));
  return df_norm(s, r.h / (2.f * s));
}
__device__ __forceinline__ df df_wsum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df u{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = df_add(v, u);
  }
  return v;
}


}  // namespace mg
