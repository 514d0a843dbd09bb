// Row-parallel complex GEMV used by the coarse stencil kernels.
//
// A CTA owns one coarse site; warp w owns rows [w*rpw, (w+1)*rpw) of the
// site's link block (row-major, K complex per row).  The lanes stride over
// the row in float4 units (two complex numbers), and every lane keeps one
// accumulator per owned row, so each step issues rpw independent 16-byte
// loads per lane and every warp load instruction reads 512 contiguous bytes.
#pragma once
#include "common.cuh"

namespace mg {

constexpr int kGemvMaxRows = 8;  // rows per warp (nc <= 64 with 8 warps)

__device__ __forceinline__ float gemv_wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// res[r] = sum_k M[row_r][k] * v[k] for the warp's rows row_r = row0 + w*rpw + r
// (r < rpw, row_r < row1).  M: global, row stride K complex (K even,
// 16-byte aligned rows); v: shared memory, K complex, 16-byte aligned.
// After the call every lane holds the full sums.
__device__ __forceinline__ void warp_gemv_rows(const float2* __restrict__ M, int row0, int row1, int K,
                                               const float2* v, int w, int rpw, int lane,
                                               float2 res[kGemvMaxRows]) {
  const float4* M4 = reinterpret_cast<const float4*>(M);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const int K4 = K >> 1;
  float re[kGemvMaxRows], im[kGemvMaxRows];
#pragma unroll
  for (int r = 0; r < kGemvMaxRows; r++) re[r] = im[r] = 0.f;
  // batches of kSteps lane-steps: all loads of a batch are issued before any
  // is used, so a warp has up to kSteps * rpw loads in flight per lane
  constexpr int kSteps = 2;
  for (int q0 = lane; q0 < K4; q0 += 32 * kSteps) {
    float4 m[kSteps][kGemvMaxRows];
#pragma unroll
    for (int u = 0; u < kSteps; u++)
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        const int i = row0 + w * rpw + r, q = q0 + 32 * u;
        m[u][r] = (r < rpw && i < row1 && q < K4) ? M4[(size_t)i * K4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
    for (int u = 0; u < kSteps; u++) {
      const int q = q0 + 32 * u;
      const float4 x = q < K4 ? v4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        if (r < rpw) {
          re[r] = fmaf(m[u][r].x, x.x, re[r]);
          re[r] = fmaf(-m[u][r].y, x.y, re[r]);
          re[r] = fmaf(m[u][r].z, x.z, re[r]);
          re[r] = fmaf(-m[u][r].w, x.w, re[r]);
          im[r] = fmaf(m[u][r].x, x.y, im[r]);
          im[r] = fmaf(m[u][r].y, x.x, im[r]);
          im[r] = fmaf(m[u][r].z, x.w, im[r]);
          im[r] = fmaf(m[u][r].w, x.z, im[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvMaxRows; r++) {
    if (r < rpw) res[r] = make_float2(gemv_wsum(re[r]), gemv_wsum(im[r]));
  }
}

__device__ __forceinline__ void warp_gemv(const float2* __restrict__ M, int nrows, int K, const float2* v, int w,
                                          int rpw, int lane, float2 res[kGemvMaxRows]) {
  warp_gemv_rows(M, 0, nrows, K, v, w, rpw, lane, res);
}

}  // namespace mg
