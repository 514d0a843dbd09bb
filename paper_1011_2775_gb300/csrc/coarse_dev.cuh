// Row-parallel complex GEMV used by the coarse stencil kernels.
//
// A CTA owns one coarse site; warp w owns rows [w*rpw, (w+1)*rpw) of the
// site's link block (row-major, K complex per row).  The lanes stride over
// the row in float4 units (two complex numbers), and every lane keeps one
// accumulator per owned row, so each step issues rpw independent 16-byte
// loads per lane and every warp load instruction reads 512 contiguous bytes.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"

namespace mg {

constexpr int kGemvMaxRows = 8;  // rows per warp (nc <= 64 with 8 warps)

__device__ __forceinline__ float gemv_wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Storage formats of link blocks (the values of mg::Store): FP32 complex
// (8 bytes) or FP16 / BF16 complex (4 bytes), the latter multiplied by a
// per-tile scale that the callers fold into the vector.
constexpr int kStF32 = 0, kStF16 = 1, kStBF16 = 2;
template <int ST>
constexpr size_t link_bytes() { return ST == kStF32 ? 8 : 4; }

// complex pair q (elements 2q, 2q+1) of a link row: loaded raw (16 bytes
// FP32, 8 bytes FP16/BF16) and decoded to {re0, im0, re1, im1} where used, so
// that the loads in flight hold no more registers than the FP32 ones
template <int ST>
struct LinkPair {
  using raw = typename std::conditional<ST == kStF32, float4, uint2>::type;
  static __device__ __forceinline__ raw load(const void* M, size_t q) { return reinterpret_cast<const raw*>(M)[q]; }
  static __device__ __forceinline__ raw zero() {
    raw z;
    memset(&z, 0, sizeof(z));
    return z;
  }
  static __device__ __forceinline__ float4 decode(const raw& u) {
    if constexpr (ST == kStF32) {
      return u;
    } else {
      float2 a, b;
      if constexpr (ST == kStF16) {
        a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
      } else {
        a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
      }
      return make_float4(a.x, a.y, b.x, b.y);
    }
  }
};

// res[r] = sum_k M[row_r][k] * v[k] for the warp's rows row_r = row0 + w*rpw + r
// (r < rpw, row_r < row1).  M: global, storage format ST, row stride K
// complex (K even; rows 16-byte (FP32) / 8-byte (FP16, BF16) aligned); v:
// shared memory, K complex, 16-byte aligned.  After the call every lane holds
// the full sums.
template <int ST = kStF32>
__device__ __forceinline__ void warp_gemv_rows(const void* __restrict__ M, int row0, int row1, int K,
                                               const float2* v, int w, int rpw, int lane,
                                               float2 res[kGemvMaxRows]) {
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const int K4 = K >> 1;
  float re[kGemvMaxRows], im[kGemvMaxRows];
#pragma unroll
  for (int r = 0; r < kGemvMaxRows; r++) re[r] = im[r] = 0.f;
  // batches of kSteps lane-steps: all loads of a batch are issued before any
  // is used, so a warp has up to kSteps * rpw loads in flight per lane
  // (twice as many steps for the 8-byte loads of 16-bit links)
  constexpr int kSteps = ST == kStF32 ? 2 : 4;
  for (int q0 = lane; q0 < K4; q0 += 32 * kSteps) {
    typename LinkPair<ST>::raw m[kSteps][kGemvMaxRows];
#pragma unroll
    for (int u = 0; u < kSteps; u++)
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        const int i = row0 + w * rpw + r, q = q0 + 32 * u;
        m[u][r] = (r < rpw && i < row1 && q < K4) ? LinkPair<ST>::load(M, (size_t)i * K4 + q) : LinkPair<ST>::zero();
      }
#pragma unroll
    for (int u = 0; u < kSteps; u++) {
      const int q = q0 + 32 * u;
      const float4 x = q < K4 ? v4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        if (r < rpw) {
          const float4 a = LinkPair<ST>::decode(m[u][r]);
          re[r] = fmaf(a.x, x.x, re[r]);
          re[r] = fmaf(-a.y, x.y, re[r]);
          re[r] = fmaf(a.z, x.z, re[r]);
          re[r] = fmaf(-a.w, x.w, re[r]);
          im[r] = fmaf(a.x, x.y, im[r]);
          im[r] = fmaf(a.y, x.x, im[r]);
          im[r] = fmaf(a.z, x.w, im[r]);
          im[r] = fmaf(a.w, x.z, im[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvMaxRows; r++) {
    if (r < rpw) res[r] = make_float2(gemv_wsum(re[r]), gemv_wsum(im[r]));
  }
}

// Multi-vector form for RB consecutive rows i0 .. i0+RB-1 (rows >= nrows are
// skipped): res[r][p] = sum_k M[i0+r][k] * v_p[k] for np <= PB vectors
// v_p = v + p * vstride (shared memory, vstride complex, even).  Each link
// pair is loaded once and applied to all np vectors; callers loop over row
// blocks so that the accumulators stay at RB * PB complex numbers.
template <int ST, int RB, int PB>
__device__ __forceinline__ void warp_gemv_multi(const void* __restrict__ M, int i0, int nrows, int K,
                                                const float2* v, int vstride, int np, int lane,
                                                float2 res[RB][PB]) {
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const int K4 = K >> 1, vs4 = vstride >> 1;
  float re[RB][PB], im[RB][PB];
#pragma unroll
  for (int r = 0; r < RB; r++)
#pragma unroll
    for (int p = 0; p < PB; p++) re[r][p] = im[r][p] = 0.f;
  for (int q = lane; q < K4; q += 32) {
    float4 a[RB];
#pragma unroll
    for (int r = 0; r < RB; r++)
      a[r] = (i0 + r < nrows) ? LinkPair<ST>::decode(LinkPair<ST>::load(M, (size_t)(i0 + r) * K4 + q))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int p = 0; p < PB; p++) {
      if (p >= np) break;
      const float4 x = v4[p * vs4 + q];
#pragma unroll
      for (int r = 0; r < RB; r++) {
        re[r][p] = fmaf(a[r].x, x.x, re[r][p]);
        re[r][p] = fmaf(-a[r].y, x.y, re[r][p]);
        re[r][p] = fmaf(a[r].z, x.z, re[r][p]);
        re[r][p] = fmaf(-a[r].w, x.w, re[r][p]);
        im[r][p] = fmaf(a[r].x, x.y, im[r][p]);
        im[r][p] = fmaf(a[r].y, x.x, im[r][p]);
        im[r][p] = fmaf(a[r].z, x.w, im[r][p]);
        im[r][p] = fmaf(a[r].w, x.z, im[r][p]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RB; r++)
#pragma unroll
    for (int p = 0; p < PB; p++) res[r][p] = make_float2(gemv_wsum(re[r][p]), gemv_wsum(im[r][p]));
}

template <int ST = kStF32>
__device__ __forceinline__ void warp_gemv(const void* __restrict__ M, int nrows, int K, const float2* v, int w,
                                          int rpw, int lane, float2 res[kGemvMaxRows]) {
  warp_gemv_rows<ST>(M, 0, nrows, K, v, w, rpw, lane, res);
}

}  // namespace mg
