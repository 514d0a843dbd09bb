// Minimal-residual smoothing on the fine level, fused (section "Adaptive
// multigrid": the cycle's smoother; FP32, like the rest of the cycle).
//
// One MR step on D_r y = y - H_eo A_o^{-1} H_oe A_e^{-1} y with residual r:
//   w = D_r r,  alpha = <w, r> / <w, w>,  e += alpha r,  r -= alpha w.
// The unfused step runs five kernels (clover apply, two dslash, the two-dot
// reduction, the update).  Here it runs three:
//   k_dslash<EPI_CH>               t_o = A_o^{-1} H_oe s_e       (s_e = A_e^{-1} r_e)
//   k_mr_dslash_dot                w_e = r_e - H_eo t_o, and <w, w>, <w, r>
//   k_mr_update_clover             e += alpha r, r -= alpha w, s_e = A_e^{-1} r_e
// The clover product A_e^{-1} r of the next step is taken from the update
// (site-local), and the two inner products from the dslash epilogue (w and r
// are in registers there).  Sums: FP32 per site (12 components), FP64 across
// sites, per-block partials added by the last block in a fixed order, so the
// result does not depend on block scheduling.
#include "internal.h"
#include "wilson_dev.cuh"

namespace mg {
namespace {

constexpr int kMRThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// the three sums of the CTA into partials[blockIdx.x][0..2]; the last CTA to
// finish adds all partials in block order into out[0..2] and resets the counter
__device__ void mr_reduce3(double v0, double v1, double v2, double* partials, unsigned* counter, double* out) {
  __shared__ double sm[3][kMRThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v[3] = {v0, v1, v2};
#pragma unroll
  for (int q = 0; q < 3; q++) {
    const double t = warp_sum_d(v[q]);
    if (lane == 0) sm[q][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kMRThreads / 32; w++) t += sm[threadIdx.x][w];
    partials[(size_t)blockIdx.x * 3 + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 3; q++) t[q] += __ldcg(&partials[(size_t)b * 3 + q]);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; q++) {
    const double s = warp_sum_d(t[q]);
    if (lane == 0) sm[q][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kMRThreads / 32; w++) s += sm[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// w_e = r_e - H_eo t_o on even sites (grid-stride over sites), with
// out[0] = <w, w>, out[1] + i out[2] = <w, r> = sum conj(w) r
__global__ void __launch_bounds__(kMRThreads) k_mr_dslash_dot(Geom g, float* __restrict__ w, const float* __restrict__ t,
                                                              const float* __restrict__ gauge,
                                                              const float* __restrict__ r, double* partials,
                                                              unsigned* counter, double* out) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x) {
    int c[4];
    cb_coords(g, i, 0, c);
    cx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = mkc<float>(0.f, 0.f);
    hop_sum<float>(g, t, gauge, 0, i, c, 0xff, acc);
    cx<float> rv[12], wv[12];
    SpinorIO<float>::load(r, g.Vh, i, rv);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      // r - H_eo t with H = -1/2 sum (1 -+ gamma) U shift: r + acc / 2
      wv[k] = mkc(rv[k].re + 0.5f * acc[k].re, rv[k].im + 0.5f * acc[k].im);
      a0 = fmaf(wv[k].re, wv[k].re, fmaf(wv[k].im, wv[k].im, a0));
      a1 = fmaf(wv[k].re, rv[k].re, fmaf(wv[k].im, rv[k].im, a1));
      a2 = fmaf(wv[k].re, rv[k].im, fmaf(-wv[k].im, rv[k].re, a2));
    }
    SpinorIO<float>::store(w, g.Vh, i, wv);
    s0 += a0;
    s1 += a1;
    s2 += a2;
  }
  mr_reduce3(s0, s1, s2, partials, counter, out);
}

// e += alpha r, r -= alpha w (alpha = in[1..2] / in[0]), and s = A_e^{-1} r
// of the updated r on even sites
__global__ void __launch_bounds__(128) k_mr_update_clover(Geom g, float* __restrict__ e, float* __restrict__ r,
                                                          const float* __restrict__ w, const double* __restrict__ in,
                                                          const float* __restrict__ clov, float* __restrict__ s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Vh) return;
  const double ww = in[0] > 0 ? in[0] : 1.0;
  const float ar = (float)(in[1] / ww), ai = (float)(in[2] / ww);
  cx<float> ev[12], rv[12], wv[12], sv[12];
  SpinorIO<float>::load(e, g.Vh, i, ev);
  SpinorIO<float>::load(r, g.Vh, i, rv);
  SpinorIO<float>::load(w, g.Vh, i, wv);
#pragma unroll
  for (int k = 0; k < 12; k++) {
    ev[k].re += ar * rv[k].re - ai * rv[k].im;
    ev[k].im += ar * rv[k].im + ai * rv[k].re;
    rv[k].re -= ar * wv[k].re - ai * wv[k].im;
    rv[k].im -= ar * wv[k].im + ai * wv[k].re;
  }
  SpinorIO<float>::store(e, g.Vh, i, ev);
  SpinorIO<float>::store(r, g.Vh, i, rv);
  clover_mul<float>(clov, g.Vh, i, rv, sv);
  SpinorIO<float>::store(s, g.Vh, i, sv);
}

}  // namespace

void mr_smooth_fine(Ctx* c, float* e, float* r, float* w, float* s, float* t, int nu, double* d_scr) {
  const Geom& g = c->g;
  const size_t n = 12 * c->Vh;
  cudaStream_t st = c->stream;
  blas_zero<float>(e, n, st);
  if (nu <= 0) return;
  clover_apply<float>(g, s, r, c->Ainv<float>(0), st);   // s_e = A_e^{-1} r_e
  const int grid_dot = (int)std::min<long long>(Workspace::kMaxBlocks, ((long long)c->Vh + kMRThreads - 1) / kMRThreads);
  for (int it = 0; it < nu; it++) {
    dslash<float>(g, EPI_CH, 1, t, s, c->gauge<float>(), c->Ainv<float>(1), nullptr, 0.0, 0xff, st);
    k_mr_dslash_dot<<<grid_dot, kMRThreads, 0, st>>>(g, w, t, c->gauge<float>(), r, c->ws.partials.as<double>(),
                                                     c->ws.counter.as<unsigned>(), d_scr);
    MG_LAUNCH();
    c->dslash_launches += 2;
    if (it + 1 < nu) {
      k_mr_update_clover<<<(c->Vh + 127) / 128, 128, 0, st>>>(g, e, r, w, d_scr, c->Ainv<float>(0), s);
      MG_LAUNCH();
    } else {
      blas_mr_update<float>(e, r, w, d_scr, n, st);
    }
  }
}

}  // namespace mg
