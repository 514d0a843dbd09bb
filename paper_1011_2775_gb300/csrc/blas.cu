// BLAS-1 kernels and deterministic reductions for the GCR solvers
// (section "Adaptive multigrid": GCR is the outer solver; section
// "Implementation": GCR again on every coarse level).
//
// All inner products accumulate in FP64 regardless of the vector precision.
// Reductions are deterministic: a fixed grid (a function of n only), per-block
// partials written to the workspace, and an ordered final sum by the last
// block to finish (threadfence + atomic ticket).  The GCR kernels fuse the
// orthogonalisation update with the norms it needs and read their
// coefficients from device memory, so a GCR iteration needs no host round
// trip except the optional convergence check.
#include "internal.h"

namespace mg {

namespace {
constexpr int kBS = 256;

inline int red_grid(size_t n) {
  size_t b = (n + kBS - 1) / kBS;
  if (b < 1) b = 1;
  if (b > (size_t)Workspace::kMaxBlocks) b = Workspace::kMaxBlocks;
  return (int)b;
}
inline int ew_grid(size_t n) {
  size_t b = (n + kBS - 1) / kBS;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce v[0..NR) then finish the grid reduction deterministically.
template <int NR>
__device__ __forceinline__ void grid_reduce(double (&v)[NR], double* partials, unsigned* counter, double* out) {
  __shared__ double sm[NR > 0 ? NR : 1][kBS / 32];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int r = 0; r < NR; r++) {
    double t = warp_sum(v[r]);
    if (lane == 0) sm[r][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int r = 0; r < NR; r++) {
      double t = lane < nw ? sm[r][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) partials[(size_t)blockIdx.x * NR + r] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
#pragma unroll
  for (int r = 0; r < NR; r++) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(&partials[(size_t)b * NR + r]);
    t = warp_sum(t);
    __syncthreads();
    if (lane == 0) sm[r][wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; w++) s += sm[r][w];
      out[r] = s;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

template <typename T>
struct VecPtrs {
  const cx<T>* p[8];
};

// Per-thread accumulation type: a thread sums only its few grid-stride
// elements, in the vectors' own precision (FP64 for FP64 vectors); the
// cross-thread tree is always FP64.  On GB300 this keeps the FP32 reductions
// off the (slow) FP64 pipe.
template <typename T>
using acc_t = typename std::conditional<sizeof(T) == 4, float, double>::type;
}  // namespace

// --------------------------------------------------------------------------- elementwise
template <typename T>
__global__ void k_zero(cx<T>* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = mkc<T>(0, 0);
}
template <typename T>
void blas_zero(T* x, size_t n, cudaStream_t s) {
  k_zero<T><<<ew_grid(n), kBS, 0, s>>>((cx<T>*)x, n);
  MG_LAUNCH();
}

template <typename TI, typename TO>
__global__ void k_convert(cx<TO>* y, const cx<TI>* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = mkc<TO>((TO)x[i].re, (TO)x[i].im);
}
template <typename TI, typename TO>
void blas_convert(TO* y, const TI* x, size_t n, cudaStream_t s) {
  k_convert<TI, TO><<<ew_grid(n), kBS, 0, s>>>((cx<TO>*)y, (const cx<TI>*)x, n);
  MG_LAUNCH();
}

template <typename T>
__global__ void k_axpby(T a, const cx<T>* __restrict__ x, T b, cx<T>* y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> xv = x[i], yv = y[i];
    y[i] = mkc<T>(a * xv.re + b * yv.re, a * xv.im + b * yv.im);
  }
}
template <typename T>
void blas_axpby(double a, const T* x, double b, T* y, size_t n, cudaStream_t s) {
  k_axpby<T><<<ew_grid(n), kBS, 0, s>>>((T)a, (const cx<T>*)x, (T)b, (cx<T>*)y, n);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- reductions
template <typename T>
__global__ void k_norm2(const cx<T>* __restrict__ x, size_t n, double* partials, unsigned* counter, double* out) {
  acc_t<T> s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = x[i];
    s = fma((acc_t<T>)a.re, (acc_t<T>)a.re, s);
    s = fma((acc_t<T>)a.im, (acc_t<T>)a.im, s);
  }
  double v[1] = {(double)s};
  grid_reduce<1>(v, partials, counter, out);
}
template <typename T>
void blas_norm2(const T* x, size_t n, double* d_out, Workspace& ws, cudaStream_t s) {
  k_norm2<T><<<red_grid(n), kBS, 0, s>>>((const cx<T>*)x, n, ws.partials.as<double>(), ws.counter.as<unsigned>(), d_out);
  MG_LAUNCH();
}

template <typename T>
__global__ void k_cdot(const cx<T>* __restrict__ x, const cx<T>* __restrict__ y, size_t n, double* partials,
                       unsigned* counter, double* out) {
  acc_t<T> s0 = 0, s1 = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = x[i], b = y[i];
    s0 = fma((acc_t<T>)a.re, (acc_t<T>)b.re, s0);
    s0 = fma((acc_t<T>)a.im, (acc_t<T>)b.im, s0);
    s1 = fma((acc_t<T>)a.re, (acc_t<T>)b.im, s1);
    s1 = fma(-(acc_t<T>)a.im, (acc_t<T>)b.re, s1);
  }
  double v[2] = {(double)s0, (double)s1};
  grid_reduce<2>(v, partials, counter, out);
}
template <typename T>
void blas_cdot(const T* x, const T* y, size_t n, double* d_out, Workspace& ws, cudaStream_t s) {
  k_cdot<T><<<red_grid(n), kBS, 0, s>>>((const cx<T>*)x, (const cx<T>*)y, n, ws.partials.as<double>(),
                                        ws.counter.as<unsigned>(), d_out);
  MG_LAUNCH();
}

template <typename T>
__global__ void k_dot2(const cx<T>* __restrict__ w, const cx<T>* __restrict__ r, size_t n, double* partials,
                       unsigned* counter, double* out) {
  acc_t<T> s0 = 0, s1 = 0, s2 = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = w[i], b = r[i];
    s0 = fma((acc_t<T>)a.re, (acc_t<T>)a.re, s0);
    s0 = fma((acc_t<T>)a.im, (acc_t<T>)a.im, s0);
    s1 = fma((acc_t<T>)a.re, (acc_t<T>)b.re, s1);
    s1 = fma((acc_t<T>)a.im, (acc_t<T>)b.im, s1);
    s2 = fma((acc_t<T>)a.re, (acc_t<T>)b.im, s2);
    s2 = fma(-(acc_t<T>)a.im, (acc_t<T>)b.re, s2);
  }
  double v[3] = {(double)s0, (double)s1, (double)s2};
  grid_reduce<3>(v, partials, counter, out);
}
// nrhs pairs (w_q, r_q) at `stride` complex apart: d_out[4q .. 4q+2] per pair,
// one launch (blockIdx.y = q, a separate reduction per pair)
template <typename T>
__global__ void k_dot2_multi(const cx<T>* __restrict__ w, const cx<T>* __restrict__ r, size_t n, size_t stride,
                             double* partials, unsigned* counters, double* out) {
  const int q = blockIdx.y;
  w += q * stride;
  r += q * stride;
  acc_t<T> s0 = 0, s1 = 0, s2 = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = w[i], b = r[i];
    s0 = fma((acc_t<T>)a.re, (acc_t<T>)a.re, s0);
    s0 = fma((acc_t<T>)a.im, (acc_t<T>)a.im, s0);
    s1 = fma((acc_t<T>)a.re, (acc_t<T>)b.re, s1);
    s1 = fma((acc_t<T>)a.im, (acc_t<T>)b.im, s1);
    s2 = fma((acc_t<T>)a.re, (acc_t<T>)b.im, s2);
    s2 = fma(-(acc_t<T>)a.im, (acc_t<T>)b.re, s2);
  }
  double v[3] = {(double)s0, (double)s1, (double)s2};
  grid_reduce<3>(v, partials + (size_t)q * gridDim.x * 3, counters + q, out + 4 * q);
}
template <typename T>
void blas_dot2_multi(const T* w, const T* r, size_t n, size_t stride, int nrhs, double* d_out, Workspace& ws,
                     cudaStream_t s) {
  if (nrhs > Workspace::kMultiCounters) raise(MG_ERR_ARG, "too many vectors for one multi-reduction");
  int g = red_grid(n);
  const int cap = Workspace::kMaxBlocks * Workspace::kMaxResults / (3 * nrhs);
  if (g > cap) g = cap;
  k_dot2_multi<T><<<dim3(g, nrhs), kBS, 0, s>>>((const cx<T>*)w, (const cx<T>*)r, n, stride / 2,
                                                 ws.partials.as<double>(), ws.mcounters.as<unsigned>(), d_out);
  MG_LAUNCH();
}

template <typename T>
__global__ void k_mr_update_multi(cx<T>* e, cx<T>* r, const cx<T>* __restrict__ w, const double* __restrict__ in,
                                  size_t n, size_t stride) {
  const int q = blockIdx.y;
  e += q * stride;
  r += q * stride;
  w += q * stride;
  in += 4 * q;
  const double ww = in[0] > 0 ? in[0] : 1.0;
  const T ar = (T)(in[1] / ww), ai = (T)(in[2] / ww);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> rv = r[i], wv = w[i], ev = e[i];
    ev.re += ar * rv.re - ai * rv.im;
    ev.im += ar * rv.im + ai * rv.re;
    rv.re -= ar * wv.re - ai * wv.im;
    rv.im -= ar * wv.im + ai * wv.re;
    e[i] = ev;
    r[i] = rv;
  }
}
template <typename T>
void blas_mr_update_multi(T* e, T* r, const T* w, const double* d_in, size_t n, size_t stride, int nrhs,
                          cudaStream_t s) {
  int g = ew_grid(n);
  if (g * nrhs > 152 * 16) g = (152 * 16 + nrhs - 1) / nrhs;
  k_mr_update_multi<T><<<dim3(g, nrhs), kBS, 0, s>>>((cx<T>*)e, (cx<T>*)r, (const cx<T>*)w, d_in, n, stride / 2);
  MG_LAUNCH();
}
template void blas_dot2_multi<float>(const float*, const float*, size_t, size_t, int, double*, Workspace&, cudaStream_t);
template void blas_mr_update_multi<float>(float*, float*, const float*, const double*, size_t, size_t, int,
                                          cudaStream_t);

template <typename T>
void blas_dot2(const T* w, const T* r, size_t n, double* d_out, Workspace& ws, cudaStream_t s) {
  k_dot2<T><<<red_grid(n), kBS, 0, s>>>((const cx<T>*)w, (const cx<T>*)r, n, ws.partials.as<double>(),
                                        ws.counter.as<unsigned>(), d_out);
  MG_LAUNCH();
}

// d_out[2j..] = <V_j, w>, j < K
template <typename T, int K>
__global__ void k_multidot(VecPtrs<T> V, const cx<T>* __restrict__ w, size_t n, double* partials, unsigned* counter,
                           double* out) {
  acc_t<T> s[2 * K];
#pragma unroll
  for (int r = 0; r < 2 * K; r++) s[r] = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> b = w[i];
#pragma unroll
    for (int j = 0; j < K; j++) {
      cx<T> a = V.p[j][i];
      s[2 * j] = fma((acc_t<T>)a.re, (acc_t<T>)b.re, s[2 * j]);
      s[2 * j] = fma((acc_t<T>)a.im, (acc_t<T>)b.im, s[2 * j]);
      s[2 * j + 1] = fma((acc_t<T>)a.re, (acc_t<T>)b.im, s[2 * j + 1]);
      s[2 * j + 1] = fma(-(acc_t<T>)a.im, (acc_t<T>)b.re, s[2 * j + 1]);
    }
  }
  double v[2 * K];
#pragma unroll
  for (int r = 0; r < 2 * K; r++) v[r] = (double)s[r];
  grid_reduce<2 * K>(v, partials, counter, out);
}

template <typename T>
void blas_multidot(const T* const* V, int k, const T* w, size_t n, double* d_out, Workspace& ws, cudaStream_t s) {
  for (int j0 = 0; j0 < k; j0 += 8) {
    const int kk = (k - j0) < 8 ? (k - j0) : 8;
    VecPtrs<T> P;
    for (int j = 0; j < 8; j++) P.p[j] = (const cx<T>*)(j < kk ? V[j0 + j] : V[j0]);
    double* o = d_out + 2 * j0;
    const int grid = red_grid(n);
    double* pa = ws.partials.as<double>();
    unsigned* ct = ws.counter.as<unsigned>();
    const cx<T>* wp = (const cx<T>*)w;
    switch (kk) {
      case 1: k_multidot<T, 1><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      case 2: k_multidot<T, 2><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      case 3: k_multidot<T, 3><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      case 4: k_multidot<T, 4><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      case 5: k_multidot<T, 5><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      case 6: k_multidot<T, 6><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      case 7: k_multidot<T, 7><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
      default: k_multidot<T, 8><<<grid, kBS, 0, s>>>(P, wp, n, pa, ct, o); break;
    }
    MG_LAUNCH();
  }
}

// w -= sum_{j<K} beta_j V_j; if RED: {||w||^2, <w, r>} -> out
template <typename T, int K, bool RED>
__global__ void k_orth_update(cx<T>* w, VecPtrs<T> V, const double* __restrict__ beta, const cx<T>* __restrict__ r,
                              size_t n, double* partials, unsigned* counter, double* out) {
  T br[K > 0 ? K : 1], bi[K > 0 ? K : 1];
#pragma unroll
  for (int j = 0; j < K; j++) {
    br[j] = (T)beta[2 * j];
    bi[j] = (T)beta[2 * j + 1];
  }
  acc_t<T> s0 = 0, s1 = 0, s2 = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = w[i];
#pragma unroll
    for (int j = 0; j < K; j++) {
      cx<T> q = V.p[j][i];
      a.re -= br[j] * q.re - bi[j] * q.im;
      a.im -= br[j] * q.im + bi[j] * q.re;
    }
    if (K > 0) w[i] = a;
    if (RED) {
      cx<T> b = r[i];
      s0 = fma((acc_t<T>)a.re, (acc_t<T>)a.re, s0);
      s0 = fma((acc_t<T>)a.im, (acc_t<T>)a.im, s0);
      s1 = fma((acc_t<T>)a.re, (acc_t<T>)b.re, s1);
      s1 = fma((acc_t<T>)a.im, (acc_t<T>)b.im, s1);
      s2 = fma((acc_t<T>)a.re, (acc_t<T>)b.im, s2);
      s2 = fma(-(acc_t<T>)a.im, (acc_t<T>)b.re, s2);
    }
  }
  double v[3] = {(double)s0, (double)s1, (double)s2};
  if (RED) grid_reduce<3>(v, partials, counter, out);
}

template <typename T>
void blas_orth_update(T* w, const T* const* V, const double* d_beta, int k, const T* r, size_t n, double* d_out,
                      Workspace& ws, cudaStream_t s) {
  const int grid = red_grid(n);
  double* pa = ws.partials.as<double>();
  unsigned* ct = ws.counter.as<unsigned>();
  cx<T>* wp = (cx<T>*)w;
  const cx<T>* rp = (const cx<T>*)r;
  if (k == 0) {
    VecPtrs<T> P{};
    k_orth_update<T, 0, true><<<grid, kBS, 0, s>>>(wp, P, d_beta, rp, n, pa, ct, d_out);
    MG_LAUNCH();
    return;
  }
  for (int j0 = 0; j0 < k; j0 += 8) {
    const int kk = (k - j0) < 8 ? (k - j0) : 8;
    const bool last = j0 + kk >= k;
    VecPtrs<T> P;
    for (int j = 0; j < 8; j++) P.p[j] = (const cx<T>*)(j < kk ? V[j0 + j] : V[j0]);
    const double* b = d_beta + 2 * j0;
#define MG_ORTH_CASE(KK)                                                                         \
  case KK:                                                                                       \
    if (last)                                                                                    \
      k_orth_update<T, KK, true><<<grid, kBS, 0, s>>>(wp, P, b, rp, n, pa, ct, d_out);           \
    else                                                                                         \
      k_orth_update<T, KK, false><<<grid, kBS, 0, s>>>(wp, P, b, rp, n, pa, ct, d_out);          \
    break;
    switch (kk) {
      MG_ORTH_CASE(1)
      MG_ORTH_CASE(2)
      MG_ORTH_CASE(3)
      MG_ORTH_CASE(4)
      MG_ORTH_CASE(5)
      MG_ORTH_CASE(6)
      MG_ORTH_CASE(7)
      default:
        if (last)
          k_orth_update<T, 8, true><<<grid, kBS, 0, s>>>(wp, P, b, rp, n, pa, ct, d_out);
        else
          k_orth_update<T, 8, false><<<grid, kBS, 0, s>>>(wp, P, b, rp, n, pa, ct, d_out);
    }
#undef MG_ORTH_CASE
    MG_LAUNCH();
  }
}

template <typename T>
__global__ void k_r_update(cx<T>* w, cx<T>* r, size_t n, const double* __restrict__ in, double* alpha_out,
                           double* gamma_out, double* partials, unsigned* counter, double* out) {
  const double g2 = in[0];
  const double gam = g2 > 0 ? sqrt(g2) : 1.0;
  const double ar = in[1] / gam, ai = in[2] / gam;  // alpha = <w/gamma, r>
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    alpha_out[0] = ar;
    alpha_out[1] = ai;
    gamma_out[0] = gam;
  }
  const T ig = (T)(1.0 / gam), a_r = (T)ar, a_i = (T)ai;
  acc_t<T> s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> q = w[i];
    q.re *= ig;
    q.im *= ig;
    w[i] = q;
    cx<T> b = r[i];
    b.re -= a_r * q.re - a_i * q.im;
    b.im -= a_r * q.im + a_i * q.re;
    r[i] = b;
    s = fma((acc_t<T>)b.re, (acc_t<T>)b.re, s);
    s = fma((acc_t<T>)b.im, (acc_t<T>)b.im, s);
  }
  double v[1] = {(double)s};
  grid_reduce<1>(v, partials, counter, out);
}

template <typename T>
void blas_r_update(T* w, T* r, size_t n, const double* d_in, double* d_alpha, double* d_gamma, double* d_rnorm2,
                   Workspace& ws, cudaStream_t s) {
  k_r_update<T><<<red_grid(n), kBS, 0, s>>>((cx<T>*)w, (cx<T>*)r, n, d_in, d_alpha, d_gamma, ws.partials.as<double>(),
                                            ws.counter.as<unsigned>(), d_rnorm2);
  MG_LAUNCH();
}

template <typename T, typename TZ, int K>
__global__ void k_lincomb(cx<T>* x, VecPtrs<TZ> Z, const double* __restrict__ c, double scale, size_t n) {
  double cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; j++) {
    cr[j] = scale * c[2 * j];
    ci[j] = scale * c[2 * j + 1];
  }
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = x[i];
    double re = (double)a.re, im = (double)a.im;
#pragma unroll
    for (int j = 0; j < K; j++) {
      cx<TZ> z = Z.p[j][i];
      re += cr[j] * (double)z.re - ci[j] * (double)z.im;
      im += cr[j] * (double)z.im + ci[j] * (double)z.re;
    }
    x[i] = mkc<T>((T)re, (T)im);
  }
}

template <typename T, typename TZ>
void blas_lincomb(T* x, const TZ* const* Z, const double* d_c, int k, double scale, size_t n, cudaStream_t s) {
  for (int j0 = 0; j0 < k; j0 += 8) {
    const int kk = (k - j0) < 8 ? (k - j0) : 8;
    VecPtrs<TZ> P;
    for (int j = 0; j < 8; j++) P.p[j] = (const cx<TZ>*)(j < kk ? Z[j0 + j] : Z[j0]);
    const double* c = d_c + 2 * j0;
    const int grid = ew_grid(n);
    cx<T>* xp = (cx<T>*)x;
    switch (kk) {
      case 1: k_lincomb<T, TZ, 1><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      case 2: k_lincomb<T, TZ, 2><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      case 3: k_lincomb<T, TZ, 3><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      case 4: k_lincomb<T, TZ, 4><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      case 5: k_lincomb<T, TZ, 5><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      case 6: k_lincomb<T, TZ, 6><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      case 7: k_lincomb<T, TZ, 7><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
      default: k_lincomb<T, TZ, 8><<<grid, kBS, 0, s>>>(xp, P, c, scale, n); break;
    }
    MG_LAUNCH();
  }
}

__global__ void k_backsub(const double* beta, int ld, const double* alpha, const double* gamma, int k, double* c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = k - 1; j >= 0; j--) {
    double re = alpha[2 * j], im = alpha[2 * j + 1];
    for (int l = j + 1; l < k; l++) {
      const double br = beta[(j + (size_t)ld * l) * 2], bi = beta[(j + (size_t)ld * l) * 2 + 1];
      const double cr = c[2 * l], ci = c[2 * l + 1];
      re -= br * cr - bi * ci;
      im -= br * ci + bi * cr;
    }
    c[2 * j] = re / gamma[j];
    c[2 * j + 1] = im / gamma[j];
  }
}

void gcr_backsub(const double* d_beta, int ld, const double* d_alpha, const double* d_gamma, int k, double* d_c,
                 cudaStream_t s) {
  k_backsub<<<1, 32, 0, s>>>(d_beta, ld, d_alpha, d_gamma, k, d_c);
  MG_LAUNCH();
}

template <typename T>
__global__ void k_mr_update(cx<T>* e, cx<T>* r, const cx<T>* __restrict__ w, const double* __restrict__ in, size_t n) {
  const double ww = in[0] > 0 ? in[0] : 1.0;
  const T ar = (T)(in[1] / ww), ai = (T)(in[2] / ww);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> rv = r[i], wv = w[i], ev = e[i];
    ev.re += ar * rv.re - ai * rv.im;
    ev.im += ar * rv.im + ai * rv.re;
    rv.re -= ar * wv.re - ai * wv.im;
    rv.im -= ar * wv.im + ai * wv.re;
    e[i] = ev;
    r[i] = rv;
  }
}
template <typename T>
void blas_mr_update(T* e, T* r, const T* w, const double* d_in, size_t n, cudaStream_t s) {
  k_mr_update<T><<<ew_grid(n), kBS, 0, s>>>((cx<T>*)e, (cx<T>*)r, (const cx<T>*)w, d_in, n);
  MG_LAUNCH();
}

template <typename T>
__global__ void k_normalize(cx<T>* x, const double* __restrict__ nrm2, size_t n) {
  const T f = (T)(nrm2[0] > 0 ? 1.0 / sqrt(nrm2[0]) : 1.0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<T> a = x[i];
    x[i] = mkc<T>(a.re * f, a.im * f);
  }
}
template <typename T>
void blas_normalize(T* x, const double* d_norm2, size_t n, cudaStream_t s) {
  k_normalize<T><<<ew_grid(n), kBS, 0, s>>>((cx<T>*)x, d_norm2, n);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- instantiations
#define MG_INST(T)                                                                                             \
  template void blas_zero<T>(T*, size_t, cudaStream_t);                                                        \
  template void blas_axpby<T>(double, const T*, double, T*, size_t, cudaStream_t);                             \
  template void blas_norm2<T>(const T*, size_t, double*, Workspace&, cudaStream_t);                            \
  template void blas_cdot<T>(const T*, const T*, size_t, double*, Workspace&, cudaStream_t);                   \
  template void blas_dot2<T>(const T*, const T*, size_t, double*, Workspace&, cudaStream_t);                   \
  template void blas_multidot<T>(const T* const*, int, const T*, size_t, double*, Workspace&, cudaStream_t);   \
  template void blas_orth_update<T>(T*, const T* const*, const double*, int, const T*, size_t, double*,        \
                                    Workspace&, cudaStream_t);                                                 \
  template void blas_r_update<T>(T*, T*, size_t, const double*, double*, double*, double*, Workspace&,         \
                                 cudaStream_t);                                                                \
  template void blas_mr_update<T>(T*, T*, const T*, const double*, size_t, cudaStream_t);                      \
  template void blas_normalize<T>(T*, const double*, size_t, cudaStream_t);
MG_INST(float)
MG_INST(double)
#undef MG_INST
template void blas_convert<float, double>(double*, const float*, size_t, cudaStream_t);
template void blas_convert<double, float>(float*, const double*, size_t, cudaStream_t);
template void blas_convert<float, float>(float*, const float*, size_t, cudaStream_t);
template void blas_convert<double, double>(double*, const double*, size_t, cudaStream_t);
template void blas_lincomb<double, float>(double*, const float* const*, const double*, int, double, size_t,
                                          cudaStream_t);
template void blas_lincomb<double, double>(double*, const double* const*, const double*, int, double, size_t,
                                           cudaStream_t);
template void blas_lincomb<float, float>(float*, const float* const*, const double*, int, double, size_t,
                                         cudaStream_t);

}  // namespace mg
