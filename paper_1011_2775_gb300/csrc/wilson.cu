// Fine-level Wilson-clover kernels for sm_103a.
//
//  * ABI <-> internal packing of spinors and gauge links
//  * clover construction A = (4+m0) + csw (i/4) sum_{mu!=nu} sigma_{mu nu} F_{mu nu}; anisotropic
//    reading: (sum_mu w_mu + m0) + (i/4) sum_{mu!=nu} c_{mu nu} sigma F with the hopping weights w_mu of the
//    directions and c = csw_t (planes containing t) or csw_s (spatial planes)
//    and its site inverse (FP64), the D_ee / D_oo of the paper's even-odd
//    split ("Red-black preconditioning": D_ee, D_oo are site-diagonal)
//  * the fused hopping kernel ("dslash") with clover / axpy epilogues, from
//    which D, D_p = 1 + H A^{-1}, D_r = 1 - H_eo A_o^{-1} H_oe A_e^{-1} and
//    b_r = b_e - H_eo A_o^{-1} b_o are composed
//  * the eight directional hopping terms (Galerkin coarse-link construction)
//  * Philox4x32-10 Gaussian start vectors of the null-vector setup
//
// One thread per lattice site; spinors, links and clover are read as
// 16-byte (float4 / double2) or 8-byte chunks in structure-of-chunks order so
// that a warp reads contiguous 512-byte spans.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "philox.cuh"
#include "wilson_dev.cuh"

namespace mg {

// --------------------------------------------------------------------------- sigma blocks
// sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] in the DeGrand-Rossi basis is
// block diagonal in chirality; c_sigma[plane][block][s][t] holds the 2x2
// blocks for the planes (01, 02, 03, 12, 13, 23).
__constant__ double c_sigma[6][2][2][2][2];

namespace {
struct HC {
  double re, im;
};
HC hmul(HC a, HC b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Uploads the table to the current device (every clover build: 384 bytes).
void upload_sigma() {
  // gamma_mu as 4x4 complex, rows of the DeGrand-Rossi table
  HC G[4][4][4] = {};
  auto set = [&](int mu, int r, int col, double re, double im) { G[mu][r][col] = {re, im}; };
  set(0, 0, 3, 0, 1); set(0, 1, 2, 0, 1); set(0, 2, 1, 0, -1); set(0, 3, 0, 0, -1);   // gamma_x
  set(1, 0, 3, -1, 0); set(1, 1, 2, 1, 0); set(1, 2, 1, 1, 0); set(1, 3, 0, -1, 0);   // gamma_y
  set(2, 0, 2, 0, 1); set(2, 1, 3, 0, -1); set(2, 2, 0, 0, -1); set(2, 3, 1, 0, 1);   // gamma_z
  set(3, 0, 2, 1, 0); set(3, 1, 3, 1, 0); set(3, 2, 0, 1, 0); set(3, 3, 1, 1, 0);     // gamma_t
  double host[6][2][2][2][2];
  int plane = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++, plane++) {
      HC S[4][4];
      for (int r = 0; r < 4; r++)
        for (int q = 0; q < 4; q++) {
          HC acc{0, 0};
          for (int k = 0; k < 4; k++) {
            HC a = hmul(G[mu][r][k], G[nu][k][q]);
            HC b = hmul(G[nu][r][k], G[mu][k][q]);
            acc.re += a.re - b.re;
            acc.im += a.im - b.im;
          }
          S[r][q] = {-0.5 * acc.im, 0.5 * acc.re};  // (i/2) * commutator
        }
      for (int b = 0; b < 2; b++)
        for (int s = 0; s < 2; s++)
          for (int t = 0; t < 2; t++) {
            host[plane][b][s][t][0] = S[2 * b + s][2 * b + t].re;
            host[plane][b][s][t][1] = S[2 * b + s][2 * b + t].im;
          }
      for (int s = 0; s < 2; s++)
        for (int t = 0; t < 2; t++)
          if (std::fabs(S[s][2 + t].re) + std::fabs(S[s][2 + t].im) > 1e-14)
            raise(MG_ERR_ARG, "sigma not block diagonal");
    }
  MG_CUDA(cudaMemcpyToSymbol(c_sigma, host, sizeof(host)));
}
}  // namespace

// --------------------------------------------------------------------------- packing
template <typename T>
__global__ void k_pack_spinor(Geom g, const double2* __restrict__ abi, T* even, T* odd) {
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= 2 * g.Vh) return;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int cb = lex >> 1;
  cx<T> s[12];
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 v = abi[(size_t)lex * 12 + k];
    s[k] = mkc<T>((T)v.x, (T)v.y);
  }
  SpinorIO<T>::store(par ? odd : even, g.Vh, cb, s);
}

template <typename T>
__global__ void k_unpack_spinor(Geom g, const T* even, const T* odd, double2* __restrict__ abi) {
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= 2 * g.Vh) return;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  cx<T> s[12];
  SpinorIO<T>::load(par ? odd : even, g.Vh, lex >> 1, s);
#pragma unroll
  for (int k = 0; k < 12; k++) abi[(size_t)lex * 12 + k] = make_double2((double)s[k].re, (double)s[k].im);
}

void pack_spinor(const Geom& g, const double* abi, void* even, void* odd, bool fp32, cudaStream_t s) {
  const int n = 2 * g.Vh, bs = 128;
  if (fp32)
    k_pack_spinor<float><<<(n + bs - 1) / bs, bs, 0, s>>>(g, (const double2*)abi, (float*)even, (float*)odd);
  else
    k_pack_spinor<double><<<(n + bs - 1) / bs, bs, 0, s>>>(g, (const double2*)abi, (double*)even, (double*)odd);
  MG_LAUNCH();
}

void unpack_spinor(const Geom& g, const void* even, const void* odd, bool fp32, double* abi, cudaStream_t s) {
  const int n = 2 * g.Vh, bs = 128;
  if (fp32)
    k_unpack_spinor<float><<<(n + bs - 1) / bs, bs, 0, s>>>(g, (const float*)even, (const float*)odd, (double2*)abi);
  else
    k_unpack_spinor<double><<<(n + bs - 1) / bs, bs, 0, s>>>(g, (const double*)even, (const double*)odd, (double2*)abi);
  MG_LAUNCH();
}

__global__ void k_pack_gauge(Geom g, const double2* __restrict__ abi, double2* g64, float2* g32) {
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= 2 * g.Vh) return;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int cb = lex >> 1;
  for (int mu = 0; mu < 4; mu++)
    for (int e = 0; e < 9; e++) {
      double2 v = abi[((size_t)lex * 4 + mu) * 9 + e];
      size_t o = ((size_t)(par * 4 + mu) * 9 + e) * g.Vh + cb;
      g64[o] = v;
      g32[o] = make_float2((float)v.x, (float)v.y);
    }
}

void pack_gauge(const Geom& g, const double* abi, double* g64, float* g32, cudaStream_t s) {
  const int n = 2 * g.Vh, bs = 128;
  k_pack_gauge<<<(n + bs - 1) / bs, bs, 0, s>>>(g, (const double2*)abi, (double2*)g64, (float2*)g32);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- clover construction
namespace {
typedef cx<double> cd;

__device__ void link_at(const Geom& g, const double* gauge, const int y[4], int mu, cd u[9]) {
  const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  load_link<double>(gauge, g.Vh, par, mu, cb_index(g, y), u);
}
__device__ void step(const Geom& g, const int x[4], int mu, int d, int y[4]) {
  for (int k = 0; k < 4; k++) y[k] = x[k];
  y[mu] = (x[mu] + d + g.L[mu]) % g.L[mu];
}
// c = a b, a^dag b, a b^dag
__device__ void mm(const cd a[9], const cd b[9], cd c[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cd s = mkc(0.0, 0.0);
      for (int k = 0; k < 3; k++) s = cfma(a[i * 3 + k], b[k * 3 + j], s);
      c[i * 3 + j] = s;
    }
}
__device__ void mdm(const cd a[9], const cd b[9], cd c[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cd s = mkc(0.0, 0.0);
      for (int k = 0; k < 3; k++) s = cfma_conj(a[k * 3 + i], b[k * 3 + j], s);
      c[i * 3 + j] = s;
    }
}
__device__ void mmd(const cd a[9], const cd b[9], cd c[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cd s = mkc(0.0, 0.0);
      for (int k = 0; k < 3; k++) s = cfma(a[i * 3 + k], conj(b[j * 3 + k]), s);
      c[i * 3 + j] = s;
    }
}

// Q_{mu nu}(x): sum of the four counter-clockwise plaquette leaves at x.
__device__ void clover_leaves(const Geom& g, const double* gauge, const int x[4], int mu, int nu, cd q[9]) {
  int y[4], z[4];
  cd a[9], b[9], t1[9], t2[9];
  for (int e = 0; e < 9; e++) q[e] = mkc(0.0, 0.0);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  link_at(g, gauge, x, mu, a);
  step(g, x, mu, +1, y); link_at(g, gauge, y, nu, b);
  mm(a, b, t1);
  step(g, x, nu, +1, y); link_at(g, gauge, y, mu, a);
  mmd(t1, a, t2);
  link_at(g, gauge, x, nu, a);
  mmd(t2, a, t1);
  for (int e = 0; e < 9; e++) q[e] = q[e] + t1[e];
  // leaf 2: U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  link_at(g, gauge, x, nu, a);
  step(g, x, nu, +1, y); step(g, y, mu, -1, z); link_at(g, gauge, z, mu, b);
  mmd(a, b, t1);
  step(g, x, mu, -1, y); link_at(g, gauge, y, nu, a);
  mmd(t1, a, t2);
  link_at(g, gauge, y, mu, a);
  mm(t2, a, t1);
  for (int e = 0; e < 9; e++) q[e] = q[e] + t1[e];
  // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  step(g, x, mu, -1, y); link_at(g, gauge, y, mu, a);
  step(g, y, nu, -1, z); link_at(g, gauge, z, nu, b);
  // t1 = a^dag b^dag = (b a)^dag
  mm(b, a, t2);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) t1[i * 3 + j] = conj(t2[j * 3 + i]);
  link_at(g, gauge, z, mu, a);
  mm(t1, a, t2);
  step(g, x, nu, -1, y); link_at(g, gauge, y, nu, a);
  mm(t2, a, t1);
  for (int e = 0; e < 9; e++) q[e] = q[e] + t1[e];
  // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
  step(g, x, nu, -1, y); link_at(g, gauge, y, nu, a);
  link_at(g, gauge, y, mu, b);
  mdm(a, b, t1);
  step(g, y, mu, +1, z); link_at(g, gauge, z, nu, a);
  mm(t1, a, t2);
  link_at(g, gauge, x, mu, a);
  mmd(t2, a, t1);
  for (int e = 0; e < 9; e++) q[e] = q[e] + t1[e];
}

// In-place inverse of a 6x6 complex matrix by Gauss-Jordan with partial
// pivoting; returns false if a pivot falls below 1e-12 of the largest entry.
__device__ bool invert6(cd m[36], cd inv[36]) {
  double amax = 0;
  for (int e = 0; e < 36; e++) amax = fmax(amax, fabs(m[e].re) + fabs(m[e].im));
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) inv[i * 6 + j] = mkc(i == j ? 1.0 : 0.0, 0.0);
  bool ok = amax > 0;
  for (int col = 0; col < 6; col++) {
    int piv = col;
    double best = -1;
    for (int r = col; r < 6; r++) {
      double v = m[r * 6 + col].re * m[r * 6 + col].re + m[r * 6 + col].im * m[r * 6 + col].im;
      if (v > best) { best = v; piv = r; }
    }
    if (!(sqrt(best) > 1e-12 * amax)) { ok = false; best = 1.0; }
    if (piv != col)
      for (int j = 0; j < 6; j++) {
        cd t = m[col * 6 + j]; m[col * 6 + j] = m[piv * 6 + j]; m[piv * 6 + j] = t;
        t = inv[col * 6 + j]; inv[col * 6 + j] = inv[piv * 6 + j]; inv[piv * 6 + j] = t;
      }
    cd p = m[col * 6 + col];
    double den = p.re * p.re + p.im * p.im;
    if (den == 0) den = 1;
    cd pinv = mkc(p.re / den, -p.im / den);
    for (int j = 0; j < 6; j++) {
      m[col * 6 + j] = pinv * m[col * 6 + j];
      inv[col * 6 + j] = pinv * inv[col * 6 + j];
    }
    for (int r = 0; r < 6; r++) {
      if (r == col) continue;
      cd f = m[r * 6 + col];
      for (int j = 0; j < 6; j++) {
        m[r * 6 + j] = m[r * 6 + j] - f * m[col * 6 + j];
        inv[r * 6 + j] = inv[r * 6 + j] - f * inv[col * 6 + j];
      }
    }
  }
  return ok;
}

__device__ void pack_herm(const cd m[36], double r[36]) {
  for (int i = 0; i < 6; i++) r[i] = m[i * 6 + i].re;
  for (int i = 1; i < 6; i++)
    for (int j = 0; j < i; j++) {
      const int k = i * (i - 1) / 2 + j;
      r[6 + 2 * k] = m[i * 6 + j].re;
      r[6 + 2 * k + 1] = m[i * 6 + j].im;
    }
}
}  // namespace

__global__ void k_build_clover(Geom g, const double* __restrict__ gauge, CloverCoef cf, double m0, double* A64,
                               double* Ainv64, float* A32, float* Ainv32, int* flags) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 2 * g.Vh) return;
  const int par = gid / g.Vh, i = gid % g.Vh;
  int x[4];
  cb_coords(g, i, par, x);
  // lower triangles (i >= j) of the two chiral blocks
  cd L[2][21];
  for (int b = 0; b < 2; b++)
    for (int e = 0; e < 21; e++) L[b][e] = mkc(0.0, 0.0);
  int plane = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++, plane++) {
      cd q[9], F[9];
      clover_leaves(g, gauge, x, mu, nu, q);
      for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) F[a * 3 + c] = 0.125 * (q[a * 3 + c] - conj(q[c * 3 + a]));
      cd tr = mkc((F[0].re + F[4].re + F[8].re) / 3.0, (F[0].im + F[4].im + F[8].im) / 3.0);
      F[0] = F[0] - tr; F[4] = F[4] - tr; F[8] = F[8] - tr;
      // sum over mu != nu of both orders gives 2x the mu < nu term:
      // A += (i c_{mu nu} / 2) sigma_{mu nu} (x) F_{mu nu}, c = csw_t for the planes
      // that contain t, csw_s for the spatial ones (one csw when isotropic)
      const cd pre = mkc(0.0, 0.5 * (nu == 3 ? cf.csw_t : cf.csw_s));
      for (int b = 0; b < 2; b++)
        for (int ii = 0; ii < 6; ii++)
          for (int jj = 0; jj <= ii; jj++) {
            const int si = ii / 3, ci = ii % 3, sj = jj / 3, cj = jj % 3;
            cd sg = mkc(c_sigma[plane][b][si][sj][0], c_sigma[plane][b][si][sj][1]);
            L[b][ii * (ii + 1) / 2 + jj] = L[b][ii * (ii + 1) / 2 + jj] + pre * (sg * F[ci * 3 + cj]);
          }
    }
  for (int b = 0; b < 2; b++) {
    cd M[36], Minv[36];
    for (int ii = 0; ii < 6; ii++)
      for (int jj = 0; jj <= ii; jj++) {
        cd v = L[b][ii * (ii + 1) / 2 + jj];
        if (ii == jj) v = mkc(v.re + (g.w[0] + g.w[1] + g.w[2] + g.w[3]) + m0, 0.0);   // 4 + m0 when isotropic
        M[ii * 6 + jj] = v;
        M[jj * 6 + ii] = conj(v);
      }
    double r[36];
    pack_herm(M, r);
    CloverIO<double>::store_block(A64 + (size_t)par * 72 * g.Vh, g.Vh, i, b, r);
    float rf[36];
    for (int e = 0; e < 36; e++) rf[e] = (float)r[e];
    CloverIO<float>::store_block(A32 + (size_t)par * 72 * g.Vh, g.Vh, i, b, rf);
    if (!invert6(M, Minv)) atomicExch(&flags[FLAG_SINGULAR], 1);
    // symmetrise: store the Hermitian part of the inverse
    for (int ii = 0; ii < 6; ii++)
      for (int jj = 0; jj <= ii; jj++) {
        cd a = Minv[ii * 6 + jj], c = conj(Minv[jj * 6 + ii]);
        Minv[ii * 6 + jj] = mkc(0.5 * (a.re + c.re), 0.5 * (a.im + c.im));
      }
    pack_herm(Minv, r);
    CloverIO<double>::store_block(Ainv64 + (size_t)par * 72 * g.Vh, g.Vh, i, b, r);
    for (int e = 0; e < 36; e++) rf[e] = (float)r[e];
    CloverIO<float>::store_block(Ainv32 + (size_t)par * 72 * g.Vh, g.Vh, i, b, rf);
  }
}

void build_clover(const Geom& g, const double* g64, CloverCoef cf, double m0, double* A64, double* Ainv64,
                  float* A32, float* Ainv32, int* flags, cudaStream_t s) {
  upload_sigma();
  const int n = 2 * g.Vh, bs = 64;
  k_build_clover<<<(n + bs - 1) / bs, bs, 0, s>>>(g, g64, cf, m0, A64, Ainv64, A32, Ainv32, flags);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- clover apply
template <typename T>
__global__ void k_clover_apply(Geom g, T* out, const T* __restrict__ in, const T* __restrict__ clov) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Vh) return;
  cx<T> x[12], y[12];
  SpinorIO<T>::load(in, g.Vh, i, x);
  clover_mul<T>(clov, g.Vh, i, x, y);
  SpinorIO<T>::store(out, g.Vh, i, y);
}

template <typename T>
void clover_apply(const Geom& g, T* out, const T* in, const T* clov, cudaStream_t s) {
  const int bs = 128;
  k_clover_apply<T><<<(g.Vh + bs - 1) / bs, bs, 0, s>>>(g, out, in, clov);
  MG_LAUNCH();
}
template void clover_apply<float>(const Geom&, float*, const float*, const float*, cudaStream_t);
template void clover_apply<double>(const Geom&, double*, const double*, const double*, cudaStream_t);

// --------------------------------------------------------------------------- dslash
// One output site: out = epilogue(-1/2 H in) (see Epilogue).
template <typename T, int EPI>
__device__ __forceinline__ void dslash_site(const Geom& g, int par, int i, T* out, const T* __restrict__ in,
                                            const T* __restrict__ gauge, const T* __restrict__ clov,
                                            const T* __restrict__ x, T a, int dirmask) {
  int c[4];
  cb_coords(g, i, par, c);
  cx<T> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = mkc<T>(0, 0);
  hop_sum<T>(g, in, gauge, par, i, c, dirmask, acc);
  const T half = (T)-0.5;
  cx<T> res[12];
  if (EPI == EPI_H) {
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = half * acc[k];
  } else if (EPI == EPI_CH) {
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = half * acc[k];
    clover_mul<T>(clov, g.Vh, i, acc, res);
  } else if (EPI == EPI_XPAY) {
    cx<T> xv[12];
    SpinorIO<T>::load(x, g.Vh, i, xv);
    const T f = half * a;
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = xv[k] + f * acc[k];
  } else if (EPI == EPI_CX_PAY) {
    cx<T> xv[12];
    SpinorIO<T>::load(x, g.Vh, i, xv);
    clover_mul<T>(clov, g.Vh, i, xv, res);
    const T f = half * a;
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = res[k] + f * acc[k];
  } else {  // EPI_C_XPAY
    cx<T> xv[12];
    SpinorIO<T>::load(x, g.Vh, i, xv);
    const T f = half * a;
#pragma unroll
    for (int k = 0; k < 12; k++) xv[k] = xv[k] + f * acc[k];
    clover_mul<T>(clov, g.Vh, i, xv, res);
  }
  SpinorIO<T>::store(out, g.Vh, i, res);
}

template <typename T, int EPI>
__global__ void __launch_bounds__(128) k_dslash(Geom g, int par, T* out, const T* __restrict__ in,
                                                 const T* __restrict__ gauge, const T* __restrict__ clov,
                                                 const T* __restrict__ x, T a, int dirmask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Vh) return;
  dslash_site<T, EPI>(g, par, i, out, in, gauge, clov, x, a, dirmask);
}

// The epilogues of the multi-RHS kernels for the nr <= NR right-hand sides
// r0 .. r0 + nr - 1 of site i (acc: the hop sums without the -1/2).
template <typename T, int EPI, int NR>
__device__ __forceinline__ void mrhs_epilogue(const Geom& g, int i, cx<T> (&acc)[NR][12], int nr, int r0,
                                              size_t stride, T* out, const T* __restrict__ clov,
                                              const T* __restrict__ x, T a) {
  const T half = (T)-0.5;
#pragma unroll
  for (int r = 0; r < NR; r++) {
    if (r >= nr) break;
    const size_t o = (size_t)(r0 + r) * stride;
    cx<T> res[12];
    if (EPI == EPI_H) {
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = half * acc[r][k];
    } else if (EPI == EPI_CH) {
#pragma unroll
      for (int k = 0; k < 12; k++) acc[r][k] = half * acc[r][k];
      clover_mul<T>(clov, g.Vh, i, acc[r], res);
    } else if (EPI == EPI_XPAY) {
      cx<T> xv[12];
      SpinorIO<T>::load(x + o, g.Vh, i, xv);
      const T f = half * a;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = xv[k] + f * acc[r][k];
    } else if (EPI == EPI_CX_PAY) {
      cx<T> xv[12];
      SpinorIO<T>::load(x + o, g.Vh, i, xv);
      clover_mul<T>(clov, g.Vh, i, xv, res);
      const T f = half * a;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = res[k] + f * acc[r][k];
    } else {  // EPI_C_XPAY
      cx<T> xv[12];
      SpinorIO<T>::load(x + o, g.Vh, i, xv);
      const T f = half * a;
#pragma unroll
      for (int k = 0; k < 12; k++) xv[k] = xv[k] + f * acc[r][k];
      clover_mul<T>(clov, g.Vh, i, xv, res);
    }
    SpinorIO<T>::store(out + o, g.Vh, i, res);
  }
}

// Multi-RHS form: nrhs vectors at a fixed stride (in elements of T).  A
// thread owns one site and NR right-hand sides (the block index selects the
// site block and the group of NR, group fastest): every link is loaded once
// into registers and applied to the NR
// neighbour spinors, so link bytes are paid once per site and NR rhs while
// the spinor loads stay coalesced over consecutive sites.
template <typename T, int EPI, int NR, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_dslash_mrhs(Geom g, int par, int nrhs, size_t stride, T* out,
                                                    const T* __restrict__ in, const T* __restrict__ gauge,
                                                    const T* __restrict__ clov, const T* __restrict__ x, T a,
                                                    int dirmask) {
  // 1-D grid, rhs group fastest: CTAs that run together share the sites
  // (and so the link and clover lines in L2) of consecutive rhs groups
  const int ngroups = (nrhs + NR - 1) / NR;
  const int i = (int)(blockIdx.x / ngroups) * BS + threadIdx.x;
  if (i >= g.Vh) return;
  const int r0 = (int)(blockIdx.x % ngroups) * NR;
  const int nr = nrhs - r0 < NR ? nrhs - r0 : NR;
  int c[4];
  cb_coords(g, i, par, c);
  cx<T> acc[NR][12];
#pragma unroll
  for (int r = 0; r < NR; r++)
#pragma unroll
    for (int k = 0; k < 12; k++) acc[r][k] = mkc<T>(0, 0);
  hop_sum_nr<T, NR>(g, in + (size_t)r0 * stride, stride, nr, gauge, par, i, c, dirmask, acc);
  mrhs_epilogue<T, EPI, NR>(g, i, acc, nr, r0, stride, out, clov, x, a);
}

template <typename T>
void dslash(const Geom& g, Epilogue epi, int parity, T* out, const T* in, const T* gauge, const T* clov, const T* x,
            double a, int dirmask, cudaStream_t s) {
  const int bs = 128;
  const int nb = (g.Vh + bs - 1) / bs;
  switch (epi) {
    case EPI_H: k_dslash<T, EPI_H><<<nb, bs, 0, s>>>(g, parity, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_CH: k_dslash<T, EPI_CH><<<nb, bs, 0, s>>>(g, parity, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_XPAY: k_dslash<T, EPI_XPAY><<<nb, bs, 0, s>>>(g, parity, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_CX_PAY: k_dslash<T, EPI_CX_PAY><<<nb, bs, 0, s>>>(g, parity, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_C_XPAY: k_dslash<T, EPI_C_XPAY><<<nb, bs, 0, s>>>(g, parity, out, in, gauge, clov, x, (T)a, dirmask); break;
  }
  MG_LAUNCH();
}
template void dslash<float>(const Geom&, Epilogue, int, float*, const float*, const float*, const float*,
                            const float*, double, int, cudaStream_t);
template void dslash<double>(const Geom&, Epilogue, int, double*, const double*, const double*, const double*,
                             const double*, double, int, cudaStream_t);

// Second mapping: one (site, rhs) per thread, the CTA is 32 consecutive sites
// (threadIdx.x) x NY right-hand sides (threadIdx.y).  Each warp reads 32
// consecutive sites of one rhs (coalesced spinors) with the register
// footprint of the single-RHS kernel; the NY warps of a CTA read the same
// link and clover lines, which the first one brings into L1.
template <typename T, int EPI, int NY>
__global__ void __launch_bounds__(32 * NY) k_dslash_mrhs_y(Geom g, int par, int nrhs, size_t stride, T* out,
                                                            const T* __restrict__ in, const T* __restrict__ gauge,
                                                            const T* __restrict__ clov, const T* __restrict__ x, T a,
                                                            int dirmask) {
  const int ngroups = (nrhs + NY - 1) / NY;   // rhs group fastest in the 1-D grid
  const int i = (int)(blockIdx.x / ngroups) * 32 + threadIdx.x;
  const int r = (int)(blockIdx.x % ngroups) * NY + threadIdx.y;
  if (i >= g.Vh || r >= nrhs) return;
  const size_t o = (size_t)r * stride;
  dslash_site<T, EPI>(g, par, i, out + o, in + o, gauge, clov, x ? x + o : nullptr, a, dirmask);
}

template <typename T, int NY>
void dslash_mrhs_y(const Geom& g, Epilogue epi, int parity, int nrhs, size_t stride, T* out, const T* in,
                   const T* gauge, const T* clov, const T* x, double a, int dirmask, cudaStream_t s) {
  const dim3 grid((unsigned)(((g.Vh + 31) / 32) * ((nrhs + NY - 1) / NY))), block(32, NY);
  switch (epi) {
    case EPI_H: k_dslash_mrhs_y<T, EPI_H, NY><<<grid, block, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_CH: k_dslash_mrhs_y<T, EPI_CH, NY><<<grid, block, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_XPAY: k_dslash_mrhs_y<T, EPI_XPAY, NY><<<grid, block, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_CX_PAY: k_dslash_mrhs_y<T, EPI_CX_PAY, NY><<<grid, block, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_C_XPAY: k_dslash_mrhs_y<T, EPI_C_XPAY, NY><<<grid, block, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
  }
  MG_LAUNCH();
}

// Third mapping (FP32): the CTA stages the links of its S consecutive output
// sites -- both hops of every dimension, 8 x 9 complex per site -- and, when
// the epilogue multiplies by a clover term, that term (18 float4 per site) in
// shared memory once, and then runs every right-hand side over them: thread
// (s, q) owns site s and the right-hand sides q, q + NQ, ...  Link and clover
// bytes leave L2 once per site for all nrhs (not once per rhs group), the
// neighbour spinors are read per rhs exactly as by the single-RHS kernel, and
// each thread keeps the single-RHS register footprint.
constexpr bool epi_has_clover(int epi) { return epi == EPI_CH || epi == EPI_CX_PAY || epi == EPI_C_XPAY; }

template <int S>
__device__ __forceinline__ void clover_mul_smem(const float4* sc, int s, const cx<float> x[12], cx<float> y[12]) {
#pragma unroll
  for (int b = 0; b < 2; b++) {
    float r[36];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const float4 v = sc[(9 * b + k) * S + s];
      r[4 * k] = v.x;
      r[4 * k + 1] = v.y;
      r[4 * k + 2] = v.z;
      r[4 * k + 3] = v.w;
    }
    herm6_apply<float>(r, x + 6 * b, y + 6 * b);
  }
}

// hop D (D = 2 mu + 1 for the backward hop) of one rhs with its link from shared memory
template <int D, int S>
__device__ __forceinline__ void smem_hop(const Geom& g, const float* __restrict__ in, const float2* sl, int s, int j,
                                         float sgw, cx<float> acc[12]) {
  cx<float> psi[12];
  SpinorIO<float>::load(in, g.Vh, j, psi);
  cx<float> u[9];
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const float2 v = sl[(D * 9 + e) * S + s];
    u[e] = mkc(v.x, v.y);
  }
  hop_apply<float, D / 2, (D & 1) == 0>(psi, u, sgw, acc);
}

template <int D>
__device__ __forceinline__ int dir_bit() { return (D & 1) ? 16 << (D / 2) : 1 << (D / 2); }

// Site block of the CTA launched as `b`.  Natural order (tt == 0): block b.
// Tiled order (tt > 0, which needs S to divide the xh Ly sites of a (z, t)
// plane -- nyb blocks per plane -- and tt to divide Lt): the lattice is cut
// into slabs of tt time slices, taken one after the other; inside a slab the
// blocks of a plane come first, then the next time slice, then the next z.
// A neighbour in t is then nyb launches away and one in z nyb * tt launches
// away, instead of a whole time slice (Vh / Lt sites) for t: with all
// right-hand sides of a site in flight at once, the spinors of a time slice
// no longer fit in L2 between their uses, those of a slab's window do.
__device__ __forceinline__ int mrhs_block(const Geom& g, int b, int nyb, int tt) {
  if (tt <= 0) return b;
  const int yb = b % nyb;
  int r = b / nyb;
  const int tin = r % tt;
  r /= tt;
  const int z = r % g.L[2];
  const int t = (r / g.L[2]) * tt + tin;
  return yb + nyb * (z + g.L[2] * t);
}

template <int EPI, int S, int NQ, int MINB>
__global__ void __launch_bounds__(S * NQ, MINB) k_dslash_mrhs_smem(Geom g, int par, int nrhs, size_t stride,
                                                                    float* out, const float* __restrict__ in,
                                                                    const float* __restrict__ gauge,
                                                                    const float* __restrict__ clov,
                                                                    const float* __restrict__ x, float a, int dirmask,
                                                                    int nyb, int tt) {
  extern __shared__ float4 dsm[];
  float2* sl = reinterpret_cast<float2*>(dsm);   // [8 hops][9][S]
  float4* sc = dsm + 36 * S;                      // [18][S], after the 72 S float2 of links
  __shared__ int snb[8][S];                       // neighbour index of every hop of the CTA's sites
  __shared__ float ssg[8][S];                     // boundary sign x hopping weight of every hop
  const int s = (int)threadIdx.x % S, q = (int)threadIdx.x / S;
  const int i = mrhs_block(g, (int)blockIdx.x, nyb, tt) * S + s;
  const bool valid = i < g.Vh;
  if (valid) {
    int c[4];
    cb_coords(g, i, par, c);
    int nb[8];
    float sg[8];
    int sgn;
#define MG_SMEM_NB(D, MU, FWD)                \
  nb[D] = neighbour<MU, FWD>(g, c, sgn);        \
  sg[D] = (float)sgn * (float)g.w[MU];
    MG_SMEM_NB(0, 0, true) MG_SMEM_NB(1, 0, false) MG_SMEM_NB(2, 1, true) MG_SMEM_NB(3, 1, false)
    MG_SMEM_NB(4, 2, true) MG_SMEM_NB(5, 2, false) MG_SMEM_NB(6, 3, true) MG_SMEM_NB(7, 3, false)
#undef MG_SMEM_NB
    if (q == 0) {
#pragma unroll
      for (int d = 0; d < 8; d++) {
        snb[d][s] = nb[d];
        ssg[d][s] = sg[d];
      }
    }
    // links: U_mu(x) of this parity for the forward hops, U_mu(x - mu) of the
    // other parity for the backward ones
    const float2* gl = reinterpret_cast<const float2*>(gauge);
#pragma unroll
    for (int d = 0; d < 8; d++) {
      const int bit = (d & 1) ? 16 << (d / 2) : 1 << (d / 2);
      if (d % NQ != q || !(dirmask & bit)) continue;
      const int site = (d & 1) ? nb[d] : i;
      const float2* p = gl + (size_t)((((d & 1) ? 1 - par : par) * 4) + d / 2) * 9 * g.Vh;
#pragma unroll
      for (int e = 0; e < 9; e++) sl[(d * 9 + e) * S + s] = p[(size_t)e * g.Vh + site];
    }
    if (epi_has_clover(EPI)) {
      const float4* cp = reinterpret_cast<const float4*>(clov);
      for (int k = q; k < 18; k += NQ) sc[k * S + s] = cp[(size_t)k * g.Vh + i];
    }
  }
  __syncthreads();
  if (!valid) return;
  const float half = -0.5f;
  for (int r = q; r < nrhs; r += NQ) {
    const size_t o = (size_t)r * stride;
    const float* inr = in + o;
    cx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = mkc<float>(0, 0);
    if (dirmask & dir_bit<0>()) smem_hop<0, S>(g, inr, sl, s, snb[0][s], ssg[0][s], acc);
    if (dirmask & dir_bit<1>()) smem_hop<1, S>(g, inr, sl, s, snb[1][s], ssg[1][s], acc);
    if (dirmask & dir_bit<2>()) smem_hop<2, S>(g, inr, sl, s, snb[2][s], ssg[2][s], acc);
    if (dirmask & dir_bit<3>()) smem_hop<3, S>(g, inr, sl, s, snb[3][s], ssg[3][s], acc);
    if (dirmask & dir_bit<4>()) smem_hop<4, S>(g, inr, sl, s, snb[4][s], ssg[4][s], acc);
    if (dirmask & dir_bit<5>()) smem_hop<5, S>(g, inr, sl, s, snb[5][s], ssg[5][s], acc);
    if (dirmask & dir_bit<6>()) smem_hop<6, S>(g, inr, sl, s, snb[6][s], ssg[6][s], acc);
    if (dirmask & dir_bit<7>()) smem_hop<7, S>(g, inr, sl, s, snb[7][s], ssg[7][s], acc);
    cx<float> res[12];
    if (EPI == EPI_H) {
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = half * acc[k];
    } else if (EPI == EPI_CH) {
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = half * acc[k];
      clover_mul_smem<S>(sc, s, acc, res);
    } else if (EPI == EPI_XPAY) {
      cx<float> xv[12];
      SpinorIO<float>::load(x + o, g.Vh, i, xv);
      const float f = half * a;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = xv[k] + f * acc[k];
    } else if (EPI == EPI_CX_PAY) {
      cx<float> xv[12];
      SpinorIO<float>::load(x + o, g.Vh, i, xv);
      clover_mul_smem<S>(sc, s, xv, res);
      const float f = half * a;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = res[k] + f * acc[k];
    } else {  // EPI_C_XPAY
      cx<float> xv[12];
      SpinorIO<float>::load(x + o, g.Vh, i, xv);
      const float f = half * a;
#pragma unroll
      for (int k = 0; k < 12; k++) xv[k] = xv[k] + f * acc[k];
      clover_mul_smem<S>(sc, s, xv, res);
    }
    SpinorIO<float>::store(out + o, g.Vh, i, res);
  }
}

template <int EPI, int S, int NQ, int MINB>
void launch_mrhs_smem(const Geom& g, int parity, int nrhs, size_t stride, float* out, const float* in,
                      const float* gauge, const float* clov, const float* x, double a, int dirmask, int tt,
                      cudaStream_t s) {
  const int plane = g.xh * g.L[1];   // sites of one (z, t) plane of a parity
  if (plane % S != 0 || tt <= 0 || g.L[3] % tt != 0) tt = 0;   // tiled order needs whole blocks and slabs
  const int nyb = plane / S;
  const size_t smem = sizeof(float2) * 72 * S + (epi_has_clover(EPI) ? sizeof(float4) * 18 * S : 0);
  auto kern = k_dslash_mrhs_smem<EPI, S, NQ, MINB>;
  static std::atomic<unsigned> attr_set{0u};   // devices on which this instantiation may take `smem` bytes
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev >= 32 || !(attr_set.load() & (1u << dev))) {
    MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (dev < 32) attr_set.fetch_or(1u << dev);
  }
  kern<<<(unsigned)((g.Vh + S - 1) / S), S * NQ, smem, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (float)a,
                                                           dirmask, nyb, tt);
  MG_LAUNCH();
}

template <int S, int NQ, int MINB>
void dslash_mrhs_smem(const Geom& g, Epilogue epi, int parity, int nrhs, size_t stride, float* out, const float* in,
                      const float* gauge, const float* clov, const float* x, double a, int dirmask, int tt,
                      cudaStream_t s) {
  switch (epi) {
    case EPI_H: launch_mrhs_smem<EPI_H, S, NQ, MINB>(g, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s); break;
    case EPI_CH: launch_mrhs_smem<EPI_CH, S, NQ, MINB>(g, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s); break;
    case EPI_XPAY: launch_mrhs_smem<EPI_XPAY, S, NQ, MINB>(g, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s); break;
    case EPI_CX_PAY: launch_mrhs_smem<EPI_CX_PAY, S, NQ, MINB>(g, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s); break;
    case EPI_C_XPAY: launch_mrhs_smem<EPI_C_XPAY, S, NQ, MINB>(g, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s); break;
  }
}

template <typename T, int NR, int BS, int MINB = 1>
void dslash_mrhs_cfg(const Geom& g, Epilogue epi, int parity, int nrhs, size_t stride, T* out, const T* in,
                     const T* gauge, const T* clov, const T* x, double a, int dirmask, cudaStream_t s) {
  const dim3 grid((unsigned)(((g.Vh + BS - 1) / BS) * ((nrhs + NR - 1) / NR)));
  switch (epi) {
    case EPI_H: k_dslash_mrhs<T, EPI_H, NR, BS, MINB><<<grid, BS, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_CH: k_dslash_mrhs<T, EPI_CH, NR, BS, MINB><<<grid, BS, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_XPAY: k_dslash_mrhs<T, EPI_XPAY, NR, BS, MINB><<<grid, BS, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_CX_PAY: k_dslash_mrhs<T, EPI_CX_PAY, NR, BS, MINB><<<grid, BS, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
    case EPI_C_XPAY: k_dslash_mrhs<T, EPI_C_XPAY, NR, BS, MINB><<<grid, BS, 0, s>>>(g, parity, nrhs, stride, out, in, gauge, clov, x, (T)a, dirmask); break;
  }
  MG_LAUNCH();
}

// config = NR * 1000 + CTA size (NR right-hand sides per thread; FP32: NR in
// {2, 4}, FP64: NR in {1, 2}) [+ 10000, FP32 only: register cap for more
// resident CTAs, __launch_bounds__ minimum of 4 (NR = 2) or 3 (NR = 4) CTAs of 128], or
// 100000 + NY (rhs in threadIdx.y, NY in {4, 8}), or (FP32 only) 200000 +
// 100 S + NQ [+ 10: tiled CTA order] (links staged in shared memory: S sites
// x NQ rhs lanes per CTA; 203204, 203208, 206404, and 203214, 206414 tiled)
template <typename T>
void dslash_mrhs(const Geom& g, Epilogue epi, int parity, int nrhs, size_t stride, T* out, const T* in,
                 const T* gauge, const T* clov, const T* x, double a, int dirmask, int config, cudaStream_t s) {
  if (nrhs < 1) raise(MG_ERR_ARG, "nrhs must be positive");
  if (config >= 100000 && config < 200000) {
    if (config % 100 == 8)
      dslash_mrhs_y<T, 8>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
    else
      dslash_mrhs_y<T, 4>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
    return;
  }
  constexpr bool f32 = std::is_same<T, float>::value;
  constexpr int NA = f32 ? 2 : 1, NB = f32 ? 4 : 2;
  if (!f32 && config >= 200000) raise(MG_ERR_ARG, "the shared-memory multi-RHS dslash is FP32 only");
  if constexpr (f32) {
    if (config >= 200000) {   // links (and clover) staged in shared memory once for all rhs
      const int tt = (config / 10) % 10 == 1 ? 8 : 0;   // tiled CTA order, slabs of 8 time slices
      const int base = config - 10 * ((config / 10) % 10);
      if (base == 203208)
        dslash_mrhs_smem<32, 8, 3>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s);
      else if (base == 206404)
        dslash_mrhs_smem<64, 4, 3>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s);
      else
        dslash_mrhs_smem<32, 4, 5>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, tt, s);
      return;
    }
    if (config >= 10000) {   // register-capped variants (FP32 only: FP64 would spill), CTA of 128
      if ((config - 10000) / 1000 == 4)
        dslash_mrhs_cfg<T, 4, 128, 3>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
      else
        dslash_mrhs_cfg<T, 2, 128, 4>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
      return;
    }
  }
  const int nr = config / 1000, bs = config % 1000;
  if (nr == NB) {
    if (bs == 64)
      dslash_mrhs_cfg<T, NB, 64>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
    else
      dslash_mrhs_cfg<T, NB, 128>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
  } else {
    if (bs == 64)
      dslash_mrhs_cfg<T, NA, 64>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
    else
      dslash_mrhs_cfg<T, NA, 128>(g, epi, parity, nrhs, stride, out, in, gauge, clov, x, a, dirmask, s);
  }
}
template void dslash_mrhs<float>(const Geom&, Epilogue, int, int, size_t, float*, const float*, const float*,
                                 const float*, const float*, double, int, int, cudaStream_t);
template void dslash_mrhs<double>(const Geom&, Epilogue, int, int, size_t, double*, const double*, const double*,
                                  const double*, const double*, double, int, int, cudaStream_t);

std::vector<int> dslash_mrhs_configs(bool fp32) {
  return fp32 ? std::vector<int>{2064, 2128, 4064, 4128, 12128, 14128, 100004, 100008, 203204, 203208, 206404, 203214, 206414}
              : std::vector<int>{1064, 1128, 2064, 2128, 100004, 100008};
}
int dslash_mrhs_default(bool fp32) { (void)fp32; return 100004; }

// clover multiply of nrhs vectors (one thread per (site, rhs); the rhs is the
// fastest block index, so the clover lines of a site block are shared in L2)
template <typename T>
__global__ void k_clover_apply_mrhs(Geom g, int nrhs, size_t stride, T* out, const T* __restrict__ in,
                                    const T* __restrict__ clov) {
  const int i = (int)(blockIdx.x / nrhs) * blockDim.x + threadIdx.x, r = (int)(blockIdx.x % nrhs);
  if (i >= g.Vh) return;
  cx<T> x[12], y[12];
  SpinorIO<T>::load(in + (size_t)r * stride, g.Vh, i, x);
  clover_mul<T>(clov, g.Vh, i, x, y);
  SpinorIO<T>::store(out + (size_t)r * stride, g.Vh, i, y);
}

template <typename T>
void clover_apply_mrhs(const Geom& g, int nrhs, size_t stride, T* out, const T* in, const T* clov, cudaStream_t s) {
  const int bs = 128;
  k_clover_apply_mrhs<T><<<(unsigned)(((g.Vh + bs - 1) / bs) * nrhs), bs, 0, s>>>(g, nrhs, stride, out, in, clov);
  MG_LAUNCH();
}
template void clover_apply_mrhs<float>(const Geom&, int, size_t, float*, const float*, const float*, cudaStream_t);
template void clover_apply_mrhs<double>(const Geom&, int, size_t, double*, const double*, const double*, cudaStream_t);

// --------------------------------------------------------------------------- directional terms
struct DirOut {
  float* p[8];
};

template <int MU, bool FWD>
__device__ __forceinline__ void one_dir(const Geom& g, const float* in, const float* gauge, int par, int i,
                                        const int c[4], float* out_full) {
  cx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = mkc(0.f, 0.f);
  hop_term<float, MU, FWD>(g, in, gauge, par, i, c, acc);
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = -0.5f * acc[k];
  SpinorIO<float>::store(out_full + (size_t)par * 24 * g.Vh, g.Vh, i, acc);
}

__global__ void k_hop_directions(Geom g, DirOut o, const float* __restrict__ in_even, const float* __restrict__ in_odd,
                                 const float* __restrict__ gauge) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 2 * g.Vh) return;
  const int par = gid / g.Vh, i = gid % g.Vh;
  int c[4];
  cb_coords(g, i, par, c);
  const float* in = par ? in_even : in_odd;  // neighbours have the other parity
  one_dir<0, true>(g, in, gauge, par, i, c, o.p[0]);
  one_dir<1, true>(g, in, gauge, par, i, c, o.p[1]);
  one_dir<2, true>(g, in, gauge, par, i, c, o.p[2]);
  one_dir<3, true>(g, in, gauge, par, i, c, o.p[3]);
  one_dir<0, false>(g, in, gauge, par, i, c, o.p[4]);
  one_dir<1, false>(g, in, gauge, par, i, c, o.p[5]);
  one_dir<2, false>(g, in, gauge, par, i, c, o.p[6]);
  one_dir<3, false>(g, in, gauge, par, i, c, o.p[7]);
}

void hop_directions(const Geom& g, float* const out[8], const float* in_even, const float* in_odd, const float* gauge,
                    cudaStream_t s) {
  DirOut o;
  for (int d = 0; d < 8; d++) o.p[d] = out[d];
  const int n = 2 * g.Vh, bs = 128;
  k_hop_directions<<<(n + bs - 1) / bs, bs, 0, s>>>(g, o, in_even, in_odd, gauge);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- Philox start vectors
__global__ void k_philox_fine(Geom g, uint64_t seed, int level, int k, float* even, float* odd) {
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= 2 * g.Vh) return;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  cx<float> s[12];
  for (int d = 0; d < 12; d++) {
    cx<double> z = philox_gauss(seed, level, k, lex, d);
    s[d] = mkc((float)z.re, (float)z.im);
  }
  SpinorIO<float>::store(par ? odd : even, g.Vh, lex >> 1, s);
}

void philox_fine_vector(const Geom& g, uint64_t seed, int level, int k, float* even, float* odd, cudaStream_t s) {
  const int n = 2 * g.Vh, bs = 128;
  k_philox_fine<<<(n + bs - 1) / bs, bs, 0, s>>>(g, seed, level, k, even, odd);
  MG_LAUNCH();
}

}  // namespace mg
