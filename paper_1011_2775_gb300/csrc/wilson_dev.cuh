// Directional terms of the Wilson hopping operator (device functions).
//
//   H psi(x) = -1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                          + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
//
// (Wilson r = 1; the paper's operator D(U) of Eq. 1 with the clover term
// kept site-local.)  In the DeGrand-Rossi chiral basis every gamma_mu has the
// off-diagonal block form [[0, a_mu], [b_mu, 0]] with b_mu a_mu = 1:
//   a_x = i sigma_1, a_y = -i sigma_2, a_z = i sigma_3, a_t = 1,
//   b_x = -i sigma_1, b_y = i sigma_2, b_z = -i sigma_3, b_t = 1.
// Hence (1 -/+ gamma_mu) psi = [h ; -/+ b_mu h] with h = psi_up -/+ a_mu psi_dn,
// so each term needs one 2-spin half spinor, two SU(3) mat-vecs and a
// reconstruction with permutations and factors of +-1, +-i only.
// The -1/2 is applied by the caller.  Fermions are antiperiodic in t.
#pragma once
#include "common.cuh"

namespace mg {

// (a_mu d)[0], (a_mu d)[1] for a lower-spin pair d0 = psi_2, d1 = psi_3
template <int MU, typename T>
__device__ __forceinline__ void mul_a(cx<T> d0, cx<T> d1, cx<T>& o0, cx<T>& o1) {
  if (MU == 0) { o0 = times_i(d1); o1 = times_i(d0); }
  if (MU == 1) { o0 = -d1; o1 = d0; }
  if (MU == 2) { o0 = times_i(d0); o1 = -times_i(d1); }
  if (MU == 3) { o0 = d0; o1 = d1; }
}

// (b_mu g)[0], (b_mu g)[1]
template <int MU, typename T>
__device__ __forceinline__ void mul_b(cx<T> g0, cx<T> g1, cx<T>& o0, cx<T>& o1) {
  if (MU == 0) { o0 = -times_i(g1); o1 = -times_i(g0); }
  if (MU == 1) { o0 = g1; o1 = -g0; }
  if (MU == 2) { o0 = -times_i(g0); o1 = times_i(g1); }
  if (MU == 3) { o0 = g0; o1 = g1; }
}

// Neighbour of site c in direction MU (FWD: +mu, else -mu): its checkerboard
// index and the boundary sign (-1 when the hop crosses the t boundary with
// antiperiodic fermions).
template <int MU, bool FWD>
__device__ __forceinline__ int neighbour(const Geom& g, const int c[4], int& sgn) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  sgn = 1;
  if (FWD) {
    n[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    if (MU == 3 && g.apbc && c[3] == g.L[3] - 1) sgn = -1;
  } else {
    n[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    if (MU == 3 && g.apbc && c[3] == 0) sgn = -1;
  }
  return cb_index(g, n);
}

// The arithmetic of one hop term: acc += (1 -/+ gamma_mu) U psi for the
// neighbour spinor psi and the link u (U_mu(x) for FWD, U_mu(x - mu) to be
// used daggered otherwise), s = boundary sign x hopping weight.
template <typename T, int MU, bool FWD>
__device__ __forceinline__ void hop_apply(const cx<T> psi[12], const cx<T> u[9], T s, cx<T> acc[12]) {
  cx<T> h0[3], h1[3];
#pragma unroll
  for (int col = 0; col < 3; col++) {
    cx<T> a0, a1;
    mul_a<MU, T>(psi[6 + col], psi[9 + col], a0, a1);
    if (FWD) {
      h0[col] = s * (psi[col] - a0);
      h1[col] = s * (psi[3 + col] - a1);
    } else {
      h0[col] = s * (psi[col] + a0);
      h1[col] = s * (psi[3 + col] + a1);
    }
  }
  cx<T> g0[3], g1[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    g0[a] = mkc<T>(0, 0);
    g1[a] = mkc<T>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
      if (FWD) {
        g0[a] = cfma(u[a * 3 + b], h0[b], g0[a]);
        g1[a] = cfma(u[a * 3 + b], h1[b], g1[a]);
      } else {
        g0[a] = cfma_conj(u[b * 3 + a], h0[b], g0[a]);
        g1[a] = cfma_conj(u[b * 3 + a], h1[b], g1[a]);
      }
    }
  }
#pragma unroll
  for (int col = 0; col < 3; col++) {
    acc[col] = acc[col] + g0[col];
    acc[3 + col] = acc[3 + col] + g1[col];
    cx<T> b0, b1;
    mul_b<MU, T>(g0[col], g1[col], b0, b1);
    if (FWD) {
      acc[6 + col] = acc[6 + col] - b0;
      acc[9 + col] = acc[9 + col] - b1;
    } else {
      acc[6 + col] = acc[6 + col] + b0;
      acc[9 + col] = acc[9 + col] + b1;
    }
  }
}

// acc += (1 -/+ gamma_mu) U psi(neighbour), without the -1/2.
//  in:    spinor half of parity 1-par (the neighbours' parity)
//  gauge: full internal gauge field
//  par,i,c: parity, checkerboard index and coordinates of the output site
template <typename T, int MU, bool FWD>
__device__ __forceinline__ void hop_term(const Geom& g, const T* __restrict__ in, const T* __restrict__ gauge,
                                         int par, int i, const int c[4], cx<T> acc[12]) {
  int sgn;
  const int j = neighbour<MU, FWD>(g, c, sgn);
  cx<T> psi[12];
  SpinorIO<T>::load(in, g.Vh, j, psi);
  cx<T> u[9];
  if (FWD)
    load_link<T>(gauge, g.Vh, par, MU, i, u);      // U_mu(x)
  else
    load_link<T>(gauge, g.Vh, 1 - par, MU, j, u);  // U_mu(x - mu)
  hop_apply<T, MU, FWD>(psi, u, (T)sgn * (T)g.w[MU], acc);   // boundary sign and the direction's hopping weight
}

// Sum of the hop terms selected by `dirmask` (bit d: d < 4 forward mu = d,
// d >= 4 backward mu = d - 4), without the -1/2.
template <typename T>
__device__ __forceinline__ void hop_sum(const Geom& g, const T* __restrict__ in, const T* __restrict__ gauge,
                                        int par, int i, const int c[4], int dirmask, cx<T> acc[12]) {
  if (dirmask & 0x01) hop_term<T, 0, true>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x10) hop_term<T, 0, false>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x02) hop_term<T, 1, true>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x20) hop_term<T, 1, false>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x04) hop_term<T, 2, true>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x40) hop_term<T, 2, false>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x08) hop_term<T, 3, true>(g, in, gauge, par, i, c, acc);
  if (dirmask & 0x80) hop_term<T, 3, false>(g, in, gauge, par, i, c, acc);
}

// Multi-RHS form of hop_term: the link is loaded once and applied to the
// neighbour spinors of nr <= NR right-hand sides (in + r * stride).
template <typename T, int MU, bool FWD, int NR>
__device__ __forceinline__ void hop_term_nr(const Geom& g, const T* __restrict__ in, size_t stride, int nr,
                                            const T* __restrict__ gauge, int par, int i, const int c[4],
                                            cx<T> acc[NR][12]) {
  int sgn;
  const int j = neighbour<MU, FWD>(g, c, sgn);
  cx<T> u[9];
  if (FWD)
    load_link<T>(gauge, g.Vh, par, MU, i, u);
  else
    load_link<T>(gauge, g.Vh, 1 - par, MU, j, u);
  const T s = (T)sgn * (T)g.w[MU];   // boundary sign and the direction's hopping weight
#pragma unroll
  for (int r = 0; r < NR; r++) {
    if (r >= nr) break;
    cx<T> psi[12];
    SpinorIO<T>::load(in + r * stride, g.Vh, j, psi);
    cx<T> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; col++) {
      cx<T> a0, a1;
      mul_a<MU, T>(psi[6 + col], psi[9 + col], a0, a1);
      if (FWD) {
        h0[col] = s * (psi[col] - a0);
        h1[col] = s * (psi[3 + col] - a1);
      } else {
        h0[col] = s * (psi[col] + a0);
        h1[col] = s * (psi[3 + col] + a1);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<T> g0 = mkc<T>(0, 0), g1 = mkc<T>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; b++) {
        if (FWD) {
          g0 = cfma(u[a * 3 + b], h0[b], g0);
          g1 = cfma(u[a * 3 + b], h1[b], g1);
        } else {
          g0 = cfma_conj(u[b * 3 + a], h0[b], g0);
          g1 = cfma_conj(u[b * 3 + a], h1[b], g1);
        }
      }
      acc[r][a] = acc[r][a] + g0;
      acc[r][3 + a] = acc[r][3 + a] + g1;
      cx<T> b0, b1;
      mul_b<MU, T>(g0, g1, b0, b1);
      if (FWD) {
        acc[r][6 + a] = acc[r][6 + a] - b0;
        acc[r][9 + a] = acc[r][9 + a] - b1;
      } else {
        acc[r][6 + a] = acc[r][6 + a] + b0;
        acc[r][9 + a] = acc[r][9 + a] + b1;
      }
    }
  }
}

template <typename T, int NR>
__device__ __forceinline__ void hop_sum_nr(const Geom& g, const T* __restrict__ in, size_t stride, int nr,
                                           const T* __restrict__ gauge, int par, int i, const int c[4], int dirmask,
                                           cx<T> acc[NR][12]) {
  if (dirmask & 0x01) hop_term_nr<T, 0, true, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x10) hop_term_nr<T, 0, false, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x02) hop_term_nr<T, 1, true, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x20) hop_term_nr<T, 1, false, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x04) hop_term_nr<T, 2, true, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x40) hop_term_nr<T, 2, false, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x08) hop_term_nr<T, 3, true, NR>(g, in, stride, nr, gauge, par, i, c, acc);
  if (dirmask & 0x80) hop_term_nr<T, 3, false, NR>(g, in, stride, nr, gauge, par, i, c, acc);
}

// out = C x for a packed two-block clover (A or A^{-1}) at site i.
template <typename T>
__device__ __forceinline__ void clover_mul(const T* __restrict__ clov, int Vh, int i, const cx<T> x[12], cx<T> y[12]) {
#pragma unroll
  for (int b = 0; b < 2; b++) {
    T r[36];
    CloverIO<T>::load_block(clov, Vh, i, b, r);
    herm6_apply<T>(r, x + 6 * b, y + 6 * b);
  }
}

}  // namespace mg
