// Gauge-link derivative of the Wilson-clover operator, for the gradient of a
// solve (the paper has no gradient; this is the adjoint-method extension).
//
// For fixed fine vectors lam and psi, f(U) = -Re <lam, D(U) psi> changes under
// a complex variation dU of the links by  df = Re sum_{x,mu} tr(dU_mu(x) K_mu(x)).
// With psi = D^{-1} eta and lam = D^{-dag} chi this is the derivative of
// L = Re <chi, D^{-1} eta>.  The kernels return K^dag (the unconstrained
// gradient in the convention dL/dRe U + i dL/dIm U) or the su(3) force
// sum_a F^a T_a, F^a = df/d omega^a for U -> exp(i omega^a T_a) U, which is
// (H - tr(H)/3)/2 with G = i U K and H = (G + G^dag)/2.
//
// K has a hopping part (one outer product per end of the link) and a clover
// part.  The clover part: lam^dag (sigma_{mu nu} x dF_{mu nu}) psi = tr(dF S),
// S = sum_s (sigma psi)_s lam_s^dag; with C = -(i csw/4) S, C0 = C - tr(C)/3
// and F = (Q - Q^dag)/8 - trace, the clover variation is
// Re sum_{mu<nu} tr(dQ_{mu nu} W_{mu nu}) with W = (C0 - C0^dag)/4 (both
// orders mu,nu and nu,mu give the same term).  Every plaquette of a plane is
// a leaf of Q at each of its four corners, so the link's own position in the
// plaquette collects the cyclic product of the other three links with W of
// every corner inserted where that corner's leaf begins.
//
// Two kernels: k_force_insertion writes W_{mu nu}(x) for the six planes of
// every site ([parity][plane][9][Vh]); k_force_links computes K (or the
// force) of every link and writes it in the ABI gauge layout (complex128).
// Both run in FP64 or, on request, in FP32 (FP32 gauge copy, vectors and W,
// FP32 arithmetic; the result is widened to complex128 on output).  With the
// anisotropic reading every hop carries its direction's weight w_mu and the
// planes containing t their own clover coefficient csw_t.
#include <cstring>

#include "internal.h"
#include "wilson_dev.cuh"

namespace mg {
void set_last_error(const std::string& what);

namespace {
template <typename T>
struct V2of;
template <>
struct V2of<double> {
  typedef double2 type;
};
template <>
struct V2of<float> {
  typedef float2 type;
};

template <typename T>
__device__ __forceinline__ typename V2of<T>::type mk2(T x, T y);
template <>
__device__ __forceinline__ double2 mk2<double>(double x, double y) {
  return make_double2(x, y);
}
template <>
__device__ __forceinline__ float2 mk2<float>(float x, float y) {
  return make_float2(x, y);
}

template <typename T>
__device__ __forceinline__ void m_mul(const cx<T> a[9], const cx<T> b[9], cx<T> c[9]) {
  typedef cx<T> cd;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cd s = a[i * 3] * b[j];
      s = cfma(a[i * 3 + 1], b[3 + j], s);
      s = cfma(a[i * 3 + 2], b[6 + j], s);
      c[i * 3 + j] = s;
    }
}
template <typename T>
__device__ __forceinline__ void m_mul_acc(const cx<T> a[9], const cx<T> b[9], cx<T> c[9]) {
  typedef cx<T> cd;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cd s = c[i * 3 + j];
      s = cfma(a[i * 3], b[j], s);
      s = cfma(a[i * 3 + 1], b[3 + j], s);
      s = cfma(a[i * 3 + 2], b[6 + j], s);
      c[i * 3 + j] = s;
    }
}
template <typename T>
__device__ __forceinline__ void m_dag_inplace(cx<T> a[9]) {
  typedef cx<T> cd;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    a[i * 3 + i] = conj(a[i * 3 + i]);
#pragma unroll
    for (int j = i + 1; j < 3; j++) {
      const cd t = a[i * 3 + j];
      a[i * 3 + j] = conj(a[j * 3 + i]);
      a[j * 3 + i] = conj(t);
    }
  }
}

// gamma_mu psi in the block form [[0, a_mu], [b_mu, 0]] (see wilson_dev.cuh)
template <int MU, typename T>
__device__ __forceinline__ void gamma_mul(const cx<T> in[12], cx<T> out[12]) {
#pragma unroll
  for (int col = 0; col < 3; col++) {
    mul_a<MU, T>(in[6 + col], in[9 + col], out[col], out[3 + col]);
    mul_b<MU, T>(in[col], in[3 + col], out[6 + col], out[9 + col]);
  }
}
template <typename T>
__device__ __forceinline__ void gamma_dyn(int mu, const cx<T> in[12], cx<T> out[12]) {
  switch (mu) {
    case 0: gamma_mul<0, T>(in, out); break;
    case 1: gamma_mul<1, T>(in, out); break;
    case 2: gamma_mul<2, T>(in, out); break;
    default: gamma_mul<3, T>(in, out); break;
  }
}

__device__ __forceinline__ int plane_of(int a, int b) { return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5); }

__device__ __forceinline__ void step(const Geom& g, int c[4], int mu, int d) {
  c[mu] += d;
  if (c[mu] < 0) c[mu] += g.L[mu];
  if (c[mu] >= g.L[mu]) c[mu] -= g.L[mu];
}

template <typename T>
__device__ __forceinline__ void link_at(const Geom& g, const T* gauge, const int c[4], int mu, cx<T> u[9]) {
  load_link<T>(gauge, g.Vh, (c[0] + c[1] + c[2] + c[3]) & 1, mu, cb_index(g, c), u);
}

template <typename T>
__device__ __forceinline__ void w_at(const Geom& g, const typename V2of<T>::type* W, const int c[4], int p,
                                     cx<T> w[9]) {
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const typename V2of<T>::type* q = W + (size_t)(par * 6 + p) * 9 * g.Vh + cb_index(g, c);
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const typename V2of<T>::type v = q[(size_t)e * g.Vh];
    w[e] = mkc(v.x, v.y);
  }
}

// W_{mu nu}(x) for the six planes mu < nu of every site.
template <typename T>
__global__ void __launch_bounds__(128) k_force_insertion(Geom g, const T* lam_e, const T* lam_o, const T* psi_e,
                                                         const T* psi_o, T csw, T csw_t, typename V2of<T>::type* W) {
  typedef cx<T> cd;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.Vh) return;
  const int par = t >= g.Vh;
  const int i = t - par * g.Vh;
  cd lam[12], psi[12];
  SpinorIO<T>::load(par ? lam_o : lam_e, g.Vh, i, lam);
  SpinorIO<T>::load(par ? psi_o : psi_e, g.Vh, i, psi);
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      const T q = (T)-0.25 * (nu == 3 ? csw_t : csw);   // C = -(i c_{mu nu}/4) S = q * (i S)
      cd gn[12], gmn[12];
      gamma_dyn(nu, psi, gn);
      gamma_dyn(mu, gn, gmn);            // sigma_{mu nu} psi = i gamma_mu gamma_nu psi
      cd C[9];
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
          cd s = mkc((T)0, (T)0);
#pragma unroll
          for (int sp = 0; sp < 4; sp++) s = cfma_conj(lam[3 * sp + b], gmn[3 * sp + a], s);
          // S_ab = sum_s (sigma psi)_{s a} conj(lam_{s b}) = i * s;  C = q * i * S = -q * s
          C[a * 3 + b] = mkc(-q * s.re, -q * s.im);
        }
      const cd tr3 = mkc((C[0].re + C[4].re + C[8].re) / (T)3, (C[0].im + C[4].im + C[8].im) / (T)3);
      C[0] = C[0] - tr3;
      C[4] = C[4] - tr3;
      C[8] = C[8] - tr3;
      const int p = plane_of(mu, nu);
      typename V2of<T>::type* out = W + (size_t)(par * 6 + p) * 9 * g.Vh + i;
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
          const cd w = C[a * 3 + b] - conj(C[b * 3 + a]);
          out[(size_t)(a * 3 + b) * g.Vh] = mk2<T>((T)0.25 * w.re, (T)0.25 * w.im);
        }
    }
}

// K_mu(x) (or the force) of every link; thread = (site, mu = blockIdx.y).
template <typename T>
__global__ void __launch_bounds__(128) k_force_links(Geom g, const T* lam_e, const T* lam_o, const T* psi_e,
                                                     const T* psi_o, const T* gauge,
                                                     const typename V2of<T>::type* W, int kind, double2* out) {
  typedef cx<T> cd;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.Vh) return;
  const int mu = blockIdx.y;
  const int par = t >= g.Vh;
  const int i = t - par * g.Vh;
  int x[4];
  cb_coords(g, i, par, x);
  cd K[9];

  // ---- hopping part: (s/2) [ sum_t psi(x+mu)_t ((1-g)lam(x))_t^dag + sum_s lam(x+mu)_s ((1+g)psi(x))_s^dag ]
  {
    int y[4] = {x[0], x[1], x[2], x[3]};
    step(g, y, mu, +1);
    const int j = cb_index(g, y);
    // boundary sign times the direction's hopping weight
    const T sgn = ((mu == 3 && g.apbc && x[3] == g.L[3] - 1) ? (T)-1 : (T)1) * (T)g.w[mu];
    cd a[12], b[12], ga[12];
    // first outer product: psi(x+mu) against (1 - gamma) lam(x)
    SpinorIO<T>::load(par ? lam_o : lam_e, g.Vh, i, a);
    gamma_dyn<T>(mu, a, ga);
#pragma unroll
    for (int k = 0; k < 12; k++) a[k] = a[k] - ga[k];
    SpinorIO<T>::load(par ? psi_e : psi_o, g.Vh, j, b);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        cd s = mkc((T)0, (T)0);
#pragma unroll
        for (int sp = 0; sp < 4; sp++) s = cfma_conj(a[3 * sp + c], b[3 * sp + r], s);
        K[r * 3 + c] = s;
      }
    // second: lam(x+mu) against (1 + gamma) psi(x)
    SpinorIO<T>::load(par ? psi_o : psi_e, g.Vh, i, a);
    gamma_dyn<T>(mu, a, ga);
#pragma unroll
    for (int k = 0; k < 12; k++) a[k] = a[k] + ga[k];
    SpinorIO<T>::load(par ? lam_e : lam_o, g.Vh, j, b);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        cd s = K[r * 3 + c];
#pragma unroll
        for (int sp = 0; sp < 4; sp++) s = cfma_conj(a[3 * sp + c], b[3 * sp + r], s);
        K[r * 3 + c] = mkc((T)0.5 * sgn * s.re, (T)0.5 * sgn * s.im);
      }
  }

  // ---- clover part: two plaquettes per plane containing mu
  for (int nu = 0; nu < 4; nu++) {
    if (nu == mu) continue;
    const int al = mu < nu ? mu : nu, be = mu < nu ? nu : mu;
    const int p = plane_of(al, be);
    for (int h = 0; h < 2; h++) {
      // base corner b and the link's position j in the plaquette
      //   L0 = U_al(b), L1 = U_be(b+al), L2 = U_al(b+be)^dag, L3 = U_be(b)^dag
      int jpos;
      int b[4] = {x[0], x[1], x[2], x[3]};
      if (mu == al) {
        if (h == 0) { jpos = 0; } else { jpos = 2; step(g, b, be, -1); }
      } else {
        if (h == 0) { jpos = 1; step(g, b, al, -1); } else { jpos = 3; }
      }
      int cr[4][4];
#pragma unroll
      for (int k = 0; k < 4; k++)
#pragma unroll
        for (int m = 0; m < 4; m++) cr[k][m] = b[m];
      step(g, cr[1], al, +1);
      step(g, cr[2], al, +1);
      step(g, cr[2], be, +1);
      step(g, cr[3], be, +1);
      // factor k of the plaquette
      auto factor = [&](int k, cd u[9]) {
        switch (k & 3) {
          case 0: link_at<T>(g, gauge, cr[0], al, u); break;
          case 1: link_at<T>(g, gauge, cr[1], be, u); break;
          case 2: link_at<T>(g, gauge, cr[3], al, u); m_dag_inplace<T>(u); break;
          default: link_at<T>(g, gauge, cr[0], be, u); m_dag_inplace<T>(u); break;
        }
      };
      // R = ((W1 A1 + A1 W2) A2 + A1 A2 W3) A3 + A1 A2 A3 W0, A_n = L_{j+n}, W_n = W(corner j+n)
      cd A[9], M[9], Q[9], P[9], R[9];
      factor(jpos + 1, A);
      w_at<T>(g, W, cr[(jpos + 1) & 3], p, M);
      m_mul<T>(M, A, Q);
      w_at<T>(g, W, cr[(jpos + 2) & 3], p, M);
      m_mul_acc<T>(A, M, Q);
#pragma unroll
      for (int e = 0; e < 9; e++) P[e] = A[e];
      factor(jpos + 2, A);
      m_mul<T>(Q, A, R);
      m_mul<T>(P, A, Q);                     // Q = A1 A2
      w_at<T>(g, W, cr[(jpos + 3) & 3], p, M);
      m_mul_acc<T>(Q, M, R);                 // R = (W1 A1 + A1 W2) A2 + A1 A2 W3
      factor(jpos + 3, A);
      m_mul<T>(R, A, P);                     // P = R A3
      m_mul<T>(Q, A, R);                     // R = A1 A2 A3
      w_at<T>(g, W, cr[jpos], p, M);
      m_mul_acc<T>(R, M, P);                 // P = full R
      if (jpos >= 2) m_dag_inplace<T>(P);
#pragma unroll
      for (int e = 0; e < 9; e++) K[e] = K[e] + P[e];
    }
  }

  // ---- output
  cd o[9];
  if (kind == MG_FORCE_WIRTINGER) {
#pragma unroll
    for (int e = 0; e < 9; e++) o[e] = K[e];
    m_dag_inplace<T>(o);
  } else {
    cd u[9], G[9];
    load_link<T>(gauge, g.Vh, par, mu, i, u);
    m_mul<T>(u, K, G);                       // G = i U K (the i is applied below)
#pragma unroll
    for (int e = 0; e < 9; e++) G[e] = times_i(G[e]);
    // H = (G + G^dag)/2, F = (H - tr(H)/3)/2
    const T trh = (G[0].re + G[4].re + G[8].re) / (T)3;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        cd hh = G[a * 3 + c] + conj(G[c * 3 + a]);
        hh = mkc((T)0.5 * hh.re, (T)0.5 * hh.im);
        if (a == c) hh.re -= trh;
        o[a * 3 + c] = mkc((T)0.5 * hh.re, (T)0.5 * hh.im);
      }
  }
  const size_t lex = ((((size_t)x[3] * g.L[2] + x[2]) * g.L[1] + x[1]) * g.L[0] + x[0]);
  double2* dst = out + (lex * 4 + mu) * 9;
#pragma unroll
  for (int e = 0; e < 9; e++) dst[e] = make_double2((double)o[e].re, (double)o[e].im);
}

// psi <- gamma_5 psi on an ABI fine vector (complex128 [site][spin][colour])
__global__ void k_gamma5_abi(double2* v, size_t sites) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= sites * 6) return;
  const size_t site = t / 6, k = 6 + t % 6;   // spins 2, 3
  double2 z = v[site * 12 + k];
  v[site * 12 + k] = make_double2(-z.x, -z.y);
}
}  // namespace

void gamma5_abi(double* v, size_t sites, cudaStream_t s) {
  const size_t n = sites * 6;
  const int bs = 256;
  k_gamma5_abi<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>((double2*)v, sites);
  MG_LAUNCH();
}

template <typename T>
void gauge_force_t(Ctx* c, double* out_abi, const double* lam_abi, const double* psi_abi, int kind) {
  const Geom& g = c->g;
  const size_t half = 24 * c->Vh;   // reals per half vector
  DBuf vec(sizeof(T) * 4 * half);
  DBuf W(sizeof(T) * 2 * 6 * 9 * c->V);
  T* lam_e = vec.as<T>();
  T* lam_o = lam_e + half;
  T* psi_e = lam_o + half;
  T* psi_o = psi_e + half;
  constexpr bool f32 = std::is_same<T, float>::value;
  pack_spinor(g, lam_abi, lam_e, lam_o, f32, c->stream);
  pack_spinor(g, psi_abi, psi_e, psi_o, f32, c->stream);
  const int bs = 128;
  const int nb = (int)((2 * c->Vh + bs - 1) / bs);
  typedef typename V2of<T>::type V2;
  k_force_insertion<T><<<nb, bs, 0, c->stream>>>(g, lam_e, lam_o, psi_e, psi_o, (T)c->csw, (T)c->csw_t, W.as<V2>());
  MG_LAUNCH();
  k_force_links<T><<<dim3(nb, 4), bs, 0, c->stream>>>(g, lam_e, lam_o, psi_e, psi_o, c->gauge<T>(), W.as<V2>(), kind,
                                                      (double2*)out_abi);
  MG_LAUNCH();
  c->sync();
}

void gauge_force(Ctx* c, double* out_abi, const double* lam_abi, const double* psi_abi, int kind) {
  if (kind & MG_FORCE_FP32)
    gauge_force_t<float>(c, out_abi, lam_abi, psi_abi, kind & ~MG_FORCE_FP32);
  else
    gauge_force_t<double>(c, out_abi, lam_abi, psi_abi, kind);
}
}  // namespace mg
