// Device-side building blocks shared by the kernels: complex arithmetic,
// even-odd lattice geometry and the internal field layouts.
//
// Internal layouts (chosen for coalesced, vectorised access on sm_103a; the
// C ABI exchanges complex128 in lexicographic order and pack/unpack kernels
// convert):
//  * fine spinor, one parity: structure-of-chunks, 6 chunks of two complex
//    numbers per site -- FP32: float4[6][Vh], FP64: (2 x double2)[6][Vh] --
//    so both precisions order the complex numbers identically.  Complex
//    index within a site is 3*spin + colour.  A whole-lattice fine vector is
//    [even half][odd half].
//  * gauge, per (parity p, direction mu): complex[9][Vh], entry a*3+b of
//    U_mu(x) for the site x of parity p with checkerboard index i.
//  * clover (A or A^{-1}), per parity: 72 reals per site, float4[18][Vh] or
//    double2[36][Vh]; two Hermitian 6x6 chiral blocks, each stored as 6 real
//    diagonal entries then the 15 strictly-lower entries (i > j, index
//    i(i-1)/2 + j) as (re, im).
//  * coarse vectors: [site][ndof] complex, sites in even-odd order (all even
//    sites, then all odd) when every coarse extent is even, lexicographic
//    otherwise.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace mg {

template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mkc(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mkc(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mkc(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a) { return mkc(-a.re, -a.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mkc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mkc(s * a.re, s * a.im); }
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return mkc(a.re, -a.im); }
// i * a
template <typename T>
__device__ __forceinline__ cx<T> times_i(cx<T> a) { return mkc(-a.im, a.re); }
// acc + a * b
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename T>
__device__ __forceinline__ cx<T> cfma_conj(cx<T> a, cx<T> b, cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}

// --------------------------------------------------------------------------- geometry
struct Geom {
  int L[4];      // Lx, Ly, Lz, Lt (all even on the fine level)
  int Vh;        // half volume
  int xh;        // Lx / 2
  int apbc;      // 1: antiperiodic fermion boundary in t
  double w[4];   // hopping weight of each direction (1 everywhere: the isotropic operator)
};

// Coordinates of checkerboard index `cb` of parity `par`.
__device__ __forceinline__ void cb_coords(const Geom& g, int cb, int par, int c[4]) {
  int xhh = cb % g.xh;
  int r = cb / g.xh;
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
  c[0] = 2 * xhh + ((par + c[1] + c[2] + c[3]) & 1);
}

__device__ __forceinline__ int cb_index(const Geom& g, const int c[4]) {
  return ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.xh + (c[0] >> 1);
}

// --------------------------------------------------------------------------- fine spinor IO
template <typename T>
struct SpinorIO;

template <>
struct SpinorIO<float> {
  // 6 float4 chunks per site
  static __device__ __forceinline__ void load(const float* base, int Vh, int i, cx<float> s[12]) {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int q = 0; q < 6; q++) {
      float4 v = p[(size_t)q * Vh + i];
      s[2 * q] = mkc(v.x, v.y);
      s[2 * q + 1] = mkc(v.z, v.w);
    }
  }
  static __device__ __forceinline__ void store(float* base, int Vh, int i, const cx<float> s[12]) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int q = 0; q < 6; q++) p[(size_t)q * Vh + i] = make_float4(s[2 * q].re, s[2 * q].im, s[2 * q + 1].re, s[2 * q + 1].im);
  }
  // complex component c (0..11) of site i
  static __device__ __forceinline__ cx<float> get(const float* base, int Vh, int i, int c) {
    const float2* p = reinterpret_cast<const float2*>(base);
    float2 v = p[((size_t)(c >> 1) * Vh + i) * 2 + (c & 1)];
    return mkc(v.x, v.y);
  }
  static __device__ __forceinline__ void put(float* base, int Vh, int i, int c, cx<float> z) {
    float2* p = reinterpret_cast<float2*>(base);
    p[((size_t)(c >> 1) * Vh + i) * 2 + (c & 1)] = make_float2(z.re, z.im);
  }
};

// FP64 uses the same complex ordering as FP32 -- 6 chunks of two complex
// numbers (32 bytes) per site -- so that element-wise precision conversion
// of whole vectors (the mixed-precision GCR) keeps every component in place.
template <>
struct SpinorIO<double> {
  static __device__ __forceinline__ void load(const double* base, int Vh, int i, cx<double> s[12]) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int q = 0; q < 6; q++) {
      const double2 a = p[((size_t)q * Vh + i) * 2];
      const double2 b = p[((size_t)q * Vh + i) * 2 + 1];
      s[2 * q] = mkc(a.x, a.y);
      s[2 * q + 1] = mkc(b.x, b.y);
    }
  }
  static __device__ __forceinline__ void store(double* base, int Vh, int i, const cx<double> s[12]) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int q = 0; q < 6; q++) {
      p[((size_t)q * Vh + i) * 2] = make_double2(s[2 * q].re, s[2 * q].im);
      p[((size_t)q * Vh + i) * 2 + 1] = make_double2(s[2 * q + 1].re, s[2 * q + 1].im);
    }
  }
  static __device__ __forceinline__ cx<double> get(const double* base, int Vh, int i, int c) {
    const double2* p = reinterpret_cast<const double2*>(base);
    double2 v = p[((size_t)(c >> 1) * Vh + i) * 2 + (c & 1)];
    return mkc(v.x, v.y);
  }
  static __device__ __forceinline__ void put(double* base, int Vh, int i, int c, cx<double> z) {
    double2* p = reinterpret_cast<double2*>(base);
    p[((size_t)(c >> 1) * Vh + i) * 2 + (c & 1)] = make_double2(z.re, z.im);
  }
};

// --------------------------------------------------------------------------- gauge IO
template <typename T>
__device__ __forceinline__ void load_link(const T* gauge, int Vh, int par, int mu, int i, cx<T> u[9]) {
  using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const V2* p = reinterpret_cast<const V2*>(gauge) + (size_t)(par * 4 + mu) * 9 * Vh;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    V2 v = p[(size_t)e * Vh + i];
    u[e] = mkc(v.x, v.y);
  }
}

// --------------------------------------------------------------------------- clover IO
// Loads chiral block `b` (36 reals) of the packed clover at site i.
template <typename T>
struct CloverIO;

template <>
struct CloverIO<float> {
  static __device__ __forceinline__ void load_block(const float* base, int Vh, int i, int b, float r[36]) {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int q = 0; q < 9; q++) {
      float4 v = p[(size_t)(9 * b + q) * Vh + i];
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  }
  static __device__ __forceinline__ void store_block(float* base, int Vh, int i, int b, const float r[36]) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int q = 0; q < 9; q++) p[(size_t)(9 * b + q) * Vh + i] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  }
};

template <>
struct CloverIO<double> {
  static __device__ __forceinline__ void load_block(const double* base, int Vh, int i, int b, double r[36]) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int q = 0; q < 18; q++) {
      double2 v = p[(size_t)(18 * b + q) * Vh + i];
      r[2 * q] = v.x;
      r[2 * q + 1] = v.y;
    }
  }
  static __device__ __forceinline__ void store_block(double* base, int Vh, int i, int b, const double r[36]) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int q = 0; q < 18; q++) p[(size_t)(18 * b + q) * Vh + i] = make_double2(r[2 * q], r[2 * q + 1]);
  }
};

// y = C x for one packed Hermitian 6x6 block r[36] (diag, then lower (i>j)).
template <typename T>
__device__ __forceinline__ void herm6_apply(const T r[36], const cx<T> x[6], cx<T> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; i++) y[i] = mkc(r[i] * x[i].re, r[i] * x[i].im);
#pragma unroll
  for (int i = 1; i < 6; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      const int m = i * (i - 1) / 2 + j;
      cx<T> a = mkc(r[6 + 2 * m], r[6 + 2 * m + 1]);  // A_ij, i > j
      y[i] = cfma(a, x[j], y[i]);
      y[j] = cfma_conj(a, x[i], y[j]);                 // A_ji = conj(A_ij)
    }
  }
}

}  // namespace mg
