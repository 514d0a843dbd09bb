// Krylov solvers the paper compares multigrid against (section "Results"):
// BiCGStab, CG on the normal equations (CGNR) and, built on BiCGStab, a
// mixed-precision solver by iterative refinement (driven from solver.cu).
// They run on the even-odd reduced operator D_r with the same fine kernels as
// the multigrid solve; the scalars of each iteration go through the host.
#include <complex>

#include "internal.h"

namespace mg {

namespace {
using cplx = std::complex<double>;

// gamma_5 = diag(1, 1, -1, -1) in spin (chiral basis).  A half vector in the
// internal layout is six chunks of two complex components (component =
// 3 spin + colour), chunk-major over the sites, so spins 2 and 3 are the last
// three chunks: the second half of the vector.
template <typename T>
void gamma5_half(Ctx* c, T* v) {
  T* hi = v + 12 * (size_t)c->Vh;  // 6 Vh complex numbers in
  blas_axpby<T>(0.0, hi, -1.0, hi, 6 * (size_t)c->Vh, c->stream);
}
}  // namespace

// D_r = S A_e^{-1} with S = A_e - H_eo A_o^{-1} H_oe the Schur complement.
// gamma_5-hermiticity of D (H_eo^dag = gamma_5 H_oe gamma_5) and the clover
// blocks being Hermitian and commuting with gamma_5 give S^dag = gamma_5 S
// gamma_5, so D_r^dag = A_e^{-1} gamma_5 S gamma_5 = gamma_5 A_e^{-1} D_r A_e gamma_5.
template <typename T>
void dr_dagger(Ctx* c, FineOps<T>& F, T* out, const T* in, T* tmp) {
  const size_t n = 12 * (size_t)c->Vh;
  blas_convert<T, T>(tmp, in, n, c->stream);
  gamma5_half(c, tmp);
  clover_apply<T>(c->g, out, tmp, c->A<T>(0), c->stream);     // A_e gamma_5 in
  F.Dr(tmp, out);                                               // D_r A_e gamma_5 in
  clover_apply<T>(c->g, out, tmp, c->Ainv<T>(0), c->stream);  // A_e^{-1} D_r A_e gamma_5 in
  gamma5_half(c, out);
}

template <typename T>
Krylov<T>::Krylov(Ctx* c, size_t n) : c_(c), n_(n) {
  for (DBuf* d : {&r_, &rh_, &p_, &v_, &s_, &t_, &q_}) {
    d->alloc(sizeof(T) * 2 * n);
    MG_CUDA(cudaMemsetAsync(d->get(), 0, sizeof(T) * 2 * n, c->stream));
  }
  sc_.alloc(sizeof(double) * 16);
  coef_.alloc(sizeof(double) * 16);
  MG_CUDA(cudaMallocHost(&hcoef_, sizeof(double) * 16));
}

template <typename T>
Krylov<T>::~Krylov() {
  if (hcoef_) cudaFreeHost(hcoef_);
}

// complex coefficients for blas_lincomb, through pinned memory: every caller
// writes them after a host synchronisation, so the previous copy has run
template <typename T>
const double* Krylov<T>::coefs(std::initializer_list<cplx> z) {
  int k = 0;
  for (const cplx& v : z) {
    hcoef_[2 * k] = v.real();
    hcoef_[2 * k + 1] = v.imag();
    k++;
  }
  MG_CUDA(cudaMemcpyAsync(coef_.get(), hcoef_, sizeof(double) * 2 * k, cudaMemcpyHostToDevice, c_->stream));
  return coef_.as<double>();
}

// BiCGStab (van der Vorst) on A x = b.  Restarts (rh = r, p = v = 0) when
// <rh, r> or <rh, A p> vanishes or omega does, and stops unconverged when the
// breakdown recurs on the restart itself.  Convergence is tested on the
// recursively updated residual at the half step (s) and the full step (r).
template <typename T>
typename Krylov<T>::Result Krylov<T>::bicgstab(const Op& A, T* x, const T* b, bool x0_zero, double tol_abs,
                                               int maxit) {
  Result res;
  cudaStream_t s = c_->stream;
  const size_t n = n_;
  T* r = r_.as<T>();
  T* rh = rh_.as<T>();
  T* p = p_.as<T>();
  T* v = v_.as<T>();
  T* sv = s_.as<T>();
  T* t = t_.as<T>();
  double* d = sc_.as<double>();
  double h[8];
  if (x0_zero) {
    blas_zero<T>(x, n, s);
    blas_convert<T, T>(r, b, n, s);
  } else {
    A(r, x);
    blas_axpby<T>(1.0, b, -1.0, r, n, s);  // r = b - A x
  }
  blas_norm2<T>(r, n, d, c_->ws, s);
  double rn = std::sqrt(c_->read_scalar(d));
  res.rnorm = rn;
  if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite residual in BiCGStab");
  if (rn <= tol_abs) {
    res.converged = true;
    return res;
  }
  bool fresh = true;
  cplx rho(1.0, 0.0), alpha(1.0, 0.0), omega(1.0, 0.0), rho_new;
  while (res.iterations < maxit) {
    const bool restarted = fresh;
    if (fresh) {
      blas_convert<T, T>(rh, r, n, s);
      blas_convert<T, T>(p, r, n, s);
      rho_new = cplx(rn * rn, 0.0);
    } else {
      const cplx beta = (rho_new / rho) * (alpha / omega);
      blas_convert<T, T>(q_.as<T>(), r, n, s);            // p = r + beta p - beta omega v
      const T* Z[2] = {p, v};
      blas_lincomb<T, T>(q_.as<T>(), Z, coefs({beta, -beta * omega}), 2, 1.0, n, s);
      std::swap(p_, q_);
      p = p_.as<T>();
    }
    fresh = false;
    A(v, p);
    blas_cdot<T>(rh, v, n, d, c_->ws, s);
    c_->read_scalars(d, h, 2);
    const cplx rv(h[0], h[1]);
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) raise(MG_ERR_NAN, "non-finite scalar in BiCGStab");
    if (std::abs(rv) <= 1e-30 * rn * rn) {
      // breakdown: restart from the current residual, unless this step already
      // was the restart (<r, A r> = 0: no progress possible from here)
      if (restarted) break;
      res.restarts++;
      fresh = true;
      continue;
    }
    alpha = rho_new / rv;
    blas_convert<T, T>(sv, r, n, s);  // s = r - alpha v
    {
      const T* Z[1] = {v};
      blas_lincomb<T, T>(sv, Z, coefs({-alpha}), 1, 1.0, n, s);
    }
    A(t, sv);
    {
      // {<t,t>, Re<t,s>, Im<t,s>} and ||s||^2
      blas_dot2<T>(t, sv, n, d, c_->ws, s);
      blas_norm2<T>(sv, n, d + 3, c_->ws, s);
      c_->read_scalars(d, h, 4);
    }
    res.iterations++;
    const double sn = std::sqrt(h[3]);
    if (!std::isfinite(sn) || !std::isfinite(h[0])) raise(MG_ERR_NAN, "non-finite scalar in BiCGStab");
    if (sn <= tol_abs || h[0] == 0.0) {  // converged at the half step (or A s = 0: s is the exact residual)
      const T* Z[1] = {p};
      blas_lincomb<T, T>(x, Z, coefs({alpha}), 1, 1.0, n, s);
      blas_convert<T, T>(r, sv, n, s);
      res.rnorm = sn;
      res.converged = sn <= tol_abs;
      if (res.converged) break;
      fresh = true;
      rn = sn;
      res.restarts++;
      continue;
    }
    omega = cplx(h[1], h[2]) / h[0];
    {
      const T* Z[2] = {p, sv};  // x += alpha p + omega s
      const double* cf = coefs({alpha, omega, -omega});
      blas_lincomb<T, T>(x, Z, cf, 2, 1.0, n, s);
      blas_convert<T, T>(r, sv, n, s);  // r = s - omega t
      const T* Zt[1] = {t};
      blas_lincomb<T, T>(r, Zt, cf + 4, 1, 1.0, n, s);
    }
    // <rh, r> for the next step and ||r||^2 in one reduction
    const T* V[2] = {rh, r};
    blas_multidot<T>(V, 2, r, n, d, c_->ws, s);
    c_->read_scalars(d, h, 4);
    rn = std::sqrt(h[2]);
    res.rnorm = rn;
    if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite residual in BiCGStab");
    if (rn <= tol_abs) {
      res.converged = true;
      break;
    }
    rho = rho_new;
    rho_new = cplx(h[0], h[1]);
    if (std::abs(omega) == 0.0 || std::abs(rho_new) <= 1e-30 * rn * rn) {
      res.restarts++;
      fresh = true;
    }
  }
  return res;
}

// CG on A^dag A x = A^dag b (CGLS form: the residual r = b - A x is updated
// alongside, and the stopping test is ||r|| <= tol_abs).
template <typename T>
typename Krylov<T>::Result Krylov<T>::cgnr(const Op& A, const Op& Adag, T* x, const T* b, bool x0_zero,
                                           double tol_abs, int maxit) {
  Result res;
  cudaStream_t s = c_->stream;
  const size_t n = n_;
  T* r = r_.as<T>();
  T* z = rh_.as<T>();
  T* p = p_.as<T>();
  T* w = v_.as<T>();
  double* d = sc_.as<double>();
  double h[2];
  if (x0_zero) {
    blas_zero<T>(x, n, s);
    blas_convert<T, T>(r, b, n, s);
  } else {
    A(r, x);
    blas_axpby<T>(1.0, b, -1.0, r, n, s);
  }
  Adag(z, r);
  blas_convert<T, T>(p, z, n, s);
  blas_norm2<T>(r, n, d, c_->ws, s);
  blas_norm2<T>(z, n, d + 1, c_->ws, s);
  c_->read_scalars(d, h, 2);
  double rn = std::sqrt(h[0]), zz = h[1];
  res.rnorm = rn;
  if (!std::isfinite(rn) || !std::isfinite(zz)) raise(MG_ERR_NAN, "non-finite residual in CGNR");
  if (rn <= tol_abs) {
    res.converged = true;
    return res;
  }
  while (res.iterations < maxit && zz > 0.0) {
    A(w, p);
    blas_norm2<T>(w, n, d, c_->ws, s);
    const double ww = c_->read_scalar(d);
    if (!(ww > 0.0) || !std::isfinite(ww)) raise(MG_ERR_NAN, "non-finite or zero <Ap, Ap> in CGNR");
    const double a = zz / ww;
    blas_axpby<T>(a, p, 1.0, x, n, s);
    blas_axpby<T>(-a, w, 1.0, r, n, s);
    Adag(z, r);
    blas_norm2<T>(r, n, d, c_->ws, s);
    blas_norm2<T>(z, n, d + 1, c_->ws, s);
    c_->read_scalars(d, h, 2);
    res.iterations++;
    rn = std::sqrt(h[0]);
    res.rnorm = rn;
    if (!std::isfinite(rn) || !std::isfinite(h[1])) raise(MG_ERR_NAN, "non-finite residual in CGNR");
    if (rn <= tol_abs) {
      res.converged = true;
      break;
    }
    const double beta = h[1] / zz;
    zz = h[1];
    blas_axpby<T>(1.0, z, beta, p, n, s);  // p = z + beta p
  }
  return res;
}

template void dr_dagger<double>(Ctx*, FineOps<double>&, double*, const double*, double*);
template void dr_dagger<float>(Ctx*, FineOps<float>&, float*, const float*, float*);
template class Krylov<double>;
template class Krylov<float>;

}  // namespace mg
