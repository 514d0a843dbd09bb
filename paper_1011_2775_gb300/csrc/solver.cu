// Host orchestration of the even-odd solve (section "Red-black
// preconditioning") and the flexible GCR used at every level (sections
// "Adaptive multigrid" and "Implementation").
//
// GCR(m) keeps all Krylov scalars on the device: one fused multi-dot, one
// fused orthogonalise-and-norm pass and one fused residual update per
// iteration, with the solution update deferred to the end of each restart
// cycle (back substitution of the triangular system).  In exact arithmetic
// this is the textbook flexible GCR; deferring the update lets the
// preconditioned directions z_j stay in the preconditioner's precision.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace mg {

// --------------------------------------------------------------------------- errors / memory
void raise(int code, const std::string& what) { throw Error{code, what}; }

void cuda_check(cudaError_t e, const char* expr, const char* file, int line) {
  if (e == cudaSuccess) return;
  std::string msg = std::string(cudaGetErrorString(e)) + " in " + expr + " at " + file + ":" + std::to_string(line);
  if (e == cudaErrorMemoryAllocation) raise(MG_ERR_ALLOC, msg);
  raise(MG_ERR_CUDA, msg);
}

namespace {
std::atomic<long long> g_launches{0};
}

void launch_check(const char* file, int line) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cuda_check(cudaGetLastError(), "kernel launch", file, line);
}

long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void DBuf::alloc(size_t bytes) {
  release();
  if (bytes == 0) return;
  MG_CUDA(cudaMalloc(&p_, bytes));
  bytes_ = bytes;
}

void DBuf::release() {
  if (p_) cudaFree(p_);
  p_ = nullptr;
  bytes_ = 0;
}

void Workspace::init() {
  partials.alloc(sizeof(double) * kMaxBlocks * kMaxResults);
  counter.alloc(sizeof(unsigned) * 4);
  MG_CUDA(cudaMemset(counter.get(), 0, sizeof(unsigned) * 4));
  scalars.alloc(sizeof(double) * kScalars);
  MG_CUDA(cudaMemset(scalars.get(), 0, sizeof(double) * kScalars));
  flags.alloc(sizeof(int) * FLAG_COUNT);
  MG_CUDA(cudaMemset(flags.get(), 0, sizeof(int) * FLAG_COUNT));
  mcounters.alloc(sizeof(unsigned) * kMultiCounters);
  MG_CUDA(cudaMemset(mcounters.get(), 0, sizeof(unsigned) * kMultiCounters));
  if (!host) MG_CUDA(cudaMallocHost((void**)&host, sizeof(double) * 256));
}

Workspace::~Workspace() {
  if (host) cudaFreeHost(host);
  host = nullptr;
}

void Ctx::sync() { MG_CUDA(cudaStreamSynchronize(stream)); }

double Ctx::read_scalar(const double* d) {
  MG_CUDA(cudaMemcpyAsync(ws.host, d, sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  return ws.host[0];
}

void Ctx::read_scalars(const double* d, double* h, int n) {
  MG_CUDA(cudaMemcpyAsync(ws.host, d, sizeof(double) * n, cudaMemcpyDeviceToHost, stream));
  sync();
  std::memcpy(h, ws.host, sizeof(double) * n);
}

int Ctx::read_flag(int which, bool clear) {
  int v = 0;
  MG_CUDA(cudaMemcpyAsync(&v, ws.flags.as<int>() + which, sizeof(int), cudaMemcpyDeviceToHost, stream));
  sync();
  if (clear && v) MG_CUDA(cudaMemsetAsync(ws.flags.as<int>() + which, 0, sizeof(int), stream));
  return v;
}

// --------------------------------------------------------------------------- fine operators
template <typename T>
FineOps<T>::FineOps(Ctx* ctx) : c(ctx) {
  t1.alloc(sizeof(T) * 24 * c->Vh);
  t2.alloc(sizeof(T) * 24 * c->Vh);
}

template <typename T>
void FineOps<T>::Dr(T* out_e, const T* in_e) {
  const Geom& g = c->g;
  T* s = t1.as<T>();
  T* t = t2.as<T>();
  clover_apply<T>(g, s, in_e, c->Ainv<T>(0), c->stream);                                     // s_e = A_e^{-1} y_e
  dslash<T>(g, EPI_CH, 1, t, s, c->gauge<T>(), c->Ainv<T>(1), nullptr, 0.0, 0xff, c->stream);  // t_o = A_o^{-1} H_oe s_e
  dslash<T>(g, EPI_XPAY, 0, out_e, t, c->gauge<T>(), nullptr, in_e, -1.0, 0xff, c->stream);    // y_e - H_eo t_o
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::br(T* out_e, const T* b_e, const T* b_o) {
  const Geom& g = c->g;
  T* t = t1.as<T>();
  clover_apply<T>(g, t, b_o, c->Ainv<T>(1), c->stream);
  dslash<T>(g, EPI_XPAY, 0, out_e, t, c->gauge<T>(), nullptr, b_e, -1.0, 0xff, c->stream);
  c->dslash_launches += 1;
}

template <typename T>
void FineOps<T>::reconstruct(T* x_e, T* x_o, const T* y_e, const T* b_o) {
  const Geom& g = c->g;
  clover_apply<T>(g, x_e, y_e, c->Ainv<T>(0), c->stream);
  dslash<T>(g, EPI_C_XPAY, 1, x_o, x_e, c->gauge<T>(), c->Ainv<T>(1), b_o, -1.0, 0xff, c->stream);
  c->dslash_launches += 1;
}

template <typename T>
void FineOps<T>::D(T* oe, T* oo, const T* ie, const T* io) {
  const Geom& g = c->g;
  dslash<T>(g, EPI_CX_PAY, 0, oe, io, c->gauge<T>(), c->A<T>(0), ie, 1.0, 0xff, c->stream);
  dslash<T>(g, EPI_CX_PAY, 1, oo, ie, c->gauge<T>(), c->A<T>(1), io, 1.0, 0xff, c->stream);
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::Dp(T* oe, T* oo, const T* ie, const T* io) {
  const Geom& g = c->g;
  T* se = t1.as<T>();
  T* so = t2.as<T>();
  clover_apply<T>(g, se, ie, c->Ainv<T>(0), c->stream);
  clover_apply<T>(g, so, io, c->Ainv<T>(1), c->stream);
  dslash<T>(g, EPI_XPAY, 0, oe, so, c->gauge<T>(), nullptr, ie, 1.0, 0xff, c->stream);
  dslash<T>(g, EPI_XPAY, 1, oo, se, c->gauge<T>(), nullptr, io, 1.0, 0xff, c->stream);
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::H(T* oe, T* oo, const T* ie, const T* io) {
  const Geom& g = c->g;
  dslash<T>(g, EPI_H, 0, oe, io, c->gauge<T>(), nullptr, nullptr, 0.0, 0xff, c->stream);
  dslash<T>(g, EPI_H, 1, oo, ie, c->gauge<T>(), nullptr, nullptr, 0.0, 0xff, c->stream);
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::M(T* oe, T* oo, const T* ie, const T* io, bool inverse) {
  const Geom& g = c->g;
  clover_apply<T>(g, oe, ie, inverse ? c->Ainv<T>(0) : c->A<T>(0), c->stream);
  clover_apply<T>(g, oo, io, inverse ? c->Ainv<T>(1) : c->A<T>(1), c->stream);
}

// ---- multi-RHS forms
template <typename T>
void FineOps<T>::reserve_multi(int nrhs) {
  const size_t need = sizeof(T) * 24 * c->Vh * (size_t)nrhs;
  if (mcap >= need) return;
  m1.alloc(need);
  m2.alloc(need);
  mcap = need;
}

template <typename T>
int FineOps<T>::block_for(const char* kernel, int nrhs, const std::function<void(int)>& launch) {
  TuneKey k{kernel, {c->dims[0], c->dims[1], c->dims[2], c->dims[3]}, nrhs, std::is_same<T, float>::value ? 1 : 0};
  return tuned_block(k, dslash_mrhs_configs(std::is_same<T, float>::value), launch, c->stream);
}

template <typename T>
void FineOps<T>::Dr_multi(T* out_e, const T* in_e, int nrhs, size_t stride) {
  const Geom& g = c->g;
  cudaStream_t st = c->stream;
  reserve_multi(nrhs);
  const size_t ts = 24 * c->Vh;  // temporaries are packed at half-vector stride
  if (stride != ts) raise(MG_ERR_ARG, "multi-RHS operators take packed half vectors");
  T* s = m1.as<T>();
  T* t = m2.as<T>();
  clover_apply_mrhs<T>(g, nrhs, stride, s, in_e, c->Ainv<T>(0), st);
  auto k1 = [&](int b) {
    dslash_mrhs<T>(g, EPI_CH, 1, nrhs, ts, t, s, c->gauge<T>(), c->Ainv<T>(1), nullptr, 0.0, 0xff, b, st);
  };
  auto k2 = [&](int b) {
    dslash_mrhs<T>(g, EPI_XPAY, 0, nrhs, ts, out_e, t, c->gauge<T>(), nullptr, in_e, -1.0, 0xff, b, st);
  };
  k1(block_for("dslash_ch", nrhs, k1));
  k2(block_for("dslash_xpay", nrhs, k2));
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::br_multi(T* out_e, const T* b_e, const T* b_o, int nrhs, size_t stride) {
  const Geom& g = c->g;
  if (stride != 24 * c->Vh) raise(MG_ERR_ARG, "multi-RHS operators take packed half vectors");
  reserve_multi(nrhs);
  T* t = m1.as<T>();
  clover_apply_mrhs<T>(g, nrhs, stride, t, b_o, c->Ainv<T>(1), c->stream);
  dslash_mrhs<T>(g, EPI_XPAY, 0, nrhs, stride, out_e, t, c->gauge<T>(), nullptr, b_e, -1.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  c->dslash_launches += 1;
}

template <typename T>
void FineOps<T>::reconstruct_multi(T* x_e, T* x_o, const T* y_e, const T* b_o, int nrhs, size_t stride) {
  const Geom& g = c->g;
  clover_apply_mrhs<T>(g, nrhs, stride, x_e, y_e, c->Ainv<T>(0), c->stream);
  dslash_mrhs<T>(g, EPI_C_XPAY, 1, nrhs, stride, x_o, x_e, c->gauge<T>(), c->Ainv<T>(1), b_o, -1.0, 0xff,
                 dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  c->dslash_launches += 1;
}

template <typename T>
void FineOps<T>::D_multi(T* oe, T* oo, const T* ie, const T* io, int nrhs, size_t stride) {
  const Geom& g = c->g;
  dslash_mrhs<T>(g, EPI_CX_PAY, 0, nrhs, stride, oe, io, c->gauge<T>(), c->A<T>(0), ie, 1.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  dslash_mrhs<T>(g, EPI_CX_PAY, 1, nrhs, stride, oo, ie, c->gauge<T>(), c->A<T>(1), io, 1.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::Dp_multi(T* oe, T* oo, const T* ie, const T* io, int nrhs, size_t stride) {
  const Geom& g = c->g;
  if (stride != 24 * c->Vh) raise(MG_ERR_ARG, "multi-RHS operators take packed half vectors");
  reserve_multi(nrhs);
  T* se = m1.as<T>();
  T* so = m2.as<T>();
  clover_apply_mrhs<T>(g, nrhs, stride, se, ie, c->Ainv<T>(0), c->stream);
  clover_apply_mrhs<T>(g, nrhs, stride, so, io, c->Ainv<T>(1), c->stream);
  dslash_mrhs<T>(g, EPI_XPAY, 0, nrhs, stride, oe, so, c->gauge<T>(), nullptr, ie, 1.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  dslash_mrhs<T>(g, EPI_XPAY, 1, nrhs, stride, oo, se, c->gauge<T>(), nullptr, io, 1.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::H_multi(T* oe, T* oo, const T* ie, const T* io, int nrhs, size_t stride) {
  const Geom& g = c->g;
  dslash_mrhs<T>(g, EPI_H, 0, nrhs, stride, oe, io, c->gauge<T>(), nullptr, nullptr, 0.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  dslash_mrhs<T>(g, EPI_H, 1, nrhs, stride, oo, ie, c->gauge<T>(), nullptr, nullptr, 0.0, 0xff, dslash_mrhs_default(std::is_same<T, float>::value), c->stream);
  c->dslash_launches += 2;
}

template <typename T>
void FineOps<T>::M_multi(T* oe, T* oo, const T* ie, const T* io, bool inverse, int nrhs, size_t stride) {
  const Geom& g = c->g;
  clover_apply_mrhs<T>(g, nrhs, stride, oe, ie, inverse ? c->Ainv<T>(0) : c->A<T>(0), c->stream);
  clover_apply_mrhs<T>(g, nrhs, stride, oo, io, inverse ? c->Ainv<T>(1) : c->A<T>(1), c->stream);
}

template struct FineOps<float>;
template struct FineOps<double>;

// --------------------------------------------------------------------------- GCR
template <typename T, typename TZ>
GCR<T, TZ>::GCR(Ctx* c, size_t n, int m) : c_(c), n_(n), m_(m) {
  W_.resize(m);
  Z_.resize(m);
  for (int k = 0; k < m; k++) {
    W_[k].alloc(sizeof(T) * 2 * n);
    Z_[k].alloc(sizeof(TZ) * 2 * n);
  }
  r_.alloc(sizeof(T) * 2 * n);
  tmp_.alloc(sizeof(T) * 2 * n);
  scal_.alloc(sizeof(double) * (2 * (size_t)m * m + 5 * (size_t)m + 16));
  s_ = scal_.as<double>();
}

template <typename T, typename TZ>
typename GCR<T, TZ>::Result GCR<T, TZ>::solve(const Op& A, const Pre* M, T* x, const T* b, bool x0_zero,
                                                double tol_abs, int maxit, bool check, const LowOp* Al) {
  cudaStream_t s = c_->stream;
  const int m = m_;
  const size_t n = n_;
  T* r = r_.as<T>();
  T* tmp = tmp_.as<T>();
  double* beta = s_;
  double* alpha = beta + 2 * (size_t)m * m;
  double* gam = alpha + 2 * m;
  double* cc = gam + m;
  double* orth = cc + 2 * m;
  double* rn2 = orth + 4;
  std::vector<const T*> Wp(m);
  std::vector<const TZ*> Zp(m);
  for (int k = 0; k < m; k++) {
    Wp[k] = W_[k].as<T>();
    Zp[k] = Z_[k].as<TZ>();
  }
  Result res;
  if (x0_zero) {
    blas_zero<T>(x, n, s);
    blas_convert<T, T>(r, b, n, s);
  } else {
    A(tmp, x);
    blas_convert<T, T>(r, b, n, s);
    blas_axpby<T>(-1.0, tmp, 1.0, r, n, s);
  }
  if (check) {
    blas_norm2<T>(r, n, rn2, c_->ws, s);
    const double rr = c_->read_scalar(rn2);
    if (!std::isfinite(rr)) raise(MG_ERR_NAN, "non-finite residual");
    res.rnorm = std::sqrt(rr);
    if (res.rnorm <= tol_abs) {
      res.converged = true;
      return res;
    }
  }
  while (res.iterations < maxit) {
    int k = 0;
    bool done = false;
    while (k < m && res.iterations < maxit) {
      Range range(std::is_same<T, double>::value ? "outer gcr iteration" : "coarse gcr iteration");
      TZ* z = Z_[k].as<TZ>();
      T* w = W_[k].as<T>();
      if (M)
        (*M)(z, r);
      else
        blas_convert<T, TZ>(z, r, n, s);
      if (Al) {
        (*Al)(w, z);
      } else if (std::is_same<T, TZ>::value) {
        A(w, reinterpret_cast<const T*>(z));
      } else {
        blas_convert<TZ, T>(tmp, z, n, s);
        A(w, tmp);
      }
      if (k > 0) blas_multidot<T>(Wp.data(), k, w, n, beta + 2 * (size_t)m * k, c_->ws, s);
      blas_orth_update<T>(w, Wp.data(), beta + 2 * (size_t)m * k, k, r, n, orth, c_->ws, s);
      blas_r_update<T>(w, r, n, orth, alpha + 2 * k, gam + k, rn2, c_->ws, s);
      k++;
      res.iterations++;
      if (check) {
        const double rr = c_->read_scalar(rn2);
        if (!std::isfinite(rr)) raise(MG_ERR_NAN, "non-finite residual in GCR");
        res.rnorm = std::sqrt(rr);
        if (res.rnorm <= tol_abs) {
          done = true;
          break;
        }
      }
    }
    gcr_backsub(beta, m, alpha, gam, k, cc, s);
    blas_lincomb<T, TZ>(x, Zp.data(), cc, k, 1.0, n, s);
    res.restarts++;
    if (!check) continue;  // recurrence residual carries over
    // true residual at every restart
    A(tmp, x);
    blas_convert<T, T>(r, b, n, s);
    blas_axpby<T>(-1.0, tmp, 1.0, r, n, s);
    blas_norm2<T>(r, n, rn2, c_->ws, s);
    const double rr = c_->read_scalar(rn2);
    if (!std::isfinite(rr)) raise(MG_ERR_NAN, "non-finite true residual");
    res.rnorm = std::sqrt(rr);
    if (res.rnorm <= tol_abs) {
      res.converged = true;
      break;
    }
    (void)done;
  }
  return res;
}

template class GCR<double, float>;
template class GCR<double, double>;
template class GCR<float, float>;

template <typename T>
void mr_smooth(Ctx* c, const std::function<void(T*, const T*)>& A, T* e, T* r, T* w, size_t n, int nu, double* d_scr) {
  blas_zero<T>(e, n, c->stream);
  for (int it = 0; it < nu; it++) {
    A(w, r);
    blas_dot2<T>(w, r, n, d_scr, c->ws, c->stream);
    blas_mr_update<T>(e, r, w, d_scr, n, c->stream);
  }
}
template void mr_smooth<float>(Ctx*, const std::function<void(float*, const float*)>&, float*, float*, float*, size_t,
                               int, double*);
template void mr_smooth<double>(Ctx*, const std::function<void(double*, const double*)>&, double*, double*, double*,
                                size_t, int, double*);

// --------------------------------------------------------------------------- solve driver
namespace {
struct SolveBuffers {
  DBuf be, bo, xe, xo, y, br, te, to;
  DBuf r32, z32, w32;
  std::unique_ptr<FineOps<double>> F64;
  std::unique_ptr<GCR<double, float>> gcr_mg;
  std::unique_ptr<GCR<double, double>> gcr_eo;
  std::unique_ptr<FineOps<float>> F32;      // the comparison solvers' FP32 operator
  std::unique_ptr<Krylov<double>> kry64;
  std::unique_ptr<Krylov<float>> kry32;
  DBuf dag;                                 // D_r^dag temporary
  int restart = 0;
};

// inner solve of the mixed-precision BiCGStab: residual reduction per
// refinement step (FP32 BiCGStab)
constexpr double kMixedInnerTol = 1e-4;
}  // namespace


int solve_fine(Ctx* c, double* psi_abi, const double* eta_abi, double tol, int mode, mg_solve_info* info) {
  const size_t n = 12 * c->Vh;
  cudaStream_t s = c->stream;
  const int restart = c->params.restart_fine > 0 ? c->params.restart_fine : 16;
  SolveBuffers* B = static_cast<SolveBuffers*>(c->solve_work.get());
  if (!B || B->restart != restart) {
    c->solve_work.reset();
    std::shared_ptr<SolveBuffers> nb(new SolveBuffers());
    c->solve_work = nb;
    B = nb.get();
    for (DBuf* d : {&B->be, &B->bo, &B->xe, &B->xo, &B->y, &B->br, &B->te, &B->to}) d->alloc(sizeof(double) * 2 * n);
    B->r32.alloc(sizeof(float) * 2 * n);
    B->z32.alloc(sizeof(float) * 2 * n);
    B->w32.alloc(sizeof(float) * 2 * n);
    B->F64.reset(new FineOps<double>(c));
    B->restart = restart;
  }
  double* be = B->be.as<double>();
  double* bo = B->bo.as<double>();
  double* xe = B->xe.as<double>();
  double* xo = B->xo.as<double>();
  double* y = B->y.as<double>();
  double* br = B->br.as<double>();
  double* te = B->te.as<double>();
  double* to = B->to.as<double>();
  double* d_scr = c->ws.scalars.as<double>();
  FineOps<double>& F = *B->F64;

  pack_spinor(c->g, eta_abi, be, bo, false, s);
  blas_norm2<double>(be, n, d_scr, c->ws, s);
  blas_norm2<double>(bo, n, d_scr + 1, c->ws, s);
  double nn[2];
  c->read_scalars(d_scr, nn, 2);
  const double bnorm = std::sqrt(nn[0] + nn[1]);
  if (!std::isfinite(bnorm)) raise(MG_ERR_NAN, "non-finite source");
  if (bnorm == 0.0) {
    MG_CUDA(cudaMemsetAsync(psi_abi, 0, sizeof(double) * 24 * c->V, s));
    if (info) info->true_residual = 0.0;
    c->sync();
    return MG_OK;
  }
  F.br(br, be, bo);
  const double tol_r = 0.5 * tol * bnorm;
  auto Aop = [&](double* out, const double* in) { F.Dr(out, in); };
  const int maxit = c->params.maxit_fine > 0 ? c->params.maxit_fine : 500;
  int used = 0, restarts = 0;
  double true_res = INFINITY;
  bool first = true;
  for (int attempt = 0; attempt < 8 && used < maxit; attempt++) {
    if (mode == MG_MODE_MG) {
      if (!B->gcr_mg) B->gcr_mg.reset(new GCR<double, float>(c, n, restart));
      float* r32 = B->r32.as<float>();
      GCR<double, float>::Pre pre = [&](float* z, const double* r) {
        if (mg_precondition_graph(c, z, r, r32)) return;
        blas_convert<double, float>(r32, r, n, s);
        mg_precondition(c, z, r32);
      };
      // the Krylov directions' product in FP32 (the true residuals stay FP64)
      if (!B->F32) B->F32.reset(new FineOps<float>(c));
      float* w32 = B->w32.as<float>();
      GCR<double, float>::LowOp low = [&](double* w, const float* z) {
        B->F32->Dr(w32, z);
        blas_convert<float, double>(w, w32, n, s);
      };
      auto res = B->gcr_mg->solve(Aop, &pre, y, br, first, tol_r, maxit - used, true,
                                  c->params.outer_prec == MG_FP32 ? &low : nullptr);
      used += res.iterations;
      restarts += res.restarts;
    } else if (mode == MG_MODE_EO_GCR) {
      if (!B->gcr_eo) B->gcr_eo.reset(new GCR<double, double>(c, n, restart));
      auto res = B->gcr_eo->solve(Aop, nullptr, y, br, first, tol_r, maxit - used, true);
      used += res.iterations;
      restarts += res.restarts;
    } else if (mode == MG_MODE_BICGSTAB || mode == MG_MODE_CGNR) {
      if (!B->kry64) B->kry64.reset(new Krylov<double>(c, n));
      Krylov<double>::Result res;
      if (mode == MG_MODE_BICGSTAB) {
        res = B->kry64->bicgstab(Aop, y, br, first, tol_r, maxit - used);
      } else {
        if (!B->dag.get()) B->dag.alloc(sizeof(double) * 2 * n);
        auto Adag = [&](double* out, const double* in) { dr_dagger<double>(c, F, out, in, B->dag.as<double>()); };
        res = B->kry64->cgnr(Aop, Adag, y, br, first, tol_r, maxit - used);
      }
      used += res.iterations;
      restarts += res.restarts;
    } else {
      // mixed precision by iterative refinement: FP64 residual r = b_r - D_r y,
      // FP32 BiCGStab for D_r e = r to kMixedInnerTol ||r||, y += e
      if (!B->F32) B->F32.reset(new FineOps<float>(c));
      if (!B->kry32) B->kry32.reset(new Krylov<float>(c, n));
      FineOps<float>& F32 = *B->F32;
      auto A32 = [&](float* out, const float* in) { F32.Dr(out, in); };
      float* r32 = B->r32.as<float>();
      float* e32 = B->z32.as<float>();
      double* r = to;
      if (first) blas_zero<double>(y, n, s);
      while (used < maxit) {
        F.Dr(te, y);
        blas_convert<double, double>(r, br, n, s);
        blas_axpby<double>(-1.0, te, 1.0, r, n, s);  // r = b_r - D_r y
        blas_norm2<double>(r, n, d_scr, c->ws, s);
        const double rn = std::sqrt(c->read_scalar(d_scr));
        if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite residual in the refinement");
        if (rn <= tol_r) break;
        blas_convert<double, float>(r32, r, n, s);
        auto res = B->kry32->bicgstab(A32, e32, r32, true, std::max(kMixedInnerTol * rn, tol_r), maxit - used);
        used += res.iterations;
        restarts++;
        if (res.iterations == 0) break;
        const float* Z[1] = {e32};
        const double one[2] = {1.0, 0.0};
        MG_CUDA(cudaMemcpyAsync(d_scr + 8, one, sizeof(one), cudaMemcpyHostToDevice, s));
        blas_lincomb<double, float>(y, Z, d_scr + 8, 1, 1.0, n, s);  // y += e
      }
    }
    first = false;
    F.reconstruct(xe, xo, y, bo);
    F.D(te, to, xe, xo);
    blas_axpby<double>(1.0, be, -1.0, te, n, s);  // te = b_e - (Dx)_e
    blas_axpby<double>(1.0, bo, -1.0, to, n, s);
    blas_norm2<double>(te, n, d_scr, c->ws, s);
    blas_norm2<double>(to, n, d_scr + 1, c->ws, s);
    c->read_scalars(d_scr, nn, 2);
    true_res = std::sqrt(nn[0] + nn[1]) / bnorm;
    if (!std::isfinite(true_res)) raise(MG_ERR_NAN, "non-finite solution");
    if (true_res <= tol) break;
  }
  unpack_spinor(c->g, xe, xo, false, psi_abi, s);
  c->sync();
  if (info) {
    info->outer_iterations += used;
    info->restarts += restarts;
    if (true_res > info->true_residual || info->true_residual != info->true_residual) info->true_residual = true_res;
  }
  return true_res <= tol ? MG_OK : MG_ERR_NOT_CONVERGED;
}

}  // namespace mg
