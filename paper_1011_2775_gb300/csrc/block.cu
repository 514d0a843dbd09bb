// Several right-hand sides of one lattice solved together.
//
// The outer solver is the same flexible GCR(m) on D_r as solver.cu (section
// "Red-black preconditioning"; section "Implementation"), run for nb
// right-hand sides in lock-step: every iteration applies the multigrid cycle
// to all residuals at once (mg_precondition_batch: multi-RHS D_r in the
// smoother, all coarsest-level solves in one persistent launch) and the FP64
// D_r to all new directions in one multi-RHS launch; the Krylov space,
// scalars, convergence test and restart of every right-hand side are its own.
// A right-hand side that has converged stops updating (its slot in the
// multi-RHS launches is carried along).  Vectors are packed half vectors:
// rhs q of a half at base + q * 24 Vh doubles.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mg {

namespace {
struct BlockBuffers {
  int nb = 0, m = 0;
  DBuf be, bo, y, br, r, tmp, xe, xo, te, to;   // FP64, nb half vectors each
  DBuf r32;                                     // FP32, nb half vectors
  std::vector<DBuf> W, Z;                       // W[k] FP64, Z[k] FP32: nb half vectors each
  DBuf scal;                                    // per rhs: beta[2 m m], alpha[2 m], gam[m], c[2 m], orth[4]
  DBuf rn2;                                     // per rhs: ||r||^2 (and a second slot)
  std::unique_ptr<FineOps<double>> F64;
  size_t per_rhs() const { return 2 * (size_t)m * m + 5 * (size_t)m + 8; }
};
}  // namespace

int solve_fine_block(Ctx* c, double* psi_abi, const double* eta_abi, int nb, double tol, mg_solve_info* info) {
  const size_t n = 12 * c->Vh, hs = 24 * c->Vh;   // complex / doubles per half vector
  cudaStream_t s = c->stream;
  const int m = c->params.restart_fine > 0 ? c->params.restart_fine : 16;
  BlockBuffers* Bp = static_cast<BlockBuffers*>(c->block_work.get());
  if (!Bp || Bp->nb < nb || Bp->m != m) {
    c->block_work.reset();
    std::shared_ptr<BlockBuffers> nbuf(new BlockBuffers());
    c->block_work = nbuf;
    Bp = nbuf.get();
    Bp->nb = nb;
    Bp->m = m;
    for (DBuf* d : {&Bp->be, &Bp->bo, &Bp->y, &Bp->br, &Bp->r, &Bp->tmp, &Bp->xe, &Bp->xo, &Bp->te, &Bp->to})
      d->alloc(sizeof(double) * hs * nb);
    Bp->r32.alloc(sizeof(float) * hs * nb);
    Bp->W.resize(m);
    Bp->Z.resize(m);
    for (int k = 0; k < m; k++) {
      Bp->W[k].alloc(sizeof(double) * hs * nb);
      Bp->Z[k].alloc(sizeof(float) * hs * nb);
    }
    Bp->scal.alloc(sizeof(double) * Bp->per_rhs() * nb);
    Bp->rn2.alloc(sizeof(double) * 2 * nb);
    Bp->F64.reset(new FineOps<double>(c));
  }
  BlockBuffers& B = *Bp;
  FineOps<double>& F = *B.F64;
  double* be = B.be.as<double>();
  double* bo = B.bo.as<double>();
  double* y = B.y.as<double>();
  double* br = B.br.as<double>();
  double* r = B.r.as<double>();
  double* tmp = B.tmp.as<double>();
  double* xe = B.xe.as<double>();
  double* xo = B.xo.as<double>();
  double* te = B.te.as<double>();
  double* to = B.to.as<double>();
  float* r32 = B.r32.as<float>();
  double* rn2 = B.rn2.as<double>();
  const size_t ns = B.per_rhs();
  auto beta = [&](int q) { return B.scal.as<double>() + q * ns; };
  auto alpha = [&](int q) { return beta(q) + 2 * (size_t)m * m; };
  auto gam = [&](int q) { return alpha(q) + 2 * m; };
  auto cc = [&](int q) { return gam(q) + m; };
  auto orth = [&](int q) { return cc(q) + 2 * m; };

  for (int q = 0; q < nb; q++) pack_spinor(c->g, eta_abi + (size_t)q * 24 * c->V, be + q * hs, bo + q * hs, false, s);
  std::vector<double> h(2 * (size_t)nb);
  auto read_norms = [&](const double* ve, const double* vo, const std::vector<char>& which) {
    for (int q = 0; q < nb; q++) {
      if (!which[q]) continue;
      blas_norm2<double>(ve + q * hs, n, rn2 + 2 * q, c->ws, s);
      if (vo) blas_norm2<double>(vo + q * hs, n, rn2 + 2 * q + 1, c->ws, s);
    }
    if (!vo)
      for (int q = 0; q < nb; q++)
        if (which[q]) MG_CUDA(cudaMemsetAsync(rn2 + 2 * q + 1, 0, sizeof(double), s));
    MG_CUDA(cudaMemcpyAsync(h.data(), rn2, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s));
    c->sync();
  };
  std::vector<char> all(nb, 1), active(nb, 1), run(nb, 0);
  read_norms(be, bo, all);
  std::vector<double> bnorm(nb), tol_r(nb), true_res(nb, INFINITY);
  for (int q = 0; q < nb; q++) {
    bnorm[q] = std::sqrt(h[2 * q] + h[2 * q + 1]);
    if (!std::isfinite(bnorm[q])) raise(MG_ERR_NAN, "non-finite source");
    tol_r[q] = 0.5 * tol * bnorm[q];
    if (bnorm[q] == 0.0) {
      active[q] = 0;
      true_res[q] = 0.0;
    }
  }
  F.br_multi(br, be, bo, nb, hs);
  blas_zero<double>(y, n * nb, s);
  blas_convert<double, double>(r, br, n * nb, s);
  const int maxit = c->params.maxit_fine > 0 ? c->params.maxit_fine : 500;
  std::vector<int> used(nb, 0);
  int it = 0, restarts = 0;
  auto any = [&](const std::vector<char>& f) {
    for (char v : f)
      if (v) return true;
    return false;
  };
  std::vector<const double*> Wp(m);
  std::vector<const float*> Zp(m);
  for (int attempt = 0; attempt < 8 && any(active) && it < maxit; attempt++) {
    while (any(active) && it < maxit) {
      int k = 0;
      std::vector<int> kp(nb, 0);
      run = active;
      while (k < m && it < maxit && any(run)) {
        float* zk = B.Z[k].as<float>();
        double* wk = B.W[k].as<double>();
        blas_convert<double, float>(r32, r, n * nb, s);
        mg_precondition_batch(c, zk, r32, nb);
        blas_convert<float, double>(tmp, zk, n * nb, s);
        F.Dr_multi(wk, tmp, nb, hs);
        for (int q = 0; q < nb; q++) {
          if (!run[q]) continue;
          for (int j = 0; j < k; j++) Wp[j] = B.W[j].as<double>() + q * hs;
          double* w = wk + q * hs;
          double* bk = beta(q) + 2 * (size_t)m * k;
          if (k > 0) blas_multidot<double>(Wp.data(), k, w, n, bk, c->ws, s);
          blas_orth_update<double>(w, Wp.data(), bk, k, r + q * hs, n, orth(q), c->ws, s);
          blas_r_update<double>(w, r + q * hs, n, orth(q), alpha(q) + 2 * k, gam(q) + k, rn2 + 2 * q, c->ws, s);
        }
        MG_CUDA(cudaMemcpyAsync(h.data(), rn2, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s));
        c->sync();
        k++;
        it++;
        for (int q = 0; q < nb; q++) {
          if (!run[q]) continue;
          kp[q] = k;
          used[q]++;
          const double rn = std::sqrt(h[2 * q]);
          if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite residual in block GCR");
          if (rn <= tol_r[q]) run[q] = 0;
        }
      }
      // per rhs: back substitution and y += sum_j c_j z_j
      for (int q = 0; q < nb; q++) {
        if (!kp[q]) continue;
        for (int j = 0; j < kp[q]; j++) Zp[j] = B.Z[j].as<float>() + q * hs;
        gcr_backsub(beta(q), m, alpha(q), gam(q), kp[q], cc(q), s);
        blas_lincomb<double, float>(y + q * hs, Zp.data(), cc(q), kp[q], 1.0, n, s);
      }
      restarts++;
      // true residuals of the reduced systems
      F.Dr_multi(tmp, y, nb, hs);
      blas_convert<double, double>(r, br, n * nb, s);
      blas_axpby<double>(-1.0, tmp, 1.0, r, n * nb, s);
      read_norms(r, nullptr, active);
      for (int q = 0; q < nb; q++) {
        if (!active[q]) continue;
        const double rn = std::sqrt(h[2 * q]);
        if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite true residual");
        if (rn <= tol_r[q]) active[q] = 0;
      }
    }
    // reconstruction and the true residual of the full system
    F.reconstruct_multi(xe, xo, y, bo, nb, hs);
    F.D_multi(te, to, xe, xo, nb, hs);
    blas_axpby<double>(1.0, be, -1.0, te, n * nb, s);
    blas_axpby<double>(1.0, bo, -1.0, to, n * nb, s);
    std::vector<char> nz(nb);
    for (int q = 0; q < nb; q++) nz[q] = bnorm[q] > 0.0;
    read_norms(te, to, nz);
    for (int q = 0; q < nb; q++) {
      if (!nz[q]) continue;
      true_res[q] = std::sqrt(h[2 * q] + h[2 * q + 1]) / bnorm[q];
      if (!std::isfinite(true_res[q])) raise(MG_ERR_NAN, "non-finite solution");
      active[q] = true_res[q] > tol;
    }
  }
  for (int q = 0; q < nb; q++) {
    if (bnorm[q] == 0.0) {
      MG_CUDA(cudaMemsetAsync(psi_abi + (size_t)q * 24 * c->V, 0, sizeof(double) * 24 * c->V, s));
      continue;
    }
    unpack_spinor(c->g, xe + q * hs, xo + q * hs, false, psi_abi + (size_t)q * 24 * c->V, s);
  }
  c->sync();
  int status = MG_OK;
  if (info) {
    for (int q = 0; q < nb; q++) {
      info->outer_iterations += used[q];
      if (true_res[q] > info->true_residual || info->true_residual != info->true_residual)
        info->true_residual = true_res[q];
    }
    info->restarts += restarts;
  }
  for (int q = 0; q < nb; q++)
    if (!(true_res[q] <= tol)) status = MG_ERR_NOT_CONVERGED;
  return status;
}

}  // namespace mg
