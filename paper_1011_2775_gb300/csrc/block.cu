// Several right-hand sides -- of one lattice, or of several lattices (contexts)
// of uneven size -- solved together.
//
// The outer solver is the same flexible GCR(m) on D_r as solver.cu (section
// "Red-black preconditioning"; section "Implementation"), run for every
// right-hand side in lock-step: every iteration applies the multigrid cycle to
// all residuals of a context at once (multi-RHS D_r in the smoother) and the
// FP64 D_r to all its new directions in one multi-RHS launch, and the
// coarsest-level solves of ALL right-hand sides of all contexts go into one
// persistent launch (coarse_gcr_solve_multi: one coarse lattice per context,
// systems of one lattice sharing link reads).  The Krylov space, scalars,
// convergence test and restarts of every right-hand side are its own; a
// right-hand side that has converged stops updating (its slot in the
// multi-RHS launches is carried along).  Vectors are packed half vectors: rhs
// q of a half at base + q * 24 Vh doubles.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "coarse.h"
#include "internal.h"

namespace mg {

namespace {
struct BlockBuffers {
  int nb = 0, m = 0;
  DBuf be, bo, y, br, r, tmp, xe, xo, te, to;   // FP64, nb half vectors each
  DBuf r32, w32;                                // FP32, nb half vectors
  std::vector<DBuf> W, Z;                       // W[k] FP64, Z[k] FP32: nb half vectors each
  DBuf scal;                                    // per rhs: beta[2 m m], alpha[2 m], gam[m], c[2 m], orth[4]
  DBuf rn2;                                     // per rhs: two norms
  std::unique_ptr<FineOps<double>> F64;
  std::unique_ptr<FineOps<float>> F32;
  size_t per_rhs() const { return 2 * (size_t)m * m + 5 * (size_t)m + 8; }
};

// one context's share of a block solve
struct Run {
  Ctx* c = nullptr;
  int nb = 0;
  const double* eta = nullptr;   // nb ABI vectors (device)
  double* psi = nullptr;
  mg_solve_info* info = nullptr;
  BlockBuffers* B = nullptr;
  size_t n = 0, hs = 0;
  int m = 0, maxit = 0;
  std::vector<double> bnorm, tol_r, true_res, h;
  std::vector<char> active, run;
  std::vector<int> used, kp;
  int restarts = 0;
  double* beta(int q) const { return B->scal.as<double>() + q * B->per_rhs(); }
  double* alpha(int q) const { return beta(q) + 2 * (size_t)m * m; }
  double* gam(int q) const { return alpha(q) + 2 * m; }
  double* cc(int q) const { return gam(q) + m; }
  double* orth(int q) const { return cc(q) + 2 * m; }
};

bool any_of(const std::vector<char>& f) {
  for (char v : f)
    if (v) return true;
  return false;
}

void prepare(Run& R, double tol) {
  Ctx* c = R.c;
  R.n = 12 * c->Vh;
  R.hs = 24 * c->Vh;
  R.m = c->params.restart_fine > 0 ? c->params.restart_fine : 16;
  R.maxit = c->params.maxit_fine > 0 ? c->params.maxit_fine : 500;
  BlockBuffers* Bp = static_cast<BlockBuffers*>(c->block_work.get());
  if (!Bp || Bp->nb < R.nb || Bp->m != R.m) {
    c->block_work.reset();
    std::shared_ptr<BlockBuffers> nbuf(new BlockBuffers());
    c->block_work = nbuf;
    Bp = nbuf.get();
    Bp->nb = R.nb;
    Bp->m = R.m;
    for (DBuf* d : {&Bp->be, &Bp->bo, &Bp->y, &Bp->br, &Bp->r, &Bp->tmp, &Bp->xe, &Bp->xo, &Bp->te, &Bp->to})
      d->alloc(sizeof(double) * R.hs * R.nb);
    Bp->r32.alloc(sizeof(float) * R.hs * R.nb);
    Bp->w32.alloc(sizeof(float) * R.hs * R.nb);
    Bp->W.resize(R.m);
    Bp->Z.resize(R.m);
    for (int k = 0; k < R.m; k++) {
      Bp->W[k].alloc(sizeof(double) * R.hs * R.nb);
      Bp->Z[k].alloc(sizeof(float) * R.hs * R.nb);
    }
    Bp->scal.alloc(sizeof(double) * Bp->per_rhs() * R.nb);
    Bp->rn2.alloc(sizeof(double) * 2 * R.nb);
    Bp->F64.reset(new FineOps<double>(c));
    Bp->F32.reset(new FineOps<float>(c));
  }
  R.B = Bp;
  const int nb = R.nb;
  R.h.assign(2 * (size_t)nb, 0.0);
  R.bnorm.assign(nb, 0.0);
  R.tol_r.assign(nb, 0.0);
  R.true_res.assign(nb, INFINITY);
  R.active.assign(nb, 1);
  R.run.assign(nb, 0);
  R.used.assign(nb, 0);
  R.kp.assign(nb, 0);
  (void)tol;
}

// norms of the nb half vectors ve (+ vo) of the selected rhs -> R.h (one host sync)
void read_norms(Run& R, const double* ve, const double* vo, const std::vector<char>& which) {
  Ctx* c = R.c;
  double* rn2 = R.B->rn2.as<double>();
  for (int q = 0; q < R.nb; q++) {
    if (!which[q]) continue;
    blas_norm2<double>(ve + q * R.hs, R.n, rn2 + 2 * q, c->ws, c->stream);
    if (vo)
      blas_norm2<double>(vo + q * R.hs, R.n, rn2 + 2 * q + 1, c->ws, c->stream);
    else
      MG_CUDA(cudaMemsetAsync(rn2 + 2 * q + 1, 0, sizeof(double), c->stream));
  }
  MG_CUDA(cudaMemcpyAsync(R.h.data(), rn2, sizeof(double) * 2 * R.nb, cudaMemcpyDeviceToHost, c->stream));
  c->sync();
}

// the cycle for every run, with the coarsest solves of the joinable runs in
// shared launches (the others solve their own)
void precondition_all(std::vector<Run*>& runs, int k) {
  std::vector<Run*> joint, own;
  for (Run* R : runs) (mg_batch_joinable(R->c) ? joint : own).push_back(R);
  // runs that can share a launch: same device, coarse storage, restart, cap and even-odd structure
  std::vector<Run*> shared, alone = own;
  for (Run* R : joint) {
    if (shared.empty()) {
      shared.push_back(R);
      continue;
    }
    const mg_params& a = shared[0]->c->params;
    const mg_params& b = R->c->params;
    const bool ok = R->c->device == shared[0]->c->device && a.storage == b.storage &&
                    a.restart_coarse == b.restart_coarse && a.maxit_coarse == b.maxit_coarse;
    (ok ? shared : alone).push_back(R);
  }
  if (shared.size() == 1) {   // one context: its own batched coarse solve (timed against one-by-one solves)
    alone.push_back(shared[0]);
    shared.clear();
  }
  for (Run* R : runs) {
    float* zk = R->B->Z[k].as<float>();
    float* r32 = R->B->r32.as<float>();
    blas_convert<double, float>(r32, R->B->r.as<double>(), R->n * R->nb, R->c->stream);
    mg_batch_pre(R->c, zk, r32, R->nb);
  }
  for (Run* R : alone) mg_batch_coarse(R->c, R->nb);
  if (!shared.empty()) {
    // all systems, in groups the persistent kernel accepts; the first context's stream
    // runs the shared launches after every participant's restriction
    Ctx* c0 = shared[0]->c;
    std::vector<CoarseSystem> sys;
    std::vector<std::vector<CoarseSystem>> launches;
    std::vector<const void*> lattices;
    for (Run* R : shared) {
      std::vector<CoarseSystem> mine;
      mg_batch_systems(R->c, R->nb, mine);
      for (const CoarseSystem& cs : mine) {
        const bool new_lattice = std::find(lattices.begin(), lattices.end(), (const void*)cs.G) == lattices.end();
        if ((int)sys.size() == coarse_gcr_batch_max() ||
            (new_lattice && (int)lattices.size() == coarse_gcr_group_max()) ||
            (!sys.empty() && (cs.G->eo != sys[0].G->eo))) {
          launches.push_back(sys);
          sys.clear();
          lattices.clear();
        }
        if (std::find(lattices.begin(), lattices.end(), (const void*)cs.G) == lattices.end()) lattices.push_back(cs.G);
        sys.push_back(cs);
      }
    }
    if (!sys.empty()) launches.push_back(sys);
    std::vector<cudaEvent_t> ev;
    for (Run* R : shared)
      if (R->c->stream != c0->stream) {
        cudaEvent_t e;
        MG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        MG_CUDA(cudaEventRecord(e, R->c->stream));
        MG_CUDA(cudaStreamWaitEvent(c0->stream, e, 0));
        ev.push_back(e);
      }
    const mg_params& p0 = c0->params;
    const int restart = p0.restart_coarse > 0 ? p0.restart_coarse : 32;
    for (const auto& L : launches) {
      // the systems of one FP16 lattice on tensor cores (mg_params.coarse_impl 0 or 4)
      if ((p0.coarse_impl == 0 || p0.coarse_impl == 4) &&
          coarse_gcr_tc_try(L, mg_batch_buffers(c0), restart, p0.maxit_coarse, c0->ws.flags.as<int>(), c0->stream))
        continue;
      coarse_gcr_solve_multi(L, mg_batch_buffers(c0), restart, p0.maxit_coarse, c0->ws.flags.as<int>(), c0->stream);
    }
    cudaEvent_t done;
    MG_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    MG_CUDA(cudaEventRecord(done, c0->stream));
    for (Run* R : shared)
      if (R->c->stream != c0->stream) MG_CUDA(cudaStreamWaitEvent(R->c->stream, done, 0));
    MG_CUDA(cudaStreamSynchronize(c0->stream));   // the events may be destroyed once the launches ran
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    cudaEventDestroy(done);
  }
  for (Run* R : runs) mg_batch_post(R->c, R->B->Z[k].as<float>(), R->B->r32.as<float>(), R->nb);
}

int solve_runs(std::vector<Run>& runs, double tol) {
  for (Run& R : runs) prepare(R, tol);
  const int m = runs[0].m;
  for (Run& R : runs)
    if (R.m != m) raise(MG_ERR_ARG, "contexts solved together need the same restart_fine");
  // sources, their norms, b_r
  for (Run& R : runs) {
    BlockBuffers& B = *R.B;
    Ctx* c = R.c;
    for (int q = 0; q < R.nb; q++)
      pack_spinor(c->g, R.eta + (size_t)q * 24 * c->V, B.be.as<double>() + q * R.hs, B.bo.as<double>() + q * R.hs,
                  false, c->stream);
    read_norms(R, B.be.as<double>(), B.bo.as<double>(), std::vector<char>(R.nb, 1));
    for (int q = 0; q < R.nb; q++) {
      R.bnorm[q] = std::sqrt(R.h[2 * q] + R.h[2 * q + 1]);
      if (!std::isfinite(R.bnorm[q])) raise(MG_ERR_NAN, "non-finite source");
      R.tol_r[q] = 0.5 * tol * R.bnorm[q];
      if (R.bnorm[q] == 0.0) {
        R.active[q] = 0;
        R.true_res[q] = 0.0;
      }
    }
    B.F64->br_multi(B.br.as<double>(), B.be.as<double>(), B.bo.as<double>(), R.nb, R.hs);
    blas_zero<double>(B.y.as<double>(), R.n * R.nb, c->stream);
    blas_convert<double, double>(B.r.as<double>(), B.br.as<double>(), R.n * R.nb, c->stream);
  }
  auto any_active = [&]() {
    for (Run& R : runs)
      if (any_of(R.active)) return true;
    return false;
  };
  auto any_running = [&]() {
    for (Run& R : runs)
      if (any_of(R.run)) return true;
    return false;
  };
  int it = 0;
  int maxit = 0;
  for (Run& R : runs) maxit = std::max(maxit, R.maxit);
  std::vector<const double*> Wp(m);
  std::vector<const float*> Zp(m);
  for (int attempt = 0; attempt < 8 && any_active() && it < maxit; attempt++) {
    while (any_active() && it < maxit) {
      int k = 0;
      for (Run& R : runs) {
        std::fill(R.kp.begin(), R.kp.end(), 0);
        R.run = R.active;
        if (it >= R.maxit) std::fill(R.run.begin(), R.run.end(), 0);
      }
      while (k < m && it < maxit && any_running()) {
        // contexts whose right-hand sides have all stopped drop out of the iteration
        std::vector<Run*> live;
        for (Run& R : runs)
          if (any_of(R.run)) live.push_back(&R);
        precondition_all(live, k);
        for (Run* Rp : live) {
          Run& R = *Rp;
          BlockBuffers& B = *R.B;
          Ctx* c = R.c;
          double* wk = B.W[k].as<double>();
          double* tmp = B.tmp.as<double>();
          double* r = B.r.as<double>();
          if (c->params.outer_prec == MG_FP32) {   // the directions' product in FP32, true residuals FP64
            B.F32->Dr_multi(B.w32.as<float>(), B.Z[k].as<float>(), R.nb, R.hs);
            blas_convert<float, double>(wk, B.w32.as<float>(), R.n * R.nb, c->stream);
          } else {
            blas_convert<float, double>(tmp, B.Z[k].as<float>(), R.n * R.nb, c->stream);
            B.F64->Dr_multi(wk, tmp, R.nb, R.hs);
          }
          for (int q = 0; q < R.nb; q++) {
            if (!R.run[q]) continue;
            for (int j = 0; j < k; j++) Wp[j] = B.W[j].as<double>() + q * R.hs;
            double* w = wk + q * R.hs;
            double* bk = R.beta(q) + 2 * (size_t)m * k;
            if (k > 0) blas_multidot<double>(Wp.data(), k, w, R.n, bk, c->ws, c->stream);
            blas_orth_update<double>(w, Wp.data(), bk, k, r + q * R.hs, R.n, R.orth(q), c->ws, c->stream);
            blas_r_update<double>(w, r + q * R.hs, R.n, R.orth(q), R.alpha(q) + 2 * k, R.gam(q) + k,
                                  B.rn2.as<double>() + 2 * q, c->ws, c->stream);
          }
        }
        for (Run* Rp : live) {
          Run& R = *Rp;
          MG_CUDA(cudaMemcpyAsync(R.h.data(), R.B->rn2.as<double>(), sizeof(double) * 2 * R.nb,
                                  cudaMemcpyDeviceToHost, R.c->stream));
          R.c->sync();
          for (int q = 0; q < R.nb; q++) {
            if (!R.run[q]) continue;
            R.kp[q] = k + 1;
            R.used[q]++;
            const double rn = std::sqrt(R.h[2 * q]);
            if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite residual in block GCR");
            if (rn <= R.tol_r[q] || it + 1 >= R.maxit) R.run[q] = 0;
          }
        }
        k++;
        it++;
      }
      for (Run& R : runs) {
        if (!any_of(R.active)) continue;   // nothing changed since its last check
        BlockBuffers& B = *R.B;
        Ctx* c = R.c;
        double* y = B.y.as<double>();
        for (int q = 0; q < R.nb; q++) {
          if (!R.kp[q]) continue;
          for (int j = 0; j < R.kp[q]; j++) Zp[j] = B.Z[j].as<float>() + q * R.hs;
          gcr_backsub(R.beta(q), m, R.alpha(q), R.gam(q), R.kp[q], R.cc(q), c->stream);
          blas_lincomb<double, float>(y + q * R.hs, Zp.data(), R.cc(q), R.kp[q], 1.0, R.n, c->stream);
        }
        R.restarts++;
        // true residuals of the reduced systems
        double* tmp = B.tmp.as<double>();
        double* r = B.r.as<double>();
        B.F64->Dr_multi(tmp, y, R.nb, R.hs);
        blas_convert<double, double>(r, B.br.as<double>(), R.n * R.nb, c->stream);
        blas_axpby<double>(-1.0, tmp, 1.0, r, R.n * R.nb, c->stream);
        read_norms(R, r, nullptr, R.active);
        for (int q = 0; q < R.nb; q++) {
          if (!R.active[q]) continue;
          const double rn = std::sqrt(R.h[2 * q]);
          if (!std::isfinite(rn)) raise(MG_ERR_NAN, "non-finite true residual");
          if (rn <= R.tol_r[q] || it >= R.maxit) R.active[q] = 0;
        }
      }
    }
    // reconstruction and the true residual of the full systems
    for (Run& R : runs) {
      BlockBuffers& B = *R.B;
      double *xe = B.xe.as<double>(), *xo = B.xo.as<double>(), *te = B.te.as<double>(), *to = B.to.as<double>();
      B.F64->reconstruct_multi(xe, xo, B.y.as<double>(), B.bo.as<double>(), R.nb, R.hs);
      B.F64->D_multi(te, to, xe, xo, R.nb, R.hs);
      blas_axpby<double>(1.0, B.be.as<double>(), -1.0, te, R.n * R.nb, R.c->stream);
      blas_axpby<double>(1.0, B.bo.as<double>(), -1.0, to, R.n * R.nb, R.c->stream);
      std::vector<char> nz(R.nb);
      for (int q = 0; q < R.nb; q++) nz[q] = R.bnorm[q] > 0.0;
      read_norms(R, te, to, nz);
      for (int q = 0; q < R.nb; q++) {
        if (!nz[q]) continue;
        R.true_res[q] = std::sqrt(R.h[2 * q] + R.h[2 * q + 1]) / R.bnorm[q];
        if (!std::isfinite(R.true_res[q])) raise(MG_ERR_NAN, "non-finite solution");
        R.active[q] = R.true_res[q] > tol && it < R.maxit;
      }
    }
  }
  int status = MG_OK;
  for (Run& R : runs) {
    BlockBuffers& B = *R.B;
    Ctx* c = R.c;
    for (int q = 0; q < R.nb; q++) {
      double* dst = R.psi + (size_t)q * 24 * c->V;
      if (R.bnorm[q] == 0.0) {
        MG_CUDA(cudaMemsetAsync(dst, 0, sizeof(double) * 24 * c->V, c->stream));
        continue;
      }
      unpack_spinor(c->g, B.xe.as<double>() + q * R.hs, B.xo.as<double>() + q * R.hs, false, dst, c->stream);
    }
    c->sync();
    if (R.info) {
      for (int q = 0; q < R.nb; q++) {
        R.info->outer_iterations += R.used[q];
        if (R.true_res[q] > R.info->true_residual || R.info->true_residual != R.info->true_residual)
          R.info->true_residual = R.true_res[q];
      }
      R.info->restarts += R.restarts;
    }
    for (int q = 0; q < R.nb; q++)
      if (!(R.true_res[q] <= tol)) status = MG_ERR_NOT_CONVERGED;
  }
  return status;
}
}  // namespace

int solve_fine_block(Ctx* c, double* psi_abi, const double* eta_abi, int nb, double tol, mg_solve_info* info) {
  std::vector<Run> runs(1);
  runs[0].c = c;
  runs[0].nb = nb;
  runs[0].eta = eta_abi;
  runs[0].psi = psi_abi;
  runs[0].info = info;
  return solve_runs(runs, tol);
}

int solve_multi_block(const std::vector<BlockPart>& parts, double tol) {
  std::vector<Run> runs(parts.size());
  for (size_t i = 0; i < parts.size(); i++) {
    runs[i].c = parts[i].c;
    runs[i].nb = parts[i].nb;
    runs[i].eta = parts[i].eta;
    runs[i].psi = parts[i].psi;
    runs[i].info = parts[i].info;
  }
  return solve_runs(runs, tol);
}

}  // namespace mg
