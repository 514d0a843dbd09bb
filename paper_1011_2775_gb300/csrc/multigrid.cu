// Host driver of the adaptive multigrid preconditioner.
//
// Setup (section "Setup procedure"): for every transfer l, Nv near-null
// vectors of level l's D_p by inverse iteration -- repeated GCR relaxations
// on a random (Philox) vector, kept globally orthogonal to the vectors
// already found, stopped when the Rayleigh quotient ||D_p v||^2 settles --
// then the chirality split and block Gram-Schmidt into P_l, the Galerkin
// coarse links R D_p P and their site inverses.
//
// Solve (section "Implementation"): the truly adaptive recursive cycle.  The
// level-l cycle restricts (r_e, 0), solves the next level's reduced
// even-odd system with GCR to a relative residual tol_coarse -- itself
// preconditioned by the next cycle, down to an unpreconditioned GCR on the
// coarsest lattice (without even-odd if an extent is odd) -- prolongs, keeps
// the even part and post-smooths with minimal-residual steps on D_r.  For
// D_p = [[1, X], [Y, 1]] the solution of D_p u = (r_e, 0) has
// u_e = D_r^{-1} r_e, which is why a coarse space of D_p serves D_r.
// The whole preconditioner runs in FP32.
#include <chrono>
#include <cmath>

#include "coarse.h"

namespace mg {

// --------------------------------------------------------------------------- geometry
void LevelGeom::init(const int dims[4], int ndof_, bool wilson_) {
  nsites = 1;
  eo = true;
  for (int m = 0; m < 4; m++) {
    L[m] = dims[m];
    nsites *= dims[m];
    if (dims[m] % 2) eo = false;
  }
  ndof = ndof_;
  wilson = wilson_;
  half = eo ? nsites / 2 : 0;
  Vh = nsites / 2;
  lex_of.assign(nsites, 0);
  store_of.assign(nsites, 0);
  for (int lex = 0; lex < nsites; lex++) {
    int c[4], r = lex;
    for (int m = 0; m < 4; m++) {
      c[m] = r % L[m];
      r /= L[m];
    }
    const int s = coord_to_store(c);
    store_of[lex] = s;
    lex_of[s] = lex;
  }
  if (!wilson) {
    std::vector<int> nbr((size_t)nsites * 8);
    for (int s = 0; s < nsites; s++) {
      int c[4], r = lex_of[s];
      for (int m = 0; m < 4; m++) {
        c[m] = r % L[m];
        r /= L[m];
      }
      for (int d = 0; d < 8; d++) {
        int n[4] = {c[0], c[1], c[2], c[3]};
        const int mu = d & 3;
        n[mu] = (c[mu] + (d < 4 ? 1 : -1) + L[mu]) % L[mu];
        nbr[(size_t)s * 8 + d] = coord_to_store(n);
      }
    }
    d_nbr.alloc(sizeof(int) * nbr.size());
    MG_CUDA(cudaMemcpy(d_nbr.get(), nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice));
    d_lex_of.alloc(sizeof(int) * nsites);
    MG_CUDA(cudaMemcpy(d_lex_of.get(), lex_of.data(), sizeof(int) * nsites, cudaMemcpyHostToDevice));
  }
}

int LevelGeom::coord_to_store(const int c[4]) const {
  const int lex = c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
  if (wilson || eo) {
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    return par * (nsites / 2) + lex / 2;
  }
  return lex;
}

// --------------------------------------------------------------------------- hierarchy
struct LevelWork {
  DBuf tA, tB;             // coarse: full-vector temporaries of the even-odd operators
  DBuf br, y;              // coarse: reduced rhs / solution
  std::unique_ptr<GCR<float, float>> gcr;
  CoarseGCRBuffers cg;     // coarsest level: buffers of the persistent solver
  DBuf rc, ec;             // next level's rhs / solution (this level's cycle)
  DBuf res, w, e, z0;      // this level's half vectors for smoothing
  int coarse_impl = -1;    // coarsest level: persistent solver chosen by the autotuner (-1: not yet)
  DBuf tune_iters;         // iteration counter of the tuning runs
  // coarsest level of a batched cycle of nb systems: 0 the batched launches,
  // 1 one single-system solve after another (-1: not yet timed)
  int batch_impl[17] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
};

// level-0 temporaries of the batched cycle (allocated for up to `cap` rhs)
struct BatchWork {
  int cap = 0;
  DBuf rc, ec, res, w, e, z0, scr;
};

// The 2-level cycle of level 0 as a captured CUDA graph (see mg_precondition_graph)
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;   // private stream the capture runs on
  const double* r = nullptr;    // the input the graph was captured for
  float* r32 = nullptr;
  bool failed = false;
  long long dslash = 0, kernels = 0;   // launches one replay executes (for the statistics)
  DBuf zc;                      // the graph's output
  // the captured cycle bakes in the smoothing steps, coarse tolerance and caps:
  // drop it when they change so that the next solve captures it afresh
  void drop() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    r = nullptr;
    r32 = nullptr;
    failed = false;
  }
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
  }
};

struct Hierarchy {
  BatchWork bw;
  CycleGraph graph;
  int L = 0;
  std::vector<LevelGeom> geo;
  std::vector<CoarseOp> cop;
  std::vector<TransferOp> tr;
  std::vector<DBuf> nullvecs;
  std::vector<LevelWork> work;
  std::unique_ptr<FineOps<float>> F32;
  std::vector<long long> iters;
  DBuf d_iters;            // long long[MG_MAX_LEVELS]: iterations counted on the device
  DBuf gs_scratch;
};

namespace {

size_t half_n(const Hierarchy& H, int l) {
  const LevelGeom& G = H.geo[l];
  return (size_t)(l == 0 ? G.Vh : G.half) * G.ndof;
}
size_t full_n(const Hierarchy& H, int l) { return H.geo[l].vec_complex(); }

// ----- level operators (FP32); vectors are full-vector base pointers, even sites first
void Dr_level(Ctx* c, Hierarchy& H, int l, float* out, const float* in) {
  if (l == 0) {
    H.F32->Dr(out, in);
    return;
  }
  const LevelGeom& G = H.geo[l];
  const CoarseOp& C = H.cop[l];
  LevelWork& W = H.work[l];
  float* tA = W.tA.as<float>();
  float* tB = W.tB.as<float>();
  coarse_site_mul(G, C, true, 0, G.half, tA, in, c->stream);                                    // X_e^{-1} y_e
  coarse_hop(G, C, EPI_CH, true, G.half, G.nsites, tB, tA, nullptr, 0.f, 0xff, c->stream);      // X_o^{-1} Y_oe .
  coarse_hop(G, C, EPI_XPAY, false, 0, G.half, out, tB, in, -1.f, 0xff, c->stream);            // y_e - Y_eo .
}

void br_level(Ctx* c, Hierarchy& H, int l, float* br, const float* b) {
  const LevelGeom& G = H.geo[l];
  const CoarseOp& C = H.cop[l];
  float* tB = H.work[l].tB.as<float>();
  coarse_site_mul(G, C, true, G.half, G.nsites, tB, b, c->stream);
  coarse_hop(G, C, EPI_XPAY, false, 0, G.half, br, tB, b, -1.f, 0xff, c->stream);
}

void recon_level(Ctx* c, Hierarchy& H, int l, float* x, const float* y, const float* b) {
  const LevelGeom& G = H.geo[l];
  const CoarseOp& C = H.cop[l];
  coarse_site_mul(G, C, true, 0, G.half, x, y, c->stream);
  coarse_hop(G, C, EPI_C_XPAY, true, G.half, G.nsites, x, x, b, -1.f, 0xff, c->stream);
}

void Dfull_level(Ctx* c, Hierarchy& H, int l, float* out, const float* in) {
  if (l == 0) {
    H.F32->D(out, out + 24 * c->Vh, in, in + 24 * c->Vh);
    return;
  }
  const LevelGeom& G = H.geo[l];
  coarse_hop(G, H.cop[l], EPI_CX_PAY, false, 0, G.nsites, out, in, in, 1.f, 0xff, c->stream);
}

void Dp_level(Ctx* c, Hierarchy& H, int l, float* out, const float* in) {
  if (l == 0) {
    H.F32->Dp(out, out + 24 * c->Vh, in, in + 24 * c->Vh);
    return;
  }
  const LevelGeom& G = H.geo[l];
  float* tA = H.work[l].tA.as<float>();
  coarse_site_mul(G, H.cop[l], true, 0, G.nsites, tA, in, c->stream);
  coarse_hop(G, H.cop[l], EPI_XPAY, false, 0, G.nsites, out, tA, in, 1.f, 0xff, c->stream);
}

void Minv_level(Ctx* c, Hierarchy& H, int l, float* out, const float* in, bool inverse) {
  if (l == 0) {
    H.F32->M(out, out + 24 * c->Vh, in, in + 24 * c->Vh, inverse);
    return;
  }
  const LevelGeom& G = H.geo[l];
  coarse_site_mul(G, H.cop[l], inverse, 0, G.nsites, out, in, c->stream);
}

void coarse_solve(Ctx* c, Hierarchy& H, int l, float* x, const float* b);

// ----- the cycle: z_e ~ D_r^{-1} r_e on level l
void cycle(Ctx* c, Hierarchy& H, int l, float* z, const float* r) {
  Range range(level_range_name(RANGE_CYCLE, l));
  LevelTime timer(c, l == 0 ? 0 : -1);
  const mg_params& p = c->params;
  LevelWork& W = H.work[l];
  const TransferOp& T = H.tr[l];
  const size_t n = half_n(H, l);
  cudaStream_t s = c->stream;
  double* scr = c->ws.scalars.as<double>() + 64 + 8 * l;
  auto Dr = [&](float* o, const float* i) { Dr_level(c, H, l, o, i); };
  float* res = W.res.as<float>();
  float* w = W.w.as<float>();
  float* e = W.e.as<float>();
  const float* rin = r;
  if (p.nu_pre > 0) {
    blas_convert<float, float>(res, r, n, s);
    mr_smooth<float>(c, Dr, z, res, w, n, p.nu_pre, scr);  // z = MR(r)
    Dr(w, z);
    blas_convert<float, float>(res, r, n, s);
    blas_axpby<float>(-1.0, w, 1.0, res, n, s);
    rin = res;
  }
  restrict_vec(T, W.rc.as<float>(), rin, true, s);
  coarse_solve(c, H, l + 1, W.ec.as<float>(), W.rc.as<float>());
  if (p.nu_pre > 0) {
    float* z0 = W.z0.as<float>();
    prolong_vec(T, z0, W.ec.as<float>(), true, s);
    blas_axpby<float>(1.0, z0, 1.0, z, n, s);
  } else {
    prolong_vec(T, z, W.ec.as<float>(), true, s);
  }
  if (p.nu_post > 0) {
    Dr(w, z);
    blas_convert<float, float>(res, r, n, s);
    blas_axpby<float>(-1.0, w, 1.0, res, n, s);
    if (l == 0)   // fused fine-level steps (three kernels per step)
      mr_smooth_fine(c, e, res, w, H.F32->t1.as<float>(), H.F32->t2.as<float>(), p.nu_post, scr);
    else
      mr_smooth<float>(c, Dr, e, res, w, n, p.nu_post, scr);
    blas_axpby<float>(1.0, e, 1.0, z, n, s);
  }
}

void coarse_solve(Ctx* c, Hierarchy& H, int l, float* x, const float* b) {
  Range range(level_range_name(RANGE_COARSE_SOLVE, l));
  LevelTime timer(c, l);
  const mg_params& p = c->params;
  const LevelGeom& G = H.geo[l];
  LevelWork& W = H.work[l];
  cudaStream_t s = c->stream;
  if (l + 1 == H.L) {
    // coarsest level: one persistent kernel, no host round trip.  Two
    // implementations of the same GCR: the single-system kernel (on the full
    // grid, or on a smaller one whose grid barriers have fewer blocks), and the
    // batched kernel with one system (row-blocked GEMV: fewer registers, more
    // co-resident CTAs).  The autotuner times them on the first solve of this
    // lattice (the tuning runs do not count towards the iteration statistics).
    // The streamed kernel (links through shared memory by bulk copies, even-odd
    // levels) is a third implementation, on the full grid or on the largest
    // grid that splits its work evenly; candidates 100 + k.
    const int restart = p.restart_coarse > 0 ? p.restart_coarse : 32;
    long long* d_it = H.d_iters.as<long long>() + l;
    const std::vector<int> smaller = coarse_gcr_smaller_grids(G, W.cg);
    const std::vector<int> streamed =
        coarse_gcr_stream_ok(G, H.cop[l]) ? coarse_gcr_stream_grids(G, H.cop[l]) : std::vector<int>();
    const std::vector<int> tensor =
        coarse_gcr_tc_ok(G, H.cop[l], 1) ? coarse_gcr_tc_grids(G, H.cop[l], 1) : std::vector<int>();
    auto run = [&](int which, long long* it) {
      if (which >= 200) {
        const double tol = p.tol_coarse;
        const size_t nf = G.vec_complex();
        coarse_gcr_tc_solve(G, H.cop[l], W.cg, restart, p.maxit_coarse, &tol, 1, b, nf, x, nf, it,
                            c->ws.flags.as<int>(), s, tensor[which - 200]);
      } else if (which >= 100)
        coarse_gcr_stream_solve(G, H.cop[l], W.cg, restart, p.maxit_coarse, p.tol_coarse, b, x, it,
                                c->ws.flags.as<int>(), s, streamed[which - 100]);
      else if (which == 1)
        coarse_gcr_solve_batch(G, H.cop[l], W.cg, restart, p.maxit_coarse, p.tol_coarse, 1, b, x, it,
                               c->ws.flags.as<int>(), s);
      else
        coarse_gcr_solve(G, H.cop[l], W.cg, restart, p.maxit_coarse, p.tol_coarse, b, x, it, c->ws.flags.as<int>(), s,
                         which >= 2 ? smaller[which - 2] : 0);
    };
    if (W.coarse_impl < 0) {
      if (!W.tune_iters.get()) W.tune_iters.alloc(sizeof(long long));
      TuneKey key{"coarse_gcr3", {G.L[0], G.L[1], G.L[2], G.L[3]}, H.cop[l].nc, H.cop[l].store};
      std::vector<int> cands = {0, 1};
      for (size_t k = 0; k < smaller.size(); k++) cands.push_back(2 + (int)k);
      for (size_t k = 0; k < streamed.size(); k++) cands.push_back(100 + (int)k);
      const int forced = c->params.coarse_impl;
      // one system on tensor cores uses one column of eight of every MMA and
      // pays two site-inverse passes per iteration: measured slower than the
      // streamed kernel on GB300, so it runs only when forced
      if (forced == 4)
        for (size_t k = 0; k < tensor.size(); k++) cands.push_back(200 + (int)k);
      if (forced > 0) {
        // a forced implementation (mg_params.coarse_impl): 1 original, 2 batched,
        // 3 streamed, 4 tensor cores; the grid is still chosen by timing
        std::vector<int> f;
        for (int cnd : cands)
          if ((forced == 1 && (cnd == 0 || (cnd >= 2 && cnd < 100))) || (forced == 2 && cnd == 1) ||
              (forced == 3 && cnd >= 100 && cnd < 200) || (forced == 4 && cnd >= 200))
            f.push_back(cnd);
        if (f.empty()) f.push_back(0);
        W.coarse_impl = f.size() == 1 ? f[0]
                                      : tuned_block(TuneKey{forced == 3 ? "coarse_gcr_stream" : forced == 4 ? "coarse_gcr_tc"
                                                                                                            : "coarse_gcr_single",
                                                            {G.L[0], G.L[1], G.L[2], G.L[3]}, H.cop[l].nc, H.cop[l].store},
                                                    f, [&](int which) { run(which, W.tune_iters.as<long long>()); }, s);
      } else {
        W.coarse_impl = tuned_block(key, cands, [&](int which) { run(which, W.tune_iters.as<long long>()); }, s);
      }
      const bool valid = (W.coarse_impl >= 0 && W.coarse_impl < 2 + (int)smaller.size()) ||
                         (W.coarse_impl >= 100 && W.coarse_impl < 100 + (int)streamed.size()) ||
                         (W.coarse_impl >= 200 && W.coarse_impl < 200 + (int)tensor.size());
      if (!valid) W.coarse_impl = 0;  // a cached choice from other grids
    }
    run(W.coarse_impl, d_it);
    return;
  }
  double* scr = c->ws.scalars.as<double>() + 32 + l;
  blas_norm2<float>(b, full_n(H, l), scr, c->ws, s);
  const double bn = std::sqrt(c->read_scalar(scr));
  if (bn == 0.0) {
    blas_zero<float>(x, full_n(H, l), s);
    return;
  }
  const double tol = p.tol_coarse * bn;
  const bool has_next = l + 1 < H.L;
  if (G.eo) {
    float* br = W.br.as<float>();
    float* y = W.y.as<float>();
    br_level(c, H, l, br, b);
    auto A = [&](float* o, const float* i) { Dr_level(c, H, l, o, i); };
    GCR<float, float>::Pre pre = [&](float* z, const float* r) { cycle(c, H, l, z, r); };
    auto res = W.gcr->solve(A, has_next ? &pre : nullptr, y, br, true, tol, p.maxit_coarse, true);
    H.iters[l] += res.iterations;
    recon_level(c, H, l, x, y, b);
  } else {
    auto A = [&](float* o, const float* i) { Dfull_level(c, H, l, o, i); };
    auto res = W.gcr->solve(A, nullptr, x, b, true, tol, p.maxit_coarse, true);
    H.iters[l] += res.iterations;
  }
}

// ----- setup
void fill_start_vector(Ctx* c, Hierarchy& H, int l, int k, float* v) {
  const uint64_t seed = c->params.seed;
  if (l == 0)
    philox_fine_vector(c->g, seed, l, k, v, v + 24 * c->Vh, c->stream);
  else
    philox_coarse_vector(H.geo[l], seed, l, k, v, c->stream);
}

void find_null_vectors(Ctx* c, Hierarchy& H, int l, mg_setup_info* info) {
  Range range(level_range_name(RANGE_NULL_VECTORS, l));
  const mg_params& p = c->params;
  const int nv = p.nv[l];
  const size_t n = full_n(H, l);
  cudaStream_t s = c->stream;
  float* base = H.nullvecs[l].as<float>();
  std::vector<const float*> found(nv);
  for (int k = 0; k < nv; k++) found[k] = base + (size_t)k * 2 * n;
  if (l < (int)c->injected.size() && !c->injected[l].empty()) {
    DBuf stage(sizeof(double) * 2 * n);
    for (int k = 0; k < nv; k++) {
      MG_CUDA(cudaMemcpyAsync(stage.get(), c->injected[l].data() + (size_t)k * 2 * n, sizeof(double) * 2 * n,
                              cudaMemcpyHostToDevice, s));
      float* v = base + (size_t)k * 2 * n;
      if (l == 0)
        pack_spinor(c->g, stage.as<double>(), v, v + 24 * c->Vh, true, s);
      else
        pack_coarse(H.geo[l], stage.as<double>(), v, s);
    }
    c->sync();
    if (info) info->vectors[l] = nv;
    return;
  }
  const int inner = p.setup_inner > 0 ? p.setup_inner : 8;
  GCR<float, float> gcr(c, n, inner);
  DBuf vb(sizeof(float) * 2 * n), wb(sizeof(float) * 2 * n);
  float* v = vb.as<float>();
  float* w = wb.as<float>();
  double* scr = c->ws.scalars.as<double>() + 256;
  auto Dp = [&](float* o, const float* i) { Dp_level(c, H, l, o, i); };
  int passes = 0;
  double rq = 0;
  for (int k = 0; k < nv; k++) {
    float* x = base + (size_t)k * 2 * n;
    fill_start_vector(c, H, l, k, v);
    double rq_prev = -1;
    for (int it = 0; it < p.setup_iters; it++) {
      gcr.solve(Dp, nullptr, x, v, true, 0.0, inner, false);
      for (int rep = 0; rep < 2 && k > 0; rep++) {
        blas_multidot<float>(found.data(), k, x, n, scr, c->ws, s);
        blas_lincomb<float, float>(x, found.data(), scr, k, -1.0, n, s);
      }
      blas_norm2<float>(x, n, scr + 200, c->ws, s);
      blas_normalize<float>(x, scr + 200, n, s);
      Dp(w, x);
      blas_norm2<float>(w, n, scr + 201, c->ws, s);
      rq = c->read_scalar(scr + 201);
      if (!std::isfinite(rq)) raise(MG_ERR_NAN, "non-finite Rayleigh quotient in setup");
      passes++;
      blas_convert<float, float>(v, x, n, s);
      if (rq_prev >= 0 && std::fabs(rq - rq_prev) < p.setup_rq_tol * rq) break;
      rq_prev = rq;
    }
  }
  if (info) {
    info->vectors[l] = nv;
    info->passes[l] = passes;
    info->rq_last[l] = rq;
  }
}

void build_coarse_links(Ctx* c, Hierarchy& H, int l) {
  Range range(level_range_name(RANGE_COARSE_LINKS, l));
  const mg_params& p = c->params;
  TransferOp& T = H.tr[l];
  CoarseOp& C = H.cop[l + 1];
  const LevelGeom& Gc = H.geo[l + 1];
  const int nv = T.nv, nc = 2 * nv;
  const size_t n = full_n(H, l);
  cudaStream_t s = c->stream;
  C.nc = nc;
  C.store = STORE_F32;
  C.Y.alloc(sizeof(float2) * (size_t)Gc.nsites * nc * 8 * nc);
  C.X.alloc(sizeof(float2) * (size_t)Gc.nsites * nc * nc);
  C.Xinv.alloc(sizeof(float2) * (size_t)Gc.nsites * nc * nc);
  C.Yscale.alloc(sizeof(float) * (size_t)Gc.nsites * 8);
  {
    std::vector<float> ones((size_t)Gc.nsites * 8, 1.f);
    MG_CUDA(cudaMemcpyAsync(C.Yscale.get(), ones.data(), sizeof(float) * ones.size(), cudaMemcpyHostToDevice, s));
    c->sync();
  }
  DBuf pb(sizeof(float) * 2 * n), ub(sizeof(float) * 2 * n), mb(sizeof(float) * 2 * n);
  std::vector<DBuf> Wb(8);
  for (auto& b : Wb) b.alloc(sizeof(float) * 2 * n);
  float* pv = pb.as<float>();
  float* u = ub.as<float>();
  float* mp = mb.as<float>();
  float* Wp[8];
  for (int d = 0; d < 8; d++) Wp[d] = Wb[d].as<float>();
  const bool galerkin_dp = p.coarse_op != MG_COARSE_D;
  for (int ch = 0; ch < 2; ch++)
    for (int k = 0; k < nv; k++) {
      extract_column(T, pv, ch, k, s);
      const float* slot8 = pv;
      const float* hop_in = pv;
      if (galerkin_dp) {
        Minv_level(c, H, l, u, pv, true);
        hop_in = u;
      } else {
        Minv_level(c, H, l, mp, pv, false);
        slot8 = mp;
      }
      if (l == 0) {
        hop_directions(c->g, Wp, hop_in, hop_in + 24 * c->Vh, c->gauge<float>(), s);
      } else {
        const LevelGeom& G = H.geo[l];
        for (int d = 0; d < 8; d++)
          coarse_hop(G, H.cop[l], EPI_H, false, 0, G.nsites, Wp[d], hop_in, nullptr, 0.f, 1 << d, s);
      }
      const float* W9[9] = {Wp[0], Wp[1], Wp[2], Wp[3], Wp[4], Wp[5], Wp[6], Wp[7], slot8};
      restrict9(T, C, W9, ch * nv + k, s);
    }
  coarse_invert(Gc, C, c->ws.flags.as<int>(), s);
  if (c->read_flag(FLAG_SINGULAR, true)) raise(MG_ERR_SINGULAR_CLOVER, "singular coarse diagonal block");
  quantize_links(Gc, C, T.store, s);               // 16-bit storage of Y (FP32: no-op)
  if (l + 2 == H.L) coarse_fold_links(Gc, C, s);  // the coarsest level runs the persistent solver
}

void alloc_work(Ctx* c, Hierarchy& H) {
  const mg_params& p = c->params;
  for (int l = 0; l < H.L; l++) {
    LevelWork& W = H.work[l];
    const size_t nh = half_n(H, l), nf = full_n(H, l);
    if (l >= 1) {
      W.tA.alloc(sizeof(float) * 2 * nf);
      W.tB.alloc(sizeof(float) * 2 * nf);
      MG_CUDA(cudaMemset(W.tA.get(), 0, sizeof(float) * 2 * nf));
      MG_CUDA(cudaMemset(W.tB.get(), 0, sizeof(float) * 2 * nf));
      const int restart = p.restart_coarse > 0 ? p.restart_coarse : 32;
      if (H.geo[l].eo) {
        W.br.alloc(sizeof(float) * 2 * nh);
        W.y.alloc(sizeof(float) * 2 * nh);
        W.gcr.reset(new GCR<float, float>(c, nh, restart));
      } else {
        W.gcr.reset(new GCR<float, float>(c, nf, restart));
      }
      if (l + 1 == H.L) W.cg.init(H.geo[l], H.geo[l].ndof, restart);
    }
    if (l + 1 < H.L) {
      const size_t nfc = full_n(H, l + 1);
      W.rc.alloc(sizeof(float) * 2 * nfc);
      W.ec.alloc(sizeof(float) * 2 * nfc);
      const size_t vec = l == 0 ? 2 * nh : 2 * nf;  // fine: half vectors; coarse: full-vector base
      W.res.alloc(sizeof(float) * vec);
      W.w.alloc(sizeof(float) * vec);
      W.e.alloc(sizeof(float) * vec);
      W.z0.alloc(sizeof(float) * vec);
      MG_CUDA(cudaMemset(W.res.get(), 0, sizeof(float) * vec));
      MG_CUDA(cudaMemset(W.w.get(), 0, sizeof(float) * vec));
      MG_CUDA(cudaMemset(W.e.get(), 0, sizeof(float) * vec));
      MG_CUDA(cudaMemset(W.z0.get(), 0, sizeof(float) * vec));
    }
  }
}

}  // namespace

// --------------------------------------------------------------------------- entry points
void mg_destroy_hierarchy(Ctx* c) { c->mg.reset(); }

void mg_build(Ctx* c, mg_setup_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  const mg_params& p = c->params;
  c->mg.reset();
  std::unique_ptr<Hierarchy> H(new Hierarchy());
  H->L = p.levels;
  H->geo.resize(p.levels);
  H->cop.resize(p.levels);
  H->tr.resize(p.levels > 1 ? p.levels - 1 : 0);
  H->nullvecs.resize(p.levels > 1 ? p.levels - 1 : 0);
  H->work.resize(p.levels);
  H->iters.assign(p.levels, 0);
  H->d_iters.alloc(sizeof(long long) * MG_MAX_LEVELS);
  MG_CUDA(cudaMemset(H->d_iters.get(), 0, sizeof(long long) * MG_MAX_LEVELS));
  H->F32.reset(new FineOps<float>(c));
  H->geo[0].init(c->dims, 12, true);
  for (int l = 0; l + 1 < p.levels; l++) {
    int cd[4];
    for (int m = 0; m < 4; m++) cd[m] = H->geo[l].L[m] / p.block[l][m];
    H->geo[l + 1].init(cd, 2 * p.nv[l], false);
  }
  alloc_work(c, *H);
  for (int l = 0; l + 1 < p.levels; l++) {
    const LevelGeom& G = H->geo[l];
    const LevelGeom& Gc = H->geo[l + 1];
    TransferOp& T = H->tr[l];
    T.nv = p.nv[l];
    T.fine_ndof = G.ndof;
    T.nb = 1;
    for (int m = 0; m < 4; m++) {
      T.block[m] = p.block[l][m];
      T.cdims[m] = Gc.L[m];
      T.nb *= p.block[l][m];
    }
    T.ncoarse = Gc.nsites;
    T.fine_half = l == 0 ? G.Vh : (G.eo ? G.half : G.nsites);
    T.store = (p.storage == MG_STORE_FP16) ? STORE_F16 : (p.storage == MG_STORE_BF16 ? STORE_BF16 : STORE_F32);
    T.fa.wilson = l == 0;
    T.flags = c->ws.flags.as<int>();
    T.fa.Vh = G.Vh;
    T.fa.ndof = G.ndof;
    // block map: coarse storage index -> fine storage indices of its block (bx fastest)
    std::vector<int> bm((size_t)T.ncoarse * T.nb);
    for (int cs = 0; cs < Gc.nsites; cs++) {
      int cc[4], r = Gc.lex_of[cs];
      for (int m = 0; m < 4; m++) {
        cc[m] = r % Gc.L[m];
        r /= Gc.L[m];
      }
      for (int i = 0; i < T.nb; i++) {
        int lc[4], q = i;
        for (int m = 0; m < 4; m++) {
          lc[m] = q % T.block[m];
          q /= T.block[m];
        }
        int fc[4];
        for (int m = 0; m < 4; m++) fc[m] = cc[m] * T.block[m] + lc[m];
        bm[(size_t)cs * T.nb + i] = G.coord_to_store(fc);
      }
    }
    T.blockmap.alloc(sizeof(int) * bm.size());
    MG_CUDA(cudaMemcpy(T.blockmap.get(), bm.data(), sizeof(int) * bm.size(), cudaMemcpyHostToDevice));
    std::vector<int> el;
    T.nbe = -1;
    for (int cs = 0; cs < Gc.nsites; cs++) {
      int n = 0;
      for (int i = 0; i < T.nb; i++)
        if (bm[(size_t)cs * T.nb + i] < T.fine_half) {
          el.push_back(i);
          n++;
        }
      if (cs == 0) T.nbe = n;
      if (n != T.nbe || n == 0) {
        T.nbe = -1;
        break;
      }
    }
    if (T.nbe > 0) {
      T.evenlist.alloc(sizeof(int) * el.size());
      MG_CUDA(cudaMemcpy(T.evenlist.get(), el.data(), sizeof(int) * el.size(), cudaMemcpyHostToDevice));
    }
    const size_t esz = T.store == STORE_F32 ? sizeof(float2) : 4;
    T.P.alloc(esz * (size_t)T.ncoarse * T.nb * T.fine_ndof * T.nv);
    T.Pscale.alloc(sizeof(float) * 2 * (size_t)T.ncoarse);
    H->nullvecs[l].alloc(sizeof(float) * 2 * full_n(*H, l) * T.nv);
    MG_CUDA(cudaMemset(H->nullvecs[l].get(), 0, sizeof(float) * 2 * full_n(*H, l) * T.nv));

    find_null_vectors(c, *H, l, info);
    std::vector<const float*> V(T.nv);
    for (int k = 0; k < T.nv; k++) V[k] = H->nullvecs[l].as<float>() + (size_t)k * 2 * full_n(*H, l);
    block_orthonormalize(T, V.data(), H->gs_scratch, c->ws.flags.as<int>(), c->stream);
    if (c->read_flag(FLAG_GS_BREAKDOWN, true)) raise(MG_ERR_GS_BREAKDOWN, "block Gram-Schmidt breakdown");
    build_coarse_links(c, *H, l);
    if (info) info->coarse_sites[l] = Gc.nsites;
  }
  H->gs_scratch.release();
  c->sync();
  c->mg = std::move(H);
  if (info) info->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// The cycle of level 0 for nb right-hand sides at once (packed half vectors,
// stride 24 Vh floats): multi-RHS D_r in the smoother, all coarsest-level
// solves in one persistent launch per group of up to coarse_gcr_batch_max().
// Each rhs gets exactly the arithmetic of mg_precondition.  It is split around
// the coarsest solve so that several contexts can share that launch:
// mg_batch_pre (pre-smoothing, restriction to bw.rc), the coarse solve
// (bw.rc -> bw.ec), mg_batch_post (prolongation, post-smoothing).
namespace {
struct BatchCtx {
  Hierarchy& H;
  const mg_params& p;
  cudaStream_t s;
  size_t n, hs, nfc, cs;
  BatchCtx(Ctx* c, int nb) : H(*c->mg), p(c->params), s(c->stream) {
    n = half_n(H, 0);
    hs = 2 * n;
    nfc = full_n(H, 1);
    cs = 2 * nfc;
    BatchWork& bw = H.bw;
    if (bw.cap < nb) {
      bw.rc.alloc(sizeof(float) * cs * nb);
      bw.ec.alloc(sizeof(float) * cs * nb);
      for (DBuf* d : {&bw.res, &bw.w, &bw.e, &bw.z0}) d->alloc(sizeof(float) * hs * nb);
      bw.scr.alloc(sizeof(double) * 4 * nb);
      bw.cap = nb;
    }
  }
};

// e = MR_nu(D_r, r) for nb rhs (r consumed)
void batch_mr(Ctx* c, BatchCtx& b, float* ev, float* rv, int nu, int nb) {
  float* w = b.H.bw.w.as<float>();
  double* scr = b.H.bw.scr.as<double>();
  blas_zero<float>(ev, b.n * nb, b.s);
  for (int it = 0; it < nu; it++) {
    b.H.F32->Dr_multi(w, rv, nb, b.hs);
    blas_dot2_multi<float>(w, rv, b.n, b.hs, nb, scr, c->ws, b.s);
    blas_mr_update_multi<float>(ev, rv, w, scr, b.n, b.hs, nb, b.s);
  }
}
}  // namespace

void mg_batch_pre(Ctx* c, float* z, const float* r, int nb) {
  if (!c->mg) raise(MG_ERR_STATE, "multigrid not set up");
  BatchCtx b(c, nb);
  BatchWork& bw = b.H.bw;
  float* res = bw.res.as<float>();
  const float* rin = r;
  if (b.p.nu_pre > 0) {
    float* w = bw.w.as<float>();
    blas_convert<float, float>(res, r, b.n * nb, b.s);
    batch_mr(c, b, z, res, b.p.nu_pre, nb);
    b.H.F32->Dr_multi(w, z, nb, b.hs);
    blas_convert<float, float>(res, r, b.n * nb, b.s);
    blas_axpby<float>(-1.0, w, 1.0, res, b.n * nb, b.s);
    rin = res;
  }
  restrict_vec_multi(b.H.tr[0], nb, bw.rc.as<float>(), b.cs, rin, b.hs, true, b.s);
}

bool mg_batch_joinable(Ctx* c) { return c->mg && c->mg->L == 2; }

void mg_batch_systems(Ctx* c, int nb, std::vector<CoarseSystem>& out) {
  if (!mg_batch_joinable(c)) raise(MG_ERR_STATE, "only 2-level hierarchies join a shared coarsest solve");
  Hierarchy& H = *c->mg;
  const size_t cs = 2 * full_n(H, 1);
  for (int q = 0; q < nb; q++)
    out.push_back(CoarseSystem{&H.geo[1], &H.cop[1], H.bw.rc.as<float>() + q * cs, H.bw.ec.as<float>() + q * cs,
                               c->params.tol_coarse, H.d_iters.as<long long>() + 1});
}

CoarseGCRBuffers& mg_batch_buffers(Ctx* c) { return c->mg->work[1].cg; }

void mg_batch_coarse(Ctx* c, int nb) {
  LevelTime timer(c, 1);
  BatchCtx b(c, nb);
  if (b.H.L == 2) {
    const int restart = b.p.restart_coarse > 0 ? b.p.restart_coarse : 32;
    const int gmax = coarse_gcr_batch_max();
    std::vector<CoarseSystem> sys;
    mg_batch_systems(c, nb, sys);
    const LevelGeom& G1 = b.H.geo[1];
    const CoarseOp& C1 = b.H.cop[1];
    const bool tc = b.p.coarse_impl == 0 || b.p.coarse_impl == 4;
    auto batched = [&]() {
      for (int q0 = 0; q0 < nb; q0 += gmax) {
        std::vector<CoarseSystem> part(sys.begin() + q0, sys.begin() + std::min(nb, q0 + gmax));
        // tensor cores for FP16 links (the group's systems are consecutive vectors of this context)
        if (tc && coarse_gcr_tc_try(part, b.H.work[1].cg, restart, b.p.maxit_coarse, c->ws.flags.as<int>(), b.s))
          continue;
        coarse_gcr_solve_multi(part, b.H.work[1].cg, restart, b.p.maxit_coarse, c->ws.flags.as<int>(), b.s);
      }
    };
    auto one_by_one = [&]() {   // the single-system solver the autotuner chose for this level
      for (int q = 0; q < nb; q++)
        coarse_solve(c, b.H, 1, b.H.bw.ec.as<float>() + q * b.cs, b.H.bw.rc.as<float>() + q * b.cs);
    };
    int& choice = b.H.work[1].batch_impl[std::min(nb, 16)];
    if (choice < 0) {
      if (b.p.coarse_impl != 0) {
        choice = 0;   // a forced implementation keeps the batched launches
      } else {
        // time both on the real systems; the tuning runs leave the iteration counters as they were
        long long* d_it = b.H.d_iters.as<long long>();
        DBuf keep(sizeof(long long) * MG_MAX_LEVELS);
        MG_CUDA(cudaMemcpyAsync(keep.get(), d_it, sizeof(long long) * MG_MAX_LEVELS, cudaMemcpyDeviceToDevice, b.s));
        choice = tuned_block(TuneKey{"coarse_batch", {G1.L[0], G1.L[1], G1.L[2], G1.L[3]}, nb, C1.store}, {0, 1},
                             [&](int which) {
                               if (which)
                                 one_by_one();
                               else
                                 batched();
                             },
                             b.s);
        MG_CUDA(cudaMemcpyAsync(d_it, keep.get(), sizeof(long long) * MG_MAX_LEVELS, cudaMemcpyDeviceToDevice, b.s));
        MG_CUDA(cudaStreamSynchronize(b.s));
      }
    }
    if (choice == 1)
      one_by_one();
    else
      batched();
  } else {
    for (int q = 0; q < nb; q++)
      coarse_solve(c, b.H, 1, b.H.bw.ec.as<float>() + q * b.cs, b.H.bw.rc.as<float>() + q * b.cs);
  }
}

void mg_batch_post(Ctx* c, float* z, const float* r, int nb) {
  BatchCtx b(c, nb);
  BatchWork& bw = b.H.bw;
  const TransferOp& T = b.H.tr[0];
  float* ec = bw.ec.as<float>();
  if (b.p.nu_pre > 0) {
    float* z0 = bw.z0.as<float>();
    prolong_vec_multi(T, nb, z0, b.hs, ec, b.cs, true, b.s);
    blas_axpby<float>(1.0, z0, 1.0, z, b.n * nb, b.s);
  } else {
    prolong_vec_multi(T, nb, z, b.hs, ec, b.cs, true, b.s);
  }
  if (b.p.nu_post > 0) {
    float* w = bw.w.as<float>();
    float* res = bw.res.as<float>();
    float* e = bw.e.as<float>();
    b.H.F32->Dr_multi(w, z, nb, b.hs);
    blas_convert<float, float>(res, r, b.n * nb, b.s);
    blas_axpby<float>(-1.0, w, 1.0, res, b.n * nb, b.s);
    batch_mr(c, b, e, res, b.p.nu_post, nb);
    blas_axpby<float>(1.0, e, 1.0, z, b.n * nb, b.s);
  }
}

void mg_precondition_batch(Ctx* c, float* z, const float* r, int nb) {
  LevelTime timer(c, 0);
  mg_batch_pre(c, z, r, nb);
  mg_batch_coarse(c, nb);
  mg_batch_post(c, z, r, nb);
}

void mg_cycle_batch(Ctx* c, double* out_abi, const double* in_abi, int nb) {
  if (!c->mg) raise(MG_ERR_STATE, "multigrid not set up");
  if (c->mg->L < 2) raise(MG_ERR_ARG, "no coarser level");
  const size_t hs = 24 * c->Vh;
  cudaStream_t s = c->stream;
  DBuf ib(sizeof(float) * 2 * hs * nb), ob(sizeof(float) * 2 * hs * nb);
  MG_CUDA(cudaMemsetAsync(ob.get(), 0, sizeof(float) * 2 * hs * nb, s));
  float* ie = ib.as<float>();
  float* io = ie + hs * nb;
  float* oe = ob.as<float>();
  float* oo = oe + hs * nb;   // stays zero: the cycle writes even sites only
  for (int q = 0; q < nb; q++) pack_spinor(c->g, in_abi + (size_t)q * 24 * c->V, ie + q * hs, io + q * hs, true, s);
  mg_precondition_batch(c, oe, ie, nb);
  for (int q = 0; q < nb; q++) unpack_spinor(c->g, oe + q * hs, oo + q * hs, true, out_abi + (size_t)q * 24 * c->V, s);
  c->sync();
}

// z_e = K(r_e) for an FP64 residual: the conversion to FP32 and the whole
// 2-level cycle (restriction, persistent coarsest solve, prolongation, MR
// smoothing: ~30 launches, no host synchronisation) are captured once into a
// CUDA graph on a private stream and replayed with one launch; the output is
// copied to z_e.  Returns false (nothing launched) when graphs are off or
// unavailable -- deeper hierarchies (their intermediate GCRs test convergence
// on the host), before the autotuner has chosen the coarsest solver (it
// synchronises), or after a failed capture -- and the caller runs the cycle
// directly.
bool mg_precondition_graph(Ctx* c, float* z_e, const double* r_e, float* r32) {
  if (!c->mg || !c->params.cuda_graphs || c->params.level_timing) return false;
  Hierarchy& H = *c->mg;
  CycleGraph& G = H.graph;
  if (H.L != 2 || G.failed || H.work[1].coarse_impl < 0) return false;
  const size_t n = half_n(H, 0);
  if (!G.exec || G.r != r_e || G.r32 != r32) {
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
    if (!G.zc.get()) G.zc.alloc(sizeof(float) * 2 * n);
    if (!G.cap) MG_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    cudaStream_t saved = c->stream;
    c->stream = G.cap;
    const long long d0 = c->dslash_launches, k0 = launches_so_far();
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
      try {
        blas_convert<double, float>(r32, r_e, n, G.cap);
        cycle(c, H, 0, G.zc.as<float>(), r32);
      } catch (const Error&) {
        ok = false;
      }
      ok = cudaStreamEndCapture(G.cap, &graph) == cudaSuccess && ok && graph;
    }
    c->stream = saved;
    // the captured launches did not run: count them when a replay runs them
    G.dslash = c->dslash_launches - d0;
    G.kernels = launches_so_far() - k0;
    c->dslash_launches = d0;
    add_launches(-G.kernels);
    if (ok) ok = cudaGraphInstantiate(&G.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      G.exec = nullptr;
      G.failed = true;
      (void)cudaGetLastError();   // clear the capture error; run the cycle directly from now on
      return false;
    }
    G.r = r_e;
    G.r32 = r32;
  }
  MG_CUDA(cudaGraphLaunch(G.exec, c->stream));
  c->dslash_launches += G.dslash;
  add_launches(G.kernels);
  MG_CUDA(cudaMemcpyAsync(z_e, G.zc.get(), sizeof(float) * 2 * n, cudaMemcpyDeviceToDevice, c->stream));
  return true;
}

void mg_solve_params_changed(Ctx* c) {
  if (!c->mg) return;
  for (LevelWork& W : c->mg->work) {   // choose (or force) the coarsest solver again
    W.coarse_impl = -1;
    for (int& v : W.batch_impl) v = -1;
  }
  if (!c->mg->graph.exec) return;
  MG_CUDA(cudaStreamSynchronize(c->stream));   // no replay in flight
  c->mg->graph.drop();
}

void mg_precondition(Ctx* c, float* z_e, const float* r_e) {
  if (!c->mg) raise(MG_ERR_STATE, "multigrid not set up");
  cycle(c, *c->mg, 0, z_e, r_e);
}

void mg_benchmark_coarse(Ctx* c, int warmup, int iters, double* avg_ms, double* bytes) {
  if (!c->mg || c->mg->L < 2) raise(MG_ERR_STATE, "multigrid not set up");
  Hierarchy& H = *c->mg;
  const LevelGeom& G = H.geo[1];
  if (!G.eo) raise(MG_ERR_DIMS, "level 1 has an odd extent");
  const size_t n = full_n(H, 1);
  DBuf ib(sizeof(float) * 2 * n), ob(sizeof(float) * 2 * n);
  philox_coarse_vector(G, 777, 1, 0, ib.as<float>(), c->stream);
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  for (int w = 0; w < warmup; w++) Dr_level(c, H, 1, ob.as<float>(), ib.as<float>());
  MG_CUDA(cudaEventRecord(e0, c->stream));
  for (int it = 0; it < iters; it++) Dr_level(c, H, 1, ob.as<float>(), ib.as<float>());
  MG_CUDA(cudaEventRecord(e1, c->stream));
  MG_CUDA(cudaEventSynchronize(e1));
  float t = 0;
  MG_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *avg_ms = t / iters;
  const double nc = H.cop[1].nc;
  *bytes = (double)G.half * (18.0 * nc * nc + 7.0 * nc) * sizeof(float2);
}

void mg_benchmark_transfer(Ctx* c, bool restrict, int nrhs, int warmup, int iters, double* avg_ms, double* bytes) {
  if (!c->mg || c->mg->L < 2) raise(MG_ERR_STATE, "multigrid not set up");
  Hierarchy& H = *c->mg;
  const TransferOp& T = H.tr[0];
  const size_t fn = (size_t)48 * c->Vh, cn = (size_t)2 * 2 * T.nv * T.ncoarse;
  DBuf fb(sizeof(float) * fn * nrhs), cb(sizeof(float) * cn * nrhs);
  for (int q = 0; q < nrhs; q++) {
    float* f = fb.as<float>() + q * fn;
    philox_fine_vector(c->g, 4242, 0, q, f, f + fn / 2, c->stream);
    philox_coarse_vector(H.geo[1], 4243, 1, q, cb.as<float>() + q * cn, c->stream);
  }
  auto once = [&]() {
    if (restrict)
      restrict_vec_multi(T, nrhs, cb.as<float>(), cn, fb.as<float>(), fn, true, c->stream);
    else
      prolong_vec_multi(T, nrhs, fb.as<float>(), fn, cb.as<float>(), cn, true, c->stream);
  };
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  for (int w = 0; w < warmup; w++) once();
  MG_CUDA(cudaEventRecord(e0, c->stream));
  for (int it = 0; it < iters; it++) once();
  MG_CUDA(cudaEventRecord(e1, c->stream));
  MG_CUDA(cudaEventSynchronize(e1));
  float t = 0;
  MG_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *avg_ms = t / iters;
  // P rows of the even sites once, the even half of each fine vector and each
  // coarse vector once
  const double esz = T.store == STORE_F32 ? 8.0 : 4.0;
  const double neven = T.nbe > 0 ? (double)T.nbe * T.ncoarse : (double)c->Vh;
  *bytes = neven * 12.0 * T.nv * esz + nrhs * ((double)c->Vh * 24 * sizeof(float) + (double)cn * sizeof(float));
}

void mg_benchmark_coarse_floor(Ctx* c, double* barrier_us, double* stream_us, double* stream_bytes, int* grid) {
  if (!c->mg || c->mg->L < 2) raise(MG_ERR_STATE, "multigrid not set up");
  Hierarchy& H = *c->mg;
  const int l = H.L - 1;
  if (!coarse_gcr_stream_ok(H.geo[l], H.cop[l])) raise(MG_ERR_STATE, "the coarsest level has no streamed solver");
  *grid = coarse_gcr_stream_grids(H.geo[l], H.cop[l])[0];
  coarse_floor(H.geo[l], H.cop[l], *grid, c->ws.flags.as<int>(), c->stream, barrier_us, stream_us, stream_bytes);
  if (c->read_flag(FLAG_TIMEOUT, true)) raise(MG_ERR_CUDA, "a wait in the coarse floor benchmark ran out of time");
}

void mg_benchmark_coarse_solve(Ctx* c, int warmup, int iters, double* avg_ms, double* bytes, double* its) {
  if (!c->mg || c->mg->L < 2) raise(MG_ERR_STATE, "multigrid not set up");
  Hierarchy& H = *c->mg;
  const int l = H.L - 1;
  const LevelGeom& G = H.geo[l];
  const CoarseOp& C = H.cop[l];
  const size_t n = full_n(H, l);
  DBuf bb(sizeof(float) * 2 * n), xb(sizeof(float) * 2 * n);
  philox_coarse_vector(G, 777, l, 0, bb.as<float>(), c->stream);
  long long* d_it = H.d_iters.as<long long>() + l;
  long long before = 0, after = 0;
  for (int w = 0; w < warmup; w++) coarse_solve(c, H, l, xb.as<float>(), bb.as<float>());
  MG_CUDA(cudaMemcpyAsync(&before, d_it, sizeof(before), cudaMemcpyDeviceToHost, c->stream));
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  MG_CUDA(cudaEventRecord(e0, c->stream));
  for (int it = 0; it < iters; it++) coarse_solve(c, H, l, xb.as<float>(), bb.as<float>());
  MG_CUDA(cudaEventRecord(e1, c->stream));
  MG_CUDA(cudaEventSynchronize(e1));
  MG_CUDA(cudaMemcpyAsync(&after, d_it, sizeof(after), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  float t = 0;
  MG_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (c->read_flag(FLAG_TIMEOUT, true)) raise(MG_ERR_CUDA, "a wait in the persistent coarse solve ran out of time");
  *avg_ms = t / iters;
  *its = (double)(after - before) / iters;
  // links of one application of the reduced operator: the folded odd-site links
  // (FP32) and the even-site Y in the storage format, each half x 8 Nc^2 complex
  const double esz = C.store == STORE_F32 ? 8.0 : 4.0;
  const double nc = C.nc;
  const double per_app = G.eo ? (double)G.half * 8.0 * nc * nc * (8.0 + esz) : (double)G.nsites * 9.0 * nc * nc * 8.0;
  *bytes = per_app * (*its + (G.eo ? 1.5 : 1.0));
}

void mg_reset_counters(Ctx* c) {
  if (!c->mg) return;
  c->mg->iters.assign(c->mg->L, 0);
  MG_CUDA(cudaMemsetAsync(c->mg->d_iters.get(), 0, sizeof(long long) * MG_MAX_LEVELS, c->stream));
}

void mg_read_counters(Ctx* c, long long* coarse_iters) {
  for (int l = 0; l < MG_MAX_LEVELS; l++) coarse_iters[l] = 0;
  if (!c->mg) return;
  long long dev[MG_MAX_LEVELS];
  MG_CUDA(cudaMemcpyAsync(dev, c->mg->d_iters.get(), sizeof(dev), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  for (int l = 0; l < c->mg->L && l < MG_MAX_LEVELS; l++) coarse_iters[l] = c->mg->iters[l] + dev[l];
  if (c->read_flag(FLAG_NAN, true)) raise(MG_ERR_NAN, "non-finite residual in the coarse solve");
  if (c->read_flag(FLAG_TIMEOUT, true)) raise(MG_ERR_CUDA, "a wait in the persistent coarse solve ran out of time");
}

void mg_level_dims(Ctx* c, int level, int dims[4], int* ndof) {
  if (level == 0) {
    for (int m = 0; m < 4; m++) dims[m] = c->dims[m];
    *ndof = 12;
    return;
  }
  if (!c->mg || level >= c->mg->L) raise(MG_ERR_STATE, "level not set up");
  for (int m = 0; m < 4; m++) dims[m] = c->mg->geo[level].L[m];
  *ndof = c->mg->geo[level].ndof;
}

void mg_get_links(Ctx* c, int level, double* Y_abi, double* X_abi) {
  if (!c->mg || level < 1 || level >= c->mg->L) raise(MG_ERR_STATE, "coarse level not set up");
  Hierarchy& H = *c->mg;
  coarse_links_abi(H.geo[level], H.cop[level], Y_abi, X_abi, c->stream);
}

// Adaptive refinement of the null vectors of transfer `level` (the alpha-SA idea the
// paper plans for the clover case, section "Setup procedure"): every vector v
// is relaxed on the homogeneous system D_p v = 0 with the current multigrid
// solver, v <- v - M D_p v, normalised after each step, where M ~ D_p^{-1} is
// the even-odd form of the current cycle K ~ D_r^{-1}: with D_p = [[1, X],
// [Y, 1]] (X = H_eo A_o^{-1}, Y = H_oe A_e^{-1}, D_r = 1 - X Y),
//   u_e = K (f_e - X f_o),   u_o = f_o - Y u_e   solves D_p u = f when K = D_r^{-1}.
// Components the current coarse space represents well are removed; what is
// left is rich in the modes the solver resolves poorly.  The caller rebuilds
// the hierarchy from the relaxed vectors.
void mg_relax_null_vectors(Ctx* c, int level, int relax) {
  if (!c->mg || level < 0 || level + 1 >= c->mg->L) raise(MG_ERR_STATE, "no transfer from this level");
  Hierarchy& H = *c->mg;
  const int l = level;
  const size_t nf = full_n(H, l), nh = half_n(H, l), hs = 2 * nh;
  cudaStream_t s = c->stream;
  if (l > 0 && !H.geo[l].eo) raise(MG_ERR_DIMS, "level has an odd extent");
  DBuf ub(sizeof(float) * 2 * nf), gb(sizeof(float) * 2 * nf), sb(sizeof(float) * 2 * nf);
  float* ue = ub.as<float>();
  float* uo = ue + hs;
  float* ge = gb.as<float>();
  float* se = sb.as<float>();
  double* scr = c->ws.scalars.as<double>() + 1024;
  const int nv = H.tr[l].nv;
  float* base = H.nullvecs[l].as<float>();
  std::vector<const float*> prev(nv);
  for (int k = 0; k < nv; k++) prev[k] = base + (size_t)k * 2 * nf;
  // inverse subspace iteration with the current solver of the level as the
  // approximate inverse: v_k <- M v_k, M = D_p^{-1} through the even-odd
  // reduction and one cycle, then Gram-Schmidt against v_0 .. v_{k-1}
  for (int k = 0; k < nv; k++) {
    float* ve = base + (size_t)k * 2 * nf;
    float* vo = ve + hs;
    for (int it = 0; it < relax; it++) {
      if (l == 0) {
        FineOps<float>& F = *H.F32;
        F.br(ge, ve, vo);                                                    // g_e = v_e - X v_o
        cycle(c, H, 0, ue, ge);                                              // u_e = K g_e
        clover_apply<float>(c->g, se, ue, c->Ainv<float>(0), s);            // A_e^{-1} u_e
        dslash<float>(c->g, EPI_XPAY, 1, uo, se, c->gauge<float>(), nullptr, vo, -1.0, 0xff, s);  // u_o = v_o - Y u_e
      } else {
        // the same on a coarse level: vectors are full coarse vectors, even sites first
        const LevelGeom& G = H.geo[l];
        const CoarseOp& C = H.cop[l];
        br_level(c, H, l, ge, ve);                                           // g_e = v_e - Y_eo X_o^{-1} v_o
        blas_zero<float>(ue, nf, s);
        cycle(c, H, l, ue, ge);                                              // u_e = K g_e
        coarse_site_mul(G, C, true, 0, G.half, se, ue, s);                   // X_e^{-1} u_e
        coarse_hop(G, C, EPI_XPAY, false, G.half, G.nsites, ue, se, ve, -1.f, 0xff, s);  // u_o = v_o - Y_oe .
      }
      blas_convert<float, float>(ve, ue, nf, s);                            // v = M v
      for (int rep = 0; rep < 2 && k > 0; rep++) {
        blas_multidot<float>(prev.data(), k, ve, nf, scr, c->ws, s);
        blas_lincomb<float, float>(ve, prev.data(), scr, k, -1.0, nf, s);
      }
      blas_norm2<float>(ve, nf, scr + 512, c->ws, s);
      const double nn = c->read_scalar(scr + 512);
      if (!std::isfinite(nn) || nn == 0.0) raise(MG_ERR_GS_BREAKDOWN, "null vector lost in the adaptive iteration");
      blas_normalize<float>(ve, scr + 512, nf, s);
    }
  }
  c->sync();
}

void mg_get_vectors(Ctx* c, int level, double* V_abi, int nv) {
  if (!c->mg || level + 1 >= c->mg->L) raise(MG_ERR_STATE, "transfer not set up");
  Hierarchy& H = *c->mg;
  if (nv != H.tr[level].nv) raise(MG_ERR_NV, "nv does not match the setup");
  const size_t n = full_n(H, level);
  for (int k = 0; k < nv; k++) {
    const float* v = H.nullvecs[level].as<float>() + (size_t)k * 2 * n;
    if (level == 0)
      unpack_spinor(c->g, v, v + 24 * c->Vh, true, V_abi + (size_t)k * 2 * n, c->stream);
    else
      unpack_coarse(H.geo[level], v, V_abi + (size_t)k * 2 * n, c->stream);
  }
  c->sync();
}

// Apply `op` on a coarse level (level >= 1), or R / P from any level.
void mg_apply_level(Ctx* c, int op, int level, double* out_abi, const double* in_abi) {
  if (!c->mg) raise(MG_ERR_STATE, "multigrid not set up");
  Hierarchy& H = *c->mg;
  cudaStream_t s = c->stream;
  auto pack = [&](int l, const double* abi, float* v) {
    if (l == 0)
      pack_spinor(c->g, abi, v, v + 24 * c->Vh, true, s);
    else
      pack_coarse(H.geo[l], abi, v, s);
  };
  auto unpack = [&](int l, const float* v, double* abi) {
    if (l == 0)
      unpack_spinor(c->g, v, v + 24 * c->Vh, true, abi, s);
    else
      unpack_coarse(H.geo[l], v, abi, s);
  };
  if (op == MG_OP_R || op == MG_OP_P) {
    if (level < 0 || level + 1 >= H.L) raise(MG_ERR_ARG, "no transfer from this level");
    DBuf fb(sizeof(float) * 2 * full_n(H, level)), cb(sizeof(float) * 2 * full_n(H, level + 1));
    if (op == MG_OP_R) {
      pack(level, in_abi, fb.as<float>());
      restrict_vec(H.tr[level], cb.as<float>(), fb.as<float>(), false, s);
      unpack(level + 1, cb.as<float>(), out_abi);
    } else {
      pack(level + 1, in_abi, cb.as<float>());
      prolong_vec(H.tr[level], fb.as<float>(), cb.as<float>(), false, s);
      unpack(level, fb.as<float>(), out_abi);
    }
    c->sync();
    return;
  }
  if (op == MG_OP_CYCLE) {
    if (level + 1 >= H.L) raise(MG_ERR_ARG, "no coarser level");
    const size_t n = full_n(H, level);
    DBuf ib(sizeof(float) * 2 * n), ob(sizeof(float) * 2 * n);
    MG_CUDA(cudaMemsetAsync(ib.get(), 0, sizeof(float) * 2 * n, s));
    MG_CUDA(cudaMemsetAsync(ob.get(), 0, sizeof(float) * 2 * n, s));
    pack(level, in_abi, ib.as<float>());
    if (level > 0) {  // even sites only: zero the odd half of the input
      const LevelGeom& G = H.geo[level];
      if (!G.eo) raise(MG_ERR_DIMS, "level has an odd extent");
      MG_CUDA(cudaMemsetAsync(ib.as<float>() + 2 * (size_t)G.half * G.ndof, 0,
                              sizeof(float) * 2 * (size_t)(G.nsites - G.half) * G.ndof, s));
    }
    cycle(c, H, level, ob.as<float>(), ib.as<float>());
    unpack(level, ob.as<float>(), out_abi);
    c->sync();
    return;
  }
  if (level < 1 || level >= H.L) raise(MG_ERR_ARG, "coarse level out of range");
  const LevelGeom& G = H.geo[level];
  const size_t n = full_n(H, level);
  DBuf ib(sizeof(float) * 2 * n), ob(sizeof(float) * 2 * n);
  float* in = ib.as<float>();
  float* out = ob.as<float>();
  pack(level, in_abi, in);
  MG_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * 2 * n, s));
  switch (op) {
    case MG_OP_D: Dfull_level(c, H, level, out, in); break;
    case MG_OP_DP: Dp_level(c, H, level, out, in); break;
    case MG_OP_M: Minv_level(c, H, level, out, in, false); break;
    case MG_OP_MINV: Minv_level(c, H, level, out, in, true); break;
    case MG_OP_HOP: coarse_hop(G, H.cop[level], EPI_H, false, 0, G.nsites, out, in, nullptr, 0.f, 0xff, s); break;
    case MG_OP_DR:
      if (!G.eo) raise(MG_ERR_DIMS, "level has an odd extent");
      Dr_level(c, H, level, out, in);
      break;
    case MG_OP_BR:
      if (!G.eo) raise(MG_ERR_DIMS, "level has an odd extent");
      br_level(c, H, level, out, in);
      break;
    default: raise(MG_ERR_ARG, "unknown operator");
  }
  unpack(level, out, out_abi);
  c->sync();
}

const char* level_range_name(int what, int l) {
  static const char* names[4][MG_MAX_LEVELS] = {
      {"cycle level 0", "cycle level 1", "cycle level 2", "cycle level 3"},
      {"coarse solve level 0", "coarse solve level 1", "coarse solve level 2", "coarse solve level 3"},
      {"null vectors level 0", "null vectors level 1", "null vectors level 2", "null vectors level 3"},
      {"coarse links level 0", "coarse links level 1", "coarse links level 2", "coarse links level 3"}};
  return names[what & 3][l < 0 ? 0 : (l >= MG_MAX_LEVELS ? MG_MAX_LEVELS - 1 : l)];
}

LevelTime::LevelTime(Ctx* ctx, int l) : c(ctx), level(l) {
  if (!c->params.level_timing || level < 0 || level >= MG_MAX_LEVELS) {
    level = -1;
    return;
  }
  auto& v = c->level_events[level];
  slot = c->level_events_used[level]++;
  if (slot >= (int)v.size()) {
    cudaEvent_t a, b;
    MG_CUDA(cudaEventCreate(&a));
    MG_CUDA(cudaEventCreate(&b));
    v.emplace_back(a, b);
  }
  MG_CUDA(cudaEventRecord(v[slot].first, c->stream));
}

LevelTime::~LevelTime() {
  if (level >= 0) cudaEventRecord(c->level_events[level][slot].second, c->stream);
}

void level_times_reset(Ctx* c) {
  for (int l = 0; l < MG_MAX_LEVELS; l++) c->level_events_used[l] = 0;
}

void level_times(Ctx* c, double out_ms[MG_MAX_LEVELS]) {
  for (int l = 0; l < MG_MAX_LEVELS; l++) out_ms[l] = 0.0;
  if (!c->params.level_timing) return;
  MG_CUDA(cudaStreamSynchronize(c->stream));
  for (int l = 0; l < MG_MAX_LEVELS; l++) {
    for (int k = 0; k < c->level_events_used[l]; k++) {
      float ms = 0.f;
      MG_CUDA(cudaEventElapsedTime(&ms, c->level_events[l][k].first, c->level_events[l][k].second));
      out_ms[l] += ms;
    }
  }
  level_times_reset(c);
}

}  // namespace mg
