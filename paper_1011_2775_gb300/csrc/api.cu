// The C ABI of libmgclover (declared and documented in include/mgclover.h).
//
// Every entry point converts internal exceptions to a status code and keeps
// the message for mg_last_error().  Host buffers are staged through device
// memory owned by the context; device buffers are read and written in place.
#include <algorithm>
#include <chrono>
#include <vector>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "coarse.h"
#include "internal.h"

namespace {
thread_local std::string g_last_error;

template <typename F>
int guarded(F&& f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const mg::Error& e) {
    g_last_error = e.what;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return MG_ERR_ALLOC;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return MG_ERR_CUDA;
  }
}

mg::Ctx* as_ctx(void* p) {
  if (!p) mg::raise(MG_ERR_ARG, "null context");
  mg::Ctx* c = static_cast<mg::Ctx*>(p);
  MG_CUDA(cudaSetDevice(c->device));
  return c;
}

// size (complex numbers) of one vector of level `level` under the current params
size_t level_vec_complex(mg::Ctx* c, int level, int* ndof_out) {
  int d[4] = {c->dims[0], c->dims[1], c->dims[2], c->dims[3]};
  int ndof = 12;
  for (int l = 0; l < level; l++) {
    for (int m = 0; m < 4; m++) d[m] /= c->params.block[l][m];
    ndof = 2 * c->params.nv[l];
  }
  if (ndof_out) *ndof_out = ndof;
  return (size_t)d[0] * d[1] * d[2] * d[3] * ndof;
}

// device pointer for a caller buffer: the buffer itself or a staging copy
struct Staged {
  mg::DBuf own;
  double* ptr = nullptr;
};

void stage_in(mg::Ctx* c, Staged& st, const void* user, size_t bytes, int where) {
  if (where == MG_DEVICE) {
    st.ptr = const_cast<double*>(static_cast<const double*>(user));
    return;
  }
  st.own.alloc(bytes);
  st.ptr = st.own.as<double>();
  MG_CUDA(cudaMemcpyAsync(st.ptr, user, bytes, cudaMemcpyHostToDevice, c->stream));
}

void stage_out_alloc(Staged& st, void* user, size_t bytes, int where) {
  if (where == MG_DEVICE) {
    st.ptr = static_cast<double*>(user);
    return;
  }
  st.own.alloc(bytes);
  st.ptr = st.own.as<double>();
}

void stage_out_finish(mg::Ctx* c, Staged& st, void* user, size_t bytes, int where) {
  if (where == MG_HOST) MG_CUDA(cudaMemcpyAsync(user, st.ptr, bytes, cudaMemcpyDeviceToHost, c->stream));
  c->sync();
}

void check_where(int where) {
  if (where != MG_HOST && where != MG_DEVICE) mg::raise(MG_ERR_ARG, "where must be MG_HOST or MG_DEVICE");
}

// mg_solve / mg_solve_dagger.  The dagger form solves D^dag psi = eta as
// psi = gamma_5 D^{-1} gamma_5 eta (D^dag = gamma_5 D gamma_5).
int solve_impl(void* ctx, void* psi, const void* eta, int nrhs, double tol, int mode, int where,
               mg_solve_info* info, bool dagger) {
  const auto t0 = std::chrono::steady_clock::now();
  mg::Ctx* c = as_ctx(ctx);
  check_where(where);
  if (!psi || !eta || nrhs < 1 || !(tol > 0)) mg::raise(MG_ERR_ARG, "bad solve arguments");
  if (mode < MG_MODE_MG || mode > MG_MODE_BICGSTAB_MP) mg::raise(MG_ERR_ARG, "bad mode");
  if (!c->have_clover) mg::raise(MG_ERR_STATE, "set the gauge field and clover first");
  if (mode == MG_MODE_MG && !c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
  mg_solve_info local;
  std::memset(&local, 0, sizeof(local));
  local.true_residual = 0.0;
  mg::mg_reset_counters(c);
  mg::level_times_reset(c);
  const long long launches0 = c->dslash_launches;
  const long long kernels0 = mg::launches_so_far();
  const size_t per = sizeof(double) * 24 * c->V;
  Staged si, so;
  if (dagger && where == MG_DEVICE) {
    // gamma_5 must not touch the caller's source: work on a copy
    si.own.alloc(per * nrhs);
    si.ptr = si.own.as<double>();
    MG_CUDA(cudaMemcpyAsync(si.ptr, eta, per * nrhs, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    stage_in(c, si, eta, per * nrhs, where);
  }
  stage_out_alloc(so, psi, per * nrhs, where);
  if (dagger) mg::gamma5_abi(si.ptr, c->V * nrhs, c->stream);
  int status = MG_OK;
  const int blk = mode == MG_MODE_MG ? c->params.rhs_block : 1;
  for (int r = 0; r < nrhs; r += blk) {
    const int nb = nrhs - r < blk ? nrhs - r : blk;
    double* po = so.ptr + (size_t)r * 24 * c->V;
    const double* pi = si.ptr + (size_t)r * 24 * c->V;
    const int st = nb > 1 ? mg::solve_fine_block(c, po, pi, nb, tol, &local) : mg::solve_fine(c, po, pi, tol, mode, &local);
    if (st != MG_OK) status = st;
  }
  if (dagger) mg::gamma5_abi(so.ptr, c->V * nrhs, c->stream);
  stage_out_finish(c, so, psi, per * nrhs, where);
  mg::mg_read_counters(c, local.coarse_iterations);
  mg::level_times(c, local.level_ms);
  local.dslash_launches = c->dslash_launches - launches0;
  local.kernel_launches = mg::launches_so_far() - kernels0;
  local.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = local;
  return status;
}
}  // namespace

namespace mg {
// lets entry points defined in other files record their error detail
void set_last_error(const std::string& what) { g_last_error = what; }
}  // namespace mg

extern "C" {

const char* mg_strerror(int status) {
  switch (status) {
    case MG_OK: return "ok";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_DIMS: return "invalid lattice or block dimensions";
    case MG_ERR_NV: return "invalid number of null vectors";
    case MG_ERR_STATE: return "call out of order (missing gauge, clover, parameters or setup)";
    case MG_ERR_GS_BREAKDOWN: return "block Gram-Schmidt breakdown (locally dependent null vectors)";
    case MG_ERR_SINGULAR_CLOVER: return "singular clover or coarse diagonal block";
    case MG_ERR_NOT_CONVERGED: return "solver did not converge";
    case MG_ERR_NAN: return "NaN or Inf encountered";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_ALLOC: return "allocation failed";
    default: return "unknown status";
  }
}

const char* mg_last_error(void) { return g_last_error.c_str(); }

int mg_default_params(mg_params* p) {
  if (!p) return MG_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->levels = 2;
  for (int l = 0; l < MG_MAX_LEVELS; l++) {
    for (int m = 0; m < 4; m++) p->block[l][m] = 4;
    p->nv[l] = 24;
  }
  p->setup_iters = 20;
  p->setup_inner = 8;
  p->setup_rq_tol = 0.05;
  p->nu_pre = 0;
  p->nu_post = 4;
  p->tol_coarse = 0.1;
  p->maxit_coarse = 50;
  p->restart_coarse = 32;
  p->restart_fine = 16;
  p->maxit_fine = 500;
  p->storage = MG_STORE_FP32;
  p->coarse_op = MG_COARSE_DP;
  p->seed = 3;
  p->rhs_block = 16;
  p->cuda_graphs = 1;
  p->coarse_impl = 0;
  p->outer_prec = MG_FP32;
  p->level_timing = 0;
  return MG_OK;
}

int mg_create(void** ctx_out, const int dims[4], int device, void* cuda_stream) {
  return guarded([&]() {
    if (!ctx_out || !dims) mg::raise(MG_ERR_ARG, "null argument");
    *ctx_out = nullptr;
    for (int m = 0; m < 4; m++)
      if (dims[m] < 2 || dims[m] % 2) mg::raise(MG_ERR_DIMS, "every lattice extent must be even and >= 2");
    const double vol = (double)dims[0] * dims[1] * dims[2] * dims[3];
    if (vol > 2.0e9) mg::raise(MG_ERR_DIMS, "lattice too large");
    MG_CUDA(cudaSetDevice(device));
    std::unique_ptr<mg::Ctx> c(new mg::Ctx());
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int m = 0; m < 4; m++) {
      c->dims[m] = dims[m];
      c->g.L[m] = dims[m];
    }
    c->V = (size_t)vol;
    c->Vh = c->V / 2;
    c->g.Vh = (int)c->Vh;
    c->g.xh = dims[0] / 2;
    c->g.apbc = 1;
    for (int m = 0; m < 4; m++) c->g.w[m] = 1.0;
    c->ws.init();
    mg_default_params(&c->params);
    *ctx_out = c.release();
    return MG_OK;
  });
}

int mg_destroy(void* ctx) {
  if (!ctx) return MG_OK;
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    cudaStreamSynchronize(c->stream);
    delete c;
    return MG_OK;
  });
}

int mg_load_gauge(void* ctx, const void* U, int where) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!U) mg::raise(MG_ERR_ARG, "null gauge field");
    check_where(where);
    const size_t bytes = sizeof(double) * 2 * 36 * c->V;
    Staged st;
    stage_in(c, st, U, bytes, where);
    if (!c->gauge64.get()) {
      c->gauge64.alloc(sizeof(double) * 2 * 36 * c->V);
      c->gauge32.alloc(sizeof(float) * 2 * 36 * c->V);
    }
    mg::pack_gauge(c->g, st.ptr, c->gauge64.as<double>(), c->gauge32.as<float>(), c->stream);
    c->sync();
    c->have_gauge = true;
    c->have_clover = false;
    c->mg.reset();
    return MG_OK;
  });
}

int mg_set_clover(void* ctx, double csw, double m0) {
  const double w[4] = {1.0, 1.0, 1.0, 1.0};
  return mg_set_clover_aniso(ctx, w, csw, csw, m0);
}

int mg_set_clover_aniso(void* ctx, const double* w, double csw_s, double csw_t, double m0) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!c->have_gauge) mg::raise(MG_ERR_STATE, "load the gauge field first");
    if (!w) mg::raise(MG_ERR_ARG, "null hopping weights");
    for (int m = 0; m < 4; m++)
      if (!(std::isfinite(w[m]) && w[m] > 0)) mg::raise(MG_ERR_ARG, "hopping weights must be positive and finite");
    if (!std::isfinite(csw_s) || !std::isfinite(csw_t) || !std::isfinite(m0)) mg::raise(MG_ERR_ARG, "non-finite csw or m0");
    const double csw = csw_s;
    if (!c->clov64.get()) {
      c->clov64.alloc(sizeof(double) * 144 * c->Vh);
      c->clovinv64.alloc(sizeof(double) * 144 * c->Vh);
      c->clov32.alloc(sizeof(float) * 144 * c->Vh);
      c->clovinv32.alloc(sizeof(float) * 144 * c->Vh);
    }
    c->mg.reset();
    c->have_clover = false;
    for (int m = 0; m < 4; m++) c->g.w[m] = w[m];   // every later hop of this context carries the weights
    mg::build_clover(c->g, c->gauge64.as<double>(), mg::CloverCoef{csw_s, csw_t}, m0, c->clov64.as<double>(),
                     c->clovinv64.as<double>(), c->clov32.as<float>(), c->clovinv32.as<float>(),
                     c->ws.flags.as<int>(), c->stream);
    if (c->read_flag(mg::FLAG_SINGULAR, true)) mg::raise(MG_ERR_SINGULAR_CLOVER, "singular clover block");
    c->csw = csw;
    c->csw_t = csw_t;
    c->m0 = m0;
    c->have_clover = true;
    return MG_OK;
  });
}

int mg_set_params(void* ctx, const mg_params* p) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!p) mg::raise(MG_ERR_ARG, "null params");
    if (p->levels < 1 || p->levels > MG_MAX_LEVELS) mg::raise(MG_ERR_ARG, "levels out of range");
    if (p->setup_iters < 1 || p->setup_inner < 1 || !(p->setup_rq_tol >= 0)) mg::raise(MG_ERR_ARG, "bad setup effort");
    if (p->nu_pre < 0 || p->nu_post < 0) mg::raise(MG_ERR_ARG, "negative smoothing steps");
    if (!(p->tol_coarse > 0) || p->maxit_coarse < 1 || p->restart_coarse < 1 || p->restart_coarse > 64)
      mg::raise(MG_ERR_ARG, "bad coarse solver parameters");
    if (p->restart_fine < 1 || p->restart_fine > 64 || p->maxit_fine < 1) mg::raise(MG_ERR_ARG, "bad outer solver parameters");
    if (p->storage < MG_STORE_FP32 || p->storage > MG_STORE_BF16) mg::raise(MG_ERR_ARG, "bad storage");
    if (p->coarse_op != MG_COARSE_DP && p->coarse_op != MG_COARSE_D) mg::raise(MG_ERR_ARG, "bad coarse_op");
    if (p->rhs_block < 1 || p->rhs_block > 16) mg::raise(MG_ERR_ARG, "rhs_block must be in [1, 16]");
    if (p->cuda_graphs != 0 && p->cuda_graphs != 1) mg::raise(MG_ERR_ARG, "cuda_graphs must be 0 or 1");
    if (p->coarse_impl < 0 || p->coarse_impl > 4) mg::raise(MG_ERR_ARG, "coarse_impl must be in [0, 4]");
    if (p->outer_prec != MG_FP32 && p->outer_prec != MG_FP64) mg::raise(MG_ERR_ARG, "outer_prec must be MG_FP32 or MG_FP64");
    if (p->level_timing != 0 && p->level_timing != 1) mg::raise(MG_ERR_ARG, "level_timing must be 0 or 1");
    int d[4] = {c->dims[0], c->dims[1], c->dims[2], c->dims[3]};
    int ndof = 12;
    for (int l = 0; l + 1 < p->levels; l++) {
      int nb = 1;
      for (int m = 0; m < 4; m++) {
        const int b = p->block[l][m];
        if (b < 1 || d[m] % b) mg::raise(MG_ERR_DIMS, "block does not divide the lattice");
        nb *= b;
      }
      const int nv = p->nv[l];
      // the coarse kernels hold at most 64 complex components per coarse site
      if (nv < 1 || nv > 32) mg::raise(MG_ERR_NV, "nv must be in [1, 32]");
      if (nv > nb * ndof / 2) mg::raise(MG_ERR_NV, "nv exceeds the dimension of a block's chiral subspace");
      for (int m = 0; m < 4; m++) d[m] /= p->block[l][m];
      ndof = 2 * nv;
      // every level below the coarsest runs an even-odd preconditioned solve
      if (l + 2 < p->levels)
        for (int m = 0; m < 4; m++)
          if (d[m] % 2) mg::raise(MG_ERR_DIMS, "a level below the coarsest has an odd extent");
    }
    // the setup (hierarchy, injected vectors) depends on these fields only;
    // smoothing, tolerances, caps, restart_fine and rhs_block take effect at
    // the next solve without a new setup
    const mg_params& o = c->params;
    bool setup_changed = !c->have_params || o.levels != p->levels || o.setup_iters != p->setup_iters ||
                         o.setup_inner != p->setup_inner || o.setup_rq_tol != p->setup_rq_tol ||
                         o.restart_coarse != p->restart_coarse || o.storage != p->storage ||
                         o.coarse_op != p->coarse_op || o.seed != p->seed;
    for (int l = 0; l + 1 < p->levels && !setup_changed; l++) {
      if (o.nv[l] != p->nv[l]) setup_changed = true;
      for (int m = 0; m < 4; m++)
        if (o.block[l][m] != p->block[l][m]) setup_changed = true;
    }
    c->params = *p;
    c->have_params = true;
    if (setup_changed) {
      c->mg.reset();
      c->injected.assign(MG_MAX_LEVELS, std::vector<double>());
    } else {
      mg::mg_solve_params_changed(c);
    }
    c->solve_work.reset();
    c->block_work.reset();
    return MG_OK;
  });
}

int mg_get_params(void* ctx, mg_params* p) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!p) mg::raise(MG_ERR_ARG, "null params");
    *p = c->params;
    return MG_OK;
  });
}

int mg_setup(void* ctx, mg_setup_info* info) {
  mg::Range range("mg_setup");
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!c->have_clover) mg::raise(MG_ERR_STATE, "set the gauge field and clover first");
    if (info) std::memset(info, 0, sizeof(*info));
    mg::mg_build(c, info);
    return MG_OK;
  });
}

int mg_set_null_vectors(void* ctx, int level, const void* V, int nv, int where) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    check_where(where);
    if (!V) mg::raise(MG_ERR_ARG, "null vectors");
    if (level < 0 || level + 1 >= c->params.levels) mg::raise(MG_ERR_ARG, "no transfer from this level");
    if (nv != c->params.nv[level]) mg::raise(MG_ERR_NV, "nv does not match the parameters");
    const size_t n = level_vec_complex(c, level, nullptr);
    if (c->injected.size() < MG_MAX_LEVELS) c->injected.assign(MG_MAX_LEVELS, std::vector<double>());
    std::vector<double>& h = c->injected[level];
    h.resize(2 * n * nv);
    if (where == MG_HOST) {
      std::memcpy(h.data(), V, sizeof(double) * h.size());
    } else {
      MG_CUDA(cudaMemcpy(h.data(), V, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    }
    c->mg.reset();
    return MG_OK;
  });
}

int mg_get_null_vectors(void* ctx, int level, void* V, int nv, int where) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    check_where(where);
    if (!V) mg::raise(MG_ERR_ARG, "null vectors");
    if (level < 0 || level + 1 >= c->params.levels) mg::raise(MG_ERR_ARG, "no transfer from this level");
    if (!c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
    if (nv != c->params.nv[level]) mg::raise(MG_ERR_NV, "nv does not match the setup");
    const size_t bytes = sizeof(double) * 2 * level_vec_complex(c, level, nullptr) * nv;
    Staged st;
    stage_out_alloc(st, V, bytes, where);
    mg::mg_get_vectors(c, level, st.ptr, nv);
    stage_out_finish(c, st, V, bytes, where);
    return MG_OK;
  });
}

// ---- setup reuse (the paper saves null vectors and coarse operators for later use)
namespace {
constexpr char kSetupMagic[8] = {'M', 'G', 'C', 'L', 'S', 'E', 'T', '3'};

struct SetupHeader {
  char magic[8];
  int32_t dims[4];
  mg_params params;
  double csw, m0;
  int32_t levels;
  double w[4], csw_t;   // hopping weights and the temporal clover coefficient
};

// the raw null vectors of every transfer of the current setup, complex128 on the host
std::vector<std::vector<double>> current_vectors(mg::Ctx* c) {
  std::vector<std::vector<double>> out;
  for (int l = 0; l + 1 < c->params.levels; l++) {
    const int nv = c->params.nv[l];
    const size_t n = level_vec_complex(c, l, nullptr) * nv;
    mg::DBuf d(sizeof(double) * 2 * n);
    mg::mg_get_vectors(c, l, d.as<double>(), nv);
    out.emplace_back(2 * n);
    MG_CUDA(cudaMemcpy(out.back().data(), d.get(), sizeof(double) * 2 * n, cudaMemcpyDeviceToHost));
  }
  return out;
}

// rebuild the hierarchy from given null vectors (no inverse iteration)
void rebuild_from(mg::Ctx* c, std::vector<std::vector<double>>& vecs, mg_setup_info* info) {
  c->injected.assign(MG_MAX_LEVELS, std::vector<double>());
  for (size_t l = 0; l < vecs.size(); l++) c->injected[l] = vecs[l];
  if (info) std::memset(info, 0, sizeof(*info));
  mg::mg_build(c, info);
}
}  // namespace

int mg_save_setup(void* ctx, const char* path) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!path) mg::raise(MG_ERR_ARG, "null path");
    if (!c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
    SetupHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kSetupMagic, 8);
    for (int m = 0; m < 4; m++) h.dims[m] = c->dims[m];
    h.params = c->params;
    h.csw = c->csw;
    h.m0 = c->m0;
    for (int m = 0; m < 4; m++) h.w[m] = c->g.w[m];
    h.csw_t = c->csw_t;
    h.levels = c->params.levels;
    std::vector<std::vector<double>> vecs = current_vectors(c);
    std::FILE* f = std::fopen(path, "wb");
    if (!f) mg::raise(MG_ERR_ARG, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    for (const auto& v : vecs) ok = ok && std::fwrite(v.data(), sizeof(double), v.size(), f) == v.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) mg::raise(MG_ERR_ARG, std::string("writing ") + path + " failed");
    return MG_OK;
  });
}

int mg_load_setup(void* ctx, const char* path, mg_setup_info* info) {
  return guarded([&]() {
    const auto t0 = std::chrono::steady_clock::now();
    mg::Ctx* c = as_ctx(ctx);
    if (!path) mg::raise(MG_ERR_ARG, "null path");
    if (!c->have_clover) mg::raise(MG_ERR_STATE, "load the gauge field and set the clover first");
    std::FILE* f = std::fopen(path, "rb");
    if (!f) mg::raise(MG_ERR_ARG, std::string("cannot open ") + path);
    SetupHeader h;
    const bool hdr = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, kSetupMagic, 8) == 0;
    if (!hdr) {
      std::fclose(f);
      mg::raise(MG_ERR_ARG, std::string(path) + " is not a saved multigrid setup");
    }
    for (int m = 0; m < 4; m++)
      if (h.dims[m] != c->dims[m]) {
        std::fclose(f);
        mg::raise(MG_ERR_DIMS, "the saved setup belongs to another lattice");
      }
    const int st = mg_set_params(ctx, &h.params);
    if (st != MG_OK) {
      std::fclose(f);
      return st;
    }
    std::vector<std::vector<double>> vecs;
    bool ok = true;
    for (int l = 0; l + 1 < h.params.levels && ok; l++) {
      const size_t n = 2 * level_vec_complex(c, l, nullptr) * h.params.nv[l];
      vecs.emplace_back(n);
      ok = std::fread(vecs.back().data(), sizeof(double), n, f) == n;
    }
    std::fclose(f);
    if (!ok) mg::raise(MG_ERR_ARG, std::string(path) + " is truncated");
    rebuild_from(c, vecs, info);
    if (info)
      info->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return (int)MG_OK;
  });
}

int mg_adapt_setup(void* ctx, int passes, int relax, int transfers, mg_setup_info* info) {
  mg::Range range("mg_adapt_setup");
  return guarded([&]() {
    const auto t0 = std::chrono::steady_clock::now();
    mg::Ctx* c = as_ctx(ctx);
    if (!c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
    if (passes < 1 || relax < 1 || transfers < 0) mg::raise(MG_ERR_ARG, "passes and relax must be positive");
    const int nt = transfers == 0 ? c->params.levels - 1 : std::min(transfers, c->params.levels - 1);
    // every pass refines the transfers from the finest down; after each, the
    // coarser transfers are set up afresh (inverse iteration) on the refined
    // coarse operator, whose near-null space their old vectors no longer span
    for (int p = 0; p < passes; p++)
      for (int l = 0; l < nt; l++) {
        mg::mg_relax_null_vectors(c, l, relax);
        std::vector<std::vector<double>> vecs = current_vectors(c);
        vecs.resize(l + 1);
        rebuild_from(c, vecs, info);
      }
    if (info)
      info->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return (int)MG_OK;
  });
}

int mg_update_mass(void* ctx, double m0, mg_setup_info* info) {
  return guarded([&]() {
    const auto t0 = std::chrono::steady_clock::now();
    mg::Ctx* c = as_ctx(ctx);
    if (!c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
    if (!std::isfinite(m0)) mg::raise(MG_ERR_ARG, "non-finite m0");
    std::vector<std::vector<double>> vecs = current_vectors(c);
    const double w[4] = {c->g.w[0], c->g.w[1], c->g.w[2], c->g.w[3]};
    const int st = mg_set_clover_aniso(ctx, w, c->csw, c->csw_t, m0);
    if (st != MG_OK) return st;
    rebuild_from(c, vecs, info);
    if (info)
      info->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return (int)MG_OK;
  });
}

int mg_get_coarse_links(void* ctx, int level, void* Y, void* X, int where) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    check_where(where);
    if (!Y || !X) mg::raise(MG_ERR_ARG, "null buffer");
    if (!c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
    if (level < 1 || level >= c->params.levels) mg::raise(MG_ERR_ARG, "level must be a coarse level");
    int ndof = 0;
    const size_t sites = level_vec_complex(c, level, &ndof) / ndof;
    const size_t ybytes = sizeof(double) * 2 * sites * 8 * ndof * ndof;
    const size_t xbytes = sizeof(double) * 2 * sites * ndof * ndof;
    Staged sy, sx;
    stage_out_alloc(sy, Y, ybytes, where);
    stage_out_alloc(sx, X, xbytes, where);
    mg::mg_get_links(c, level, sy.ptr, sx.ptr);
    if (where == MG_HOST) MG_CUDA(cudaMemcpyAsync(Y, sy.ptr, ybytes, cudaMemcpyDeviceToHost, c->stream));
    stage_out_finish(c, sx, X, xbytes, where);
    return MG_OK;
  });
}

int mg_solve(void* ctx, void* psi, const void* eta, int nrhs, double tol, int mode, int where, mg_solve_info* info) {
  mg::Range range("mg_solve");
  return guarded([&]() { return solve_impl(ctx, psi, eta, nrhs, tol, mode, where, info, false); });
}

int mg_solve_dagger(void* ctx, void* psi, const void* eta, int nrhs, double tol, int mode, int where,
                    mg_solve_info* info) {
  return guarded([&]() { return solve_impl(ctx, psi, eta, nrhs, tol, mode, where, info, true); });
}

int mg_solve_batch(void* const* ctxs, int nctx, void* const* psi, const void* const* eta, const int* nrhs, double tol,
                   int where, mg_solve_info* infos) {
  mg::Range range("mg_solve_batch");
  return guarded([&]() {
    const auto t0 = std::chrono::steady_clock::now();
    check_where(where);
    if (!ctxs || !psi || !eta || !nrhs || nctx < 1 || !(tol > 0)) mg::raise(MG_ERR_ARG, "bad batch arguments");
    std::vector<mg::Ctx*> cs(nctx);
    for (int i = 0; i < nctx; i++) {
      cs[i] = as_ctx(ctxs[i]);
      if (!psi[i] || !eta[i] || nrhs[i] < 1) mg::raise(MG_ERR_ARG, "bad batch arguments");
      if (!cs[i]->have_clover || !cs[i]->mg) mg::raise(MG_ERR_STATE, "every context needs gauge, clover and mg_setup");
      if (cs[i]->device != cs[0]->device) mg::raise(MG_ERR_ARG, "contexts of one batch must share a device");
      for (int j = 0; j < i; j++)
        if (cs[j] == cs[i]) mg::raise(MG_ERR_ARG, "a context appears twice in the batch");
    }
    MG_CUDA(cudaSetDevice(cs[0]->device));
    const long long kernels0 = mg::launches_so_far();
    std::vector<Staged> si(nctx), so(nctx);
    std::vector<mg_solve_info> loc(nctx);
    for (int i = 0; i < nctx; i++) {
      mg::Ctx* c = cs[i];
      const size_t bytes = sizeof(double) * 24 * c->V * nrhs[i];
      stage_in(c, si[i], eta[i], bytes, where);
      stage_out_alloc(so[i], psi[i], bytes, where);
      std::memset(&loc[i], 0, sizeof(mg_solve_info));
      mg::mg_reset_counters(c);
    }
    // groups of right-hand sides (in context order) that one persistent launch can hold
    const int cap = std::min(16, std::max(1, cs[0]->params.rhs_block));
    int status = MG_OK;
    std::vector<mg::BlockPart> parts;
    int used = 0;
    auto flush = [&]() {
      if (parts.empty()) return;
      const int st = mg::solve_multi_block(parts, tol);
      if (st != MG_OK) status = st;
      parts.clear();
      used = 0;
    };
    for (int i = 0; i < nctx; i++) {
      int q = 0;
      // a context's right-hand sides stay in one group when they fit in a fresh one
      if (used > 0 && used + nrhs[i] > cap && nrhs[i] <= cap) flush();
      while (q < nrhs[i]) {
        const int take = std::min(nrhs[i] - q, cap - used);
        mg::Ctx* c = cs[i];
        parts.push_back(mg::BlockPart{c, take, si[i].ptr + (size_t)q * 24 * c->V, so[i].ptr + (size_t)q * 24 * c->V,
                                      &loc[i]});
        used += take;
        q += take;
        if (used == cap) flush();
      }
    }
    flush();
    for (int i = 0; i < nctx; i++) {
      mg::Ctx* c = cs[i];
      stage_out_finish(c, so[i], psi[i], sizeof(double) * 24 * c->V * nrhs[i], where);
      mg::mg_read_counters(c, loc[i].coarse_iterations);
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < nctx; i++) {
      loc[i].solve_ms = ms;
      loc[i].kernel_launches = mg::launches_so_far() - kernels0;
      if (infos) infos[i] = loc[i];
    }
    return status;
  });
}

int mg_force(void* ctx, void* F, const void* lambda, const void* psi, int kind, int where) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    check_where(where);
    if (!F || !lambda || !psi) mg::raise(MG_ERR_ARG, "null buffer");
    const int base = kind & ~MG_FORCE_FP32;
    if (base != MG_FORCE_SU3 && base != MG_FORCE_WIRTINGER) mg::raise(MG_ERR_ARG, "bad force kind");
    if (!c->have_clover) mg::raise(MG_ERR_STATE, "set the gauge field and clover first");
    const size_t vbytes = sizeof(double) * 24 * c->V, fbytes = sizeof(double) * 72 * c->V;
    Staged sl, sp, so;
    stage_in(c, sl, lambda, vbytes, where);
    stage_in(c, sp, psi, vbytes, where);
    stage_out_alloc(so, F, fbytes, where);
    mg::gauge_force(c, so.ptr, sl.ptr, sp.ptr, kind);
    stage_out_finish(c, so, F, fbytes, where);
    return MG_OK;
  });
}

int mg_apply(void* ctx, int op, int level, void* out, const void* in, int nrhs, int prec, int where) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    check_where(where);
    if (!out || !in || nrhs < 1) mg::raise(MG_ERR_ARG, "bad apply arguments");
    if (prec != MG_FP64 && prec != MG_FP32) mg::raise(MG_ERR_ARG, "bad precision");
    if (op < MG_OP_D || op > MG_OP_DR_DAG) mg::raise(MG_ERR_ARG, "bad operator");
    if (!c->have_clover) mg::raise(MG_ERR_STATE, "set the gauge field and clover first");
    if (level < 0 || level >= c->params.levels) mg::raise(MG_ERR_ARG, "level out of range");
    if (op == MG_OP_DR_DAG && level != 0) mg::raise(MG_ERR_ARG, "D_r^dag is a fine-level operator");
    if ((level > 0 || op == MG_OP_R || op == MG_OP_P || op == MG_OP_CYCLE) && !c->mg) mg::raise(MG_ERR_STATE, "run mg_setup first");
    if (op == MG_OP_CYCLE && level + 1 >= c->params.levels) mg::raise(MG_ERR_ARG, "no coarser level to cycle to");
    int ndof_in, ndof_out;
    const int lin = op == MG_OP_P ? level + 1 : level;
    const int lout = op == MG_OP_R ? level + 1 : level;
    if ((op == MG_OP_R || op == MG_OP_P) && level + 1 >= c->params.levels) mg::raise(MG_ERR_ARG, "no transfer");
    const size_t nin = level_vec_complex(c, lin, &ndof_in), nout = level_vec_complex(c, lout, &ndof_out);
    Staged si, so;
    stage_in(c, si, in, sizeof(double) * 2 * nin * nrhs, where);
    stage_out_alloc(so, out, sizeof(double) * 2 * nout * nrhs, where);
    if (op == MG_OP_CYCLE && level == 0 && nrhs > 1) {
      mg::mg_cycle_batch(c, so.ptr, si.ptr, nrhs);   // all rhs through the batched cycle
    } else if (level > 0 || op == MG_OP_R || op == MG_OP_P || op == MG_OP_CYCLE) {
      for (int r = 0; r < nrhs; r++)
        mg::mg_apply_level(c, op, level, so.ptr + (size_t)r * 2 * nout, si.ptr + (size_t)r * 2 * nin);
    } else {
      // fine level: all right-hand sides in one launch per kernel, as packed
      // half vectors [even halves of every rhs][odd halves of every rhs]
      const bool f32 = prec == MG_FP32;
      const size_t es = f32 ? sizeof(float) : sizeof(double);
      const size_t half = 24 * c->Vh;  // reals per half vector
      mg::DBuf ib(es * 2 * half * nrhs), ob(es * 2 * half * nrhs);
      MG_CUDA(cudaMemsetAsync(ob.get(), 0, es * 2 * half * nrhs, c->stream));
      char* ie = ib.as<char>();
      char* io = ie + es * half * nrhs;
      char* oe = ob.as<char>();
      char* oo = oe + es * half * nrhs;
      for (int r = 0; r < nrhs; r++)
        mg::pack_spinor(c->g, si.ptr + (size_t)r * 2 * nin, ie + es * half * r, io + es * half * r, f32, c->stream);
      auto run = [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        mg::FineOps<T> F(c);
        T *ie_ = (T*)ie, *io_ = (T*)io, *oe_ = (T*)oe, *oo_ = (T*)oo;
        if (op == MG_OP_DR_DAG) {
          mg::DBuf tmp(sizeof(T) * half);
          for (int r = 0; r < nrhs; r++) mg::dr_dagger<T>(c, F, oe_ + half * r, ie_ + half * r, tmp.as<T>());
          return;
        }
        if (nrhs == 1) {
          switch (op) {
            case MG_OP_D: F.D(oe_, oo_, ie_, io_); break;
            case MG_OP_DP: F.Dp(oe_, oo_, ie_, io_); break;
            case MG_OP_DR: F.Dr(oe_, ie_); break;
            case MG_OP_BR: F.br(oe_, ie_, io_); break;
            case MG_OP_M: F.M(oe_, oo_, ie_, io_, false); break;
            case MG_OP_MINV: F.M(oe_, oo_, ie_, io_, true); break;
            case MG_OP_HOP: F.H(oe_, oo_, ie_, io_); break;
            default: mg::raise(MG_ERR_ARG, "bad operator");
          }
          return;
        }
        switch (op) {
          case MG_OP_D: F.D_multi(oe_, oo_, ie_, io_, nrhs, half); break;
          case MG_OP_DP: F.Dp_multi(oe_, oo_, ie_, io_, nrhs, half); break;
          case MG_OP_DR: F.Dr_multi(oe_, ie_, nrhs, half); break;
          case MG_OP_BR: F.br_multi(oe_, ie_, io_, nrhs, half); break;
          case MG_OP_M: F.M_multi(oe_, oo_, ie_, io_, false, nrhs, half); break;
          case MG_OP_MINV: F.M_multi(oe_, oo_, ie_, io_, true, nrhs, half); break;
          case MG_OP_HOP: F.H_multi(oe_, oo_, ie_, io_, nrhs, half); break;
          default: mg::raise(MG_ERR_ARG, "bad operator");
        }
      };
      if (f32)
        run((float*)nullptr);
      else
        run((double*)nullptr);
      for (int r = 0; r < nrhs; r++)
        mg::unpack_spinor(c->g, oe + es * half * r, oo + es * half * r, f32, so.ptr + (size_t)r * 2 * nout, c->stream);
      c->sync();
    }
    stage_out_finish(c, so, out, sizeof(double) * 2 * nout * nrhs, where);
    return MG_OK;
  });
}

int mg_benchmark_fma(int device, int prec, double* tflops) {
  return guarded([&]() {
    if (!tflops || (prec != MG_FP64 && prec != MG_FP32)) mg::raise(MG_ERR_ARG, "bad FMA benchmark arguments");
    MG_CUDA(cudaSetDevice(device));
    *tflops = mg::fma_peak_tflops(prec);
    return MG_OK;
  });
}

int mg_benchmark_coarse_solve(void* ctx, int warmup, int iters, double* avg_ms, double* bytes_per_solve,
                              double* iterations_per_solve) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!avg_ms || !bytes_per_solve || !iterations_per_solve || iters < 1 || warmup < 0)
      mg::raise(MG_ERR_ARG, "bad benchmark arguments");
    mg::mg_benchmark_coarse_solve(c, warmup, iters, avg_ms, bytes_per_solve, iterations_per_solve);
    return MG_OK;
  });
}

int mg_benchmark_coarse_floor(void* ctx, double* barrier_us, double* stream_us, double* stream_bytes, int* grid) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!barrier_us || !stream_us || !stream_bytes || !grid) mg::raise(MG_ERR_ARG, "bad benchmark arguments");
    mg::mg_benchmark_coarse_floor(c, barrier_us, stream_us, stream_bytes, grid);
    return MG_OK;
  });
}

int mg_benchmark_kernel(void* ctx, int kernel, int prec, int warmup, int iters, double* avg_ms,
                        double* bytes_per_launch) {
  return mg_benchmark_kernel_nrhs(ctx, kernel, prec, 1, warmup, iters, avg_ms, bytes_per_launch);
}

int mg_benchmark_kernel_nrhs(void* ctx, int kernel, int prec, int nrhs, int warmup, int iters, double* avg_ms,
                             double* bytes_per_launch) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!avg_ms || !bytes_per_launch || iters < 1 || warmup < 0 || nrhs < 1) mg::raise(MG_ERR_ARG, "bad benchmark arguments");
    if (prec != MG_FP64 && prec != MG_FP32) mg::raise(MG_ERR_ARG, "bad precision");
    if (!c->have_clover) mg::raise(MG_ERR_STATE, "set the gauge field and clover first");
    if (kernel == MG_KERNEL_COARSE_DR) {
      if (nrhs != 1) mg::raise(MG_ERR_ARG, "the coarse benchmark takes one right-hand side");
      mg::mg_benchmark_coarse(c, warmup, iters, avg_ms, bytes_per_launch);
      return MG_OK;
    }
    if (kernel == MG_KERNEL_RESTRICT || kernel == MG_KERNEL_PROLONG) {
      mg::mg_benchmark_transfer(c, kernel == MG_KERNEL_RESTRICT, nrhs, warmup, iters, avg_ms, bytes_per_launch);
      return MG_OK;
    }
    if (kernel < MG_KERNEL_DSLASH_CLOVER || kernel > MG_KERNEL_DR) mg::raise(MG_ERR_ARG, "bad kernel");
    const bool f32 = prec == MG_FP32;
    const size_t half_reals = 24 * c->Vh;
    mg::DBuf a32(sizeof(float) * 2 * half_reals);
    mg::philox_fine_vector(c->g, 12345, 0, 0, a32.as<float>(), a32.as<float>() + half_reals, c->stream);
    cudaEvent_t e0, e1;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    double ms = 0, bytes = 0;
    auto run = [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      const size_t hn = half_reals * nrhs;
      mg::DBuf in(sizeof(T) * hn), x(sizeof(T) * hn), out(sizeof(T) * hn);
      for (int q = 0; q < nrhs; q++) {
        mg::blas_convert<float, T>(in.as<T>() + q * half_reals, a32.as<float>(), half_reals / 2, c->stream);
        mg::blas_convert<float, T>(x.as<T>() + q * half_reals, a32.as<float>() + half_reals, half_reals / 2, c->stream);
      }
      mg::FineOps<T> F(c);
      const mg::Geom& g = c->g;
      int blk_ch = 0, blk_xp = 0;
      if (nrhs > 1) {   // the autotuned CTA sizes the solver would use
        auto kch = [&](int b) {
          mg::dslash_mrhs<T>(g, mg::EPI_CH, 1, nrhs, half_reals, out.as<T>(), in.as<T>(), c->gauge<T>(), c->Ainv<T>(1),
                             nullptr, 0.0, 0xff, b, c->stream);
        };
        auto kxp = [&](int b) {
          mg::dslash_mrhs<T>(g, mg::EPI_XPAY, 0, nrhs, half_reals, out.as<T>(), in.as<T>(), c->gauge<T>(), nullptr,
                             x.as<T>(), -1.0, 0xff, b, c->stream);
        };
        blk_ch = F.block_for("dslash_ch", nrhs, kch);
        blk_xp = F.block_for("dslash_xpay", nrhs, kxp);
      }
      auto launch = [&]() {
        switch (kernel) {
          case MG_KERNEL_DSLASH_CLOVER:
            if (nrhs == 1)
              mg::dslash<T>(g, mg::EPI_CH, 1, out.as<T>(), in.as<T>(), c->gauge<T>(), c->Ainv<T>(1), nullptr, 0.0,
                            0xff, c->stream);
            else
              mg::dslash_mrhs<T>(g, mg::EPI_CH, 1, nrhs, half_reals, out.as<T>(), in.as<T>(), c->gauge<T>(),
                                 c->Ainv<T>(1), nullptr, 0.0, 0xff, blk_ch, c->stream);
            break;
          case MG_KERNEL_DSLASH_XPAY:
            if (nrhs == 1)
              mg::dslash<T>(g, mg::EPI_XPAY, 0, out.as<T>(), in.as<T>(), c->gauge<T>(), nullptr, x.as<T>(), -1.0,
                            0xff, c->stream);
            else
              mg::dslash_mrhs<T>(g, mg::EPI_XPAY, 0, nrhs, half_reals, out.as<T>(), in.as<T>(), c->gauge<T>(),
                                 nullptr, x.as<T>(), -1.0, 0xff, blk_xp, c->stream);
            break;
          default:
            if (nrhs == 1)
              F.Dr(out.as<T>(), in.as<T>());
            else
              F.Dr_multi(out.as<T>(), in.as<T>(), nrhs, half_reals);
            break;
        }
      };
      for (int w = 0; w < warmup; w++) launch();
      MG_CUDA(cudaEventRecord(e0, c->stream));
      for (int it = 0; it < iters; it++) launch();
      MG_CUDA(cudaEventRecord(e1, c->stream));
      MG_CUDA(cudaEventSynchronize(e1));
      float t = 0;
      MG_CUDA(cudaEventElapsedTime(&t, e0, e1));
      ms = t / iters;
      // reals per output site: links and clover once, spinors once per rhs
      double reals;
      if (kernel == MG_KERNEL_DSLASH_CLOVER)
        reals = 144.0 + 72.0 + 48.0 * nrhs;
      else if (kernel == MG_KERNEL_DSLASH_XPAY)
        reals = 144.0 + 72.0 * nrhs;
      else
        reals = 432.0 + 168.0 * nrhs;
      bytes = reals * sizeof(T) * (double)c->Vh;
    };
    if (f32)
      run((float*)nullptr);
    else
      run((double*)nullptr);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *avg_ms = ms;
    *bytes_per_launch = bytes;
    return MG_OK;
  });
}

int mg_level_info(void* ctx, int level, int dims_out[4], int* ndof_out) {
  return guarded([&]() {
    mg::Ctx* c = as_ctx(ctx);
    if (!dims_out || !ndof_out) mg::raise(MG_ERR_ARG, "null output");
    if (level < 0 || level >= c->params.levels) mg::raise(MG_ERR_ARG, "level out of range");
    int d[4] = {c->dims[0], c->dims[1], c->dims[2], c->dims[3]};
    int ndof = 12;
    for (int l = 0; l < level; l++) {
      for (int m = 0; m < 4; m++) d[m] /= c->params.block[l][m];
      ndof = 2 * c->params.nv[l];
    }
    for (int m = 0; m < 4; m++) dims_out[m] = d[m];
    *ndof_out = ndof;
    return MG_OK;
  });
}

}  // extern "C"
