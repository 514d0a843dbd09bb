// Host-side internals of libmgclover: the context, device workspace, error
// handling and the kernel launchers each translation unit provides.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <complex>
#include <functional>
#include <initializer_list>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "mgclover.h"

namespace mg {

// An NVTX range for the duration of a scope (setup, solve, outer iteration,
// level cycle, coarse solve); free when no tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
struct Ctx;
// With mg_params.level_timing on, records a CUDA event pair on the context
// stream around its scope into the level's list (level_times() sums them).
struct LevelTime {
  LevelTime(Ctx* c, int level);
  ~LevelTime();
  Ctx* c;
  int level;
  int slot = -1;
};
// sums and clears the recorded pairs of every level (synchronises the stream)
void level_times(Ctx* c, double out_ms[MG_MAX_LEVELS]);
void level_times_reset(Ctx* c);
// "<what> level <l>" for l < MG_MAX_LEVELS (static strings)
const char* level_range_name(int what, int l);
enum { RANGE_CYCLE = 0, RANGE_COARSE_SOLVE = 1, RANGE_NULL_VECTORS = 2, RANGE_COARSE_LINKS = 3 };


// --------------------------------------------------------------------------- errors
struct Error {
  int code;
  std::string what;
};

[[noreturn]] void raise(int code, const std::string& what);
void cuda_check(cudaError_t e, const char* expr, const char* file, int line);
// counts one kernel launch and checks its launch error (configuration errors
// only; no sync)
void launch_check(const char* file, int line);
long long launches_so_far();
// adjusts the launch count (kernels a CUDA-graph replay runs, or captured ones that did not run)
void add_launches(long long n);
#define MG_CUDA(expr) ::mg::cuda_check((expr), #expr, __FILE__, __LINE__)
#define MG_LAUNCH() ::mg::launch_check(__FILE__, __LINE__)

// --------------------------------------------------------------------------- device memory
// Owning device allocation (cudaMalloc / cudaFree).
class DBuf {
 public:
  DBuf() = default;
  explicit DBuf(size_t bytes) { alloc(bytes); }
  ~DBuf() { release(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p_(o.p_), bytes_(o.bytes_) { o.p_ = nullptr; o.bytes_ = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p_ = o.p_; bytes_ = o.bytes_; o.p_ = nullptr; o.bytes_ = 0; }
    return *this;
  }
  void alloc(size_t bytes);
  void release();
  template <typename T>
  T* as() const { return static_cast<T*>(p_); }
  void* get() const { return p_; }
  size_t bytes() const { return bytes_; }

 private:
  void* p_ = nullptr;
  size_t bytes_ = 0;
};

// --------------------------------------------------------------------------- workspace
// Reduction scratch, device scalars and error flags shared by all kernels of
// one context.  Reductions are deterministic: fixed grid, per-block FP64
// partials, then an ordered sum by the last block to finish.
struct Workspace {
  static constexpr int kMaxBlocks = 608;       // 4 x 152 SMs
  static constexpr int kMaxResults = 136;      // doubles per reduction
  static constexpr int kScalars = 16384;       // device scalar pool (doubles)
  DBuf partials;                               // [kMaxBlocks][kMaxResults]
  DBuf counter;                                // unsigned, self-resetting
  DBuf scalars;                                // doubles
  DBuf flags;                                  // int[16]
  static constexpr int kMultiCounters = 64;    // separate reductions in one launch (multi-RHS)
  DBuf mcounters;                              // unsigned[kMultiCounters], self-resetting
  double* host = nullptr;                      // pinned mirror of the first scalars
  void init();
  ~Workspace();
};

enum Flag { FLAG_SINGULAR = 0, FLAG_GS_BREAKDOWN = 1, FLAG_NAN = 2, FLAG_TIMEOUT = 3, FLAG_COUNT = 16 };

// --------------------------------------------------------------------------- fine level
// dslash epilogues: out = f(H in), H the hopping term including its -1/2
enum Epilogue { EPI_H = 0, EPI_CH = 1, EPI_XPAY = 2, EPI_CX_PAY = 3, EPI_C_XPAY = 4 };
//  EPI_H:      out = H in
//  EPI_CH:     out = C (H in)
//  EPI_XPAY:   out = x + a H in
//  EPI_CX_PAY: out = C x + a H in
//  EPI_C_XPAY: out = C (x + a H in)

void pack_spinor(const Geom& g, const double* abi, void* even, void* odd, bool fp32, cudaStream_t s);
void unpack_spinor(const Geom& g, const void* even, const void* odd, bool fp32, double* abi, cudaStream_t s);
void pack_gauge(const Geom& g, const double* abi, double* g64, float* g32, cudaStream_t s);
// clover coefficients of the spatial planes and of the planes that contain t
struct CloverCoef {
  double csw_s, csw_t;
};
void build_clover(const Geom& g, const double* g64, CloverCoef cf, double m0, double* A64, double* Ainv64,
                  float* A32, float* Ainv32, int* flags, cudaStream_t s);
template <typename T>
void clover_apply(const Geom& g, T* out, const T* in, const T* clov, cudaStream_t s);
template <typename T>
void dslash(const Geom& g, Epilogue epi, int parity, T* out, const T* in, const T* gauge, const T* clov,
            const T* x, double a, int dirmask, cudaStream_t s);
// nrhs right-hand sides at `stride` elements of T apart (out, in and x alike),
// one launch; `config` = (right-hand sides per thread) * 1000 + CTA size, one
// of dslash_mrhs_configs()
template <typename T>
void dslash_mrhs(const Geom& g, Epilogue epi, int parity, int nrhs, size_t stride, T* out, const T* in,
                 const T* gauge, const T* clov, const T* x, double a, int dirmask, int config, cudaStream_t s);
std::vector<int> dslash_mrhs_configs(bool fp32);
int dslash_mrhs_default(bool fp32);
template <typename T>
void clover_apply_mrhs(const Geom& g, int nrhs, size_t stride, T* out, const T* in, const T* clov, cudaStream_t s);
// the 8 directional terms H_d in (without summation), written to out[d]
// (whole-lattice FP32 vectors, [even half][odd half] each)
void hop_directions(const Geom& g, float* const out[8], const float* in_even, const float* in_odd,
                    const float* gauge, cudaStream_t s);
// Philox4x32-10 Gaussian start vector (see the generator's definition in coarse.cu)
void philox_fine_vector(const Geom& g, uint64_t seed, int level, int k, float* even, float* odd, cudaStream_t s);

// --------------------------------------------------------------------------- BLAS
// Vectors are flat arrays of n complex numbers of precision T.
template <typename T>
void blas_zero(T* x, size_t n, cudaStream_t s);
template <typename TI, typename TO>
void blas_convert(TO* y, const TI* x, size_t n, cudaStream_t s);
// y = a x + b y  (real a, b)
template <typename T>
void blas_axpby(double a, const T* x, double b, T* y, size_t n, cudaStream_t s);
// ||x||^2 -> d_out[0] (device)
template <typename T>
void blas_norm2(const T* x, size_t n, double* d_out, Workspace& ws, cudaStream_t s);
// <x, y> -> d_out[0..1] (device)
template <typename T>
void blas_cdot(const T* x, const T* y, size_t n, double* d_out, Workspace& ws, cudaStream_t s);
// d_out[2j..2j+1] = <V_j, w>, j < k (k <= 64)
template <typename T>
void blas_multidot(const T* const* V, int k, const T* w, size_t n, double* d_out, Workspace& ws, cudaStream_t s);
// w -= sum_j beta_j V_j (beta device complex, k may be 0), then
// d_out = {||w||^2, Re<w,r>, Im<w,r>}
template <typename T>
void blas_orth_update(T* w, const T* const* V, const double* d_beta, int k, const T* r, size_t n, double* d_out,
                      Workspace& ws, cudaStream_t s);
// gamma = sqrt(d_in[0]); alpha = (d_in[1] + i d_in[2]) / gamma; w /= gamma;
// r -= alpha w; stores alpha (2 doubles), gamma; d_rnorm2 = ||r||^2
template <typename T>
void blas_r_update(T* w, T* r, size_t n, const double* d_in, double* d_alpha, double* d_gamma, double* d_rnorm2,
                   Workspace& ws, cudaStream_t s);
// x += scale * sum_j c_j Z_j (c device complex)
template <typename T, typename TZ>
void blas_lincomb(T* x, const TZ* const* Z, const double* d_c, int k, double scale, size_t n, cudaStream_t s);
// GCR back substitution: c_j = (alpha_j - sum_{l>j} beta_{j,l} c_l) / gamma_j,
// beta column-major with leading dimension ld: beta[(j + ld*l)*2 + {re,im}]
void gcr_backsub(const double* d_beta, int ld, const double* d_alpha, const double* d_gamma, int k, double* d_c,
                 cudaStream_t s);
// minimal-residual step: alpha = <w,r>/<w,w> from d_in = {<w,w>, Re<w,r>, Im<w,r>};
// e += alpha r; r -= alpha w
template <typename T>
void blas_mr_update(T* e, T* r, const T* w, const double* d_in, size_t n, cudaStream_t s);
// x *= 1/sqrt(d_norm2[0])
template <typename T>
void blas_normalize(T* x, const double* d_norm2, size_t n, cudaStream_t s);
// {<w,w>, Re<w,r>, Im<w,r>} -> d_out
template <typename T>
void blas_dot2(const T* w, const T* r, size_t n, double* d_out, Workspace& ws, cudaStream_t s);
// the same for nrhs pairs at `stride` reals apart: d_out[4q .. 4q+2] (one launch)
template <typename T>
void blas_dot2_multi(const T* w, const T* r, size_t n, size_t stride, int nrhs, double* d_out, Workspace& ws,
                     cudaStream_t s);
// blas_mr_update for nrhs triples at `stride` reals apart with d_in[4q ..] (one launch)
template <typename T>
void blas_mr_update_multi(T* e, T* r, const T* w, const double* d_in, size_t n, size_t stride, int nrhs,
                          cudaStream_t s);

// --------------------------------------------------------------------------- autotuner (tune.cu)
struct TuneKey {
  const char* kernel;
  int dims[4];
  int nrhs;
  int prec;   // 0 FP64, 1 FP32
};
// CTA size for `k`: looked up, or chosen by timing `launch(block)` for every
// candidate on stream `s` (the launches must be idempotent: no output aliases
// an input).  Thread-safe.
int tuned_block(const TuneKey& k, const std::vector<int>& candidates, const std::function<void(int)>& launch,
                cudaStream_t s);
int tune_entries();

// --------------------------------------------------------------------------- context
struct Level;     // multigrid level (coarse.cu / multigrid.cu)
struct Hierarchy;

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Geom g{};
  int dims[4] = {0, 0, 0, 0};
  size_t V = 0, Vh = 0;
  Workspace ws;

  // fields (internal layouts, see common.cuh)
  DBuf gauge64, gauge32;                 // [2][4][9][Vh] complex
  DBuf clov64, clovinv64;                // [2][72 Vh] doubles
  DBuf clov32, clovinv32;                // [2][72 Vh] floats
  bool have_gauge = false, have_clover = false;
  double csw = 0, m0 = 0;
  double csw_t = 0;                      // clover coefficient of the planes that contain t (= csw when isotropic)
  bool anisotropic() const { return g.w[0] != 1.0 || g.w[1] != 1.0 || g.w[2] != 1.0 || g.w[3] != 1.0 || csw_t != csw; }

  mg_params params{};
  bool have_params = false;
  std::shared_ptr<Hierarchy> mg;         // null until mg_setup (shared_ptr: Hierarchy is incomplete here)
  std::vector<std::vector<double>> injected;  // per transfer: injected raw null vectors (host, complex128)
  std::vector<int> injected_nv;

  // host I/O staging
  DBuf stage_in, stage_out;              // complex128 whole-lattice staging
  long long dslash_launches = 0;
  // mg_params.level_timing: CUDA event pairs around each level's work, per level
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> level_events[MG_MAX_LEVELS];
  int level_events_used[MG_MAX_LEVELS] = {0, 0, 0, 0};
  ~Ctx() {
    for (auto& v : level_events)
      for (auto& e : v) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
  }
  std::shared_ptr<void> solve_work;      // solve buffers (solver.cu), kept between calls
  std::shared_ptr<void> block_work;      // block-solve buffers (block.cu), kept between calls

  const double* A64(int p) const { return clov64.as<double>() + (size_t)p * 72 * Vh; }
  const double* Ainv64(int p) const { return clovinv64.as<double>() + (size_t)p * 72 * Vh; }
  const float* A32(int p) const { return clov32.as<float>() + (size_t)p * 72 * Vh; }
  const float* Ainv32(int p) const { return clovinv32.as<float>() + (size_t)p * 72 * Vh; }
  template <typename T>
  const T* gauge() const;
  template <typename T>
  const T* A(int p) const;
  template <typename T>
  const T* Ainv(int p) const;

  void sync();
  double read_scalar(const double* d);            // sync + copy one double
  void read_scalars(const double* d, double* h, int n);
  int read_flag(int which, bool clear);
};

template <>
inline const double* Ctx::gauge<double>() const { return gauge64.as<double>(); }
template <>
inline const float* Ctx::gauge<float>() const { return gauge32.as<float>(); }
template <>
inline const double* Ctx::A<double>(int p) const { return A64(p); }
template <>
inline const float* Ctx::A<float>(int p) const { return A32(p); }
template <>
inline const double* Ctx::Ainv<double>(int p) const { return Ainv64(p); }
template <>
inline const float* Ctx::Ainv<float>(int p) const { return Ainv32(p); }

// --------------------------------------------------------------------------- fine operators
// Even-odd operators of the fine level in precision T on half-lattice vectors
// (12 Vh complex).  Temporaries are owned by the object.
template <typename T>
struct FineOps {
  Ctx* c;
  DBuf t1, t2;
  explicit FineOps(Ctx* ctx);
  size_t half_n() const { return 12 * c->Vh; }
  // D_r y = y - H_eo A_o^{-1} H_oe A_e^{-1} y
  void Dr(T* out_e, const T* in_e);
  // b_r = b_e - H_eo A_o^{-1} b_o
  void br(T* out_e, const T* b_e, const T* b_o);
  // x_e = A_e^{-1} y_e, x_o = A_o^{-1}(b_o - H_oe x_e)
  void reconstruct(T* x_e, T* x_o, const T* y_e, const T* b_o);
  // full-lattice D, D_p, H, M, M^{-1}
  void D(T* oe, T* oo, const T* ie, const T* io);
  void Dp(T* oe, T* oo, const T* ie, const T* io);
  void H(T* oe, T* oo, const T* ie, const T* io);
  void M(T* oe, T* oo, const T* ie, const T* io, bool inverse);
  // nrhs vectors as packed half vectors: rhs r of a half at base + r * stride
  // with stride = 24 Vh elements of T (the even halves of all rhs, and
  // separately the odd halves, are contiguous).
  // Multi-RHS kernels: links and clover are read once per site for all rhs.
  DBuf m1, m2;
  size_t mcap = 0;
  void reserve_multi(int nrhs);
  int block_for(const char* kernel, int nrhs, const std::function<void(int)>& launch);
  void Dr_multi(T* out_e, const T* in_e, int nrhs, size_t stride);
  void br_multi(T* out_e, const T* b_e, const T* b_o, int nrhs, size_t stride);
  void reconstruct_multi(T* x_e, T* x_o, const T* y_e, const T* b_o, int nrhs, size_t stride);
  void D_multi(T* oe, T* oo, const T* ie, const T* io, int nrhs, size_t stride);
  void Dp_multi(T* oe, T* oo, const T* ie, const T* io, int nrhs, size_t stride);
  void H_multi(T* oe, T* oo, const T* ie, const T* io, int nrhs, size_t stride);
  void M_multi(T* oe, T* oo, const T* ie, const T* io, bool inverse, int nrhs, size_t stride);
};

// --------------------------------------------------------------------------- GCR
// Flexible GCR(m) with deferred solution update (see solver.cu).
template <typename T, typename TZ>
class GCR {
 public:
  using Op = std::function<void(T* out, const T* in)>;
  using Pre = std::function<void(TZ* z, const T* r)>;
  using LowOp = std::function<void(T* out, const TZ* in)>;   // A applied to a preconditioner output
  struct Result {
    int iterations = 0;
    int restarts = 0;
    double rnorm = 0;
    bool converged = false;
  };
  GCR(Ctx* c, size_t n, int m);
  // Solves A x = b.  x0_zero: start from x = 0 (x is overwritten), else from x.
  // Checks ||r|| <= tol_abs after every iteration when check is true (one
  // host sync per iteration); with check false it runs exactly maxit
  // iterations without restarts and without host syncs.
  // Al (optional): the product A z of the Krylov directions inside a restart
  // cycle, from the preconditioner output z directly (e.g. in lower
  // precision); A itself still forms every true residual.
  Result solve(const Op& A, const Pre* M, T* x, const T* b, bool x0_zero, double tol_abs, int maxit, bool check,
               const LowOp* Al = nullptr);
  T* residual() { return r_.as<T>(); }

 private:
  Ctx* c_;
  size_t n_;
  int m_;
  std::vector<DBuf> W_, Z_;
  DBuf r_, tmp_;
  DBuf scal_;
  double* s_;  // device scalars: beta[m*m*2], alpha[m*2], gamma[m], c[m*2], misc
};

// --------------------------------------------------------------------------- comparison Krylov solvers (krylov.cu)
// D_r^dag in = gamma_5 A_e^{-1} D_r A_e gamma_5 in on even half vectors (tmp: one half vector)
template <typename T>
void dr_dagger(Ctx* c, FineOps<T>& F, T* out, const T* in, T* tmp);

// BiCGStab and CGNR on n complex unknowns; the iteration scalars go through
// the host (a few synchronisations per iteration)
template <typename T>
class Krylov {
 public:
  using Op = std::function<void(T* out, const T* in)>;
  struct Result {
    int iterations = 0;
    int restarts = 0;
    double rnorm = 0;
    bool converged = false;
  };
  Krylov(Ctx* c, size_t n);
  ~Krylov();
  Krylov(const Krylov&) = delete;
  Krylov& operator=(const Krylov&) = delete;
  // A x = b from x = 0 (x0_zero) or from x, until ||b - A x|| <= tol_abs
  // (recursive residual) or maxit iterations (two applications of A each)
  Result bicgstab(const Op& A, T* x, const T* b, bool x0_zero, double tol_abs, int maxit);
  // CG on A^dag A x = A^dag b until ||b - A x|| <= tol_abs or maxit
  // iterations (one application of A and one of A^dag each)
  Result cgnr(const Op& A, const Op& Adag, T* x, const T* b, bool x0_zero, double tol_abs, int maxit);

 private:
  const double* coefs(std::initializer_list<std::complex<double>> z);
  Ctx* c_;
  size_t n_;
  DBuf r_, rh_, p_, v_, s_, t_, q_;
  DBuf sc_, coef_;
  double* hcoef_ = nullptr;  // pinned staging of lincomb coefficients
};

// MR smoothing: e = MR_nu(A, r) from e = 0 (r is consumed as scratch)
// nu MR steps on the fine D_r in FP32 with the fused kernels of mr.cu: e = the
// correction (zeroed first), r the residual (updated), w, s, t scratch half
// vectors; d_scr receives the last step's inner products
void mr_smooth_fine(Ctx* c, float* e, float* r, float* w, float* s, float* t, int nu, double* d_scr);
template <typename T>
void mr_smooth(Ctx* c, const std::function<void(T*, const T*)>& A, T* e, T* r, T* w, size_t n, int nu,
               double* d_scr);

// --------------------------------------------------------------------------- solve drivers (solver.cu)
int solve_fine(Ctx* c, double* psi_abi, const double* eta_abi, double tol, int mode, mg_solve_info* info);
// nb right-hand sides (ABI vectors, consecutive) solved together by
// lock-step multigrid-preconditioned FGCR (block.cu)
int solve_fine_block(Ctx* c, double* psi_abi, const double* eta_abi, int nb, double tol, mg_solve_info* info);
// right-hand sides of several contexts (lattices) solved together, their
// coarsest-level solves sharing persistent launches (block.cu)
struct BlockPart {
  Ctx* c;
  int nb;
  const double* eta;   // nb ABI vectors on the device
  double* psi;
  mg_solve_info* info;
};
int solve_multi_block(const std::vector<BlockPart>& parts, double tol);

// --------------------------------------------------------------------------- gauge derivative (force.cu)
// gamma_5 in place on ABI fine vectors (`sites` sites of 12 complex128)
void gamma5_abi(double* v, size_t sites, cudaStream_t s);
// derivative of -Re<lam, D(U) psi> with respect to the links (ABI layouts;
// kind = MG_FORCE_SU3 or MG_FORCE_WIRTINGER), see force.cu
void gauge_force(Ctx* c, double* out_abi, const double* lam_abi, const double* psi_abi, int kind);

// --------------------------------------------------------------------------- multigrid (multigrid.cu)
void mg_build(Ctx* c, mg_setup_info* info);
void mg_destroy_hierarchy(Ctx* c);
// preconditioner of the fine D_r in FP32 (z_e, r_e half vectors)
void mg_precondition(Ctx* c, float* z_e, const float* r_e);
// the same from an FP64 residual through a captured CUDA graph (r32: FP32
// staging); false when graphs are off or unavailable (see multigrid.cu)
bool mg_precondition_graph(Ctx* c, float* z_e, const double* r_e, float* r32);
// solve parameters changed with the setup kept: drop what was captured with the old ones
void mg_solve_params_changed(Ctx* c);
// the same for nb right-hand sides (packed half vectors, stride 24 Vh floats)
void mg_precondition_batch(Ctx* c, float* z_e, const float* r_e, int nb);
// mg_precondition_batch in three steps around the coarsest solve, so that
// several contexts can share one coarsest launch (see multigrid.cu)
void mg_batch_pre(Ctx* c, float* z_e, const float* r_e, int nb);
void mg_batch_coarse(Ctx* c, int nb);
void mg_batch_post(Ctx* c, float* z_e, const float* r_e, int nb);
bool mg_batch_joinable(Ctx* c);
// MG_OP_CYCLE of level 0 for nb ABI vectors through mg_precondition_batch
void mg_cycle_batch(Ctx* c, double* out_abi, const double* in_abi, int nb);
void mg_apply_level(Ctx* c, int op, int level, double* out_abi, const double* in_abi);
void mg_get_vectors(Ctx* c, int level, double* V_abi, int nv);
// relaxes the null vectors of transfer `level` with the current solver (multigrid.cu)
void mg_relax_null_vectors(Ctx* c, int level, int relax);
// dequantised coarse links of level >= 1 (ABI layouts, see mg_get_coarse_links)
void mg_get_links(Ctx* c, int level, double* Y_abi, double* X_abi);
void mg_level_dims(Ctx* c, int level, int dims[4], int* ndof);
void mg_reset_counters(Ctx* c);
// times `iters` applications of the level-1 coarse D_hat_r (see mg_benchmark_kernel)
void mg_benchmark_coarse(Ctx* c, int warmup, int iters, double* avg_ms, double* bytes);
void mg_read_counters(Ctx* c, long long* coarse_iters);
// measured CUDA-core FMA throughput of the current GPU (peaks.cu), TFLOP/s
double fma_peak_tflops(int prec);
// times the level-0 restriction (restrict = true) or prolongation on the even
// sites for nrhs right-hand sides (see mg_benchmark_kernel_nrhs)
void mg_benchmark_transfer(Ctx* c, bool restrict, int nrhs, int warmup, int iters, double* avg_ms, double* bytes);
// floors of one coarsest-level GCR iteration (see mg_benchmark_coarse_floor)
void mg_benchmark_coarse_floor(Ctx* c, double* barrier_us, double* stream_us, double* stream_bytes, int* grid);
// times `iters` coarsest-level solves (see mg_benchmark_coarse_solve)
void mg_benchmark_coarse_solve(Ctx* c, int warmup, int iters, double* avg_ms, double* bytes, double* its);

}  // namespace mg
