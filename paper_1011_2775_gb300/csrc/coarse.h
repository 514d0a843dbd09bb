// Multigrid data structures and the launchers of coarse.cu.
//
// A level is a lattice with `ndof` complex components per site.  The fine
// level (Wilson, ndof = 12) stores vectors in the chunked even-odd layout of
// common.cuh; coarse levels store [site][ndof] complex FP32 with sites in
// even-odd order when every extent is even (lexicographic otherwise).  A
// site's "storage index" is parity * half + checkerboard index (even-odd
// levels) or its lexicographic index.
//
// Transfer l -> l+1 (prolongation P, restriction R = P^dag; sections
// "Adaptive multigrid" and "Red-black preconditioning"): P is stored per
// coarse site c and block-local fine site i as P[c][i][dof][k], k < Nv; the
// column of entry (c, i, dof, k) is coarse dof chir(dof) * Nv + k with
// chir(dof) = dof / (ndof/2) (the chirality split of the null vectors).
// Coarse links (Galerkin operator): Y[c][row][d][col] for the 8 hops
// d (d < 4: from c + mu, d >= 4: from c - mu) and X[c][row][col], Xinv.
#pragma once
#include <vector>

#include "internal.h"

namespace mg {

struct CoarseSystem;   // one coarse system of a batched solve (below)

// Storage format of prolongators / coarse links
enum Store { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2 };

struct LevelGeom {
  int L[4] = {0, 0, 0, 0};
  int nsites = 0;
  bool eo = false;     // even-odd ordering / preconditioning available
  int half = 0;        // nsites / 2 when eo
  int ndof = 0;
  bool wilson = false; // fine level (chunked layout)
  int Vh = 0;          // fine level: half volume (chunk stride)
  std::vector<int> lex_of;  // storage -> lexicographic
  std::vector<int> store_of;  // lexicographic -> storage
  DBuf d_nbr;          // coarse levels: int[nsites][8] neighbour storage indices
  DBuf d_lex_of;       // int[nsites]
  void init(const int dims[4], int ndof_, bool wilson_);
  int coord_to_store(const int c[4]) const;
  size_t vec_complex() const { return (size_t)nsites * ndof; }
};

struct FineAccess {
  int wilson;
  int Vh;
  int ndof;
};

struct TransferOp {
  int block[4] = {1, 1, 1, 1};
  int cdims[4] = {1, 1, 1, 1};
  int nv = 0, fine_ndof = 0, nb = 0, ncoarse = 0;
  int fine_half = 0;       // storage index < fine_half <=> even site (fine level even-odd)
  int store = STORE_F32;
  FineAccess fa{};
  DBuf blockmap;           // int[ncoarse][nb] fine storage index
  // The block-local indices of each block's even fine sites, in order
  // (int[ncoarse][nbe]); nbe = -1 when blocks differ in their number of even
  // sites, and the transfers restricted to even sites then scan the whole block.
  DBuf evenlist;
  int nbe = -1;
  int* flags = nullptr;    // the context's error flags (FLAG_TIMEOUT from the pipelined transfers)
  DBuf P;                  // [ncoarse][nb][fine_ndof][nv] in `store` format
  DBuf Pscale;             // float[ncoarse][2]: per (block, chirality) scale (1 for FP32)
};

struct CoarseOp {
  int nc = 0;
  int store = STORE_F32;
  DBuf Y;                  // [site][nc][8][nc] in `store` format
  DBuf Yscale;             // float[site][8]: per (site, direction) scale
  DBuf X, Xinv;            // [site][nc][nc] complex FP32
  // Links with the site inverses folded in, for the persistent coarsest solve:
  //  even-odd levels: A[o - half][nc][8][nc] = X_o^{-1} Y_d(o) X^{-1}(o + d) on odd
  //  sites, so that (X_o^{-1} Y_oe X_e^{-1} y)(o) = sum_d A_d(o) y(o + d);
  //  other levels: [site][nc][9][nc] = [Y_0 .. Y_7 | X], so D_hat v is one GEMV.
  // The folded links are products, built in FP32 from the stored (dequantised)
  // Y, so the persistent solve applies exactly the operator of Y and X.
  DBuf A;
};

// Quantises Y from FP32 to `store` (FP16 / BF16) with one scale per
// (site, direction) tile: the largest |Re|, |Im| of the tile, so that every
// stored value lies in [-1, 1].  X and X^{-1} stay FP32.  Runs before
// coarse_fold_links.
void quantize_links(const LevelGeom& G, CoarseOp& C, int store, cudaStream_t s);
// dequantised links in ABI order: Y_abi[lex][8][nc][nc], X_abi[lex][nc][nc] complex128
void coarse_links_abi(const LevelGeom& G, const CoarseOp& C, double* Y_abi, double* X_abi, cudaStream_t s);

// builds C.A from the stored Y, X, Xinv (see CoarseOp)
void coarse_fold_links(const LevelGeom& G, CoarseOp& C, cudaStream_t s);

// ---- transfer kernels (coarse.cu)
// out_c (coarse full vector) = R v; even_only: v's odd sites are taken as zero
void restrict_vec(const TransferOp& T, float* out_c, const float* v, bool even_only, cudaStream_t s);
// v = P in_c; even_only: only even sites of v are written
void prolong_vec(const TransferOp& T, float* v, const float* in_c, bool even_only, cudaStream_t s);
// the same for nrhs vectors (strides in floats), one launch
void restrict_vec_multi(const TransferOp& T, int nrhs, float* out_c, size_t cstride, const float* v, size_t vstride,
                        bool even_only, cudaStream_t s);
void prolong_vec_multi(const TransferOp& T, int nrhs, float* v, size_t vstride, const float* in_c, size_t cstride,
                       bool even_only, cudaStream_t s);
// p = column (chir, k) of P as a whole-lattice vector of the fine level
void extract_column(const TransferOp& T, float* p, int chir, int k, cudaStream_t s);
// Galerkin accumulation of one column: W[0..7] directional hops of u = M^{-1} p,
// W[8] the identity-slot vector; writes column `col` of Y (faces) and X.
void restrict9(const TransferOp& T, CoarseOp& C, const float* const W[9], int col, cudaStream_t s);

// ---- coarse stencil kernels
// out[s] = epi(sum_{d in mask} Y_d(s) in[nbr_d(s)]) for storage sites
// s in [s0, s1); epilogues as the fine dslash (EPI_*), C = X or Xinv.
void coarse_hop(const LevelGeom& G, const CoarseOp& C, Epilogue epi, bool use_inv, int s0, int s1, float* out,
                const float* in, const float* x, float a, int dirmask, cudaStream_t s);
// out[s] = C(s) in[s] (+ a x[s] if x) for s in [s0, s1)
void coarse_site_mul(const LevelGeom& G, const CoarseOp& C, bool use_inv, int s0, int s1, float* out, const float* in,
                     cudaStream_t s);
// Xinv = X^{-1} per site (FP64 Gauss-Jordan); sets FLAG_SINGULAR on a tiny pivot
void coarse_invert(const LevelGeom& G, CoarseOp& C, int* flags, cudaStream_t s);

// ---- the coarsest-level solve as one persistent cooperative kernel (coarse_gcr.cu)
struct CoarseGCRBuffers {
  int grid = 0;            // co-resident blocks of the cooperative launch
  int nsplit = 1;          // work items per site in the stencil phases (row split)
  DBuf r, y, br, tA, tB, W, Z, partials, scal;
  // batched solves (coarse_batch.cu; grown on demand)
  DBuf bx_r, bx_y, bx_br, bx_tB, bx_W, bx_Z, bx_part, bx_scal;
  // streamed solve (coarse_stream.cu; grown on demand): partial sums, the
  // Gram-Schmidt coefficients, grid-barrier counter and abort flag
  DBuf st_part, st_beta, st_sync;
  // tensor-core solve (coarse_tc.cu; grown on demand)
  DBuf tc_y, tc_r, tc_br, tc_s, tc_sy, tc_t, tc_tb, tc_W, tc_Z, tc_part, tc_sync;
  void init(const LevelGeom& G, int nc, int m);
};
// x = D_hat^{-1} b to ||b - D_hat x|| <= tol_rel ||b|| (or maxit iterations) by
// GCR(m) on the reduced even-odd system (or on D_hat itself when the level has
// an odd extent); adds the iterations run to *d_iters (device)
// (grid: blocks of the cooperative launch, 0 for B.grid; at most B.grid)
void coarse_gcr_solve(const LevelGeom& G, const CoarseOp& C, const CoarseGCRBuffers& B, int m, int maxit,
                      double tol_rel, const float* b, float* x, long long* d_iters, int* flags, cudaStream_t s,
                      int grid = 0);
// The same solve with the links streamed through shared memory by bulk
// asynchronous copies and three grid barriers per iteration
// (coarse_stream.cu): even-odd levels only.  grid: blocks of the cooperative
// launch, one of coarse_gcr_stream_grids().  Raises FLAG_TIMEOUT if a wait
// runs out of time.
bool coarse_gcr_stream_ok(const LevelGeom& G, const CoarseOp& C);
// floors of one coarsest-level GCR iteration on `grid` CTAs: the time of one
// grid barrier and of streaming the iteration's links (A and the even-site Y)
// L2 -> shared memory without arithmetic (floor.cu)
void coarse_floor(const LevelGeom& G, const CoarseOp& C, int grid, int* flags, cudaStream_t s, double* barrier_us,
                  double* stream_us, double* stream_bytes);
std::vector<int> coarse_gcr_stream_grids(const LevelGeom& G, const CoarseOp& C);
void coarse_gcr_stream_solve(const LevelGeom& G, const CoarseOp& C, CoarseGCRBuffers& B, int m, int maxit,
                             double tol_rel, const float* b, float* x, long long* d_iters, int* flags, cudaStream_t s,
                             int grid);
// The same GCR for nb (1 .. 16) systems of one even-odd lattice whose links
// are stored in FP16, with the hop terms on tensor cores (coarse_tc.cu):
// system p's right-hand side at b + 2 p bstride floats, its solution at
// x + 2 p xstride floats (full coarse vectors), tolerance tol_rel[p]; grid:
// one of coarse_gcr_tc_grids().  Raises FLAG_TIMEOUT if a wait runs out of time.
bool coarse_gcr_tc_ok(const LevelGeom& G, const CoarseOp& C, int nb);
std::vector<int> coarse_gcr_tc_grids(const LevelGeom& G, const CoarseOp& C, int nb);
void coarse_gcr_tc_solve(const LevelGeom& G, const CoarseOp& C, CoarseGCRBuffers& B, int m, int maxit,
                         const double* tol_rel, int nb, const float* b, size_t bstride, float* x, size_t xstride,
                         long long* d_iters, int* flags, cudaStream_t s, int grid);
// the systems on tensor cores when they are consecutive vectors of one FP16
// lattice that coarse_gcr_tc_ok accepts (returns false, launching nothing,
// otherwise)
bool coarse_gcr_tc_try(const std::vector<CoarseSystem>& sys, CoarseGCRBuffers& B, int m, int maxit, int* flags,
                       cudaStream_t s);
// smaller grids worth timing against B.grid: the fewest blocks that keep the
// largest number of stencil sites per block, and one more site per block
// (fewer blocks at every grid barrier)
std::vector<int> coarse_gcr_smaller_grids(const LevelGeom& G, const CoarseGCRBuffers& B);

// ---- batched coarsest solves (coarse_batch.cu)
// One coarse system: the lattice and operator (a level of some context), its
// right-hand side and solution (full FP32 coarse vectors), its relative
// tolerance and the device counter its iterations are added to.
struct CoarseSystem {
  const LevelGeom* G;
  const CoarseOp* C;
  const float* b;
  float* x;
  double tol_rel;
  long long* iters;
};
// Solves up to coarse_gcr_batch_max() systems -- of at most
// coarse_gcr_group_max() different lattices, all even-odd or none, one link
// storage format -- in one cooperative launch, each to its own tolerance, by
// the GCR(m) of coarse_gcr_solve.  Buffers in B grow on demand.
int coarse_gcr_batch_max();
int coarse_gcr_group_max();
void coarse_gcr_solve_multi(const std::vector<CoarseSystem>& sys, CoarseGCRBuffers& B, int m, int maxit, int* flags,
                            cudaStream_t s);
// nb right-hand sides of one lattice (b, x: [nb][nsites nc] floats x 2)
void coarse_gcr_solve_batch(const LevelGeom& G, const CoarseOp& C, CoarseGCRBuffers& B, int m, int maxit,
                            double tol_rel, int nb, const float* b, float* x, long long* d_iters, int* flags,
                            cudaStream_t s);

// the coarsest systems of a context's batched cycle (2-level hierarchies; the
// right-hand sides were written by mg_batch_pre) and the buffers of its
// batched solves (multigrid.cu)
void mg_batch_systems(Ctx* c, int nb, std::vector<CoarseSystem>& out);
CoarseGCRBuffers& mg_batch_buffers(Ctx* c);

// ---- setup kernels
// Philox start vector on a coarse level (AoS)
void philox_coarse_vector(const LevelGeom& G, uint64_t seed, int level, int k, float* out, cudaStream_t s);
// chirality split + block Gram-Schmidt of nv vectors V[k] (level vectors)
// into T.P (and T.Pscale); sets FLAG_GS_BREAKDOWN on breakdown
void block_orthonormalize(TransferOp& T, const float* const* V, DBuf& scratch, int* flags, cudaStream_t s);

// ---- ABI packing of coarse vectors ([lex][ndof] complex128 <-> storage FP32)
void pack_coarse(const LevelGeom& G, const double* abi, float* v, cudaStream_t s);
void unpack_coarse(const LevelGeom& G, const float* v, double* abi, cudaStream_t s);

}  // namespace mg
