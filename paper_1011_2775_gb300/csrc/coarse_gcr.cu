// The coarsest-level solve as one persistent cooperative kernel.
//
// Section "Implementation": the coarsest lattice is solved by an
// unpreconditioned GCR to a residual tolerance relative to its right-hand
// side (about 0.1); section "Red-black preconditioning": the coarse system
// is solved through its reduced even-odd form.  The host-driven GCR of
// solver.cu does the same arithmetic, but on the coarsest lattice each
// iteration is a handful of tiny kernels plus a host round trip for the
// convergence test, so latency dominates.  Here the whole solve -- b_r, the
// GCR(m) iterations with restarts and true-residual recomputation, the
// convergence test and the reconstruction of both parities -- runs in one
// launch: phases are separated by grid-wide barriers of a cooperative launch
// (all blocks co-resident), every inner product is reduced deterministically
// (per-block FP64 partials, then the same ordered sum in every block, so all
// blocks take identical decisions), and the host reads nothing until the
// next level up needs the result.
//
// Algorithm per GCR iteration k (flexible GCR with z_k = r_k, the solution
// update deferred to the end of each restart cycle, as in solver.cu):
//   w = D_r r;  beta_j = <w_j, w>;  w -= sum_j beta_j w_j;  gamma = |w|;
//   w /= gamma;  alpha = <w, r>;  r -= alpha w;  test |r| <= tol.
#include <cooperative_groups.h>

#include <cstring>

#include "coarse.h"
#include "coarse_dev.cuh"

namespace cg = cooperative_groups;

namespace mg {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxRestart = 64;
constexpr int kNR = 2 * kMaxRestart + 8;  // reduction slots per block
// Consecutive reductions of one iteration use disjoint slot regions: a block
// may start writing the next reduction while a slower block still sums the
// previous one (there is no barrier between a read and the next write).
constexpr int RA = 0;                      // <w_j, w>: 2 (m - 1) slots
constexpr int RB = 2 * kMaxRestart;        // ||w||^2, <w, r>
constexpr int RC = RB + 3;                 // ||r||^2 (recurrence)
constexpr int RD = RC + 1;                 // ||b||^2, true residual

struct CGArgs {
  int nc, half, nsites, m, maxit, eo, nsplit;
  double tol_rel;
  const int* nbr;
  const void* Y;     // links, storage format of the kernel's ST
  const float* Ys;   // Y tile scales [site][8]
  const float2* X;
  const float2* Xinv;
  const float2* A;   // folded links (CoarseOp::A), FP32
  const float2* b;   // full right-hand side
  float2* x;         // full solution
  float2* r;         // residual (half when eo, else full)
  float2* y;         // GCR iterate (half when eo, else full)
  float2* br;        // reduced right-hand side (eo)
  float2* tA;        // full temporaries
  float2* tB;
  float2* W;         // [m][n]
  float2* Z;         // [m][n]
  double* partials;  // [gridDim][kNR]
  double* scal;      // beta [m][m][2], alpha [m][2], gamma [m], c [m][2]
  long long* iters;  // accumulated iteration count (device)
  int* flags;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce nq values (one per thread-slot array v[q]) and store the block's
// partial sums in partials[q0 + q][blockIdx.x] (slot-major, so that the
// totals below read them coalesced).
__device__ void block_partials(const CGArgs& a, double* v, int nq, int q0, double* sred) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < nq; q++) {
    const double t = wsum(v[q]);
    if (lane == 0) sred[q * 8 + wid] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += sred[q * 8 + w];
    a.partials[(size_t)(q0 + q) * gridDim.x + blockIdx.x] = s;
  }
  __syncthreads();
}

// After a grid barrier: the totals of slots [q0, q0+nq), identical in every
// block (same lane partitions, same shuffle tree).  One warp per slot; the
// lanes read the per-block partials in parallel.
__device__ void grid_totals(const CGArgs& a, int q0, int nq, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int U = 4;  // slots per warp per round, loaded together
  const int G = gridDim.x;
  for (int qb = wid; qb < nq; qb += nw * U) {
    double s[U];
#pragma unroll
    for (int u = 0; u < U; u++) s[u] = 0.0;
#pragma unroll 2
    for (int g = lane; g < G; g += 32) {
      double t[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int q = qb + u * nw;
        t[u] = q < nq ? __ldcg(a.partials + (size_t)(q0 + q) * G + g) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; u++) s[u] += t[u];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const double r = wsum(s[u]);
      const int q = qb + u * nw;
      if (lane == 0 && q < nq) out[q] = r;
    }
  }
  __syncthreads();
}

// out[s] = C(s) in[s] for storage sites s in [s0, s1)
__device__ void site_mul(const CGArgs& a, const float2* C, int s0, int s1, float2* out, const float2* in,
                         float2* sv) {
  const int nc = a.nc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rpw = (nc + nw - 1) / nw;
  for (int s = s0 + blockIdx.x; s < s1; s += gridDim.x) {
    for (int t = threadIdx.x; t < nc; t += blockDim.x) sv[t] = in[(size_t)s * nc + t];
    __syncthreads();
    float2 res[kGemvMaxRows];
    warp_gemv(C + (size_t)s * nc * nc, nc, nc, sv, w, rpw, lane, res);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        const int i = w * rpw + r;
        if (r < rpw && i < nc) out[(size_t)s * nc + i] = res[r];
      }
    __syncthreads();
  }
}

// Hopping term for storage sites [s0, s1), one site per block at a time:
//   mode 0: out = x_self - hop(in)             (D_r last step / residual)
//   mode 1: out = Xinv (hop(in))               (D_r middle step)
//   mode 2: out = Xinv (x_self - hop(in))      (reconstruction of the odd sites)
//   mode 3: out = X x_self + hop(in)           (full D_hat, no even-odd)
// x_self is read from `xs`.
template <int ST>
__device__ void hop_phase(const CGArgs& a, int mode, int s0, int s1, float2* out, const float2* in, const float2* xs,
                          float2* sm) {
  const int nc = a.nc;
  float2* vin = sm;            // [8 nc]
  float2* tv = sm + 8 * nc;    // [nc]
  float2* vx = tv + nc;        // [nc]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rpw = (nc + nw - 1) / nw;
  for (int s = s0 + blockIdx.x; s < s1; s += gridDim.x) {
    for (int t = threadIdx.x; t < 8 * nc; t += blockDim.x) {
      const int d = t / nc, j = t % nc;
      float2 v = in[(size_t)a.nbr[(size_t)s * 8 + d] * nc + j];
      const float sc = a.Ys[(size_t)s * 8 + d];
      vin[t] = make_float2(v.x * sc, v.y * sc);
    }
    for (int t = threadIdx.x; t < nc; t += blockDim.x) vx[t] = xs[(size_t)s * nc + t];
    __syncthreads();
    float2 res[kGemvMaxRows];
    warp_gemv<ST>(static_cast<const char*>(a.Y) + (size_t)s * nc * 8 * nc * link_bytes<ST>(), nc, 8 * nc, vin, w, rpw,
                  lane, res);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        const int i = w * rpw + r;
        if (r < rpw && i < nc) {
          if (mode == 0) out[(size_t)s * nc + i] = make_float2(vx[i].x - res[r].x, vx[i].y - res[r].y);
          else if (mode == 2) tv[i] = make_float2(vx[i].x - res[r].x, vx[i].y - res[r].y);
          else tv[i] = res[r];
        }
      }
    __syncthreads();
    if (mode != 0) {
      const float2* Cm = mode == 3 ? a.X : a.Xinv;
      const float2* src = mode == 3 ? vx : tv;
      warp_gemv(Cm + (size_t)s * nc * nc, nc, nc, src, w, rpw, lane, res);
      if (lane == 0)
#pragma unroll
        for (int r = 0; r < kGemvMaxRows; r++) {
          const int i = w * rpw + r;
          if (r < rpw && i < nc) {
            if (mode == 3) out[(size_t)s * nc + i] = make_float2(res[r].x + tv[i].x, res[r].y + tv[i].y);
            else out[(size_t)s * nc + i] = res[r];
          }
        }
      __syncthreads();
    }
  }
}

// One GEMV per site with the site's rows split over a.nsplit work items, so
// the blocks stay balanced when there are fewer sites than 2x blocks.
// Links L (storage format ST): site s uses L + (s - lbase) * nc * nb * nc
// (row-major, nb blocks of nc columns) with tile scales
// scale[(s - lbase) * nb + block] (null: 1); its vector gathers the 8
// neighbours (and, for nb == 9, the site itself).  subtract: out = xs - L v,
// else out = L v.
template <int ST>
__device__ void hop_rows(const CGArgs& a, const void* L, const float* scale, int lbase, int nb, bool subtract,
                         int s0, int s1, float2* out, const float2* in, const float2* xs, float2* sm) {
  const int nc = a.nc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (nc + a.nsplit - 1) / a.nsplit;
  const int rpw = (per + nw - 1) / nw;
  const int nitems = (s1 - s0) * a.nsplit;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int s = s0 + it / a.nsplit, part = it % a.nsplit;
    const int row0 = part * per, row1 = row0 + per < nc ? row0 + per : nc;
    for (int t = threadIdx.x; t < nb * nc; t += blockDim.x) {
      const int d = t / nc, j = t % nc;
      float2 x = d < 8 ? in[(size_t)a.nbr[(size_t)s * 8 + d] * nc + j] : in[(size_t)s * nc + j];
      if (scale) {
        const float sc = scale[(size_t)(s - lbase) * nb + d];
        x = make_float2(sc * x.x, sc * x.y);
      }
      sm[t] = x;
    }
    __syncthreads();
    float2 res[kGemvMaxRows];
    warp_gemv_rows<ST>(static_cast<const char*>(L) + (size_t)(s - lbase) * nc * nb * nc * link_bytes<ST>(), row0, row1,
                       nb * nc, sm, w, rpw, lane, res);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < kGemvMaxRows; r++) {
        const int i = row0 + w * rpw + r;
        if (r < rpw && i < row1) {
          if (subtract) {
            const float2 x = xs[(size_t)s * nc + i];
            out[(size_t)s * nc + i] = make_float2(x.x - res[r].x, x.y - res[r].y);
          } else {
            out[(size_t)s * nc + i] = res[r];
          }
        }
      }
    __syncthreads();
  }
}

// w = A v with A = D_r on the even sites (folded links: two GEMV phases, one
// barrier) or the full D_hat (one GEMV phase over [Y | X])
template <int ST>
__device__ void apply_A(const CGArgs& a, cg::grid_group& grid, float2* w, const float2* v, float2* sm) {
  if (a.eo) {
    hop_rows<kStF32>(a, a.A, nullptr, a.half, 8, false, a.half, a.nsites, a.tB, v, nullptr, sm);  // X_o^-1 Y_oe X_e^-1 v_e
    grid.sync();
    hop_rows<ST>(a, a.Y, a.Ys, 0, 8, true, 0, a.half, w, a.tB, v, sm);                            // w_e = v_e - Y_eo t_o
  } else {
    hop_rows<kStF32>(a, a.A, nullptr, 0, 9, false, 0, a.nsites, w, v, nullptr, sm);               // w = [Y | X] v
  }
}

// Each block owns a contiguous chunk [e0, e1) of every (half) vector for the
// element-wise phases; the stencil phases own whole sites.  Phases with
// different ownership are always separated by a grid barrier.
template <int ST>
__global__ void __launch_bounds__(kThreads) k_coarse_gcr(CGArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) double dsm[];
  double* sred = dsm;                      // [kNR][8]
  double* tot = sred + kNR * 8;            // [kNR]
  float2* sm = reinterpret_cast<float2*>(tot + kNR);  // [10 nc]
  const int nc = a.nc;
  const int m = a.m;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t n = (size_t)(a.eo ? a.half : a.nsites) * nc;
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t e0 = (size_t)blockIdx.x * chunk;
  const size_t e1 = e0 + chunk < n ? e0 + chunk : n;
  double* beta = a.scal;
  double* alpha = beta + 2 * (size_t)m * m;
  double* gam = alpha + 2 * m;
  double v[4];

  // ---- ||b|| (full rhs) and the reduced right-hand side
  {
    const size_t nf = (size_t)a.nsites * nc;
    const size_t cf = (nf + gridDim.x - 1) / gridDim.x;
    const size_t f0 = (size_t)blockIdx.x * cf, f1 = f0 + cf < nf ? f0 + cf : nf;
    v[0] = 0.0;
    for (size_t e = f0 + threadIdx.x; e < f1; e += blockDim.x) {
      const float2 q = a.b[e];
      v[0] += (double)q.x * q.x + (double)q.y * q.y;
    }
    block_partials(a, v, 1, RD, sred);
  }
  const float2* rhs = a.b;
  if (a.eo) {
    site_mul(a, a.Xinv, a.half, a.nsites, a.tB, a.b, sm);        // t_o = X_o^{-1} b_o
    grid.sync();
    hop_rows<ST>(a, a.Y, a.Ys, 0, 8, true, 0, a.half, a.br, a.tB, a.b, sm);  // b_r = b_e - Y_eo t_o
    rhs = a.br;
  }
  grid.sync();
  grid_totals(a, RD, 1, tot);
  const double bnorm = sqrt(tot[0]);
  const double tol = a.tol_rel * bnorm;
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {   // y = 0, r = rhs
    a.y[e] = make_float2(0.f, 0.f);
    a.r[e] = rhs[e];
  }
  long long its = 0;
  bool done = !(bnorm > 0.0);
  grid.sync();
  while (!done && its < a.maxit) {
    int k = 0;
    double rn = 0.0;
    while (k < m && its < a.maxit) {
      float2* wk = a.W + (size_t)k * n;
      float2* zk = a.Z + (size_t)k * n;
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) zk[e] = a.r[e];
      apply_A<ST>(a, grid, wk, a.r, sm);
      grid.sync();
      // beta_j = <w_j, w> over this block's chunk: warp w owns j = w + u*nw,
      // u < 4, and issues the loads of all four before reducing
      for (int jb = wid; jb < k; jb += 4 * nw) {
        double re[4] = {0.0, 0.0, 0.0, 0.0}, im[4] = {0.0, 0.0, 0.0, 0.0};
        for (size_t e = e0 + lane; e < e1; e += 32) {
          const float2 x = wk[e];
          float2 p[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int j = jb + u * nw;
            p[u] = j < k ? a.W[(size_t)j * n + e] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; u++) {
            re[u] += (double)p[u].x * x.x + (double)p[u].y * x.y;
            im[u] += (double)p[u].x * x.y - (double)p[u].y * x.x;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int j = jb + u * nw;
          const double sr = wsum(re[u]), si = wsum(im[u]);
          if (lane == 0 && j < k) {
            a.partials[(size_t)(RA + 2 * j) * gridDim.x + blockIdx.x] = sr;
            a.partials[(size_t)(RA + 2 * j + 1) * gridDim.x + blockIdx.x] = si;
          }
        }
      }
      grid.sync();
      if (k) grid_totals(a, RA, 2 * k, tot);
      // w -= sum beta_j w_j; then ||w||^2 and <w, r>
      v[0] = v[1] = v[2] = 0.0;
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 x = wk[e];
        for (int j = 0; j < k; j++) {
          const float2 p = a.W[(size_t)j * n + e];
          const float br = (float)tot[2 * j], bi = (float)tot[2 * j + 1];
          x.x -= br * p.x - bi * p.y;
          x.y -= br * p.y + bi * p.x;
        }
        wk[e] = x;
        const float2 rr = a.r[e];
        v[0] += (double)x.x * x.x + (double)x.y * x.y;
        v[1] += (double)x.x * rr.x + (double)x.y * rr.y;
        v[2] += (double)x.x * rr.y - (double)x.y * rr.x;
      }
      if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
          beta[(j + (size_t)m * k) * 2] = tot[2 * j];
          beta[(j + (size_t)m * k) * 2 + 1] = tot[2 * j + 1];
        }
      block_partials(a, v, 3, RB, sred);
      grid.sync();
      grid_totals(a, RB, 3, tot);
      const double g = tot[0] > 0 ? sqrt(tot[0]) : 1.0;
      const double ar = tot[1] / g, ai = tot[2] / g;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        alpha[2 * k] = ar;
        alpha[2 * k + 1] = ai;
        gam[k] = g;
      }
      const float ig = (float)(1.0 / g), far = (float)ar, fai = (float)ai;
      v[0] = 0.0;
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 x = wk[e];
        x.x *= ig;
        x.y *= ig;
        wk[e] = x;
        float2 rr = a.r[e];
        rr.x -= far * x.x - fai * x.y;
        rr.y -= far * x.y + fai * x.x;
        a.r[e] = rr;
        v[0] += (double)rr.x * rr.x + (double)rr.y * rr.y;
      }
      block_partials(a, v, 1, RC, sred);
      grid.sync();
      grid_totals(a, RC, 1, tot);
      rn = sqrt(tot[0]);
      k++;
      its++;
      if (!(rn == rn)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&a.flags[FLAG_NAN], 1);
        done = true;
        break;
      }
      if (rn <= tol) break;
    }
    // back substitution (every block, identical) and y += sum c_j z_j
    if (threadIdx.x == 0) {
      for (int j = k - 1; j >= 0; j--) {
        double re = alpha[2 * j], im = alpha[2 * j + 1];
        for (int l = j + 1; l < k; l++) {
          const double br = beta[(j + (size_t)m * l) * 2], bi = beta[(j + (size_t)m * l) * 2 + 1];
          re -= br * tot[2 * l + 8] - bi * tot[2 * l + 9];
          im -= br * tot[2 * l + 9] + bi * tot[2 * l + 8];
        }
        tot[2 * j + 8] = re / gam[j];
        tot[2 * j + 9] = im / gam[j];
      }
    }
    __syncthreads();
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      float2 yy = a.y[e];
      double re = yy.x, im = yy.y;
      for (int j = 0; j < k; j++) {
        const float2 z = a.Z[(size_t)j * n + e];
        const double cr = tot[2 * j + 8], ci = tot[2 * j + 9];
        re += cr * z.x - ci * z.y;
        im += cr * z.y + ci * z.x;
      }
      a.y[e] = make_float2((float)re, (float)im);
    }
    grid.sync();
    if (done) break;
    // true residual r = rhs - A y
    apply_A<ST>(a, grid, a.r, a.y, sm);
    grid.sync();
    v[0] = 0.0;
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const float2 ay = a.r[e], bb = rhs[e];
      const float2 rr = make_float2(bb.x - ay.x, bb.y - ay.y);
      a.r[e] = rr;
      v[0] += (double)rr.x * rr.x + (double)rr.y * rr.y;
    }
    block_partials(a, v, 1, RD, sred);
    grid.sync();
    grid_totals(a, RD, 1, tot);
    rn = sqrt(tot[0]);
    if (rn <= tol || !(rn == rn)) done = true;
  }
  // reconstruction
  if (a.eo) {
    site_mul(a, a.Xinv, 0, a.half, a.x, a.y, sm);                 // x_e = X_e^{-1} y_e
    grid.sync();
    hop_phase<ST>(a, 2, a.half, a.nsites, a.x, a.x, a.b, sm);     // x_o = X_o^{-1}(b_o - Y_oe x_e)
  } else {
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) a.x[e] = a.y[e];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters += its;
}

}  // namespace

size_t coarse_gcr_scalars(int m) { return 2 * (size_t)m * m + 5 * (size_t)m + 16; }

int coarse_gcr_grid(int nc) {
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  int sms = 0;
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = sizeof(double) * (kNR * 8 + kNR) + sizeof(float2) * 10 * (size_t)nc;
  // the smallest residency of the three storage instantiations, so that any
  // of them can be launched cooperatively on this grid
  int per = 1 << 20;
  const void* kernels[3] = {(const void*)k_coarse_gcr<kStF32>, (const void*)k_coarse_gcr<kStF16>,
                            (const void*)k_coarse_gcr<kStBF16>};
  for (const void* k : kernels) {
    int p = 0;
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, k, kThreads, smem));
    per = p < per ? p : per;
  }
  if (per < 1) raise(MG_ERR_CUDA, "persistent coarse GCR cannot be resident");
  return sms * (per < 4 ? per : 4);
}

std::vector<int> coarse_gcr_smaller_grids(const LevelGeom& G, const CoarseGCRBuffers& B) {
  const int target = G.eo ? G.half : G.nsites;
  const int per = (target + B.grid - 1) / B.grid;  // sites per block on the full grid
  std::vector<int> out;
  for (int k = per; k <= per + 1; k++) {
    const int g = (target + k - 1) / k;
    if (g >= 1 && g < B.grid && (out.empty() || g < out.back())) out.push_back(g);
  }
  return out;
}

void coarse_gcr_solve(const LevelGeom& G, const CoarseOp& C, const CoarseGCRBuffers& B, int m, int maxit,
                      double tol_rel, const float* b, float* x, long long* d_iters, int* flags, cudaStream_t s,
                      int grid_blocks) {
  if (m > kMaxRestart) raise(MG_ERR_ARG, "coarse restart too long for the persistent solver");
  CGArgs a;
  a.nc = C.nc;
  a.half = G.half;
  a.nsites = G.nsites;
  a.m = m;
  a.maxit = maxit;
  a.eo = G.eo ? 1 : 0;
  a.tol_rel = tol_rel;
  a.nbr = G.d_nbr.as<int>();
  a.Y = C.Y.get();
  a.Ys = C.Yscale.as<float>();
  a.X = C.X.as<float2>();
  a.Xinv = C.Xinv.as<float2>();
  a.A = C.A.as<float2>();
  if (!a.A) raise(MG_ERR_STATE, "folded coarse links missing");
  a.nsplit = B.nsplit;
  a.b = reinterpret_cast<const float2*>(b);
  a.x = reinterpret_cast<float2*>(x);
  a.r = B.r.as<float2>();
  a.y = B.y.as<float2>();
  a.br = B.br.as<float2>();
  a.tA = B.tA.as<float2>();
  a.tB = B.tB.as<float2>();
  a.W = B.W.as<float2>();
  a.Z = B.Z.as<float2>();
  a.partials = B.partials.as<double>();
  a.scal = B.scal.as<double>();
  a.iters = d_iters;
  a.flags = flags;
  const size_t smem = sizeof(double) * (kNR * 8 + kNR) + sizeof(float2) * 10 * (size_t)C.nc;
  const int grid = grid_blocks > 0 && grid_blocks < B.grid ? grid_blocks : B.grid;
  void* params[] = {&a};
  const void* kern = C.store == STORE_F16    ? (const void*)k_coarse_gcr<kStF16>
                     : C.store == STORE_BF16 ? (const void*)k_coarse_gcr<kStBF16>
                                             : (const void*)k_coarse_gcr<kStF32>;
  MG_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kThreads), params, smem, s));
  MG_LAUNCH();
}

void CoarseGCRBuffers::init(const LevelGeom& G, int nc, int m) {
  const size_t nfull = (size_t)G.nsites * nc;
  const size_t n = G.eo ? (size_t)G.half * nc : nfull;
  // one stencil site per block and phase where possible, at least one block per SM
  const int most = coarse_gcr_grid(nc);
  int sms = 0, dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int target = G.eo ? G.half : G.nsites;
  grid = target < most ? target : most;
  if (grid < sms) grid = sms < most ? sms : most;
  // One work item per site.  Splitting a site's rows over several items was
  // measured slower on GB300: a block then walks its items one after another,
  // each with its own gather and load latency.
  nsplit = 1;
  r.alloc(sizeof(float2) * n);
  y.alloc(sizeof(float2) * n);
  br.alloc(sizeof(float2) * (G.eo ? n : 1));
  tA.alloc(sizeof(float2) * nfull);
  tB.alloc(sizeof(float2) * nfull);
  MG_CUDA(cudaMemset(tA.get(), 0, sizeof(float2) * nfull));
  MG_CUDA(cudaMemset(tB.get(), 0, sizeof(float2) * nfull));
  W.alloc(sizeof(float2) * n * m);
  Z.alloc(sizeof(float2) * n * m);
  partials.alloc(sizeof(double) * (size_t)grid * kNR);
  scal.alloc(sizeof(double) * coarse_gcr_scalars(m));
}

}  // namespace mg
