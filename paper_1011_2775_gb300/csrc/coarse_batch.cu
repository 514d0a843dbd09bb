// Batched coarsest-level solves: several systems -- right-hand sides of one
// lattice and systems of several lattices of uneven size -- in one
// cooperative launch.
//
// The coarsest solve of section "Implementation" (unpreconditioned GCR on the
// reduced even-odd coarse system to ~0.1 relative residual) is latency-bound:
// grid barriers and L2 round trips, not bytes.  Solving B systems in
// lock-step costs little more per iteration than solving one:
//  * systems are grouped by geometry (one coarse lattice and its links); a
//    stencil work item is one site of one group, processed for every active
//    system of the group -- the neighbour vectors of all of them are gathered
//    once and every link pair loaded serves kPB systems (warp_gemv_multi);
//  * element-wise phases: the CTAs are split into B groups of Gp; CTA group p
//    owns system p's vectors, so a CTA reduces and reads only its own system's
//    partial sums (Gp per slot); the residual norms that decide convergence
//    are read for every system by every CTA (B * Gp partials).
// Each system keeps its own Krylov space, scalars, tolerance, convergence test
// and restart decisions; a converged system is skipped.  All decisions derive
// from sums every CTA computes in the same order, so the barriers stay
// uniform.  The arithmetic per system is that of the single-system kernel of
// coarse_gcr.cu (flexible GCR with z = r, deferred solution update).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>

#include "coarse.h"
#include "coarse_dev.cuh"

namespace cg = cooperative_groups;

namespace mg {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxRestart = 64;
constexpr int kMaxBatch = 16;
constexpr int kMaxGroups = 8;
constexpr int kPB = 4;   // systems per link pass of the multi-vector GEMV
constexpr int kRB = 2;   // rows per pass of the multi-vector GEMV
constexpr int kNR = 2 * kMaxRestart + 8;
constexpr int RA = 0;                      // <w_j, w>: 2 (m - 1) slots
constexpr int RB = 2 * kMaxRestart;        // ||w||^2, <w, r>
constexpr int RC = RB + 3;                 // ||r||^2 (recurrence)
constexpr int RD = RC + 1;                 // ||b||^2, true residual

size_t scalars_per_system(int m) { return 2 * (size_t)m * m + 5 * (size_t)m + 16; }

struct Group {          // one coarse lattice and its operator
  int nc, half, nsites;
  const int* nbr;
  const void* Y;        // links in the launch's storage format
  const float* Ys;
  const float2* Xinv;
  const float2* A;      // folded links (FP32)
  unsigned mask;        // systems of this group
};

struct MArgs {
  int B, ng, Gp, m, maxit, eo, maxnc;
  Group grp[kMaxGroups];
  int group_of[kMaxBatch];
  double tol_rel[kMaxBatch];
  size_t n[kMaxBatch];        // half (eo) or full vector length of each system
  size_t nf[kMaxBatch];       // full vector length
  size_t off[kMaxBatch];      // offset of each system in the packed [sum n] buffers
  size_t offf[kMaxBatch];     // offset in the packed [sum nf] buffer
  size_t ntot;                // sum n: stride of W, Z per Krylov index
  const float2* b[kMaxBatch]; // right-hand sides (full coarse vectors)
  float2* x[kMaxBatch];       // solutions (full coarse vectors)
  float2* r;                  // packed [sum n]
  float2* y;
  float2* br;
  float2* tB;                 // packed [sum nf]
  float2* W;                  // [m][sum n]
  float2* Z;
  double* partials;           // [kNR][B][Gp]
  double* scal;               // [B][nscal]
  size_t nscal;
  long long* iters[kMaxBatch];   // each system's iteration counter (several may share one)
  int* flags;
};

// vector selectors of the stencil phases
enum VecKind { V_R = 0, V_Y, V_BR, V_TB, V_B, V_X, V_W };
struct Vec {
  int kind;
  int k;  // Krylov index for V_W
};
__device__ __forceinline__ float2* vec_ptr(const MArgs& A, Vec v, int p) {
  switch (v.kind) {
    case V_R: return A.r + A.off[p];
    case V_Y: return A.y + A.off[p];
    case V_BR: return A.br + A.off[p];
    case V_TB: return A.tB + A.offf[p];
    case V_B: return const_cast<float2*>(A.b[p]);
    case V_X: return A.x[p];
    default: return A.W + (size_t)v.k * A.ntot + A.off[p];
  }
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block partial sums of nq values of system p: slot (q0 + q, p, gi)
__device__ void own_partials(const MArgs& A, const double* v, int nq, int q0, int p, int gi, double* sred) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < nq; q++) {
    const double t = wsum(v[q]);
    if (lane == 0) sred[q * 8 + wid] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += sred[q * 8 + w];
    A.partials[((size_t)(q0 + q) * A.B + p) * A.Gp + gi] = s;
  }
  __syncthreads();
}

// totals of slots [q0, q0+nq) of system p: out[q] (one warp per slot)
__device__ void own_totals(const MArgs& A, int q0, int nq, int p, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = wid; q < nq; q += nw) {
    double s = 0.0;
    for (int g = lane; g < A.Gp; g += 32) s += __ldcg(A.partials + ((size_t)(q0 + q) * A.B + p) * A.Gp + g);
    s = wsum(s);
    if (lane == 0) out[q] = s;
  }
  __syncthreads();
}

// slot q of every system: out[p] (one warp per system)
__device__ void all_totals(const MArgs& A, int q, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = wid; p < A.B; p += nw) {
    double s = 0.0;
    for (int g = lane; g < A.Gp; g += 32) s += __ldcg(A.partials + ((size_t)q * A.B + p) * A.Gp + g);
    s = wsum(s);
    if (lane == 0) out[p] = s;
  }
  __syncthreads();
}

// the systems of `mask` as a list in shared memory; returns their number
__device__ int list_of(unsigned mask, int* slist) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int q = 0;
    for (int p = 0; p < kMaxBatch; p++)
      if ((mask >> p) & 1u) slist[q++] = p;
  }
  __syncthreads();
  return __popc(mask);
}

enum Range { R_EVEN = 0, R_ODD = 1, R_ALL = 2 };
__device__ __forceinline__ void range_of(const Group& g, int range, int& s0, int& s1) {
  s0 = range == R_ODD ? g.half : 0;
  s1 = range == R_EVEN ? g.half : g.nsites;
}
enum LinkKind { L_FOLDED = 0, L_Y = 1 };

// Stencil over the sites of `range` in every group, for the systems of `mask`:
//   out_p[s] = [xs_p[s] -] L(s) v_p,  v_p gathered from in_p at the 8
// neighbours (and s itself for the folded [Y | X] links of an odd-extent
// lattice), with the Y tile scales folded into the gathered vector.
template <int ST>
__device__ void msites(const MArgs& A, unsigned mask, int* plist, int links, int range, bool subtract, Vec out,
                       Vec in, Vec xs, float2* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int total = 0;
  for (int gi = 0; gi < A.ng; gi++) {
    int s0, s1;
    range_of(A.grp[gi], range, s0, s1);
    if (A.grp[gi].mask & mask) total += s1 - s0;
  }
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    // find the group and site of this item
    int gidx = 0, s = 0, acc = 0;
    for (int gi = 0; gi < A.ng; gi++) {
      int s0, s1;
      range_of(A.grp[gi], range, s0, s1);
      if (!(A.grp[gi].mask & mask)) continue;
      if (it < acc + (s1 - s0)) {
        gidx = gi;
        s = s0 + (it - acc);
        break;
      }
      acc += s1 - s0;
    }
    const Group& g = A.grp[gidx];
    const int np = list_of(mask & g.mask, plist);
    const int nc = g.nc;
    const bool folded = links == L_FOLDED;
    const int nb = (folded && !A.eo) ? 9 : 8;
    const int lbase = (folded && A.eo) ? g.half : 0;
    const float* scale = folded ? nullptr : g.Ys;
    const int per = nb * nc;
    const int rpw = (nc + nw - 1) / nw;
    {  // four elements per thread and round: indices, then loads, in flight together
      constexpr int U = 4;
      const int total = np * per;
      for (int t0 = threadIdx.x; t0 < total; t0 += U * blockDim.x) {
        const float2* src[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int t = t0 + u * blockDim.x;
          const int tt = t < total ? t : 0;
          const int q = tt / per, rem = tt % per, d = rem / nc, j = rem % nc;
          const float2* inp = vec_ptr(A, in, plist[q]);
          src[u] = d < 8 ? inp + (size_t)g.nbr[(size_t)s * 8 + d] * nc + j : inp + (size_t)s * nc + j;
          sc[u] = scale ? scale[(size_t)s * 8 + d] : 1.f;
        }
        float2 x[U];
#pragma unroll
        for (int u = 0; u < U; u++) x[u] = *src[u];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int t = t0 + u * blockDim.x;
          if (t < total) sm[t] = make_float2(sc[u] * x[u].x, sc[u] * x[u].y);
        }
      }
    }
    __syncthreads();
    for (int q0 = 0; q0 < np; q0 += kPB) {
      const int cnt = np - q0 < kPB ? np - q0 : kPB;
      for (int rb = 0; rb < rpw; rb += kRB) {
        const int i0 = w * rpw + rb;
        if (i0 >= nc) break;
        float2 res[kRB][kPB];
        if (folded)
          warp_gemv_multi<kStF32, kRB, kPB>(g.A + (size_t)(s - lbase) * nc * per, i0, nc, per, sm + q0 * per, per,
                                             cnt, lane, res);
        else
          warp_gemv_multi<ST, kRB, kPB>(static_cast<const char*>(g.Y) + (size_t)s * nc * per * link_bytes<ST>(), i0,
                                        nc, per, sm + q0 * per, per, cnt, lane, res);
        if (lane == 0)
#pragma unroll
          for (int r = 0; r < kRB; r++) {
            const int i = i0 + r;
            if (rb + r < rpw && i < nc)
#pragma unroll
              for (int pp = 0; pp < kPB; pp++) {
                if (pp >= cnt) break;
                const int p = plist[q0 + pp];
                float2 o = res[r][pp];
                if (subtract) {
                  const float2 xv = vec_ptr(A, xs, p)[(size_t)s * nc + i];
                  o = make_float2(xv.x - o.x, xv.y - o.y);
                }
                vec_ptr(A, out, p)[(size_t)s * nc + i] = o;
              }
          }
      }
    }
    __syncthreads();
  }
}

// out_p[s] = X^{-1}(s) in_p[s] for the sites of `range`, systems of `mask`
__device__ void msite_inv(const MArgs& A, unsigned mask, int* plist, int range, Vec out, Vec in, float2* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int total = 0;
  for (int gi = 0; gi < A.ng; gi++) {
    int s0, s1;
    range_of(A.grp[gi], range, s0, s1);
    if (A.grp[gi].mask & mask) total += s1 - s0;
  }
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    int gidx = 0, s = 0, acc = 0;
    for (int gi = 0; gi < A.ng; gi++) {
      int s0, s1;
      range_of(A.grp[gi], range, s0, s1);
      if (!(A.grp[gi].mask & mask)) continue;
      if (it < acc + (s1 - s0)) {
        gidx = gi;
        s = s0 + (it - acc);
        break;
      }
      acc += s1 - s0;
    }
    const Group& g = A.grp[gidx];
    const int np = list_of(mask & g.mask, plist);
    const int nc = g.nc;
    const int rpw = (nc + nw - 1) / nw;
    for (int t = threadIdx.x; t < np * nc; t += blockDim.x)
      sm[t] = vec_ptr(A, in, plist[t / nc])[(size_t)s * nc + t % nc];
    __syncthreads();
    for (int q0 = 0; q0 < np; q0 += kPB) {
      const int cnt = np - q0 < kPB ? np - q0 : kPB;
      for (int rb = 0; rb < rpw; rb += kRB) {
        const int i0 = w * rpw + rb;
        if (i0 >= nc) break;
        float2 res[kRB][kPB];
        warp_gemv_multi<kStF32, kRB, kPB>(g.Xinv + (size_t)s * nc * nc, i0, nc, nc, sm + q0 * nc, nc, cnt, lane,
                                          res);
        if (lane == 0)
#pragma unroll
          for (int r = 0; r < kRB; r++) {
            const int i = i0 + r;
            if (rb + r < rpw && i < nc)
#pragma unroll
              for (int pp = 0; pp < kPB; pp++) {
                if (pp >= cnt) break;
                vec_ptr(A, out, plist[q0 + pp])[(size_t)s * nc + i] = res[r][pp];
              }
          }
      }
    }
    __syncthreads();
  }
}

// w_p = A v_p (the reduced D_r, or D_hat itself when the lattices have an odd extent)
template <int ST>
__device__ void mapply(const MArgs& A, unsigned mask, int* plist, cg::grid_group& grid, Vec w, Vec v, float2* sm) {
  if (A.eo) {
    msites<ST>(A, mask, plist, L_FOLDED, R_ODD, false, Vec{V_TB, 0}, v, Vec{V_R, 0}, sm);   // X_o^-1 Y_oe X_e^-1 v_e
    grid.sync();
    msites<ST>(A, mask, plist, L_Y, R_EVEN, true, w, Vec{V_TB, 0}, v, sm);                   // w_e = v_e - Y_eo t_o
  } else {
    msites<ST>(A, mask, plist, L_FOLDED, R_ALL, false, w, v, Vec{V_R, 0}, sm);                // w = [Y | X] v
  }
}

template <int ST>
__global__ void __launch_bounds__(kThreads) k_coarse_gcr_multi(MArgs A) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) double dsm[];
  double* sred = dsm;                        // [8][8]
  double* tot = sred + 64;                   // own totals [kNR]
  double* allv = tot + kNR;                  // per-system values [kMaxBatch]
  double* stol = allv + kMaxBatch;           // per-system absolute tolerances [kMaxBatch]
  double* cc = stol + kMaxBatch;             // own back-substitution coefficients [2 kMaxRestart]
  int* slist = reinterpret_cast<int*>(cc + 2 * kMaxRestart);                        // [kMaxBatch]
  int* scount = slist + kMaxBatch;                                                   // [kMaxBatch] iterations
  float2* sm = reinterpret_cast<float2*>(cc + 2 * kMaxRestart + kMaxBatch);         // gather
  const int B = A.B, m = A.m;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // this CTA's system (element-wise phases)
  const int myp = blockIdx.x / A.Gp, gi = blockIdx.x % A.Gp;
  const bool mine = myp < B;
  const int pp_ = mine ? myp : 0;
  const size_t n = A.n[pp_], nf = A.nf[pp_];
  const size_t chunk = (n + A.Gp - 1) / A.Gp;
  const size_t e0 = mine ? (size_t)gi * chunk : 0;
  const size_t e1 = mine ? (e0 + chunk < n ? e0 + chunk : n) : 0;
  float2* r = A.r + A.off[pp_];
  float2* y = A.y + A.off[pp_];
  double* beta = A.scal + pp_ * A.nscal;
  double* alpha = beta + 2 * (size_t)m * m;
  double* gam = alpha + 2 * m;
  const unsigned allm = B >= 32 ? 0xffffffffu : ((1u << B) - 1u);
  unsigned act = allm, run = 0u;
  double v[4];
  if (threadIdx.x < kMaxBatch) scount[threadIdx.x] = 0;

  // ---- ||b_p|| and the reduced right-hand sides
  {
    const size_t cf = (nf + A.Gp - 1) / A.Gp;
    const size_t f0 = mine ? (size_t)gi * cf : 0, f1 = mine ? (f0 + cf < nf ? f0 + cf : nf) : 0;
    v[0] = 0.0;
    for (size_t e = f0 + threadIdx.x; e < f1; e += blockDim.x) {
      const float2 q = A.b[pp_][e];
      v[0] += (double)q.x * q.x + (double)q.y * q.y;
    }
    if (mine) own_partials(A, v, 1, RD, myp, gi, sred);
  }
  Vec rhs{V_B, 0};
  if (A.eo) {
    msite_inv(A, act, slist, R_ODD, Vec{V_TB, 0}, Vec{V_B, 0}, sm);                            // t_o = X_o^{-1} b_o
    grid.sync();
    msites<ST>(A, act, slist, L_Y, R_EVEN, true, Vec{V_BR, 0}, Vec{V_TB, 0}, Vec{V_B, 0}, sm);  // b_r = b_e - Y_eo t_o
    rhs = Vec{V_BR, 0};
  }
  grid.sync();
  all_totals(A, RD, allv);
  act = 0u;
  for (int p = 0; p < B; p++)
    if (allv[p] > 0.0) act |= 1u << p;
  if (threadIdx.x < B) stol[threadIdx.x] = A.tol_rel[threadIdx.x] * sqrt(allv[threadIdx.x]);
  __syncthreads();
  const float2* rhsp = vec_ptr(A, rhs, pp_);
  if (mine)
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      y[e] = make_float2(0.f, 0.f);
      r[e] = rhsp[e];
    }
  long long its = 0;
  grid.sync();
  while (act && its < A.maxit) {
    int k = 0, kmy = 0;
    run = act;
    while (k < m && its < A.maxit && run) {
      const bool me = mine && ((run >> myp) & 1u);
      float2* Wk = A.W + (size_t)k * A.ntot + A.off[pp_];
      float2* Zk = A.Z + (size_t)k * A.ntot + A.off[pp_];
      if (me)
        for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) Zk[e] = r[e];
      mapply<ST>(A, run, slist, grid, Vec{V_W, k}, Vec{V_R, 0}, sm);
      grid.sync();
      // beta_j = <w_j, w> for this CTA's system: warp wid owns j = wid + u*nw (u < 4)
      if (me)
        for (int jb = wid; jb < k; jb += 4 * nw) {
          double re[4] = {0.0, 0.0, 0.0, 0.0}, im[4] = {0.0, 0.0, 0.0, 0.0};
          for (size_t e = e0 + lane; e < e1; e += 32) {
            const float2 x = Wk[e];
#pragma unroll
            for (int u = 0; u < 4; u++) {
              const int j = jb + u * nw;
              const float2 q = j < k ? A.W[(size_t)j * A.ntot + A.off[myp] + e] : make_float2(0.f, 0.f);
              re[u] += (double)q.x * x.x + (double)q.y * x.y;
              im[u] += (double)q.x * x.y - (double)q.y * x.x;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int j = jb + u * nw;
            const double sr = wsum(re[u]), si = wsum(im[u]);
            if (lane == 0 && j < k) {
              A.partials[((size_t)(RA + 2 * j) * B + myp) * A.Gp + gi] = sr;
              A.partials[((size_t)(RA + 2 * j + 1) * B + myp) * A.Gp + gi] = si;
            }
          }
        }
      grid.sync();
      if (me && k) own_totals(A, RA, 2 * k, myp, tot);
      // w -= sum_j beta_j w_j, then ||w||^2 and <w, r>
      if (me) {
        v[0] = v[1] = v[2] = 0.0;
        for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          float2 x = Wk[e];
          for (int j = 0; j < k; j++) {
            const float2 q = A.W[(size_t)j * A.ntot + A.off[myp] + e];
            const float br = (float)tot[2 * j], bi = (float)tot[2 * j + 1];
            x.x -= br * q.x - bi * q.y;
            x.y -= br * q.y + bi * q.x;
          }
          Wk[e] = x;
          const float2 rr = r[e];
          v[0] += (double)x.x * x.x + (double)x.y * x.y;
          v[1] += (double)x.x * rr.x + (double)x.y * rr.y;
          v[2] += (double)x.x * rr.y - (double)x.y * rr.x;
        }
        if (gi == 0)
          for (int j = threadIdx.x; j < k; j += blockDim.x) {
            beta[(j + (size_t)m * k) * 2] = tot[2 * j];
            beta[(j + (size_t)m * k) * 2 + 1] = tot[2 * j + 1];
          }
        own_partials(A, v, 3, RB, myp, gi, sred);
      }
      grid.sync();
      if (me) {
        own_totals(A, RB, 3, myp, tot);
        const double g = tot[0] > 0 ? sqrt(tot[0]) : 1.0;
        const double ar = tot[1] / g, ai = tot[2] / g;
        if (gi == 0 && threadIdx.x == 0) {
          alpha[2 * k] = ar;
          alpha[2 * k + 1] = ai;
          gam[k] = g;
        }
        const float ig = (float)(1.0 / g), far = (float)ar, fai = (float)ai;
        v[0] = 0.0;
        for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          float2 x = Wk[e];
          x.x *= ig;
          x.y *= ig;
          Wk[e] = x;
          float2 rr = r[e];
          rr.x -= far * x.x - fai * x.y;
          rr.y -= far * x.y + fai * x.x;
          r[e] = rr;
          v[0] += (double)rr.x * rr.x + (double)rr.y * rr.y;
        }
        own_partials(A, v, 1, RC, myp, gi, sred);
      }
      grid.sync();
      all_totals(A, RC, allv);
      k++;
      its++;
      if (me) kmy = k;
      if (threadIdx.x == 0)
        for (int p = 0; p < B; p++)
          if ((run >> p) & 1u) scount[p]++;
      unsigned next = run;
      for (int p = 0; p < B; p++) {
        if (!((run >> p) & 1u)) continue;
        const double rn = sqrt(allv[p]);
        if (!(rn == rn)) {
          if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&A.flags[FLAG_NAN], 1);
          next &= ~(1u << p);
          act &= ~(1u << p);
        } else if (rn <= stol[p]) {
          next &= ~(1u << p);
        }
      }
      run = next;
    }
    // back substitution of this CTA's system and y += sum c_j z_j
    if (mine && kmy > 0) {
      if (threadIdx.x == 0) {
        for (int j = kmy - 1; j >= 0; j--) {
          double re = alpha[2 * j], im = alpha[2 * j + 1];
          for (int l = j + 1; l < kmy; l++) {
            const double br = beta[(j + (size_t)m * l) * 2], bi = beta[(j + (size_t)m * l) * 2 + 1];
            re -= br * cc[2 * l] - bi * cc[2 * l + 1];
            im -= br * cc[2 * l + 1] + bi * cc[2 * l];
          }
          cc[2 * j] = re / gam[j];
          cc[2 * j + 1] = im / gam[j];
        }
      }
      __syncthreads();
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 yy = y[e];
        double re = yy.x, im = yy.y;
        for (int j = 0; j < kmy; j++) {
          const float2 z = A.Z[(size_t)j * A.ntot + A.off[myp] + e];
          re += cc[2 * j] * z.x - cc[2 * j + 1] * z.y;
          im += cc[2 * j] * z.y + cc[2 * j + 1] * z.x;
        }
        y[e] = make_float2((float)re, (float)im);
      }
    }
    grid.sync();
    // true residuals r_p = rhs_p - A y_p of the systems still active
    mapply<ST>(A, act, slist, grid, Vec{V_R, 0}, Vec{V_Y, 0}, sm);
    grid.sync();
    if (mine && ((act >> myp) & 1u)) {
      v[0] = 0.0;
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const float2 ay = r[e], bb = rhsp[e];
        const float2 rr = make_float2(bb.x - ay.x, bb.y - ay.y);
        r[e] = rr;
        v[0] += (double)rr.x * rr.x + (double)rr.y * rr.y;
      }
      own_partials(A, v, 1, RD, myp, gi, sred);
    }
    grid.sync();
    all_totals(A, RD, allv);
    unsigned next = act;
    for (int p = 0; p < B; p++) {
      if (!((act >> p) & 1u)) continue;
      const double rn = sqrt(allv[p]);
      if (rn <= stol[p] || !(rn == rn)) next &= ~(1u << p);
    }
    act = next;
  }
  // reconstruction of every system
  if (A.eo) {
    msite_inv(A, allm, slist, R_EVEN, Vec{V_X, 0}, Vec{V_Y, 0}, sm);                           // x_e = X_e^{-1} y_e
    grid.sync();
    msites<ST>(A, allm, slist, L_Y, R_ODD, true, Vec{V_TB, 0}, Vec{V_X, 0}, Vec{V_B, 0}, sm);   // t_o = b_o - Y_oe x_e
    grid.sync();
    msite_inv(A, allm, slist, R_ODD, Vec{V_X, 0}, Vec{V_TB, 0}, sm);                           // x_o = X_o^{-1} t_o
  } else if (mine) {
    float2* xp = A.x[myp];
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) xp[e] = y[e];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int p = 0; p < B; p++) atomicAdd(reinterpret_cast<unsigned long long*>(A.iters[p]), (unsigned long long)scount[p]);
}

size_t multi_smem(int maxnc, int nb) {
  return sizeof(double) * (64 + kNR + 2 * kMaxBatch + 2 * kMaxRestart + kMaxBatch) +
         sizeof(float2) * (size_t)nb * 9 * maxnc;
}

// co-resident grid per (kernel, batch size, largest nc)
std::map<std::tuple<const void*, int, int>, int> g_per_sm;
}  // namespace

int coarse_gcr_batch_max() { return kMaxBatch; }
int coarse_gcr_group_max() { return kMaxGroups; }

void coarse_gcr_solve_multi(const std::vector<CoarseSystem>& sys, CoarseGCRBuffers& Bf, int m, int maxit,
                            int* flags, cudaStream_t s) {
  const int nb = (int)sys.size();
  if (m > kMaxRestart) raise(MG_ERR_ARG, "coarse restart too long for the persistent solver");
  if (nb < 1 || nb > kMaxBatch) raise(MG_ERR_ARG, "coarse batch size out of range");
  MArgs A;
  std::memset(&A, 0, sizeof(A));
  A.B = nb;
  A.m = m;
  A.maxit = maxit;
  A.flags = flags;
  const int store = sys[0].C->store;
  A.eo = sys[0].G->eo ? 1 : 0;
  size_t ntot = 0, nftot = 0;
  for (int p = 0; p < nb; p++) {
    const LevelGeom& G = *sys[p].G;
    const CoarseOp& C = *sys[p].C;
    if (C.store != store) raise(MG_ERR_ARG, "batched coarse systems must share the link storage format");
    if ((G.eo ? 1 : 0) != A.eo) raise(MG_ERR_ARG, "batched coarse systems must all (or none) be even-odd");
    if (!C.A.get()) raise(MG_ERR_STATE, "folded coarse links missing");
    int gi = -1;
    for (int q = 0; q < A.ng; q++)
      if (A.grp[q].nbr == G.d_nbr.as<int>() && A.grp[q].Y == C.Y.get()) gi = q;
    if (gi < 0) {
      if (A.ng == kMaxGroups) raise(MG_ERR_ARG, "too many coarse lattices in one batch");
      gi = A.ng++;
      Group& g = A.grp[gi];
      g.nc = C.nc;
      g.half = G.half;
      g.nsites = G.nsites;
      g.nbr = G.d_nbr.as<int>();
      g.Y = C.Y.get();
      g.Ys = C.Yscale.as<float>();
      g.Xinv = C.Xinv.as<float2>();
      g.A = C.A.as<float2>();
      g.mask = 0u;
      A.maxnc = std::max(A.maxnc, C.nc);
    }
    A.grp[gi].mask |= 1u << p;
    A.group_of[p] = gi;
    A.tol_rel[p] = sys[p].tol_rel;
    A.nf[p] = (size_t)G.nsites * C.nc;
    A.n[p] = A.eo ? (size_t)G.half * C.nc : A.nf[p];
    A.off[p] = ntot;
    A.offf[p] = nftot;
    ntot += A.n[p];
    nftot += A.nf[p];
    A.b[p] = reinterpret_cast<const float2*>(sys[p].b);
    A.x[p] = reinterpret_cast<float2*>(sys[p].x);
    A.iters[p] = sys[p].iters;
  }
  A.ntot = ntot;
  const size_t smem = multi_smem(A.maxnc, nb);
  const void* kern = store == STORE_F16    ? (const void*)k_coarse_gcr_multi<kStF16>
                     : store == STORE_BF16 ? (const void*)k_coarse_gcr_multi<kStBF16>
                                           : (const void*)k_coarse_gcr_multi<kStF32>;
  int dev = 0, sms = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int& per = g_per_sm[std::make_tuple(kern, nb, A.maxnc)];
  if (per == 0) MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem));
  if (per < 1) raise(MG_ERR_CUDA, "batched coarse GCR cannot be resident");
  const int most = sms * (per < 4 ? per : 4);
  // enough CTAs for the largest stencil phase, at least one per SM, and the
  // same number for every system's element-wise group
  long long sites = 0;
  for (int q = 0; q < A.ng; q++) sites += A.eo ? A.grp[q].half : A.grp[q].nsites;
  int grid = (int)std::min<long long>(most, std::max<long long>(sites, sms));
  A.Gp = grid / nb;
  if (A.Gp < 1) raise(MG_ERR_ARG, "batch larger than the co-resident grid");
  // buffers (grown on demand)
  A.nscal = scalars_per_system(m);
  auto grow = [&](DBuf& d, size_t bytes) {
    if (d.bytes() < bytes) d.alloc(bytes);
  };
  grow(Bf.bx_r, sizeof(float2) * ntot);
  grow(Bf.bx_y, sizeof(float2) * ntot);
  grow(Bf.bx_br, sizeof(float2) * ntot);
  if (Bf.bx_tB.bytes() < sizeof(float2) * nftot) {
    Bf.bx_tB.alloc(sizeof(float2) * nftot);
    MG_CUDA(cudaMemsetAsync(Bf.bx_tB.get(), 0, sizeof(float2) * nftot, s));
  }
  grow(Bf.bx_W, sizeof(float2) * ntot * m);
  grow(Bf.bx_Z, sizeof(float2) * ntot * m);
  grow(Bf.bx_part, sizeof(double) * (size_t)kNR * nb * A.Gp);
  grow(Bf.bx_scal, sizeof(double) * A.nscal * nb);
  A.r = Bf.bx_r.as<float2>();
  A.y = Bf.bx_y.as<float2>();
  A.br = Bf.bx_br.as<float2>();
  A.tB = Bf.bx_tB.as<float2>();
  A.W = Bf.bx_W.as<float2>();
  A.Z = Bf.bx_Z.as<float2>();
  A.partials = Bf.bx_part.as<double>();
  A.scal = Bf.bx_scal.as<double>();
  void* params[] = {&A};
  MG_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kThreads), params, smem, s));
  MG_LAUNCH();
}

void coarse_gcr_solve_batch(const LevelGeom& G, const CoarseOp& C, CoarseGCRBuffers& Bf, int m, int maxit,
                            double tol_rel, int nb, const float* b, float* x, long long* d_iters, int* flags,
                            cudaStream_t s) {
  std::vector<CoarseSystem> sys(nb);
  const size_t nfull = (size_t)G.nsites * C.nc;
  for (int p = 0; p < nb; p++) sys[p] = CoarseSystem{&G, &C, b + 2 * nfull * p, x + 2 * nfull * p, tol_rel, d_iters};
  coarse_gcr_solve_multi(sys, Bf, m, maxit, flags, s);
}

}  // namespace mg
