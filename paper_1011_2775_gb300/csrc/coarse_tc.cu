// The coarsest-level GCR of up to 16 systems of one even-odd coarse lattice on
// tensor cores (links stored in FP16).
//
// Section "Implementation": the coarsest lattice is solved by unpreconditioned
// GCR to a residual tolerance relative to its right-hand side; section
// "Red-black preconditioning": through its reduced even-odd system, here in
// unfolded form
//   D_r y = y - Y_eo t,   t = X_o^{-1} Y_oe s,   s = X_e^{-1} y,
// which is exactly the operator of the stored (dequantised) Y and the FP32
// site inverses.  The coarse operator looks like a staggered operator with
// Nc = 2 Nv colours ("Implementation"); applied to nb right-hand sides at once
// its link blocks form a real dense contraction, so the hop terms run on
// mma.sync.m16n8k16 with FP16 operands and FP32 accumulation:
//
//  * complex arithmetic in real form: an M tile is 8 complex link rows, its
//    16 real rows are the real and the imaginary row of each, built in
//    registers from the stored (re, im) FP16 pairs (a sign flip and a half
//    swap); the vectors are the B operand, one FP16 (re, im) pair per element;
//  * every vector is multiplied by a power-of-two scale per system (its
//    largest component maps to [0.5, 1)) and split into FP16 hi + lo parts, so
//    the product keeps about 22 bits; the tile scale of Y (per site and
//    direction) is folded in before the split;
//  * a block owns whole sites for the hop phases (its link rows stream through
//    two shared-memory stages per warp by cp.async.bulk, one row per copy into
//    rows padded by 16 bytes so the fragment loads are free of bank
//    conflicts), and whole sites of one system for the element-wise phases,
//    so the site inverses X^{-1} act on complete sites locally;
//  * one iteration: hop phase A (t on odd sites) | barrier | hop phase B
//    (w = r - Y_eo t) | barrier | Gram-Schmidt dots | barrier | projection of
//    w and z, with the norm of the projected w | barrier | update of w, z, y, r
//    and s = X_e^{-1} r | barrier.  Reductions are double-float on the FP32
//    pipes and deterministic; maxima (for the vector scales) go through
//    integer atomics, which are exact.
// Every wait is bounded in time (async_copy.cuh); FLAG_TIMEOUT on expiry.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "async_copy.cuh"
#include "coarse.h"
#include "coarse_dev.cuh"
#include "dfloat.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRestart = 64;
constexpr int kMaxSys = 16;
constexpr int kTile = 8;         // complex rows of an M tile (16 real rows of m16n8k16)
constexpr int kPad = 4;          // 32-bit words of padding per staged row
constexpr int kSplit = 2;        // FP16 hi + lo
// per-system reduction slots of the element-wise phases
constexpr int kDot = 2 * kMaxRestart;       // beta (2k)
constexpr int QR = kDot;                    // ||r||^2 (also ||b||^2 at the start)
constexpr int QE = QR + 1;                  // ||w''||^2, Re/Im <w'', r> of the projected w
constexpr int kSlots = QE + 3;

struct TArgs {
  int nc, half, m, maxit, nb, MT, pitch;   // pitch: 32-bit words per staged row (M tiles MT = nc / 8)
  int Gp;                                   // blocks per system in the element-wise phases
  float tol_rel[kMaxSys];
  const int* nbr;
  const unsigned* Y;        // FP16 (re, im) pairs: [site][nc][8 nc]
  const float* Ys;          // [site][8]
  const float2* Xinv;       // [site][nc][nc]
  const float2* b;          // system p: full vector at b + p * bstride
  size_t bstride;
  float2* x;                // system p: full solution at x + p * xstride
  size_t xstride;
  float2 *y, *r, *br, *s, *sy;   // [p][n], n = half nc (even sites)
  float2 *t, *tb;                // [p][n] (odd sites, local index)
  float2 *W, *Z;                 // [j][p][n]
  float2* part;                  // [slot][p][Gp] double-float partial sums
  unsigned* vmax;                // [2][kMaxSys]: max |component| of s (0) and t (1), float bits
  long long* iters;
  int* flags;
  unsigned* bar;
  int* abort;
};

__device__ __forceinline__ unsigned h2_bits(__half2 h) { return *reinterpret_cast<unsigned*>(&h); }

// the m16n8k16 FP16 MMA with FP32 accumulation
__device__ __forceinline__ void mma16816(float c[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// power-of-two scale mapping a largest magnitude m into [0.5, 1)
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
  int e;
  frexpf(m, &e);
  return ldexpf(1.f, -e);
}

// stage of warp position p; item of a warp position: (kind, site)
struct Stream {
  unsigned char* ring;
  uint64_t* full;
  int e0, e1, o0, o1;   // the block's even and odd sites (local index)
  long long t;          // this warp's next sequence position
};

__device__ __forceinline__ void seq_site(const Stream& st, long long p, int& kind, int& site) {
  const int nA = st.o1 - st.o0, nB = st.e1 - st.e0;
  if (p < nB) {
    kind = 1;
    site = st.e0 + (int)p;
    return;
  }
  const int off = (int)((p - nB) % (nA + nB));
  if (off < nA) {
    kind = 0;
    site = st.o0 + off;
  } else {
    kind = 1;
    site = st.e0 + off - nA;
  }
}

// lane 0 of warp w: the rows of M tile w of the position's site, one bulk copy
// per row into the padded stage
__device__ __forceinline__ void issue(const TArgs& a, const Stream& st, long long p, int stage_bytes, int spw) {
  const int w = threadIdx.x >> 5;
  if (st.o1 - st.o0 + st.e1 - st.e0 == 0) return;
  int kind, site;
  seq_site(st, p, kind, site);
  const int nc = a.nc, K = 8 * nc;
  const int storage = kind == 0 ? a.half + site : site;
  const int stage = w * spw + (int)(p % spw);
  unsigned char* dst = st.ring + (size_t)stage * stage_bytes;
  const unsigned row_bytes = (unsigned)K * 4u;
  mbar_arrive_expect_tx(&st.full[stage], row_bytes * kTile);
  for (int r = 0; r < kTile; r++) {
    const unsigned* src = a.Y + ((size_t)storage * nc + w * kTile + r) * K;
    bulk_copy_g2s(dst + (size_t)r * a.pitch * 4, src, row_bytes, &st.full[stage]);
  }
}

// Gathers the vectors of `site` (storage index) for the nb systems: the 8
// neighbours' nc components of in_p (neighbour storage index nbr at element
// (nbr - nbase) nc of in_p), times the tile scale of Y and the system's
// power-of-two scale, split into FP16 hi and lo parts: gv[split][p][pitch
// words].  Systems nb .. NB-1 are zero.
template <int NB>
__device__ void gather(const TArgs& a, int site, const float2* in, size_t instride, int nbase, const float* sc,
                       unsigned* gv) {
  const int nc = a.nc, K = 8 * nc;
  const int total = NB * K;
  // four elements per thread and round: their indices and scales, then their
  // loads, are in flight together
  constexpr int U = 4;
  for (int q0 = threadIdx.x; q0 < total; q0 += U * blockDim.x) {
    size_t src[U];
    float f[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int q = q0 + u * blockDim.x;
      const int qq = q < total ? q : 0;
      const int p = qq / K, rem = qq - p * K, d = rem / nc, j = rem - d * nc;
      live[u] = q < total && p < a.nb;
      src[u] = live[u] ? (size_t)p * instride + (size_t)(a.nbr[(size_t)site * 8 + d] - nbase) * nc + j : 0;
      f[u] = live[u] ? a.Ys[(size_t)site * 8 + d] * sc[p] : 0.f;
    }
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; u++) v[u] = live[u] ? __ldcg(in + src[u]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int q = q0 + u * blockDim.x;
      if (q >= total) continue;
      const int p = q / K, rem = q - p * K;
      unsigned hi = 0u, lo = 0u;
      if (live[u]) {
        const float2 x = make_float2(v[u].x * f[u], v[u].y * f[u]);
        const __half2 h = __floats2half2_rn(x.x, x.y);
        const float2 hf = __half22float2(h);
        hi = h2_bits(h);
        lo = h2_bits(__floats2half2_rn(x.x - hf.x, x.y - hf.y));
      }
      gv[(size_t)p * a.pitch + rem] = hi;
      gv[((size_t)NB + p) * a.pitch + rem] = lo;
    }
  }
  __syncthreads();
}

// M tile w of a staged site times the gathered vectors: acc[nt][4] as the
// m16n8k16 C fragments (rows: real parts of the tile's rows 0-7, then their
// imaginary parts; columns: systems 8 nt + 0..7)
template <int NB>
__device__ __forceinline__ void tile_mma(const TArgs& a, const unsigned* stage, const unsigned* gv, float acc[NB / 8][4]) {
  constexpr int NT = NB / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int K = 8 * a.nc;
#pragma unroll
  for (int nt = 0; nt < NT; nt++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
  const unsigned* arow = stage + (size_t)g * a.pitch + t;
  const unsigned* brow = gv + (size_t)g * a.pitch + t;
#pragma unroll 2
  for (int kc = 0; kc < K; kc += 8) {
    const unsigned w0 = arow[kc], w1 = arow[kc + 4];
    const unsigned a0 = w0 ^ 0x80000000u, a1 = __byte_perm(w0, 0, 0x1032);
    const unsigned a2 = w1 ^ 0x80000000u, a3 = __byte_perm(w1, 0, 0x1032);
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
#pragma unroll
      for (int sp = 0; sp < kSplit; sp++) {
        const unsigned* bp = brow + ((size_t)sp * NB + nt * 8) * a.pitch;
        mma16816(acc[nt], a0, a1, a2, a3, bp[kc], bp[kc + 4]);
      }
    }
  }
}

// one hop phase over the block's sites of `kind` (0: odd sites, Y_oe; 1:
// even sites, Y_eo): per site the gather, the M tiles on warps 0 .. MT-1 with
// epi(site, p, row, value) for every (system, row), then done(site) on the
// whole block; false on a timeout (uniform)
template <int NB, typename Epi, typename Done>
__device__ bool hop_phase(const TArgs& a, Stream& st, int kind, const float2* in, const float* sc, unsigned* gv,
                          int stage_bytes, int spw, int* s_fail, Epi epi, Done done) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int s0 = kind ? st.e0 : st.o0, s1 = kind ? st.e1 : st.o1;
  const size_t n = (size_t)a.half * a.nc;
  for (int site = s0; site < s1; site++) {
    const int storage = kind ? site : a.half + site;
    gather<NB>(a, storage, in, n, kind ? a.half : 0, sc, gv);
    if (w < a.MT) {
      const int stage = w * spw + (int)(st.t % spw);
      const unsigned par = (unsigned)((st.t / spw) & 1);
      if (!mbar_wait(&st.full[stage], par)) {
        atomicExch(s_fail, 1);
      } else {
        float acc[NB / 8][4];
        tile_mma<NB>(a, reinterpret_cast<const unsigned*>(st.ring + (size_t)stage * stage_bytes), gv, acc);
        const int row = w * kTile + g;
#pragma unroll
        for (int nt = 0; nt < NB / 8; nt++)
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const int p = nt * 8 + 2 * t + h;
            if (p < a.nb) {
              const float inv = 1.f / sc[p];
              epi(site, p, row, make_float2(acc[nt][h] * inv, acc[nt][2 + h] * inv));
            }
          }
        __syncwarp();
        if (lane == 0) issue(a, st, st.t + spw, stage_bytes, spw);
        st.t++;
      }
    }
    __syncthreads();
    if (*(volatile int*)s_fail) return false;
    done(site);
  }
  return true;
}

// out = X in for the nc x nc site block X (global) and np vectors in shared
// memory (in[p][nc]); every output element goes to f(p, i, value)
template <typename F>
__device__ void site_gemv(const TArgs& a, const float2* X, const float2* in, int np, F f) {
  const int nc = a.nc;
  for (int q = threadIdx.x; q < np * nc; q += blockDim.x) {
    const int p = q / nc, i = q - p * nc;
    const float2* xr = X + (size_t)i * nc;
    const float2* v = in + (size_t)p * nc;
    float re = 0.f, im = 0.f;
    for (int j = 0; j < nc; j++) {
      const float2 m = xr[j], x = v[j];
      re = fmaf(m.x, x.x, fmaf(-m.y, x.y, re));
      im = fmaf(m.x, x.y, fmaf(m.y, x.x, im));
    }
    f(p, i, make_float2(re, im));
  }
}

__device__ __forceinline__ void atomic_fmax(unsigned* addr, float2 u) {
  // non-negative floats order like their bit patterns
  atomicMax(addr, __float_as_uint(fmaxf(fabsf(u.x), fabsf(u.y))));
}

// block partial sums (double-float) of nq per-thread floats of system p,
// stored at part[q0 + q][p][gi]
__device__ void block_partials(const TArgs& a, const float* v, int nq, int q0, int p, int gi, df* sred) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < nq; q++) {
    const df u = df_wsum(df_of(v[q]));
    if (lane == 0) sred[q * kWarps + wid] = u;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    df s = sred[q * kWarps];
    for (int w = 1; w < kWarps; w++) s = df_add(s, sred[q * kWarps + w]);
    a.part[((size_t)(q0 + q) * kMaxSys + p) * a.Gp + gi] = make_float2(s.h, s.l);
  }
  __syncthreads();
}

// totals of slots [q0, q0 + nq) of system p (one warp per slot)
__device__ void sys_totals(const TArgs& a, int q0, int nq, int p, df* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = wid; q < nq; q += kWarps) {
    const float2* src = a.part + ((size_t)(q0 + q) * kMaxSys + p) * a.Gp;
    df s = df_of(0.f);
    for (int g = lane; g < a.Gp; g += 32) {
      const float2 x = __ldcg(src + g);
      s = df_add(s, df{x.x, x.y});
    }
    s = df_wsum(s);
    if (lane == 0) out[q] = s;
  }
  __syncthreads();
}

// slot q of every system into out[p] (warp w sums systems w, w + 8)
__device__ void all_totals(const TArgs& a, int q, df* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int p = wid; p < a.nb; p += kWarps) {
    df s = df_of(0.f);
    for (int g = lane; g < a.Gp; g += 32) {
      const float2 x = __ldcg(a.part + ((size_t)q * kMaxSys + p) * a.Gp + g);
      s = df_add(s, df{x.x, x.y});
    }
    s = df_wsum(s);
    if (lane == 0) out[p] = s;
  }
  __syncthreads();
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 1) k_coarse_gcr_tc(TArgs a, int stage_bytes, int spw) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kWarps * 2];
  __shared__ float s_sc[2][kMaxSys];        // vector scales of the hop inputs: s / sy (0), t (1)
  __shared__ float2 s_beta[kMaxRestart];
  __shared__ float s_coef[4];
  __shared__ float s_tol2[kMaxSys];
  __shared__ int s_fail;
  __shared__ unsigned s_act, s_run;
  const int nc = a.nc, m = a.m;
  const int G = gridDim.x, bid = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t n = (size_t)a.half * nc;
  // shared memory: stages | gathered vectors | site buffer | reductions
  unsigned* gv = reinterpret_cast<unsigned*>(smem + (size_t)a.MT * spw * stage_bytes);
  float2* sbuf = reinterpret_cast<float2*>(gv + (size_t)kSplit * NB * a.pitch);   // [NB][nc]
  df* sred = reinterpret_cast<df*>(sbuf + (size_t)NB * nc);                       // [kSlots][kWarps]
  df* tot = sred + (size_t)kSlots * kWarps;                                        // [kSlots]

  Stream st;
  st.ring = smem;
  st.full = full;
  st.e0 = (int)((long long)bid * a.half / G);
  st.e1 = (int)((long long)(bid + 1) * a.half / G);
  st.o0 = st.e0;
  st.o1 = st.e1;
  st.t = 0;
  // element-wise ownership: system myp, its sites [q0, q1)
  const int myp = bid / a.Gp, gi = bid % a.Gp;
  const bool mine = myp < a.nb;
  const int q0 = mine ? (int)((long long)gi * a.half / a.Gp) : 0;
  const int q1 = mine ? (int)((long long)(gi + 1) * a.half / a.Gp) : 0;
  const size_t E0 = (size_t)q0 * nc, E1 = (size_t)q1 * nc;
  const size_t pn = (size_t)(mine ? myp : 0) * n;
  float2* r = a.r + pn;
  float2* y = a.y + pn;
  auto Wj = [&](int j) { return a.W + ((size_t)j * a.nb) * n + pn; };
  auto Zj = [&](int j) { return a.Z + ((size_t)j * a.nb) * n + pn; };
  unsigned target = 0;
  int ep = 0;   // max-reduction epoch: buffer ep % 4 of vmax
  bool ok = true;
  float v[4];
  auto vmax_slot = [&](int e, int p) { return a.vmax + (size_t)(e & 3) * kMaxSys + p; };
  // after the barrier that ends epoch ep's maxima: read them into scale slot
  // `which`, clear the buffer of epoch ep + 2, advance
  auto take_max = [&](int which) {
    if (threadIdx.x < a.nb) s_sc[which][threadIdx.x] = pow2_scale(__uint_as_float(__ldcg(vmax_slot(ep, threadIdx.x))));
    if (bid == 0 && threadIdx.x < kMaxSys) *vmax_slot(ep + 2, threadIdx.x) = 0u;
    ep++;
    __syncthreads();
  };
  // X_e^{-1} applied to the owned sites of vector src (system myp) into dst, maxima into epoch ep
  auto even_inverse = [&](const float2* src, float2* dst) {
    for (int site = q0; site < q1; site++) {
      for (int q = threadIdx.x; q < nc; q += blockDim.x) sbuf[q] = __ldcg(src + (size_t)site * nc + q);
      __syncthreads();
      site_gemv(a, a.Xinv + (size_t)site * nc * nc, sbuf, 1, [&](int, int i, float2 u) {
        dst[(size_t)site * nc + i] = u;
        atomic_fmax(vmax_slot(ep, myp), u);
      });
      __syncthreads();
    }
  };
  // the odd-site hop phase: t = X_o^{-1} Y_oe in (maxima into epoch ep)
  auto phase_a = [&](const float2* in) {
    return hop_phase<NB>(
        a, st, 0, in, s_sc[0], gv, stage_bytes, spw, &s_fail,
        [&](int, int p, int row, float2 u) { sbuf[(size_t)p * nc + row] = u; },
        [&](int site) {
          site_gemv(a, a.Xinv + (size_t)(a.half + site) * nc * nc, sbuf, a.nb, [&](int p, int i, float2 u) {
            a.t[(size_t)p * n + (size_t)site * nc + i] = u;
            atomic_fmax(vmax_slot(ep, p), u);
          });
          __syncthreads();
        });
  };

  if (threadIdx.x == 0) {
    for (int q = 0; q < a.MT * spw; q++) mbar_init(&full[q], 1);
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  if (lane == 0 && wid < a.MT)
    for (long long p = 0; p < spw; p++) issue(a, st, p, stage_bytes, spw);

  // ---- start: tb = t = X_o^{-1} b_o on the block's odd sites (all systems)
  for (int site = st.o0; site < st.o1; site++) {
    const int o = a.half + site;
    for (int q = threadIdx.x; q < a.nb * nc; q += blockDim.x) {
      const int p = q / nc, j = q - p * nc;
      sbuf[q] = a.b[(size_t)p * a.bstride + (size_t)o * nc + j];
    }
    __syncthreads();
    site_gemv(a, a.Xinv + (size_t)o * nc * nc, sbuf, a.nb, [&](int p, int i, float2 u) {
      a.tb[(size_t)p * n + (size_t)site * nc + i] = u;
      a.t[(size_t)p * n + (size_t)site * nc + i] = u;
      atomic_fmax(vmax_slot(ep, p), u);
    });
    __syncthreads();
  }
  // ||b_p||^2 over the full vector, on the system's element-wise blocks
  if (mine) {
    const size_t nf = 2 * n, cf = (nf + a.Gp - 1) / a.Gp;
    const size_t f0 = (size_t)gi * cf, f1 = f0 + cf < nf ? f0 + cf : nf;
    v[0] = 0.f;
    for (size_t e = f0 + threadIdx.x; e < f1; e += blockDim.x) {
      const float2 q = a.b[(size_t)myp * a.bstride + e];
      v[0] = fmaf(q.x, q.x, fmaf(q.y, q.y, v[0]));
    }
    block_partials(a, v, 1, QR, myp, gi, sred);
  }
  ok = grid_barrier(a.bar, a.abort, target);
  // ---- b_r = b_e - Y_eo t on the block's even sites: r = b_r, y = 0
  if (ok) {
    take_max(1);
    ok = hop_phase<NB>(
        a, st, 1, a.t, s_sc[1], gv, stage_bytes, spw, &s_fail,
        [&](int site, int p, int row, float2 u) {
          const size_t i = (size_t)site * nc + row;
          const float2 bb = a.b[(size_t)p * a.bstride + i];
          const float2 o = make_float2(bb.x - u.x, bb.y - u.y);
          a.br[(size_t)p * n + i] = o;
          a.r[(size_t)p * n + i] = o;
          a.y[(size_t)p * n + i] = make_float2(0.f, 0.f);
          a.sy[(size_t)p * n + i] = make_float2(0.f, 0.f);
        },
        [](int) {});
  }
  if (ok) ok = grid_barrier(a.bar, a.abort, target);
  // ---- s = X_e^{-1} r on the owned sites; then the tolerances and the scale of s
  if (ok && mine) even_inverse(r, a.s + pn);
  if (ok) ok = grid_barrier(a.bar, a.abort, target);
  if (ok) {
    all_totals(a, QR, tot);
    if (threadIdx.x < a.nb)
      s_tol2[threadIdx.x] = a.tol_rel[threadIdx.x] * a.tol_rel[threadIdx.x] * (tot[threadIdx.x].h + tot[threadIdx.x].l);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned act = 0u;
      for (int p = 0; p < a.nb; p++)
        if (s_tol2[p] > 0.f) act |= 1u << p;
      s_act = act;
    }
    take_max(0);
  }
  long long its = 0;
  while (ok && s_act && its < a.maxit) {
    int k = 0;
    if (threadIdx.x == 0) s_run = s_act;
    __syncthreads();
    while (k < m && its < a.maxit && s_run) {
      const bool me = mine && ((s_run >> myp) & 1u);
      // A: t = X_o^{-1} Y_oe s on the block's odd sites
      if (!(ok = phase_a(a.s))) break;
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      take_max(1);
      // B: w = r - Y_eo t on the block's even sites
      float2* Wk = a.W + ((size_t)k * a.nb) * n;
      if (!(ok = hop_phase<NB>(
                a, st, 1, a.t, s_sc[1], gv, stage_bytes, spw, &s_fail,
                [&](int site, int p, int row, float2 u) {
                  const size_t i = (size_t)p * n + (size_t)site * nc + row;
                  const float2 rr = __ldcg(a.r + i);
                  Wk[i] = make_float2(rr.x - u.x, rr.y - u.y);
                },
                [](int) {})))
        break;
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      // dots of the owned slice: beta_j = <w_j, w> (warp wid owns j = wid + 8 u), ||w||^2, <w, r>
      float2* wk = Wj(k);
      if (me) {
        for (int jb = wid; jb < k; jb += 4 * kWarps) {
          float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
          for (size_t e = E0 + lane; e < E1; e += 32) {
            const float2 x = __ldcg(wk + e);
#pragma unroll
            for (int u = 0; u < 4; u++) {
              const int j = jb + u * kWarps;
              const float2 q = j < k ? Wj(j)[e] : make_float2(0.f, 0.f);
              re[u] = fmaf(q.x, x.x, fmaf(q.y, x.y, re[u]));
              im[u] = fmaf(q.x, x.y, fmaf(-q.y, x.x, im[u]));
            }
          }
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int j = jb + u * kWarps;
            const df sr = df_wsum(df_of(re[u])), si = df_wsum(df_of(im[u]));
            if (lane == 0 && j < k) {
              a.part[((size_t)(2 * j) * kMaxSys + myp) * a.Gp + gi] = make_float2(sr.h, sr.l);
              a.part[((size_t)(2 * j + 1) * kMaxSys + myp) * a.Gp + gi] = make_float2(si.h, si.l);
            }
          }
        }
      }
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      // coefficients of the own system: beta_j, then w'' = w - sum beta_j w_j and
      // z'' = r - sum beta_j z_j on the slice with the exact ||w''||^2, <w'', r>
      // (classical Gram-Schmidt with the norm taken after the projection)
      float2* zk = Zj(k);
      if (me) {
        if (k) sys_totals(a, 0, 2 * k, myp, tot);
        if (threadIdx.x < k)
          s_beta[threadIdx.x] = make_float2(tot[2 * threadIdx.x].h + tot[2 * threadIdx.x].l,
                                            tot[2 * threadIdx.x + 1].h + tot[2 * threadIdx.x + 1].l);
        __syncthreads();
        v[0] = v[1] = v[2] = 0.f;
        for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x) {
          float2 x = __ldcg(wk + e);
          const float2 rr = __ldcg(r + e);
          float2 z = rr;
          // four independent partial sums over j, loads of four j issued together
          float sw[4][2] = {}, sz[4][2] = {};
          int j = 0;
          for (; j + 4 <= k; j += 4) {
            float2 q[4], zq[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
              q[u] = Wj(j + u)[e];
              zq[u] = Zj(j + u)[e];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
              const float2 bj = s_beta[j + u];
              sw[u][0] += bj.x * q[u].x - bj.y * q[u].y;
              sw[u][1] += bj.x * q[u].y + bj.y * q[u].x;
              sz[u][0] += bj.x * zq[u].x - bj.y * zq[u].y;
              sz[u][1] += bj.x * zq[u].y + bj.y * zq[u].x;
            }
          }
          for (; j < k; j++) {
            const float2 bj = s_beta[j], q = Wj(j)[e], zq = Zj(j)[e];
            sw[0][0] += bj.x * q.x - bj.y * q.y;
            sw[0][1] += bj.x * q.y + bj.y * q.x;
            sz[0][0] += bj.x * zq.x - bj.y * zq.y;
            sz[0][1] += bj.x * zq.y + bj.y * zq.x;
          }
          x.x -= (sw[0][0] + sw[1][0]) + (sw[2][0] + sw[3][0]);
          x.y -= (sw[0][1] + sw[1][1]) + (sw[2][1] + sw[3][1]);
          z.x -= (sz[0][0] + sz[1][0]) + (sz[2][0] + sz[3][0]);
          z.y -= (sz[0][1] + sz[1][1]) + (sz[2][1] + sz[3][1]);
          wk[e] = x;
          zk[e] = z;
          v[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, v[0]));
          v[1] = fmaf(x.x, rr.x, fmaf(x.y, rr.y, v[1]));
          v[2] = fmaf(x.x, rr.y, fmaf(-x.y, rr.x, v[2]));
        }
        block_partials(a, v, 3, QE, myp, gi, sred);
      }
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      // gamma = ||w''||, alpha = <w'', r> / gamma; w_k = w'' / gamma, z_k = z'' / gamma,
      // y += alpha z_k, r -= alpha w_k; s = X_e^{-1} r
      if (me) {
        sys_totals(a, QE, 3, myp, tot + QE);
        if (threadIdx.x == 0) {
          const df g = df_sqrt(tot[QE]);
          const bool gz = !(g.h > 0.f);
          s_coef[0] = gz ? 1.f : 1.f / g.h;
          const df ar = gz ? tot[QE + 1] : df_div(tot[QE + 1], g);
          const df ai = gz ? tot[QE + 2] : df_div(tot[QE + 2], g);
          s_coef[1] = ar.h + ar.l;
          s_coef[2] = ai.h + ai.l;
        }
        __syncthreads();
        const float ig = s_coef[0], far = s_coef[1], fai = s_coef[2];
        v[0] = 0.f;
        for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x) {
          float2 x = wk[e], z = zk[e];
          x.x *= ig;
          x.y *= ig;
          z.x *= ig;
          z.y *= ig;
          wk[e] = x;
          zk[e] = z;
          float2 yy = __ldcg(y + e);
          yy.x += far * z.x - fai * z.y;
          yy.y += far * z.y + fai * z.x;
          y[e] = yy;
          float2 rr = __ldcg(r + e);
          rr.x -= far * x.x - fai * x.y;
          rr.y -= far * x.y + fai * x.x;
          r[e] = rr;
          v[0] = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, v[0]));
        }
        block_partials(a, v, 1, QR, myp, gi, sred);
        even_inverse(r, a.s + pn);
      }
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      // every block: residual norms and cancellations of all systems, the scale of s
      all_totals(a, QR, tot);
      if (threadIdx.x < a.nb && ((s_run >> threadIdx.x) & 1u)) {
        const int p = threadIdx.x;
        const df rn2 = tot[p];
        bool stop = rn2.h <= s_tol2[p];
        if (!(rn2.h == rn2.h)) {
          stop = true;
          atomicExch(&a.flags[FLAG_NAN], 1);
        }
        if (stop) atomicAnd(&s_run, ~(1u << p));
      }
      take_max(0);
      k++;
      its++;
    }
    if (!ok) break;
    // ---- end of the Krylov cycle: true residual r = b_r - D_r y of the active systems
    if (mine && ((s_act >> myp) & 1u)) even_inverse(y, a.sy + pn);
    if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
    take_max(0);
    if (!(ok = phase_a(a.sy))) break;
    if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
    take_max(1);
    if (!(ok = hop_phase<NB>(
              a, st, 1, a.t, s_sc[1], gv, stage_bytes, spw, &s_fail,
              [&](int site, int p, int row, float2 u) {
                const size_t i = (size_t)p * n + (size_t)site * nc + row;
                const float2 yy = __ldcg(a.y + i), bb = __ldcg(a.br + i);
                a.r[i] = make_float2(bb.x - (yy.x - u.x), bb.y - (yy.y - u.y));
              },
              [](int) {})))
      break;
    if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
    if (mine) {
      v[0] = 0.f;
      for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x) {
        const float2 rr = __ldcg(r + e);
        v[0] = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, v[0]));
      }
      block_partials(a, v, 1, QR, myp, gi, sred);
      even_inverse(r, a.s + pn);
    }
    if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
    all_totals(a, QR, tot);
    if (threadIdx.x < a.nb && ((s_act >> threadIdx.x) & 1u)) {
      const int p = threadIdx.x;
      const df rn2 = tot[p];
      if (rn2.h <= s_tol2[p] || !(rn2.h == rn2.h)) atomicAnd(&s_act, ~(1u << p));
    }
    take_max(0);
  }
  // ---- x_e = X_e^{-1} y (sy of the last true residual), x_o = t_b - X_o^{-1} Y_oe x_e (t of it)
  if (ok) {
    if (mine)
      for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x)
        a.x[(size_t)myp * a.xstride + e] = __ldcg(a.sy + pn + e);
    for (int q = threadIdx.x; q < a.nb * (st.o1 - st.o0) * nc; q += blockDim.x) {
      const int p = q / ((st.o1 - st.o0) * nc), i = q - p * (st.o1 - st.o0) * nc;
      const size_t li = (size_t)st.o0 * nc + i;
      const float2 tb = a.tb[(size_t)p * n + li], tt = __ldcg(a.t + (size_t)p * n + li);
      a.x[(size_t)p * a.xstride + n + li] = make_float2(tb.x - tt.x, tb.y - tt.y);
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(&a.flags[FLAG_TIMEOUT], 1);
    atomicExch(a.abort, 1);
  }
  // drain: the copies this warp issued beyond what it consumed land before exit
  if (lane == 0 && wid < a.MT && st.o1 - st.o0 + st.e1 - st.e0 > 0)
    for (long long p = st.t; p < st.t + spw; p++)
      (void)mbar_wait(&full[wid * spw + (int)(p % spw)], (unsigned)((p / spw) & 1));
  if (bid == 0 && threadIdx.x == 0) *a.iters += its;
}

struct Plan {
  int grid, pitch, stage_bytes, spw, MT;
  size_t smem;
};

Plan make_plan(const LevelGeom& G, const CoarseOp& C, int grid, int nb) {
  Plan p;
  const int nc = C.nc, K = 8 * nc;
  const int NB = nb <= 8 ? 8 : 16;
  p.MT = nc / kTile;
  p.pitch = K + kPad;
  p.stage_bytes = kTile * p.pitch * 4;
  p.grid = std::min(grid, std::max(G.half, nb));   // blocks without sites still own element-wise slices
  int dev = 0, optin = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t other = (size_t)kSplit * NB * p.pitch * 4 + sizeof(float2) * (size_t)NB * nc +
                       sizeof(df) * (size_t)kSlots * (kWarps + 1);
  const size_t budget = (size_t)optin - 4096;
  p.spw = 2;
  p.smem = (size_t)p.MT * 2 * p.stage_bytes + other;
  if (p.smem > budget) {
    p.spw = 1;
    p.smem = (size_t)p.MT * p.stage_bytes + other;
  }
  return p;
}

int sm_count() {
  int dev = 0, sms = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

}  // namespace

bool coarse_gcr_tc_ok(const LevelGeom& G, const CoarseOp& C, int nb) {
  if (!G.eo || C.store != STORE_F16 || C.nc % kTile || C.nc > 64 || nb < 1 || nb > kMaxSys) return false;
  int dev = 0, optin = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const Plan p = make_plan(G, C, sm_count(), nb);
  return p.smem + 4096 <= (size_t)optin;
}

std::vector<int> coarse_gcr_tc_grids(const LevelGeom& G, const CoarseOp& C, int nb) {
  const int full = std::min(sm_count(), std::max(G.half, nb));
  std::vector<int> out = {full};
  // the largest grid that splits the sites evenly
  for (int g = full - 1; g >= full / 2 && g >= nb; g--)
    if (G.half % g == 0) {
      out.push_back(g);
      break;
    }
  (void)C;
  return out;
}

bool coarse_gcr_tc_try(const std::vector<CoarseSystem>& sys, CoarseGCRBuffers& B, int m, int maxit, int* flags,
                       cudaStream_t s) {
  const int nb = (int)sys.size();
  if (nb < 1) return false;
  const LevelGeom& G = *sys[0].G;
  const CoarseOp& C = *sys[0].C;
  if (!coarse_gcr_tc_ok(G, C, nb)) return false;
  const size_t nf = G.vec_complex();
  std::vector<double> tols(nb);
  for (int p = 0; p < nb; p++) {
    // one lattice, consecutive vectors, one iteration counter
    if (sys[p].G != sys[0].G || sys[p].C != sys[0].C || sys[p].iters != sys[0].iters ||
        sys[p].b != sys[0].b + 2 * nf * p || sys[p].x != sys[0].x + 2 * nf * p)
      return false;
    tols[p] = sys[p].tol_rel;
  }
  const std::vector<int> grids = coarse_gcr_tc_grids(G, C, nb);
  coarse_gcr_tc_solve(G, C, B, m, maxit, tols.data(), nb, sys[0].b, nf, sys[0].x, nf, sys[0].iters, flags, s,
                      grids.back());
  return true;
}

void coarse_gcr_tc_solve(const LevelGeom& G, const CoarseOp& C, CoarseGCRBuffers& B, int m, int maxit,
                         const double* tol_rel, int nb, const float* b, size_t bstride, float* x, size_t xstride,
                         long long* d_iters, int* flags, cudaStream_t s, int grid) {
  if (m > kMaxRestart) raise(MG_ERR_ARG, "coarse restart too long for the persistent solver");
  if (!coarse_gcr_tc_ok(G, C, nb)) raise(MG_ERR_STATE, "tensor-core coarse solve not applicable to this level");
  const Plan p = make_plan(G, C, grid, nb);
  if (p.grid < nb) raise(MG_ERR_ARG, "grid smaller than the number of systems");
  const int sms = sm_count();
  const bool wide = nb > 8;
  const void* kern = wide ? (const void*)k_coarse_gcr_tc<16> : (const void*)k_coarse_gcr_tc<8>;
  int per = 0;
  MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, p.smem));
  if (per < 1 || p.grid > per * sms) raise(MG_ERR_CUDA, "tensor-core coarse GCR cannot be resident");
  const size_t n = (size_t)G.half * C.nc;
  auto need = [&](DBuf& d, size_t bytes) {
    if (d.bytes() < bytes) d.alloc(bytes);
  };
  const size_t vb = sizeof(float2) * n * nb;
  need(B.tc_y, vb);
  need(B.tc_r, vb);
  need(B.tc_br, vb);
  need(B.tc_s, vb);
  need(B.tc_sy, vb);
  need(B.tc_t, vb);
  need(B.tc_tb, vb);
  need(B.tc_W, vb * m);
  need(B.tc_Z, vb * m);
  const int Gp = p.grid / nb;
  need(B.tc_part, sizeof(float2) * (size_t)kSlots * kMaxSys * Gp);
  need(B.tc_sync, 512);
  TArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nc = C.nc;
  a.half = G.half;
  a.m = m;
  a.maxit = maxit;
  a.nb = nb;
  a.MT = p.MT;
  a.pitch = p.pitch;
  a.Gp = Gp;
  for (int q = 0; q < nb; q++) a.tol_rel[q] = (float)tol_rel[q];
  a.nbr = G.d_nbr.as<int>();
  a.Y = C.Y.as<unsigned>();
  a.Ys = C.Yscale.as<float>();
  a.Xinv = C.Xinv.as<float2>();
  a.b = reinterpret_cast<const float2*>(b);
  a.bstride = bstride;
  a.x = reinterpret_cast<float2*>(x);
  a.xstride = xstride;
  a.y = B.tc_y.as<float2>();
  a.r = B.tc_r.as<float2>();
  a.br = B.tc_br.as<float2>();
  a.s = B.tc_s.as<float2>();
  a.sy = B.tc_sy.as<float2>();
  a.t = B.tc_t.as<float2>();
  a.tb = B.tc_tb.as<float2>();
  a.W = B.tc_W.as<float2>();
  a.Z = B.tc_Z.as<float2>();
  a.part = B.tc_part.as<float2>();
  unsigned char* sync = B.tc_sync.as<unsigned char>();
  a.bar = reinterpret_cast<unsigned*>(sync);
  a.abort = reinterpret_cast<int*>(sync + 128);
  a.vmax = reinterpret_cast<unsigned*>(sync + 256);   // [4][kMaxSys]
  a.iters = d_iters;
  a.flags = flags;
  MG_CUDA(cudaMemsetAsync(B.tc_sync.get(), 0, 512, s));
  int stage_bytes = p.stage_bytes, spw = p.spw;
  void* params[] = {&a, &stage_bytes, &spw};
  MG_CUDA(cudaLaunchCooperativeKernel(kern, dim3(p.grid), dim3(kThreads), params, p.smem, s));
  MG_LAUNCH();
}

}  // namespace mg
