// The coarsest-level GCR of an even-odd coarse lattice with its links
// streamed through shared memory.
//
// Same method as coarse_gcr.cu (section "Implementation": unpreconditioned
// GCR on the coarsest lattice to a relative residual tolerance; section
// "Red-black preconditioning": the reduced even-odd system
// D_r = 1 - Y_eo X_o^{-1} Y_oe X_e^{-1}), arranged for the GB300 memory
// system:
//
//  * Work items are row blocks of one site's link matrix (rows x 8 Nc):
//    phase A uses the folded odd-site links X_o^{-1} Y_d X^{-1}(o + d) (FP32),
//    phase B the even-site links Y_eo in their storage format.  Every block
//    owns a fixed, contiguous range of A items and of B items, and warp w of
//    the block takes every eighth item of each range.
//  * The links do not change during the solve, so the order in which a warp
//    consumes them is known in advance: its B items (for b_r), then its A
//    items and B items once per operator application.  Each warp keeps two
//    shared-memory stages filled along its sequence with bulk asynchronous
//    copies (cp.async.bulk, completion on one mbarrier per stage), so the
//    warps stream and compute independently and the links of the next phase
//    arrive while the block waits at a grid barrier.  A warp computes all
//    rows of its item: every lane strides along the row, the gathered vector
//    element is loaded once for all rows, and one transposing shuffle
//    reduction finishes up to eight rows.
//  * The element-wise work belongs to the block that computed those rows in
//    phase B, so the Gram-Schmidt dots follow phase B without a barrier:
//    one iteration is phase A | barrier | phase B + dots | barrier |
//    coefficients, update, ||r||^2 | barrier.  The norm of the orthogonalised
//    w comes from Pythagoras (the w_j are orthonormal), with an exact second
//    reduction when that subtraction loses more than three digits; <w', r>
//    = <w, r> / gamma because r is orthogonal to the w_j.  The block's slice
//    of the Krylov vectors w_j stays in shared memory when it is small.
//  * Every inner product is reduced deterministically (per-block FP64
//    partials summed in the same order by every block), so all blocks take
//    identical decisions and the result is reproducible bit for bit.
//  * Every wait (mbarrier, grid barrier) is bounded in time; a block that
//    times out raises an abort flag that releases the others, sets
//    FLAG_TIMEOUT and the kernel returns after its copies in flight land.
//
// The site-local parts around it -- t_o = X_o^{-1} b_o before, and the
// reconstruction x_e = X_e^{-1} y_e, x_o = X_o^{-1}(b_o - Y_oe x_e) after --
// are separate launches of the coarse stencil kernels.
#include <algorithm>
#include <cstring>

#include "async_copy.cuh"
#include "dfloat.cuh"
#include "coarse.h"
#include "coarse_dev.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStagesPerWarp = 2;
constexpr int kStages = kWarps * kStagesPerWarp;
constexpr int kMaxRows = 8;        // rows of one item (16 accumulators per lane)
constexpr int kMaxGroups = 8;      // thread groups sharing the sum over j of the Gram-Schmidt update
constexpr int kMaxRestart = 64;
// reduction slots: [0, 2 kMaxRestart) <w_j, w>; then ||w||^2, Re/Im <w, r>;
// ||r||^2; ||b||^2 / true residual; the exact ||w'||^2, Re/Im <w', r>
constexpr int RA = 0;
constexpr int RB = 2 * kMaxRestart;
constexpr int RC = RB + 3;
constexpr int RD = RC + 1;
constexpr int RE = RD + 1;
constexpr int kNR = RE + 3;

struct SArgs {
  int nc, half, m, maxit;
  int rowsA, rowsB, ipsA, ipsB, NA, NB, eszB;
  int stage_bytes, gmax, wsm_ld;   // wsm_ld > 0: the w_j slice in shared memory, leading dimension
  double tol_rel;
  const int* nbr;
  const unsigned char* Y;     // even-site links [e][nc][8][nc], storage format
  const float* Ys;            // their tile scales [e][8]
  const unsigned char* Af;    // folded odd-site links [o - half][nc][8][nc], FP32
  const float2* b;            // full right-hand side
  float2* y;                  // half: GCR iterate
  float2* r;                  // half: residual
  float2* br;                 // half: reduced right-hand side
  float2* tB;                 // full: odd part holds X_o^{-1} b_o on entry, A outputs after
  float2* W;                  // [m][half nc] (when the slice is not in shared memory)
  float2* Z;                  // [m][half nc]
  float2* partials;           // [kNR][grid] double-float partial sums
  long long* iters;
  int* flags;
  unsigned* bar;              // grid barrier counter (0 at launch)
  int* abort;
};

// first element (of the half vector) of item i: site i / ips, rows from (i % ips) rows
__device__ __forceinline__ size_t item_elem(int i, int ips, int rows, int nc) {
  return (size_t)(i / ips) * nc + (size_t)(i % ips) * rows;
}

// Per-warp state of the link stream.
struct Stream {
  unsigned char* ring;
  uint64_t* full;
  int a0, a1, b0, b1;    // the block's item ranges
  int cA, cB;            // this warp's items per A phase and per B phase
  long long t;           // this warp's next sequence position (uniform in the warp)
};

// warp sequence position -> (kind 0: A, 1: B, item index)
__device__ __forceinline__ void seq_item(const Stream& st, long long p, int& kind, int& it) {
  const int w = threadIdx.x >> 5;
  if (p < st.cB) {
    kind = 1;
    it = st.b0 + w + kWarps * (int)p;
    return;
  }
  const long long q = p - st.cB;
  const int off = (int)(q % (st.cA + st.cB));
  if (off < st.cA) {
    kind = 0;
    it = st.a0 + w + kWarps * off;
  } else {
    kind = 1;
    it = st.b0 + w + kWarps * (off - st.cA);
  }
}

// lane 0: bulk copy of the item at warp position p into its stage
__device__ __forceinline__ void issue(const SArgs& a, const Stream& st, long long p) {
  if (st.cA + st.cB == 0) return;
  int kind, it;
  seq_item(st, p, kind, it);
  const int nc = a.nc, K = 8 * nc;
  const unsigned char* src;
  unsigned bytes;
  if (kind == 0) {
    const int s = it / a.ipsA, r0 = (it % a.ipsA) * a.rowsA;
    const int nr = min(a.rowsA, nc - r0);
    src = a.Af + ((size_t)s * nc + r0) * K * 8;
    bytes = (unsigned)(nr * K * 8);
  } else {
    const int s = it / a.ipsB, r0 = (it % a.ipsB) * a.rowsB;
    const int nr = min(a.rowsB, nc - r0);
    src = a.Y + ((size_t)s * nc + r0) * K * a.eszB;
    bytes = (unsigned)(nr * K * a.eszB);
  }
  const int stage = (threadIdx.x >> 5) * kStagesPerWarp + (int)(p % kStagesPerWarp);
  mbar_arrive_expect_tx(&st.full[stage], bytes);
  bulk_copy_g2s(st.ring + (size_t)stage * a.stage_bytes, src, bytes, &st.full[stage]);
}

// Gathers the vectors of the sites of items [i0, i1) (the whole block): for
// each site, the 8 neighbours' nc components of `in`, times the tile scale of
// Y (phase B).
__device__ void gather(const SArgs& a, int i0, int i1, int ips, int site_base, const float2* in, const float* scale,
                       float2* gv) {
  if (i1 > i0) {
    const int nc = a.nc, K = 8 * nc;
    const int s0 = i0 / ips, s1 = (i1 - 1) / ips;
    const int total = (s1 - s0 + 1) * K;
    // four elements per thread and round: their neighbour indices, then their
    // loads, are in flight together (two L2 round trips per round)
    constexpr int U = 4;
    for (int t0 = threadIdx.x; t0 < total; t0 += U * blockDim.x) {
      int src[U];
      float sc[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int t = t0 + u * blockDim.x;
        const int tt = t < total ? t : 0;
        const int sl = tt / K, rem = tt % K, d = rem / nc, j = rem % nc;
        src[u] = a.nbr[(size_t)(site_base + s0 + sl) * 8 + d] * nc + j;
        sc[u] = scale ? scale[(size_t)(s0 + sl) * 8 + d] : 1.f;
      }
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; u++) v[u] = __ldcg(in + (size_t)src[u]);
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int t = t0 + u * blockDim.x;
        if (t < total) gv[t] = make_float2(sc[u] * v[u].x, sc[u] * v[u].y);
      }
    }
  }
  __syncthreads();
}

// Sum over the warp of V per-lane values (V = 2, 4, 8, 16): each of the first
// log2 V levels keeps half of the values and passes the other half to its
// partner, the remaining levels add whole values.  Afterwards lane l holds the
// total of value (l >> log2(32 / V)) & (V - 1).
template <int V>
__device__ __forceinline__ float reduce_values(float v[V]) {
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int half = V / 2; half >= 1; half /= 2, off /= 2) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; i++) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float t = v[0];
#pragma unroll
  for (int o = 16 / V; o >= 1; o /= 2) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// reduce_values for double-float sums: lane l ends with the warp total of
// v[(l >> (5 - log2 V)) & (V - 1)], added in a fixed order.
template <int V>
__device__ __forceinline__ df reduce_df(df v[V]) {
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int half = V / 2; half >= 1; half /= 2, off /= 2) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; i++) {
      const df send = up ? v[i] : v[i + half];
      const df keep = up ? v[i + half] : v[i];
      v[i] = df_add(keep, df{__shfl_xor_sync(0xffffffffu, send.h, off), __shfl_xor_sync(0xffffffffu, send.l, off)});
    }
  }
  df t = v[0];
#pragma unroll
  for (int o = 16 / V; o >= 1; o /= 2)
    t = df_add(t, df{__shfl_xor_sync(0xffffffffu, t.h, o), __shfl_xor_sync(0xffffffffu, t.l, o)});
  return t;
}

// out[row] = sum_k L[row][k] v[k] for the NR rows of a staged item (row-major,
// K complex per row, storage format ST).  Every lane strides along the rows
// two float4 steps at a time, loading the vector element once for all rows.
// Returns true on the lane that holds row `row`'s {re, im} in `res`.
template <int ST, int NR>
__device__ __forceinline__ bool item_rows(const unsigned char* stage, int K, const float2* v, float2& res, int& row) {
  constexpr int V = NR <= 1 ? 2 : NR <= 2 ? 4 : NR <= 4 ? 8 : 16;
  constexpr int SH = V == 2 ? 4 : V == 4 ? 3 : V == 8 ? 2 : 1;   // log2(32 / V)
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const int lane = threadIdx.x & 31;
  const int K2 = K >> 1;
  float acc[V];
#pragma unroll
  for (int i = 0; i < V; i++) acc[i] = 0.f;
  auto step = [&](int q) {
    const float4 x = v4[q];
#pragma unroll
    for (int r = 0; r < NR; r++) {
      float4 m;
      if constexpr (ST == kStF32)
        m = reinterpret_cast<const float4*>(stage)[(size_t)r * K2 + q];
      else
        m = LinkPair<ST>::decode(reinterpret_cast<const uint2*>(stage)[(size_t)r * K2 + q]);
      acc[2 * r] = fmaf(m.x, x.x, acc[2 * r]);
      acc[2 * r] = fmaf(-m.y, x.y, acc[2 * r]);
      acc[2 * r] = fmaf(m.z, x.z, acc[2 * r]);
      acc[2 * r] = fmaf(-m.w, x.w, acc[2 * r]);
      acc[2 * r + 1] = fmaf(m.x, x.y, acc[2 * r + 1]);
      acc[2 * r + 1] = fmaf(m.y, x.x, acc[2 * r + 1]);
      acc[2 * r + 1] = fmaf(m.z, x.w, acc[2 * r + 1]);
      acc[2 * r + 1] = fmaf(m.w, x.z, acc[2 * r + 1]);
    }
  };
  int q = lane;
  for (; q + 32 < K2; q += 64) {
    step(q);
    step(q + 32);
  }
  if (q < K2) step(q);
  const float t = reduce_values<V>(acc);                       // lane l: value (l >> SH) & (V - 1)
  const float im = __shfl_down_sync(0xffffffffu, t, 1 << SH);  // value 2 row + 1
  res = make_float2(t, im);
  row = lane >> (SH + 1);
  return (lane & ((2 << SH) - 1)) == 0 && row < NR;
}

template <int ST>
__device__ __forceinline__ bool item_rows_n(int nr, const unsigned char* stage, int K, const float2* v, float2& res,
                                            int& row) {
  switch (nr) {
    case 1: return item_rows<ST, 1>(stage, K, v, res, row);
    case 2: return item_rows<ST, 2>(stage, K, v, res, row);
    case 3: return item_rows<ST, 3>(stage, K, v, res, row);
    case 4: return item_rows<ST, 4>(stage, K, v, res, row);
    case 5: return item_rows<ST, 5>(stage, K, v, res, row);
    case 6: return item_rows<ST, 6>(stage, K, v, res, row);
    case 7: return item_rows<ST, 7>(stage, K, v, res, row);
    default: return item_rows<ST, 8>(stage, K, v, res, row);
  }
}

// One phase of this warp's items: waits for each staged item, computes its
// rows, hands row results to epi(kind-specific index, row value) and refills
// the stage two positions ahead.  false on a timeout (uniform in the block
// after the closing barrier).
template <int ST, typename Epi>
__device__ bool run_items(const SArgs& a, Stream& st, int kind, const float2* gv, Epi epi, int* s_fail) {
  const int nc = a.nc, K = 8 * nc;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = kind ? st.b0 : st.a0, i1 = kind ? st.b1 : st.a1;
  const int ips = kind ? a.ipsB : a.ipsA, rows = kind ? a.rowsB : a.rowsA;
  const int sbase = i0 / ips;
  bool ok = true;
  for (int it = i0 + w; it < i1; it += kWarps) {
    const int stage = w * kStagesPerWarp + (int)(st.t % kStagesPerWarp);
    const unsigned par = (unsigned)((st.t / kStagesPerWarp) & 1);
    if (!mbar_wait(&st.full[stage], par)) {
      ok = false;
      break;
    }
    const int s = it / ips, r0 = (it % ips) * rows;
    const int nr = min(rows, nc - r0);
    float2 res;
    int row;
    const unsigned char* sp = st.ring + (size_t)stage * a.stage_bytes;
    const float2* vp = gv + (size_t)(s - sbase) * K;
    const bool mine = kind == 0 ? item_rows_n<kStF32>(nr, sp, K, vp, res, row) : item_rows_n<ST>(nr, sp, K, vp, res, row);
    if (mine) epi((size_t)s * nc + r0 + row, res);
    __syncwarp();
    if (lane == 0) issue(a, st, st.t + kStagesPerWarp);
    st.t++;
  }
  if (!ok) atomicExch(s_fail, 1);
  __syncthreads();
  return *(volatile int*)s_fail == 0;
}

// block partial sums of nq per-thread float values v[q]: warp sums, then the
// eight warp sums added by one thread per slot; partials[q0 + q][block]
__device__ void block_partials(const SArgs& a, const float* v, int nq, int q0, df* sred) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < nq; q++) {
    const df t = df_wsum(df_of(v[q]));
    if (lane == 0) sred[q * kWarps + wid] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    df s = sred[q * kWarps];
    for (int w = 1; w < kWarps; w++) s = df_add(s, sred[q * kWarps + w]);
    a.partials[(size_t)(q0 + q) * gridDim.x + blockIdx.x] = make_float2(s.h, s.l);
  }
  __syncthreads();
}

// totals of slots [q0, q0 + nq) after a grid barrier, identical in every
// block.  Warp w sums slots w, w + 8, ...; each round issues the loads of
// kTotU slots (up to kTotG / 32 per lane and slot) before adding any, so that a
// round costs one L2 round trip; the kTotU sums leave the warp through one
// transposing reduction.
constexpr int kTotG = 160;   // grids up to this size take the one-pass path
constexpr int kTotU = 4;     // slots per warp and round
__device__ void grid_totals(const SArgs& a, int q0, int nq, df* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = gridDim.x;
  if (G <= kTotG) {
    for (int qb = wid; qb < nq; qb += kTotU * kWarps) {
      float2 t[kTotU][kTotG / 32];
#pragma unroll
      for (int u = 0; u < kTotU; u++) {
        const int q = qb + u * kWarps;
        const float2* p = a.partials + (size_t)(q0 + (q < nq ? q : 0)) * G;
#pragma unroll
        for (int i = 0; i < kTotG / 32; i++) {
          const int g = lane + 32 * i;
          t[u][i] = (q < nq && g < G) ? __ldcg(p + g) : make_float2(0.f, 0.f);
        }
      }
      df sv[kTotU];
#pragma unroll
      for (int u = 0; u < kTotU; u++) {
        sv[u] = df{t[u][0].x, t[u][0].y};
#pragma unroll
        for (int i = 1; i < kTotG / 32; i++) sv[u] = df_add(sv[u], df{t[u][i].x, t[u][i].y});
      }
      const df s = reduce_df<kTotU>(sv);   // lane l: slot qb + (l >> 3) * kWarps
      const int q = qb + (lane >> 3) * kWarps;
      if ((lane & 7) == 0 && q < nq) out[q] = s;
    }
  } else {
    for (int q = wid; q < nq; q += kWarps) {
      const float2* p = a.partials + (size_t)(q0 + q) * G;
      df s = df_of(0.f);
      for (int g = lane; g < G; g += 32) {
        const float2 x = __ldcg(p + g);
        s = df_add(s, df{x.x, x.y});
      }
      s = df_wsum(s);
      if (lane == 0) out[q] = s;
    }
  }
  __syncthreads();
}

template <int ST>
__global__ void __launch_bounds__(kThreads, 1) k_coarse_gcr_stream(SArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ float2 s_beta[kMaxRestart];   // <w_j, w> of this iteration, as floats
  __shared__ float s_coef[4];              // 1/gamma, Re alpha, Im alpha, exact flag
  __shared__ int s_fail;
  const int nc = a.nc, K = 8 * nc, m = a.m;
  const int G = gridDim.x, bid = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2* gv = reinterpret_cast<float2*>(smem + (size_t)kStages * a.stage_bytes);
  df* sred = reinterpret_cast<df*>(gv + (size_t)a.gmax * K);          // [kNR][kWarps]
  df* tot = sred + kNR * kWarps;                                       // [kNR]
  float2* upd = reinterpret_cast<float2*>(tot + kNR);                  // [2][kThreads] update partial sums
  float2* wsm = upd + 2 * kThreads;                                    // [m][wsm_ld] when used

  Stream st;
  st.ring = smem;
  st.full = full;
  st.a0 = (int)((long long)bid * a.NA / G);
  st.a1 = (int)((long long)(bid + 1) * a.NA / G);
  st.b0 = (int)((long long)bid * a.NB / G);
  st.b1 = (int)((long long)(bid + 1) * a.NB / G);
  st.cA = st.a1 - st.a0 > wid ? (st.a1 - st.a0 - wid + kWarps - 1) / kWarps : 0;
  st.cB = st.b1 - st.b0 > wid ? (st.b1 - st.b0 - wid + kWarps - 1) / kWarps : 0;
  st.t = 0;
  const size_t E0 = item_elem(st.b0, a.ipsB, a.rowsB, nc);
  const size_t E1 = st.b1 == a.NB ? (size_t)a.half * nc : item_elem(st.b1, a.ipsB, a.rowsB, nc);
  const int E = (int)(E1 - E0);
  const size_t n = (size_t)a.half * nc;
  // the block's slices of w_j and z_j: element e at Wj(j)[e - E0], Zj(j)[e - E0]
  float2* const wbase = a.wsm_ld > 0 ? wsm : a.W + E0;
  const size_t wld = a.wsm_ld > 0 ? (size_t)a.wsm_ld : n;
  auto Wj = [&](int j) { return wbase + (size_t)j * wld; };
  auto Zj = [&](int j) { return a.Z + (size_t)j * n + E0; };
  // the j sums of the Gram-Schmidt update are split over ngrp thread groups
  // when the slice has at most one element per thread
  const int ngrp = (E > 0 && E <= (int)blockDim.x) ? min((int)blockDim.x / E, kMaxGroups) : 0;
  unsigned target = 0;
  bool ok = true;
  float v[4];

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(&full[s], 1);
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  if (lane == 0)
    for (long long p = 0; p < kStagesPerWarp; p++) issue(a, st, p);

  // ||b||^2 over the full right-hand side (any partition of it)
  {
    const size_t nf = 2 * n;
    const size_t cf = (nf + G - 1) / G;
    const size_t f0 = (size_t)bid * cf, f1 = f0 + cf < nf ? f0 + cf : nf;
    v[0] = 0.f;
    for (size_t e = f0 + threadIdx.x; e < f1; e += blockDim.x) {
      const float2 q = a.b[e];
      v[0] = fmaf(q.x, q.x, fmaf(q.y, q.y, v[0]));
    }
    block_partials(a, v, 1, RD, sred);
  }
  // b_r = b_e - Y_eo X_o^{-1} b_o on the owned rows; r = b_r, y = 0
  gather(a, st.b0, st.b1, a.ipsB, 0, a.tB, a.Ys, gv);
  ok = run_items<ST>(a, st, 1, gv, [&](size_t i, float2 u) {
    const float2 bb = a.b[i];
    const float2 o = make_float2(bb.x - u.x, bb.y - u.y);
    a.br[i] = o;
    a.r[i] = o;
    a.y[i] = make_float2(0.f, 0.f);
  }, &s_fail);
  // ||b_r||^2 over the owned rows (written by this block's own items)
  v[0] = 0.f;
  for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x) {
    const float2 rr = a.r[e];
    v[0] = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, v[0]));
  }
  block_partials(a, v, 1, RC, sred);
  if (ok) ok = grid_barrier(a.bar, a.abort, target);
  long long its = 0;
  bool done = true;
  df tol2 = df_of(0.f);
  if (ok) {
    grid_totals(a, RC, 2, tot + RC);   // ||b_r||^2 (the running ||r||^2) and ||b||^2
    const df tr = df_of((float)a.tol_rel);
    tol2 = df_mul(df_mul(tr, tr), tot[RD]);
    done = !(tot[RD].h > 0.f);
  }
  while (ok && !done && its < a.maxit) {
    int k = 0;
    while (k < m && its < a.maxit) {
      float2* wk = Wj(k);
      // w = D_r r: phase A, barrier, phase B
      gather(a, st.a0, st.a1, a.ipsA, a.half, a.r, nullptr, gv);
      if (!(ok = run_items<ST>(a, st, 0, gv, [&](size_t i, float2 u) { a.tB[(size_t)a.half * nc + i] = u; }, &s_fail)))
        break;
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      gather(a, st.b0, st.b1, a.ipsB, 0, a.tB, a.Ys, gv);
      if (!(ok = run_items<ST>(a, st, 1, gv, [&](size_t i, float2 u) {
              const float2 rr = a.r[i];
              wk[i - E0] = make_float2(rr.x - u.x, rr.y - u.y);
            }, &s_fail)))
        break;
      // beta_j = <w_j, w> (warp wid owns j = wid + 8 u, u < 4), ||w||^2, <w, r>
      for (int jb = wid; jb < k; jb += 4 * kWarps) {
        float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
        for (int e = lane; e < E; e += 32) {
          const float2 x = wk[e];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int j = jb + u * kWarps;
            const float2 p = j < k ? Wj(j)[e] : make_float2(0.f, 0.f);
            re[u] = fmaf(p.x, x.x, fmaf(p.y, x.y, re[u]));
            im[u] = fmaf(p.x, x.y, fmaf(-p.y, x.x, im[u]));
          }
        }
        df sv[8];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          sv[2 * u] = df_of(re[u]);
          sv[2 * u + 1] = df_of(im[u]);
        }
        const df sr = reduce_df<8>(sv);   // lane l: sum (l >> 2) = 2 u + {re, im}
        const int j = jb + (lane >> 3) * kWarps;
        if ((lane & 3) == 0 && j < k) a.partials[(size_t)(RA + 2 * j + ((lane >> 2) & 1)) * G + bid] = make_float2(sr.h, sr.l);
      }
      v[0] = v[1] = v[2] = 0.f;
      for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x) {
        const float2 x = wk[e - E0], rr = a.r[e];
        v[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, v[0]));
        v[1] = fmaf(x.x, rr.x, fmaf(x.y, rr.y, v[1]));
        v[2] = fmaf(x.x, rr.y, fmaf(-x.y, rr.x, v[2]));
      }
      block_partials(a, v, 3, RA + 2 * k, sred);   // after the beta slots: one pass reads all of them
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      grid_totals(a, RA, 2 * k + 3, tot);
      {  // move them to their own slots (the ranges may overlap: read all, then write)
        df moved = df_of(0.f);
        if (threadIdx.x < 3) moved = tot[2 * k + threadIdx.x];
        __syncthreads();
        if (threadIdx.x < 3) tot[RB + threadIdx.x] = moved;
        __syncthreads();
      }
      // sum_j |beta_j|^2 (warp 0, lanes over j) and the beta_j as floats
      if (wid == 0) {
        df bb = df_of(0.f);
        for (int j = lane; j < k; j += 32) {
          bb = df_add(bb, df_mul(tot[2 * j], tot[2 * j]));
          bb = df_add(bb, df_mul(tot[2 * j + 1], tot[2 * j + 1]));
          s_beta[j] = make_float2(tot[2 * j].h + tot[2 * j].l, tot[2 * j + 1].h + tot[2 * j + 1].l);
        }
        bb = df_wsum(bb);
        if (lane == 0) {
          const df g2 = df_add(tot[RB], df_neg(bb));
          s_coef[3] = (g2.h > 1e-3f * tot[RB].h) ? 0.f : 1.f;   // Pythagoras lost more than three digits
          tot[RE] = g2;
        }
      }
      __syncthreads();
      const bool exact = s_coef[3] != 0.f;
      // S_w = sum_j beta_j w_j, S_z = sum_j beta_j z_j on the owned rows
      if (ngrp) {
        const int gi = threadIdx.x / E, ei = threadIdx.x - gi * E;
        if (gi < ngrp) {
          float swr = 0.f, swi = 0.f, szr = 0.f, szi = 0.f;
#pragma unroll 4
          for (int j = gi; j < k; j += ngrp) {
            const float2 bj = s_beta[j];
            const float2 p = Wj(j)[ei], q = Zj(j)[ei];
            swr = fmaf(bj.x, p.x, fmaf(-bj.y, p.y, swr));
            swi = fmaf(bj.x, p.y, fmaf(bj.y, p.x, swi));
            szr = fmaf(bj.x, q.x, fmaf(-bj.y, q.y, szr));
            szi = fmaf(bj.x, q.y, fmaf(bj.y, q.x, szi));
          }
          upd[gi * E + ei] = make_float2(swr, swi);
          upd[kThreads + gi * E + ei] = make_float2(szr, szi);
        }
        __syncthreads();
      }
      // w'' = w - S_w kept in place; with the exact path its norm and <w'', r>
      v[0] = v[1] = v[2] = 0.f;
      for (int ei = threadIdx.x; ei < E; ei += blockDim.x) {
        float2 x = wk[ei];
        if (ngrp) {
          for (int g = 0; g < ngrp; g++) {
            const float2 u = upd[g * E + ei];
            x.x -= u.x;
            x.y -= u.y;
          }
        } else {
#pragma unroll 4
          for (int j = 0; j < k; j++) {
            const float2 bj = s_beta[j], p = Wj(j)[ei];
            x.x -= bj.x * p.x - bj.y * p.y;
            x.y -= bj.x * p.y + bj.y * p.x;
          }
        }
        wk[ei] = x;
        if (exact) {
          const float2 rr = a.r[E0 + ei];
          v[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, v[0]));
          v[1] = fmaf(x.x, rr.x, fmaf(x.y, rr.y, v[1]));
          v[2] = fmaf(x.x, rr.y, fmaf(-x.y, rr.x, v[2]));
        }
      }
      if (exact) {  // uniform: every block took the same decision from the same totals
        block_partials(a, v, 3, RE, sred);
        if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
        grid_totals(a, RE, 3, tot + RB);   // the exact ||w''||^2, <w'', r> replace the estimates
        if (threadIdx.x == 0) tot[RE] = tot[RB];
        __syncthreads();
      }
      // gamma = ||w''||, alpha = <w'', r> / gamma; with w_k = w'' / gamma of
      // unit norm, ||r - alpha w_k||^2 = ||r||^2 - |alpha|^2 (the running norm)
      if (threadIdx.x == 0) {
        const df g = df_sqrt(tot[RE]);
        const bool gz = !(g.h > 0.f);
        s_coef[0] = gz ? 1.f : 1.f / g.h;
        const df ar = gz ? tot[RB + 1] : df_div(tot[RB + 1], g);
        const df ai = gz ? tot[RB + 2] : df_div(tot[RB + 2], g);
        s_coef[1] = ar.h + ar.l;
        s_coef[2] = ai.h + ai.l;
        if (!gz) {
          const df rn = df_add(tot[RC], df_neg(df_add(df_mul(ar, ar), df_mul(ai, ai))));
          tot[RC] = rn.h > 0.f ? rn : df_of(0.f);
        }
      }
      __syncthreads();
      // w_k = w'' / gamma, z_k = (r - S_z) / gamma, y += alpha z_k, r -= alpha w_k
      const float ig = s_coef[0], far = s_coef[1], fai = s_coef[2];
      v[0] = 0.f;
      for (int ei = threadIdx.x; ei < E; ei += blockDim.x) {
        const size_t e = E0 + ei;
        float2 x = wk[ei];
        x.x *= ig;
        x.y *= ig;
        wk[ei] = x;
        float2 rr = a.r[e];
        float2 z = rr;
        if (ngrp) {
          for (int g = 0; g < ngrp; g++) {
            const float2 u = upd[kThreads + g * E + ei];
            z.x -= u.x;
            z.y -= u.y;
          }
        } else {
#pragma unroll 4
          for (int j = 0; j < k; j++) {
            const float2 bj = s_beta[j], q = Zj(j)[ei];
            z.x -= bj.x * q.x - bj.y * q.y;
            z.y -= bj.x * q.y + bj.y * q.x;
          }
        }
        z.x *= ig;
        z.y *= ig;
        Zj(k)[ei] = z;
        float2 yy = a.y[e];
        yy.x += far * z.x - fai * z.y;
        yy.y += far * z.y + fai * z.x;
        a.y[e] = yy;
        rr.x -= far * x.x - fai * x.y;
        rr.y -= far * x.y + fai * x.x;
        a.r[e] = rr;
      }
      // r complete on every block before the next iteration's phase A reads it
      if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
      k++;
      its++;
      const df rn2 = tot[RC];
      if (!(rn2.h == rn2.h)) {
        if (bid == 0 && threadIdx.x == 0) atomicExch(&a.flags[FLAG_NAN], 1);
        done = true;
        break;
      }
      if (rn2.h <= tol2.h) break;
    }
    if (!ok || done) break;
    // true residual r = b_r - D_r y (y complete on every block after the last barrier)
    gather(a, st.a0, st.a1, a.ipsA, a.half, a.y, nullptr, gv);
    if (!(ok = run_items<ST>(a, st, 0, gv, [&](size_t i, float2 u) { a.tB[(size_t)a.half * nc + i] = u; }, &s_fail)))
      break;
    if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
    gather(a, st.b0, st.b1, a.ipsB, 0, a.tB, a.Ys, gv);
    if (!(ok = run_items<ST>(a, st, 1, gv, [&](size_t i, float2 u) {
            const float2 yy = a.y[i], bb = a.br[i];
            a.r[i] = make_float2(bb.x - (yy.x - u.x), bb.y - (yy.y - u.y));
          }, &s_fail)))
      break;
    v[0] = 0.f;
    for (size_t e = E0 + threadIdx.x; e < E1; e += blockDim.x) {
      const float2 rr = a.r[e];
      v[0] = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, v[0]));
    }
    block_partials(a, v, 1, RC, sred);
    if (!(ok = grid_barrier(a.bar, a.abort, target))) break;
    grid_totals(a, RC, 1, tot + RC);   // the true ||r||^2 restarts the running norm
    const df rn2 = tot[RC];
    if (rn2.h <= tol2.h || !(rn2.h == rn2.h)) done = true;
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(&a.flags[FLAG_TIMEOUT], 1);
    atomicExch(a.abort, 1);
  }
  // drain: the copies this warp issued beyond what it consumed land before exit
  if (lane == 0 && st.cA + st.cB > 0)
    for (long long p = st.t; p < st.t + kStagesPerWarp; p++)
      (void)mbar_wait(&full[wid * kStagesPerWarp + (int)(p % kStagesPerWarp)],
                      (unsigned)((p / kStagesPerWarp) & 1));
  if (bid == 0 && threadIdx.x == 0) *a.iters += its;
}

struct Plan {
  int grid, stage_bytes, rowsA, rowsB, ipsA, ipsB, NA, NB, gmax, wsm_ld, emax;
  size_t smem;
};

// items, the sites a block's item ranges touch, and the shared memory they need
void plan_items(Plan& p, int half, int nc, int esz) {
  const int K = 8 * nc;
  p.rowsA = std::min(kMaxRows, std::min(nc, p.stage_bytes / (K * 8)));
  p.rowsB = std::min(kMaxRows, std::min(nc, p.stage_bytes / (K * esz)));
  p.ipsA = p.rowsA > 0 ? (nc + p.rowsA - 1) / p.rowsA : 0;
  p.ipsB = p.rowsB > 0 ? (nc + p.rowsB - 1) / p.rowsB : 0;
  p.NA = half * p.ipsA;
  p.NB = half * p.ipsB;
  p.gmax = 1;
  p.emax = 0;
  const int G = std::min(p.grid, std::min(p.NA, p.NB));
  auto elem = [&](int i) -> long long {   // item_elem of the kernel
    return i == p.NB ? (long long)half * nc : (long long)(i / p.ipsB) * nc + (long long)(i % p.ipsB) * p.rowsB;
  };
  for (int b = 0; b < G && p.rowsA > 0 && p.rowsB > 0; b++) {
    const int a0 = (int)((long long)b * p.NA / G), a1 = (int)((long long)(b + 1) * p.NA / G);
    const int b0 = (int)((long long)b * p.NB / G), b1 = (int)((long long)(b + 1) * p.NB / G);
    if (a1 > a0) p.gmax = std::max(p.gmax, (a1 - 1) / p.ipsA - a0 / p.ipsA + 1);
    if (b1 > b0) p.gmax = std::max(p.gmax, (b1 - 1) / p.ipsB - b0 / p.ipsB + 1);
    p.emax = std::max(p.emax, (int)(elem(b1) - elem(b0)));
  }
}

Plan make_plan(const LevelGeom& G, const CoarseOp& C, int grid, int m) {
  Plan p;
  const int nc = C.nc, K = 8 * nc;
  const int esz = C.store == STORE_F32 ? 8 : 4;
  int dev = 0, optin = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t budget = (size_t)optin - 4096;   // static shared memory and slack
  const size_t fixed = sizeof(float2) * (kNR * kWarps + kNR) + sizeof(float2) * 2 * kThreads;
  p.grid = grid;
  // the w_j slice in shared memory only when it is small (a sixteenth of the
  // budget): measured on GB300 at Nc = 48, m = 64, a deeper link ring gains
  // more than shared-memory Gram-Schmidt vectors save.  A block's slice has
  // at most ceil(n / grid) elements plus the rows of the partial items at
  // both ends of its range.
  const size_t n = (size_t)G.half * nc;
  const int gb = std::max(1, grid);
  const int ebound = (int)((n + gb - 1) / gb) + (int)((7LL * G.half + gb - 1) / gb) + 2 * kMaxRows;
  const bool wsmem = (size_t)m * ebound * sizeof(float2) <= budget / 16;
  const size_t wbytes = wsmem ? (size_t)m * ebound * sizeof(float2) : 0;
  int gsites = 4;
  for (int pass = 0; pass < 3; pass++) {
    const size_t other = fixed + wbytes + sizeof(float2) * (size_t)gsites * K;
    p.stage_bytes = budget > other ? (int)(((budget - other) / kStages) / 16 * 16) : 0;
    plan_items(p, G.half, nc, esz);
    if (p.gmax <= gsites) break;
    gsites = p.gmax;
  }
  p.grid = std::min(grid, std::min(p.NA, p.NB));
  p.smem = (size_t)kStages * p.stage_bytes + fixed + wbytes + sizeof(float2) * (size_t)std::max(gsites, p.gmax) * K;
  p.gmax = std::max(gsites, p.gmax);
  p.wsm_ld = wsmem ? ebound : 0;
  if (wsmem && p.emax > ebound) raise(MG_ERR_STATE, "streamed coarse GCR: Krylov slice larger than planned");
  return p;
}

const void* kernel_for(int store) {
  return store == STORE_F16    ? (const void*)k_coarse_gcr_stream<kStF16>
         : store == STORE_BF16 ? (const void*)k_coarse_gcr_stream<kStBF16>
                               : (const void*)k_coarse_gcr_stream<kStF32>;
}

int sm_count() {
  int dev = 0, sms = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

}  // namespace

bool coarse_gcr_stream_ok(const LevelGeom& G, const CoarseOp& C) {
  if (!G.eo || C.nc % 2 || !C.A.get()) return false;
  const Plan p = make_plan(G, C, sm_count(), kMaxRestart);
  return p.rowsA >= 1 && p.rowsB >= 1 && p.smem <= 232448;
}

std::vector<int> coarse_gcr_stream_grids(const LevelGeom& G, const CoarseOp& C) {
  const Plan p = make_plan(G, C, sm_count(), kMaxRestart);
  std::vector<int> out = {p.grid};
  // the largest grid that splits both item lists evenly (no block waits at a
  // barrier for a neighbour with one more item)
  for (int g = p.grid - 1; g >= p.grid / 2 && g >= 1; g--)
    if (p.NA % g == 0 && p.NB % g == 0) {
      out.push_back(g);
      break;
    }
  return out;
}

void coarse_gcr_stream_solve(const LevelGeom& G, const CoarseOp& C, CoarseGCRBuffers& B, int m, int maxit,
                             double tol_rel, const float* b, float* x, long long* d_iters, int* flags, cudaStream_t s,
                             int grid) {
  if (m > kMaxRestart) raise(MG_ERR_ARG, "coarse restart too long for the persistent solver");
  if (!coarse_gcr_stream_ok(G, C)) raise(MG_ERR_STATE, "streamed coarse solve not applicable to this level");
  const Plan p = make_plan(G, C, grid, m);
  const int sms = sm_count();
  int per = 0;
  const void* kern = kernel_for(C.store);
  MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, p.smem));
  if (per < 1 || p.grid > per * sms) raise(MG_ERR_CUDA, "streamed coarse GCR cannot be resident");
  const size_t n = (size_t)G.half * C.nc;
  auto need = [&](DBuf& d, size_t bytes) {
    if (d.bytes() < bytes) d.alloc(bytes);
  };
  need(B.st_part, sizeof(float2) * (size_t)kNR * p.grid);
  need(B.st_sync, 256);
  if (B.W.bytes() < sizeof(float2) * n * m || B.Z.bytes() < sizeof(float2) * n * m)
    raise(MG_ERR_STATE, "coarse GCR buffers too small for this restart length");
  float* tB = B.tB.as<float>();
  coarse_site_mul(G, C, true, G.half, G.nsites, tB, b, s);     // t_o = X_o^{-1} b_o
  MG_CUDA(cudaMemsetAsync(B.st_sync.get(), 0, 256, s));
  SArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nc = C.nc;
  a.half = G.half;
  a.m = m;
  a.maxit = maxit;
  a.rowsA = p.rowsA;
  a.rowsB = p.rowsB;
  a.ipsA = p.ipsA;
  a.ipsB = p.ipsB;
  a.NA = p.NA;
  a.NB = p.NB;
  a.eszB = C.store == STORE_F32 ? 8 : 4;
  a.stage_bytes = p.stage_bytes;
  a.gmax = p.gmax;
  a.wsm_ld = p.wsm_ld;
  a.tol_rel = tol_rel;
  a.nbr = G.d_nbr.as<int>();
  a.Y = static_cast<const unsigned char*>(C.Y.get());
  a.Ys = C.Yscale.as<float>();
  a.Af = static_cast<const unsigned char*>(C.A.get());
  a.b = reinterpret_cast<const float2*>(b);
  a.y = B.y.as<float2>();
  a.r = B.r.as<float2>();
  a.br = B.br.as<float2>();
  a.tB = B.tB.as<float2>();
  a.W = B.W.as<float2>();
  a.Z = B.Z.as<float2>();
  a.partials = B.st_part.as<float2>();
  a.iters = d_iters;
  a.flags = flags;
  a.bar = B.st_sync.as<unsigned>();
  a.abort = reinterpret_cast<int*>(B.st_sync.as<unsigned char>() + 128);
  void* params[] = {&a};
  MG_CUDA(cudaLaunchCooperativeKernel(kern, dim3(p.grid), dim3(kThreads), params, p.smem, s));
  MG_LAUNCH();
  // reconstruction: x_e = X_e^{-1} y_e, x_o = X_o^{-1} (b_o - Y_oe x_e)
  coarse_site_mul(G, C, true, 0, G.half, x, B.y.as<float>(), s);
  coarse_hop(G, C, EPI_C_XPAY, true, G.half, G.nsites, x, x, b, -1.f, 0xff, s);
}

}  // namespace mg
