// Coarse-level kernels of the adaptive multigrid (sm_103a).
//
//  * restriction R = P^dag and prolongation P with the chirality split of
//    the null vectors (section "Red-black preconditioning": P is built from
//    the low modes of D_p, split into the two chiralities inside each block;
//    R = P^dag gamma_5 gives the same coarse correction as R = P^dag for a
//    chirality-split P, so R = P^dag is applied)
//  * Galerkin coarse links D_hat = R D_p P ("Red-black preconditioning"):
//    one P column at a time, the eight directional hops of M^{-1} p are
//    projected onto the receiving block's P, hops across a block face into
//    Y_d and all others into X
//  * the coarse stencil D_hat v = X v + sum_d Y_d v(. + d) with the same
//    epilogues as the fine dslash, which give the coarse even-odd operators
//    (the coarse system is solved by its reduced even-odd form)
//  * FP64 batched Gauss-Jordan for X^{-1}
//  * block Gram-Schmidt (FP64 accumulation) and coarse-vector packing
//
// Coarse operators look like a staggered operator with Nc = 2 Nv colours
// ("Implementation"); a CTA owns one coarse site, its warps own rows of the
// 2Nv x 8*2Nv link block, and the neighbour vectors are staged in shared
// memory so each link row is read once, coalesced.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "async_copy.cuh"
#include "coarse.h"
#include "coarse_dev.cuh"
#include "philox.cuh"

namespace mg {

namespace {
constexpr int kBS = 256;

__device__ __forceinline__ cx<float> fget(const FineAccess& fa, const float* base, int idx, int c) {
  if (fa.wilson) {
    const int par = idx >= fa.Vh;
    const int cb = idx - par * fa.Vh;
    return SpinorIO<float>::get(base + (size_t)par * 24 * fa.Vh, fa.Vh, cb, c);
  }
  const float2 v = reinterpret_cast<const float2*>(base)[(size_t)idx * fa.ndof + c];
  return mkc(v.x, v.y);
}

__device__ __forceinline__ void fput(const FineAccess& fa, float* base, int idx, int c, cx<float> z) {
  if (fa.wilson) {
    const int par = idx >= fa.Vh;
    const int cb = idx - par * fa.Vh;
    SpinorIO<float>::put(base + (size_t)par * 24 * fa.Vh, fa.Vh, cb, c, z);
    return;
  }
  reinterpret_cast<float2*>(base)[(size_t)idx * fa.ndof + c] = make_float2(z.re, z.im);
}

// element e of a stored complex array in format ST
template <int ST>
__device__ __forceinline__ cx<float> sget(const void* p, size_t e) {
  if (ST == STORE_F32) {
    const float2 v = reinterpret_cast<const float2*>(p)[e];
    return mkc(v.x, v.y);
  } else if (ST == STORE_F16) {
    const float2 v = __half22float2(reinterpret_cast<const __half2*>(p)[e]);
    return mkc(v.x, v.y);
  } else {
    const float2 v = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(p)[e]);
    return mkc(v.x, v.y);
  }
}

template <int ST>
__device__ __forceinline__ void sput(void* p, size_t e, cx<float> z) {
  if (ST == STORE_F32) {
    reinterpret_cast<float2*>(p)[e] = make_float2(z.re, z.im);
  } else if (ST == STORE_F16) {
    reinterpret_cast<__half2*>(p)[e] = __floats2half2_rn(z.re, z.im);
  } else {
    reinterpret_cast<__nv_bfloat162*>(p)[e] = __floats2bfloat162_rn(z.re, z.im);
  }
}

struct TArgs {
  int nv, ndof, nb, fine_half, nbe;
  int b[4], cd[4];
  FineAccess fa;
  const int* blockmap;
  const int* evenlist;
  const void* P;
  const float* Ps;
  int* flags;
};

TArgs targs(const TransferOp& T) {
  TArgs a;
  a.nv = T.nv;
  a.ndof = T.fine_ndof;
  a.nb = T.nb;
  a.fine_half = T.fine_half;
  for (int m = 0; m < 4; m++) {
    a.b[m] = T.block[m];
    a.cd[m] = T.cdims[m];
  }
  a.fa = T.fa;
  a.nbe = T.nbe;
  a.blockmap = T.blockmap.as<int>();
  a.evenlist = T.evenlist.as<int>();
  a.P = T.P.get();
  a.Ps = T.Pscale.as<float>();
  a.flags = T.flags;
  return a;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

// --------------------------------------------------------------------------- restriction
// One CTA per coarse site.  Warp w takes the block's fine sites w, w+8, ...;
// lane k (and k+32 when Nv > 32) accumulates conj(P[i][c][k]) v[i][c] for the
// two chiralities.  The site's components are read once by lanes 0..ndof-1
// and broadcast with shuffles; P rows are read coalesced, several components
// in flight at a time.  Per-warp sums are combined in FP64 at the end.
template <int ST>
__global__ void __launch_bounds__(256) k_restrict(TArgs a, float* __restrict__ out, const float* __restrict__ v,
                                                  int even_only, int nrhs, size_t vstride, size_t cstride) {
  extern __shared__ float2 sacc[];  // [nwarps][2 nv]
  // one CTA per (coarse site, rhs), rhs fastest: the CTAs of a site share its P rows in L2
  const int cc = blockIdx.x / nrhs, rq = blockIdx.x % nrhs;
  v += rq * vstride;
  out += rq * cstride;
  const int nv = a.nv, hd = a.ndof / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float acc[2][2][2] = {};  // [k-half][chirality][re, im]
  for (int i = w; i < a.nb; i += nw) {
    const int idx = a.blockmap[cc * a.nb + i];
    if (even_only && idx >= a.fine_half) continue;
    const cx<float> x0 = lane < a.ndof ? fget(a.fa, v, idx, lane) : mkc(0.f, 0.f);
    const cx<float> x1 = lane + 32 < a.ndof ? fget(a.fa, v, idx, lane + 32) : mkc(0.f, 0.f);
    const size_t base = (size_t)(cc * a.nb + i) * a.ndof;
#pragma unroll 4
    for (int c = 0; c < a.ndof; c++) {
      const float xr = __shfl_sync(0xffffffffu, c < 32 ? x0.re : x1.re, c & 31);
      const float xi = __shfl_sync(0xffffffffu, c < 32 ? x0.im : x1.im, c & 31);
      const int ch = c >= hd;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int k = lane + 32 * h;
        if (k < nv) {
          const cx<float> p = sget<ST>(a.P, (base + c) * nv + k);
          acc[h][ch][0] += p.re * xr + p.im * xi;
          acc[h][ch][1] += p.re * xi - p.im * xr;
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int k = lane + 32 * h;
    if (k < nv) {
      sacc[(size_t)w * 2 * nv + k] = make_float2(acc[h][0][0], acc[h][0][1]);
      sacc[(size_t)w * 2 * nv + nv + k] = make_float2(acc[h][1][0], acc[h][1][1]);
    }
  }
  __syncthreads();
  const float s0 = a.Ps[cc * 2], s1 = a.Ps[cc * 2 + 1];
  for (int t = threadIdx.x; t < 2 * nv; t += blockDim.x) {
    double re = 0, im = 0;
    for (int q = 0; q < nw; q++) {
      re += sacc[(size_t)q * 2 * nv + t].x;
      im += sacc[(size_t)q * 2 * nv + t].y;
    }
    const float sc = t < nv ? s0 : s1;
    reinterpret_cast<float2*>(out)[(size_t)cc * 2 * nv + t] = make_float2((float)(sc * re), (float)(sc * im));
  }
}

// Fine-level (Wilson) transfers.  One CTA per (coarse site, chirality, group
// of NR right-hand sides) walks the block's selected fine sites (all, or the
// even ones from the block's list) in tiles of kFTile sites through a
// kFStages-deep shared-memory pipeline.  A producer warp fills a stage --
// per site its P rows of the chirality, 6 Nv contiguous elements, with one
// bulk asynchronous copy each, and for the restriction the chirality's three
// float4 chunks of each right-hand side with 16-byte cp.async copies spread
// over its lanes (many tiny bulk copies would queue on the copy engine) --
// completed on the stage's "full" mbarrier; the consumer warps compute from
// the stage and release it on its "empty" mbarrier.  The bytes in flight per SM are set by the shared-memory budget
// (2-3 stages of each resident CTA), not by registers.  Every wait is bounded;
// a wait that runs out raises FLAG_TIMEOUT and the kernel carries on without
// it (every address stays in bounds), so the launch always ends.
constexpr int kFTile = 8;
constexpr int kFStages = 3;
constexpr int kFineMaxSites = 512;   // selected fine sites per block (indices kept in shared memory)

template <int ST>
__host__ __device__ constexpr int fine_esz() {
  return ST == STORE_F32 ? 8 : 4;
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

bool fine_transfer_ok(const TransferOp& T, bool even_only, const void* fine, size_t fstride, const void* coarse,
                      size_t cstride) {
  return T.fa.wilson && T.nv <= 32 && T.nv % 2 == 0 && T.nb <= kFineMaxSites && (!even_only || T.nbe > 0) &&
         reinterpret_cast<uintptr_t>(fine) % 16 == 0 && reinterpret_cast<uintptr_t>(coarse) % 16 == 0 &&
         fstride % 4 == 0 && cstride % 4 == 0;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// an arrival on bar once all of the calling thread's earlier cp.async copies
// have landed (the barrier's expected count includes this arrival)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Restriction.  Consumer warp w takes the tile's sites w, w + 4; lane k < Nv
// accumulates conj(P[site][d][k]) x[site][d] (P from consecutive addresses, x
// as a broadcast).  The four warp sums are added in a fixed order.
constexpr int kRCons = 4;

template <int ST, int NR>
struct RestrictSmem {
  static constexpr int esz = fine_esz<ST>();
  int rowb, xoff, stb;
  size_t sacc, stage0, idx, total;
  __host__ __device__ RestrictSmem(int nv, int nsel) {
    rowb = 6 * nv * esz;
    xoff = kFTile * rowb;
    stb = xoff + kFTile * NR * 48;
    sacc = align16(sizeof(uint64_t) * 2 * kFStages);
    stage0 = align16(sacc + sizeof(float2) * kRCons * NR * 32);
    idx = stage0 + (size_t)kFStages * stb;
    total = idx + sizeof(int) * 2 * nsel;
  }
};

template <int ST, int NR>
__global__ void __launch_bounds__((kRCons + 1) * 32) k_restrict_fine(TArgs a, float* __restrict__ out,
                                                                     const float* __restrict__ v, int even_only,
                                                                     int nrhs, size_t vstride, size_t cstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int esz = fine_esz<ST>();
  const int nv = a.nv, Vh = a.fa.Vh;
  const int nsel = even_only ? a.nbe : a.nb;
  const RestrictSmem<ST, NR> L(nv, nsel);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kFStages;
  float2* sacc = reinterpret_cast<float2*>(smem_raw + L.sacc);   // [kRCons][NR][32]
  unsigned char* stage0 = smem_raw + L.stage0;
  int* si = reinterpret_cast<int*>(smem_raw + L.idx);            // [nsel] block-local index
  int* sx = si + nsel;                                           // [nsel] storage index
  const int nrg = (nrhs + NR - 1) / NR;
  const int cc = blockIdx.x / (2 * nrg), rem = blockIdx.x % (2 * nrg);
  const int ch = rem / nrg, r0 = (rem % nrg) * NR;
  const int nr = min(NR, nrhs - r0);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    for (int st = 0; st < kFStages; st++) {
      mbar_init(&full[st], 1 + 32);   // lane 0's arrival + every producer lane's cp.async arrival
      mbar_init(&empty[st], kRCons);
    }
    mbar_fence_init();
  }
  for (int t = tid; t < nsel; t += blockDim.x) {
    const int i = even_only ? a.evenlist[cc * a.nbe + t] : t;
    si[t] = i;
    sx[t] = a.blockmap[cc * a.nb + i];
  }
  __syncthreads();
  const int ntile = (nsel + kFTile - 1) / kFTile;
  bool ok = true;
  if (w == kRCons) {   // producer
    const unsigned char* Pb = static_cast<const unsigned char*>(a.P);
    for (int T = 0; T < ntile; T++) {
      const int st = T % kFStages, use = T / kFStages;
      if (use > 0) ok &= mbar_wait(&empty[st], (unsigned)((use - 1) & 1));
      const int s0 = T * kFTile, ns = min(kFTile, nsel - s0);
      unsigned char* sp = stage0 + (size_t)st * L.stb;
      if (lane == 0) mbar_expect_tx(&full[st], (unsigned)(ns * L.rowb));
      __syncwarp();
      if (lane < ns)
        bulk_copy_g2s(sp + lane * L.rowb, Pb + (((size_t)(cc * a.nb + si[s0 + lane]) * 12 + 6 * ch) * nv) * esz,
                      (unsigned)L.rowb, &full[st]);
      for (int u = lane; u < ns * nr * 3; u += 32) {
        const int s = u / (nr * 3), rq = u - s * nr * 3, r = rq / 3, q = rq - r * 3;
        const int idx = sx[s0 + s], par = idx >= Vh, cb = idx - par * Vh;
        cp_async16(sp + L.xoff + ((s * NR + r) * 3 + q) * 16,
                   reinterpret_cast<const float4*>(v + (size_t)(r0 + r) * vstride + (size_t)par * 24 * Vh) +
                       (size_t)(3 * ch + q) * Vh + cb);
      }
      cp_async_arrive(&full[st]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[st]);
    }
  } else {   // consumers
    float acc[NR][2];
#pragma unroll
    for (int r = 0; r < NR; r++) acc[r][0] = acc[r][1] = 0.f;
    for (int T = 0; T < ntile; T++) {
      const int st = T % kFStages, use = T / kFStages;
      ok &= mbar_wait(&full[st], (unsigned)(use & 1));
      const unsigned char* sp = stage0 + (size_t)st * L.stb;
      const float4* xs = reinterpret_cast<const float4*>(sp + L.xoff);
      const int ns = min(kFTile, nsel - T * kFTile);
      if (lane < nv) {
        for (int s = w; s < ns; s += kRCons) {
          const void* prow = sp + s * L.rowb;
#pragma unroll
          for (int d = 0; d < 6; d++) {
            const cx<float> p = sget<ST>(prow, (size_t)d * nv + lane);
#pragma unroll
            for (int r = 0; r < NR; r++) {
              if (r < nr) {
                const float4 c4 = xs[(s * NR + r) * 3 + (d >> 1)];
                const float xr = (d & 1) ? c4.z : c4.x, xi = (d & 1) ? c4.w : c4.y;
                acc[r][0] = fmaf(p.re, xr, fmaf(p.im, xi, acc[r][0]));
                acc[r][1] = fmaf(p.re, xi, fmaf(-p.im, xr, acc[r][1]));
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
#pragma unroll
    for (int r = 0; r < NR; r++) sacc[(w * NR + r) * 32 + lane] = make_float2(acc[r][0], acc[r][1]);
    consumer_sync(kRCons * 32);
    const float sc = a.Ps[cc * 2 + ch];
    for (int t = tid; t < nr * nv; t += kRCons * 32) {
      const int r = t / nv, k = t - r * nv;
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int q = 0; q < kRCons; q++) {
        re += sacc[(q * NR + r) * 32 + k].x;
        im += sacc[(q * NR + r) * 32 + k].y;
      }
      reinterpret_cast<float2*>(out + (size_t)(r0 + r) * cstride)[(size_t)cc * 2 * nv + ch * nv + k] =
          make_float2(sc * re, sc * im);
    }
  }
  if (!ok && a.flags) atomicExch(&a.flags[FLAG_TIMEOUT], 1);
}

template <int ST, int NR>
void launch_restrict_fine(const TArgs& a, int ncoarse, int nrhs, float* out, const float* v, bool even_only,
                          size_t vstride, size_t cstride, cudaStream_t s) {
  const unsigned grid = (unsigned)((size_t)ncoarse * 2 * ((nrhs + NR - 1) / NR));
  const RestrictSmem<ST, NR> L(a.nv, even_only ? a.nbe : a.nb);
  MG_CUDA(cudaFuncSetAttribute(k_restrict_fine<ST, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  k_restrict_fine<ST, NR><<<grid, (kRCons + 1) * 32, L.total, s>>>(a, out, v, even_only, nrhs, vstride, cstride);
  MG_LAUNCH();
}

template <int ST>
void restrict_fine(const TArgs& a, int ncoarse, int nrhs, float* out, const float* v, bool even_only,
                   size_t vstride, size_t cstride, cudaStream_t s) {
  if (nrhs >= 4)
    launch_restrict_fine<ST, 4>(a, ncoarse, nrhs, out, v, even_only, vstride, cstride, s);
  else if (nrhs >= 2)
    launch_restrict_fine<ST, 2>(a, ncoarse, nrhs, out, v, even_only, vstride, cstride, s);
  else
    launch_restrict_fine<ST, 1>(a, ncoarse, nrhs, out, v, even_only, vstride, cstride, s);
}

void restrict_vec_multi(const TransferOp& T, int nrhs, float* out_c, size_t cstride, const float* v, size_t vstride,
                        bool even_only, cudaStream_t s) {
  TArgs a = targs(T);
  if (fine_transfer_ok(T, even_only, v, vstride, out_c, cstride)) {
    switch (T.store) {
      case STORE_F32: restrict_fine<STORE_F32>(a, T.ncoarse, nrhs, out_c, v, even_only, vstride, cstride, s); break;
      case STORE_F16: restrict_fine<STORE_F16>(a, T.ncoarse, nrhs, out_c, v, even_only, vstride, cstride, s); break;
      default: restrict_fine<STORE_BF16>(a, T.ncoarse, nrhs, out_c, v, even_only, vstride, cstride, s); break;
    }
    return;
  }
  const size_t sm = sizeof(float2) * (kBS / 32) * 2 * (size_t)T.nv;
  const unsigned grid = (unsigned)((size_t)T.ncoarse * nrhs);
  switch (T.store) {
    case STORE_F32: k_restrict<STORE_F32><<<grid, kBS, sm, s>>>(a, out_c, v, even_only, nrhs, vstride, cstride); break;
    case STORE_F16: k_restrict<STORE_F16><<<grid, kBS, sm, s>>>(a, out_c, v, even_only, nrhs, vstride, cstride); break;
    default: k_restrict<STORE_BF16><<<grid, kBS, sm, s>>>(a, out_c, v, even_only, nrhs, vstride, cstride); break;
  }
  MG_LAUNCH();
}

void restrict_vec(const TransferOp& T, float* out_c, const float* v, bool even_only, cudaStream_t s) {
  restrict_vec_multi(T, 1, out_c, 0, v, 0, even_only, s);
}

// --------------------------------------------------------------------------- prolongation
template <int ST>
__global__ void k_prolong(TArgs a, float* __restrict__ v, const float* __restrict__ in_c, int even_only, int nrhs,
                          size_t vstride, size_t cstride) {
  extern __shared__ float2 svc[];  // [2 nv]
  const int cc = blockIdx.x / nrhs, rq = blockIdx.x % nrhs;   // (coarse site, rhs), rhs fastest
  v += rq * vstride;
  in_c += rq * cstride;
  const int nv = a.nv, hd = a.ndof / 2;
  for (int t = threadIdx.x; t < 2 * nv; t += blockDim.x)
    svc[t] = reinterpret_cast<const float2*>(in_c)[(size_t)cc * 2 * nv + t];
  __syncthreads();
  const float s0 = a.Ps[cc * 2], s1 = a.Ps[cc * 2 + 1];
  for (int t = threadIdx.x; t < a.nb * a.ndof; t += blockDim.x) {
    const int i = t / a.ndof, c = t % a.ndof;
    const int idx = a.blockmap[cc * a.nb + i];
    if (even_only && idx >= a.fine_half) continue;
    const int ch = c >= hd;
    const float2* vc = svc + ch * nv;
    const size_t base = ((size_t)(cc * a.nb + i) * a.ndof + c) * nv;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < nv; k++) {
      const cx<float> p = sget<ST>(a.P, base + k);
      re += p.re * vc[k].x - p.im * vc[k].y;
      im += p.re * vc[k].y + p.im * vc[k].x;
    }
    const float sc = ch ? s1 : s0;
    fput(a.fa, v, idx, c, mkc(sc * re, sc * im));
  }
}

// Prolongation onto the fine (Wilson) level, with the pipeline of the
// restriction (one CTA per (coarse site, chirality, group of NR right-hand
// sides)); the producer also copies the coarse vectors of the chirality once.
// Consumer warp w forms the float4 chunk 3 ch + w (spin-colour components
// 6 ch + 2w, +1) of the tile's sites: lane = site (lane & 7) + 8 g, the four
// g lanes of a site taking its NR right-hand sides, each split over 4 / NR
// lanes that share the Nv/2 pairs of null vectors and add their sums with
// shuffles; one lane per (site, right-hand side) stores the chunk with one
// 16-byte store.  A staged site occupies an odd
// number of 16-byte units, so the eight sites of a quarter-warp read
// different banks; the coarse vector is read as a broadcast.
constexpr int kPCons = 3;

template <int ST, int NR>
struct ProlongSmem {
  static constexpr int esz = fine_esz<ST>();
  int rowb, pitch, stb;
  size_t svc, stage0, idx, total;
  __host__ __device__ ProlongSmem(int nv, int nsel) {
    rowb = 6 * nv * esz;
    pitch = 16 * ((rowb / 16) | 1);
    stb = kFTile * pitch;
    svc = align16(sizeof(uint64_t) * (2 * kFStages + 1));
    stage0 = align16(svc + sizeof(float2) * NR * nv);
    idx = stage0 + (size_t)kFStages * stb;
    total = idx + sizeof(int) * 2 * nsel;
  }
};

template <int ST, int NR>
__global__ void __launch_bounds__((kPCons + 1) * 32) k_prolong_fine(TArgs a, float* __restrict__ v,
                                                                    const float* __restrict__ in_c, int even_only,
                                                                    int nrhs, size_t vstride, size_t cstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int esz = fine_esz<ST>();
  const int nv = a.nv, Vh = a.fa.Vh;
  const int nsel = even_only ? a.nbe : a.nb;
  const ProlongSmem<ST, NR> L(nv, nsel);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kFStages;
  uint64_t* cbar = empty + kFStages;
  const float2* svc = reinterpret_cast<const float2*>(smem_raw + L.svc);   // [NR][nv]
  unsigned char* stage0 = smem_raw + L.stage0;
  int* si = reinterpret_cast<int*>(smem_raw + L.idx);
  int* sx = si + nsel;
  const int nrg = (nrhs + NR - 1) / NR;
  const int cc = blockIdx.x / (2 * nrg), rem = blockIdx.x % (2 * nrg);
  const int ch = rem / nrg, r0 = (rem % nrg) * NR;
  const int nr = min(NR, nrhs - r0);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    for (int st = 0; st < kFStages; st++) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kPCons);
    }
    mbar_init(cbar, 1);
    mbar_fence_init();
  }
  for (int t = tid; t < nsel; t += blockDim.x) {
    const int i = even_only ? a.evenlist[cc * a.nbe + t] : t;
    si[t] = i;
    sx[t] = a.blockmap[cc * a.nb + i];
  }
  __syncthreads();
  const int ntile = (nsel + kFTile - 1) / kFTile;
  bool ok = true;
  if (w == kPCons) {   // producer
    if (lane == 0) mbar_expect_tx(cbar, (unsigned)(nr * nv * 8));
    __syncwarp();
    if (lane < nr)
      bulk_copy_g2s(smem_raw + L.svc + (size_t)lane * nv * 8,
                    in_c + (size_t)(r0 + lane) * cstride + ((size_t)cc * 2 * nv + ch * nv) * 2, (unsigned)(nv * 8),
                    cbar);
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    const unsigned char* Pb = static_cast<const unsigned char*>(a.P);
    for (int T = 0; T < ntile; T++) {
      const int st = T % kFStages, use = T / kFStages;
      if (use > 0) ok &= mbar_wait(&empty[st], (unsigned)((use - 1) & 1));
      const int s0 = T * kFTile, ns = min(kFTile, nsel - s0);
      if (lane == 0) mbar_expect_tx(&full[st], (unsigned)(ns * L.rowb));
      __syncwarp();
      if (lane < ns)
        bulk_copy_g2s(stage0 + (size_t)st * L.stb + lane * L.pitch,
                      Pb + (((size_t)(cc * a.nb + si[s0 + lane]) * 12 + 6 * ch) * nv) * esz, (unsigned)L.rowb,
                      &full[st]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[st]);
    }
  } else {   // consumers
    ok &= mbar_wait(cbar, 0u);
    constexpr int KQ = 4 / NR;   // lanes sharing the pairs of one (site, right-hand side)
    const int s = lane & 7, g = lane >> 3, rq = g / KQ, kq = g % KQ;
    const int npair = nv / 2;
    const float4* c2p = reinterpret_cast<const float4*>(svc + rq * nv);
    for (int T = 0; T < ntile; T++) {
      const int st = T % kFStages, use = T / kFStages;
      ok &= mbar_wait(&full[st], (unsigned)(use & 1));
      const int s0 = T * kFTile, ns = min(kFTile, nsel - s0);
      const unsigned char* row0 = stage0 + (size_t)st * L.stb + s * L.pitch + 2 * w * nv * esz;
      const unsigned char* row1 = row0 + nv * esz;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      if (s < ns && rq < nr) {
        for (int kp = kq; kp < npair; kp += KQ) {
          float2 p0[2], p1[2];
          if (ST == STORE_F32) {
            const float4 u0 = reinterpret_cast<const float4*>(row0)[kp];
            const float4 u1 = reinterpret_cast<const float4*>(row1)[kp];
            p0[0] = make_float2(u0.x, u0.y);
            p0[1] = make_float2(u0.z, u0.w);
            p1[0] = make_float2(u1.x, u1.y);
            p1[1] = make_float2(u1.z, u1.w);
          } else {
            const uint2 u0 = reinterpret_cast<const uint2*>(row0)[kp];
            const uint2 u1 = reinterpret_cast<const uint2*>(row1)[kp];
            if (ST == STORE_F16) {
              p0[0] = __half22float2(*reinterpret_cast<const __half2*>(&u0.x));
              p0[1] = __half22float2(*reinterpret_cast<const __half2*>(&u0.y));
              p1[0] = __half22float2(*reinterpret_cast<const __half2*>(&u1.x));
              p1[1] = __half22float2(*reinterpret_cast<const __half2*>(&u1.y));
            } else {
              p0[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u0.x));
              p0[1] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u0.y));
              p1[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u1.x));
              p1[1] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u1.y));
            }
          }
          const float4 c2 = c2p[kp];
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const float cr = h ? c2.z : c2.x, ci = h ? c2.w : c2.y;
            acc[0] = fmaf(p0[h].x, cr, fmaf(-p0[h].y, ci, acc[0]));
            acc[1] = fmaf(p0[h].x, ci, fmaf(p0[h].y, cr, acc[1]));
            acc[2] = fmaf(p1[h].x, cr, fmaf(-p1[h].y, ci, acc[2]));
            acc[3] = fmaf(p1[h].x, ci, fmaf(p1[h].y, cr, acc[3]));
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);   // the stage is read; what follows uses registers
#pragma unroll
      for (int o = 8; o < 8 * KQ; o <<= 1)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
      if (s < ns && rq < nr && kq == 0) {
        const float sc = a.Ps[cc * 2 + ch];
        const int idx = sx[s0 + s], par = idx >= Vh, cb = idx - par * Vh;
        reinterpret_cast<float4*>(v + (size_t)(r0 + rq) * vstride + (size_t)par * 24 * Vh)[(size_t)(3 * ch + w) * Vh +
                                                                                           cb] =
            make_float4(sc * acc[0], sc * acc[1], sc * acc[2], sc * acc[3]);
      }
    }
  }
  if (!ok && a.flags) atomicExch(&a.flags[FLAG_TIMEOUT], 1);
}

template <int ST, int NR>
void launch_prolong_fine(const TArgs& a, const TransferOp& T, int nrhs, float* v, const float* in_c, bool even_only,
                         size_t vstride, size_t cstride, cudaStream_t s) {
  const unsigned grid = (unsigned)((size_t)T.ncoarse * 2 * ((nrhs + NR - 1) / NR));
  const ProlongSmem<ST, NR> L(T.nv, even_only ? T.nbe : T.nb);
  MG_CUDA(cudaFuncSetAttribute(k_prolong_fine<ST, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  k_prolong_fine<ST, NR><<<grid, (kPCons + 1) * 32, L.total, s>>>(a, v, in_c, even_only, nrhs, vstride, cstride);
  MG_LAUNCH();
}

template <int ST>
void prolong_fine(const TArgs& a, const TransferOp& T, int nrhs, float* v, const float* in_c, bool even_only,
                  size_t vstride, size_t cstride, cudaStream_t s) {
  if (nrhs >= 4)
    launch_prolong_fine<ST, 4>(a, T, nrhs, v, in_c, even_only, vstride, cstride, s);
  else if (nrhs >= 2)
    launch_prolong_fine<ST, 2>(a, T, nrhs, v, in_c, even_only, vstride, cstride, s);
  else
    launch_prolong_fine<ST, 1>(a, T, nrhs, v, in_c, even_only, vstride, cstride, s);
}

void prolong_vec_multi(const TransferOp& T, int nrhs, float* v, size_t vstride, const float* in_c, size_t cstride,
                       bool even_only, cudaStream_t s) {
  TArgs a = targs(T);
  if (fine_transfer_ok(T, even_only, v, vstride, in_c, cstride)) {
    switch (T.store) {
      case STORE_F32: prolong_fine<STORE_F32>(a, T, nrhs, v, in_c, even_only, vstride, cstride, s); break;
      case STORE_F16: prolong_fine<STORE_F16>(a, T, nrhs, v, in_c, even_only, vstride, cstride, s); break;
      default: prolong_fine<STORE_BF16>(a, T, nrhs, v, in_c, even_only, vstride, cstride, s); break;
    }
    return;
  }
  const size_t sm = sizeof(float2) * 2 * T.nv;
  const unsigned grid = (unsigned)((size_t)T.ncoarse * nrhs);
  switch (T.store) {
    case STORE_F32: k_prolong<STORE_F32><<<grid, kBS, sm, s>>>(a, v, in_c, even_only, nrhs, vstride, cstride); break;
    case STORE_F16: k_prolong<STORE_F16><<<grid, kBS, sm, s>>>(a, v, in_c, even_only, nrhs, vstride, cstride); break;
    default: k_prolong<STORE_BF16><<<grid, kBS, sm, s>>>(a, v, in_c, even_only, nrhs, vstride, cstride); break;
  }
  MG_LAUNCH();
}

void prolong_vec(const TransferOp& T, float* v, const float* in_c, bool even_only, cudaStream_t s) {
  prolong_vec_multi(T, 1, v, 0, in_c, 0, even_only, s);
}

// --------------------------------------------------------------------------- column extraction
template <int ST>
__global__ void k_extract_column(TArgs a, float* p, int chir, int k) {
  const size_t total = (size_t)a.nb * a.ndof;
  const int cc = blockIdx.x;
  const int hd = a.ndof / 2;
  for (size_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = (int)(t / a.ndof), c = (int)(t % a.ndof);
    const int idx = a.blockmap[cc * a.nb + i];
    cx<float> z = mkc(0.f, 0.f);
    if ((c >= hd) == (chir == 1)) {
      z = sget<ST>(a.P, ((size_t)(cc * a.nb + i) * a.ndof + c) * a.nv + k);
      const float sc = a.Ps[cc * 2 + chir];
      z = mkc(sc * z.re, sc * z.im);
    }
    fput(a.fa, p, idx, c, z);
  }
}

void extract_column(const TransferOp& T, float* p, int chir, int k, cudaStream_t s) {
  TArgs a = targs(T);
  switch (T.store) {
    case STORE_F32: k_extract_column<STORE_F32><<<T.ncoarse, kBS, 0, s>>>(a, p, chir, k); break;
    case STORE_F16: k_extract_column<STORE_F16><<<T.ncoarse, kBS, 0, s>>>(a, p, chir, k); break;
    default: k_extract_column<STORE_BF16><<<T.ncoarse, kBS, 0, s>>>(a, p, chir, k); break;
  }
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- Galerkin column
struct W9 {
  const float* p[9];
};

template <int ST>
__global__ void k_restrict9(TArgs a, W9 W, float2* __restrict__ Y, float2* __restrict__ X, int col) {
  extern __shared__ double sred[];  // [G][nv][2][2]
  const int cc = blockIdx.x;
  const int nv = a.nv, G = blockDim.x / nv, nc = 2 * nv;
  const int k = threadIdx.x % nv, g = threadIdx.x / nv;
  const int hd = a.ndof / 2;
  double acc[9][2][2];
#pragma unroll
  for (int t = 0; t < 9; t++)
#pragma unroll
    for (int ch = 0; ch < 2; ch++) acc[t][ch][0] = acc[t][ch][1] = 0.0;
  if (g < G) {
    for (int i = g; i < a.nb; i += G) {
      const int idx = a.blockmap[cc * a.nb + i];
      int l[4];
      l[0] = i % a.b[0];
      l[1] = (i / a.b[0]) % a.b[1];
      l[2] = (i / (a.b[0] * a.b[1])) % a.b[2];
      l[3] = i / (a.b[0] * a.b[1] * a.b[2]);
      bool face[8];
#pragma unroll
      for (int d = 0; d < 8; d++) {
        const int mu = d & 3;
        face[d] = a.cd[mu] > 1 && (d < 4 ? l[mu] == a.b[mu] - 1 : l[mu] == 0);
      }
      const size_t base = (size_t)(cc * a.nb + i) * a.ndof;
#pragma unroll
      for (int ch = 0; ch < 2; ch++) {
        const float sc = a.Ps[cc * 2 + ch];
        for (int c = ch * hd; c < (ch + 1) * hd; c++) {
          cx<float> p = sget<ST>(a.P, (base + c) * nv + k);
          p = mkc(sc * p.re, sc * p.im);
#pragma unroll
          for (int d = 0; d < 9; d++) {
            const cx<float> w = fget(a.fa, W.p[d], idx, c);
            const double re = (double)p.re * w.re + (double)p.im * w.im;
            const double im = (double)p.re * w.im - (double)p.im * w.re;
            if (d < 8 && face[d < 8 ? d : 0]) {
              acc[d][ch][0] += re;
              acc[d][ch][1] += im;
            } else {
              acc[8][ch][0] += re;
              acc[8][ch][1] += im;
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 9; t++) {
    __syncthreads();
    if (g < G) {
      double* me = sred + ((size_t)g * nv + k) * 4;
      me[0] = acc[t][0][0];
      me[1] = acc[t][0][1];
      me[2] = acc[t][1][0];
      me[3] = acc[t][1][1];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      const int ch = q / nv, kk = q % nv;
      double re = 0, im = 0;
      for (int gg = 0; gg < G; gg++) {
        re += sred[((size_t)gg * nv + kk) * 4 + 2 * ch];
        im += sred[((size_t)gg * nv + kk) * 4 + 2 * ch + 1];
      }
      const int row = q;
      if (t < 8)
        Y[(((size_t)cc * nc + row) * 8 + t) * nc + col] = make_float2((float)re, (float)im);
      else
        X[((size_t)cc * nc + row) * nc + col] = make_float2((float)re, (float)im);
    }
  }
}

void restrict9(const TransferOp& T, CoarseOp& C, const float* const W[9], int col, cudaStream_t s) {
  TArgs a = targs(T);
  W9 w;
  for (int d = 0; d < 9; d++) w.p[d] = W[d];
  const int G = kBS / T.nv;
  const size_t sm = sizeof(double) * 4 * (size_t)G * T.nv;
  float2* Y = C.Y.as<float2>();
  float2* X = C.X.as<float2>();
  switch (T.store) {
    case STORE_F32: k_restrict9<STORE_F32><<<T.ncoarse, kBS, sm, s>>>(a, w, Y, X, col); break;
    case STORE_F16: k_restrict9<STORE_F16><<<T.ncoarse, kBS, sm, s>>>(a, w, Y, X, col); break;
    default: k_restrict9<STORE_BF16><<<T.ncoarse, kBS, sm, s>>>(a, w, Y, X, col); break;
  }
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- coarse stencil
struct HopArgs {
  int nc, s0, dirmask;
  const int* nbr;
  const void* Y;    // links in the level's storage format
  const float* Ys;
  const float2* C;  // X or Xinv
  float2* out;
  const float2* in;
  const float2* x;
  float a;
};

template <int EPI, int ST>
__global__ void __launch_bounds__(256) k_coarse_hop(HopArgs h) {
  extern __shared__ __align__(16) float2 sm[];  // vin[8 nc], t[nc], vx[nc]
  const int nc = h.nc;
  const int s = h.s0 + blockIdx.x;
  float2* vin = sm;
  float2* tv = sm + 8 * nc;
  float2* vx = tv + nc;
  for (int t = threadIdx.x; t < 8 * nc; t += blockDim.x) {
    const int d = t / nc, j = t % nc;
    float2 v = make_float2(0.f, 0.f);
    if ((h.dirmask >> d) & 1) {
      const float sc = h.Ys[(size_t)s * 8 + d];
      v = h.in[(size_t)h.nbr[(size_t)s * 8 + d] * nc + j];
      v.x *= sc;
      v.y *= sc;
    }
    vin[t] = v;
  }
  if (EPI == EPI_CX_PAY || EPI == EPI_XPAY || EPI == EPI_C_XPAY)
    for (int t = threadIdx.x; t < nc; t += blockDim.x) vx[t] = h.x[(size_t)s * nc + t];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rpw = (nc + nw - 1) / nw;
  float2 res[kGemvMaxRows];
  warp_gemv<ST>(static_cast<const char*>(h.Y) + (size_t)s * nc * 8 * nc * link_bytes<ST>(), nc, 8 * nc, vin, w, rpw,
                lane, res);
  if (lane == 0)
#pragma unroll
    for (int r = 0; r < kGemvMaxRows; r++) {
      const int i = w * rpw + r;
      if (r < rpw && i < nc) {
        if (EPI == EPI_H) h.out[(size_t)s * nc + i] = res[r];
        else if (EPI == EPI_XPAY)
          h.out[(size_t)s * nc + i] = make_float2(vx[i].x + h.a * res[r].x, vx[i].y + h.a * res[r].y);
        else if (EPI == EPI_CH || EPI == EPI_CX_PAY) tv[i] = res[r];
        else tv[i] = make_float2(vx[i].x + h.a * res[r].x, vx[i].y + h.a * res[r].y);  // EPI_C_XPAY
      }
    }
  if (EPI == EPI_H || EPI == EPI_XPAY) return;
  __syncthreads();
  const float2* src = (EPI == EPI_CX_PAY) ? vx : tv;
  warp_gemv(h.C + (size_t)s * nc * nc, nc, nc, src, w, rpw, lane, res);
  if (lane == 0)
#pragma unroll
    for (int r = 0; r < kGemvMaxRows; r++) {
      const int i = w * rpw + r;
      if (r < rpw && i < nc) {
        if (EPI == EPI_CX_PAY)
          h.out[(size_t)s * nc + i] = make_float2(res[r].x + h.a * tv[i].x, res[r].y + h.a * tv[i].y);
        else
          h.out[(size_t)s * nc + i] = res[r];
      }
    }
}

void coarse_hop(const LevelGeom& G, const CoarseOp& C, Epilogue epi, bool use_inv, int s0, int s1, float* out,
                const float* in, const float* x, float a, int dirmask, cudaStream_t s) {
  if (s1 <= s0) return;
  HopArgs h;
  h.nc = C.nc;
  h.s0 = s0;
  h.dirmask = dirmask;
  h.nbr = G.d_nbr.as<int>();
  h.Y = C.Y.get();
  h.Ys = C.Yscale.as<float>();
  h.C = use_inv ? C.Xinv.as<float2>() : C.X.as<float2>();
  h.out = (float2*)out;
  h.in = (const float2*)in;
  h.x = (const float2*)x;
  h.a = a;
  const size_t sm = sizeof(float2) * 10 * (size_t)C.nc;
  const int nb = s1 - s0;
  auto launch = [&](auto st) {
    constexpr int ST = decltype(st)::value;
    switch (epi) {
      case EPI_H: k_coarse_hop<EPI_H, ST><<<nb, 256, sm, s>>>(h); break;
      case EPI_CH: k_coarse_hop<EPI_CH, ST><<<nb, 256, sm, s>>>(h); break;
      case EPI_XPAY: k_coarse_hop<EPI_XPAY, ST><<<nb, 256, sm, s>>>(h); break;
      case EPI_CX_PAY: k_coarse_hop<EPI_CX_PAY, ST><<<nb, 256, sm, s>>>(h); break;
      case EPI_C_XPAY: k_coarse_hop<EPI_C_XPAY, ST><<<nb, 256, sm, s>>>(h); break;
    }
  };
  switch (C.store) {
    case STORE_F32: launch(std::integral_constant<int, kStF32>()); break;
    case STORE_F16: launch(std::integral_constant<int, kStF16>()); break;
    default: launch(std::integral_constant<int, kStBF16>()); break;
  }
  MG_LAUNCH();
}

__global__ void __launch_bounds__(256) k_site_mul(int nc, int s0, const float2* __restrict__ C, float2* out,
                                                   const float2* __restrict__ in) {
  extern __shared__ __align__(16) float2 sv[];
  const int s = s0 + blockIdx.x;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) sv[t] = in[(size_t)s * nc + t];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rpw = (nc + nw - 1) / nw;
  float2 res[kGemvMaxRows];
  warp_gemv(C + (size_t)s * nc * nc, nc, nc, sv, w, rpw, lane, res);
  if (lane == 0)
#pragma unroll
    for (int r = 0; r < kGemvMaxRows; r++) {
      const int i = w * rpw + r;
      if (r < rpw && i < nc) out[(size_t)s * nc + i] = res[r];
    }
}

void coarse_site_mul(const LevelGeom& G, const CoarseOp& C, bool use_inv, int s0, int s1, float* out, const float* in,
                     cudaStream_t s) {
  (void)G;
  if (s1 <= s0) return;
  const float2* M = use_inv ? C.Xinv.as<float2>() : C.X.as<float2>();
  k_site_mul<<<s1 - s0, 256, sizeof(float2) * C.nc, s>>>(C.nc, s0, M, (float2*)out, (const float2*)in);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- coarse inverse
__global__ void k_coarse_invert(int nc, const float2* __restrict__ X, float2* Xinv, int* flags) {
  extern __shared__ double2 A[];  // [nc][2 nc]
  __shared__ double2 fac[128];
  __shared__ int piv_s;
  __shared__ double amax_s;
  const int s = blockIdx.x;
  const int w2 = 2 * nc;
  for (int t = threadIdx.x; t < nc * w2; t += blockDim.x) {
    const int i = t / w2, j = t % w2;
    double2 v;
    if (j < nc) {
      const float2 x = X[((size_t)s * nc + i) * nc + j];
      v = make_double2(x.x, x.y);
    } else {
      v = make_double2(i == j - nc ? 1.0 : 0.0, 0.0);
    }
    A[t] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0;
    for (int i = 0; i < nc; i++)
      for (int j = 0; j < nc; j++) m = fmax(m, fabs(A[i * w2 + j].x) + fabs(A[i * w2 + j].y));
    amax_s = m;
  }
  __syncthreads();
  for (int col = 0; col < nc; col++) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = col;
      for (int r = col + threadIdx.x; r < nc; r += 32) {
        const double2 v = A[r * w2 + col];
        const double m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        piv_s = bi;
        if (!(sqrt(best) > 1e-12 * amax_s)) atomicExch(&flags[FLAG_SINGULAR], 1);
      }
    }
    __syncthreads();
    const int piv = piv_s;
    if (piv != col)
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        const double2 t = A[col * w2 + j];
        A[col * w2 + j] = A[piv * w2 + j];
        A[piv * w2 + j] = t;
      }
    __syncthreads();
    double2 p = A[col * w2 + col];
    double den = p.x * p.x + p.y * p.y;
    if (den == 0) den = 1;
    const double2 pinv = make_double2(p.x / den, -p.y / den);
    __syncthreads();
    for (int j = threadIdx.x; j < w2; j += blockDim.x) {
      const double2 a = A[col * w2 + j];
      A[col * w2 + j] = make_double2(pinv.x * a.x - pinv.y * a.y, pinv.x * a.y + pinv.y * a.x);
    }
    for (int r = threadIdx.x; r < nc; r += blockDim.x) fac[r] = A[r * w2 + col];
    __syncthreads();
    for (int t = threadIdx.x; t < nc * w2; t += blockDim.x) {
      const int r = t / w2, j = t % w2;
      if (r == col) continue;
      const double2 f = fac[r], a = A[col * w2 + j];
      A[t].x -= f.x * a.x - f.y * a.y;
      A[t].y -= f.x * a.y + f.y * a.x;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
    const int i = t / nc, j = t % nc;
    const double2 v = A[i * w2 + nc + j];
    Xinv[((size_t)s * nc + i) * nc + j] = make_float2((float)v.x, (float)v.y);
  }
}

void coarse_invert(const LevelGeom& G, CoarseOp& C, int* flags, cudaStream_t s) {
  const size_t sm = sizeof(double2) * 2 * (size_t)C.nc * C.nc;
  MG_CUDA(cudaFuncSetAttribute(k_coarse_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_coarse_invert<<<G.nsites, 256, sm, s>>>(C.nc, C.X.as<float2>(), C.Xinv.as<float2>(), flags);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- folded links
// One CTA per (odd site o, direction d): A_d(o) = X^{-1}(o) Y_d(o) X^{-1}(o + d).
template <int ST>
__global__ void k_fold_eo(int nc, int half, const int* __restrict__ nbr, const void* __restrict__ Y,
                          const float* __restrict__ Ys, const float2* __restrict__ Xinv, float2* A) {
  extern __shared__ __align__(16) float2 fs[];  // Xo, Yd, Xn, T: 4 nc^2
  const int o = half + blockIdx.x, d = blockIdx.y;
  const int n2 = nc * nc;
  float2* Xo = fs;
  float2* Yd = fs + n2;
  float2* Xn = fs + 2 * n2;
  float2* T = fs + 3 * n2;
  const int nb = nbr[(size_t)o * 8 + d];
  const float sc = Ys[(size_t)o * 8 + d];
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const int i = t / nc, j = t % nc;
    Xo[t] = Xinv[(size_t)o * n2 + t];
    const cx<float> y = sget<ST>(Y, (((size_t)o * nc + i) * 8 + d) * nc + j);
    Yd[t] = make_float2(sc * y.re, sc * y.im);
    Xn[t] = Xinv[(size_t)nb * n2 + t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {  // T = Yd Xn
    const int i = t / nc, j = t % nc;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < nc; k++) {
      const float2 a = Yd[i * nc + k], b = Xn[k * nc + j];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    T[t] = make_float2(re, im);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {  // A = Xo T
    const int i = t / nc, j = t % nc;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < nc; k++) {
      const float2 a = Xo[i * nc + k], b = T[k * nc + j];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    A[((((size_t)(o - half)) * nc + i) * 8 + d) * nc + j] = make_float2(re, im);
  }
}

template <int ST>
__global__ void k_cat_links(int nc, int nsites, const void* __restrict__ Y, const float* __restrict__ Ys,
                            const float2* __restrict__ X, float2* A) {
  const size_t total = (size_t)nsites * nc * 9 * nc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % nc);
    const int d = (int)((t / nc) % 9);
    const size_t row = t / ((size_t)9 * nc);  // s * nc + i
    const size_t s = row / nc;
    if (d < 8) {
      const cx<float> y = sget<ST>(Y, (row * 8 + d) * nc + j);
      const float sc = Ys[s * 8 + d];
      A[t] = make_float2(sc * y.re, sc * y.im);
    } else {
      A[t] = X[row * nc + j];
    }
  }
}

void coarse_fold_links(const LevelGeom& G, CoarseOp& C, cudaStream_t s) {
  const int nc = C.nc;
  auto run = [&](auto st) {
    constexpr int ST = decltype(st)::value;
    if (G.eo) {
      const int nodd = G.nsites - G.half;
      C.A.alloc(sizeof(float2) * (size_t)nodd * nc * 8 * nc);
      const size_t sm = sizeof(float2) * 4 * (size_t)nc * nc;
      MG_CUDA(cudaFuncSetAttribute(k_fold_eo<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_fold_eo<ST><<<dim3(nodd, 8), 256, sm, s>>>(nc, G.half, G.d_nbr.as<int>(), C.Y.get(), C.Yscale.as<float>(),
                                                   C.Xinv.as<float2>(), C.A.as<float2>());
    } else {
      C.A.alloc(sizeof(float2) * (size_t)G.nsites * nc * 9 * nc);
      k_cat_links<ST><<<152 * 8, 256, 0, s>>>(nc, G.nsites, C.Y.get(), C.Yscale.as<float>(), C.X.as<float2>(),
                                              C.A.as<float2>());
    }
    MG_LAUNCH();
  };
  switch (C.store) {
    case STORE_F32: run(std::integral_constant<int, STORE_F32>()); break;
    case STORE_F16: run(std::integral_constant<int, STORE_F16>()); break;
    default: run(std::integral_constant<int, STORE_BF16>()); break;
  }
}

// --------------------------------------------------------------------------- 16-bit links
// One CTA per tile (site s = blockIdx.x, block d = blockIdx.y) of an FP32 link
// array [nsites][nc][nb][nc]: scale = largest |Re|, |Im| of the tile (1 for
// an all-zero tile), stored value = link / scale in format ST.
template <int ST>
__global__ void k_quantize_links(int nc, int nb, const float2* __restrict__ in, void* out, float* scale) {
  __shared__ float smax[32];
  __shared__ float sc_s;
  const int s = blockIdx.x, d = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n2 = nc * nc;
  float m = 0.f;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const int i = t / nc, j = t % nc;
    const float2 z = in[(((size_t)s * nc + i) * nb + d) * nc + j];
    m = fmaxf(m, fmaxf(fabsf(z.x), fabsf(z.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) smax[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int q = 0; q < nw; q++) v = fmaxf(v, smax[q]);
    sc_s = v > 0.f ? v : 1.f;
    scale[(size_t)s * nb + d] = sc_s;
  }
  __syncthreads();
  const float inv = 1.f / sc_s;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const int i = t / nc, j = t % nc;
    const size_t e = (((size_t)s * nc + i) * nb + d) * nc + j;
    const float2 z = in[e];
    sput<ST>(out, e, mkc(z.x * inv, z.y * inv));
  }
}

namespace {
// replaces `buf` ([nsites][nc][nb][nc] FP32) by its 16-bit copy; scales -> `scale`
void quantize_array(DBuf& buf, DBuf& scale, int nsites, int nc, int nb, int store, cudaStream_t s) {
  DBuf q(sizeof(uint32_t) * (size_t)nsites * nc * nb * nc);
  scale.alloc(sizeof(float) * (size_t)nsites * nb);
  const dim3 grid(nsites, nb);
  if (store == STORE_F16)
    k_quantize_links<STORE_F16><<<grid, 256, 0, s>>>(nc, nb, buf.as<float2>(), q.get(), scale.as<float>());
  else
    k_quantize_links<STORE_BF16><<<grid, 256, 0, s>>>(nc, nb, buf.as<float2>(), q.get(), scale.as<float>());
  MG_LAUNCH();
  MG_CUDA(cudaStreamSynchronize(s));
  buf = std::move(q);
}
}  // namespace

void quantize_links(const LevelGeom& G, CoarseOp& C, int store, cudaStream_t s) {
  if (store == STORE_F32) return;
  if (C.store != STORE_F32) raise(MG_ERR_STATE, "coarse links are already quantised");
  if (C.A.get()) raise(MG_ERR_STATE, "quantise the links before folding them");
  quantize_array(C.Y, C.Yscale, G.nsites, C.nc, 8, store, s);
  C.store = store;
}

template <int ST>
__global__ void k_links_abi(int nc, int nsites, const int* __restrict__ lex_of, const void* Y,
                            const float* __restrict__ Ys, const float2* __restrict__ X, double2* Yabi, double2* Xabi) {
  const size_t per = (size_t)9 * nc * nc;
  const size_t total = (size_t)nsites * per;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t s = t / per;
    const int r = (int)(t % per);
    const int d = r / (nc * nc), i = (r / nc) % nc, j = r % nc;
    const size_t lex = (size_t)lex_of[s];
    if (d < 8) {
      const cx<float> z = sget<ST>(Y, ((s * nc + i) * 8 + d) * nc + j);
      const double sc = Ys[s * 8 + d];
      Yabi[((lex * 8 + d) * nc + i) * nc + j] = make_double2(sc * z.re, sc * z.im);
    } else {
      const float2 z = X[(s * nc + i) * nc + j];
      Xabi[(lex * nc + i) * nc + j] = make_double2(z.x, z.y);
    }
  }
}

void coarse_links_abi(const LevelGeom& G, const CoarseOp& C, double* Y_abi, double* X_abi, cudaStream_t s) {
  const int nc = C.nc;
  const int* lex = G.d_lex_of.as<int>();
  switch (C.store) {
    case STORE_F32:
      k_links_abi<STORE_F32><<<152 * 8, 256, 0, s>>>(nc, G.nsites, lex, C.Y.get(), C.Yscale.as<float>(),
                                                     C.X.as<float2>(), (double2*)Y_abi, (double2*)X_abi);
      break;
    case STORE_F16:
      k_links_abi<STORE_F16><<<152 * 8, 256, 0, s>>>(nc, G.nsites, lex, C.Y.get(), C.Yscale.as<float>(),
                                                     C.X.as<float2>(), (double2*)Y_abi, (double2*)X_abi);
      break;
    default:
      k_links_abi<STORE_BF16><<<152 * 8, 256, 0, s>>>(nc, G.nsites, lex, C.Y.get(), C.Yscale.as<float>(),
                                                      C.X.as<float2>(), (double2*)Y_abi, (double2*)X_abi);
      break;
  }
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- Philox / packing
__global__ void k_philox_coarse(int nsites, int ndof, const int* lex_of, uint64_t seed, int level, int k, float2* out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)nsites * ndof) return;
  const int s = (int)(t / ndof), d = (int)(t % ndof);
  const cx<double> z = philox_gauss(seed, level, k, lex_of[s], d);
  out[t] = make_float2((float)z.re, (float)z.im);
}

void philox_coarse_vector(const LevelGeom& G, uint64_t seed, int level, int k, float* out, cudaStream_t s) {
  const size_t n = G.vec_complex();
  k_philox_coarse<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G.nsites, G.ndof, G.d_lex_of.as<int>(), seed, level, k,
                                                              (float2*)out);
  MG_LAUNCH();
}

__global__ void k_pack_coarse(int nsites, int ndof, const int* lex_of, const double2* abi, float2* v) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)nsites * ndof) return;
  const int s = (int)(t / ndof), d = (int)(t % ndof);
  const double2 z = abi[(size_t)lex_of[s] * ndof + d];
  v[t] = make_float2((float)z.x, (float)z.y);
}

__global__ void k_unpack_coarse(int nsites, int ndof, const int* lex_of, const float2* v, double2* abi) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)nsites * ndof) return;
  const int s = (int)(t / ndof), d = (int)(t % ndof);
  const float2 z = v[t];
  abi[(size_t)lex_of[s] * ndof + d] = make_double2(z.x, z.y);
}

void pack_coarse(const LevelGeom& G, const double* abi, float* v, cudaStream_t s) {
  const size_t n = G.vec_complex();
  k_pack_coarse<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G.nsites, G.ndof, G.d_lex_of.as<int>(), (const double2*)abi,
                                                            (float2*)v);
  MG_LAUNCH();
}

void unpack_coarse(const LevelGeom& G, const float* v, double* abi, cudaStream_t s) {
  const size_t n = G.vec_complex();
  k_unpack_coarse<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G.nsites, G.ndof, G.d_lex_of.as<int>(), (const float2*)v,
                                                              (double2*)abi);
  MG_LAUNCH();
}

// --------------------------------------------------------------------------- block Gram-Schmidt
struct GSArgs {
  TArgs a;
  const float* V;       // nv level vectors, vector k at V + k * vstride
  size_t vstride;       // floats between consecutive vectors
  double2* Q;           // [ncoarse][2][nv][L]
  int L;                // nb * ndof / 2
};

__global__ void k_gs_gather(GSArgs g) {
  const int cc = blockIdx.x;
  const int nv = g.a.nv, hd = g.a.ndof / 2, L = g.L;
  const size_t per = (size_t)2 * nv * L;
  for (size_t t = threadIdx.x; t < per; t += blockDim.x) {
    const int ch = (int)(t / ((size_t)nv * L));
    const int k = (int)((t / L) % nv);
    const int l = (int)(t % L);
    const int i = l / hd, c = ch * hd + l % hd;
    const int idx = g.a.blockmap[cc * g.a.nb + i];
    const cx<float> z = fget(g.a.fa, g.V + (size_t)k * g.vstride, idx, c);
    g.Q[(size_t)cc * per + t] = make_double2(z.re, z.im);
  }
}

// one CTA per (coarse site, chirality): modified Gram-Schmidt, every vector
// projected twice, FP64 accumulation; breakdown if the norm after projection
// drops below kGSBreakdown of the norm before.  The vectors arrive in FP32,
// so dependence is only resolvable to about 1e-7: the threshold is 1e-6
// (the FP64 oracle uses 1e-10 on FP64 vectors).
constexpr double kGSBreakdown = 1e-6;

__global__ void k_block_gs(GSArgs g, int* flags) {
  __shared__ double red[2][32];
  const int blk = blockIdx.x;  // cc * 2 + ch
  const int nv = g.a.nv, L = g.L;
  double2* Q = g.Q + (size_t)blk * nv * L;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto block_sum2 = [&](double x, double y, double& ox, double& oy) {
    x = warp_sum(x);
    y = warp_sum(y);
    __syncthreads();
    if (lane == 0) {
      red[0][wid] = x;
      red[1][wid] = y;
    }
    __syncthreads();
    double sx = 0, sy = 0;
    for (int q = 0; q < nw; q++) {
      sx += red[0][q];
      sy += red[1][q];
    }
    ox = sx;
    oy = sy;
  };
  for (int k = 0; k < nv; k++) {
    double2* w = Q + (size_t)k * L;
    double n0 = 0, dummy;
    {
      double a = 0;
      for (int l = threadIdx.x; l < L; l += blockDim.x) a += w[l].x * w[l].x + w[l].y * w[l].y;
      block_sum2(a, 0.0, n0, dummy);
    }
    for (int pass = 0; pass < 2; pass++)
      for (int j = 0; j < k; j++) {
        const double2* q = Q + (size_t)j * L;
        double re = 0, im = 0;
        for (int l = threadIdx.x; l < L; l += blockDim.x) {
          re += q[l].x * w[l].x + q[l].y * w[l].y;
          im += q[l].x * w[l].y - q[l].y * w[l].x;
        }
        double dre, dim;
        block_sum2(re, im, dre, dim);
        for (int l = threadIdx.x; l < L; l += blockDim.x) {
          w[l].x -= dre * q[l].x - dim * q[l].y;
          w[l].y -= dre * q[l].y + dim * q[l].x;
        }
        __syncthreads();
      }
    double n1 = 0;
    {
      double a = 0;
      for (int l = threadIdx.x; l < L; l += blockDim.x) a += w[l].x * w[l].x + w[l].y * w[l].y;
      block_sum2(a, 0.0, n1, dummy);
    }
    if (threadIdx.x == 0 && (!(n0 > 0) || !(sqrt(n1) >= kGSBreakdown * sqrt(n0)))) atomicExch(&flags[FLAG_GS_BREAKDOWN], 1);
    const double f = n1 > 0 ? 1.0 / sqrt(n1) : 0.0;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
      w[l].x *= f;
      w[l].y *= f;
    }
    __syncthreads();
  }
}

// scale per (coarse site, chirality): 1 for FP32 storage, else the largest
// |Re|, |Im| of the tile so that the stored values lie in [-1, 1]
template <int ST>
__global__ void k_gs_scatter(GSArgs g, void* P, float* Ps) {
  __shared__ float smax[2][32];
  __shared__ float scale_s[2];
  const int cc = blockIdx.x;
  const int nv = g.a.nv, hd = g.a.ndof / 2, L = g.L;
  const size_t per = (size_t)2 * nv * L;
  const double2* Qc = g.Q + (size_t)cc * per;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float m[2] = {0.f, 0.f};
  if (ST != STORE_F32)
    for (size_t t = threadIdx.x; t < per; t += blockDim.x) {
      const int ch = (int)(t / ((size_t)nv * L));
      const double2 z = Qc[t];
      m[ch] = fmaxf(m[ch], fmaxf(fabsf((float)z.x), fabsf((float)z.y)));
    }
  for (int ch = 0; ch < 2; ch++) {
    float v = m[ch];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) smax[ch][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float v = 0.f;
    for (int q = 0; q < nw; q++) v = fmaxf(v, smax[threadIdx.x][q]);
    scale_s[threadIdx.x] = (ST == STORE_F32 || v == 0.f) ? 1.f : v;
    Ps[cc * 2 + threadIdx.x] = scale_s[threadIdx.x];
  }
  __syncthreads();
  for (size_t t = threadIdx.x; t < per; t += blockDim.x) {
    const int ch = (int)(t / ((size_t)nv * L));
    const int k = (int)((t / L) % nv);
    const int l = (int)(t % L);
    const int i = l / hd, c = ch * hd + l % hd;
    const double2 z = Qc[t];
    const float inv = 1.f / scale_s[ch];
    sput<ST>(P, ((size_t)(cc * g.a.nb + i) * g.a.ndof + c) * nv + k, mkc((float)z.x * inv, (float)z.y * inv));
  }
}

void block_orthonormalize(TransferOp& T, const float* const* V, DBuf& scratch, int* flags, cudaStream_t s) {
  GSArgs g;
  g.a = targs(T);
  g.V = V[0];
  g.vstride = (T.nv > 1) ? (size_t)(V[1] - V[0]) : 0;
  for (int k = 2; k < T.nv; k++)
    if ((size_t)(V[k] - V[0]) != k * g.vstride) raise(MG_ERR_ARG, "null vectors must be equally spaced");
  g.L = T.nb * T.fine_ndof / 2;
  const size_t need = sizeof(double2) * (size_t)T.ncoarse * 2 * T.nv * g.L;
  if (scratch.bytes() < need) scratch.alloc(need);
  g.Q = scratch.as<double2>();
  k_gs_gather<<<T.ncoarse, kBS, 0, s>>>(g);
  MG_LAUNCH();
  k_block_gs<<<T.ncoarse * 2, kBS, 0, s>>>(g, flags);
  MG_LAUNCH();
  switch (T.store) {
    case STORE_F32: k_gs_scatter<STORE_F32><<<T.ncoarse, kBS, 0, s>>>(g, T.P.get(), T.Pscale.as<float>()); break;
    case STORE_F16: k_gs_scatter<STORE_F16><<<T.ncoarse, kBS, 0, s>>>(g, T.P.get(), T.Pscale.as<float>()); break;
    default: k_gs_scatter<STORE_BF16><<<T.ncoarse, kBS, 0, s>>>(g, T.P.get(), T.Pscale.as<float>()); break;
  }
  MG_LAUNCH();
}

}  // namespace mg
