// Floors of one coarsest-level GCR iteration on this GPU (section
// "Implementation": unpreconditioned GCR on the coarsest lattice), measured
// with CUDA events on the grid the streamed solver runs on:
//
//  * a grid barrier: a cooperative kernel that does nothing but pass the
//    solver's time-bounded grid barrier (every GCR iteration passes three);
//  * the link stream: the bytes one iteration must move through shared
//    memory -- the folded odd-site links A and the even-site links Y -- copied
//    L2 -> shared memory by per-warp double-buffered bulk copies, with no
//    arithmetic, split evenly over every warp of the grid.
//
// Their sum (three barriers + one stream) is what an iteration cannot beat
// with this structure; the solver's own time per iteration is compared with it.
#include "async_copy.cuh"
#include "coarse.h"

namespace mg {
namespace {

constexpr int kFloorThreads = 256;
constexpr int kFloorWarps = kFloorThreads / 32;
constexpr unsigned kFloorStage = 8192;   // bytes per per-warp stage (two stages per warp)

__global__ void __launch_bounds__(kFloorThreads) k_barrier_floor(unsigned* count, int* abort, int nbar, int* flags) {
  unsigned target = 0;
  for (int b = 0; b < nbar; b++)
    if (!grid_barrier(count, abort, target)) {
      if (threadIdx.x == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
      break;
    }
}

struct StreamRegion {
  const unsigned char* p;
  size_t bytes;   // a multiple of 16
};

// stage k (k counts the warp's stages over all repetitions): its source and size
__device__ __forceinline__ void stage_of(const StreamRegion* R, const size_t* b0, const size_t* b1,
                                         const size_t* nst, long long k, const unsigned char** src, unsigned* n) {
  long long q = k % (long long)(nst[0] + nst[1]);
  const int r = q < (long long)nst[0] ? 0 : 1;
  if (r) q -= (long long)nst[0];
  const size_t off = b0[r] + (size_t)q * kFloorStage;
  *src = R[r].p + off;
  *n = (unsigned)min((size_t)kFloorStage, b1[r] - off);
}

__global__ void __launch_bounds__(kFloorThreads) k_stream_floor(StreamRegion A, StreamRegion Y, int reps,
                                                                float* sink, int* flags) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2 * kFloorWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane != 0) return;
  unsigned char* st = smem + (size_t)w * 2 * kFloorStage;
  mbar_init(&bar[2 * w], 1);
  mbar_init(&bar[2 * w + 1], 1);
  mbar_fence_init();
  const StreamRegion R[2] = {A, Y};
  const size_t nw = (size_t)gridDim.x * kFloorWarps, gw = (size_t)blockIdx.x * kFloorWarps + w;
  size_t b0[2], b1[2], nst[2];
  for (int r = 0; r < 2; r++) {
    const size_t units = R[r].bytes / 16;
    b0[r] = units * gw / nw * 16;
    b1[r] = units * (gw + 1) / nw * 16;
    nst[r] = (b1[r] - b0[r] + kFloorStage - 1) / kFloorStage;
  }
  const long long total = (long long)(nst[0] + nst[1]) * reps;
  auto issue = [&](long long k) {
    const unsigned char* src;
    unsigned n;
    stage_of(R, b0, b1, nst, k, &src, &n);
    uint64_t* b = &bar[2 * w + (int)(k & 1)];
    mbar_arrive_expect_tx(b, n);
    bulk_copy_g2s(st + (k & 1) * kFloorStage, src, n, b);
  };
  float acc = 0.f;
  bool ok = true;
  if (total > 0) issue(0);
  for (long long k = 0; k < total; k++) {
    if (k + 1 < total) issue(k + 1);   // into the stage consumed at k - 1
    ok &= mbar_wait(&bar[2 * w + (int)(k & 1)], (unsigned)((k >> 1) & 1));
    acc += *reinterpret_cast<const float*>(st + (k & 1) * kFloorStage);
  }
  if (!ok) atomicExch(&flags[FLAG_TIMEOUT], 1);
  if (acc == -1.2345f) sink[0] = acc;   // never true for link data of a solvable system; keeps the reads
}

}  // namespace

void coarse_floor(const LevelGeom& G, const CoarseOp& C, int grid, int* flags, cudaStream_t s, double* barrier_us,
                  double* stream_us, double* stream_bytes) {
  if (!G.eo || !C.A.get()) raise(MG_ERR_STATE, "the coarse floor needs an even-odd coarsest level");
  const size_t esz = C.store == STORE_F32 ? 8 : 4;
  const size_t lbytes = (size_t)G.half * C.nc * 8 * C.nc;   // link entries of one parity
  StreamRegion A{static_cast<const unsigned char*>(C.A.get()), lbytes * 8};
  StreamRegion Y{static_cast<const unsigned char*>(C.Y.get()), lbytes * esz};   // even sites come first
  *stream_bytes = (double)(A.bytes + Y.bytes);
  DBuf sync(256), sink(64);
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  // barriers: a warm-up launch, then one launch of nbar barriers
  const int nbar = 3000;
  int per = 0;
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_barrier_floor, kFloorThreads, 0));
  int dev = 0, sms = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per < 1 || grid > per * sms) raise(MG_ERR_CUDA, "barrier floor grid cannot be resident");
  float ms = 0;
  for (int pass = 0; pass < 2; pass++) {
    MG_CUDA(cudaMemsetAsync(sync.get(), 0, 256, s));
    unsigned* count = sync.as<unsigned>();
    int* abort = reinterpret_cast<int*>(sync.as<unsigned char>() + 128);
    int nb = pass ? nbar : 10;
    void* params[] = {&count, &abort, &nb, &flags};
    MG_CUDA(cudaEventRecord(e0, s));
    MG_CUDA(cudaLaunchCooperativeKernel((const void*)k_barrier_floor, dim3(grid), dim3(kFloorThreads), params, 0, s));
    MG_LAUNCH();
    MG_CUDA(cudaEventRecord(e1, s));
    MG_CUDA(cudaEventSynchronize(e1));
    MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  *barrier_us = 1e3 * ms / nbar;
  // link stream: a warm-up launch of one repetition, then `reps`
  const size_t smem = (size_t)kFloorWarps * 2 * kFloorStage;
  MG_CUDA(cudaFuncSetAttribute(k_stream_floor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int reps = 20;
  for (int pass = 0; pass < 2; pass++) {
    MG_CUDA(cudaEventRecord(e0, s));
    k_stream_floor<<<grid, kFloorThreads, smem, s>>>(A, Y, pass ? reps : 1, sink.as<float>(), flags);
    MG_LAUNCH();
    MG_CUDA(cudaEventRecord(e1, s));
    MG_CUDA(cudaEventSynchronize(e1));
    MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  *stream_us = 1e3 * ms / reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace mg
