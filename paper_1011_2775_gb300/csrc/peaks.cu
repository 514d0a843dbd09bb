// CUDA-core FMA throughput of this GPU in FP32 and FP64, measured with CUDA
// events: the denominators of the FP64-ALU-bound kernels' roofline (the FP64
// dslash and link derivative) and of the FP32 coarse GEMVs.
//
// Every thread runs kChains independent FMA chains of kIters steps; the grid
// fills every SM with kBlocksPerSM blocks.  Inputs come from the kernel
// arguments and the results are stored conditionally, so no step can be
// removed by the compiler.
#include "internal.h"

namespace mg {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T a, T b, int iters, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) {
      if constexpr (sizeof(T) == 4)
        x[c] = fmaf(x[c], a, b);
      else
        x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  if (s == (T)-1.2345) out[blockIdx.x] = s;   // never true for the arguments used
}

template <typename T>
double fma_tflops(int iters) {
  int dev = 0, sms = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * kBlocksPerSM;
  DBuf out(sizeof(T) * grid);
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_peak<T><<<grid, kThreads>>>(a, b, iters / 10 + 1, out.as<T>());   // warm-up
  MG_LAUNCH();
  MG_CUDA(cudaEventRecord(e0));
  k_fma_peak<T><<<grid, kThreads>>>(a, b, iters, out.as<T>());
  MG_LAUNCH();
  MG_CUDA(cudaEventRecord(e1));
  MG_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * kChains * (double)iters * kThreads * grid;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace

double fma_peak_tflops(int prec) {
  return prec == MG_FP64 ? fma_tflops<double>(1 << 14) : fma_tflops<float>(1 << 17);
}

}  // namespace mg
