// FMA throughput microbenchmark (cgl_measure_fma_peak): the measured FP64
// and FP32 ALU peaks that the SIMT kernels' roofline fractions are set
// against, next to the peaks derived from unit counts and clocks.
//
// Every thread runs kChains independent FMA chains x <- x * a + b for `iters`
// rounds (a, b runtime values, so nothing folds), on a grid of
// 8 blocks x 256 threads per SM; each thread writes its sum so the chains
// stay live.  Flops = 2 * kChains * iters * threads; the time is the CUDA
// event interval around the launch, after one untimed warm-up launch.
#include "cgl_internal.cuh"

namespace cgl {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;
constexpr int kChains = 8;

template <class T> __global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(T a, T b, int iters, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T> static int measure(int iters, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CGL_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CGL_ECUDA;
  const int blocks = sms * kPeakBlocksPerSm;
  T* out = nullptr;
  if (cudaMallocAsync(&out, (size_t)blocks * kPeakThreads * sizeof(T), s) != cudaSuccess) return CGL_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = CGL_ECUDA;
  float ms = 0;
  const T a = (T)0.999999, b = (T)1e-6;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, s>>>(a, b, iters, out);
    cudaEventRecord(e0, s);
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, s>>>(a, b, iters, out);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0) {
      const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
      *tflops = flops / (ms * 1e-3) / 1e12;
      st = CGL_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) st = CGL_ECUDA;
  return st;
}

}  // namespace cgl

extern "C" int cgl_measure_fma_peak(int precision, int iters, double* tflops, void* stream) {
  using namespace cgl;
  if (!tflops || iters < 1) return CGL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == CGL_F64) return measure<double>(iters, tflops, s);
  if (precision == CGL_F32) return measure<float>(iters, tflops, s);
  return CGL_EINVAL;
}
