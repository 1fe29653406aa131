// Arithmetic peaks of this GPU measured by the library itself (no counterpart in the paper): the FP32
// and FP64 fused multiply-add rates of the CUDA cores, the denominators of the roofline fractions of the
// FP32 path and of the FP64 reductions.  Each thread runs eight independent FMA chains (enough
// independent work to cover the FMA latency at full occupancy); the grid is eight 256-thread blocks per SM.
#include <cuda_runtime.h>

namespace tdo {

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(T *out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)threadIdx.x * (T)1e-7 + (T)i;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1.25) out[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

template <typename T>
static cudaError_t peak_t(int n_sm, int iters, cudaStream_t st, double *tflops) {
  T *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * 8 * (size_t)n_sm);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = 8 * n_sm, threads = 256;
  double best = 0.0;
  if (e == cudaSuccess) {
    k_peak_fma<T><<<blocks, threads, 0, st>>>(out, iters / 8, (T)0.9999999, (T)1e-7);   // warm-up
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, st);
      k_peak_fma<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.9999999, (T)1e-7);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      const double flop = 2.0 * 8.0 * (double)iters * blocks * threads;
      if (e == cudaSuccess && ms > 0.f && flop / (ms * 1e-3) / 1e12 > best) best = flop / (ms * 1e-3) / 1e12;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  *tflops = best;
  return e;
}

}  // namespace tdo

cudaError_t measure_fma_peak(int fp64, int n_sm, cudaStream_t st, double *tflops) {
  return fp64 ? tdo::peak_t<double>(n_sm, 1 << 12, st, tflops) : tdo::peak_t<float>(n_sm, 1 << 16, st, tflops);
}
