// sph_peak.cu -- arithmetic peaks of the GPU the library runs on, measured
// (declared in include/sph.h as sph_measure_fma_peak): the denominators of
// the ALU roofline that the pair sweeps are reported against beside HBM.
//
// Every thread runs eight independent multiply-add chains in the chosen
// precision (enough in flight to cover the pipeline latency), the grid
// holds eight 256-thread blocks per SM, and the kernel is timed with CUDA
// events after one untimed launch; each chain's final value is stored so
// that nothing is optimised away.
#include <cuda_runtime.h>

#include <string>

#include "sph_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a0, T b, int iters, T *out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = a0 + (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], b, a0);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(double *flops_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return sphk::set_error(SPH_ERR_CUDA, "sph_measure_fma_peak: no device");
  const int blocks = 8 * sms;
  const int iters = sizeof(T) == 4 ? 1 << 15 : 1 << 11;
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess)
    return sphk::set_error(SPH_ERR_ALLOC, "sph_measure_fma_peak: output buffer");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a0 and b keep the chains bounded (|b| < 1) and unknown to the compiler
  const T a0 = (T)0.5, b = (T)0.999;
  k_fma_chains<T><<<blocks, kThreads>>>(a0, b, iters, out);  // warm-up
  float best = 0.0f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, kThreads>>>(a0, b, iters, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0 || ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess)
    return sphk::set_error(SPH_ERR_CUDA, (std::string("sph_measure_fma_peak: ") + cudaGetErrorString(e)).c_str());
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *flops_out = flops / (best * 1e-3);
  return SPH_OK;
}

}  // namespace

extern "C" int sph_measure_fma_peak(int32_t precision, double *flops_per_s) {
  if (!flops_per_s || (precision != SPH_PREC_FP32 && precision != SPH_PREC_FP64))
    return sphk::set_error(SPH_ERR_ARG, "sph_measure_fma_peak: bad precision or NULL output");
  return precision == SPH_PREC_FP32 ? measure<float>(flops_per_s) : measure<double>(flops_per_s);
}
