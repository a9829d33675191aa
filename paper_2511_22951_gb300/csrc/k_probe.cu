// k_probe.cu -- FMA throughput probe for the ALU rooflines (GB300, sm_103a).
//
// The measured peaks the roofline divides by are an HBM copy and a cuBLAS
// bf16 GEMM; neither bounds the FP64 force loops or the FP32 descriptor
// kernel, whose bound is the FP64 / FP32 FMA pipe.  This probe measures
// that pipe: every thread runs 8 independent FMA chains (enough to cover
// the pipe latency at full occupancy) for `iters` iterations on a grid of
// 8 blocks of 256 threads per SM; FLOPs = 2 x 8 x iters x threads over the
// CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "mdk.h"
#include "mdk_internal.cuh"

namespace mdk {
namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T b, T c) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int k = 0; k < iters; ++k) {
    a0 = a0 * b + c;
    a1 = a1 * b + c;
    a2 = a2 * b + c;
    a3 = a3 * b + c;
    a4 = a4 * b + c;
    a5 = a5 * b + c;
    a6 = a6 * b + c;
    a7 = a7 * b + c;
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == (T)-12345.0) out[blockIdx.x] = s;  // keeps the chains live; never true
}

template <class T>
int run(int iters, double *tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MDK_ERR_CUDA;
  const int blocks = 8 * sms, threads = 256;
  T *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int r = MDK_OK;
  if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return MDK_ERR_CUDA;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = MDK_ERR_CUDA;
  // b < 1 and c small keep the values finite and normal
  const T b = (T)0.999999, c = (T)1e-7;
  if (r == MDK_OK) {
    k_fma_probe<T><<<blocks, threads>>>(out, iters / 10, b, c);  // warm-up
    cudaEventRecord(e0);
    k_fma_probe<T><<<blocks, threads>>>(out, iters, b, c);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        !(ms > 0.f))
      r = MDK_ERR_CUDA;
    else
      *tflops = 2.0 * 8.0 * (double)iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return r;
}

}  // namespace
}  // namespace mdk

extern "C" int mdk_fma_peak(int precision, double *tflops) {
  if (!tflops || (precision != MDK_FP64 && precision != MDK_MIXED)) return MDK_ERR_BAD_ARG;
  return precision == MDK_FP64 ? mdk::run<double>(1 << 14, tflops)
                               : mdk::run<float>(1 << 18, tflops);
}
