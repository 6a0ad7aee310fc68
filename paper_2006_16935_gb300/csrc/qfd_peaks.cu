// qfd_fma_rate: the measured FMA issue rate of the FP64 or the FP32 pipe, the
// roofline denominator of the passes that are bound by vector arithmetic
// rather than by HBM (the complex128 transforms run on the FP64 pipe, the
// complex64 and double-float ones on the FP32 pipe; no tensor cores are used).
//
// Every thread runs CHAINS independent fused multiply-add recurrences
// x <- x * a + b for `iters` iterations, so the pipe always has independent
// work to issue.  The grid fills every SM several times over.  The chains are
// summed and compared with a value they never take, which keeps the compiler
// from removing them; nothing is written in practice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qfd.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(THREADS) k_fma_chains(R* __restrict__ sink, int iters, R a, R b) {
  R x[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) x[j] = (R)(threadIdx.x + j) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = fma(x[j], a, b);
  }
  R s = 0;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += x[j];
  if (s == (R)-12345.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" qfd_status qfd_fma_rate(int fp64, double* tflops) {
  if (!tflops || (fp64 != 0 && fp64 != 1)) return QFD_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QFD_ERR_CUDA;
  const int blocks = sms * 8;  // 64 warps' worth of CTAs per SM, resident in turns
  // about 0.1 s per launch at the rates of this GPU class
  const int iters = fp64 ? 20000 : 1000000;
  void* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * sizeof(double)) != cudaSuccess) return QFD_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  qfd_status st = QFD_OK;
  float best = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = QFD_ERR_CUDA;
  for (int rep = 0; st == QFD_OK && rep < 6; ++rep) {  // one warm-up, best of five
    cudaEventRecord(e0, 0);
    if (fp64)
      k_fma_chains<double><<<blocks, THREADS>>>(static_cast<double*>(sink), iters, 0.9999999, 1e-7);
    else
      k_fma_chains<float><<<blocks, THREADS>>>(static_cast<float*>(sink), iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = QFD_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (st != QFD_OK) return st;
  const double flops = 2.0 * CHAINS * (double)iters * (double)blocks * THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return QFD_OK;
}
