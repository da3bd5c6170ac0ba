// hse_peaks.cu -- arithmetic-pipe throughput of the device, measured.
//
// The stages of the evaluation are bound by different pipes: the real-space
// pairs inside rc64 by FP64 multiply-adds, the outer shell and the mixed path by
// FP32, the Fourier part of FP64 plans by double-float (df64) multiply-adds on
// the FP32 pipe.  hse_measure_pipe_peaks times long chains of each operation on
// every SM, so that roofline fractions can be stated against measured
// throughputs instead of data-sheet figures.  The paper has no counterpart.
#include <cuda_runtime.h>

#include <cstdio>

#include "hse_df64.cuh"
#include "hse_internal.cuh"

namespace {

constexpr int kChains = 8;    // independent accumulators per thread
constexpr int kThreads = 256;

// kChains independent FMA chains of `iters` steps per thread; the result is
// stored so that nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T b, T c, T* out) {
  T acc[kChains];
  for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 4
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
  T s = 0;
  for (int k = 0; k < kChains; ++k) s += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the grid element multiply-accumulate of the double-float spread and gather
// (acc + a b, product unnormalised, sum renormalised)
__global__ void __launch_bounds__(kThreads) k_df64_chains(int iters, float bh, float bl, float* out) {
  using hse::df;
  df acc[kChains];
  const df b(bh, bl);
  for (int k = 0; k < kChains; ++k) acc[k] = df((float)(threadIdx.x + k) * 1e-3f, 0.f);
  // acc_k += acc_{k+1} b: the product's operands change every step, as a
  // window weight and a strength do in the spread
#pragma unroll 2
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = hse::mac(acc[k], acc[(k + 1) % kChains], b);
  float s = 0.f;
  for (int k = 0; k < kChains; ++k) s += acc[k].hi + acc[k].lo;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Seconds of one launch of `fn`, best of three after a warm-up.
template <typename F>
static cudaError_t best_time(F fn, double* seconds) {
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  double best = 1e30;
  fn();
  for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
    cudaEventRecord(e0);
    fn();
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms * 1e-3 < best) best = ms * 1e-3;
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *seconds = best;
  return err;
}

extern "C" hse_status hse_measure_pipe_peaks(hse_pipe_peaks* out) {
  if (!out) return HSE_ERR_INVALID;
  *out = hse_pipe_peaks{};
  int dev = 0, n_sm = 0, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return hse::set_err(nullptr, HSE_ERR_CUDA, "hse_measure_pipe_peaks: device query");
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int blocks = n_sm * 4;  // 1024 threads per SM
  const size_t n_out = (size_t)blocks * kThreads;
  double* buf = nullptr;
  if (cudaMalloc(&buf, n_out * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return hse::set_err(nullptr, HSE_ERR_OOM, "hse_measure_pipe_peaks: %zu bytes", n_out * sizeof(double));
  }
  const int it64 = 2048, it32 = 65536, itdf = 4096;
  double t64 = 0, t32 = 0, tdf = 0;
  cudaError_t e = best_time([&] { k_fma_chains<double><<<blocks, kThreads>>>(it64, 0.9999999, 1e-7, buf); }, &t64);
  if (e == cudaSuccess)
    e = best_time([&] { k_fma_chains<float><<<blocks, kThreads>>>(it32, 0.9999f, 1e-4f, (float*)buf); }, &t32);
  if (e == cudaSuccess)
    e = best_time([&] { k_df64_chains<<<blocks, kThreads>>>(itdf, 1e-4f, 1e-12f, (float*)buf); }, &tdf);
  cudaFree(buf);
  if (e != cudaSuccess) return hse::set_err(nullptr, HSE_ERR_CUDA, "hse_measure_pipe_peaks: %s", cudaGetErrorString(e));
  const double threads = (double)n_out;
  out->fp64_tflops = 2.0 * threads * kChains * it64 / t64 / 1e12;
  out->fp32_tflops = 2.0 * threads * kChains * it32 / t32 / 1e12;
  // one chain step is one df64 multiply-add (2 flops)
  out->df64_tflops = 2.0 * threads * kChains * itdf / tdf / 1e12;
  out->n_sm = n_sm;
  out->sm_clock_mhz = clk_khz / 1000.0;
  return HSE_OK;
}
