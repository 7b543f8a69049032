// peak.cu -- measured FP64 FMA throughput of the device: the denominator of
// the FP64 form's roofline (the plain FP64 kernel issues scalar DFMA, so its
// ceiling is the DFMA pipe, not a DGEMM rate).
//
// Every thread runs kChains independent FMA chains x <- x*b + c; with b just
// below 1 the values settle at c/(1-b) and never become subnormal.  The
// result is stored only if it equals a value it cannot take, which keeps
// the chains live without a store per thread.
#include "nbgb_internal.cuh"
#include "../../include/nbgb.h"

namespace nbgb {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 4;
constexpr int kPeakIters = 4096;

__global__ void __launch_bounds__(kPeakThreads)
    dfma_peak_kernel(double b, double c, int iters, double *out) {
  double x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == -1.0) out[blockIdx.x] = s;
}

}  // namespace nbgb

extern "C" int nb_fp64_peak_tflops(int device, double *tflops) {
  if (!tflops) return NB_EINVAL;
  *tflops = 0.0;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  if (device < 0 || device >= n_dev) return NB_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return NB_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return NB_ECUDA;
  int sms = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double *out = nullptr;
  int rc = NB_OK;
  float best_ms = 0.f;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = NB_ECUDA;
  }
  const int blocks = sms * nbgb::kPeakBlocksPerSM;
  if (rc == NB_OK &&
      cudaMalloc(&out, (size_t)(blocks > 0 ? blocks : 1) * sizeof(double)) !=
          cudaSuccess)
    rc = NB_ENOMEM;
  // one warm-up launch, then the best of three timed ones
  for (int rep = 0; rc == NB_OK && rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    nbgb::dfma_peak_kernel<<<blocks, nbgb::kPeakThreads, 0, st>>>(
        0.9999999, 1e-7, nbgb::kPeakIters, out);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = NB_ECUDA;
      break;
    }
    if (rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (rc == NB_OK && best_ms > 0.f) {
    const double fmas = (double)blocks * nbgb::kPeakThreads * nbgb::kChains *
                        nbgb::kPeakIters;
    *tflops = 2.0 * fmas / (best_ms * 1e-3) / 1e12;
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaSetDevice(prev);
  return rc;
}
