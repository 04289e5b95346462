// The FP64 roof of the device, measured: the denominator of the rooflines reported for the FP64
// kernels that run on CUDA cores (the DFMA slice products, the TBAS SpMM and block products).
// Every thread runs kPeakChains independent fused multiply-add chains on registers, so the FP64
// pipe's issue rate, not the 4-8 cycle dependence latency of one chain, sets the pace; kPeakCtasPerSm
// CTAs of kPeakThreads threads per SM give every sub-partition several warps.  x <- a x + b with
// a = 1 - 2^-20 and b = 2^-20 keeps every value near 1 (no overflow, no subnormals), and the sums are
// stored so that no chain is dead code.
#include "internal.cuh"

namespace ts {
namespace {

constexpr int kPeakChains = 8, kPeakThreads = 256, kPeakCtasPerSm = 4, kPeakIters = 16384;

__global__ void __launch_bounds__(kPeakThreads) k_dfma_peak(double* __restrict__ out, int iters, double a,
                                                            double b) {
  double x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = 1.0 + 1e-3 * c + 1e-6 * threadIdx.x;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  out[(long long)blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

}  // namespace

double fp64_fma_peak_tflops(ts_ctx* ctx, cudaStream_t st) {
  int sms = 0;
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int blocks = sms * kPeakCtasPerSm;
  double* out = static_cast<double*>(ctx->ws.get("peak_out", sizeof(double) * (size_t)blocks * kPeakThreads));
  const double a = 1.0 - 1.0 / 1048576.0, b = 1.0 / 1048576.0;
  struct Events {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Events() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } ev;
  TS_CUDA(cudaEventCreate(&ev.e0));
  TS_CUDA(cudaEventCreate(&ev.e1));
  k_dfma_peak<<<blocks, kPeakThreads, 0, st>>>(out, kPeakIters / 8, a, b);   // untimed: load and clocks
  count_launch();
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaEventRecord(ev.e0, st));
  k_dfma_peak<<<blocks, kPeakThreads, 0, st>>>(out, kPeakIters, a, b);
  count_launch();
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaEventRecord(ev.e1, st));
  TS_CUDA(cudaEventSynchronize(ev.e1));
  float ms = 0.f;
  TS_CUDA(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
  const double fmas = (double)blocks * kPeakThreads * kPeakChains * kPeakIters;
  return ms > 0.f ? 2.0 * fmas / (ms * 1e-3) / 1e12 : 0.0;
}

}  // namespace ts
