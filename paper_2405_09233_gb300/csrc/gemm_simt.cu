// Per-Fourier-slice complex products on CUDA cores, FP64 and FP32 (Algorithm 1 step 2; inside M
// it is the fused Y_k = A_k X_k - X_k B_k of Eq. (2) in the Fourier domain).
//
// GB300 runs FP64 at ~1 TFLOP/s on CUDA cores (DFMA and the m8n8k4 DMMA measure within 4% of
// each other), so this kernel is FP64-pipe bound by a wide margin: a 64x64 output tile with
// 16x16 threads of 4x4 outputs reuses every shared-memory operand 4 times, and the global
// traffic is ~1/100 of what the pipe could hide.  The one lever that matters is the number of
// FP64 operations: the complex product uses three real products (Gauss):
//   T1 = sum ar*br, T2 = sum ai*bi, T3 = sum (ar+ai)(br+bi);  re = T1 - T2, im = T3 - T1 - T2,
// 3 DFMA per complex multiply-add instead of 4.  The sums ar+ai, br+bi are formed once per
// shared-memory tile element.  Slices k = 0 and k = p/2 are real (their imaginary parts are
// exactly zero) and take a single real product.
#include "internal.cuh"
#include "gemm_tile.cuh"

namespace ts {
namespace {

template <typename Real, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(kGemmNT, 1) k_gemm_slices(GemmArgs<typename CplxOf<Real>::T> a) {
  gemm_tile<Real, BM, BN, TM, TN>(a, blockIdx.z, blockIdx.x * BM, blockIdx.y * BN);
}

template <typename Real>
__global__ void __launch_bounds__(kTinyThreads) k_gemm_tiny(GemmArgs<typename CplxOf<Real>::T> a) {
  gemm_tiny_tile<Real>(a, blockIdx.z, blockIdx.x * kTinyBM, blockIdx.y * kTinyBN);
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) TS_CUDA(cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev));
  return cached[dev];
}

// Otherwise the output tile is the largest of 64, 32, 16 whose grid still covers every SM (a product of a few large
// tiles would leave most of the FP64 pipes idle); 16 when even that does not.
template <typename Real>
void launch_slices(const GemmArgs<typename CplxOf<Real>::T>& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return;
  if (a.L1 <= kTinyL && a.L2 <= kTinyL) {
    dim3 grid((a.M + kTinyBM - 1) / kTinyBM, (a.N + kTinyBN - 1) / kTinyBN, a.K);
    TS_REQUIRE(grid.y <= 65535 && grid.z <= 65535, "slice GEMM grid too large");
    k_gemm_tiny<Real><<<grid, kTinyThreads, 0, st>>>(a);
    count_launch();
    TS_CUDA(cudaGetLastError());
    return;
  }
  const long long sms = sm_count();
  auto ctas = [&](int t) { return (long long)a.K * ((a.M + t - 1) / t) * ((a.N + t - 1) / t); };
  const int tile = ctas(64) >= sms ? 64 : (ctas(32) >= sms ? 32 : 16);
  dim3 grid((a.M + tile - 1) / tile, (a.N + tile - 1) / tile, a.K);
  TS_REQUIRE(grid.y <= 65535 && grid.z <= 65535, "slice GEMM grid too large");
  if (tile == 64) k_gemm_slices<Real, 64, 64, 4, 4><<<grid, kGemmNT, 0, st>>>(a);
  else if (tile == 32) k_gemm_slices<Real, 32, 32, 2, 2><<<grid, kGemmNT, 0, st>>>(a);
  else k_gemm_slices<Real, 16, 16, 1, 1><<<grid, kGemmNT, 0, st>>>(a);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace

void zgemm_slices_f64(const ZGemmArgs& a, cudaStream_t st) { launch_slices<double>(a, st); }

void cgemm_slices_f32(const CGemmArgs& a, cudaStream_t st) { launch_slices<float>(a, st); }

}  // namespace ts
