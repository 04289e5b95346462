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

constexpr int BM = kGemmBM, BN = kGemmBN, NT = kGemmNT;

template <typename Real>
__global__ void __launch_bounds__(NT, 1) k_gemm_slices(GemmArgs<typename CplxOf<Real>::T> a) {
  gemm_tile<Real>(a, blockIdx.z, blockIdx.x * BM, blockIdx.y * BN);
}

}  // namespace

void zgemm_slices_f64(const ZGemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return;
  dim3 grid((a.M + BM - 1) / BM, (a.N + BN - 1) / BN, a.K);
  TS_REQUIRE(grid.y <= 65535 && grid.z <= 65535, "slice GEMM grid too large");
  k_gemm_slices<double><<<grid, NT, 0, st>>>(a);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void cgemm_slices_f32(const CGemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return;
  dim3 grid((a.M + BM - 1) / BM, (a.N + BN - 1) / BN, a.K);
  TS_REQUIRE(grid.y <= 65535 && grid.z <= 65535, "slice GEMM grid too large");
  k_gemm_slices<float><<<grid, NT, 0, st>>>(a);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace ts
