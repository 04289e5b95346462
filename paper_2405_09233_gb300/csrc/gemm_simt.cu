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

namespace ts {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename Real> struct CplxOf;
template <> struct CplxOf<double> { using T = double2; };
template <> struct CplxOf<float> { using T = float2; };

template <typename Real>
__global__ void __launch_bounds__(NT, 1) k_gemm_slices(GemmArgs<typename CplxOf<Real>::T> a) {
  using Cplx = typename CplxOf<Real>::T;
  const int k = blockIdx.z;
  const bool real = (k == 0) || (k == a.nyq);
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  __shared__ Real sA[3][BK][BM];
  __shared__ Real sB[3][BK][BN];

  Real acc[3][4][4];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[c][q][r] = Real(0);

  for (int phase = 0; phase < 2; ++phase) {
    const int L = phase == 0 ? a.L1 : a.L2;
    if (L <= 0) continue;
    const Cplx* A = phase == 0 ? a.A1 + a.sA1 * k : a.A2 + a.sA2 * k;
    const Cplx* B = phase == 0 ? a.B1 + a.sB1 * k : a.B2 + a.sB2 * k;
    const int lda = phase == 0 ? a.lda1 : a.lda2;
    const int ldb = phase == 0 ? a.ldb1 : a.ldb2;
    const Real sgn = phase == 0 ? Real(1) : Real(a.sgn2);
    for (int l0 = 0; l0 < L; l0 += BK) {
      // A tile: BM rows x BK columns, column-major source; consecutive threads walk the rows.
#pragma unroll
      for (int q = 0; q < (BM * BK) / NT; ++q) {
        const int e = tid + NT * q;
        const int r = e % BM, c = e / BM;
        Cplx v;
        v.x = Real(0);
        v.y = Real(0);
        if (i0 + r < a.M && l0 + c < L) v = A[(long long)(l0 + c) * lda + i0 + r];
        if (real) v.y = Real(0);
        sA[0][c][r] = v.x;
        sA[1][c][r] = v.y;
        sA[2][c][r] = v.x + v.y;
      }
      // B tile: BK rows x BN columns; consecutive threads walk down a column (contiguous).
#pragma unroll
      for (int q = 0; q < (BN * BK) / NT; ++q) {
        const int e = tid + NT * q;
        const int c = e % BK, jj = e / BK;
        Cplx v;
        v.x = Real(0);
        v.y = Real(0);
        if (j0 + jj < a.N && l0 + c < L) v = B[(long long)(j0 + jj) * ldb + l0 + c];
        if (real) v.y = Real(0);
        v.x *= sgn;
        v.y *= sgn;
        sB[0][c][jj] = v.x;
        sB[1][c][jj] = v.y;
        sB[2][c][jj] = v.x + v.y;
      }
      __syncthreads();
      if (real) {
#pragma unroll 4
        for (int c = 0; c < BK; ++c) {
          Real ar[4], br[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) ar[q] = sA[0][c][ty * 4 + q];
#pragma unroll
          for (int r = 0; r < 4; ++r) br[r] = sB[0][c][tx * 4 + r];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[0][q][r] = fma(ar[q], br[r], acc[0][q][r]);
        }
      } else {
#pragma unroll 2
        for (int c = 0; c < BK; ++c) {
          Real av[3][4], bv[3][4];
#pragma unroll
          for (int z = 0; z < 3; ++z) {
#pragma unroll
            for (int q = 0; q < 4; ++q) av[z][q] = sA[z][c][ty * 4 + q];
#pragma unroll
            for (int r = 0; r < 4; ++r) bv[z][r] = sB[z][c][tx * 4 + r];
          }
#pragma unroll
          for (int z = 0; z < 3; ++z)
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int r = 0; r < 4; ++r) acc[z][q][r] = fma(av[z][q], bv[z][r], acc[z][q][r]);
        }
      }
      __syncthreads();
    }
  }

  Cplx* Y = a.Y + a.sY * k;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int j = j0 + tx * 4 + r;
    if (j >= a.N) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty * 4 + q;
      if (i >= a.M) continue;
      Cplx v;
      if (real) {
        v.x = acc[0][q][r];
        v.y = Real(0);
      } else {
        v.x = acc[0][q][r] - acc[1][q][r];
        v.y = acc[2][q][r] - acc[0][q][r] - acc[1][q][r];
      }
      Y[(long long)j * a.ldy + i] = v;
    }
  }
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
