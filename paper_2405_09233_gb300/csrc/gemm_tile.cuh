// One BM x BN output tile of the fused per-slice complex product (see gemm_simt.cu), shared by
// the grid-mapped kernel and the work-list kernel of the batched solver.  NT = (BM/TM)(BN/TN)
// threads, each owning TM x TN outputs.  64 x 64 tiles (4 x 4 per thread) reuse every shared
// operand four times; 32 x 32 and 16 x 16 tiles spread a small product over more SMs, which is what
// counts on GB300, whose FP64 pipe issues 2 DFMA per clock per SM: a lone 64 x 64 tile needs ~47 us
// per 16-deep reduction step however small the problem.
#pragma once
#include "internal.cuh"

namespace ts {

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmNT = 256;

template <typename Real> struct CplxOf;
template <> struct CplxOf<double> { using T = double2; };
template <> struct CplxOf<float> { using T = float2; };

// Y_k(i0.., j0..) = A1_k B1_k + sgn2 A2_k B2_k for one tile; slices k == 0 and k == nyq are real.
template <typename Real, int BM = kGemmBM, int BN = kGemmBN, int TM = 4, int TN = 4>
__device__ __forceinline__ void gemm_tile(const GemmArgs<typename CplxOf<Real>::T>& a, int k, int i0, int j0) {
  constexpr int BK = kGemmBK, TX = BN / TN, NT = (BM / TM) * TX;
  static_assert(NT == kGemmNT && (BM * BK) % NT == 0 && (BN * BK) % NT == 0, "tile shape");
  using Cplx = typename CplxOf<Real>::T;
  const bool real = (k == 0) || (k == a.nyq);
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;

  __shared__ Real sA[3][BK][BM];
  __shared__ Real sB[3][BK][BN];

  Real acc[3][TM][TN];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < TM; ++q)
#pragma unroll
      for (int r = 0; r < TN; ++r) acc[c][q][r] = Real(0);

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
          Real ar[TM], br[TN];
#pragma unroll
          for (int q = 0; q < TM; ++q) ar[q] = sA[0][c][ty * TM + q];
#pragma unroll
          for (int r = 0; r < TN; ++r) br[r] = sB[0][c][tx * TN + r];
#pragma unroll
          for (int q = 0; q < TM; ++q)
#pragma unroll
            for (int r = 0; r < TN; ++r) acc[0][q][r] = fma(ar[q], br[r], acc[0][q][r]);
        }
      } else {
#pragma unroll 2
        for (int c = 0; c < BK; ++c) {
          Real av[3][TM], bv[3][TN];
#pragma unroll
          for (int z = 0; z < 3; ++z) {
#pragma unroll
            for (int q = 0; q < TM; ++q) av[z][q] = sA[z][c][ty * TM + q];
#pragma unroll
            for (int r = 0; r < TN; ++r) bv[z][r] = sB[z][c][tx * TN + r];
          }
#pragma unroll
          for (int z = 0; z < 3; ++z)
#pragma unroll
            for (int q = 0; q < TM; ++q)
#pragma unroll
              for (int r = 0; r < TN; ++r) acc[z][q][r] = fma(av[z][q], bv[z][r], acc[z][q][r]);
        }
      }
      __syncthreads();
    }
  }

  Cplx* Y = a.Y + a.sY * k;
#pragma unroll
  for (int r = 0; r < TN; ++r) {
    const int j = j0 + tx * TN + r;
    if (j >= a.N) continue;
#pragma unroll
    for (int q = 0; q < TM; ++q) {
      const int i = i0 + ty * TM + q;
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


}  // namespace ts
