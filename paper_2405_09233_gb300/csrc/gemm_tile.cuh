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
  if (a.gate && *a.gate == 0) return;
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


// Products whose reduction lengths L1, L2 are at most kTinyL (the latency-bound small problems):
// one 8 x 4 output tile per CTA of four warps.  Each phase's operand panels (8 rows of A1 or A2,
// 4 columns of B1 or B2, over the whole reduction) go to shared memory in one round trip; then warp
// w forms the 32 outputs' partial sums over its quarter of the concatenated reduction (phase 1's l,
// then phase 2's) and warp 0 adds the four partials in order.  GB300's FP64 pipe issues one warp's
// DFMA in 64 clocks per SM sub-partition, so a single warp per tile (one sub-partition of four) ran
// ~9 us at n = s = 24, and a 16 x 16 tile of 256 threads spent most of ~19 us on padded work.
constexpr int kTinyL = 64, kTinyBM = 8, kTinyBN = 4, kTinyThreads = 128;

// One 8 x 4 tile (output rows i0.., columns j0..) of slice k; blockDim.x == kTinyThreads.
template <typename Real>
__device__ __forceinline__ void gemm_tiny_tile(const GemmArgs<typename CplxOf<Real>::T>& a, int k, int i0, int j0) {
  using Cplx = typename CplxOf<Real>::T;
  __shared__ Real sA[2][3][kTinyL][kTinyBM];
  __shared__ Real sB[2][3][kTinyL][kTinyBN];
  __shared__ Real sP[kTinyThreads / 32][3][32];
  if (a.gate && *a.gate == 0) return;
  const bool real = (k == 0) || (k == a.nyq);
  const int t = threadIdx.x;
  constexpr int QA = kTinyBM * kTinyL / kTinyThreads, QB = kTinyBN * kTinyL / kTinyThreads;
  for (int phase = 0; phase < 2; ++phase) {
    const int L = phase == 0 ? a.L1 : a.L2;
    const Cplx* A = phase == 0 ? a.A1 + a.sA1 * k : a.A2 + a.sA2 * k;
    const Cplx* B = phase == 0 ? a.B1 + a.sB1 * k : a.B2 + a.sB2 * k;
    const int lda = phase == 0 ? a.lda1 : a.lda2;
    const int ldb = phase == 0 ? a.ldb1 : a.ldb2;
    const Real sgn = phase == 0 ? Real(1) : Real(a.sgn2);
    // Every load of the phase's panels goes to registers first (fixed trip counts, predicated), so
    // all are in flight at once; a loop that stored each value to shared memory before the next load
    // ran one round trip per element.
    Cplx va[QA], vb[QB];
#pragma unroll
    for (int q = 0; q < QA; ++q) {   // A panel: rows i0.., column-major source
      const int e = t + kTinyThreads * q, r = e % kTinyBM, c = e / kTinyBM;
      va[q].x = Real(0);
      va[q].y = Real(0);
      if (e < kTinyBM * L && i0 + r < a.M) va[q] = A[(long long)c * lda + i0 + r];
    }
#pragma unroll
    for (int q = 0; q < QB; ++q) {   // B panel: columns j0.., contiguous down a column
      const int e = t + kTinyThreads * q;
      const int c = L > 0 ? e % L : 0, jj = L > 0 ? e / L : 0;
      vb[q].x = Real(0);
      vb[q].y = Real(0);
      if (e < kTinyBN * L && j0 + jj < a.N) vb[q] = B[(long long)(j0 + jj) * ldb + c];
    }
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int e = t + kTinyThreads * q, r = e % kTinyBM, c = e / kTinyBM;
      if (e < kTinyBM * L) {
        Cplx v = va[q];
        if (real) v.y = Real(0);
        sA[phase][0][c][r] = v.x;
        sA[phase][1][c][r] = v.y;
        sA[phase][2][c][r] = v.x + v.y;
      }
    }
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int e = t + kTinyThreads * q;
      if (e < kTinyBN * L) {
        const int c = e % L, jj = e / L;
        Cplx v = vb[q];
        if (real) v.y = Real(0);
        v.x *= sgn;
        v.y *= sgn;
        sB[phase][0][c][jj] = v.x;
        sB[phase][1][c][jj] = v.y;
        sB[phase][2][c][jj] = v.x + v.y;
      }
    }
  }
  __syncthreads();
  const int lane = t % 32, w = t / 32, r = lane % kTinyBM, jj = lane / kTinyBM;
  constexpr int NW = kTinyThreads / 32;
  const int Lt = a.L1 + a.L2, q0 = (Lt * w) / NW, q1 = (Lt * (w + 1)) / NW;
  Real acc[3] = {Real(0), Real(0), Real(0)};
  for (int q = q0; q < q1; ++q) {
    const int phase = q < a.L1 ? 0 : 1, c = q < a.L1 ? q : q - a.L1;
    if (real) {
      acc[0] = fma(sA[phase][0][c][r], sB[phase][0][c][jj], acc[0]);
    } else {
#pragma unroll
      for (int z = 0; z < 3; ++z) acc[z] = fma(sA[phase][z][c][r], sB[phase][z][c][jj], acc[z]);
    }
  }
#pragma unroll
  for (int z = 0; z < 3; ++z) sP[w][z][lane] = acc[z];
  __syncthreads();
  if (w != 0) return;
#pragma unroll
  for (int z = 0; z < 3; ++z) {
    Real v = sP[0][z][lane];
#pragma unroll
    for (int u = 1; u < NW; ++u) v += sP[u][z][lane];
    acc[z] = v;
  }
  const int i = i0 + r, j = j0 + jj;
  if (i < a.M && j < a.N) {
    Cplx v;
    if (real) {
      v.x = acc[0];
      v.y = Real(0);
    } else {
      v.x = acc[0] - acc[1];
      v.y = acc[2] - acc[0] - acc[1];
    }
    a.Y[a.sY * k + (long long)j * a.ldy + i] = v;
  }
}

}  // namespace ts
