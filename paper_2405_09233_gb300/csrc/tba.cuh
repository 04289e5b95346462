// Tubal Block Arnoldi / TBAS and t-Bartels-Stewart (tba.cu, small_complex.cu).
#pragma once
#include "internal.cuh"

namespace ts {

// Sparse operator: the union of the CSR patterns of A^(1..p), with the Fourier slices of the
// values on that pattern.
struct SparseOp {
  int nnz = 0;
  int* rowptr = nullptr;     // n + 1
  int* col = nullptr;        // nnz
  double2* vals = nullptr;   // K x nnz (slice k at vals + k*nnz)
  float2* vals32 = nullptr;  // FP32 copy for the inner cycle of mixed-precision TBAS, made on first use
  void release();
};

// Small complex kernels (small_complex.cu).  Matrices are column-major, one per slice.
void schur_small(double2* T, double2* Q, int s, int count, int* err, cudaStream_t st);
void shifted_lu(const double2* H, long long sH, const double2* T, double2* LU, int* piv, int N, int bw, int s, int K,
                int* err, cudaStream_t st);
void hs_solve(const double2* LU, const int* piv, const double2* G, const double2* T, double2* Z, int N, int bw, int s,
              int K, cudaStream_t st);
void small_gemm(const double2* A, long long sA, int lda, const double2* B, long long sB, int ldb, bool transB, double2* C,
                long long sC, int ldc, int M, int L, int Ncol, int K, bool accumulate, cudaStream_t st);
// Per-slice Cholesky G = R^H R with the pivot test of k_cholesky (rel, tiny2; 0, 0 for d > 0 only).
void cholesky_small(const double2* G, double2* R, int s, int K, double rel, double tiny2, int* err, int* fail_slice,
                    cudaStream_t st);

// Schur factors of the operator's B_k (computed on first use and cached in the operator).
void ensure_b_schur(ts_ctx* ctx, ts_op* op, cudaStream_t st);

}  // namespace ts
