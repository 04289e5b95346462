// Tensor-core (tcgen05) operator for the mixed-precision inner solve (gemm_tc.cu).
#pragma once
#include "internal.cuh"

namespace ts {

// Planar operand copies of A_k and B_k for the tensor cores (BF16 or TF32), owned by a ts_op.
struct TcOperands {
  int esz = 0;           // element size: 2 (BF16) or 4 (TF32 stored as FP32)
  int ldn = 0, lds = 0;  // padded row lengths (multiples of 64 elements)
  void* a_re = nullptr;  // [K][n][ldn]  row-major A_k
  void* a_im = nullptr;
  void* b_re = nullptr;  // [K][s][lds]  column-major B_k
  void* b_im = nullptr;
  bool split = false;       // split TF32: low parts v - tf32(v) below
  void* a_re_lo = nullptr;
  void* a_im_lo = nullptr;
  void* b_re_lo = nullptr;
  void* b_im_lo = nullptr;
  void release();
};

// Per-apply planar copies of X_k (workspace).
struct TcWork {
  void* xc_re = nullptr;  // [K][s][ldn]  column-major X_k
  void* xc_im = nullptr;
  void* xr_re = nullptr;  // [K][n][lds]  row-major X_k
  void* xr_im = nullptr;
  void* xc_re_lo = nullptr;  // split TF32 low parts (nullptr otherwise)
  void* xc_im_lo = nullptr;
  void* xr_re_lo = nullptr;
  void* xr_im_lo = nullptr;
};

void tc_prepare(ts_op* op, int precision, cudaStream_t st);
// Yh (float2, K slices of column-major n x s) = A_k X_k - X_k B_k on the tensor cores, from the
// FP32 tensor X (n x s x p).
void tc_apply(ts_ctx* ctx, ts_op* op, int precision, const float* X, float2* Yh, cudaStream_t st);
double gemm_flops_tc(int n, int s, int K, int nyq);

}  // namespace ts
