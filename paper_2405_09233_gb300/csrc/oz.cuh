// Emulated FP64 slice products on the tensor cores (Ozaki scheme, gemm_oz.cu).
#pragma once
#include "internal.cuh"

namespace ts {

// BF16 digit planes of A_k and B_k for the emulated FP64 product, owned by a ts_op.
struct OzOperands {
  int S = 0;                       // digits per FP64 value
  int ldn = 0, lds = 0;            // padded row lengths (multiples of 64 elements)
  void* a_re = nullptr;            // [S][K][n][ldn]  row-major A_k digits
  void* a_im = nullptr;
  void* b_re = nullptr;            // [S][K][s][lds]  column-major B_k digits
  void* b_im = nullptr;
  void* b_nre = nullptr;           // digits of -Re B_k
  int* Eop = nullptr;              // [K] shared exponent of A_k and B_k
  unsigned long long* mx = nullptr;
  void release();
};

void oz_prepare(ts_op* op, int S, cudaStream_t st);
// Y = M(X) in FP64 through the emulated product (same contract as apply_f64).
void apply_f64_oz(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, int mode, const double* C,
                  double* partials, int S, cudaStream_t st);
// BF16 tensor FLOPs one emulated application executes (all kept digit pairs).
double oz_bf16_flops(int n, int s, int K, int nyq, int S);

}  // namespace ts
