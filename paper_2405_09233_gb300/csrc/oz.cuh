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

// Per-application digit planes of X_k (caller-owned, sized by oz_buffer_sizes).
struct OzBuffers {
  void* xc_re = nullptr;           // [S][K][s][ldn]  column-major X_k digits
  void* xc_im = nullptr;
  void* xc_nim = nullptr;          //   digits of -Im X_k
  void* xr_re = nullptr;           // [S][K][n][lds]  row-major X_k digits
  void* xr_im = nullptr;
  unsigned long long* mx = nullptr;   // [K] slice maxima (FP64 bit patterns)
  int* Ex = nullptr;                  // [K] slice exponents
};
struct OzBufferSizes {
  size_t xc = 0, xr = 0;           // bytes of each xc_* / xr_* plane set
  int K = 0;                       // entries of mx and Ex
};
OzBufferSizes oz_buffer_sizes(int n, int s, int K, int S);

void oz_prepare(ts_op* op, int S, cudaStream_t st);
// Loads the kernels and sets their attributes (call before any stream capture that records them).
void oz_preload();
// Yh_k = A_k Xh_k - Xh_k B_k for the K spectral slices of op (double2, column-major n x s each),
// emulated FP64 with S digits per value; op must be prepared with at least S digits (the leading S
// digits of a longer expansion approximate an entry as closely as an S-digit expansion, within
// 0.502 of the last kept digit's unit).  gate (device, may be null): when *gate == 0
// every kernel returns at once.  Captures into a CUDA graph (no allocation, no synchronisation).
void oz_products(const ts_op* op, const double2* Xh, double2* Yh, int S, const OzBuffers& b, const int* gate,
                 int* err, cudaStream_t st);
// Y = M(X) in FP64 through the emulated product (same contract as apply_f64), with S digits per
// value; the operator's digit planes are prepared (once) with S_op >= S digits.
void apply_f64_oz(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, int mode, const double* C,
                  double* partials, int S, int S_op, cudaStream_t st);
// The emulated products alone on spectral tensors (the spectral Krylov basis): Yh = A_k Xh_k - Xh_k B_k.
void oz_apply_spectral(ts_ctx* ctx, const ts_op* op, const double2* Xh, double2* Yh, int S, int S_op,
                       cudaStream_t st);
// BF16 tensor FLOPs one emulated application executes (all kept digit pairs).
double oz_bf16_flops(int n, int s, int K, int nyq, int S);

}  // namespace ts
