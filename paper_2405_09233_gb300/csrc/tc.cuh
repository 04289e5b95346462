// Tensor-core (tcgen05) operator for the mixed-precision inner solve (gemm_tc.cu).
#pragma once
#include <cuda.h>
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

// Tensor maps of one operator application (128-byte swizzle, box 128 bytes x rows).
struct TcMaps {
  CUtensorMap a_re, a_im;      // A_k planes          [K][n][ldn]
  CUtensorMap xc_re, xc_im;    // X_k column-major    [K][s][ldn]
  CUtensorMap xr_re, xr_im;    // X_k row-major       [K][n][lds]
  CUtensorMap b_re, b_im;      // B_k column-major    [K][s][lds]
  // split TF32 (PARTS = 3): the low parts v - tf32(v) of the same planes
  CUtensorMap a_re_lo, a_im_lo, xc_re_lo, xc_im_lo, xr_re_lo, xr_im_lo, b_re_lo, b_im_lo;
};

// Batched solver: one instance's output and sizes, and its planar X copies.
struct BTcInst {
  float2* Y;             // K slices of column-major n x s (the instance's part of the batch spectrum)
  int n, s, nyq;
};
struct BTcPlanes {
  const float2* Xh;      // K slices of column-major n x s FP32 spectra
  void* xc_re;           // [K][s][ldn]  column-major planes
  void* xc_im;
  void* xr_re;           // [K][n][lds]  row-major planes
  void* xr_im;
  void* xc_re_lo;        // split TF32 low parts (nullptr otherwise)
  void* xc_im_lo;
  void* xr_re_lo;
  void* xr_im_lo;
  int n, s, ldn, lds, nyq;
};
// Column tiles the batched kernel supports (chosen per batch by the autotuner).
constexpr int kBatchTcBNs[2] = {64, 128};
// A batched product schedule, as the autotuner stores it: the column tile bn, plus 1 for the
// persistent kernel (one CTA per SM walking the work list) instead of one CTA per work item.
inline int tc_batch_sched(int bn, bool persistent) { return bn + (persistent ? 1 : 0); }
inline int tc_batch_bn(int sched) { return sched & ~1; }
inline bool tc_batch_persistent(int sched) { return (sched & 1) != 0; }
// Bytes of one instance's planar X copies (all planes) for `precision`.
size_t tc_batch_plane_bytes(int n, int s, int K, int precision);
// Fill `pl` (plane pointers carved from `base`) and `maps` (column tile bn) for one instance of a batch.
void tc_batch_instance(ts_op* op, int precision, const float2* Xh, void* base, BTcPlanes* pl, TcMaps* maps, int bn);
// Load the batched kernels and set their attributes (before any capture that records them).
void tc_batch_preload(int precision);
// Planar copies (planes work list) then the products (tiles work list, schedule sched) of the
// active instances.
void tc_batch_products(int precision, int sched, const BTcPlanes* planes, const int4* pitems, int npitems,
                       const TcMaps* maps, const BTcInst* inst, const int* active, const int4* items, int nitems,
                       int* err, cudaStream_t st);

void tc_prepare(ts_op* op, int precision, cudaStream_t st);
// Yh (float2, K slices of column-major n x s) = A_k X_k - X_k B_k on the tensor cores, from the
// FP32 tensor X (n x s x p).
void tc_apply(ts_ctx* ctx, ts_op* op, int precision, const float* X, float2* Yh, cudaStream_t st);
double gemm_flops_tc(int n, int s, int K, int nyq);

}  // namespace ts
