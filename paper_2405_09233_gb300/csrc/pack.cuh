// Packs of 4 consecutive elements moved as one float4 or two double2 accesses (16-byte aligned).
#pragma once
#include <cuda_runtime.h>

namespace ts {

// 4 consecutive elements as one or two 16-byte accesses.
__device__ __forceinline__ void ld4(const float* p, long long e, float (&v)[4]) {
  const float4 q = reinterpret_cast<const float4*>(p)[e];
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, long long e, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[2 * e], b = reinterpret_cast<const double2*>(p)[2 * e + 1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, long long e, const float (&v)[4]) {
  reinterpret_cast<float4*>(p)[e] = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, long long e, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[2 * e] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[2 * e + 1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Dot products of packs.  An FP64 pack accumulates in FP64 term by term.  An FP32 pack sums its
// products in FP32 (pack_dot) and the caller adds that sum to its FP64 accumulator once: GB300
// executes FP64 arithmetic, and conversions between FP32 and FP64, at a small fraction of its FP32
// rate, so a conversion and a DFMA per element left the FP32 streaming kernels bound by the FP64
// pipe instead of by HBM.  The FP32 partial adds at most ~4u32 of the pack's absolute products,
// the size of the rounding its FP32 operands already carry.
__device__ __forceinline__ float pack_dot(const float (&a)[4], const float (&b)[4], float f = 0.f) {
#pragma unroll
  for (int c = 0; c < 4; ++c) f = fmaf(a[c], b[c], f);
  return f;
}
__device__ __forceinline__ void acc_pack(double& acc, const float (&a)[4], const float (&b)[4]) {
  acc += (double)pack_dot(a, b);
}
__device__ __forceinline__ void acc_pack(double& acc, const double (&a)[4], const double (&b)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) acc += a[c] * b[c];
}

}  // namespace ts
