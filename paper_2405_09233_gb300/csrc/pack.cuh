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

}  // namespace ts
