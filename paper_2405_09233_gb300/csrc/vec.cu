// Streaming kernels of the Arnoldi process (Algorithm 2) and of the solution update: inner
// products and norms (Definition 2.3), the modified Gram-Schmidt sweep, scaling and the
// (*) product of §3.1.  All are HBM-bound: grid-stride loops over packs of 4 elements (16- or
// 32-byte loads, two packs in flight per thread) when N is a multiple of 4 and the tensors are
// 16-byte aligned, scalar loops otherwise; a fixed grid of kRedBlocks blocks wherever a sum is
// formed; FP64 accumulation across packs whatever the storage type (an FP32 pack sums its own few
// products in FP32 first, see pack.cuh).
//
// Reductions never use atomics: each block writes one partial sum, and whoever needs the total
// (the next MGS pass, the Givens kernel) adds the kRedBlocks partials in a fixed order.  The
// results are therefore bitwise reproducible from run to run.  A short vector is reduced by fewer
// blocks (red_blocks: one per 2048 elements, at most kRedBlocks), whose first block zeroes the
// rest of the partial array, so consumers still add kRedBlocks entries: a small solve does not pay
// for 608 mostly idle blocks in each of its dozen reductions per step.
#include <initializer_list>
#include <type_traits>
#include <cstdint>
#include "internal.cuh"
#include "reduce.cuh"
#include "pack.cuh"

namespace ts {
namespace {

// Block 0 zeroes the partial sums that no block of this (shortened) grid writes.
__device__ __forceinline__ void zero_unused_partials(double* __restrict__ partials) {
  if (blockIdx.x == 0)
    for (int b = gridDim.x + threadIdx.x; b < kRedBlocks; b += blockDim.x) partials[b] = 0.0;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_dot(const T* __restrict__ x, const T* __restrict__ y,
                                                     long long N, double* __restrict__ partials) {
  zero_unused_partials(partials);
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride)
    acc += (double)x[e] * (double)y[e];
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Packed form of k_dot: N4 packs of 4.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_dot4(const T* __restrict__ x, const T* __restrict__ y,
                                                      long long N4, double* __restrict__ partials) {
  zero_unused_partials(partials);
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N4; e += 2 * stride) {
    const long long e1 = e + stride;
    T a0[4], b0[4], a1[4], b1[4];
    ld4(x, e, a0);
    ld4(y, e, b0);
    const bool two = e1 < N4;
    if (two) {
      ld4(x, e1, a1);
      ld4(y, e1, b1);
    }
    if constexpr (sizeof(T) == 4) {   // both packs summed in FP32, one FP64 add (pack.cuh)
      float f = pack_dot(a0, b0);
      if (two) f = pack_dot(a1, b1, f);
      acc += (double)f;
    } else {
      acc_pack(acc, a0, b0);
      if (two) acc_pack(acc, a1, b1);
    }
  }
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// One modified Gram-Schmidt step fused with the inner product the next step needs:
//   h = <V_i, W> (finalised from Pin);  W -= h V_i;  Pout = partials of <V_next, W> or <W, W>.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_mgs(T* __restrict__ W, const T* __restrict__ Vi,
                                                     const T* __restrict__ Vn, long long N,
                                                     const double* __restrict__ Pin, double* __restrict__ h_out,
                                                     double* __restrict__ Pout) {
  const double h = finalize_partials(Pin);
  if (blockIdx.x == 0 && threadIdx.x == 0) *h_out = h;
  zero_unused_partials(Pout);
  const T hT = (T)h;
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const T* __restrict__ other = Vn ? Vn : W;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride) {
    const T w = W[e] - hT * Vi[e];
    W[e] = w;
    acc += (double)(Vn ? other[e] : w) * (double)w;
  }
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) Pout[blockIdx.x] = tot;
}

// Packed form of k_mgs: N4 packs of 4.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_mgs4(T* __restrict__ W, const T* __restrict__ Vi,
                                                      const T* __restrict__ Vn, long long N4,
                                                      const double* __restrict__ Pin, double* __restrict__ h_out,
                                                      double* __restrict__ Pout) {
  const double h = finalize_partials(Pin);
  if (blockIdx.x == 0 && threadIdx.x == 0) *h_out = h;
  zero_unused_partials(Pout);
  const T hT = (T)h;
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N4; e += 2 * stride) {
    const long long e1 = e + stride;
    const bool two = e1 < N4;
    T w0[4], v0[4], o0[4], w1[4], v1[4], o1[4];
    ld4(W, e, w0);
    ld4(Vi, e, v0);
    if (Vn) ld4(Vn, e, o0);
    if (two) {
      ld4(W, e1, w1);
      ld4(Vi, e1, v1);
      if (Vn) ld4(Vn, e1, o1);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      w0[c] = w0[c] - hT * v0[c];
      if (!Vn) o0[c] = w0[c];
    }
    st4(W, e, w0);
    if (two) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        w1[c] = w1[c] - hT * v1[c];
        if (!Vn) o1[c] = w1[c];
      }
      st4(W, e1, w1);
    }
    if constexpr (sizeof(T) == 4) {   // both packs summed in FP32, one FP64 add (pack.cuh)
      float f = pack_dot(o0, w0);
      if (two) f = pack_dot(o1, w1, f);
      acc += (double)f;
    } else {
      acc_pack(acc, o0, w0);
      if (two) acc_pack(acc, o1, w1);
    }
  }
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) Pout[blockIdx.x] = tot;
}

template <typename T, typename U>
__global__ void k_scale(const T* __restrict__ x, U* __restrict__ y, long long N, const double* __restrict__ s) {
  const double sc = *s;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride)
    y[e] = (U)((double)x[e] * sc);
}

template <typename T, typename U>
__global__ void k_scale4(const T* __restrict__ x, U* __restrict__ y, long long N4, const double* __restrict__ s) {
  const double sc = *s;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const float scf = (float)sc;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N4; e += stride) {
    T a[4];
    U b[4];
    ld4(x, e, a);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if constexpr (sizeof(U) == 4) b[c] = (float)a[c] * scf;   // FP32 result: FP32 product
      else b[c] = (U)((double)a[c] * sc);
    }
    st4(y, e, b);
  }
}

// X += alpha * sum_{i<k} y_i V_i ; alpha = alpha_scale * (*alpha_dev if given).
template <typename T, typename U>
__global__ void k_multi_axpy(U* __restrict__ X, const T* __restrict__ V, long long ldv, long long N,
                             const double* __restrict__ y, int k, double alpha_scale,
                             const double* __restrict__ alpha_dev) {
  __shared__ double ys[256];
  const double alpha = alpha_scale * (alpha_dev ? *alpha_dev : 1.0);
  for (int i = threadIdx.x; i < k && i < 256; i += blockDim.x) ys[i] = y[i] * alpha;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc = fma(ys[i], (double)V[(long long)i * ldv + e], acc);
    X[e] = (U)((double)X[e] + acc);
  }
}

template <typename T, typename U>
__global__ void k_multi_axpy4(U* __restrict__ X, const T* __restrict__ V, long long ldv, long long N4,
                              const double* __restrict__ y, int k, double alpha_scale,
                              const double* __restrict__ alpha_dev) {
  // FP32 basis: the combination is formed in FP32 (coefficients rounded to FP32) and added to X
  // once, so no element costs a conversion or a DFMA per basis vector (pack.cuh); an FP64 basis
  // accumulates in FP64.
  using Acc = typename std::conditional<sizeof(T) == 4, float, double>::type;
  __shared__ Acc ys[256];
  const double alpha = alpha_scale * (alpha_dev ? *alpha_dev : 1.0);
  for (int i = threadIdx.x; i < k && i < 256; i += blockDim.x) ys[i] = (Acc)(y[i] * alpha);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N4; e += stride) {
    Acc acc[4] = {0, 0, 0, 0};
    for (int i = 0; i < k; ++i) {
      T v[4];
      ld4(V + (long long)i * ldv, e, v);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fma_t(ys[i], (Acc)v[c], acc[c]);
    }
    U x[4];
    ld4(X, e, x);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if constexpr (sizeof(U) == 4) x[c] = x[c] + (float)acc[c];
      else x[c] = (U)((double)x[c] + (double)acc[c]);
    }
    st4(X, e, x);
  }
}

__global__ void k_finalize_norm(const double* __restrict__ P, double* __restrict__ out) {
  const double s = finalize_partials(P);
  if (threadIdx.x == 0) {
    const double nv = sqrt(s);
    out[0] = nv;
    out[1] = nv > 0.0 ? 1.0 / nv : 0.0;
  }
}

template <typename T>
__global__ void k_sub3(const T* __restrict__ b, const T* __restrict__ c, T* __restrict__ a, long long N) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride) a[e] = b[e] - c[e];
}

template <typename T, typename U>
__global__ void k_convert(const T* __restrict__ x, U* __restrict__ y, long long N) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride) y[e] = (U)x[e];
}

// Packed kernels need N % 4 == 0 and 16-byte aligned tensors (then every basis vector V + i N is
// aligned too).
bool packable(long long N, std::initializer_list<const void*> ptrs) {
  if (N % 4 != 0) return false;
  for (const void* p : ptrs)
    if (p && (reinterpret_cast<uintptr_t>(p) & 15) != 0) return false;
  return true;
}

// Blocks of a reduction over N elements: one per 2048 (a thread takes two packs of 4 per pass).
int red_blocks(long long N) {
  const long long b = (N + 2047) / 2048;
  return (int)(b < 1 ? 1 : (b > kRedBlocks ? kRedBlocks : b));
}

int grid_for(long long N) {
  long long b = (N + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
void dot_partials(const T* x, const T* y, long long N, double* partials, cudaStream_t st) {
  if (packable(N, {x, y})) k_dot4<T><<<red_blocks(N), kRedThreads, 0, st>>>(x, y, N / 4, partials);
  else k_dot<T><<<red_blocks(N), kRedThreads, 0, st>>>(x, y, N, partials);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename T>
void mgs_pass(T* W, const T* Vi, const T* Vnext, long long N, const double* Pin, double* h_out, double* Pout,
              cudaStream_t st) {
  if (packable(N, {W, Vi, Vnext}))
    k_mgs4<T><<<red_blocks(N), kRedThreads, 0, st>>>(W, Vi, Vnext, N / 4, Pin, h_out, Pout);
  else
    k_mgs<T><<<red_blocks(N), kRedThreads, 0, st>>>(W, Vi, Vnext, N, Pin, h_out, Pout);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename T, typename U>
void scale_dev(const T* x, U* y, long long N, const double* scale, cudaStream_t st) {
  if (packable(N, {x, y})) k_scale4<T, U><<<grid_for(N / 4), 256, 0, st>>>(x, y, N / 4, scale);
  else k_scale<T, U><<<grid_for(N), 256, 0, st>>>(x, y, N, scale);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename T, typename U>
void multi_axpy(U* X, const T* V, long long ldv, long long N, const double* y, int k, double alpha_scale,
                const double* alpha_dev, cudaStream_t st) {
  TS_REQUIRE(k <= 256, "multi_axpy: at most 256 basis vectors");
  if (k <= 0) return;
  if (packable(N, {X, V}) && ldv % 4 == 0)
    k_multi_axpy4<T, U><<<grid_for(N / 4), 256, 0, st>>>(X, V, ldv / 4 * 4, N / 4, y, k, alpha_scale, alpha_dev);
  else
    k_multi_axpy<T, U><<<grid_for(N), 256, 0, st>>>(X, V, ldv, N, y, k, alpha_scale, alpha_dev);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void finalize_norm(const double* P, double* out, cudaStream_t st) {
  k_finalize_norm<<<1, 256, 0, st>>>(P, out);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename T>
void sub3(const T* b, const T* c, T* a, long long N, cudaStream_t st) {
  k_sub3<T><<<grid_for(N), 256, 0, st>>>(b, c, a, N);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename T, typename U>
void convert(const T* x, U* y, long long N, cudaStream_t st) {
  k_convert<T, U><<<grid_for(N), 256, 0, st>>>(x, y, N);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void fill_zero(void* p, size_t bytes, cudaStream_t st) { TS_CUDA(cudaMemsetAsync(p, 0, bytes, st)); }

template void dot_partials<double>(const double*, const double*, long long, double*, cudaStream_t);
template void dot_partials<float>(const float*, const float*, long long, double*, cudaStream_t);
template void mgs_pass<double>(double*, const double*, const double*, long long, const double*, double*, double*,
                               cudaStream_t);
template void mgs_pass<float>(float*, const float*, const float*, long long, const double*, double*, double*,
                              cudaStream_t);
template void scale_dev<double, double>(const double*, double*, long long, const double*, cudaStream_t);
template void scale_dev<double, float>(const double*, float*, long long, const double*, cudaStream_t);
template void scale_dev<float, float>(const float*, float*, long long, const double*, cudaStream_t);
template void multi_axpy<double, double>(double*, const double*, long long, long long, const double*, int, double,
                                         const double*, cudaStream_t);
template void multi_axpy<float, double>(double*, const float*, long long, long long, const double*, int, double,
                                        const double*, cudaStream_t);
template void multi_axpy<float, float>(float*, const float*, long long, long long, const double*, int, double,
                                       const double*, cudaStream_t);
template void sub3<double>(const double*, const double*, double*, long long, cudaStream_t);
template void convert<double, float>(const double*, float*, long long, cudaStream_t);
template void convert<float, double>(const float*, double*, long long, cudaStream_t);

}  // namespace ts
