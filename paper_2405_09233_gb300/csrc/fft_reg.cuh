// Register-resident radix-2 FFT of a compile-time power-of-two length P <= 32, used for the DFT
// along mode 3 (one tube per thread).  The direct DFT costs P(P/2+1) complex multiply-adds per
// tube; this costs (P/2) log2 P butterflies, which moves the mode-3 transforms from instruction
// bound to HBM bound for the tube lengths of the workloads (p = 4 .. 32).
//
// Convention (MATLAB's fft): forward X_k = sum_t x_t e^{-2 pi i k t / P}; the inverse here is the
// unnormalised sum with e^{+2 pi i k t / P} (the caller applies 1/P).  Twiddle table: tc[r] =
// cos(2 pi r / P), ts[r] = sin(2 pi r / P), r < P, computed with sincospi.
#pragma once
#include <cuda_runtime.h>

namespace ts {

__host__ __device__ constexpr int ilog2c(int p) { return p <= 1 ? 0 : 1 + ilog2c(p / 2); }
__host__ __device__ constexpr int bitrevc(int x, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r = (r << 1) | ((x >> b) & 1);
  return r;
}

// One radix-2 stage of span LEN, then the next; LEN is a template argument so that every register
// index is a compile-time constant (a runtime stage loop leaves the arrays in local memory).
template <typename Real, int P, bool INVERSE, int LEN>
struct FftStages {
  static __device__ __forceinline__ void run(Real (&xr)[P], Real (&xi)[P], const Real* __restrict__ tc,
                                             const Real* __restrict__ ts) {
    constexpr int half = LEN / 2, stride = P / LEN;
#pragma unroll
    for (int start = 0; start < P; start += LEN) {
#pragma unroll
      for (int q = 0; q < half; ++q) {
        const int a = start + q, b = start + q + half;
        Real vr, vi;
        if (q == 0) {                       // twiddle 1
          vr = xr[b];
          vi = xi[b];
        } else if (4 * q == LEN) {          // twiddle -+i
          vr = INVERSE ? -xi[b] : xi[b];
          vi = INVERSE ? xr[b] : -xr[b];
        } else {
          const Real wr = tc[q * stride];
          const Real wi = INVERSE ? ts[q * stride] : -ts[q * stride];
          vr = xr[b] * wr - xi[b] * wi;
          vi = xr[b] * wi + xi[b] * wr;
        }
        xr[b] = xr[a] - vr;
        xi[b] = xi[a] - vi;
        xr[a] = xr[a] + vr;
        xi[a] = xi[a] + vi;
      }
    }
    FftStages<Real, P, INVERSE, 2 * LEN>::run(xr, xi, tc, ts);
  }
};
template <typename Real, int P, bool INVERSE>
struct FftStages<Real, P, INVERSE, 2 * P> {
  static __device__ __forceinline__ void run(Real (&)[P], Real (&)[P], const Real*, const Real*) {}
};

// In-place decimation-in-time FFT; the inputs must already sit in bit-reversed order.
template <typename Real, int P, bool INVERSE>
__device__ __forceinline__ void fft_bitrev_inplace(Real (&xr)[P], Real (&xi)[P], const Real* __restrict__ tc,
                                                   const Real* __restrict__ ts) {
  FftStages<Real, P, INVERSE, 2>::run(xr, xi, tc, ts);
}

// Forward transform of P real samples read by `load(t)`; writes the P/2+1 non-redundant outputs
// through `store(k, re, im)`.
template <typename Real, int P, typename Load, typename Store>
__device__ __forceinline__ void rfft_reg(Load load, Store store, const Real* tc, const Real* ts) {
  constexpr int LB = ilog2c(P);
  Real xr[P], xi[P];
#pragma unroll
  for (int t = 0; t < P; ++t) {
    xr[bitrevc(t, LB)] = load(t);
    xi[bitrevc(t, LB)] = Real(0);
  }
  fft_bitrev_inplace<Real, P, false>(xr, xi, tc, ts);
#pragma unroll
  for (int k = 0; k <= P / 2; ++k) store(k, xr[k], (k == 0 || k == P / 2) ? Real(0) : xi[k]);
}

// Inverse of a Hermitian half spectrum c_0..c_{P/2} read by `load(k, re, im)`: writes the P real
// samples times P (unnormalised) through `store(t, value)`.  Imaginary parts of c_0 and c_{P/2}
// are ignored (they are zero for the spectrum of a real tensor).
template <typename Real, int P, typename Load, typename Store>
__device__ __forceinline__ void irfft_reg(Load load, Store store, const Real* tc, const Real* ts) {
  constexpr int LB = ilog2c(P);
  Real xr[P], xi[P];
#pragma unroll
  for (int k = 0; k <= P / 2; ++k) {
    Real re, im;
    load(k, re, im);
    if (k == 0 || k == P / 2) im = Real(0);
    xr[bitrevc(k, LB)] = re;
    xi[bitrevc(k, LB)] = im;
    if (k > 0 && k < P / 2) {
      xr[bitrevc(P - k, LB)] = re;
      xi[bitrevc(P - k, LB)] = -im;
    }
  }
  fft_bitrev_inplace<Real, P, true>(xr, xi, tc, ts);
#pragma unroll
  for (int t = 0; t < P; ++t) store(t, xr[t]);
}

}  // namespace ts
