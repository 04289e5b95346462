// Register-resident radix-2 FFT of a compile-time power-of-two length P <= 32, used for the DFT
// along mode 3 (one tube per thread).  The direct DFT costs P(P/2+1) complex multiply-adds per
// tube; this costs (P/2) log2 P butterflies, which moves the mode-3 transforms from instruction
// bound to HBM bound for the tube lengths of the workloads (p = 4 .. 32).
//
// A real tube of length P >= 4 is transformed as one complex tube of length M = P/2 (even samples
// as real parts, odd samples as imaginary parts) plus one combining pass (the standard two-for-one
// real FFT), about 40% fewer arithmetic instructions than a complex length-P FFT with zero
// imaginary parts.  That matters for FP64 tubes, which GB300's FP64 rate makes instruction bound.
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
// TSTR: stride into the twiddle table (2 when a length-P/2 FFT uses the table of length P).
template <typename Real, int P, bool INVERSE, int LEN, int TSTR = 1>
struct FftStages {
  static __device__ __forceinline__ void run(Real (&xr)[P], Real (&xi)[P], const Real* __restrict__ tc,
                                             const Real* __restrict__ ts) {
    constexpr int half = LEN / 2, stride = TSTR * (P / LEN);
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
    FftStages<Real, P, INVERSE, 2 * LEN, TSTR>::run(xr, xi, tc, ts);
  }
};
template <typename Real, int P, bool INVERSE, int TSTR>
struct FftStages<Real, P, INVERSE, 2 * P, TSTR> {
  static __device__ __forceinline__ void run(Real (&)[P], Real (&)[P], const Real*, const Real*) {}
};

// In-place decimation-in-time FFT; the inputs must already sit in bit-reversed order.
template <typename Real, int P, bool INVERSE>
__device__ __forceinline__ void fft_bitrev_inplace(Real (&xr)[P], Real (&xi)[P], const Real* __restrict__ tc,
                                                   const Real* __restrict__ ts) {
  FftStages<Real, P, INVERSE, 2>::run(xr, xi, tc, ts);
}

// Forward transform of P real samples read by `load(t)`; writes the P/2+1 non-redundant outputs
// through `store(k, re, im)`.  Twiddle table of length P.
//
// Two-for-one (P >= 4): z_t = x_2t + i x_2t+1, Z = DFT_M(z).  With E_k, O_k the length-M DFTs of the
// even and odd samples, Z_k = E_k + i O_k and conj(Z_M-k) = E_k - i O_k, so
// E_k = (Z_k + conj Z_M-k)/2, O_k = (Z_k - conj Z_M-k)/(2i) and X_k = E_k + w^k O_k,
// X_M-k = conj(E_k) - conj(w^k O_k), w = e^{-2 pi i/P}; X_0 = Re Z_0 + Im Z_0, X_M = Re Z_0 - Im Z_0
// and X_M/2 = conj Z_M/2.
template <typename Real, int P, typename Load, typename Store>
__device__ __forceinline__ void rfft_reg(Load load, Store store, const Real* tc, const Real* ts) {
  if constexpr (P < 4) {
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
  } else {
    constexpr int M = P / 2, LB = ilog2c(M);
    Real zr[M], zi[M];
#pragma unroll
    for (int t = 0; t < M; ++t) {
      zr[bitrevc(t, LB)] = load(2 * t);
      zi[bitrevc(t, LB)] = load(2 * t + 1);
    }
    FftStages<Real, M, false, 2, 2>::run(zr, zi, tc, ts);
    store(0, zr[0] + zi[0], Real(0));
    store(M, zr[0] - zi[0], Real(0));
#pragma unroll
    for (int k = 1; 2 * k <= M; ++k) {
      if (2 * k == M) {
        store(k, zr[k], -zi[k]);
      } else {
        const Real s1 = zr[k] + zr[M - k], s2 = zi[k] - zi[M - k];
        const Real s3 = zi[k] + zi[M - k], s4 = zr[M - k] - zr[k];
        const Real hc = Real(0.5) * tc[k], hs = Real(0.5) * ts[k];
        const Real u = hc * s3 + hs * s4, v = hc * s4 - hs * s3;
        store(k, Real(0.5) * s1 + u, Real(0.5) * s2 + v);
        store(M - k, Real(0.5) * s1 - u, v - Real(0.5) * s2);
      }
    }
  }
}

// Inverse of a Hermitian half spectrum c_0..c_{P/2} read by `load(k, re, im)`: writes the P real
// samples times P (unnormalised) through `store(t, value)`.  Imaginary parts of c_0 and c_{P/2}
// are ignored (they are zero for the spectrum of a real tensor).
//
// Two-for-one (P >= 4), the forward steps reversed: Z'_k = (c_k + conj c_M-k) +
// i (c_k - conj c_M-k) w^-k (= 2 Z_k), and the unnormalised inverse DFT_M of Z' is P z, so
// x_2t = Re and x_2t+1 = Im of its entry t.
template <typename Real, int P, typename Load, typename Store>
__device__ __forceinline__ void irfft_reg(Load load, Store store, const Real* tc, const Real* ts) {
  if constexpr (P < 4) {
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
  } else {
    constexpr int M = P / 2, LB = ilog2c(M);
    Real zr[M], zi[M];
    {
      Real a, b, c, d;
      load(0, a, b);
      load(M, c, d);
      zr[0] = a + c;
      zi[0] = a - c;
    }
#pragma unroll
    for (int k = 1; 2 * k <= M; ++k) {
      Real a, b;
      load(k, a, b);
      if (2 * k == M) {
        zr[bitrevc(k, LB)] = Real(2) * a;
        zi[bitrevc(k, LB)] = Real(-2) * b;
      } else {
        Real c, d;
        load(M - k, c, d);
        const Real s1 = a + c, s2 = b - d, s3 = b + d, s4 = c - a;
        const Real co = tc[k], si = ts[k];
        const Real pp = -(s4 * co + s3 * si), qq = s3 * co - s4 * si;
        zr[bitrevc(k, LB)] = s1 - qq;
        zi[bitrevc(k, LB)] = s2 + pp;
        zr[bitrevc(M - k, LB)] = s1 + qq;
        zi[bitrevc(M - k, LB)] = pp - s2;
      }
    }
    FftStages<Real, M, true, 2, 2>::run(zr, zi, tc, ts);
#pragma unroll
    for (int t = 0; t < M; ++t) {
      store(2 * t, zr[t]);
      store(2 * t + 1, zi[t]);
    }
  }
}

}  // namespace ts
