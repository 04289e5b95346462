// DFT along mode 3 of column-major tensors (§2: fft(X, [], 3) and ifft), keeping only the
// floor(p/2)+1 non-redundant Fourier slices of a real tensor (Algorithm 1, with the Nyquist
// slice computed rather than mirrored).
//
// Every frontal slice is a contiguous block of T = n1*n2 entries, so the tube (i, j, :) is the
// strided sequence in[e], in[e + T], ..., in[e + (p-1)T] with e = i + n1*j.  One thread owns one
// tube: a warp reads 32 consecutive e for each t (coalesced), keeps the p samples in registers
// and evaluates the DFT directly from a twiddle table in shared memory (sincospi of 2r/p, so the
// k = 0 and Nyquist twiddles are exactly +-1 and 0 and those slices come out exactly real).
#include "internal.cuh"
#include "reduce.cuh"
#include "fft_reg.cuh"

namespace ts {
namespace {

template <typename Real> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };

template <typename Real>
__device__ __forceinline__ void load_twiddles(Real* c, Real* s, int p) {
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    double sv, cv;
    sincospi(2.0 * r / p, &sv, &cv);
    c[r] = (Real)cv;
    s[r] = (Real)sv;
  }
  __syncthreads();
}

template <typename Real, typename Cplx, int PMAX>
__global__ void __launch_bounds__(256) k_rfft(const Real* __restrict__ in, Cplx* __restrict__ out,
                                              long long T, int p, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;   // a cycle that already ended (launched ahead)
  __shared__ Real tc[PMAX], tsn[PMAX];
  load_twiddles(tc, tsn, p);
  const int K = p / 2 + 1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T;
       e += (long long)gridDim.x * blockDim.x) {
    Real x[PMAX];
#pragma unroll
    for (int t = 0; t < PMAX; ++t) x[t] = (t < p) ? in[t * T + e] : Real(0);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      {
        Real re = 0, im = 0;
        int r = 0;
#pragma unroll
        for (int t = 0; t < PMAX; ++t) {
          if (t < p) {
            re = fma(x[t], tc[r], re);
            im = fma(-x[t], tsn[r], im);
            r += k;
            if (r >= p) r -= p;
          }
        }
        Cplx v;
        v.x = re;
        v.y = im;
        out[k * T + e] = v;
      }
    }
  }
}

// Power-of-two p: register radix-2 FFT (fft_reg.cuh), P compile-time.
template <typename Real, typename Cplx, int P>
__global__ void __launch_bounds__(256) k_rfft_pow2(const Real* __restrict__ in, Cplx* __restrict__ out, long long T,
                                                   const int* __restrict__ gate) {
  if (gate && *gate == 0) return;   // a cycle that already ended (launched ahead)
  __shared__ Real tc[P], tsn[P];
  load_twiddles(tc, tsn, P);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T;
       e += (long long)gridDim.x * blockDim.x) {
    rfft_reg<Real, P>([&](int t) { return in[t * T + e]; },
                      [&](int k, Real re, Real im) {
                        Cplx v;
                        v.x = re;
                        v.y = im;
                        out[k * T + e] = v;
                      },
                      tc, tsn);
  }
}

template <typename Real, typename Cplx, int P, int MODE>
__global__ void __launch_bounds__(256) k_irfft_pow2(const Cplx* __restrict__ in, Real* __restrict__ out, long long T,
                                                    const Real* __restrict__ C, double* __restrict__ partials,
                                                    const int* __restrict__ gate) {
  if (gate && *gate == 0) return;   // a cycle that already ended (launched ahead)
  __shared__ Real tc[P], tsn[P];
  load_twiddles(tc, tsn, P);
  const Real invp = Real(1) / Real(P);
  double local = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T;
       e += (long long)gridDim.x * blockDim.x) {
    irfft_reg<Real, P>(
        [&](int k, Real& re, Real& im) {
          const Cplx c = in[k * T + e];
          re = c.x;
          im = c.y;
        },
        [&](int t, Real v) {
          v *= invp;
          if (MODE == IRFFT_RESIDUAL) {
            v = C[t * T + e] - v;
            local += (double)v * (double)v;
          }
          out[t * T + e] = v;
        },
        tc, tsn);
  }
  if (MODE == IRFFT_RESIDUAL) {
    const double tot = block_sum(local);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  }
}

// Any p: samples re-read from memory for every k (L1/L2 hits after the first).
template <typename Real, typename Cplx>
__global__ void __launch_bounds__(256) k_rfft_any(const Real* __restrict__ in, Cplx* __restrict__ out,
                                                  long long T, int p, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;   // a cycle that already ended (launched ahead)
  extern __shared__ unsigned char smem_raw[];
  Real* tc = reinterpret_cast<Real*>(smem_raw);
  Real* tsn = tc + p;
  load_twiddles(tc, tsn, p);
  const int K = p / 2 + 1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T;
       e += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < K; ++k) {
      Real re = 0, im = 0;
      int r = 0;
      for (int t = 0; t < p; ++t) {
        const Real xv = in[t * T + e];
        re = fma(xv, tc[r], re);
        im = fma(-xv, tsn[r], im);
        r += k;
        if (r >= p) r -= p;
      }
      Cplx v;
      v.x = re;
      v.y = im;
      out[k * T + e] = v;
    }
  }
}

// Inverse: y_t = (1/p) [Re c_0 + (-1)^t Re c_{p/2} (p even) + 2 sum_{0<k<p/2} Re(c_k e^{+2 pi i k t/p})].
template <typename Real, typename Cplx, int PMAX, int MODE>
__global__ void __launch_bounds__(256) k_irfft(const Cplx* __restrict__ in, Real* __restrict__ out,
                                               long long T, int p, const Real* __restrict__ C,
                                               double* __restrict__ partials, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;   // a cycle that already ended (launched ahead)
  __shared__ Real tc[PMAX], tsn[PMAX];
  load_twiddles(tc, tsn, p);
  const int K = p / 2 + 1;
  const int nyq = (p % 2 == 0 && p > 1) ? p / 2 : -1;
  const Real invp = Real(1) / Real(p);
  double local = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T;
       e += (long long)gridDim.x * blockDim.x) {
    Real y[PMAX];
#pragma unroll
    for (int t = 0; t < PMAX; ++t) y[t] = 0;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      {
        const Cplx c = in[k * T + e];
        const Real w = (k == 0 || k == nyq) ? Real(1) : Real(2);
        const Real cr = w * c.x, ci = w * c.y;
        int r = 0;
#pragma unroll
        for (int t = 0; t < PMAX; ++t) {
          if (t < p) {
            if (k == 0 || k == nyq) {
              y[t] = fma(cr, tc[r], y[t]);     // real slices: imaginary part is zero by symmetry
            } else {
              y[t] = fma(cr, tc[r], y[t]);
              y[t] = fma(-ci, tsn[r], y[t]);
            }
            r += k;
            if (r >= p) r -= p;
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < PMAX; ++t) {
      if (t < p) {
        Real v = y[t] * invp;
        if (MODE == IRFFT_RESIDUAL) {
          v = C[t * T + e] - v;
          local += (double)v * (double)v;
        }
        out[t * T + e] = v;
      }
    }
  }
  if (MODE == IRFFT_RESIDUAL) {
    const double tot = block_sum(local);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  }
}

template <typename Real, typename Cplx, int MODE>
__global__ void __launch_bounds__(256) k_irfft_any(const Cplx* __restrict__ in, Real* __restrict__ out,
                                                   long long T, int p, const Real* __restrict__ C,
                                                   double* __restrict__ partials, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;   // a cycle that already ended (launched ahead)
  extern __shared__ unsigned char smem_raw[];
  Real* tc = reinterpret_cast<Real*>(smem_raw);
  Real* tsn = tc + p;
  load_twiddles(tc, tsn, p);
  const int K = p / 2 + 1;
  const int nyq = (p % 2 == 0 && p > 1) ? p / 2 : -1;
  const Real invp = Real(1) / Real(p);
  double local = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T;
       e += (long long)gridDim.x * blockDim.x) {
    for (int t = 0; t < p; ++t) {
      Real y = 0;
      for (int k = 0; k < K; ++k) {
        const Cplx c = in[k * T + e];
        const int r = (int)(((long long)k * t) % p);
        if (k == 0 || k == nyq) {
          y = fma(c.x, tc[r], y);
        } else {
          y = fma(Real(2) * c.x, tc[r], y);
          y = fma(-Real(2) * c.y, tsn[r], y);
        }
      }
      Real v = y * invp;
      if (MODE == IRFFT_RESIDUAL) {
        v = C[t * T + e] - v;
        local += (double)v * (double)v;
      }
      out[t * T + e] = v;
    }
  }
  if (MODE == IRFFT_RESIDUAL) {
    const double tot = block_sum(local);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  }
}

int stream_grid(long long T) {
  long long b = (T + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename Real, typename Cplx>
void rfft_tube(const Real* in, Cplx* out, long long T, int p, cudaStream_t st, const int* gate) {
  const int g = stream_grid(T);
  if (p == 2) k_rfft_pow2<Real, Cplx, 2><<<g, 256, 0, st>>>(in, out, T, gate);
  else if (p == 4) k_rfft_pow2<Real, Cplx, 4><<<g, 256, 0, st>>>(in, out, T, gate);
  else if (p == 8) k_rfft_pow2<Real, Cplx, 8><<<g, 256, 0, st>>>(in, out, T, gate);
  else if (p == 16) k_rfft_pow2<Real, Cplx, 16><<<g, 256, 0, st>>>(in, out, T, gate);
  else if (p == 32) k_rfft_pow2<Real, Cplx, 32><<<g, 256, 0, st>>>(in, out, T, gate);
  else if (p <= 2) k_rfft<Real, Cplx, 2><<<g, 256, 0, st>>>(in, out, T, p, gate);
  else if (p <= 4) k_rfft<Real, Cplx, 4><<<g, 256, 0, st>>>(in, out, T, p, gate);
  else if (p <= 8) k_rfft<Real, Cplx, 8><<<g, 256, 0, st>>>(in, out, T, p, gate);
  else if (p <= 16) k_rfft<Real, Cplx, 16><<<g, 256, 0, st>>>(in, out, T, p, gate);
  else if (p <= 32) k_rfft<Real, Cplx, 32><<<g, 256, 0, st>>>(in, out, T, p, gate);
  else k_rfft_any<Real, Cplx><<<g, 256, 2 * p * sizeof(Real), st>>>(in, out, T, p, gate);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename Real, typename Cplx>
void irfft_tube(const Cplx* in, Real* out, long long T, int p, int mode, const Real* C,
                double* partials, cudaStream_t st, const int* gate) {
  // The residual epilogue writes one partial per block: it runs on exactly kRedBlocks blocks.
  const int g = mode == IRFFT_RESIDUAL ? kRedBlocks : stream_grid(T);
#define TS_IRFFT(PM)                                                                            \
  do {                                                                                          \
    if (mode == IRFFT_RESIDUAL)                                                                 \
      k_irfft<Real, Cplx, PM, IRFFT_RESIDUAL><<<g, 256, 0, st>>>(in, out, T, p, C, partials, gate);   \
    else                                                                                        \
      k_irfft<Real, Cplx, PM, IRFFT_STORE><<<g, 256, 0, st>>>(in, out, T, p, C, partials, gate);      \
  } while (0)
#define TS_IRFFT_POW2(PP)                                                                        \
  do {                                                                                           \
    if (mode == IRFFT_RESIDUAL)                                                                  \
      k_irfft_pow2<Real, Cplx, PP, IRFFT_RESIDUAL><<<g, 256, 0, st>>>(in, out, T, C, partials, gate);  \
    else                                                                                         \
      k_irfft_pow2<Real, Cplx, PP, IRFFT_STORE><<<g, 256, 0, st>>>(in, out, T, C, partials, gate);     \
  } while (0)
  if (p == 2) TS_IRFFT_POW2(2);
  else if (p == 4) TS_IRFFT_POW2(4);
  else if (p == 8) TS_IRFFT_POW2(8);
  else if (p == 16) TS_IRFFT_POW2(16);
  else if (p == 32) TS_IRFFT_POW2(32);
  else if (p <= 2) TS_IRFFT(2);
  else if (p <= 4) TS_IRFFT(4);
  else if (p <= 8) TS_IRFFT(8);
  else if (p <= 16) TS_IRFFT(16);
  else if (p <= 32) TS_IRFFT(32);
  else if (mode == IRFFT_RESIDUAL)
    k_irfft_any<Real, Cplx, IRFFT_RESIDUAL><<<g, 256, 2 * p * sizeof(Real), st>>>(in, out, T, p, C, partials, gate);
  else
    k_irfft_any<Real, Cplx, IRFFT_STORE><<<g, 256, 2 * p * sizeof(Real), st>>>(in, out, T, p, C, partials, gate);
#undef TS_IRFFT
#undef TS_IRFFT_POW2
  count_launch();
  TS_CUDA(cudaGetLastError());
}

namespace {
// Scaled half spectrum of the spectral Krylov basis: out_k = in_k * sqrt(w_k / p) (or its inverse),
// times *alpha when given; the imaginary parts of the real slices (k = 0 and p/2) are set to zero.
__global__ void k_spec_weight(const double2* in, double2* out, long long T, int p,
                              int inverse, const double* __restrict__ alpha) {
  const int K = p / 2 + 1;
  const double a = alpha ? *alpha : 1.0;
  const long long tot = (long long)K * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / T);
    const bool real = k == 0 || (p % 2 == 0 && k == p / 2);
    const double w = real ? 1.0 : 2.0;
    const double f = a * (inverse ? sqrt(p / w) : sqrt(w / p));
    const double2 v = in[e];
    out[e] = make_double2(v.x * f, real ? 0.0 : v.y * f);
  }
}
}  // namespace

void spec_weight(const double2* in, double2* out, long long T, int p, bool inverse, const double* alpha,
                 cudaStream_t st) {
  k_spec_weight<<<stream_grid((long long)(p / 2 + 1) * T), 256, 0, st>>>(in, out, T, p, inverse ? 1 : 0, alpha);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template void rfft_tube<double, double2>(const double*, double2*, long long, int, cudaStream_t, const int*);
template void rfft_tube<float, float2>(const float*, float2*, long long, int, cudaStream_t, const int*);
template void irfft_tube<double, double2>(const double2*, double*, long long, int, int, const double*, double*,
                                          cudaStream_t, const int*);
template void irfft_tube<float, float2>(const float2*, float*, long long, int, int, const float*, double*,
                                        cudaStream_t, const int*);

}  // namespace ts
