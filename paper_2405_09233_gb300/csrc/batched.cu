// Batched restarted tGMRES: many independent Sylvester tensor equations of uneven (n, s, p) solved
// together on one GPU, FP64 or mixed precision (FP32 Arnoldi cycle, FP64 residual and update).
//
// All instances advance in lockstep through the restart cycle of Algorithm 3; every phase is ONE
// launch over all instances:
//   * streaming phases (scaling, inner products, MGS passes, X += V (*) y) run over a block table
//     in which every block belongs to one instance (a chunk of its N = n s p unknowns), so each
//     instance's inner product is the fixed-order sum of its own blocks' partials;
//   * the mode-3 DFTs run over a tube-block table (one tube per thread, the instance's p);
//   * the per-slice products run over a work list of (instance, Fourier slice, 64 x 64 tile)
//     items, ordered by cost (largest first) so the tail of the launch stays short;
//   * the Givens update is one block per instance.
// Masks on the device (cycle participation, still iterating) let an instance stop its inner cycle
// early or drop out of the batch without changing the launch sequence, so one restart cycle is
// captured once as a CUDA graph and replayed; the host only reads the per-instance residuals at
// the end of each cycle.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>
#include <type_traits>
#include <string>
#include "internal.cuh"
#include "oz.cuh"
#include "tc.cuh"
#include "tune.cuh"
#include "apply.cuh"
#include "reduce.cuh"
#include "pack.cuh"
#include "fft_reg.cuh"
#include "gemm_tile.cuh"
#include "cycle_graph.cuh"

namespace ts {

void ensure_f32_operator(ts_op* op, cudaStream_t st);  // lowprec.cu

namespace {

constexpr int kChunk = 4096;      // unknowns per streaming block (256 threads x 16)
constexpr int kTubes = 256;       // tubes per DFT block (one per thread)

struct BInst {
  double* X;
  const double* C;
  const double2* Ah;
  const double2* Bh;
  const float2* Ah32;
  const float2* Bh32;
  long long offN, offS;   // offsets in the concatenated unknown / spectral buffers
  long long N, T;         // n s p and n s
  int n, s, p, K, nyq;
  int nb0, nb1;           // streaming-block range
  int tb0, tb1;           // tube-block range
  double tol;
};

// Per-instance scalars (16 doubles each).
enum { SC_NORMC = 0, SC_RES = 1, SC_INVRES = 2, SC_EST = 3, SC_INVH = 4, SC_H = 5, SC_K = 6, SC_FLAGS = 7,
       SC_ITERS = 8, SC_DONE = 9 };

struct BDev {
  const BInst* inst;
  int count, m;
  long long totN, totS;
  const int* nb_inst;
  const long long* nb_off;
  const int* tb_inst;
  const long long* tb_off;
  const int* cyc;   // participates in the current cycle
  int* act;         // still iterating in the current cycle
  double* sc;
  double* state;
  long long stride;
  double inner_tol;
  int mixed;
};

// Per-instance Krylov state: H and its rotated copy R ((m+1) x m each), the rotations cs, sn (m),
// the rotated right-hand side g (m+1) and the solution y (m).
struct StLayout {
  int m;
  __host__ __device__ long long H() const { return 0; }
  __host__ __device__ long long R() const { return (long long)(m + 1) * m; }
  __host__ __device__ long long cs() const { return 2ll * (m + 1) * m; }
  __host__ __device__ long long sn() const { return cs() + m; }
  __host__ __device__ long long g() const { return sn() + m; }
  __host__ __device__ long long y() const { return g() + m + 1; }
  __host__ __device__ long long end() const { return y() + m; }
};
long long state_stride(int m) { return StLayout{m}.end(); }

// Sum of an instance's block partials [b0, b1), identical in every block that calls it.
__device__ __forceinline__ double inst_sum(const double* P, int b0, int b1) {
  double v = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) v += P[b];
  return block_sum(v);
}

template <typename T>
__host__ __device__ __forceinline__ T* basis(T* V, long long totN, int j) {
  return V + (long long)j * totN;
}

// --- streaming phases ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_b_scale_R(BDev d, const double* __restrict__ R, T* __restrict__ V0) {
  const int i = d.nb_inst[blockIdx.x];
  if (!d.cyc[i]) return;
  const BInst& in = d.inst[i];
  const double sc = d.sc[16 * i + SC_INVRES];
  const long long e0 = in.offN + d.nb_off[blockIdx.x];
  const long long e1 = min(in.offN + in.N, e0 + kChunk);
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) V0[e] = (T)(R[e] * sc);
}

// Instance offsets are multiples of 4 and chunks are kChunk long, so a block's range starts
// 16-byte aligned: the streaming kernels below move packs of 4 and finish a ragged instance tail
// element by element.
template <typename T>
__global__ void __launch_bounds__(256) k_b_dot(BDev d, const T* __restrict__ x, const T* __restrict__ y,
                                               double* __restrict__ P) {
  const int i = d.nb_inst[blockIdx.x];
  if (!d.act[i]) return;
  const BInst& in = d.inst[i];
  const long long e0 = in.offN + d.nb_off[blockIdx.x];
  const long long e1 = min(in.offN + in.N, e0 + kChunk);
  const long long n4 = (e1 - e0) / 4, p0 = e0 / 4;
  double acc = 0.0;
#pragma unroll 4
  for (long long q = threadIdx.x; q < n4; q += blockDim.x) {
    T a[4], c[4];
    ld4(x, p0 + q, a);
    ld4(y, p0 + q, c);
    acc_pack(acc, a, c);   // an FP32 pack is summed in FP32 first (pack.cuh)
  }
  for (long long e = e0 + 4 * n4 + threadIdx.x; e < e1; e += blockDim.x) acc += (double)x[e] * (double)y[e];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) P[blockIdx.x] = t;
}

// ||C_i||^2 partials (C read through the instance pointer).
__global__ void __launch_bounds__(256) k_b_normC(BDev d, double* __restrict__ P) {
  const int i = d.nb_inst[blockIdx.x];
  const BInst& in = d.inst[i];
  const long long l0 = d.nb_off[blockIdx.x];
  const long long l1 = min(in.N, l0 + kChunk);
  double acc = 0.0;
  for (long long e = l0 + threadIdx.x; e < l1; e += blockDim.x) acc += in.C[e] * in.C[e];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) P[blockIdx.x] = t;
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_mgs(BDev d, T* __restrict__ W, const T* __restrict__ Vi,
                                               const T* __restrict__ Vn, const double* __restrict__ Pin,
                                               double* __restrict__ Pout, int irow, int jcol) {
  const int i = d.nb_inst[blockIdx.x];
  if (!d.act[i]) return;
  const BInst& in = d.inst[i];
  const double h = inst_sum(Pin, in.nb0, in.nb1);
  if (blockIdx.x == in.nb0 && threadIdx.x == 0) {
    StLayout L{d.m};
    d.state[i * d.stride + L.H() + irow + (long long)(d.m + 1) * jcol] = h;
  }
  const T hT = (T)h;
  const long long e0 = in.offN + d.nb_off[blockIdx.x];
  const long long e1 = min(in.offN + in.N, e0 + kChunk);
  const long long n4 = (e1 - e0) / 4, p0 = e0 / 4;
  double acc = 0.0;
#pragma unroll 4
  for (long long q = threadIdx.x; q < n4; q += blockDim.x) {
    T w[4], v[4], o[4];
    ld4(W, p0 + q, w);
    ld4(Vi, p0 + q, v);
    if (Vn) ld4(Vn, p0 + q, o);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      w[t] = w[t] - hT * v[t];
      if (!Vn) o[t] = w[t];
    }
    st4(W, p0 + q, w);
    acc_pack(acc, o, w);
  }
  for (long long e = e0 + 4 * n4 + threadIdx.x; e < e1; e += blockDim.x) {
    const T w = W[e] - hT * Vi[e];
    W[e] = w;
    acc += (double)(Vn ? Vn[e] : w) * (double)w;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) Pout[blockIdx.x] = t;
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_scale_W(BDev d, const T* __restrict__ W, T* __restrict__ Vn) {
  const int i = d.nb_inst[blockIdx.x];
  if (!d.act[i]) return;
  const BInst& in = d.inst[i];
  const T sc = (T)d.sc[16 * i + SC_INVH];
  const long long e0 = in.offN + d.nb_off[blockIdx.x];
  const long long e1 = min(in.offN + in.N, e0 + kChunk);
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) Vn[e] = W[e] * sc;
}

// X_i += sum_{q < k_i} y_q V_q  (X through the instance pointer, FP64).
template <typename T>
__global__ void __launch_bounds__(256) k_b_axpy(BDev d, const T* __restrict__ V) {
  const int i = d.nb_inst[blockIdx.x];
  if (!d.cyc[i]) return;
  const BInst& in = d.inst[i];
  // an FP32 basis is combined in FP32 and added to X once (no per-term conversion, pack.cuh)
  __shared__ T ys[256];
  StLayout L{d.m};
  const int k = (int)d.sc[16 * i + SC_K];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = (T)d.state[i * d.stride + L.y() + q];
  __syncthreads();
  const long long l0 = d.nb_off[blockIdx.x];
  const long long l1 = min(in.N, l0 + kChunk);
  for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
    T acc = 0;
    for (int q = 0; q < k; ++q) acc = fma_t(ys[q], V[(long long)q * d.totN + in.offN + l], acc);
    in.X[l] += (double)acc;
  }
}

// --- DFT along mode 3 over the tube-block table ----------------------------------------------------
// SRC 0: concatenated buffer `in` (offN); SRC 1: instance X (FP64).  MASK 0: act, 1: cyc.
template <typename Real, typename Cplx, int SRC, int MASK>
__global__ void __launch_bounds__(kTubes) k_b_rfft(BDev d, const Real* __restrict__ in, Cplx* __restrict__ out) {
  const int i = d.tb_inst[blockIdx.x];
  if (!(MASK ? d.cyc[i] : d.act[i])) return;
  const BInst& ins = d.inst[i];
  const int p = ins.p;
  __shared__ Real tc[64], tsn[64];
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    double sv, cv;
    sincospi(2.0 * r / p, &sv, &cv);
    tc[r] = (Real)cv;
    tsn[r] = (Real)sv;
  }
  __syncthreads();
  const long long e = d.tb_off[blockIdx.x] + threadIdx.x;
  if (e >= ins.T) return;
  const Real* src = SRC == 0 ? in + ins.offN : reinterpret_cast<const Real*>(ins.X);
  Cplx* dst = out + ins.offS;
  const long long T = ins.T;
  auto ld = [&](int t) { return src[t * T + e]; };
  auto stv = [&](int k, Real re, Real im) {
    Cplx v;
    v.x = re;
    v.y = im;
    dst[k * T + e] = v;
  };
  switch (p) {
    case 2: rfft_reg<Real, 2>(ld, stv, tc, tsn); break;
    case 4: rfft_reg<Real, 4>(ld, stv, tc, tsn); break;
    case 8: rfft_reg<Real, 8>(ld, stv, tc, tsn); break;
    case 16: rfft_reg<Real, 16>(ld, stv, tc, tsn); break;
    case 32: rfft_reg<Real, 32>(ld, stv, tc, tsn); break;
    default: {
      const int K = p / 2 + 1;
      for (int k = 0; k < K; ++k) {
        Real re = 0, im = 0;
        int r = 0;
        for (int t = 0; t < p; ++t) {
          const Real x = src[t * T + e];
          re = fma(x, tc[r], re);
          im = fma(-x, tsn[r], im);
          r += k;
          if (r >= p) r -= p;
        }
        stv(k, re, im);
      }
    }
  }
}

// MODE 0: out (concatenated) = y;  MODE 1: out = C_i - y (FP64) and per-block partial norms.
template <typename Real, typename Cplx, int MODE>
__global__ void __launch_bounds__(kTubes) k_b_irfft(BDev d, const Cplx* __restrict__ in, Real* __restrict__ out,
                                                    double* __restrict__ P) {
  const int i = d.tb_inst[blockIdx.x];
  const bool on = MODE ? d.cyc[i] : d.act[i];
  if (!on) return;
  const BInst& ins = d.inst[i];
  const int p = ins.p;
  __shared__ Real tc[64], tsn[64];
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    double sv, cv;
    sincospi(2.0 * r / p, &sv, &cv);
    tc[r] = (Real)cv;
    tsn[r] = (Real)sv;
  }
  __syncthreads();
  const long long e = d.tb_off[blockIdx.x] + threadIdx.x;
  double local = 0.0;
  if (e < ins.T) {
    const Cplx* src = in + ins.offS;
    Real* dst = out + ins.offN;
    const long long T = ins.T;
    const Real invp = Real(1) / Real(p);
    auto ld = [&](int k, Real& re, Real& im) {
      const Cplx c = src[k * T + e];
      re = c.x;
      im = c.y;
    };
    auto stv = [&](int t, Real v) {
      v *= invp;
      if (MODE == 1) {
        v = (Real)(ins.C[t * T + e] - (double)v);
        local += (double)v * (double)v;
      }
      dst[t * T + e] = v;
    };
    switch (p) {
      case 2: irfft_reg<Real, 2>(ld, stv, tc, tsn); break;
      case 4: irfft_reg<Real, 4>(ld, stv, tc, tsn); break;
      case 8: irfft_reg<Real, 8>(ld, stv, tc, tsn); break;
      case 16: irfft_reg<Real, 16>(ld, stv, tc, tsn); break;
      case 32: irfft_reg<Real, 32>(ld, stv, tc, tsn); break;
      default: {
        const int K = p / 2 + 1, nyq = (p % 2 == 0) ? p / 2 : -1;
        for (int t = 0; t < p; ++t) {
          Real y = 0;
          for (int k = 0; k < K; ++k) {
            const Cplx c = src[k * T + e];
            const int r = (int)(((long long)k * t) % p);
            if (k == 0 || k == nyq) {
              y = fma(c.x, tc[r], y);
            } else {
              y = fma(Real(2) * c.x, tc[r], y);
              y = fma(-Real(2) * c.y, tsn[r], y);
            }
          }
          stv(t, y);
        }
      }
    }
  }
  if (MODE == 1) {
    const double t = block_sum(local);
    if (threadIdx.x == 0) P[blockIdx.x] = t;
  }
}

// --- per-slice products over the work list ---------------------------------------------------------
// TILE 0: every instance has n, s <= kTinyL and the items are 8 x 4 tiles for kTinyThreads
// (gemm_tiny_tile); otherwise 64 x TILE tiles (TILE = 64, 32 or 16 columns; 4 x TILE/16 outputs per
// thread) for kGemmNT threads.  Every TILE > 0 sums each output entry's products in the same order
// (phase 1's reduction index, then phase 2's), so the column width, which the autotuner picks,
// changes which CTA forms an entry and how much padding it computes, never the entry's value.
template <typename Real, int MASK, int TILE>
__global__ void __launch_bounds__(kGemmNT, 1) k_b_gemm(BDev d, const int4* __restrict__ items,
                                                       const typename CplxOf<Real>::T* __restrict__ Xh,
                                                       typename CplxOf<Real>::T* __restrict__ Yh) {
  using Cplx = typename CplxOf<Real>::T;
  const int4 it = items[blockIdx.x];
  const int i = it.x;
  if (!(MASK ? d.cyc[i] : d.act[i])) return;
  const BInst& in = d.inst[i];
  GemmArgs<Cplx> a{};
  const Cplx* Ah;
  const Cplx* Bh;
  if constexpr (sizeof(Real) == 8) {
    Ah = reinterpret_cast<const Cplx*>(in.Ah);
    Bh = reinterpret_cast<const Cplx*>(in.Bh);
  } else {
    Ah = reinterpret_cast<const Cplx*>(in.Ah32);
    Bh = reinterpret_cast<const Cplx*>(in.Bh32);
  }
  const long long T = in.T;
  a.A1 = Ah; a.sA1 = (long long)in.n * in.n; a.lda1 = in.n;
  a.B1 = Xh + in.offS; a.sB1 = T; a.ldb1 = in.n; a.L1 = in.n;
  a.A2 = Xh + in.offS; a.sA2 = T; a.lda2 = in.n;
  a.B2 = Bh; a.sB2 = (long long)in.s * in.s; a.ldb2 = in.s; a.L2 = in.s;
  a.Y = Yh + in.offS; a.sY = T; a.ldy = in.n;
  a.M = in.n; a.N = in.s; a.K = in.K; a.nyq = in.nyq; a.sgn2 = -1.0;
  if constexpr (TILE == 0) gemm_tiny_tile<Real>(a, it.y, it.z, it.w);
  else gemm_tile<Real, kGemmBM, TILE, 4, TILE / 16>(a, it.y, it.z, it.w);
}

// Column widths the autotuner chooses from for the CUDA-core work-list products, and one work list.
constexpr int kBatchSimtBNs[] = {64, 32, 16};
struct SimtList {
  int bn;              // 0: the 8 x 4 tiles of an all-tiny batch
  const int4* items;   // device work list
  int count;
};

// One launch of the work-list products (no launch counting: the callers count, once per launch or
// per graph replay).
template <typename Real, int MASK>
void launch_b_gemm(const SimtList& l, const BDev& d, const void* X, void* Y, cudaStream_t st) {
  using Cplx = typename CplxOf<Real>::T;
  const Cplx* x = static_cast<const Cplx*>(X);
  Cplx* y = static_cast<Cplx*>(Y);
  switch (l.bn) {
    case 0: k_b_gemm<Real, MASK, 0><<<l.count, kTinyThreads, 0, st>>>(d, l.items, x, y); break;
    case 64: k_b_gemm<Real, MASK, 64><<<l.count, kGemmNT, 0, st>>>(d, l.items, x, y); break;
    case 32: k_b_gemm<Real, MASK, 32><<<l.count, kGemmNT, 0, st>>>(d, l.items, x, y); break;
    case 16: k_b_gemm<Real, MASK, 16><<<l.count, kGemmNT, 0, st>>>(d, l.items, x, y); break;
    default: TS_REQUIRE(false, "batched products: unknown tile width");
  }
  TS_CUDA(cudaGetLastError());
}

// --- small per-instance kernels ---------------------------------------------------------------------
__global__ void k_b_finalize_norm(BDev d, const double* __restrict__ P, int which) {
  // which 0: ||C|| from streaming partials; 1: residual from tube-block partials
  const int i = blockIdx.x;
  const BInst& in = d.inst[i];
  if (which == 1 && !d.cyc[i]) return;
  const double v = which == 0 ? inst_sum(P, in.nb0, in.nb1) : inst_sum(P, in.tb0, in.tb1);
  if (threadIdx.x == 0) {
    double* sc = d.sc + 16 * i;
    const double nv = sqrt(v);
    if (which == 0) {
      sc[SC_NORMC] = nv;
    } else {
      sc[SC_RES] = nv;
      sc[SC_INVRES] = nv > 0.0 ? 1.0 / nv : 0.0;
      const double tol = in.tol;
      sc[SC_DONE] = (nv <= tol * sc[SC_NORMC] || !isfinite(nv)) ? 1.0 : 0.0;
    }
  }
}

__global__ void k_b_ks_init(BDev d) {
  const int i = blockIdx.x;
  if (!d.cyc[i]) return;
  StLayout L{d.m};
  double* st = d.state + i * d.stride;
  const double beta = d.sc[16 * i + SC_RES];
  for (long long e = threadIdx.x; e < 2ll * (d.m + 1) * d.m; e += blockDim.x) st[e] = 0.0;
  for (int e = threadIdx.x; e <= d.m; e += blockDim.x) st[L.g() + e] = e == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    d.sc[16 * i + SC_K] = 0.0;
    d.sc[16 * i + SC_FLAGS] = 0.0;
  }
}

// Givens update of column j for every still-iterating instance; retires instances whose
// estimate passed, that broke down, or that reached the end of the cycle.
__global__ void k_b_givens(BDev d, const double* __restrict__ Pnorm, int j) {
  const int i = blockIdx.x;
  if (!d.act[i]) return;
  const BInst& in = d.inst[i];
  const double hn = sqrt(inst_sum(Pnorm, in.nb0, in.nb1));
  if (threadIdx.x != 0) return;
  StLayout L{d.m};
  const int m = d.m, ld = m + 1;
  double* st = d.state + i * d.stride;
  double* H = st + L.H();
  double* R = st + L.R();
  double* cs = st + L.cs();
  double* sn = st + L.sn();
  double* g = st + L.g();
  double* sc = d.sc + 16 * i;
  H[(j + 1) + ld * j] = hn;
  for (int r = 0; r <= j + 1; ++r) R[r + ld * j] = H[r + ld * j];
  for (int q = 0; q < j; ++q) {
    const double a = R[q + ld * j], b = R[q + 1 + ld * j];
    R[q + ld * j] = cs[q] * a + sn[q] * b;
    R[q + 1 + ld * j] = -sn[q] * a + cs[q] * b;
  }
  const double a = R[j + ld * j], b = R[j + 1 + ld * j];
  const double r = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (r > 0.0) {
    c = a / r;
    s = b / r;
  }
  cs[j] = c;
  sn[j] = s;
  R[j + ld * j] = r;
  R[j + 1 + ld * j] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  const double est = fabs(g[j + 1]);
  const double res = sc[SC_RES];
  sc[SC_EST] = est;
  sc[SC_H] = hn;
  sc[SC_INVH] = hn > 0.0 ? 1.0 / hn : 0.0;
  sc[SC_K] = j + 1;
  sc[SC_ITERS] += 1.0;
  const bool broke = hn <= 1e-14 * res;
  if (!isfinite(est) || !isfinite(hn)) sc[SC_FLAGS] = 4.0;
  if (broke || !isfinite(est) || est <= in.tol * sc[SC_NORMC] || (d.mixed && est <= d.inner_tol * res) ||
      j + 1 == m)
    d.act[i] = 0;
}

__global__ void k_b_solve_y(BDev d) {
  const int i = blockIdx.x;
  if (!d.cyc[i] || threadIdx.x != 0) return;
  StLayout L{d.m};
  const int m = d.m, ld = m + 1;
  double* st = d.state + i * d.stride;
  const double* R = st + L.R();
  const double* g = st + L.g();
  double* y = st + L.y();
  const int k = (int)d.sc[16 * i + SC_K];
  for (int r = k - 1; r >= 0; --r) {
    double v = g[r];
    for (int q = r + 1; q < k; ++q) v -= R[r + ld * q] * y[q];
    y[r] = v / R[r + ld * r];
  }
}

// Ends a nested cycle graph after the current step when no instance is still iterating.
__global__ void k_b_any_active(BDev d, cudaGraphConditionalHandle next) {
  int any = 0;
  for (int i = threadIdx.x; i < d.count; i += blockDim.x) any |= d.act[i];
  any = __syncthreads_or(any);
  if (threadIdx.x == 0 && !any) cudaGraphSetConditional(next, 0);
}

// --- host orchestration -----------------------------------------------------------------------------
// Kernels are loaded lazily on first launch, and loading is not allowed while a stream is being
// captured; every kernel of the captured cycle is therefore loaded (cudaFuncGetAttributes) first.
template <typename T, typename Real2>
void preload_cycle_kernels() {
  cudaFuncAttributes fa;
  const void* fns[] = {
      (const void*)k_b_ks_init, (const void*)k_b_scale_R<T>, (const void*)k_b_rfft<T, Real2, 0, 0>,
      (const void*)k_b_gemm<T, 0, 0>, (const void*)k_b_gemm<T, 0, 64>, (const void*)k_b_gemm<T, 0, 32>,
      (const void*)k_b_gemm<T, 0, 16>, (const void*)k_b_irfft<T, Real2, 0>,
      (const void*)k_b_dot<T>,
      (const void*)k_b_mgs<T>, (const void*)k_b_givens, (const void*)k_b_scale_W<T>, (const void*)k_b_solve_y,
      (const void*)k_b_axpy<T>, (const void*)k_b_rfft<double, double2, 1, 1>, (const void*)k_b_gemm<double, 1, 0>,
      (const void*)k_b_gemm<double, 1, 64>, (const void*)k_b_gemm<double, 1, 32>, (const void*)k_b_gemm<double, 1, 16>,
      (const void*)k_b_irfft<double, double2, 1>, (const void*)k_b_finalize_norm, (const void*)k_b_any_active};
  for (const void* f : fns) TS_CUDA(cudaFuncGetAttributes(&fa, f));
}

struct BatchPlan {
  std::vector<BInst> inst;
  std::vector<int> nb_inst, tb_inst;
  std::vector<long long> nb_off, tb_off;
  bool tiny = false;   // CUDA-core products on 8 x 4 tiles (gemm_tiny_tile) instead of 64 x BN
  long long totN = 0, totS = 0;
};

// The pieces of one restart cycle, each recorded on `st` and returning the kernels it launched:
// the prologue (Givens state reset, V_1 = R / ||R||), inner step j (DFT, inner slice products,
// inverse DFT, MGS sweep, Givens update, V_{j+1}; with a conditional handle of step j + 1 it also ends
// a nested cycle graph once no instance is iterating), and the epilogue (y, X += V y, the FP64 true
// residual).  `residual_products(st)` issues the FP64 slice products of the residual (Xh64 -> Yh64)
// and `inner_products(st)` the inner operator's (Xh -> Yh); both return their kernel counts.
// ev (may be null; flat graphs only): 2m + 2 events recorded as graph nodes around the inner products
// of step j (ev[2j], ev[2j+1]) and around the residual products (ev[2m], ev[2m+1]), for the statistics.
template <typename T, typename Real2, typename InnerProducts, typename ResidualProducts>
struct CycleRecorder {
  const BDev& d;
  const BatchPlan& plan;
  T* V;
  T* W;
  Real2* Xh;
  Real2* Yh;
  double* R;
  double2* Xh64;
  double2* Yh64;
  double* P0;
  double* P1;
  double* Pt;
  const InnerProducts& inner_products;
  const ResidualProducts& residual_products;
  const cudaEvent_t* ev;

  int prologue(cudaStream_t st) const {
    const int nbs = (int)plan.nb_inst.size();
    k_b_ks_init<<<d.count, 256, 0, st>>>(d);
    k_b_scale_R<T><<<nbs, 256, 0, st>>>(d, R, basis(V, d.totN, 0));
    TS_CUDA(cudaGetLastError());
    return 2;
  }
  int step(int j, cudaGraphConditionalHandle next, cudaStream_t st) const {
    using Real = T;
    const int nbs = (int)plan.nb_inst.size(), ntb = (int)plan.tb_inst.size();
    double* Pp[2] = {P0, P1};
    int kernels = 0;
    k_b_rfft<Real, Real2, 0, 0><<<ntb, kTubes, 0, st>>>(d, basis(V, d.totN, j), Xh);
    if (ev) TS_CUDA(cudaEventRecordWithFlags(ev[2 * j], st, cudaEventRecordExternal));
    kernels += inner_products(st);
    if (ev) TS_CUDA(cudaEventRecordWithFlags(ev[2 * j + 1], st, cudaEventRecordExternal));
    k_b_irfft<Real, Real2, 0><<<ntb, kTubes, 0, st>>>(d, Yh, W, nullptr);
    k_b_dot<T><<<nbs, 256, 0, st>>>(d, basis(V, d.totN, 0), W, Pp[0]);
    for (int i = 0; i <= j; ++i)
      k_b_mgs<T><<<nbs, 256, 0, st>>>(d, W, basis(V, d.totN, i), i < j ? basis(V, d.totN, i + 1) : nullptr,
                                      Pp[i & 1], Pp[(i + 1) & 1], i, j);
    k_b_givens<<<d.count, 256, 0, st>>>(d, Pp[(j + 1) & 1], j);
    k_b_scale_W<T><<<nbs, 256, 0, st>>>(d, W, basis(V, d.totN, j + 1));
    kernels += 5 + j + 1;
    if (next) {
      k_b_any_active<<<1, 256, 0, st>>>(d, next);
      ++kernels;
    }
    TS_CUDA(cudaGetLastError());
    return kernels;
  }
  int epilogue(cudaStream_t st) const {
    const int nbs = (int)plan.nb_inst.size(), ntb = (int)plan.tb_inst.size();
    const int m = d.m;
    int kernels = 0;
    k_b_solve_y<<<d.count, 32, 0, st>>>(d);
    k_b_axpy<T><<<nbs, 256, 0, st>>>(d, V);
    // true residual R = C - M(X) in FP64
    k_b_rfft<double, double2, 1, 1><<<ntb, kTubes, 0, st>>>(d, nullptr, Xh64);
    if (ev) TS_CUDA(cudaEventRecordWithFlags(ev[2 * m], st, cudaEventRecordExternal));
    kernels += residual_products(st);
    if (ev) TS_CUDA(cudaEventRecordWithFlags(ev[2 * m + 1], st, cudaEventRecordExternal));
    k_b_irfft<double, double2, 1><<<ntb, kTubes, 0, st>>>(d, Yh64, R, Pt);
    k_b_finalize_norm<<<d.count, 256, 0, st>>>(d, Pt, 1);
    kernels += 5;
    TS_CUDA(cudaGetLastError());
    return kernels;
  }
};

}  // namespace

ts_status batched_entry(ts_ctx* ctx, int count, const ts_instance* insts, const ts_solve_opts* opts,
                        ts_solve_info* infos, int* statuses, ts_stream stream) {
  TS_REQUIRE(count >= 1 && insts && opts, "ts_batched_solve: bad arguments");
  const auto host_t0 = std::chrono::steady_clock::now();
  auto host_ms_since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
  };
  const ts_solve_opts& o = *opts;
  TS_REQUIRE(o.restart >= 1 && o.restart <= 128, "ts_batched_solve: restart must be in 1..128");
  TS_REQUIRE(o.tol > 0.0, "ts_batched_solve: tol must be positive");
  TS_REQUIRE(o.precision >= TS_FP64 && o.precision <= TS_MIXED_TF32X3, "ts_batched_solve: unknown precision");
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  TS_REQUIRE(o.fp64_engine == TS_ENGINE_DFMA || o.fp64_engine == TS_ENGINE_OZAKI,
             "ts_batched_solve: unknown fp64_engine");
  TS_REQUIRE(o.ozaki_digits == 0 || (o.ozaki_digits >= 3 && o.ozaki_digits <= 8),
             "ts_batched_solve: ozaki_digits must be 3..8");
  const bool ozaki = o.fp64_engine == TS_ENGINE_OZAKI;
  const int oz_digits = o.ozaki_digits == 0 ? 6 : o.ozaki_digits;
  const bool mixed = o.precision != TS_FP64;
  // tensor-core inner products (BF16, TF32 or split TF32); FP32 CUDA cores for TS_MIXED_FP32
  const bool tcin = mixed && o.precision != TS_MIXED_FP32;
  std::vector<ts_op*> ops(count);
  const int m = o.restart;
  BatchPlan plan;
  plan.inst.resize(count);
  for (int i = 0; i < count; ++i) {
    const ts_instance& u = insts[i];
    TS_REQUIRE(u.op && u.C && u.X, "ts_batched_solve: instance with a null pointer");
    ts_op* op = const_cast<ts_op*>(u.op);
    ops[i] = op;
    TS_REQUIRE(!op->sp, "ts_batched_solve: dense operators only");
    TS_REQUIRE(op->p <= 64, "ts_batched_solve: p must be <= 64");
    TS_REQUIRE(is_device_ptr(u.C) && is_device_ptr(u.X), "ts_batched_solve: C and X must be device memory");
    BInst& b = plan.inst[i];
    b.X = u.X;
    b.C = u.C;
    b.Ah = op->Ah;
    b.Bh = op->Bh;
    if (mixed) {
      if (tcin) tc_prepare(op, o.precision, user);
      else ensure_f32_operator(op, user);
      b.Ah32 = op->Ah32;
      b.Bh32 = op->Bh32;
    }
    b.n = op->n; b.s = op->s; b.p = op->p; b.K = op->K; b.nyq = nyquist_index(op->p);
    b.T = (long long)b.n * b.s;
    b.N = b.T * b.p;
    b.offN = (plan.totN + 3) / 4 * 4;   // 16-byte aligned start: the streaming kernels move packs of 4
    b.offS = plan.totS;
    plan.totN = b.offN + b.N;
    plan.totS += (long long)b.K * b.T;
    b.tol = u.tol > 0 ? u.tol : o.tol;
    b.nb0 = (int)plan.nb_inst.size();
    for (long long l = 0; l < b.N; l += kChunk) {
      plan.nb_inst.push_back(i);
      plan.nb_off.push_back(l);
    }
    b.nb1 = (int)plan.nb_inst.size();
    b.tb0 = (int)plan.tb_inst.size();
    for (long long t = 0; t < b.T; t += kTubes) {
      plan.tb_inst.push_back(i);
      plan.tb_off.push_back(t);
    }
    b.tb1 = (int)plan.tb_inst.size();
  }
  plan.totN = (plan.totN + 3) / 4 * 4;   // every basis vector V + j totN starts 16-byte aligned
  TS_REQUIRE(plan.nb_inst.size() < (size_t)INT32_MAX, "batch too large");
  const size_t tsz = mixed ? sizeof(float) : sizeof(double);
  auto get = [&](const char* name, size_t bytes) { return ctx->ws.get(name, bytes); };
  char* base = (char*)get("b_tables", sizeof(BInst) * count + 16 * (plan.nb_inst.size() + plan.tb_inst.size()) +
                                          1024);
  BInst* d_inst = (BInst*)base;
  int* d_nb_inst = (int*)(d_inst + count);
  long long* d_nb_off = (long long*)(((uintptr_t)(d_nb_inst + plan.nb_inst.size()) + 15) & ~(uintptr_t)15);
  int* d_tb_inst = (int*)(d_nb_off + plan.nb_off.size());
  long long* d_tb_off = (long long*)(((uintptr_t)(d_tb_inst + plan.tb_inst.size()) + 15) & ~(uintptr_t)15);
  // the tables are copied from pageable memory: synchronous, before anything is captured
  TS_CUDA(cudaMemcpy(d_inst, plan.inst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(d_nb_inst, plan.nb_inst.data(), sizeof(int) * plan.nb_inst.size(), cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(d_nb_off, plan.nb_off.data(), sizeof(long long) * plan.nb_off.size(), cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(d_tb_inst, plan.tb_inst.data(), sizeof(int) * plan.tb_inst.size(), cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(d_tb_off, plan.tb_off.data(), sizeof(long long) * plan.tb_off.size(), cudaMemcpyHostToDevice));
  // CUDA-core slice products (FP64: the residuals on the DFMA engine and the whole cycle of a TS_FP64
  // batch on it; FP32: the inner products of TS_MIXED_FP32) run over a work list of (instance, slice,
  // row, column) tiles: warp-sized 8 x 4 tiles when every instance is tiny (a 64 x 64 tile of a
  // 24 x 24 product issues 10x the FP64 work it needs), else 64 x BN tiles, BN in kBatchSimtBNs picked
  // per element size and batch shape by the autotuner.  The FP64 pipe (2 DFMA per clock per SM) is
  // far slower than shared memory, so a narrow tile that pads s less can win for FP64 while FP32
  // wants the reuse of wide tiles.  A cached choice needs only its own list.
  const bool simt64 = !ozaki, simt32 = mixed && !tcin;
  plan.tiny = true;
  for (const BInst& b : plan.inst) plan.tiny = plan.tiny && b.n <= kTinyL && b.s <= kTinyL;
  std::string simt_shape = ":" + std::to_string(count);
  for (const BInst& b : plan.inst)
    simt_shape += ":" + std::to_string(b.n) + "x" + std::to_string(b.s) + "x" + std::to_string(b.K);
  auto simt_key = [&](int esz) { return "bsimt:" + std::to_string(esz) + simt_shape; };
  if (!ctx->tune_loaded) tune_load(ctx);
  auto simt_cands = [&](int esz) {
    if (plan.tiny) return std::vector<int>{0};
    const auto t = ctx->tune.find(simt_key(esz));
    for (int bn : kBatchSimtBNs)
      if (t != ctx->tune.end() && t->second == bn) return std::vector<int>{bn};
    return std::vector<int>(std::begin(kBatchSimtBNs), std::end(kBatchSimtBNs));
  };
  std::vector<SimtList> simt;
  {
    std::vector<int> need;
    for (int esz : {8, 4}) {
      if (!(esz == 8 ? simt64 : simt32)) continue;
      for (int bn : simt_cands(esz))
        if (std::find(need.begin(), need.end(), bn) == need.end()) need.push_back(bn);
    }
    for (int bn : need) {
      const int tbm = bn == 0 ? kTinyBM : kGemmBM, tbn = bn == 0 ? kTinyBN : bn;
      std::vector<int4> items;
      for (int i = 0; i < count; ++i) {
        const BInst& b = plan.inst[i];
        for (int k = 0; k < b.K; ++k)
          for (int i0 = 0; i0 < b.n; i0 += tbm)
            for (int j0 = 0; j0 < b.s; j0 += tbn) items.push_back(make_int4(i, k, i0, j0));
      }
      // Largest tiles first (reduction length n + s; real slices are a quarter of the work).
      std::stable_sort(items.begin(), items.end(), [&](const int4& a, const int4& b) {
        auto cost = [&](const int4& q) {
          const BInst& x = plan.inst[q.x];
          const double w = (q.y == 0 || q.y == x.nyq) ? 1.0 : 4.0;
          return w * (x.n + x.s);
        };
        return cost(a) > cost(b);
      });
      TS_REQUIRE(items.size() < (size_t)INT32_MAX, "batch too large");
      int4* dev = (int4*)get(("b_items_" + std::to_string(bn)).c_str(), sizeof(int4) * items.size());
      TS_CUDA(cudaMemcpy(dev, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
      simt.push_back(SimtList{bn, dev, (int)items.size()});
    }
  }
  auto simt_list = [&](int bn) -> const SimtList& {
    size_t q = 0;
    while (q + 1 < simt.size() && simt[q].bn != bn) ++q;
    TS_REQUIRE(!simt.empty() && simt[q].bn == bn, "batched products: no work list for the chosen tile");
    return simt[q];
  };

  void* V = get("b_V", tsz * (size_t)(m + 1) * plan.totN);
  void* W = get("b_W", tsz * (size_t)plan.totN);
  double* R = (double*)get("b_R", sizeof(double) * (size_t)plan.totN);
  void* Xh = get("b_Xh", 2 * tsz * (size_t)plan.totS);
  void* Yh = get("b_Yh", 2 * tsz * (size_t)plan.totS);
  double2* Xh64 = mixed ? (double2*)get("b_Xh64", sizeof(double2) * (size_t)plan.totS) : (double2*)Xh;
  double2* Yh64 = mixed ? (double2*)get("b_Yh64", sizeof(double2) * (size_t)plan.totS) : (double2*)Yh;
  const size_t np = std::max(plan.nb_inst.size(), plan.tb_inst.size());
  double* P0 = (double*)get("b_P0", sizeof(double) * np);
  double* P1 = (double*)get("b_P1", sizeof(double) * np);
  double* Pt = (double*)get("b_Pt", sizeof(double) * np);
  double* sc = (double*)get("b_sc", sizeof(double) * 16 * count);
  int* flags = (int*)get("b_flags", sizeof(int) * 2 * count);
  const long long stride = state_stride(m);
  double* state = (double*)get("b_state", sizeof(double) * (size_t)stride * count);
  // Emulated FP64 residual products: digit planes of every operator; the instances' products run
  // on kOzBranches side streams (parallel branches of the captured graph, since one small
  // instance fills few SMs), each branch with its own scratch set sized for the largest instance.
  // Everything is made before anything is captured.
  constexpr int kOzBranches = 8;
  std::vector<OzBuffers> ozb(kOzBranches);
  std::vector<int> order(count);
  int* tc_err = (int*)get("tc_err", sizeof(int) * 4);
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  if (ozaki) {
    OzBufferSizes zmax;
    for (int i = 0; i < count; ++i) {
      oz_prepare(ops[i], oz_digits, user);
      const OzBufferSizes z = oz_buffer_sizes(ops[i]->n, ops[i]->s, ops[i]->K, oz_digits);
      zmax.xc = std::max(zmax.xc, z.xc);
      zmax.xr = std::max(zmax.xr, z.xr);
      zmax.K = std::max(zmax.K, z.K);
    }
    oz_preload();
    for (int q = 0; q < kOzBranches; ++q) {
      const std::string sfx = "_" + std::to_string(q);
      ozb[q].xc_re = get(("b_oz_xc_re" + sfx).c_str(), zmax.xc);
      ozb[q].xc_im = get(("b_oz_xc_im" + sfx).c_str(), zmax.xc);
      ozb[q].xc_nim = get(("b_oz_xc_nim" + sfx).c_str(), zmax.xc);
      ozb[q].xr_re = get(("b_oz_xr_re" + sfx).c_str(), zmax.xr);
      ozb[q].xr_im = get(("b_oz_xr_im" + sfx).c_str(), zmax.xr);
      ozb[q].mx = (unsigned long long*)get(("b_oz_mx" + sfx).c_str(), sizeof(unsigned long long) * zmax.K);
      ozb[q].Ex = (int*)get(("b_oz_Ex" + sfx).c_str(), sizeof(int) * zmax.K);
    }
    while ((int)ctx->side.size() < kOzBranches) {
      cudaStream_t q;
      TS_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
      ctx->side.push_back(q);
    }
    TS_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    join_ev.resize(kOzBranches);
    for (auto& e : join_ev) TS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // largest products first, dealt round-robin over the branches
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      auto cost = [&](int i) { return (double)ops[i]->K * ops[i]->n * ops[i]->s * (ops[i]->n + ops[i]->s); };
      return cost(a) > cost(b);
    });
    TS_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int) * 4, user));
  }
  struct EventGuard {
    cudaEvent_t& f;
    std::vector<cudaEvent_t>& j;
    ~EventGuard() {
      if (f) cudaEventDestroy(f);
      for (auto e : j) cudaEventDestroy(e);
    }
  } ev_guard{fork_ev, join_ev};

  BDev d{};
  d.inst = d_inst;
  d.count = count;
  d.m = m;
  d.totN = plan.totN;
  d.totS = plan.totS;
  d.nb_inst = d_nb_inst;
  d.nb_off = d_nb_off;
  d.tb_inst = d_tb_inst;
  d.tb_off = d_tb_off;
  d.cyc = flags;
  d.act = flags + count;
  d.sc = sc;
  d.state = state;
  d.stride = stride;
  // default inner tolerances as in the single-instance solver (FP32 / split TF32, TF32, BF16)
  const double inner_default =
      o.precision == TS_MIXED_TF32 ? 1e-3 : (o.precision == TS_MIXED_BF16 ? 1e-2 : 1e-6);
  d.inner_tol = mixed ? (o.inner_tol > 0 ? o.inner_tol : inner_default) : 0.0;
  d.mixed = mixed ? 1 : 0;

  // A private stream for the captured cycle, ordered after the caller's stream.
  if (!ctx->bstream) TS_CUDA(cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking));
  cudaStream_t st = ctx->bstream;
  TS_CUDA(cudaEventRecord(ctx->ev0, user));
  TS_CUDA(cudaStreamWaitEvent(st, ctx->ev0, 0));
  cudaEvent_t t0, t1;
  TS_CUDA(cudaEventCreate(&t0));
  TS_CUDA(cudaEventCreate(&t1));
  TS_CUDA(cudaEventRecord(t0, st));

  std::vector<int> hflags(2 * count, 1);
  TS_CUDA(cudaMemcpyAsync(flags, hflags.data(), sizeof(int) * 2 * count, cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaMemsetAsync(sc, 0, sizeof(double) * 16 * count, st));
  const int nbs = (int)plan.nb_inst.size(), ntb = (int)plan.tb_inst.size();
  // Column widths of the CUDA-core products, tuned on one product pass of the whole batch with every
  // instance active (flags set above) from zeroed inputs; before anything is captured.
  auto simt_pick = [&](int esz) -> int {
    if (plan.tiny) return 0;
    const std::vector<int> cands = simt_cands(esz);
    if (cands.size() > 1)
      TS_CUDA(cudaMemsetAsync(esz == 8 ? (void*)Xh64 : Xh, 0, (size_t)2 * esz * plan.totS, st));
    return tune_pick(
        ctx, simt_key(esz), cands,
        [&](int bn) {
          if (esz == 8) launch_b_gemm<double, 0>(simt_list(bn), d, Xh64, Yh64, st);
          else launch_b_gemm<float, 0>(simt_list(bn), d, Xh, Yh, st);
          count_launch();
        },
        st);
  };
  const int simt_bn64 = simt64 ? simt_pick(8) : 0, simt_bn32 = simt32 ? simt_pick(4) : 0;
  // Tensor-core inner products: every instance's planar X copies, tensor maps and work lists,
  // made before anything is captured.
  struct TcTables {
    const TcMaps* maps = nullptr;
    const BTcPlanes* planes = nullptr;
    const BTcInst* inst = nullptr;
    const int4* titems = nullptr;
    const int4* pitems = nullptr;
    int n_titems = 0, n_pitems = 0;
  };
  TcTables tct;
  int tc_bn = tc_batch_sched(kBatchTcBNs[0], false);   // product schedule (column tile, persistent)
  if (tcin) {
    std::vector<size_t> poff(count);
    size_t ptot = 0;
    for (int i = 0; i < count; ++i) {
      poff[i] = ptot;
      ptot += tc_batch_plane_bytes(ops[i]->n, ops[i]->s, ops[i]->K, o.precision);
    }
    char* planes = (char*)get("b_tc_planes", ptot);
    // One set of tables per candidate column tile: the tensor maps' B boxes and the tile work list
    // depend on it, the planar X copies do not.
    auto build_tables = [&](int bn) -> TcTables {
      std::vector<TcMaps> hmaps(count);
      std::vector<BTcPlanes> hplanes(count);
      std::vector<BTcInst> hinst(count);
      std::vector<int4> titems, pitems;
      for (int i = 0; i < count; ++i) {
        const BInst& b = plan.inst[i];
        tc_batch_instance(ops[i], o.precision, (const float2*)Xh + b.offS, planes + poff[i], &hplanes[i], &hmaps[i],
                          bn);
        hinst[i] = BTcInst{(float2*)Yh + b.offS, b.n, b.s, b.nyq};
        for (int k = 0; k < b.K; ++k) {
          for (int i0 = 0; i0 < b.n; i0 += 128)
            for (int j0 = 0; j0 < b.s; j0 += bn) titems.push_back(make_int4(i, k, i0, j0));
          for (int i0 = 0; i0 < b.n; i0 += 32)
            for (int j0 = 0; j0 < b.s; j0 += 32) pitems.push_back(make_int4(i, k, i0, j0));
        }
      }
      // largest tiles first: interior slices carry four real products, the DC and Nyquist ones one
      std::stable_sort(titems.begin(), titems.end(), [&](const int4& a, const int4& b) {
        auto cost = [&](const int4& q) {
          const BInst& x = plan.inst[q.x];
          return ((q.y == 0 || q.y == x.nyq) ? 1.0 : 4.0) * (x.n + x.s);
        };
        return cost(a) > cost(b);
      });
      const std::string name = "b_tc_tables_" + std::to_string(bn);
      char* tab = (char*)get(name.c_str(), sizeof(TcMaps) * count + sizeof(BTcPlanes) * count +
                                               sizeof(BTcInst) * count + sizeof(int4) * (titems.size() + pitems.size()) +
                                               1024);
      TcMaps* m_ = (TcMaps*)tab;                                  // 2 KB each: 64-byte aligned tensor maps
      BTcPlanes* p_ = (BTcPlanes*)(m_ + count);
      BTcInst* in_ = (BTcInst*)(((uintptr_t)(p_ + count) + 15) & ~(uintptr_t)15);
      int4* ti_ = (int4*)(((uintptr_t)(in_ + count) + 15) & ~(uintptr_t)15);
      int4* pi_ = ti_ + titems.size();
      TS_CUDA(cudaMemcpy(m_, hmaps.data(), sizeof(TcMaps) * count, cudaMemcpyHostToDevice));
      TS_CUDA(cudaMemcpy(p_, hplanes.data(), sizeof(BTcPlanes) * count, cudaMemcpyHostToDevice));
      TS_CUDA(cudaMemcpy(in_, hinst.data(), sizeof(BTcInst) * count, cudaMemcpyHostToDevice));
      TS_CUDA(cudaMemcpy(ti_, titems.data(), sizeof(int4) * titems.size(), cudaMemcpyHostToDevice));
      TS_CUDA(cudaMemcpy(pi_, pitems.data(), sizeof(int4) * pitems.size(), cudaMemcpyHostToDevice));
      TcTables t;
      t.maps = m_;
      t.planes = p_;
      t.inst = in_;
      t.titems = ti_;
      t.pitems = pi_;
      t.n_titems = (int)titems.size();
      t.n_pitems = (int)pitems.size();
      return t;
    };
    tc_batch_preload(o.precision);   // shared-memory limits of the product kernels, before any launch
    // Pick the column tile by timing one product pass of the whole batch with every instance
    // active (the activity flags are all set above); the choice is cached per batch shape, and once
    // it exists only its tables are built.
    std::string key = "btc:" + std::to_string(o.precision) + ":" + std::to_string(count);
    for (int i = 0; i < count; ++i)
      key += ":" + std::to_string(plan.inst[i].n) + "x" + std::to_string(plan.inst[i].s) + "x" +
             std::to_string(plan.inst[i].K);
    if (!ctx->tune_loaded) tune_load(ctx);
    const auto tuned = ctx->tune.find(key);
    // Candidates: every usable column tile, each with the one-CTA-per-item and the persistent
    // schedule (tc_batch_sched); tables exist once per column tile.
    std::vector<int> bns, cands;
    std::vector<TcTables> bn_tables;
    int smax = 0;
    for (int i = 0; i < count; ++i) smax = std::max(smax, plan.inst[i].s);
    auto add_cands = [&](bool only_cached) {
      for (int bn : kBatchTcBNs) {
        if (!(bn == kBatchTcBNs[0] || bn / 2 < smax)) continue;
        bool any = false;
        for (bool pers : {false, true}) {
          const int c = tc_batch_sched(bn, pers);
          if (only_cached && tuned->second != c) continue;
          cands.push_back(c);
          any = true;
        }
        if (any) {
          bns.push_back(bn);
          bn_tables.push_back(build_tables(bn));
        }
      }
    };
    add_cands(tuned != ctx->tune.end());
    if (cands.empty()) {   // a cached choice this batch cannot use: tune again
      ctx->tune.erase(key);
      add_cands(false);
    }
    auto tables_of = [&](int c) -> const TcTables& {
      return bn_tables[std::find(bns.begin(), bns.end(), tc_batch_bn(c)) - bns.begin()];
    };
    TS_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int) * 4, st));
    tc_bn = tune_pick(
        ctx, key, cands,
        [&](int c) {
          const TcTables& t = tables_of(c);
          tc_batch_products(o.precision, c, t.planes, t.pitems, t.n_pitems, t.maps, t.inst, d.act, t.titems,
                            t.n_titems, tc_err, st);
        },
        st);
    tct = tables_of(tc_bn);
    TS_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int) * 4, st));
  }
  // Emulated-FP64 slice products of every instance (X -> Y, spectral FP64), each gated on the device
  // by the instance's flag in `gate`: dealt largest first over the kOzBranches side streams, forked
  // from and joined back to s2.
  auto oz_all = [&](cudaStream_t s2, const double2* X, double2* Y, const int* gate) -> int {
    // fork: every branch waits for the products' input; join: s2 waits for every branch
    TS_CUDA(cudaEventRecord(fork_ev, s2));
    for (int q = 0; q < kOzBranches; ++q) TS_CUDA(cudaStreamWaitEvent(ctx->side[q], fork_ev, 0));
    for (int r = 0; r < count; ++r) {
      const int i = order[r], q = r % kOzBranches;
      oz_products(ops[i], X + plan.inst[i].offS, Y + plan.inst[i].offS, oz_digits, ozb[q], gate + i, tc_err,
                  ctx->side[q]);
    }
    for (int q = 0; q < kOzBranches; ++q) {
      TS_CUDA(cudaEventRecord(join_ev[q], ctx->side[q]));
      TS_CUDA(cudaStreamWaitEvent(s2, join_ev[q], 0));
    }
    return 5 * count;
  };
  auto inner_products = [&](cudaStream_t s2) -> int {
    // FP64 solve on the emulated engine: the Arnoldi products too (gated by the inner-cycle flag)
    if (!mixed && ozaki) return oz_all(s2, (const double2*)Xh, (double2*)Yh, d.act);
    if (tcin) {
      tc_batch_products(o.precision, tc_bn, tct.planes, tct.pitems, tct.n_pitems, tct.maps, tct.inst, d.act,
                        tct.titems, tct.n_titems, tc_err, s2);
      return 2;
    }
    if (mixed) launch_b_gemm<float, 0>(simt_list(simt_bn32), d, Xh, Yh, s2);
    else launch_b_gemm<double, 0>(simt_list(simt_bn64), d, Xh, Yh, s2);
    return 1;
  };
  // FP64 slice products of a true residual: the (instance, slice, tile) work list on CUDA cores, or
  // one emulated-FP64 product per instance (each gated by the instance's cycle flag).
  auto residual_products = [&](cudaStream_t s2) -> int {
    if (!ozaki) {
      launch_b_gemm<double, 1>(simt_list(simt_bn64), d, Xh64, Yh64, s2);
      return 1;
    }
    return oz_all(s2, Xh64, Yh64, d.cyc);
  };
  ctx->timer.host_setup_ms += host_ms_since(host_t0);
  const auto cycles_t0 = std::chrono::steady_clock::now();
  k_b_normC<<<nbs, 256, 0, st>>>(d, P0);
  k_b_finalize_norm<<<count, 256, 0, st>>>(d, P0, 0);
  k_b_rfft<double, double2, 1, 1><<<ntb, kTubes, 0, st>>>(d, nullptr, Xh64);
  const int first = residual_products(st);
  k_b_irfft<double, double2, 1><<<ntb, kTubes, 0, st>>>(d, Yh64, R, Pt);
  k_b_finalize_norm<<<count, 256, 0, st>>>(d, Pt, 1);
  count_launch(ozaki ? 5 : 5 + first);   // the emulated products count their own launches
  TS_CUDA(cudaGetLastError());

  std::vector<double> hsc(16 * count);
  std::vector<int> done(count, 0), cycles(count, 0);
  cudaGraphExec_t exec = nullptr;
  long long cycle_fixed_kernels = 0;          // prologue and epilogue of a cycle graph
  std::vector<long long> cycle_step_kernels;  // kernels of each inner step
  bool nested_graph = false;
  int max_cycles = mixed ? (o.max_outer > 0 ? o.max_outer : 50) : o.max_restarts;
  int launched = 0;
  ts_status overall = TS_OK;
  // Statistics (while enabled): events recorded inside the cycle graph time the inner products of each
  // step and the residual products; after each replay the host adds their durations, and the
  // algorithmic work of the instances that took part (inner steps from each instance's iteration
  // count, residuals from its cycle flag), to the context's timer.
  std::vector<cudaEvent_t> tev;
  struct TevGuard {
    std::vector<cudaEvent_t>& e;
    ~TevGuard() {
      for (auto x : e) cudaEventDestroy(x);
    }
  } tev_guard{tev};
  if (ctx->timer.enabled) {
    tev.resize(2 * m + 2);
    for (auto& e : tev) TS_CUDA(cudaEventCreate(&e));
  }
  std::vector<double> iters_prev(count, 0.0), inst_flops(count), inst_pairs(count);
  for (int i = 0; i < count; ++i) {
    const ts_op* op = ops[i];
    inst_flops[i] = gemm_flops(op->n, op->s, op->n, op->s, op->K, nyquist_index(op->p));
    inst_pairs[i] = ozaki ? oz_bf16_flops(op->n, op->s, op->K, nyquist_index(op->p), oz_digits) : 0.0;
  }
  std::vector<int> in_cycle(count, 0);
  auto collect_phase_times = [&]() {
    KernelTimer& tm = ctx->timer;
    double inner_ms = 0.0, res_ms = 0.0, inner_work = 0.0, res_work = 0.0, inner_pairs = 0.0, res_pairs = 0.0;
    for (int j = 0; j < m; ++j) {
      float x = 0.f;
      TS_CUDA(cudaEventElapsedTime(&x, tev[2 * j], tev[2 * j + 1]));
      inner_ms += x;
    }
    float x = 0.f;
    TS_CUDA(cudaEventElapsedTime(&x, tev[2 * m], tev[2 * m + 1]));
    res_ms = x;
    for (int i = 0; i < count; ++i) {
      const double steps = hsc[16 * i + SC_ITERS] - iters_prev[i];
      iters_prev[i] = hsc[16 * i + SC_ITERS];
      inner_work += steps * inst_flops[i];
      inner_pairs += steps * inst_pairs[i];
      if (in_cycle[i]) {
        res_work += inst_flops[i];
        res_pairs += inst_pairs[i];
      }
    }
    // inner products: low precision (kind 2), or FP64 on the emulated (3) or DFMA (0) engine
    if (mixed) {
      tm.lowp_launches += m;
      tm.lowp_ms += inner_ms;
      tm.lowp_flops += inner_work;
    } else if (ozaki) {
      tm.oz_launches += m;
      tm.oz_ms += inner_ms;
      tm.oz_flops += inner_work;
      tm.oz_pair_flops += inner_pairs;
    } else {
      tm.gemm_launches += m;
      tm.gemm_ms += inner_ms;
      tm.gemm_flops += inner_work;
    }
    if (ozaki) {
      tm.oz_launches += 1;
      tm.oz_ms += res_ms;
      tm.oz_flops += res_work;
      tm.oz_pair_flops += res_pairs;
    } else {
      tm.gemm_launches += 1;
      tm.gemm_ms += res_ms;
      tm.gemm_flops += res_work;
    }
  };
  try {
    for (int cycle = 0; cycle <= max_cycles; ++cycle) {
      TS_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(double) * 16 * count, cudaMemcpyDeviceToHost, st));
      TS_CUDA(cudaStreamSynchronize(st));
      if (cycle > 0) {
        // kernels of the replay just done: a nested graph ran as many steps as its busiest instance
        int steps_run = m;
        if (nested_graph) {
          steps_run = 0;
          for (int i = 0; i < count; ++i)
            if (in_cycle[i]) steps_run = std::max(steps_run, (int)hsc[16 * i + SC_K]);
        }
        long long ran = cycle_fixed_kernels;
        for (int j = 0; j < steps_run && j < (int)cycle_step_kernels.size(); ++j) ran += cycle_step_kernels[j];
        count_launch(ran);
      }
      if (cycle == 0)
        for (int i = 0; i < count; ++i) iters_prev[i] = hsc[16 * i + SC_ITERS];
      else if (!tev.empty())
        collect_phase_times();
      int remaining = 0;
      for (int i = 0; i < count; ++i) {
        done[i] = hsc[16 * i + SC_DONE] != 0.0 || hsc[16 * i + SC_FLAGS] != 0.0;
        if (!done[i]) ++remaining;
      }
      if (remaining == 0 || cycle == max_cycles) break;
      for (int i = 0; i < count; ++i) {
        hflags[i] = done[i] ? 0 : 1;
        hflags[count + i] = hflags[i];
        in_cycle[i] = hflags[i];
        if (!done[i]) ++cycles[i];
      }
      TS_CUDA(cudaMemcpyAsync(flags, hflags.data(), sizeof(int) * 2 * count, cudaMemcpyHostToDevice, st));
      TS_CUDA(cudaStreamSynchronize(st));
      if (!exec) {
        const auto build_t0 = std::chrono::steady_clock::now();
        if (mixed) preload_cycle_kernels<float, float2>();
        else preload_cycle_kernels<double, double2>();
        CountSuppress no_count;   // the replays below count the recorded kernels
        auto build = [&](auto* Vt, auto* Xht) -> cudaGraph_t {
          using TT = std::remove_pointer_t<decltype(Vt)>;
          using R2 = std::remove_pointer_t<decltype(Xht)>;
          const CycleRecorder<TT, R2, decltype(inner_products), decltype(residual_products)> rec{
              d, plan, Vt, (TT*)W, Xht, (R2*)Yh, R, Xh64, Yh64, P0, P1, Pt, inner_products, residual_products,
              tev.empty() ? nullptr : tev.data()};
          if (tev.empty()) {
            // statistics off: nested conditional steps, so a cycle stops once no instance iterates
            NestedCycleCounts cnt;
            cudaGraph_t g = build_nested_cycle(
                m, st, [&](cudaStream_t q) { return rec.prologue(q); },
                [&](int j, cudaGraphConditionalHandle next, cudaStream_t q) { return rec.step(j, next, q); },
                [&](cudaStream_t q) { return rec.epilogue(q); }, cnt);
            cycle_fixed_kernels = cnt.prologue + cnt.epilogue;
            cycle_step_kernels = cnt.steps;
            return g;
          }
          // statistics on: one flat graph (event records are not allowed inside conditional bodies)
          cudaGraph_t g;
          TS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
          try {
            long long k = rec.prologue(st);
            cycle_step_kernels.clear();
            for (int j = 0; j < m; ++j) cycle_step_kernels.push_back(rec.step(j, 0, st));
            k += rec.epilogue(st);
            cycle_fixed_kernels = k;
          } catch (...) {
            cudaGraph_t dropped = nullptr;
            cudaStreamEndCapture(st, &dropped);
            if (dropped) cudaGraphDestroy(dropped);
            throw;
          }
          TS_CUDA(cudaStreamEndCapture(st, &g));
          return g;
        };
        cudaGraph_t graph = mixed ? build((float*)V, (float2*)Xh) : build((double*)V, (double2*)Xh);
        nested_graph = tev.empty();
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TS_CUDA(ie);
        ctx->timer.graph_build_ms += host_ms_since(build_t0);
      }
      TS_CUDA(cudaGraphLaunch(exec, st));
      ++launched;
    }
  } catch (...) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    throw;
  }
  TS_CUDA(cudaEventRecord(t1, st));
  TS_CUDA(cudaEventSynchronize(t1));
  ctx->timer.host_cycles_ms += host_ms_since(cycles_t0);
  float ms = 0.f;
  TS_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  if (exec) TS_CUDA(cudaGraphExecDestroy(exec));
  if (ozaki || tcin) {
    int e = 0;
    TS_CUDA(cudaMemcpy(&e, tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
      TS_CUDA(cudaEventDestroy(t0));
      TS_CUDA(cudaEventDestroy(t1));
      throw Error{TS_ERR_TIMEOUT, "tensor-core kernel wait expired (code " + std::to_string(e) + ")"};
    }
  }
  TS_CUDA(cudaEventDestroy(t0));
  TS_CUDA(cudaEventDestroy(t1));
  TS_CUDA(cudaEventRecord(ctx->ev1, st));
  TS_CUDA(cudaStreamWaitEvent(user, ctx->ev1, 0));
  for (int i = 0; i < count; ++i) {
    const double* s = hsc.data() + 16 * i;
    ts_status sti = TS_NOT_CONVERGED;
    if (s[SC_FLAGS] != 0.0 || !std::isfinite(s[SC_RES])) sti = TS_ERR_NONFINITE;
    else if (s[SC_DONE] != 0.0) sti = TS_OK;
    if (statuses) statuses[i] = sti;
    if (sti != TS_OK && overall == TS_OK) overall = sti == TS_ERR_NONFINITE ? TS_ERR_NONFINITE : TS_NOT_CONVERGED;
    if (infos) {
      ts_solve_info inf{};
      inf.iters = (int)s[SC_ITERS];
      inf.cycles = cycles[i];
      inf.outer = mixed ? cycles[i] : 0;
      inf.applies_fp64 = 1 + cycles[i] + (mixed ? 0 : inf.iters);
      inf.applies_low = mixed ? inf.iters : 0;
      inf.normC = s[SC_NORMC];
      inf.relres_true = s[SC_NORMC] > 0 ? s[SC_RES] / s[SC_NORMC] : s[SC_RES];
      inf.relres_est = s[SC_NORMC] > 0 ? s[SC_EST] / s[SC_NORMC] : s[SC_EST];
      inf.ms_total = ms;
      infos[i] = inf;
    }
  }
  (void)launched;
  return overall;
}

}  // namespace ts
