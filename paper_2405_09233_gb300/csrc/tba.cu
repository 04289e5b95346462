// Tubal Block Arnoldi (Algorithm 7) and TBAS(m) (Algorithm 8), and t-Bartels-Stewart
// (Algorithm 5), on one GB300 in FP64.
//
// Everything runs in the Fourier domain (Eq. (5)): the T-product decouples into K = p/2 + 1
// independent complex slices, the T-transpose becomes the conjugate transpose of each slice, and
// a tube becomes one complex number per slice.  So, slice by slice:
//   * Tubal-QR (Algorithm 6) of a full-rank n x s block is the thin QR with a positive real
//     diagonal -- unique, whatever algorithm computes it.  It is computed by CholeskyQR2 (Gram
//     matrix, small Cholesky, triangular multiply, twice), which keeps the work in GEMM-shaped
//     passes; slices of a (nearly) rank-deficient block run Algorithm 6's Gram-Schmidt with the
//     Normalize tie-break instead.
//   * The block MGS step H_ij = V_i^H W, W -= V_i H_ij is a tall-skinny Gram and an update.
//   * The projected equation H_m Y - Y B = C1 (Eq. (46)) is solved per slice by Hessenberg-Schur
//     (small_complex.cu) and X += V_m Y.
// Block vectors are stored slice by slice as row-major n x s complex matrices, so that a warp
// reading one row of V reads s contiguous entries: the sparse A_k V product (one warp per row,
// union CSR pattern of all frontal slices, complex values per slice), the Gram and the updates are
// all coalesced.  Norms use Parseval: ||X||^2 = (1/p) sum_k w_k ||X_k||^2, w = 1 for k = 0 and
// k = p/2, 2 otherwise.
#include <algorithm>
#include <cmath>
#include <vector>
#include <type_traits>
#include "internal.cuh"
#include "apply.cuh"
#include "reduce.cuh"
#include "tba.cuh"

namespace ts {
void ensure_f32_operator(ts_op* op, cudaStream_t st);  // lowprec.cu
namespace {

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c, FP32
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
template <typename C2> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };
__device__ __forceinline__ double2 to_c2(double2 v, double2*) { return v; }
__device__ __forceinline__ float2 to_c2(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 widen(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double slice_weight(int k, int p) {
  return (k == 0 || (p % 2 == 0 && k == p / 2)) ? 1.0 : 2.0;
}

constexpr int kMaxS = 64;           // block width supported by the row kernels

// C2: double2 (FP64), or float2 for the FP32 inner cycle of mixed-precision TBAS (MODE 0 only).
template <typename C2>
struct RowsArgsT {
  const int* rowptr;      // sparse pattern (nullptr: dense A_k column-major in Ad)
  const int* col;
  const C2* vals;         // K x nnz
  const C2* Ad;           // K x n x n column-major (dense operator)
  long long nnz;
  const C2* V;            // K x n x s row-major
  const double2* Brow;    // K x s x s row-major (B_k)
  const double2* C;       // K x n x s row-major (residual mode)
  C2* Out;                // K x n x s row-major
  double* partials;       // residual mode: one per block
  int n, s, K, p;
};
using RowsArgs = RowsArgsT<double2>;

// MODE 0: Out = A_k V_k.  MODE 1: Out = A_k V_k - V_k B_k.  MODE 2: Out = C_k - (A_k V_k - V_k B_k)
// and partials of the Parseval-weighted squared norm.
// Lane layout: LT = 1 (s <= 32): the warp's lanes form groups of sp = s rounded up to a power of two,
// one group per row and one lane per column, so a warp works on 32 / sp rows at once (an idle
// FP64 lane costs as much as a busy one); LT = 2 (32 < s <= 64): one row per warp, two columns per
// lane.
template <int MODE, int LT, typename C2>
__global__ void __launch_bounds__(256) k_sylv_rows(RowsArgsT<C2> a) {
  static_assert(MODE == 0 || sizeof(C2) == 16, "the operator with B_k and the residual run in FP64");
  const int k = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int sp = 32;
  if (LT == 1)
    while (sp / 2 >= a.s && sp > 1) sp /= 2;
  const int rpw = 32 / sp;                       // rows per warp
  const int sub = lane / sp, jl = lane % sp;
  const long long ns = (long long)a.n * a.s;
  const C2* Vk = a.V + k * ns;
  double local = 0.0;
  const int rows_step = gridDim.x * 8 * rpw;
  for (int ibase = (blockIdx.x * 8 + warp) * rpw; ibase < a.n; ibase += rows_step) {
    const int i = ibase + sub;
    const bool live = i < a.n;
    C2 acc[LT];
#pragma unroll
    for (int t = 0; t < LT; ++t) acc[t] = C2{0, 0};
    if (live) {
      if (a.rowptr) {
        const C2* vk = a.vals + (long long)k * a.nnz;
        for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
          const C2 av = vk[q];
          const C2* vr = Vk + (long long)a.col[q] * a.s;
#pragma unroll
          for (int t = 0; t < LT; ++t) {
            const int j = jl + 32 * t;
            if (j < a.s) acc[t] = cfma(av, vr[j], acc[t]);
          }
        }
      } else {
        const C2* Ak = a.Ad + (long long)k * a.n * a.n;
        for (int l = 0; l < a.n; ++l) {
          const C2 av = Ak[(long long)l * a.n + i];
          const C2* vr = Vk + (long long)l * a.s;
#pragma unroll
          for (int t = 0; t < LT; ++t) {
            const int j = jl + 32 * t;
            if (j < a.s) acc[t] = cfma(av, vr[j], acc[t]);
          }
        }
      }
      if constexpr (MODE >= 1) {
        const double2* Bk = a.Brow + (long long)k * a.s * a.s;
        const double2* xr = Vk + (long long)i * a.s;
        for (int l = 0; l < a.s; ++l) {
          const double2 xv = xr[l];
          const double2 nx = make_double2(-xv.x, -xv.y);
#pragma unroll
          for (int t = 0; t < LT; ++t) {
            const int j = jl + 32 * t;
            if (j < a.s) acc[t] = cfma(nx, Bk[(long long)l * a.s + j], acc[t]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < LT; ++t) {
        const int j = jl + 32 * t;
        if (j < a.s) {
          C2 v = acc[t];
          const long long o = k * ns + (long long)i * a.s + j;
          if constexpr (MODE == 2) {
            const double2 c = a.C[o];
            v = make_double2(c.x - v.x, c.y - v.y);
            local += v.x * v.x + v.y * v.y;
          }
          a.Out[o] = v;
        }
      }
    }
  }
  if (MODE == 2) {
    const double tot = block_sum(local) * slice_weight(k, a.p) / a.p;
    if (threadIdx.x == 0) a.partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

// Partial Gram matrices G_k = V_k^H W_k over row chunks: partials[(k*chunks + c)*s*s + a + s*b].
// Gauss's three-multiplication form: with u = conj(v), u w = (T1 - T3) + i (T1 + T2) where
// T1 = sum w_re (u_re + u_im), T2 = sum u_re (w_im - w_re), T3 = sum u_im (w_re + w_im); the sums
// of the factors are formed once per entry while staging, so a complex multiply-add costs three
// DFMA.  Each thread owns a 4 x 4 block of G; min(256 / (s/4)^2, 16) row groups split a staged row
// batch and are summed in shared memory at the end.
// C2 = float2: FP32 inputs and accumulation (the inner cycle of mixed-precision TBAS); the partial
// Grams are written in FP64 either way.
template <typename C2>
__global__ void __launch_bounds__(256) k_gram(const C2* __restrict__ V, const C2* __restrict__ W, int n, int s,
                                              int rows_per_chunk, double2* __restrict__ partials) {
  using R = typename RealOf<C2>::T;
  constexpr int RB = 16;                                 // rows staged per batch
  const int k = blockIdx.y, chunk = blockIdx.x, chunks = gridDim.x;
  // staged planes: u_re, u_im, u_re + u_im of V; w_re, w_im - w_re, w_re + w_im of W (one array, so
  // the final reduction can reuse it as one contiguous buffer)
  __shared__ R stage[6][RB][kMaxS];
  R (*vp1)[kMaxS] = stage[0];
  R (*vp2)[kMaxS] = stage[1];
  R (*vp3)[kMaxS] = stage[2];
  R (*wq1)[kMaxS] = stage[3];
  R (*wq2)[kMaxS] = stage[4];
  R (*wq3)[kMaxS] = stage[5];
  const long long ns = (long long)n * s;
  const C2* Vk = V + k * ns;
  const C2* Wk = W + k * ns;
  const int sg = (s + 3) / 4;                            // 4-wide groups per side
  const int tiles = sg * sg;
  // Row groups (>= 1 since s <= 64), at most one per staged row: more would sit idle and lengthen
  // the serial group reduction below, whose FP64 adds are expensive on this part.
  const int groups = min((int)blockDim.x / tiles, RB);
  const int t = threadIdx.x % tiles, grp = threadIdx.x / tiles;
  const int a0 = (t % sg) * 4, b0 = (t / sg) * 4;
  const bool live = grp < groups;
  R T1[4][4], T2[4][4], T3[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) T1[x][y] = T2[x][y] = T3[x][y] = R(0);
  const int r_begin = chunk * rows_per_chunk;
  const int r_end = min(n, r_begin + rows_per_chunk);
  for (int r0 = r_begin; r0 < r_end; r0 += RB) {
    for (int e = threadIdx.x; e < RB * kMaxS; e += blockDim.x) {
      const int rr = e / kMaxS, cc = e % kMaxS;
      const int r = r0 + rr;
      C2 v{0, 0}, w{0, 0};
      if (r < r_end && cc < s) {
        v = Vk[(long long)r * s + cc];
        w = Wk[(long long)r * s + cc];
      }
      vp1[rr][cc] = v.x;
      vp2[rr][cc] = -v.y;
      vp3[rr][cc] = v.x - v.y;
      wq1[rr][cc] = w.x;
      wq2[rr][cc] = w.y - w.x;
      wq3[rr][cc] = w.x + w.y;
    }
    __syncthreads();
    if (live) {
      for (int rr = grp; rr < RB; rr += groups) {
        R p1[4], p2[4], p3[4], q1[4], q2[4], q3[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int a = min(a0 + x, kMaxS - 1), b = min(b0 + x, kMaxS - 1);
          p1[x] = vp1[rr][a];
          p2[x] = vp2[rr][a];
          p3[x] = vp3[rr][a];
          q1[x] = wq1[rr][b];
          q2[x] = wq2[rr][b];
          q3[x] = wq3[rr][b];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            T1[x][y] = fma(q1[y], p3[x], T1[x][y]);
            T2[x][y] = fma(p1[x], q2[y], T2[x][y]);
            T3[x][y] = fma(p2[x], q3[y], T3[x][y]);
          }
      }
    }
    __syncthreads();
  }
  const int ss = s * s;
  double2* Pk = partials + ((long long)k * chunks + chunk) * ss;
  if (groups == 1) {
    if (live) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if (a0 + x < s && b0 + y < s)
            Pk[(a0 + x) + s * (b0 + y)] =   // combined in R, one conversion per part
                make_double2((double)(T1[x][y] - T3[x][y]), (double)(T1[x][y] + T2[x][y]));
    }
    return;
  }
  // Several row groups (then s <= 44, so 2 s^2 doubles fit in the staging arrays): sum them in a
  // fixed order through shared memory.
  R* red = &stage[0][0][0];
  for (int g = 0; g < groups; ++g) {
    if (live && grp == g) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int a = a0 + x, b = b0 + y;
          if (a < s && b < s) {
            const R re = T1[x][y] - T3[x][y], im = T1[x][y] + T2[x][y];
            const int e = a + s * b;
            if (g == 0) {
              red[2 * e] = re;
              red[2 * e + 1] = im;
            } else {
              red[2 * e] += re;
              red[2 * e + 1] += im;
            }
          }
        }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < ss; e += blockDim.x) Pk[e] = make_double2((double)red[2 * e], (double)red[2 * e + 1]);
}

// out_k (column-major, leading dimension ldo) = sum over chunks of the partial Grams (fixed order).
__global__ void k_gram_reduce(const double2* __restrict__ partials, int chunks, int s, double2* __restrict__ out,
                              long long sOut, int ldo) {
  const int k = blockIdx.x;
  const int ss = s * s;
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < chunks; ++c) {
      const double2 v = partials[((long long)k * chunks + c) * ss + e];
      acc.x += v.x;
      acc.y += v.y;
    }
    out[(long long)k * sOut + (e % s) + (long long)ldo * (e / s)] = acc;
  }
}

// Out_k = (accumulate ? Out_k : 0) + alpha * In_k M_k (in place allowed), M_k an s x s column-major
// block with leading dimension ldm.  kRowCols consecutive columns of one row per thread, all
// threads of a row in one warp; Gauss's form with the planes M_re, M_im - M_re, M_re + M_im of M_k in
// shared memory: Re = T1 - T3, Im = T1 + T2 with T1 = sum (a_re + a_im) m_re, T2 = sum a_re (m_im - m_re),
// T3 = sum a_im (m_re + m_im), three DFMA per complex multiply-add.
// Cin = float2 (the FP32 basis of mixed-precision TBAS): products in FP32; Cout may be double2 (the
// FP64 solution update X += V Y) or float2.
constexpr int kRowCols = 8;
template <typename Cin, typename Cout>
__global__ void __launch_bounds__(256) k_rows_mm(const Cin* In, Cout* Out, const double2* __restrict__ M,
                                                 long long sM, int ldm, int n, int s, double alpha, int accumulate) {
  using R = typename RealOf<Cin>::T;
  const int k = blockIdx.y;
  extern __shared__ unsigned char smm_raw[];   // three s x s planes, l-major: plane[l * s + j]
  R* mr = reinterpret_cast<R*>(smm_raw);
  R* md = mr + s * s;
  R* mq = mr + 2 * s * s;
  const double2* Mk = M + (long long)k * sM;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int l = e % s, j = e / s;
    const double2 v = Mk[l + (long long)ldm * j];
    mr[l * s + j] = (R)v.x;
    md[l * s + j] = (R)(v.y - v.x);
    mq[l * s + j] = (R)(v.x + v.y);
  }
  __syncthreads();
  // Threads per row: a power of two (1, 2, 4, 8), so a row never straddles two warps.
  int tpr = 1;
  while (tpr * kRowCols < s) tpr *= 2;
  const int cpt = (s + tpr - 1) / tpr;                   // columns per thread (<= kRowCols)
  const int rows_per_block = blockDim.x / tpr;
  const int rloc = threadIdx.x / tpr, cg = threadIdx.x % tpr;
  const int c0 = cg * cpt;
  const int c1 = min(c0 + cpt, s);
  const long long ns = (long long)n * s;
  const bool live_thread = rloc < rows_per_block;
  for (int rbase = blockIdx.x * rows_per_block; rbase < n; rbase += gridDim.x * rows_per_block) {
    const int i = rbase + rloc;
    const bool live = live_thread && i < n;
    R T1[kRowCols], T2[kRowCols], T3[kRowCols];
#pragma unroll
    for (int c = 0; c < kRowCols; ++c) T1[c] = T2[c] = T3[c] = R(0);
    const long long ro = k * ns + (long long)i * s;
    if (live) {
      for (int l = 0; l < s; ++l) {
        const Cin a = In[ro + l];
        const R sa = a.x + a.y;
#pragma unroll
        for (int c = 0; c < kRowCols; ++c) {
          const int j = min(c0 + c, c1 - 1);
          T1[c] = fma(sa, mr[l * s + j], T1[c]);
          T2[c] = fma(a.x, md[l * s + j], T2[c]);
          T3[c] = fma(a.y, mq[l * s + j], T3[c]);
        }
      }
    }
    __syncwarp();   // every thread of the row has read In before any writes Out (in place)
    if (live) {
#pragma unroll
      for (int c = 0; c < kRowCols; ++c) {
        const int j = c0 + c;
        if (j < c1) {
          if constexpr (sizeof(R) == 4) {
            // FP32 products: scale in FP32 and convert at most once, since GB300's FP64 and
            // conversion rate would otherwise make this epilogue cost more than the s-term loop
            const float al = (float)alpha;
            const float vr = al * (T1[c] - T3[c]), vi = al * (T1[c] + T2[c]);
            if constexpr (sizeof(Cout) == 8) {
              float2 v = make_float2(vr, vi);
              if (accumulate) {
                const float2 o = Out[ro + j];
                v.x += o.x;
                v.y += o.y;
              }
              Out[ro + j] = v;
            } else {
              double2 v = make_double2((double)vr, (double)vi);
              if (accumulate) {
                const double2 o = widen(Out[ro + j]);
                v.x += o.x;
                v.y += o.y;
              }
              Out[ro + j] = to_c2(v, (Cout*)nullptr);
            }
          } else {
            double2 v = make_double2(alpha * (double)(T1[c] - T3[c]), alpha * (double)(T1[c] + T2[c]));
            if (accumulate) {
              const double2 o = widen(Out[ro + j]);
              v.x += o.x;
              v.y += o.y;
            }
            Out[ro + j] = to_c2(v, (Cout*)nullptr);
          }
        }
      }
    }
  }
}

// Inverse of an upper triangular s x s matrix per slice (one warp; lanes over columns).
__global__ void k_triinv(const double2* __restrict__ Rall, double2* __restrict__ Xall, int s) {
  const double2* R = Rall + (long long)blockIdx.x * s * s;
  double2* X = Xall + (long long)blockIdx.x * s * s;
  for (int b = threadIdx.x; b < s; b += 32) {
    for (int a = 0; a < s; ++a) X[a + (long long)s * b] = make_double2(0.0, 0.0);
    // X[b][b] = 1 / R[b][b] (R has a real positive diagonal)
    X[b + (long long)s * b] = make_double2(1.0 / R[b + (long long)s * b].x, 0.0);
    for (int a = b - 1; a >= 0; --a) {
      double2 acc = make_double2(0.0, 0.0);
      for (int c = a + 1; c <= b; ++c) acc = cfma(R[a + (long long)s * c], X[c + (long long)s * b], acc);
      const double inv = 1.0 / R[a + (long long)s * a].x;
      X[a + (long long)s * b] = make_double2(-acc.x * inv, -acc.y * inv);
    }
  }
}

// Algorithm 6 with Normalization1 on the Fourier slices whose first Cholesky pivot showed a (nearly)
// rank-deficient block (fail[k] = 1; other slices return at once): modified Gram-Schmidt over the s
// columns of W_k (row-major n x s, in place -> Q_k), r_ij = q_i^H w_j, w_j -= q_i r_ij, then
// a = ||w_j||.  Column j counts as zero in this slice when a <= tiny * ref_j, ref_j the largest norm of
// column j over all K slices before orthogonalisation (the square root of max_k G_k(j, j), G the Gram
// of the original block); then r_jj = 0 and q_j is the first unit vector e_i whose component
// orthogonal to q_0..q_{j-1} has squared norm >= 1/(2n), orthogonalised twice (classical
// Gram-Schmidt) and normalised.  Writes R_k (upper triangular, column-major) to R and the identity to
// Rinv, so the CholeskyQR2 steps that follow leave the slice as it is.  One CTA per slice; rows are
// strided over the threads (each thread only reads back the rows it wrote, so the block reductions
// are the only synchronisation needed).  A fallback for rare blocks: columns are read with stride s.
template <typename C2>
__global__ void __launch_bounds__(256) k_tubal_mgs(C2* __restrict__ W, const double2* __restrict__ G,
                                                   const int* __restrict__ fail, double2* __restrict__ R,
                                                   double2* __restrict__ Rinv, int n, int s, int K, double tiny) {
  const int k = blockIdx.x;
  if (!fail[k]) return;
  __shared__ double2 coef[kMaxS];
  const long long ns = (long long)n * s;
  C2* Wk = W + k * ns;
  double2* Rk = R + (long long)k * s * s;
  double2* Ik = Rinv + (long long)k * s * s;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    Rk[e] = make_double2(0.0, 0.0);
    Ik[e] = make_double2(e % s == e / s ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  auto ld = [&](int r, int c) { return widen(Wk[(long long)r * s + c]); };
  auto st = [&](int r, int c, double2 v) { Wk[(long long)r * s + c] = to_c2(v, (C2*)nullptr); };
  for (int j = 0; j < s; ++j) {
    double ref2 = 0.0;
    for (int q = 0; q < K; ++q) ref2 = fmax(ref2, G[(long long)q * s * s + j + (long long)s * j].x);
    for (int i = 0; i < j; ++i) {                       // r_ij = q_i^H w_j; w_j -= q_i r_ij
      double re = 0.0, im = 0.0;
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 q = ld(r, i), w = ld(r, j);
        re += q.x * w.x + q.y * w.y;
        im += q.x * w.y - q.y * w.x;
      }
      re = block_sum(re);
      im = block_sum(im);
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 q = ld(r, i), w = ld(r, j);
        st(r, j, make_double2(w.x - (q.x * re - q.y * im), w.y - (q.x * im + q.y * re)));
      }
      if (threadIdx.x == 0) Rk[i + (long long)s * j] = make_double2(re, im);
    }
    double a2 = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const double2 w = ld(r, j);
      a2 += w.x * w.x + w.y * w.y;
    }
    const double a = sqrt(block_sum(a2));
    if (a > tiny * sqrt(ref2)) {                        // Normalize: q_j = w_j / a, r_jj = a
      const double inv = 1.0 / a;
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 w = ld(r, j);
        st(r, j, make_double2(w.x * inv, w.y * inv));
      }
      if (threadIdx.x == 0) Rk[j + (long long)s * j] = make_double2(a, 0.0);
      continue;
    }
    // rank-deficient slice of column j: r_jj = 0 (already), q_j = a unit vector orthogonal to q_<j
    for (int e = 0; e < n; ++e) {
      for (int r = threadIdx.x; r < n; r += blockDim.x) st(r, j, make_double2(r == e ? 1.0 : 0.0, 0.0));
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < j; ++i) {                   // c_i = q_i^H z for every i first (classical)
          double re = 0.0, im = 0.0;
          for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const double2 q = ld(r, i), z = ld(r, j);
            re += q.x * z.x + q.y * z.y;
            im += q.x * z.y - q.y * z.x;
          }
          re = block_sum(re);
          im = block_sum(im);
          if (threadIdx.x == 0) coef[i] = make_double2(re, im);
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
          double2 z = ld(r, j);
          for (int i = 0; i < j; ++i) {
            const double2 q = ld(r, i), c = coef[i];
            z.x -= q.x * c.x - q.y * c.y;
            z.y -= q.x * c.y + q.y * c.x;
          }
          st(r, j, z);
        }
        __syncthreads();                                // coef is rewritten by the next pass
      }
      double z2 = 0.0;
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 z = ld(r, j);
        z2 += z.x * z.x + z.y * z.y;
      }
      z2 = block_sum(z2);
      if (z2 >= 0.5 / n) {
        const double inv = 1.0 / sqrt(z2);
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
          const double2 z = ld(r, j);
          st(r, j, make_double2(z.x * inv, z.y * inv));
        }
        break;
      }
    }
  }
}

// Column-major spectral [k][j][i] <-> row-major [k][i][j], 32 x 32 tiles.
__global__ void k_spec_transpose(const double2* __restrict__ in, double2* __restrict__ out, int rows, int cols) {
  // in: K x (cols x rows) with rows fastest; out: K x (rows x cols) with cols fastest
  __shared__ double2 tile[32][33];
  const int k = blockIdx.z;
  const long long off = (long long)k * rows * cols;
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + threadIdx.x, c = c0 + q;
    if (r < rows && c < cols) tile[q][threadIdx.x] = in[off + (long long)c * rows + r];
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + q, c = c0 + threadIdx.x;
    if (r < rows && c < cols) out[off + (long long)r * cols + c] = tile[threadIdx.x][q];
  }
}

// sum_k w_k/p * (squared Frobenius norm of the s x s block k of E) -> out[0]; traces of G -> out.
__global__ void k_weighted_fro(const double2* __restrict__ E, int s, int K, int p, double* out) {
  double local = 0.0;
  for (int e = threadIdx.x; e < K * s * s; e += blockDim.x) {
    const int k = e / (s * s);
    const double2 v = E[e];
    local += (v.x * v.x + v.y * v.y) * slice_weight(k, p) / p;
  }
  const double tot = block_sum(local);
  if (threadIdx.x == 0) out[0] = tot;
}

__global__ void k_weighted_trace(const double2* __restrict__ G, int s, int K, int p, double* out) {
  double local = 0.0;
  for (int e = threadIdx.x; e < K * s; e += blockDim.x) {
    const int k = e / s, d = e % s;
    local += G[(long long)k * s * s + d + (long long)s * d].x * slice_weight(k, p) / p;
  }
  const double tot = block_sum(local);
  if (threadIdx.x == 0) out[0] = tot;
}

__global__ void k_fill_c1(const double2* __restrict__ H0, double2* __restrict__ C1, int s, int N, int K) {
  // C1_k = [H0_k; 0] (N x s column-major)
  const long long tot = (long long)K * N * s;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / ((long long)N * s));
    const long long r = e % ((long long)N * s);
    const int i = (int)(r % N), j = (int)(r / N);
    C1[e] = i < s ? H0[(long long)k * s * s + i + (long long)s * j] : make_double2(0.0, 0.0);
  }
}

// B_k (column-major) -> row-major copy.
__global__ void k_row_major_small(const double2* __restrict__ B, double2* __restrict__ Br, int s, int K) {
  const long long tot = (long long)K * s * s;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / ((long long)s * s));
    const long long r = e % ((long long)s * s);
    const int row = (int)(r / s), colj = (int)(r % s);
    Br[e] = B[(long long)k * s * s + row + (long long)s * colj];
  }
}

int grid1d(long long work) {
  long long g = (work + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

struct TbaWork {
  int n, s, p, K, m;
  long long blk;            // K * n * s
  double2* V;               // (m + 1) blocks
  double2* X;               // spectral X, row-major
  double2* C;               // spectral C, row-major
  double2* R;               // spectral residual
  double2* tmp;             // column-major spectral scratch
  double2* Hm;              // K x (ms x ms) column-major
  double2* H0;              // K x s x s
  double2* Hlast;           // K x s x s
  double2* G;               // K x s x s (Gram / Cholesky scratch)
  double2* R1;              // K x s x s
  double2* Rinv;            // K x s x s
  double2* R2;              // K x s x s
  double2* gram_part;       // partial Grams
  int chunks, rows_per_chunk;
  double2* LU;              // K x s x N x N
  int* piv;                 // K x s x N
  double2* Gp;              // K x N x s
  double2* Z;               // K x N x s
  double2* Y;               // K x N x s
  double2* E;               // K x s x s
  double* P;                // kRedBlocks partials
  double* sc;               // scalars
  int* err;                 // error bits
  int* fail;                // K flags: slices whose Tubal-QR took the Gram-Schmidt fallback
  KernelTimer* tm;          // per-kernel timing (kind 4: tubal Gram and block products)
};

}  // namespace

void SparseOp::release() {
  op_free(rowptr);
  op_free(col);
  op_free(vals);
  op_free(vals32);
  rowptr = col = nullptr;
  vals = nullptr;
  vals32 = nullptr;
}

void ensure_b_schur(ts_ctx* ctx, ts_op* op, cudaStream_t st) {
  if (op->schurT) return;
  const int s = op->s, K = op->K;
  op_alloc(op->schurT, sizeof(double2) * (size_t)K * s * s);
  op_alloc(op->schurQ, sizeof(double2) * (size_t)K * s * s);
  TS_CUDA(cudaMemcpyAsync(op->schurT, op->Bh, sizeof(double2) * (size_t)K * s * s, cudaMemcpyDeviceToDevice, st));
  int* err = static_cast<int*>(ctx->ws.get("schur_err", sizeof(int)));
  TS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  schur_small(op->schurT, op->schurQ, s, K, err, st);
  int e = 0;
  TS_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  if (e) {
    op_free(op->schurT);
    op_free(op->schurQ);
    op->schurT = op->schurQ = nullptr;
    throw Error{TS_SINGULAR, "complex Schur iteration of B_k did not converge"};
  }
}

namespace {

// W = A_k V_k in FP32 (the inner cycle of mixed-precision TBAS); FP32 copies of the operator's
// values are made on first use.
void rows_call_f32(ts_op* op, const float2* V, float2* Out, int n, int s, int K, int p, cudaStream_t st) {
  RowsArgsT<float2> a{};
  if (op->sp) {
    SparseOp& sp = *op->sp;
    if (!sp.vals32) {
      op_alloc(sp.vals32, sizeof(float2) * (size_t)K * sp.nnz);
      convert<double, float>(reinterpret_cast<const double*>(sp.vals), reinterpret_cast<float*>(sp.vals32),
                             2ll * K * sp.nnz, st);
    }
    a.rowptr = sp.rowptr;
    a.col = sp.col;
    a.vals = sp.vals32;
    a.nnz = sp.nnz;
  } else {
    ensure_f32_operator(op, st);
    a.Ad = op->Ah32;
  }
  a.V = V;
  a.Out = Out;
  a.n = n;
  a.s = s;
  a.K = K;
  a.p = p;
  const bool wide = s > 32;
  int sp = 32;
  while (!wide && sp / 2 >= s && sp > 1) sp /= 2;
  const int rows_per_block = 8 * (32 / sp);
  const int gx = std::max(1, std::min((n + rows_per_block - 1) / rows_per_block, 2 * 152 * 4 / K));
  if (wide) k_sylv_rows<0, 2><<<dim3(gx, K), 256, 0, st>>>(a);
  else k_sylv_rows<0, 1><<<dim3(gx, K), 256, 0, st>>>(a);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void rows_call(int mode, const ts_op* op, const double2* V, const double2* C, double2* Out, double* partials, int n,
               int s, int K, int p, cudaStream_t st) {
  RowsArgs a{};
  if (op->sp) {
    a.rowptr = op->sp->rowptr;
    a.col = op->sp->col;
    a.vals = op->sp->vals;
    a.nnz = op->sp->nnz;
  } else {
    a.Ad = op->Ah;
  }
  a.V = V;
  a.Brow = op->Bh_row;
  a.C = C;
  a.Out = Out;
  a.partials = partials;
  a.n = n;
  a.s = s;
  a.K = K;
  a.p = p;
  const bool wide = s > 32;
  int sp = 32;
  while (!wide && sp / 2 >= s && sp > 1) sp /= 2;
  const int rows_per_block = 8 * (32 / sp);
#define TS_SYLV_ROWS(M, GX)                                                           \
  do {                                                                                \
    if (wide) k_sylv_rows<M, 2><<<dim3((GX), K), 256, 0, st>>>(a);                    \
    else k_sylv_rows<M, 1><<<dim3((GX), K), 256, 0, st>>>(a);                         \
  } while (0)
  if (mode == 2) {
    const int gx = kRedBlocks / K;
    TS_CUDA(cudaMemsetAsync(partials, 0, sizeof(double) * kRedBlocks, st));
    TS_SYLV_ROWS(2, gx);
  } else {
    const int gx = std::max(1, std::min((n + rows_per_block - 1) / rows_per_block, 2 * 152 * 4 / K));
    if (mode == 0) TS_SYLV_ROWS(0, gx);
    else TS_SYLV_ROWS(1, gx);
  }
#undef TS_SYLV_ROWS
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename Cin, typename Cout>
void rows_mm(const Cin* In, Cout* Out, const double2* M, long long sM, int ldm, int n, int s, int K, double alpha,
             bool accumulate, cudaStream_t st) {
  using R = typename RealOf<Cin>::T;
  TS_REQUIRE(s <= kMaxS, "rows_mm: block width above kMaxS");
  int tpr = 1;
  while (tpr * kRowCols < s) tpr *= 2;
  const int rows_per_block = 256 / tpr;
  const int gx = std::max(1, std::min((n + rows_per_block - 1) / rows_per_block, 4 * 152 * 4 / K));
  const size_t smem = sizeof(R) * 3 * (size_t)s * s;
  set_max_dynamic_smem((const void*)k_rows_mm<Cin, Cout>, (int)(sizeof(R) * 3 * kMaxS * kMaxS));
  k_rows_mm<Cin, Cout><<<dim3(gx, K), 256, smem, st>>>(In, Out, M, sM, ldm, n, s, alpha, accumulate ? 1 : 0);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

// Algorithmic FLOPs of one (n x s)^H (n x s) or (n x s)(s x s) complex product over K slices.
double block_flops(const TbaWork& w) { return 8.0 * w.n * w.s * w.s * w.K; }

template <typename C2>
void gram(const TbaWork& w, const C2* V, const C2* W, double2* out, long long sOut, int ldo, cudaStream_t st) {
  w.tm->begin(st, 4, block_flops(w));
  k_gram<C2><<<dim3(w.chunks, w.K), 256, 0, st>>>(V, W, w.n, w.s, w.rows_per_chunk, w.gram_part);
  count_launch();
  TS_CUDA(cudaGetLastError());
  k_gram_reduce<<<w.K, 256, 0, st>>>(w.gram_part, w.chunks, w.s, out, sOut, ldo);
  count_launch();
  TS_CUDA(cudaGetLastError());
  w.tm->end(st);
}

template <typename Cin, typename Cout>
void rows_mm_timed(const TbaWork& w, const Cin* In, Cout* Out, const double2* M, long long sM, int ldm,
                   double alpha, bool accumulate, cudaStream_t st) {
  w.tm->begin(st, 4, block_flops(w));
  rows_mm(In, Out, M, sM, ldm, w.n, w.s, w.K, alpha, accumulate, st);
  w.tm->end(st);
}

void triinv(const double2* R, double2* X, int s, int K, cudaStream_t st) {
  k_triinv<<<K, 32, 0, st>>>(R, X, s);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

// Tubal-QR of the block W (in place -> Q); R written to Rout (column-major, ldr).  Per Fourier slice
// the QR with a positive real diagonal is unique for a full-rank block, and CholeskyQR2 computes it
// in GEMM-shaped passes: G = W^H W, G = R1^H R1, W <- W R1^-1, again with R2, R = R2 R1.  A slice
// whose first Cholesky pivot says that a column is (nearly) dependent on the previous ones -- its
// orthogonal part below 1e-6 of its norm in FP64 (1e-3 in FP32), or its norm below the rank-deficiency
// scale of Normalization1 -- takes Algorithm 6 itself instead (k_tubal_mgs: Gram-Schmidt with the
// Normalize tie-break), whose Q the second CholeskyQR pass then only re-orthogonalises to rounding.
// Returns false when the second Cholesky fails (not expected after either first pass).
template <typename C2>
bool tubal_qr(const TbaWork& w, C2* W, double2* Rout, long long sR, int ldr, cudaStream_t st) {
  const int s = w.s, K = w.K;
  const long long ss = (long long)s * s;
  constexpr bool f64 = sizeof(C2) == 16;
  const double tiny = f64 ? 1e-12 : 1e-4;      // Normalization1: a slice is zero below tiny * ref_j
  const double rel = f64 ? 1e-12 : 1e-6;       // CholeskyQR is trusted for orthogonal parts above sqrt(rel)
  TS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  gram(w, W, W, w.G, ss, s, st);
  cholesky_small(w.G, w.R1, s, K, rel, tiny * tiny, nullptr, w.fail, st);
  triinv(w.R1, w.Rinv, s, K, st);
  k_tubal_mgs<C2><<<K, 256, 0, st>>>(W, w.G, w.fail, w.R1, w.Rinv, w.n, s, K, tiny);
  count_launch();
  TS_CUDA(cudaGetLastError());
  rows_mm_timed(w, W, W, w.Rinv, ss, s, 1.0, false, st);
  gram(w, W, W, w.G, ss, s, st);
  cholesky_small(w.G, w.R2, s, K, 0.0, 0.0, w.err, nullptr, st);
  triinv(w.R2, w.Rinv, s, K, st);
  rows_mm_timed(w, W, W, w.Rinv, ss, s, 1.0, false, st);
  small_gemm(w.R2, ss, s, w.R1, ss, s, false, Rout, sR, ldr, s, s, s, K, false, st);   // R = R2 R1
  int e = 0;
  TS_CUDA(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  return e == 0;
}

double read_scalar(const double* d, ts_ctx* ctx, cudaStream_t st) {
  TS_CUDA(cudaMemcpyAsync(ctx->host_scalars + 32, d, sizeof(double), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  return ctx->host_scalars[32];
}

double weighted_trace(const TbaWork& w, const double2* G, ts_ctx* ctx, cudaStream_t st) {
  k_weighted_trace<<<1, 256, 0, st>>>(G, w.s, w.K, w.p, w.sc);
  count_launch();
  TS_CUDA(cudaGetLastError());
  return read_scalar(w.sc, ctx, st);
}

// R = C - M(X) in the spectral row-major layout; returns ||R||_F (real space).
double residual(ts_ctx* ctx, const ts_op* op, const TbaWork& w, cudaStream_t st) {
  rows_call(2, op, w.X, w.C, w.R, w.P, w.n, w.s, w.K, w.p, st);
  finalize_norm(w.P, w.sc, st);
  return read_scalar(w.sc, ctx, st);
}

void to_rows(const double* real, double2* spec_rows, double2* tmp, int n, int s, int p, cudaStream_t st) {
  const int K = num_slices(p);
  rfft_tube<double, double2>(real, tmp, (long long)n * s, p, st);
  k_spec_transpose<<<dim3((n + 31) / 32, (s + 31) / 32, K), dim3(32, 8), 0, st>>>(tmp, spec_rows, n, s);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void from_rows(const double2* spec_rows, double* real, double2* tmp, int n, int s, int p, cudaStream_t st) {
  const int K = num_slices(p);
  // row-major (n x s) is column-major (s x n): transpose with rows = s, cols = n
  k_spec_transpose<<<dim3((s + 31) / 32, (n + 31) / 32, K), dim3(32, 8), 0, st>>>(spec_rows, tmp, s, n);
  count_launch();
  TS_CUDA(cudaGetLastError());
  irfft_tube<double, double2>(tmp, real, (long long)n * s, p, IRFFT_STORE, nullptr, nullptr, st);
}

void ensure_brow(ts_op* op, cudaStream_t st) {
  if (op->Bh_row) return;
  const size_t b = sizeof(double2) * (size_t)op->K * op->s * op->s;
  op_alloc(op->Bh_row, b);
  k_row_major_small<<<grid1d((long long)op->K * op->s * op->s), 256, 0, st>>>(op->Bh, op->Bh_row, op->s, op->K);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

TbaWork tba_work(ts_ctx* ctx, const ts_op* op, int m) {
  TbaWork w{};
  w.n = op->n; w.s = op->s; w.p = op->p; w.K = op->K; w.m = m;
  const int n = w.n, s = w.s, K = w.K, N = m * s;
  w.blk = (long long)K * n * s;
  const size_t blk = sizeof(double2) * (size_t)w.blk, ss = sizeof(double2) * (size_t)K * s * s;
  auto get = [&](const char* name, size_t bytes) { return ctx->ws.get(name, bytes); };
  w.V = (double2*)get("tba_V", blk * (m + 1));
  w.X = (double2*)get("tba_X", blk);
  w.C = (double2*)get("tba_C", blk);
  w.R = (double2*)get("tba_R", blk);
  w.tmp = (double2*)get("tba_tmp", blk);
  w.Hm = (double2*)get("tba_Hm", sizeof(double2) * (size_t)K * N * N);
  w.H0 = (double2*)get("tba_H0", ss);
  w.Hlast = (double2*)get("tba_Hlast", ss);
  w.G = (double2*)get("tba_G", ss);
  w.R1 = (double2*)get("tba_R1", ss);
  w.R2 = (double2*)get("tba_R2", ss);
  w.Rinv = (double2*)get("tba_Rinv", ss);
  w.chunks = std::max(1, std::min(2 * 152 / K, (n + 63) / 64));
  w.rows_per_chunk = (n + w.chunks - 1) / w.chunks;
  w.gram_part = (double2*)get("tba_gram_part", sizeof(double2) * (size_t)K * w.chunks * s * s);
  w.LU = (double2*)get("tba_LU", sizeof(double2) * (size_t)K * s * N * N);
  w.piv = (int*)get("tba_piv", sizeof(int) * (size_t)K * s * N);
  w.Gp = (double2*)get("tba_Gp", sizeof(double2) * (size_t)K * N * s);
  w.Z = (double2*)get("tba_Z", sizeof(double2) * (size_t)K * N * s);
  w.Y = (double2*)get("tba_Y", sizeof(double2) * (size_t)K * N * s);
  w.E = (double2*)get("tba_E", ss);
  w.P = (double*)get("tba_P", sizeof(double) * kRedBlocks);
  w.sc = (double*)get("tba_sc", sizeof(double) * 16);
  w.err = (int*)get("tba_err", sizeof(int) * 4);
  w.fail = (int*)get("tba_fail", sizeof(int) * (size_t)K);
  w.tm = &ctx->timer;
  return w;
}

ts_status tbas_solve(ts_ctx* ctx, ts_op* op, const double* C, double* X, const ts_solve_opts& o, ts_solve_info& info,
                     cudaStream_t st) {
  const int n = op->n, s = op->s, p = op->p, K = op->K, m = o.restart;
  TS_REQUIRE(s <= kMaxS, "ts_tba_solve: block width s must be <= 64");
  TS_REQUIRE((long long)m * s <= 12000, "ts_tba_solve: m*s too large for the projected solve");
  ensure_brow(op, st);
  ensure_b_schur(ctx, op, st);
  TbaWork w = tba_work(ctx, op, m);
  const long long ss = (long long)s * s;
  int hist_len = 0, true_len = 0;
  auto push_hist = [&](double v) {
    if (o.history && hist_len < o.history_cap) o.history[hist_len] = v;
    ++hist_len;
  };
  auto push_true = [&](double v) {
    if (o.true_history && true_len < o.true_history_cap) o.true_history[true_len] = v;
    ++true_len;
  };
  to_rows(C, w.C, w.tmp, n, s, p, st);
  to_rows(X, w.X, w.tmp, n, s, p, st);
  // ||C||^2 = (1/p) sum_k w_k trace(C_k^H C_k)  (Parseval)
  gram(w, w.C, w.C, w.G, ss, s, st);
  const double normC = std::sqrt(std::max(0.0, weighted_trace(w, w.G, ctx, st)));
  double res = residual(ctx, op, w, st);
  info.normC = normC;
  info.applies_fp64 = 1;
  push_true(res);
  double last_est = res;
  auto finish = [&](ts_status stt) {
    from_rows(w.X, X, w.tmp, n, s, p, st);
    TS_CUDA(cudaStreamSynchronize(st));
    info.history_len = hist_len;
    info.true_history_len = true_len;
    if (o.precision == TS_MIXED_FP32) info.outer = info.cycles;
    info.relres_true = normC > 0 ? res / normC : res;
    info.relres_est = normC > 0 ? last_est / normC : last_est;
    return stt;
  };
  if (!std::isfinite(res) || !std::isfinite(normC)) return finish(TS_ERR_NONFINITE);
  if (normC == 0.0 || res <= o.tol * normC) return finish(TS_OK);
  const long long blk = w.blk;
  // Mixed precision (TS_MIXED_FP32): the block Krylov basis, the SpMM and the block products of each
  // cycle run in FP32; the Gram results, H_m, the projected solve, X and the true residual of every
  // restart stay FP64, so the restarts are steps of iterative refinement.
  const bool low = o.precision == TS_MIXED_FP32;
  float2* V32 = low ? (float2*)ctx->ws.get("tba_V32", sizeof(float2) * (size_t)blk * (m + 1)) : nullptr;
  const double breakdown_rel = low ? 1e-6 : 1e-13;
  // Work of one A V_j product over all K slices: the kernel forms 8 FLOPs per stored complex value
  // and block column (dense A: n^2 values per slice); algorithmically it reads the values, the
  // pattern and V once and writes W once.
  const double a_vals = op->sp ? (double)op->sp->nnz : (double)n * n;
  const double spmm_flops = 8.0 * a_vals * s * K;
  auto spmm_bytes = [&](size_t c2) {
    return (double)K * a_vals * c2 + (op->sp ? 4.0 * (a_vals + n + 1) : 0.0) + 2.0 * (double)K * n * s * c2;
  };
  for (int cycle = 0; cycle < o.max_restarts; ++cycle) {
    const int N = m * s;
    int mm = m;
    // One Tubal Block Arnoldi cycle on the basis V (double2 or float2): V_1 = Tubal-QR(R0), W = A V_j,
    // block MGS, Tubal-QR of W.  Returns false on a failed Tubal-QR.
    auto arnoldi = [&](auto* V) -> bool {
      using C2 = std::remove_pointer_t<decltype(V)>;
      if constexpr (sizeof(C2) == 16) {
        TS_CUDA(cudaMemcpyAsync(V, w.R, sizeof(double2) * blk, cudaMemcpyDeviceToDevice, st));
      } else {
        convert<double, float>(reinterpret_cast<const double*>(w.R), reinterpret_cast<float*>(V), 2 * blk, st);
      }
      if (!tubal_qr(w, V, w.H0, ss, s, st)) return false;
      TS_CUDA(cudaMemsetAsync(w.Hm, 0, sizeof(double2) * (size_t)K * N * N, st));
      for (int j = 0; j < m; ++j) {
        C2* Vj = V + (long long)j * blk;
        C2* Wb = V + (long long)(j + 1) * blk;
        w.tm->begin(st, 5, spmm_flops, spmm_bytes(sizeof(C2)));
        if constexpr (sizeof(C2) == 16) {
          rows_call(0, op, Vj, nullptr, Wb, nullptr, n, s, K, p, st);          // W = A * V_j (A, not M)
          ++info.applies_fp64;
        } else {
          rows_call_f32(op, Vj, Wb, n, s, K, p, st);
          ++info.applies_low;
        }
        w.tm->end(st);
        for (int i = 0; i <= j; ++i) {                                          // block MGS
          C2* Vi = V + (long long)i * blk;
          double2* Hij = w.Hm + (long long)i * s + (long long)N * j * s;       // block (i, j) of H_m
          gram(w, Vi, Wb, Hij, (long long)N * N, N, st);
          rows_mm_timed(w, Vi, Wb, Hij, (long long)N * N, N, -1.0, true, st);
        }
        gram(w, Wb, Wb, w.G, ss, s, st);
        const double wn = std::sqrt(std::max(0.0, weighted_trace(w, w.G, ctx, st)));
        ++info.iters;
        if (wn <= breakdown_rel * res) {                                        // block breakdown
          mm = j + 1;
          TS_CUDA(cudaMemsetAsync(w.Hlast, 0, sizeof(double2) * (size_t)K * ss, st));
          break;
        }
        double2* Hnext = (j + 1 < m) ? w.Hm + (long long)(j + 1) * s + (long long)N * j * s : w.Hlast;
        const long long sH = (j + 1 < m) ? (long long)N * N : ss;
        const int ldh = (j + 1 < m) ? N : s;
        if (!tubal_qr(w, Wb, Hnext, sH, ldh, st)) return false;
      }
      return true;
    };
    if (!(low ? arnoldi(V32) : arnoldi(w.V))) return finish(TS_BREAKDOWN);
    const int Nm = mm * s;
    // Projected equation per slice: H_m Y - Y B = C1 = [H0; 0] by Hessenberg-Schur.
    // When the block space broke down early the leading Nm x Nm part of H_m is used.
    double2* Hproj = w.Hm;
    long long sHp = (long long)N * N;
    if (Nm != N) {
      double2* Hc = (double2*)ctx->ws.get("tba_Hcompact", sizeof(double2) * (size_t)K * Nm * Nm);
      for (int k = 0; k < K; ++k)
        TS_CUDA(cudaMemcpy2DAsync(Hc + (long long)k * Nm * Nm, sizeof(double2) * Nm, w.Hm + (long long)k * N * N,
                                  sizeof(double2) * N, sizeof(double2) * Nm, Nm, cudaMemcpyDeviceToDevice, st));
      Hproj = Hc;
      sHp = (long long)Nm * Nm;
    }
    k_fill_c1<<<grid1d((long long)K * Nm * s), 256, 0, st>>>(w.H0, w.Z, s, Nm, K);     // Z <- C1
    count_launch();
    TS_CUDA(cudaGetLastError());
    small_gemm(w.Z, (long long)Nm * s, Nm, op->schurQ, ss, s, false, w.Gp, (long long)Nm * s, Nm, Nm, s, s, K, false,
               st);                                                                     // G = C1 Q
    TS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    shifted_lu(Hproj, sHp, op->schurT, w.LU, w.piv, Nm, std::min(s, Nm - 1), s, K, w.err, st);
    hs_solve(w.LU, w.piv, w.Gp, op->schurT, w.Z, Nm, std::min(s, Nm - 1), s, K, st);
    small_gemm(w.Z, (long long)Nm * s, Nm, op->schurQ, ss, s, true, w.Y, (long long)Nm * s, Nm, Nm, s, s, K, false,
               st);                                                                     // Y = Z Q^H
    // Proposition 5.2 estimate ||H_{m+1,m} E_m Y||
    small_gemm(w.Hlast, ss, s, w.Y + (long long)(mm - 1) * s, (long long)Nm * s, Nm, false, w.E, ss, s, s, s, s, K,
               false, st);
    k_weighted_fro<<<1, 256, 0, st>>>(w.E, s, K, p, w.sc + 4);
    count_launch();
    TS_CUDA(cudaGetLastError());
    // X += V_m Y
    for (int j = 0; j < mm; ++j) {
      if (low)
        rows_mm(V32 + (long long)j * blk, w.X, w.Y + (long long)j * s, (long long)Nm * s, Nm, n, s, K, 1.0, true, st);
      else
        rows_mm(w.V + (long long)j * blk, w.X, w.Y + (long long)j * s, (long long)Nm * s, Nm, n, s, K, 1.0, true, st);
    }
    int e = 0;
    TS_CUDA(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    const double est = std::sqrt(std::max(0.0, read_scalar(w.sc + 4, ctx, st)));
    if (e & 2) return finish(TS_SINGULAR);
    last_est = est;
    push_hist(est);
    ++info.cycles;
    res = residual(ctx, op, w, st);
    ++info.applies_fp64;
    push_true(res);
    if (!std::isfinite(res)) return finish(TS_ERR_NONFINITE);
    if (res <= o.tol * normC) return finish(TS_OK);
  }
  return finish(TS_NOT_CONVERGED);
}

}  // namespace

ts_status tba_entry(ts_ctx* ctx, const ts_op* cop, const double* C, double* X, const ts_solve_opts* opts,
                    ts_solve_info* info_out, ts_stream stream) {
  ts_op* op = const_cast<ts_op*>(cop);
  TS_REQUIRE(op && C && X && opts, "ts_tba_solve: null pointer");
  const ts_solve_opts& o = *opts;
  TS_REQUIRE(o.restart >= 1 && o.restart <= 256, "ts_tba_solve: restart must be in 1..256");
  TS_REQUIRE(o.max_restarts >= 1, "ts_tba_solve: max_restarts must be >= 1");
  TS_REQUIRE(o.tol > 0.0 && std::isfinite(o.tol), "ts_tba_solve: tol must be positive");
  if (o.precision != TS_FP64 && o.precision != TS_MIXED_FP32)
    throw Error{TS_ERR_UNSUPPORTED, "TBAS runs in FP64 or TS_MIXED_FP32 only"};
  if (o.fp64_engine != TS_ENGINE_DFMA) throw Error{TS_ERR_UNSUPPORTED, "TBAS runs on the FP64 DFMA engine only"};
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ts_solve_info info{};
  TS_CUDA(cudaEventRecord(ctx->ev0, st));
  const size_t N = (size_t)op->n * op->s * op->p;
  StagedIn c(ctx, "solve_inC", C, N, st);
  StagedOut x(ctx, "solve_ioX", X, N, true, st);
  ts_status s = tbas_solve(ctx, op, c.dev, x.dev, o, info, st);
  x.finish();
  TS_CUDA(cudaEventRecord(ctx->ev1, st));
  TS_CUDA(cudaEventSynchronize(ctx->ev1));
  float ms = 0.f;
  TS_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  info.ms_total = ms;
  if (info_out) *info_out = info;
  return s;
}

// Dense operator apply for a sparse op (ts_sylv_apply / residuals): X real -> Y = M(X) real.
void apply_sparse_f64(ts_ctx* ctx, const ts_op* cop, const double* X, double* Y, cudaStream_t st) {
  ts_op* op = const_cast<ts_op*>(cop);
  ensure_brow(op, st);
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  TS_REQUIRE(s <= kMaxS, "sparse operator: s must be <= 64");
  const size_t blk = sizeof(double2) * (size_t)K * n * s;
  double2* a = (double2*)ctx->ws.get("sp_a", blk);
  double2* b = (double2*)ctx->ws.get("sp_b", blk);
  double2* t = (double2*)ctx->ws.get("sp_t", blk);
  to_rows(X, a, t, n, s, p, st);
  rows_call(1, op, a, nullptr, b, nullptr, n, s, K, p, st);
  from_rows(b, Y, t, n, s, p, st);
}

// t-Bartels-Stewart (Algorithm 5) for small dense A (n x n x p), B (s x s x p): A*X - X*B = C.
void t_bartels_stewart_dev(ts_ctx* ctx, const double* A, int n, const double* B, int s, int p, const double* C,
                           double* X, cudaStream_t st) {
  const int K = num_slices(p);
  TS_REQUIRE((long long)K * s * n * n <= (1ll << 28), "ts_t_bartels_stewart: K*s*n^2 too large (small solver)");
  TS_REQUIRE(n <= 12000, "ts_t_bartels_stewart: n too large");
  double2* Ah = (double2*)ctx->ws.get("bs_Ah", sizeof(double2) * (size_t)K * n * n);
  double2* T = (double2*)ctx->ws.get("bs_T", sizeof(double2) * (size_t)K * s * s);
  double2* Q = (double2*)ctx->ws.get("bs_Q", sizeof(double2) * (size_t)K * s * s);
  double2* Ch = (double2*)ctx->ws.get("bs_Ch", sizeof(double2) * (size_t)K * n * s);
  double2* Gp = (double2*)ctx->ws.get("bs_G", sizeof(double2) * (size_t)K * n * s);
  double2* Z = (double2*)ctx->ws.get("bs_Z", sizeof(double2) * (size_t)K * n * s);
  double2* LU = (double2*)ctx->ws.get("bs_LU", sizeof(double2) * (size_t)K * s * n * n);
  int* piv = (int*)ctx->ws.get("bs_piv", sizeof(int) * (size_t)K * s * n);
  int* err = (int*)ctx->ws.get("bs_err", sizeof(int));
  rfft_tube<double, double2>(A, Ah, (long long)n * n, p, st);
  rfft_tube<double, double2>(B, T, (long long)s * s, p, st);
  rfft_tube<double, double2>(C, Ch, (long long)n * s, p, st);
  TS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  schur_small(T, Q, s, K, err, st);                                                // B_k = Q T Q^H
  const long long ss = (long long)s * s;
  small_gemm(Ch, (long long)n * s, n, Q, ss, s, false, Gp, (long long)n * s, n, n, s, s, K, false, st);   // G = C Q
  shifted_lu(Ah, (long long)n * n, T, LU, piv, n, n - 1, s, K, err, st);           // A_k - t_jj I
  hs_solve(LU, piv, Gp, T, Z, n, n - 1, s, K, st);
  small_gemm(Z, (long long)n * s, n, Q, ss, s, true, Ch, (long long)n * s, n, n, s, s, K, false, st);     // X = Z Q^H
  irfft_tube<double, double2>(Ch, X, (long long)n * s, p, IRFFT_STORE, nullptr, nullptr, st);
  int e = 0;
  TS_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  if (e & 1) throw Error{TS_SINGULAR, "complex Schur iteration of B_k did not converge"};
  if (e & 2) throw Error{TS_SINGULAR, "A_k - lambda I singular for an eigenvalue lambda of B_k (Theorem 2.1)"};
}

// Sparse operator from p CSR slices (host arrays): union pattern on the host, values' Fourier
// slices on the device.
void op_prepare_csr(ts_op* op, const int* rowptr, const int* col, const double* val, cudaStream_t st) {
  const int n = op->n, p = op->p, K = op->K;
  std::vector<int> urow(n + 1, 0);
  std::vector<int> ucol;
  std::vector<std::vector<int>> rows(n);
  for (int t = 0; t < p; ++t) {
    const int* rp = rowptr + (size_t)t * (n + 1);
    for (int i = 0; i < n; ++i) {
      TS_REQUIRE(rp[i] <= rp[i + 1], "ts_op_create_csr: row pointers must be non-decreasing");
      for (int q = rp[i]; q < rp[i + 1]; ++q) {
        TS_REQUIRE(col[q] >= 0 && col[q] < n, "ts_op_create_csr: column index out of range");
        rows[i].push_back(col[q]);
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    rows[i].erase(std::unique(rows[i].begin(), rows[i].end()), rows[i].end());
    urow[i + 1] = urow[i] + (int)rows[i].size();
    ucol.insert(ucol.end(), rows[i].begin(), rows[i].end());
  }
  const int nnz = urow[n];
  std::vector<double> uval((size_t)p * std::max(nnz, 1), 0.0);
  for (int t = 0; t < p; ++t) {
    const int* rp = rowptr + (size_t)t * (n + 1);
    for (int i = 0; i < n; ++i)
      for (int q = rp[i]; q < rp[i + 1]; ++q) {
        const int* b = ucol.data() + urow[i];
        const int* e = ucol.data() + urow[i + 1];
        const int pos = (int)(std::lower_bound(b, e, col[q]) - ucol.data());
        uval[(size_t)t * nnz + pos] += val[q];
      }
  }
  op->sp = new SparseOp();
  op->sp->nnz = nnz;
  op_alloc(op->sp->rowptr, sizeof(int) * (n + 1));
  op_alloc(op->sp->col, sizeof(int) * std::max(nnz, 1));
  op_alloc(op->sp->vals, sizeof(double2) * (size_t)K * std::max(nnz, 1));
  double* dval = (double*)op->ctx->ws.get("csr_stage_vals", sizeof(double) * (size_t)p * std::max(nnz, 1));
  TS_CUDA(cudaMemcpyAsync(op->sp->rowptr, urow.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
  if (nnz > 0) {
    TS_CUDA(cudaMemcpyAsync(op->sp->col, ucol.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
    TS_CUDA(cudaMemcpyAsync(dval, uval.data(), sizeof(double) * (size_t)p * nnz, cudaMemcpyHostToDevice, st));
    rfft_tube<double, double2>(dval, op->sp->vals, nnz, p, st);
  }
  TS_CUDA(cudaStreamSynchronize(st));
}

}  // namespace ts
