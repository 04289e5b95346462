// Small dense complex FP64 kernels for the projected equation of TBAS and for t-Bartels-Stewart
// (§4, Algorithm 5; §5.2, the projected equation H_m*Y - Y*B = C1).
//
// Per Fourier slice the tensor equation is the matrix Sylvester equation H_k Y_k - Y_k B_k = F_k.
// It is solved by the Hessenberg-Schur form of Bartels-Stewart: only B_k (s x s) is reduced to
// complex Schur form B_k = Q T Q^H (schur.cu); with Z = Y Q and G = F Q,
// column j of Z solves (H_k - t_jj I) z_j = g_j + sum_{i<j} t_ij z_i.  The shifted matrices are
// factorised in parallel (one CTA per (slice, j), LU with partial pivoting restricted to the lower
// bandwidth, which is s for the block Hessenberg H_m of TBA and n-1 for a general matrix), then one
// CTA per slice sweeps j in order.  All matrices are column-major complex (double2).
#include "internal.cuh"
#include "reduce.cuh"
#include "tba.cuh"
#include "complex_ops.cuh"

namespace ts {
namespace {

// LU with partial pivoting of M = H_k - t_jj I, lower bandwidth bw, one CTA per (j, k).
// LU[(k*s + j)] is an N x N column-major factor; piv holds the row chosen at each step.  Per column
// c: warp 0 finds the pivot among rows c..c+bw (shuffle argmax, first index on ties), swaps it into
// column c, and forms the multipliers (kept in column c, and the first kLuMaxBw in shared memory);
// then every thread takes columns q > c, applies the row interchange to its column and subtracts
// the multipliers times M[c, q] down the band: two barriers per column.  (The first version reduced
// the pivot candidates of all 256 threads serially and used five barriers per column.)
constexpr int kLuMaxBw = 256;
__global__ void __launch_bounds__(256) k_shifted_lu(const double2* __restrict__ H, long long sH,
                                                    const double2* __restrict__ T, double2* __restrict__ LU,
                                                    int* __restrict__ piv, int N, int bw, int s, int* err) {
  const int j = blockIdx.x, k = blockIdx.y;
  const double2* Hk = H + (long long)k * sH;
  const double2 shift = T[(long long)k * s * s + (long long)j * s + j];
  double2* M = LU + ((long long)k * s + j) * N * N;
  int* pv = piv + ((long long)k * s + j) * N;
  for (long long e = threadIdx.x; e < (long long)N * N; e += blockDim.x) {
    double2 v = Hk[e];
    if ((e % N) == (e / N)) v = csub(v, shift);
    M[e] = v;
  }
  __shared__ int sp;
  __shared__ double sbest[256];
  __shared__ double2 sl[kLuMaxBw];
  __syncthreads();
  // max-norm of M: a pivot below N * 1e-14 * max|M| marks a (numerically) singular shift
  double mx = 0.0;
  for (long long e = threadIdx.x; e < (long long)N * N; e += blockDim.x) mx = fmax(mx, cabs2(M[e]));
  sbest[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m0 = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) m0 = fmax(m0, sbest[t]);
    sbest[0] = m0;
  }
  __syncthreads();
  const double tiny = 1e-14 * N * sbest[0];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < N; ++c) {
    const int rmax = (c + bw < N - 1) ? c + bw : N - 1, nr = rmax - c;
    double2* Mc = M + (long long)N * c;
    if (warp == 0) {
      double best = -1.0;
      int bi = c;
      for (int r = c + lane; r <= rmax; r += 32) {
        const double v = cabs2(Mc[r]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      const int p = bi;
      if (lane == 0) {
        pv[c] = p;
        sp = p;
        if (best <= tiny) atomicOr(err, 2);
        if (p != c) {
          const double2 t0 = Mc[c];
          Mc[c] = Mc[p];
          Mc[p] = t0;
        }
      }
      __syncwarp();
      const double2 dinv = cdiv(make_double2(1.0, 0.0), Mc[c]);
      for (int r = lane; r < nr; r += 32) {
        const double2 l = cmul(Mc[c + 1 + r], dinv);
        Mc[c + 1 + r] = l;
        if (r < kLuMaxBw) sl[r] = l;
      }
    }
    __syncthreads();
    const int p = sp;
    for (int q = c + 1 + (int)threadIdx.x; q < N; q += blockDim.x) {
      double2* Mq = M + (long long)N * q;
      if (p != c) {
        const double2 t0 = Mq[c];
        Mq[c] = Mq[p];
        Mq[p] = t0;
      }
      const double2 u = Mq[c];
      for (int r = 0; r < nr; ++r)
        Mq[c + 1 + r] = csub(Mq[c + 1 + r], cmul(r < kLuMaxBw ? sl[r] : Mc[c + 1 + r], u));
    }
    __syncthreads();
  }
}

// One CTA per slice: Z[:, j] for j = 0..s-1 in order, using the factors of k_shifted_lu.  Both
// triangular solves are blocked by kHsB columns so that the long dependent chains run inside one
// warp on shared memory:
//   forward  for each block of columns: stage the pivots and, for bands up to kHsBandStage wide,
//            the L band (rows c+1 .. c+bw), then one warp applies the row interchanges and
//            eliminations of the block in order (the same operations, in the same order, as the
//            unblocked solve); wider bands (t-Bartels-Stewart, bw = n - 1) are read from global memory;
//   backward for each block from the last: stage the diagonal kHsB x kHsB block of U, one warp
//            solves it, then all threads subtract the block's columns from the rows above (GEMV).
constexpr int kHsB = 32;
constexpr int kHsBandStage = 64;
__global__ void __launch_bounds__(256) k_hs_solve(const double2* __restrict__ LU, const int* __restrict__ piv,
                                                  const double2* __restrict__ G, const double2* __restrict__ T,
                                                  double2* __restrict__ Z, int N, int bw, int s) {
  const int k = blockIdx.x;
  const double2* Gk = G + (long long)k * N * s;
  const double2* Tk = T + (long long)k * s * s;
  double2* Zk = Z + (long long)k * N * s;
  extern __shared__ double2 hs_smem[];
  double2* rhs = hs_smem;                       // N
  const bool stage = bw <= kHsBandStage;
  double2* Lb = rhs + N;                        // kHsB x bw  (band of the block's L columns), if staged
  double2* Ub = Lb + (stage ? (size_t)kHsB * bw : 0);   // kHsB x (kHsB + 1)
  __shared__ int spv[kHsB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < s; ++j) {
    const double2* M = LU + ((long long)k * s + j) * N * N;
    const int* pv = piv + ((long long)k * s + j) * N;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      double2 v = Gk[r + (long long)N * j];
      for (int i = 0; i < j; ++i) v = cadd(v, cmul(Tk[i + (long long)s * j], Zk[r + (long long)N * i]));
      rhs[r] = v;
    }
    __syncthreads();
    // forward: row interchanges and the unit lower factor
    for (int c0 = 0; c0 < N; c0 += kHsB) {
      const int nb = min(kHsB, N - c0);
      for (int e = threadIdx.x; stage && e < nb * bw; e += blockDim.x) {
        const int cc = e / bw, t = e % bw, c = c0 + cc, r = c + 1 + t;
        Lb[e] = r < N ? M[r + (long long)N * c] : make_double2(0.0, 0.0);
      }
      for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) spv[cc] = pv[c0 + cc];
      __syncthreads();
      if (warp == 0) {
        for (int cc = 0; cc < nb; ++cc) {
          const int c = c0 + cc, p = spv[cc];
          if (p != c && lane == 0) {
            const double2 t0 = rhs[c];
            rhs[c] = rhs[p];
            rhs[p] = t0;
          }
          __syncwarp();
          const double2 rc = rhs[c];
          const int nr = min(bw, N - 1 - c);
          for (int t = lane; t < nr; t += 32) {
            const double2 l = stage ? Lb[cc * bw + t] : M[(c + 1 + t) + (long long)N * c];
            rhs[c + 1 + t] = csub(rhs[c + 1 + t], cmul(l, rc));
          }
          __syncwarp();
        }
      }
      __syncthreads();
    }
    // backward: the upper factor, by blocks from the last
    for (int c1 = N; c1 > 0; c1 -= kHsB) {
      const int c0 = max(0, c1 - kHsB), nb = c1 - c0;
      for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int rr = e % nb, cc = e / nb;
        Ub[rr + (kHsB + 1) * cc] = M[(c0 + rr) + (long long)N * (c0 + cc)];
      }
      __syncthreads();
      if (warp == 0) {
        for (int cc = nb - 1; cc >= 0; --cc) {
          if (lane == 0) rhs[c0 + cc] = cdiv(rhs[c0 + cc], Ub[cc + (kHsB + 1) * cc]);
          __syncwarp();
          const double2 zc = rhs[c0 + cc];
          if (lane < cc) rhs[c0 + lane] = csub(rhs[c0 + lane], cmul(Ub[lane + (kHsB + 1) * cc], zc));
          __syncwarp();
        }
      }
      __syncthreads();
      for (int r = threadIdx.x; r < c0; r += blockDim.x) {
        double2 v = rhs[r];
        for (int cc = 0; cc < nb; ++cc) v = csub(v, cmul(M[r + (long long)N * (c0 + cc)], rhs[c0 + cc]));
        rhs[r] = v;
      }
      __syncthreads();
    }
    for (int r = threadIdx.x; r < N; r += blockDim.x) Zk[r + (long long)N * j] = rhs[r];
    __syncthreads();
  }
}

// C = A * op(B) for small column-major complex matrices per slice: op = none or conjugate
// transpose.  A: M x L (lda), B: L x Ncol (or Ncol x L when conjugate-transposed).
__global__ void k_small_gemm(const double2* __restrict__ A, long long sA, int lda, const double2* __restrict__ B,
                             long long sB, int ldb, int transB, double2* __restrict__ C, long long sC, int ldc, int M,
                             int L, int Ncol, int accumulate) {
  const int k = blockIdx.y;
  const double2* Ak = A + (long long)k * sA;
  const double2* Bk = B + (long long)k * sB;
  double2* Ck = C + (long long)k * sC;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)M * Ncol;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    double2 acc = accumulate ? Ck[i + (long long)ldc * j] : make_double2(0.0, 0.0);
    for (int l = 0; l < L; ++l) {
      const double2 b = transB ? cconj(Bk[j + (long long)ldb * l]) : Bk[l + (long long)ldb * j];
      acc = cadd(acc, cmul(Ak[i + (long long)lda * l], b));
    }
    Ck[i + (long long)ldc * j] = acc;
  }
}

// Cholesky G = R^H R of a Hermitian positive definite s x s matrix per slice (one warp each).
// R is written upper triangular (zeros below).  A pivot d_j (the squared norm of column j's part
// orthogonal to the previous columns, when G is a Gram matrix) fails when it is not above
// max(rel * g_jj, tiny2 * max_k g_jj(k)), the second maximum taken over the Grams of all K slices;
// rel = tiny2 = 0 asks for d_j > 0 only.  A failed slice stops early (R partly written), sets
// fail_slice[slice] = 1 (each slice's entry is reset to 0 first) and err bit 4 (err may be NULL).
__global__ void k_cholesky(const double2* __restrict__ Gall, double2* __restrict__ Rall, int s, int K, double rel,
                           double tiny2, int* err, int* fail_slice) {
  const double2* G = Gall + (long long)blockIdx.x * s * s;
  double2* R = Rall + (long long)blockIdx.x * s * s;
  const int lane = threadIdx.x & 31;
  if (fail_slice && lane == 0) fail_slice[blockIdx.x] = 0;
  for (int e = lane; e < s * s; e += 32) R[e] = make_double2(0.0, 0.0);
  __syncwarp();
  for (int j = 0; j < s; ++j) {
    // r_jj = sqrt(g_jj - sum_{i<j} |r_ij|^2)
    const double gjj = G[j + (long long)s * j].x;
    double d = gjj;
    for (int i = 0; i < j; ++i) {
      const double2 r = R[i + (long long)s * j];
      d -= r.x * r.x + r.y * r.y;
    }
    double floor_d = rel * gjj;
    if (tiny2 > 0.0) {
      double ref2 = 0.0;
      for (int q = 0; q < K; ++q) ref2 = fmax(ref2, Gall[(long long)q * s * s + j + (long long)s * j].x);
      floor_d = fmax(floor_d, tiny2 * ref2);
    }
    if (!(d > floor_d)) {
      if (lane == 0) {
        if (err) atomicOr(err, 4);
        if (fail_slice) fail_slice[blockIdx.x] = 1;
      }
      return;
    }
    const double rjj = sqrt(d);
    if (lane == 0) R[j + (long long)s * j] = make_double2(rjj, 0.0);
    // r_jq = (g_jq - sum_{i<j} conj(r_ij) r_iq) / r_jj for q > j
    for (int q = j + 1 + lane; q < s; q += 32) {
      double2 v = G[j + (long long)s * q];
      for (int i = 0; i < j; ++i) v = csub(v, cmulc(R[i + (long long)s * j], R[i + (long long)s * q]));
      R[j + (long long)s * q] = cscale(v, 1.0 / rjj);
    }
    __syncwarp();
  }
}

}  // namespace

void shifted_lu(const double2* H, long long sH, const double2* T, double2* LU, int* piv, int N, int bw, int s, int K,
                int* err, cudaStream_t st) {
  k_shifted_lu<<<dim3(s, K), 256, 0, st>>>(H, sH, T, LU, piv, N, bw, s, err);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void hs_solve(const double2* LU, const int* piv, const double2* G, const double2* T, double2* Z, int N, int bw, int s,
              int K, cudaStream_t st) {
  const size_t band = bw <= kHsBandStage ? (size_t)kHsB * bw : 0;
  const size_t smem = sizeof(double2) * ((size_t)N + band + (size_t)kHsB * (kHsB + 1));
  TS_REQUIRE(smem <= 200 * 1024, "projected system too large");
  if (smem > 48 * 1024) TS_CUDA(cudaFuncSetAttribute(k_hs_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_hs_solve<<<K, 256, smem, st>>>(LU, piv, G, T, Z, N, bw, s);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void small_gemm(const double2* A, long long sA, int lda, const double2* B, long long sB, int ldb, bool transB, double2* C,
                long long sC, int ldc, int M, int L, int Ncol, int K, bool accumulate, cudaStream_t st) {
  long long tot = (long long)M * Ncol;
  int g = (int)((tot + 255) / 256);
  if (g > 1024) g = 1024;
  k_small_gemm<<<dim3(g, K), 256, 0, st>>>(A, sA, lda, B, sB, ldb, transB ? 1 : 0, C, sC, ldc, M, L, Ncol,
                                           accumulate ? 1 : 0);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void cholesky_small(const double2* G, double2* R, int s, int K, double rel, double tiny2, int* err, int* fail_slice,
                    cudaStream_t st) {
  k_cholesky<<<K, 32, 0, st>>>(G, R, s, K, rel, tiny2, err, fail_slice);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace ts
