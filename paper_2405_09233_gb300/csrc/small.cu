// The small FP64 problems of tGMRES and tFOM, kept on the device so the Arnoldi loop never
// waits for the host between steps.
//
// tGMRES (§3.3): y = argmin || beta e1 - Htilde_k y ||_2.  The QR factorisation of Htilde_k that
// Proposition 3.4 refers to is built one column at a time with Givens rotations: column j of H
// receives the j earlier rotations, a new rotation zeroes h_{j+1,j}, and the rotated right-hand
// side g gives the residual norm |gamma_{j+1}| = |g_{j+1}| without forming y.
// tFOM (§3.2): H_k y = beta e1 by Gaussian elimination with partial pivoting (a Hessenberg
// matrix only needs a choice between rows c and c+1 at column c); the estimate is
// h_{k+1,k} |y_k| (Proposition 3.3).
#include <algorithm>
#include "internal.cuh"
#include "reduce.cuh"

namespace ts {
namespace {

struct Layout {
  int m;
  __host__ __device__ size_t H() const { return 0; }
  __host__ __device__ size_t R() const { return (size_t)(m + 1) * m; }
  __host__ __device__ size_t cs() const { return R() + (size_t)(m + 1) * m; }
  __host__ __device__ size_t sn() const { return cs() + m; }
  __host__ __device__ size_t g() const { return sn() + m; }
  __host__ __device__ size_t y() const { return g() + m + 1; }
  __host__ __device__ size_t est() const { return y() + m; }
  __host__ __device__ size_t beta() const { return est() + 8; }
  __host__ __device__ size_t lu() const { return beta() + 8; }
  __host__ __device__ size_t hist() const { return lu() + (size_t)m * m + m; }
  __host__ __device__ size_t total() const { return hist() + m; }
};

constexpr double kBreakdownRel = 1e-14;

__global__ void k_ks_init(double* st, int m, const double* beta_in) {
  Layout L{m};
  const double beta = beta_in[0];
  for (int i = threadIdx.x; i < (m + 1) * m; i += blockDim.x) {
    st[L.H() + i] = 0.0;
    st[L.R() + i] = 0.0;
  }
  for (int i = threadIdx.x; i <= m; i += blockDim.x) st[L.g() + i] = (i == 0) ? beta : 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) st[L.y() + i] = 0.0;
  if (threadIdx.x == 0) {
    st[L.beta()] = beta;
    st[L.beta() + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int q = 0; q < 8; ++q) st[L.est() + q] = 0.0;
  }
}

// est[0] = estimate, est[1] = 1/h_{j+1,j}, est[2] = h_{j+1,j}, est[3] = flags (1 breakdown,
// 2 singular, 4 non-finite), est[4] = steps taken in this cycle (j + 1), est[8 + j] = estimate of
// step j.  In a graph-captured cycle, `handle` is the conditional handle of step j + 1 (0 for the
// last step) and the kernel decides whether the cycle goes on: it sets that handle to 0 on breakdown,
// a bad step, an estimate <= stop[0] (the tolerance times ||C||) or <= stop[1] (the inner tolerance
// of mixed precision, or -1).
// Columns of the Givens state staged in shared memory (tGMRES, m <= kStageMax): thread 0 then
// rotates without a chain of dependent global loads (~0.7 us each; ~8 us at j = 10 before).
constexpr int kStageMax = 256;

// Step j's update given h_{j+1,j} = hn; called by every thread of the block (one block).
__device__ void ks_update(double* st, int m, int j, int method, double hn, cudaGraphConditionalHandle handle,
                          const double* stop, int* gate = nullptr) {
  __shared__ double s_col[kStageMax + 2], s_cs[kStageMax], s_sn[kStageMax];
  Layout L{m};
  double* H = st + L.H();
  const int ld = m + 1;
  const bool staged = method == 0 && m <= kStageMax;
  if (staged) {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) s_col[i] = H[i + ld * j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      s_cs[i] = st[L.cs() + i];
      s_sn[i] = st[L.sn() + i];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  H[(j + 1) + ld * j] = hn;
  const double beta = st[L.beta()];
  double flags = (hn <= kBreakdownRel * beta) ? 1.0 : 0.0;
  double est;
  if (method == 0) {
    double* R = st + L.R();
    double* cs = st + L.cs();
    double* sn = st + L.sn();
    double* g = st + L.g();
    double* col = staged ? s_col : R + ld * j;
    const double* c_cs = staged ? s_cs : cs;
    const double* c_sn = staged ? s_sn : sn;
    if (!staged)
      for (int i = 0; i <= j; ++i) col[i] = H[i + ld * j];
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = col[i], b = col[i + 1];
      col[i] = c_cs[i] * a + c_sn[i] * b;
      col[i + 1] = -c_sn[i] * a + c_cs[i] * b;
    }
    const double a = col[j], b = col[j + 1];
    const double r = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (r > 0.0) {
      c = a / r;
      s = b / r;
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    if (staged)
      for (int i = 0; i <= j + 1; ++i) R[i + ld * j] = col[i];
    const double gj = g[j];
    g[j + 1] = -s * gj;
    g[j] = c * gj;
    est = fabs(g[j + 1]);
  } else {
    // Gaussian elimination with partial pivoting on H_k (k = j+1), right-hand side beta e1.
    const int k = j + 1;
    double* M = st + L.lu();   // k x k, column-major, followed by the right-hand side
    double* rhs = M + (size_t)m * m;
    for (int c = 0; c < k; ++c)
      for (int r = 0; r < k; ++r) M[r + k * c] = (r <= c + 1) ? H[r + ld * c] : 0.0;
    for (int r = 0; r < k; ++r) rhs[r] = (r == 0) ? beta : 0.0;
    bool singular = false;
    for (int c = 0; c < k; ++c) {
      if (c + 1 < k && fabs(M[c + 1 + k * c]) > fabs(M[c + k * c])) {
        for (int q = c; q < k; ++q) {
          const double t = M[c + k * q];
          M[c + k * q] = M[c + 1 + k * q];
          M[c + 1 + k * q] = t;
        }
        const double t = rhs[c];
        rhs[c] = rhs[c + 1];
        rhs[c + 1] = t;
      }
      const double piv = M[c + k * c];
      if (piv == 0.0) {
        singular = true;
        break;
      }
      if (c + 1 < k) {
        const double f = M[c + 1 + k * c] / piv;
        for (int q = c; q < k; ++q) M[c + 1 + k * q] -= f * M[c + k * q];
        rhs[c + 1] -= f * rhs[c];
      }
    }
    double* y = st + L.y();
    if (!singular) {
      for (int r = k - 1; r >= 0; --r) {
        double v = rhs[r];
        for (int q = r + 1; q < k; ++q) v -= M[r + k * q] * y[q];
        y[r] = v / M[r + k * r];
      }
      est = hn * fabs(y[k - 1]);
    } else {
      flags += 2.0;
      est = INFINITY;
    }
  }
  if (!isfinite(est) || !isfinite(hn)) flags += 4.0;
  st[L.est()] = est;
  st[L.est() + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
  st[L.est() + 2] = hn;
  st[L.est() + 3] = flags;
  st[L.est() + 4] = j + 1;
  st[L.hist() + j] = est;
  if (handle || gate) {
    const bool go = flags == 0.0 && !(est <= stop[0]) && !(est <= stop[1]);
    if (!go) {
      if (handle) cudaGraphSetConditional(handle, 0);
      if (gate) *gate = 0;
    }
  }
}

__global__ void k_ks_step(double* st, int m, int j, int method, const double* Pnorm,
                          cudaGraphConditionalHandle handle, const double* stop) {
  const double hn = sqrt(finalize_partials(Pnorm));
  ks_update(st, m, j, method, hn, handle, stop);
}

// Everything of inner step j after W = M(V_j), for vectors of at most kArnMaxN entries, in one
// launch of a thread-block cluster of CL <= kArnCL CTAs: the modified Gram-Schmidt sweep
// h_ij = <V_i, W>, W -= h_ij V_i (i = 0..j, in order), the norm h_{j+1,j} = ||W||, the Givens /
// Hessenberg update (ks_update, by CTA 0) and V_{j+1} = W / h_{j+1,j}.  CTA c owns a contiguous part
// of the vectors, kept in registers (W) or loaded one pass ahead (the next V_i).  An inner product
// is summed per warp (butterfly), every warp's partial is stored into every CTA's shared memory
// (distributed shared memory), and after one cluster barrier each warp adds all partials in the same
// fixed order, so every thread of every CTA holds the same value, bit for bit.  GB300's FP64 pipe
// issues one warp's DFMA in 64 clocks per SM sub-partition, so one CTA spent ~2.3 us per MGS pass at
// 2304 entries in FP64 issue alone; eight SMs cut that eightfold, and the pass is left with two short
// reduction trees and the barrier.  Same arithmetic as the multi-block kernels (FP64 sums; an FP32
// basis sums each thread's products in FP32 first), in a different summation order.  All CTAs pass
// the same barriers (j is a kernel argument; the gate is read once, before the first barrier, and
// written by CTA 0 only after the last), the first barrier precedes every remote store and no remote
// store follows the last one.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

constexpr int kArnCL = 8, kArnMaxThreads = 512, kArnMaxN = kArnCL * kArnMaxThreads * 16;

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <typename T, int R>
__global__ void __launch_bounds__(kArnMaxThreads, 1)
    k_arnoldi_cluster(T* __restrict__ W, T* __restrict__ V, long long ldv, int N, int j, int m, double* st,
                      int method, cudaGraphConditionalHandle handle, const double* stop, int* gate) {
  if (gate && *gate == 0) return;   // launched ahead of a cycle that has already ended (all CTAs alike)
  __shared__ double slots[2][kArnCL * (kArnMaxThreads / 32)];
  uint32_t rank, ncta;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
  const int nt = blockDim.x, nw = nt / 32, t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int Nc = (N + (int)ncta - 1) / (int)ncta, e0 = (int)rank * Nc;
  auto idx = [&](int r) {   // element of (thread, r), or -1
    const int q = t + nt * r, e = e0 + q;
    return (q < Nc && e < N) ? e : -1;
  };
  Layout L{m};
  double* H = st + L.H();
  const int ld = m + 1;
  T w[R], v[R], vn[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = idx(r);
    w[r] = e >= 0 ? W[e] : T(0);
    v[r] = e >= 0 ? V[e] : T(0);
  }
  auto dot = [&](const T (&x)[R]) {
    if constexpr (sizeof(T) == 4) {
      float f = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) f = fmaf(x[r], w[r], f);
      return (double)f;
    } else {
      double acc = 0.0;
#pragma unroll
      for (int r = 0; r < R; ++r) acc += x[r] * w[r];
      return acc;
    }
  };
  int buf = 0;
  auto cluster_sum = [&](double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) {
      const uint32_t local = smem_addr(&slots[buf][(int)rank * nw + wp]);
      for (uint32_t c = 0; c < ncta; ++c) {
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(c));
        asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(x) : "memory");
      }
    }
    cluster_sync_all();
    double y = 0.0;
    for (int q = lane; q < (int)ncta * nw; q += 32) y += slots[buf][q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    buf ^= 1;
    return y;
  };
  cluster_sync_all();   // every CTA of the cluster runs before any remote store
  for (int i = 0; i <= j; ++i) {
    const double part = dot(v);
    if (i < j) {
      const T* Vn = V + (long long)(i + 1) * ldv;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = idx(r);
        vn[r] = e >= 0 ? Vn[e] : T(0);
      }
    }
    const double h = cluster_sum(part);
    if (rank == 0 && t == 0) H[i + ld * j] = h;
    const T hT = (T)h;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      w[r] = w[r] - hT * v[r];
      v[r] = vn[r];
    }
  }
  const double hn = sqrt(cluster_sum(dot(w)));
  if (rank == 0) ks_update(st, m, j, method, hn, handle, stop, gate);
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  T* Vj1 = V + (long long)(j + 1) * ldv;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = idx(r);
    if (e >= 0) {
      if constexpr (sizeof(T) == 4) Vj1[e] = w[r] * (float)inv;
      else Vj1[e] = w[r] * inv;
    }
  }
}

// tGMRES: back substitution R_k y = g_k.  tFOM: y is already the solution of the last step.
// R_k and g_k are staged in shared memory first (k <= kSolveStage) so that one thread's substitution
// does not wait on a global load per term (~29 us at k = 18 before).
constexpr int kSolveStage = 64;
__global__ void k_ks_solve(double* st, int m, int k, int method) {
  if (method != 0) return;
  __shared__ double sR[kSolveStage * kSolveStage], sg[kSolveStage], sy[kSolveStage];
  Layout L{m};
  const int ld = m + 1;
  const double* R = st + L.R();
  const double* g = st + L.g();
  double* y = st + L.y();
  const bool staged = k <= kSolveStage;
  if (staged) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int r = e % k, q = e / k;
      sR[r + kSolveStage * q] = R[r + ld * q];
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) sg[r] = g[r];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (staged) {
    for (int r = k - 1; r >= 0; --r) {
      double v = sg[r];
      for (int q = r + 1; q < k; ++q) v -= sR[r + kSolveStage * q] * sy[q];
      sy[r] = v / sR[r + kSolveStage * r];
    }
    for (int r = 0; r < k; ++r) y[r] = sy[r];
    return;
  }
  for (int r = k - 1; r >= 0; --r) {
    double v = g[r];
    for (int q = r + 1; q < k; ++q) v -= R[r + ld * q] * y[q];
    y[r] = v / R[r + ld * r];
  }
}

}  // namespace

size_t krylov_state_bytes(int m) { return Layout{m}.total() * sizeof(double); }
double* ks_H(void* s, int m) { return static_cast<double*>(s) + Layout{m}.H(); }
double* ks_y(void* s, int m) { return static_cast<double*>(s) + Layout{m}.y(); }
double* ks_est(void* s, int m) { return static_cast<double*>(s) + Layout{m}.est(); }
double* ks_beta(void* s, int m) { return static_cast<double*>(s) + Layout{m}.beta(); }

void ks_init(void* state, int m, const double* beta_and_inv, cudaStream_t st) {
  k_ks_init<<<1, 256, 0, st>>>(static_cast<double*>(state), m, beta_and_inv);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

double* ks_hist(void* s, int m) { return static_cast<double*>(s) + Layout{m}.hist(); }

void ks_step(void* state, int m, int j, int method, const double* Pnorm, cudaStream_t st,
             cudaGraphConditionalHandle handle, const double* stop) {
  k_ks_step<<<1, 256, 0, st>>>(static_cast<double*>(state), m, j, method, Pnorm, handle, stop);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

bool arnoldi_small_ok(long long N) { return N >= 1 && N <= kArnMaxN; }

template <typename T, int R>
void launch_arnoldi_cluster(int cl, int nt, T* W, T* V, long long ldv, int n, int j, int m, double* s, int method,
                            cudaGraphConditionalHandle handle, const double* stop, int* gate, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(nt, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TS_CUDA(cudaLaunchKernelEx(&cfg, k_arnoldi_cluster<T, R>, W, V, ldv, n, j, m, s, method, handle, stop, gate));
}

template <typename T>
void arnoldi_small(T* W, T* V, long long ldv, long long N, int j, int m, void* state, int method, cudaStream_t st,
                   cudaGraphConditionalHandle handle, const double* stop, int* gate) {
  TS_REQUIRE(arnoldi_small_ok(N) && j >= 0 && j < m, "arnoldi_small: bad size");
  double* s = static_cast<double*>(state);
  const int n = (int)N;
  // CTAs: one per 64 entries up to kArnCL; threads: the CTA's share in R-element runs, whole warps
  const int cl = (int)std::min<long long>(kArnCL, std::max<long long>(1, (N + 63) / 64));
  const long long nc = (N + cl - 1) / cl;
  auto threads = [&](int R) { return (int)((nc + 32LL * R - 1) / (32LL * R) * 32); };
  if (nc <= kArnMaxThreads * 2LL)
    launch_arnoldi_cluster<T, 2>(cl, threads(2), W, V, ldv, n, j, m, s, method, handle, stop, gate, st);
  else if (nc <= kArnMaxThreads * 4LL)
    launch_arnoldi_cluster<T, 4>(cl, threads(4), W, V, ldv, n, j, m, s, method, handle, stop, gate, st);
  else if (nc <= kArnMaxThreads * 8LL)
    launch_arnoldi_cluster<T, 8>(cl, threads(8), W, V, ldv, n, j, m, s, method, handle, stop, gate, st);
  else
    launch_arnoldi_cluster<T, 16>(cl, threads(16), W, V, ldv, n, j, m, s, method, handle, stop, gate, st);
  count_launch();
  TS_CUDA(cudaGetLastError());
}
template void arnoldi_small<double>(double*, double*, long long, long long, int, int, void*, int, cudaStream_t,
                                    cudaGraphConditionalHandle, const double*, int*);
template void arnoldi_small<float>(float*, float*, long long, long long, int, int, void*, int, cudaStream_t,
                                   cudaGraphConditionalHandle, const double*, int*);

void ks_solve(void* state, int m, int k, int method, cudaStream_t st) {
  k_ks_solve<<<1, 256, 0, st>>>(static_cast<double*>(state), m, k, method);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace ts
