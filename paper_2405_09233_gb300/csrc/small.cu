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
__global__ void k_ks_step(double* st, int m, int j, int method, const double* Pnorm,
                          cudaGraphConditionalHandle handle, const double* stop) {
  Layout L{m};
  const double hn = sqrt(finalize_partials(Pnorm));
  if (threadIdx.x != 0) return;
  double* H = st + L.H();
  const int ld = m + 1;
  H[(j + 1) + ld * j] = hn;
  const double beta = st[L.beta()];
  double flags = (hn <= kBreakdownRel * beta) ? 1.0 : 0.0;
  double est;
  if (method == 0) {
    double* R = st + L.R();
    double* cs = st + L.cs();
    double* sn = st + L.sn();
    double* g = st + L.g();
    for (int i = 0; i <= j + 1; ++i) R[i + ld * j] = H[i + ld * j];
    for (int i = 0; i < j; ++i) {
      const double a = R[i + ld * j], b = R[i + 1 + ld * j];
      R[i + ld * j] = cs[i] * a + sn[i] * b;
      R[i + 1 + ld * j] = -sn[i] * a + cs[i] * b;
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
  if (handle) {
    const bool go = flags == 0.0 && !(est <= stop[0]) && !(est <= stop[1]);
    if (!go) cudaGraphSetConditional(handle, 0);
  }
}

// tGMRES: back substitution R_k y = g_k.  tFOM: y is already the solution of the last step.
__global__ void k_ks_solve(double* st, int m, int k, int method) {
  if (threadIdx.x != 0 || method != 0) return;
  Layout L{m};
  const int ld = m + 1;
  const double* R = st + L.R();
  const double* g = st + L.g();
  double* y = st + L.y();
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

void ks_solve(void* state, int m, int k, int method, cudaStream_t st) {
  k_ks_solve<<<1, 32, 0, st>>>(static_cast<double*>(state), m, k, method);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace ts
