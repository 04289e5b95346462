// Internal declarations of libtstar (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <atomic>
#include <map>
#include <vector>
#include "../../include/tstar.h"

namespace ts {

// ----------------------------------------------------------------------------------------------
// Errors
// ----------------------------------------------------------------------------------------------
struct Error {
  ts_status status;
  std::string msg;
};

#define TS_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::ts::Error{TS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define TS_REQUIRE(cond, msg)                                   \
  do {                                                          \
    if (!(cond)) throw ::ts::Error{TS_ERR_ARG, std::string(msg)}; \
  } while (0)

// ----------------------------------------------------------------------------------------------
// Device workspace: named buffers that grow on demand and live as long as the context.
// ----------------------------------------------------------------------------------------------
// Every buffer carries a guard band of kGuardBytes filled with kGuardByte after its usable bytes;
// check() reports a buffer whose guard was overwritten (an out-of-bounds write).
struct Workspace {
  static constexpr size_t kGuardBytes = 4096;
  static constexpr unsigned char kGuardByte = 0xA5;
  struct Buf { void* ptr = nullptr; size_t bytes = 0; };
  std::map<std::string, Buf> bufs;
  void* get(const std::string& name, size_t bytes);
  std::string check() const;   // "" when every guard is intact, else the first damaged buffer
  void release_all();
};

// ----------------------------------------------------------------------------------------------
// Operator buffers (Fourier slices, low-precision and digit planes, Schur factors, sparse pattern):
// taken from a process-wide stream-ordered memory pool of the current device that keeps up to
// kOpPoolKeepBytes of freed memory reserved, so creating and destroying operators of recurring
// shapes does not map and unmap device memory every time.  op_malloc returns memory usable on
// every stream (like cudaMalloc) and throws TS_ERR_NOMEM on failure.  op_free defers the release:
// buffers are kept (unusable by anyone) until 2 GiB of them have gathered, an allocation of the same
// size asks for one, an allocation fails or a context is destroyed; then one device synchronisation
// makes them all idle, so that no pending kernel can still read them, and they are kept (up to 8 GiB)
// for allocations of exactly their size, which then need no CUDA call; nullptr is ignored.
// ----------------------------------------------------------------------------------------------
constexpr unsigned long long kOpPoolKeepBytes = 16ull << 30;
void* op_malloc(size_t bytes);
void op_free(void* p);
void op_free_flush();   // return every deferred buffer of the current device's pool now
template <typename T>
inline void op_alloc(T*& p, size_t bytes) {
  p = static_cast<T*>(op_malloc(bytes));
}
// Stream-ordered form: the buffer is usable on `st` (and on work ordered after it) without any host
// synchronisation; for buffers that a call prepares on `st` and that are only used after it.
void* op_malloc_on(size_t bytes, cudaStream_t st);
template <typename T>
inline void op_alloc_on(T*& p, size_t bytes, cudaStream_t st) {
  p = static_cast<T*>(op_malloc_on(bytes, st));
}

// ----------------------------------------------------------------------------------------------
// Reductions: a fixed grid so that the summation order (hence the result) is reproducible.
// ----------------------------------------------------------------------------------------------
constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;

// Process-wide count of kernel launches (reported by ts_stats_get).
extern std::atomic<long long> g_launches;
// Launches recorded into a CUDA graph are counted when the graph is replayed, not while it is
// captured: CountSuppress turns counting off on this thread for its lifetime.
extern thread_local int g_count_suppress;
inline void count_launch(long long n = 1) {
  if (!g_count_suppress) g_launches.fetch_add(n, std::memory_order_relaxed);
}
struct CountSuppress {
  CountSuppress() { ++g_count_suppress; }
  ~CountSuppress() { --g_count_suppress; }
};

// Event timing of selected kernels while a context has statistics enabled.
struct TimedRegion {
  cudaEvent_t a, b;
  int kind;        // 0 = FP64 GEMM, 1 = FFT, 2 = low-precision GEMM, 3 = emulated FP64 GEMM, 4 = TBAS block products,
                   // 5 = sparse A_k V products (TBAS)
  double work;     // algorithmic FLOPs (GEMM, sparse products) or bytes (FFT)
  double work2;    // sparse products: algorithmic bytes
};
struct KernelTimer {
  bool enabled = false;
  std::vector<TimedRegion> done;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  long long gemm_launches = 0, fft_launches = 0, lowp_launches = 0, oz_launches = 0;
  double gemm_ms = 0, gemm_flops = 0, fft_ms = 0, fft_bytes = 0, lowp_ms = 0, lowp_flops = 0;
  double oz_ms = 0, oz_flops = 0, oz_pair_flops = 0;   // oz_pair_flops: added at launch time
  long long tba_launches = 0;
  double tba_ms = 0, tba_flops = 0;
  long long spmm_launches = 0;
  double spmm_ms = 0, spmm_flops = 0, spmm_bytes = 0;
  double host_setup_ms = 0, graph_build_ms = 0, host_cycles_ms = 0;   // host clock, always collected
  void begin(cudaStream_t st, int kind, double work, double work2 = 0.0);
  void end(cudaStream_t st);
  void collect();  // synchronise the recorded events and accumulate
  void reset();
  void destroy();
};

}  // namespace ts

namespace ts { struct TcOperands; struct SparseOp; struct OzOperands; }

struct ts_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  ts::Workspace ws;
  double* host_scalars = nullptr;  // pinned, 1024 doubles, for small host<->device transfers
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // Operator creation from host arrays: copies done (the caller's arrays are free again), and the
  // DFTs that read the staging buffers done (the next creation may overwrite them).
  cudaEvent_t ev_stage_copied = nullptr, ev_stage_free = nullptr;
  cudaStream_t bstream = nullptr;  // private stream of the batched solver (graph capture)
  std::vector<cudaStream_t> side;  // side streams of the batched solver's parallel branches
  std::map<std::string, int> tune; // launch shapes chosen by the autotuner (tune.cuh), by problem key
  bool tune_loaded = false;        // the on-disk tuning cache (TSTAR_TUNE_CACHE) has been read
  int f64_engine = 0;              // how the current call computes FP64 applications (ts_fp64_engine)
  int oz_digits = 6;               // digits per value of the emulated FP64 product
  int oz_step_digits = 0;          // fewer digits for the current application (0: oz_digits)
  ts::KernelTimer timer;
};

struct ts_op {
  ts_ctx* ctx = nullptr;
  int n = 0, s = 0, p = 0, K = 0;
  double2* Ah = nullptr;   // K slices, column-major n x n complex (FP64)
  double2* Bh = nullptr;   // K slices, column-major s x s complex (FP64)
  float2* Ah32 = nullptr;  // FP32 copies, made on first mixed-precision use
  float2* Bh32 = nullptr;
  ts::TcOperands* tc = nullptr;  // tensor-core operand planes (BF16 or TF32), made on first use
  ts::OzOperands* oz = nullptr;  // BF16 digit planes of the emulated FP64 product, made on first use
  int tc_prec = -1;
  ts::SparseOp* sp = nullptr;    // sparse A (union CSR pattern + Fourier slices of the values)
  double2* Bh_row = nullptr;     // K slices of B_k, row-major (row kernels of TBAS)
  double2* schurT = nullptr;     // K slices: complex Schur factor T of B_k
  double2* schurQ = nullptr;     // K slices: Schur vectors Q of B_k
};

namespace ts {

inline int nyquist_index(int p) { return (p % 2 == 0 && p > 1) ? p / 2 : -1; }
inline int num_slices(int p) { return p / 2 + 1; }

// Memory-kind helper: true for device (or managed) memory of the current device, false for host
// memory; throws TS_ERR_ARG for memory of another device, which a kernel here must not be given.
bool is_device_ptr(const void* p);
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device (once per kernel and
// device; thread-safe).
void set_max_dynamic_smem(const void* func, int bytes);

// ---------------- FFT along mode 3 (fft_tube.cu) ----------------
// Forward: out[k*T + e] = sum_{t<p} in[t*T + e] exp(-2 pi i k t / p), k < K = p/2+1.
// gate (device, may be null) in this and the inverse: when *gate == 0 the kernel returns at once
// (a launched-ahead step of a restart cycle that has already ended).
template <typename Real, typename Cplx>
void rfft_tube(const Real* in, Cplx* out, long long T, int p, cudaStream_t st, const int* gate = nullptr);
// Inverse: out[t*T + e] = (1/p) sum over the full Hermitian spectrum; mode selects the epilogue.
enum IrfftMode { IRFFT_STORE = 0, IRFFT_RESIDUAL = 1 };
// IRFFT_STORE: out = y.  IRFFT_RESIDUAL: out = C - y and partials[b] = block sums of out^2.
template <typename Real, typename Cplx>
void irfft_tube(const Cplx* in, Real* out, long long T, int p, int mode, const Real* C,
                double* partials, cudaStream_t st, const int* gate = nullptr);

// Spectral Krylov basis: out_k = alpha * sqrt(w_k / p) * in_k (inverse: sqrt(p / w_k)) over K = p/2+1
// slices of T entries, w_k = 1 for k = 0 and p/2, else 2; real slices get zero imaginary parts.
// alpha is a device scalar (nullptr: 1).  in and out may alias.
void spec_weight(const double2* in, double2* out, long long T, int p, bool inverse, const double* alpha,
                 cudaStream_t st);

// ---------------- per-slice complex GEMM on CUDA cores, FP64 / FP32 (gemm_simt.cu) ----------------
// Y_k = A1_k B1_k + sgn2 * A2_k B2_k for k < K (phase 2 skipped when L2 == 0);
// slices k == 0 and k == nyq are treated as real (imaginary parts ignored, result imag = 0).
template <typename Cplx>
struct GemmArgs {
  const Cplx* A1; long long sA1; int lda1;
  const Cplx* B1; long long sB1; int ldb1; int L1;
  const Cplx* A2; long long sA2; int lda2;
  const Cplx* B2; long long sB2; int ldb2; int L2;
  Cplx* Y; long long sY; int ldy;
  int M, N, K, nyq;
  double sgn2;
  const int* gate;   // device, may be null: when *gate == 0 the product is skipped (see rfft_tube)
};
using ZGemmArgs = GemmArgs<double2>;
using CGemmArgs = GemmArgs<float2>;
void zgemm_slices_f64(const ZGemmArgs& a, cudaStream_t st);
// Measured FP64 fused multiply-add rate of ctx's device in TFLOP/s (peak.cu); synchronises st.
double fp64_fma_peak_tflops(ts_ctx* ctx, cudaStream_t st);
void cgemm_slices_f32(const CGemmArgs& a, cudaStream_t st);

// ---------------- vector kernels (vec.cu) ----------------
// All reductions write kRedBlocks partial sums; consumers finalise them in a fixed order.
template <typename T> void dot_partials(const T* x, const T* y, long long N, double* partials, cudaStream_t st);
// W -= h * Vi with h = finalize(Pin) (stored to *h_out by block 0); Pout = partials of <Vnext, W>
// (or of <W, W> when Vnext == nullptr).
template <typename T> void mgs_pass(T* W, const T* Vi, const T* Vnext, long long N, const double* Pin,
                                    double* h_out, double* Pout, cudaStream_t st);
// y = x * (*scale)
template <typename T, typename U> void scale_dev(const T* x, U* y, long long N, const double* scale, cudaStream_t st);
// X += sum_{i<k} y[i] * V[i*ldv ...]
template <typename T, typename U> void multi_axpy(U* X, const T* V, long long ldv, long long N, const double* y, int k,
                                                  double alpha_scale, const double* alpha_dev, cudaStream_t st);
// out = sqrt(finalize(P)) to a device scalar; also writes 1/out to out[1].
void finalize_norm(const double* P, double* out, cudaStream_t st);
// a = b - c (elementwise)
template <typename T> void sub3(const T* b, const T* c, T* a, long long N, cudaStream_t st);
// convert
template <typename T, typename U> void convert(const T* x, U* y, long long N, cudaStream_t st);
void fill_zero(void* p, size_t bytes, cudaStream_t st);

// ---------------- small FP64 Hessenberg kernels (small.cu) ----------------
struct KrylovState;  // device-resident, see small.cu
size_t krylov_state_bytes(int m);
void ks_init(void* state, int m, const double* beta_and_inv, cudaStream_t st);
// GMRES (method 0) / FOM (method 1) step j: consumes column j of H (rows 0..j written by MGS) and
// ||W|| from Pnorm partials; writes the estimate and 1/h_{j+1,j} into the state.  Inside a
// graph-captured cycle, `handle` is the conditional handle of step j + 1, which it sets to 0 when the
// cycle stops after this step (breakdown, bad step, estimate <= stop[0] or <= stop[1]).
void ks_step(void* state, int m, int j, int method, const double* Pnorm, cudaStream_t st,
             cudaGraphConditionalHandle handle = 0, const double* stop = nullptr);
// Solve for y over the first k columns; result in the state's y array.
void ks_solve(void* state, int m, int k, int method, cudaStream_t st);
// Inner step j after W = M(V_j), in one cluster launch for short vectors (arnoldi_small_ok(N)): the MGS sweep
// against V_0..V_j (writing column j of H), h_{j+1,j} = ||W||, the ks_step update (same handle and
// stop semantics) and V_{j+1} = W / h_{j+1,j} (always formed; W itself is left as M(V_j)).  The basis
// vectors are V + i ldv.  gate (device, may be null): the kernel returns at once when *gate == 0,
// and sets *gate = 0 where ks_step would end a graph-captured cycle (stop must then be given).
bool arnoldi_small_ok(long long N);
template <typename T>
void arnoldi_small(T* W, T* V, long long ldv, long long N, int j, int m, void* state, int method, cudaStream_t st,
                   cudaGraphConditionalHandle handle = 0, const double* stop = nullptr, int* gate = nullptr);
// Device addresses inside the state block.
double* ks_H(void* state, int m);          // column-major (m+1) x m, H[i + (m+1)*j]
double* ks_y(void* state, int m);
double* ks_est(void* state, int m);        // [0] = estimate, [1] = 1/h_{j+1,j}, [2] = h_{j+1,j}, [3] = flags,
                                           // [4] = steps taken in the cycle
double* ks_hist(void* state, int m);       // the estimate of every step of the cycle (m entries)
double* ks_beta(void* state, int m);       // [0] = beta, [1] = 1/beta

}  // namespace ts
