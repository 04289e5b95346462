// Host-side helpers shared by the entry points: host/device staging and the operator pipeline.
#pragma once
#include "internal.cuh"

namespace ts {

// A read-only tensor argument: used in place when it is device memory, else copied into a
// named workspace buffer on `st`.
struct StagedIn {
  const double* dev = nullptr;
  bool staged = false;
  StagedIn(ts_ctx* ctx, const std::string& name, const double* p, size_t count, cudaStream_t st);
};

// An output (or in/out) tensor argument: written in place when it is device memory, else through
// a workspace buffer that finish() copies back (and synchronises).
struct StagedOut {
  double* dev = nullptr;
  double* host = nullptr;
  size_t count = 0;
  bool staged = false;
  cudaStream_t stream = nullptr;
  StagedOut(ts_ctx* ctx, const std::string& name, double* p, size_t count, bool copy_in, cudaStream_t st);
  void finish();
};

// Sets the FP64 engine of ctx for the duration of one API call.
struct EngineScope {
  ts_ctx* c;
  int e0, d0;
  EngineScope(ts_ctx* ctx, int engine, int digits) : c(ctx), e0(ctx->f64_engine), d0(ctx->oz_digits) {
    c->f64_engine = engine;
    c->oz_digits = digits;
  }
  ~EngineScope() {
    c->f64_engine = e0;
    c->oz_digits = d0;
  }
};

// Y = M(X) in FP64 (rfft -> fused per-slice GEMMs -> irfft).  mode IRFFT_RESIDUAL writes
// Y = C - M(X) and the kRedBlocks partial sums of Y^2 to `partials`.  gate (device, may be null; dense
// operators on the DFMA engine only): when *gate == 0 the three kernels return at once.
void apply_f64(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, int mode, const double* C,
               double* partials, cudaStream_t st, const int* gate = nullptr);

// Yh = A_k Xh_k - Xh_k B_k slice by slice on spectral tensors (K slices of n x s, column-major), on the
// context's FP64 engine: the operator of the spectral Krylov basis (no mode-3 DFTs).
void apply_f64_spectral(ts_ctx* ctx, const ts_op* op, const double2* Xh, double2* Yh, cudaStream_t st);

// Algorithmic FLOPs of one fused slice-GEMM launch (8 per complex, 2 per real multiply-add).
double gemm_flops(int M, int N, int L1, int L2, int K, int nyq);

// Sparse operator: Y = M(X) (real FP64 in and out).
void apply_sparse_f64(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, cudaStream_t st);
void op_prepare_csr(ts_op* op, const int* rowptr, const int* col, const double* val, cudaStream_t st);
ts_status tba_entry(ts_ctx* ctx, const ts_op* op, const double* C, double* X, const ts_solve_opts* opts,
                    ts_solve_info* info, ts_stream stream);
void t_bartels_stewart_dev(ts_ctx* ctx, const double* A, int n, const double* B, int s, int p, const double* C,
                           double* X, cudaStream_t st);

ts_status batched_entry(ts_ctx* ctx, int count, const ts_instance* insts, const ts_solve_opts* opts,
                        ts_solve_info* infos, int* statuses, ts_stream stream);

// Low-precision apply used by the inner solve of mixed precision: X, Y FP32.
void apply_low(ts_ctx* ctx, ts_op* op, int precision, const float* X, float* Y, cudaStream_t st);

}  // namespace ts
