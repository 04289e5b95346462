/*
 * tstar.h -- C ABI of libtstar: tensor Krylov solvers for the Sylvester tensor
 * equation  M(X) = A*X - X*B = C  under the Kilmer-Martin T-product
 * (Bouyghf, El Guide, El Ichi, "Tensor Krylov subspace methods via the
 * T-product for large Sylvester tensor equations", arXiv:2405.09233).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.  A third-order tensor X in R^{n1 x n2 x p} is stored column-major,
 *   X(i, j, k) at X[i + n1*(j + n2*k)]: frontal slice k is a contiguous
 *   column-major n1 x n2 matrix (the MATLAB layout the paper uses, §2).
 *   In PyTorch this is a contiguous tensor of shape (p, n2, n1).
 * Memory.  Unless stated otherwise a tensor pointer may be device memory or
 *   host memory (pageable or pinned); the library detects which with
 *   cudaPointerGetAttributes and stages host data through its own device
 *   workspace.  The caller owns every pointer it passes; the library never
 *   frees caller memory.  Pointers must stay valid until the call returns.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *   ts_tstar, ts_sylv_apply and ts_op_create_dense with device pointers are
 *   asynchronous on that stream; every other call returns after its work on
 *   the stream completed.
 * Errors.  Every call returns a ts_status; nothing throws, exits or aborts.
 *   ts_last_error(ctx) describes the last failure on that context.
 * Threads.  A ts_ctx (and the ts_op objects made from it) must be used by one
 *   host thread at a time.
 */
#ifndef TSTAR_H
#define TSTAR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ts_stream; /* identical to cudaStream_t */

typedef enum {
  TS_OK = 0,
  TS_BREAKDOWN = 1,      /* Krylov breakdown and the true residual still misses tol; X = best iterate */
  TS_NOT_CONVERGED = 2,  /* iteration budget exhausted; X = last iterate */
  TS_SINGULAR = 3,       /* a small projected system was singular */
  TS_ERR_ARG = -1,       /* invalid argument (sizes, null pointers, tolerances) */
  TS_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  TS_ERR_NOMEM = -3,     /* device or host allocation failed */
  TS_ERR_NONFINITE = -4, /* NaN/Inf met in a residual or norm */
  TS_ERR_TIMEOUT = -5,   /* a bounded device-side wait expired */
  TS_ERR_UNSUPPORTED = -6,
  TS_ERR_CORRUPTION = -7 /* a workspace guard band was overwritten (ts_workspace_check) */
} ts_status;

typedef enum {
  TS_FP64 = 0,        /* every step in FP64 */
  TS_MIXED_FP32 = 1,  /* FP64 refinement around an FP32 inner tGMRES (FP32 CUDA-core GEMMs) */
  TS_MIXED_TF32 = 2,  /* inner GEMMs on tcgen05 tensor cores, TF32 inputs, FP32 accumulation */
  TS_MIXED_BF16 = 3,  /* inner GEMMs on tcgen05 tensor cores, BF16 inputs, FP32 accumulation */
  TS_MIXED_TF32X3 = 4 /* inner GEMMs on tcgen05 in split TF32 (hi*hi + hi*lo + lo*hi): FP32-level
                         accuracy at tensor-core speed */
} ts_precision;

typedef struct ts_ctx ts_ctx; /* device, workspace, scratch, error text */
typedef struct ts_op ts_op;   /* a prepared operator M: Fourier slices of A and B */

/* Create a context on CUDA device `device`.  Allocates nothing on the device
 * until first use.  Returns TS_ERR_CUDA if the device cannot be selected. */
ts_status ts_create(ts_ctx** ctx, int device);
/* Free the context and all of its workspace.  NULL is ignored. */
void ts_destroy(ts_ctx* ctx);
/* Text of the last error on ctx ("" if none).  Valid until the next call on ctx. */
const char* ts_last_error(const ts_ctx* ctx);
/* Static name of a status code. */
const char* ts_status_string(ts_status s);

/* T-product C = A*B (Definition 2.1), evaluated through the block
 * diagonalisation of Eq. (5) as Algorithm 1 does: a real DFT along mode 3
 * that keeps the floor(p/2)+1 non-redundant Fourier slices (the Nyquist slice
 * is computed, not mirrored), one complex matrix product per slice, and the
 * inverse DFT.  A is n1 x n2 x p, B is n2 x m x p, C is n1 x m x p (FP64).
 * n1, n2, m, p >= 1.  C must not alias A or B. */
ts_status ts_tstar(ts_ctx* ctx, const double* A, int n1, int n2, const double* B, int m, int p,
                   double* C, ts_stream stream);

/* Prepare the operator M(X) = A*X - X*B of Eq. (2) from dense A (n x n x p)
 * and B (s x s x p): computes and keeps the Fourier slices A_k, B_k for
 * k = 0..floor(p/2) (FP64; lower-precision copies are made on first use by a
 * mixed-precision solve).  `flags` is reserved (pass 0).  *op is owned by the
 * caller and freed with ts_op_destroy before ts_destroy(ctx).  With A and B in
 * device memory the preparation is asynchronous on `stream`: the operator may
 * be used on that stream at once, on another stream once `stream` has been
 * synchronised.  Host inputs are staged through the context's buffers; the call
 * returns once they have been copied (the caller may then reuse its arrays),
 * and the operator follows the same stream rule. */
ts_status ts_op_create_dense(ts_ctx* ctx, const double* A, int n, const double* B, int s, int p,
                             unsigned flags, ts_op** op, ts_stream stream);
/* Prepare M(X) = A*X - X*B with a sparse A given by its p frontal slices in CSR form (host
 * arrays): slice t (0-based) has row pointers rowptr[t*(n+1) .. t*(n+1)+n], which index the
 * shared arrays col[] and val[] (0-based columns, duplicates summed).  The library forms the
 * union of the p patterns and keeps, per Fourier slice k <= p/2, the complex values of A_k on it
 * (a complex CSR matrix per slice).  B is dense s x s x p (host or device).  Sparse operators run
 * in FP64 (ts_sylv_apply, ts_tgmres_solve, ts_tfom_solve, ts_tba_solve); s <= 64. */
ts_status ts_op_create_csr(ts_ctx* ctx, int n, int p, const int* rowptr, const int* col, const double* val,
                           const double* B, int s, unsigned flags, ts_op** op, ts_stream stream);
/* Free an operator.  NULL is ignored.  Its device buffers return to the library's operator pool
 * once work that may still read them is known to have finished (they are collected and released
 * together after one device synchronisation, at the latest when the context is destroyed). */
void ts_op_destroy(ts_op* op);
/* Sizes of a prepared operator (any output pointer may be NULL). */
ts_status ts_op_shape(const ts_op* op, int* n, int* s, int* p);

/* Y = M(X) = A*X - X*B (Eq. (2)) for X, Y of size n x s x p (FP64).  Y must
 * not alias X.  Asynchronous when X and Y are device pointers. */
ts_status ts_sylv_apply(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, ts_stream stream);

/* Y = M(X) as ts_sylv_apply, with the slice products on the emulated-FP64 tensor-core engine
 * (TS_ENGINE_OZAKI) and `digits` digits per value (3..8; 0 = 6).  Dense operators, p <= any.  The
 * operator's digit planes are built on first use; an operator already holding more digits is used
 * through its leading `digits` digits (an approximation as close as a `digits`-digit expansion,
 * within 0.502 of the last kept digit's unit), a larger count rebuilds them.
 *
 * Mixed-precision solves on this engine with the default digit count (opts.ozaki_digits = 0) form
 * each true residual with the fewest digits the next inner solve needs (at least 3), from the inner
 * estimate of its norm, and form any residual that would end the solve again with all 6 digits; a
 * residual that fails to halve turns this off for the rest of the solve. */
ts_status ts_sylv_apply_ozaki(ts_ctx* ctx, const ts_op* op, int digits, const double* X, double* Y,
                              ts_stream stream);

/* Y = M(X) in a lower precision, the operator of the mixed-precision inner solve: X, Y are
 * FP32 device tensors (n x s x p).  precision TS_MIXED_FP32: FP32 DFT and FP32 CUDA-core slice
 * GEMMs; TS_MIXED_TF32 / TS_MIXED_BF16 / TS_MIXED_TF32X3: the slice GEMMs run on the tcgen05
 * tensor cores with TF32 / BF16 / split-TF32 inputs and FP32 accumulation (p <= 32).  The first call with a precision builds
 * that precision's copy of the operator's Fourier slices.  Asynchronous on `stream`. */
ts_status ts_sylv_apply_lowp(ts_ctx* ctx, const ts_op* op, int precision, const float* X, float* Y,
                             ts_stream stream);

/* How FP64 operator applications are computed.  TS_ENGINE_DFMA: FP64 CUDA-core slice GEMMs.
 * TS_ENGINE_OZAKI: the slice products are emulated on the BF16 tensor cores (Ozaki scheme):
 * every FP64 Fourier slice is split into `ozaki_digits` 8-bit integer digits under one exponent
 * per slice, the digit products are summed exactly in FP32 tensor memory and combined in 64-bit
 * fixed point.  Its error is below 2^(-8 ozaki_digits + 2) max|A_k| max|X_k| per term of the
 * reduction (n + s terms per slice entry), i.e. at FP64 level for 6 digits, in normwise rather than
 * componentwise form.  The mode-3 DFTs stay FP64. */
typedef enum { TS_ENGINE_DFMA = 0, TS_ENGINE_OZAKI = 1 } ts_fp64_engine;

typedef struct {
  int restart;           /* m, the Krylov dimension per cycle (Algorithm 3), 1..256 */
  int max_restarts;      /* Iter_max (Algorithm 3): cycles allowed (per inner solve when mixed) */
  double tol;            /* stop when ||C - M(X)||_F <= tol * ||C||_F (true residual) */
  int precision;         /* ts_precision */
  double inner_tol;      /* mixed precision: relative tolerance of each inner solve (0 = 1e-6 FP32 and split
                            TF32, 1e-3 TF32, 1e-2 BF16) */
  int max_outer;         /* mixed precision: refinement steps allowed (0 = 50) */
  double* history;       /* optional host array: residual estimate after every inner step */
  int history_cap;       /* capacity of history (entries); extra entries are dropped */
  double* true_history;  /* optional host array: true residual norm at every restart / outer step */
  int true_history_cap;
  int fp64_engine;       /* ts_fp64_engine of every FP64 application (the whole FP64 solve, or the true
                            residuals of mixed precision); dense operators of ts_tgmres/ts_tfom only */
  int ozaki_digits;      /* TS_ENGINE_OZAKI: digits per value, 3..8 (0 = 6) */
  int spectral_basis;    /* TS_FP64 tGMRES / tFOM with a dense operator: 1 keeps the Krylov basis in the
                            Fourier domain (the K = p/2 + 1 slices of each basis tensor, slice k scaled by
                            sqrt(w_k / p), w_k = 1 for k = 0 and p/2, else 2, so that the Euclidean inner
                            product of the scaled slices is the tensor inner product of Definition 2.3 by
                            Parseval); every inner step then applies M slice by slice without the two
                            mode-3 DFTs, which only the residuals and the solution update still need.  The
                            same iterates as 0 (the default, real-space basis) up to rounding. */
} ts_solve_opts;

typedef struct {
  int iters;             /* inner Krylov steps taken (all cycles, all outer steps) */
  int cycles;            /* restart cycles run */
  int outer;             /* refinement steps (mixed precision), else 0 */
  int history_len;       /* entries the solver produced for history (may exceed history_cap) */
  int true_history_len;
  int applies_fp64;      /* FP64 operator applications */
  int applies_low;       /* low-precision operator applications */
  double normC;          /* ||C||_F */
  double relres_true;    /* final ||C - M(X)||_F / ||C||_F, computed in FP64 */
  double relres_est;     /* last residual estimate / ||C||_F */
  double ms_total;       /* wall time of the call on the stream (CUDA events), ms */
} ts_solve_info;

/* Fill opts with defaults: restart 20, max_restarts 200, tol 1e-10, FP64. */
void ts_solve_opts_default(ts_solve_opts* opts);

/* Restarted tGMRES(m) (§3.3, Algorithm 3 with the minimum-residual small
 * problem of Proposition 3.4, solved by Givens rotations).  C: right-hand
 * side, X: initial guess on entry, solution on return (both n x s x p, FP64).
 * info may be NULL.  Returns TS_OK when the true relative residual is
 * <= opts->tol, TS_NOT_CONVERGED / TS_BREAKDOWN otherwise (X holds the last
 * iterate).  With opts->precision != TS_FP64 the FP64 tGMRES becomes the outer
 * iterative refinement X += d, d from an inner low-precision tGMRES on
 * M(d) = C - M(X). */
ts_status ts_tgmres_solve(ts_ctx* ctx, const ts_op* op, const double* C, double* X,
                          const ts_solve_opts* opts, ts_solve_info* info, ts_stream stream);

/* Restarted tFOM(m) (§3.2, Algorithm 3 with the Galerkin small problem
 * H_m y = ||R0|| e1 and the estimate of Proposition 3.3).  Arguments and
 * results as ts_tgmres_solve; FP64 only (TS_ERR_UNSUPPORTED otherwise). */
ts_status ts_tfom_solve(ts_ctx* ctx, const ts_op* op, const double* C, double* X,
                        const ts_solve_opts* opts, ts_solve_info* info, ts_stream stream);

/* One instance of a batch: its prepared dense operator, right-hand side and initial guess /
 * solution (device pointers, n x s x p of that operator), and its own relative tolerance
 * (<= 0: opts->tol). */
typedef struct {
  const ts_op* op;
  const double* C;
  double* X;
  double tol;
} ts_instance;

/* Many independent STEs of uneven (n, s, p) solved together by restarted tGMRES(m) (Algorithm 3)
 * in lockstep: every phase of a restart cycle is one launch over all instances (block tables for
 * the streaming phases and the mode-3 DFTs, a cost-ordered (instance, slice, tile) work list for
 * the slice products), device-side masks retire converged instances, and one cycle is captured
 * as a CUDA graph and replayed.  opts->precision: TS_FP64, or a mixed precision -- an FP32 Arnoldi
 * cycle with FP64 residual and update, whose slice products run on FP32 CUDA cores
 * (TS_MIXED_FP32) or on the tcgen05 tensor cores (TS_MIXED_TF32, TS_MIXED_BF16, TS_MIXED_TF32X3);
 * the cycle's inner tolerance is opts->inner_tol (0: 1e-6 for FP32 and split TF32, 1e-3 TF32,
 * 1e-2 BF16).  opts->fp64_engine picks the engine of every FP64 product (the residuals, and the
 * whole cycle of a TS_FP64 batch): TS_ENGINE_DFMA or TS_ENGINE_OZAKI (opts->ozaki_digits).
 * The first call for a batch shape times the candidate launch shapes of its slice products (the
 * autotuner; see ts_tune_entries) before the cycle is captured; later calls reuse the choice.
 * opts->restart <= 128; dense operators with p <= 64.  infos / statuses (count entries each, may
 * be NULL) receive each instance's result; the call returns TS_OK when every instance reached its
 * tolerance, TS_NOT_CONVERGED (or TS_ERR_NONFINITE) otherwise.  Synchronous. */
ts_status ts_batched_solve(ts_ctx* ctx, int count, const ts_instance* insts, const ts_solve_opts* opts,
                           ts_solve_info* infos, int* statuses, ts_stream stream);

/* ts_tstar without allocating: C = A*B exactly as ts_tstar computes it, for callers that cannot
 * allocate device memory when they need a T-product: latency-critical loops that must not risk the
 * device-wide synchronisation a cudaMalloc or cudaFree can cause, and processes whose device memory
 * is already claimed by another allocator (a framework's caching pool), where a fresh cudaMalloc can
 * fail.  The paper has no counterpart; this is a deployment variant of the T-product entry point.
 *
 * Scratch: a fixed array of TS_NOALLOC_MAX_COMPLEX complex doubles (32 MiB) in the library's own
 * device memory, present on every GPU that loads the library until the process exits.  The call
 * needs K*(n1*n2 + n2*m + n1*m) <= TS_NOALLOC_MAX_COMPLEX with K = p/2 + 1, else it returns
 * TS_ERR_ARG without doing anything.  A, B and C must be device memory of the current device
 * (TS_ERR_ARG for host memory or another device's memory); no context is used and nothing is
 * allocated or freed (no cudaMalloc, cudaFree or allocating library routine).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and caches it; make that first call before any stream capture.  All calls
 * share the one array and every call overwrites what it uses (nothing has to start at zero), so
 * calls whose work overlaps on the GPU (other streams, or other host threads) race and must be
 * serialised by the caller.  Asynchronous on `stream`. */
#define TS_NOALLOC_MAX_COMPLEX (2LL * 1024 * 1024)
ts_status ts_tstar_noalloc(const double* A, int n1, int n2, const double* B, int m, int p, double* C,
                           ts_stream stream);

/* Restarted TBAS(m) (§5.2, Algorithm 8): Tubal Block Arnoldi (Algorithm 7) on A with block width
 * s, started from R0 = C - M(X0); the projected equation H_m*Y - Y*B = V_m^T*R0 (Eq. (46)) is
 * solved by t-Bartels-Stewart; X = X0 + V_m*Y; restart until ||C - M(X)||_F <= tol ||C||_F.
 * opts->restart is m (block steps per cycle, m*s <= 12000), opts->max_restarts the cycle budget;
 * history receives the Proposition 5.2 estimate per cycle and true_history the true residual.
 * opts->precision TS_FP64, or TS_MIXED_FP32: the block Krylov basis, the SpMM and the block
 * products of every cycle run in FP32 while the Gram results, H_m, the projected solve, X and the
 * true residual of every restart stay FP64, so the restarts are steps of iterative refinement
 * (info->outer = cycles).  s <= 64.  Arguments and results otherwise as ts_tgmres_solve. */
ts_status ts_tba_solve(ts_ctx* ctx, const ts_op* op, const double* C, double* X, const ts_solve_opts* opts,
                       ts_solve_info* info, ts_stream stream);

/* t-Bartels-Stewart (§4, Algorithm 5) for a small dense STE A*X - X*B = C (A n x n x p,
 * B s x s x p, C and X n x s x p, FP64): per Fourier slice k <= p/2, B_k = Q T Q^H (complex
 * Schur), then column j of X_k Q solves (A_k - t_jj I) z_j = (C_k Q)_j + sum_{i<j} t_ij z_i.
 * Needs K*s*n^2 <= 2^28 complex entries of workspace.  Returns TS_SINGULAR when A_k and B_k
 * share an eigenvalue (Theorem 2.1's condition fails) or the Schur iteration does not converge. */
ts_status ts_t_bartels_stewart(ts_ctx* ctx, const double* A, int n, const double* B, int s, int p,
                               const double* C, double* X, ts_stream stream);

/* Verify the guard bands that follow every workspace buffer of ctx (4 KiB of a fixed pattern
 * each): TS_ERR_CORRUPTION, with the buffer named by ts_last_error, when a kernel wrote past the
 * end of a buffer.  Synchronises the device.  A debugging and testing aid. */
ts_status ts_workspace_check(ts_ctx* ctx);

/* Launch shapes chosen by the autotuner (no counterpart in the paper: the column-tile width of the
 * tcgen05 slice products, and in batched solves the tensor-core product schedule and the column
 * width of the CUDA-core work-list tiles, timed over their candidates on the first call of each shape
 * and precision, then cached in the context; with the environment variable TSTAR_TUNE_CACHE naming a file, also
 * read from and appended to that file, per device).  Writes the context's entries as
 * "<key> <value>\n" lines, NUL-terminated, into `buf` (host memory of `cap` bytes; nothing is
 * written if buf is NULL or cap is 0) and stores the bytes needed, terminator included, in
 * *needed.  TS_ERR_ARG if ctx or needed is NULL; a short buffer is not an error (the text is cut
 * and still NUL-terminated).  No device work. */
ts_status ts_tune_entries(ts_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* Kernel statistics, for measurement.  Launch counts are process-wide (every libtstar kernel
 * launch on any context); kernel timings are per context and only collected while enabled,
 * by CUDA events recorded on the launching stream around each timed launch. */
typedef struct {
  long long launches;      /* libtstar kernels launched since the last ts_stats_reset */
  long long gemm_launches; /* FP64 per-Fourier-slice GEMM launches timed while enabled */
  double gemm_ms;          /* their summed event durations */
  double gemm_flops;       /* their algorithmic FLOPs: 8 per complex and 2 per real multiply-add */
  long long lowp_launches; /* low-precision slice GEMM launches (FP32 CUDA cores or tcgen05) */
  double lowp_ms;
  double lowp_flops;
  long long fft_launches;  /* forward and inverse DFT launches timed while enabled */
  double fft_ms;
  double fft_bytes;        /* their algorithmic HBM bytes (input read + output written once) */
  long long oz_launches;   /* emulated FP64 slice products (TS_ENGINE_OZAKI), digit split included */
  double oz_ms;
  double oz_flops;         /* their algorithmic FLOPs, counted as for gemm_flops */
  long long tba_launches;  /* TBAS tubal Gram and block products (V^H W, W - V H), FP64 */
  double tba_ms;
  double tba_flops;        /* 8 n s^2 per complex slice product */
  double oz_pair_flops;    /* BF16 FLOPs of the emulated products' digit pairs (S(S+1)/2 products per
                              FP64 product, S the digits of each launch) */
  long long spmm_launches; /* sparse products A_k V of TBAS (Algorithm 7 step 3(a)), FP64 or FP32 */
  double spmm_ms;
  double spmm_flops;       /* FLOPs the kernel executes: 8 per stored complex value and block column */
  double spmm_bytes;       /* algorithmic bytes: values, column indices, row pointers, V read and W
                              written once */
  double host_setup_ms;    /* host clock (always collected): batched solves' preparation before the
                              first residual (operator copies, work lists, tensor maps, tuning) */
  double graph_build_ms;   /* capture and instantiation of restart-cycle graphs (batched and small
                              single-instance solves) */
  double host_cycles_ms;   /* batched solves: the restart cycles (graph replays and the host's look at
                              each cycle's residuals) */
} ts_stats;

/* Enable (1) or disable (0) per-kernel event timing on ctx. */
ts_status ts_stats_enable(ts_ctx* ctx, int enable);
/* Read the statistics (synchronises the recorded events). */
ts_status ts_stats_get(ts_ctx* ctx, ts_stats* out);
/* Zero the statistics and the process-wide launch counter. */
ts_status ts_stats_reset(ts_ctx* ctx);

/* The FP64 roof of ctx's device, measured (no counterpart in the paper: the denominator of the
 * rooflines reported for FP64 kernels on CUDA cores).  Launches on `stream` a kernel in which every
 * thread runs 8 independent fused multiply-add chains on registers (4 CTAs of 256 threads per SM;
 * one short untimed launch, then one timed with CUDA events, ~30 ms on a GB300) and stores
 * 2 x (multiply-adds) / seconds / 1e12 in *tflops (host memory).  Uses ~1.2 MB of the context's
 * workspace.  TS_ERR_ARG if ctx or tflops is NULL.  Synchronous. */
ts_status ts_probe_fp64_peak(ts_ctx* ctx, double* tflops, ts_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* TSTAR_H */
