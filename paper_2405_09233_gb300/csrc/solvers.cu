// Restarted tGMRES(m) and tFOM(m) (Algorithm 3), and their mixed-precision form.
//
// One cycle:  R = C - M(X) (FP64, fused into the inverse FFT with the norm partials),
//             V_1 = R / ||R||, then for j = 1..m: W = M(V_j); MGS against V_1..V_j
//             (Algorithm 2); h_{j+1,j} = ||W||; Givens (tGMRES) or Hessenberg LU (tFOM) on the
//             device gives the residual estimate; stop early when it reaches the tolerance;
//             V_{j+1} = W / h_{j+1,j}.  Then y, X += V_k (*) y, and the true residual.
// The host reads 4 doubles per inner step (estimate, 1/h, h, flags) to decide whether to stop --
// except for small problems, which are bound by launch latency and by that look at every step.
// Vectors of at most 65536 entries run everything after W = M(V_j) in one launch (arnoldi_small, a
// thread-block cluster), and
// on the FP64 DFMA engine (real basis, dense operator) a cycle's steps are launched ahead in chunks
// behind a device gate that the step ending the cycle closes, so the host looks once per chunk.
// Other problems of at most kGraphCycleMaxN unknowns run, from their second cycle on, each restart
// cycle as one CUDA graph in which step j is the body of a conditional (IF) node (step j + 1's node
// nested inside it) and the step's Givens / Hessenberg kernel switches the remaining steps off on the
// device, so the host looks once per cycle.  All forms run the same kernels in the same order, so
// they give identical results.
//
// Mixed precision: the Arnoldi cycle (basis, W, operator) runs in FP32 storage with a FP32 or
// tensor-core operator, while R = C - M(X), the small problem, and X += ||R|| (V (*) y) stay in
// FP64.  Every cycle is thus one step of iterative refinement with an inner tGMRES whose own
// stopping tolerance is inner_tol relative to ||R||; only the residual needs an FP64 apply.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <vector>
#include "internal.cuh"
#include "apply.cuh"
#include "cycle_graph.cuh"

namespace ts {

namespace {

// Problems of at most this many unknowns run their restart cycles, from the second one on, as CUDA
// graphs (unless the environment sets TSTAR_NO_GRAPH_CYCLE=1, or statistics are being collected:
// event timing is not allowed inside the conditional bodies).
constexpr long long kGraphCycleMaxN = 1ll << 20;

// One restart cycle (Algorithm 2 up to m steps) as an executable graph: a prologue (Givens state
// reset, V_1 = R / ||R||), then m conditional (IF) nodes, node j holding inner step j and, nested at
// its end, node j + 1; the kernels of each part are counted once while captured, so replays can be
// counted as the steps they ran.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  long long prologue_kernels = 0;
  std::vector<long long> step_kernels;
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

struct Result {
  ts_status status = TS_NOT_CONVERGED;
};

template <typename T>
T* basis_ptr(T* V, long long N, int i) {
  return V + (long long)i * N;
}

void apply_basis(ts_ctx* ctx, ts_op* op, int prec, const double* x, double* y, cudaStream_t st) {
  (void)prec;
  apply_f64(ctx, op, x, y, IRFFT_STORE, nullptr, nullptr, st);
}
void apply_basis(ts_ctx* ctx, ts_op* op, int prec, const float* x, float* y, cudaStream_t st) {
  apply_low(ctx, op, prec, x, y, st);
}

// Digits for an emulated-FP64 residual that the next inner solve needs only to relative accuracy
// ~inner_tol, when its norm is expected near rho ||C||.  An S-digit product of an output entry
// carries n + s terms, each off by about 256^-S of its operands' largest entries, so its error is
// taken as 10 (n + s) 256^-S ||C|| (a factor 10 for cancellation between C and M(X)); the fewest
// S whose error stays below a tenth of inner_tol rho ||C|| is used, at least 3 and at most S_full.
int progressive_digits(double rho, double inner_tol, int n, int s, int S_full) {
  const double need = 0.1 * inner_tol * rho;
  for (int S = 3; S < S_full; ++S)
    if (10.0 * (n + s) * std::pow(256.0, -S) <= need) return S;
  return S_full;
}

template <typename T>
ts_status krylov_solve(ts_ctx* ctx, ts_op* op, const double* C, double* X, const ts_solve_opts& o,
                       ts_solve_info& info, cudaStream_t st, int method, int prec) {
  const long long N = (long long)op->n * op->s * op->p;
  const int m = o.restart;
  const bool mixed = prec != TS_FP64;
  const int max_cycles = mixed ? (o.max_outer > 0 ? o.max_outer : 50) : o.max_restarts;
  // Default inner tolerance: a little above what the inner operator's rounding lets the inner
  // tGMRES resolve (FP32 ~1e-7, TF32 ~5e-4, BF16 ~4e-3 relative).
  const double inner_default =
      (prec == TS_MIXED_FP32 || prec == TS_MIXED_TF32X3) ? 1e-6 : (prec == TS_MIXED_TF32 ? 1e-3 : 1e-2);
  const double inner_tol = mixed ? (o.inner_tol > 0 ? o.inner_tol : inner_default) : 0.0;

  // Spectral basis (FP64, dense operators): basis tensors are the K scaled Fourier slices, 2 K n s
  // doubles each, on which the tensor inner product is the Euclidean one (Parseval).
  const bool spectral = sizeof(T) == 8 && o.spectral_basis != 0;
  const long long Ts = (long long)op->n * op->s;
  const long long Nb = spectral ? 2ll * op->K * Ts : N;      // length of a basis vector, in T
  T* V = static_cast<T*>(ctx->ws.get("krylov_V", sizeof(T) * (size_t)(m + 1) * Nb));
  T* W = static_cast<T*>(ctx->ws.get("krylov_W", sizeof(T) * (size_t)Nb));
  double2* Rh = spectral ? static_cast<double2*>(ctx->ws.get("krylov_Rh", sizeof(double2) * (size_t)op->K * Ts))
                         : nullptr;
  double* R = static_cast<double*>(ctx->ws.get("krylov_R", sizeof(double) * (size_t)N));
  double* P = static_cast<double*>(ctx->ws.get("krylov_P", sizeof(double) * 3 * kRedBlocks));
  double* Pp[2] = {P, P + kRedBlocks};
  double* P2 = P + 2 * kRedBlocks;
  double* sc = static_cast<double*>(ctx->ws.get("krylov_scalars", sizeof(double) * 64));
  ctx->host_scalars[13] = 1.0;
  TS_CUDA(cudaMemcpyAsync(sc + 12, ctx->host_scalars + 13, sizeof(double), cudaMemcpyHostToDevice, st));
  void* state = ctx->ws.get("krylov_state", krylov_state_bytes(m));
  double* hs = ctx->host_scalars;
  int* tc_err = static_cast<int*>(ctx->ws.get("tc_err", sizeof(int) * 4));
  const bool ozaki = ctx->f64_engine == TS_ENGINE_OZAKI;
  if (mixed || ozaki) TS_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int) * 4, st));
  // Progressive digits: mixed precision on the emulated engine with the default digit count.
  bool progressive = mixed && ozaki && o.ozaki_digits == 0;
  struct StepDigitsReset {   // an exception never leaves reduced digits behind in the context
    ts_ctx* c;
    ~StepDigitsReset() { c->oz_step_digits = 0; }
  } step_digits_reset{ctx};

  int hist_len = 0, true_len = 0;
  auto push_hist = [&](double v) {
    if (o.history && hist_len < o.history_cap) o.history[hist_len] = v;
    ++hist_len;
  };
  auto push_true = [&](double v) {
    if (o.true_history && true_len < o.true_history_cap) o.true_history[true_len] = v;
    ++true_len;
  };

  // ||C|| and the initial residual R = C - M(X0) (Algorithm 3, step 3).  M(0) = 0 exactly, so
  // for X0 = 0 the residual is C itself and the FP64 apply is skipped.
  dot_partials<double>(C, C, N, P2, st);
  finalize_norm(P2, sc + 0, st);
  dot_partials<double>(X, X, N, P2, st);
  finalize_norm(P2, sc + 4, st);
  TS_CUDA(cudaMemcpyAsync(hs, sc, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  const double normC = hs[0];
  double res;
  if (hs[4] == 0.0) {
    TS_CUDA(cudaMemcpyAsync(R, C, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, st));
    TS_CUDA(cudaMemcpyAsync(sc + 2, sc + 0, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    res = normC;
  } else {
    apply_f64(ctx, op, X, R, IRFFT_RESIDUAL, C, P2, st);
    ++info.applies_fp64;
    finalize_norm(P2, sc + 2, st);
    TS_CUDA(cudaMemcpyAsync(hs, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaStreamSynchronize(st));
    res = hs[2];
  }
  info.normC = normC;
  push_true(res);
  ts_status status = TS_NOT_CONVERGED;
  double last_est = res;

  auto finish = [&](ts_status s) {
    info.history_len = hist_len;
    info.true_history_len = true_len;
    info.relres_true = normC > 0 ? res / normC : res;
    info.relres_est = normC > 0 ? last_est / normC : last_est;
    return s;
  };

  if (!std::isfinite(res) || !std::isfinite(normC)) return finish(TS_ERR_NONFINITE);
  if (normC == 0.0) {
    // C = 0: the solution is X = 0 (M is invertible under Theorem 2.1's condition).
    fill_zero(X, sizeof(double) * (size_t)N, st);
    res = 0.0;
    return finish(TS_OK);
  }
  if (res <= o.tol * normC) return finish(TS_OK);

  // Inner step j of a cycle: W = M(V_j), the MGS sweep (fused with the next dot), the Givens /
  // Hessenberg update (which, inside a graph, also decides whether the cycle goes on), and
  // V_{j+1} = W / h_{j+1,j} when `scale_next` (the graph always forms it; unused after the last step).
  double* stop_dev = sc + 8;   // [tol ||C||, inner threshold or -1] for the graph's stopping test
  const bool small_steps = arnoldi_small_ok(Nb);   // the post-apply part of a step is one launch
  // Small FP64 problems on the DFMA engine: a cycle's steps are launched ahead, kAheadChunk at a
  // time, without waiting for each step's estimate; a step that ends the cycle closes a device gate
  // and the kernels of the steps launched after it return at once.  (Each step of such a problem
  // is a few short kernels; the host round trip per step had cost about as much as they do.)
  const char* no_ahead = std::getenv("TSTAR_NO_LAUNCH_AHEAD");
  const bool ahead = small_steps && sizeof(T) == 8 && !mixed && !spectral && !op->sp && !ozaki &&
                     !ctx->timer.enabled && !(no_ahead && no_ahead[0] == '1');
  constexpr int kAheadChunk = 8;
  int* gate = ahead ? static_cast<int*>(ctx->ws.get("krylov_gate", sizeof(int))) : nullptr;
  auto inner_step = [&](int j, cudaGraphConditionalHandle handle, bool scale_next, cudaStream_t q) {
    if constexpr (sizeof(T) == 8) {
      if (spectral)   // W = M(V_j) slice by slice: the scaling commutes with the per-slice operator
        apply_f64_spectral(ctx, op, reinterpret_cast<const double2*>(basis_ptr(V, Nb, j)),
                           reinterpret_cast<double2*>(W), q);
      else if (ahead)
        apply_f64(ctx, op, basis_ptr(V, Nb, j), W, IRFFT_STORE, nullptr, nullptr, q, gate);
      else
        apply_basis(ctx, op, prec, basis_ptr(V, Nb, j), W, q);     // W = M(V_j)
    } else {
      apply_basis(ctx, op, prec, basis_ptr(V, Nb, j), W, q);
    }
    if (small_steps) {   // sweep, norm, Givens / Hessenberg update and V_{j+1} in one launch
      arnoldi_small<T>(W, V, Nb, Nb, j, m, state, method, q, handle, stop_dev, ahead ? gate : nullptr);
      return;
    }
    dot_partials<T>(basis_ptr(V, Nb, 0), W, Nb, Pp[0], q);
    for (int i = 0; i <= j; ++i) {                                  // MGS sweep, fused with the next dot
      const T* Vn = i < j ? basis_ptr(V, Nb, i + 1) : nullptr;
      mgs_pass<T>(W, basis_ptr(V, Nb, i), Vn, Nb, Pp[i & 1], ks_H(state, m) + i + (size_t)(m + 1) * j,
                  Pp[(i + 1) & 1], q);
    }
    ks_step(state, m, j, method, Pp[(j + 1) & 1], q, handle, stop_dev);
    if (scale_next) scale_dev<T, T>(W, basis_ptr(V, Nb, j + 1), Nb, ks_est(state, m) + 1, q);   // V_{j+1}
  };
  // V_1 = R / ||R|| (in the spectral basis: the scaled Fourier slices of R, over ||R||)
  auto init_v1 = [&](cudaStream_t q) {
    if constexpr (sizeof(T) == 8) {
      if (spectral) {
        rfft_tube<double, double2>(R, Rh, Ts, op->p, q);
        spec_weight(Rh, reinterpret_cast<double2*>(basis_ptr(V, Nb, 0)), Ts, op->p, false, sc + 3, q);
        return;
      }
    }
    scale_dev<double, T>(R, basis_ptr(V, Nb, 0), N, sc + 3, q);
  };
  const char* no_graph = std::getenv("TSTAR_NO_GRAPH_CYCLE");
  const bool graph_allowed =
      !ahead && !ctx->timer.enabled && N <= kGraphCycleMaxN && !(no_graph && no_graph[0] == '1');
  std::unique_ptr<CycleGraph> cg;
  // Built when a second cycle starts: a one-cycle solve would not earn the graph back, and by then every
  // workspace buffer, operator copy and tuning choice a step needs exists (nothing may allocate or
  // tune inside a capture).
  auto build_cycle_graph = [&]() {
    // captured on and replayed from the context's private stream (a capture cannot start on the
    // legacy default stream), ordered after the caller's stream by an event
    if (!ctx->bstream) TS_CUDA(cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking));
    TS_CUDA(cudaStreamSynchronize(st));
    cg.reset(new CycleGraph());
    const cudaStream_t gst = ctx->bstream;
    const long long launches0 = g_launches.load();
    const auto build_t0 = std::chrono::steady_clock::now();
    try {
      auto counted = [&](auto&& record) {   // kernels a piece records, from the launch counter
        const long long c0 = g_launches.load();
        record();
        return g_launches.load() - c0;
      };
      NestedCycleCounts cnt;
      cg->graph = build_nested_cycle(
          m, gst,
          [&](cudaStream_t q) {
            return counted([&] {
              ks_init(state, m, sc + 2, q);
              init_v1(q);
            });
          },
          [&](int j, cudaGraphConditionalHandle next, cudaStream_t q) {
            return counted([&] { inner_step(j, next, j + 1 < m, q); });
          },
          [&](cudaStream_t) { return 0ll; }, cnt);
      cg->prologue_kernels = cnt.prologue;
      cg->step_kernels = cnt.steps;
      const auto inst_t0 = std::chrono::steady_clock::now();
      TS_CUDA(cudaGraphInstantiate(&cg->exec, cg->graph, 0));
      const char* dbg = std::getenv("TSTAR_DEBUG_GRAPH");
      if (dbg && dbg[0] == '1')
        std::fprintf(stderr, "tstar: cycle graph of %d steps: capture %.3f ms, instantiate %.3f ms\n", m,
                     std::chrono::duration<double, std::milli>(inst_t0 - build_t0).count(),
                     std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - inst_t0).count());
    } catch (const Error& e) {
      // not capturable here (the apply path of this precision did something a capture forbids):
      // keep the per-step form (TSTAR_DEBUG_GRAPH=1 reports why on stderr)
      const char* dbg = std::getenv("TSTAR_DEBUG_GRAPH");
      if (dbg && dbg[0] == '1') std::fprintf(stderr, "tstar: restart-cycle graph not used: %s\n", e.msg.c_str());
      cg.reset();
    }
    g_launches.fetch_sub(g_launches.load() - launches0);   // captured launches did not run
    ctx->timer.graph_build_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - build_t0).count();
  };

  for (int cycle = 0; cycle < max_cycles; ++cycle) {
    int k = 0;
    double flags = 0.0;
    if (cycle == 1 && graph_allowed) build_cycle_graph();
    if (cg) {
      double* hstop = hs + 64;
      hstop[0] = o.tol * normC;
      hstop[1] = mixed ? inner_tol * res : -1.0;
      const cudaStream_t gst = ctx->bstream;
      TS_CUDA(cudaEventRecord(ctx->ev1, st));                  // the cycle follows the caller's stream
      TS_CUDA(cudaStreamWaitEvent(gst, ctx->ev1, 0));
      TS_CUDA(cudaMemcpyAsync(stop_dev, hstop, 2 * sizeof(double), cudaMemcpyHostToDevice, gst));
      TS_CUDA(cudaGraphLaunch(cg->exec, gst));
      double* hest = hs + 96;
      double* hhist = hs + 256;
      TS_CUDA(cudaMemcpyAsync(hest, ks_est(state, m), 8 * sizeof(double), cudaMemcpyDeviceToHost, gst));
      TS_CUDA(cudaMemcpyAsync(hhist, ks_hist(state, m), m * sizeof(double), cudaMemcpyDeviceToHost, gst));
      TS_CUDA(cudaStreamSynchronize(gst));                     // later work on the caller's stream follows it
      k = (int)hest[4];
      flags = hest[3];
      long long ran = cg->prologue_kernels;
      for (int j = 0; j < k; ++j) {
        ran += cg->step_kernels[j];
        push_hist(hhist[j]);
      }
      count_launch(ran);
      info.iters += k;
      if (mixed) info.applies_low += k; else info.applies_fp64 += k;
      last_est = k > 0 ? hhist[k - 1] : last_est;
    } else if (ahead) {
      double* hstop = hs + 64;
      hstop[0] = o.tol * normC;
      hstop[1] = -1.0;
      TS_CUDA(cudaMemcpyAsync(stop_dev, hstop, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
      TS_CUDA(cudaMemsetAsync(gate, 1, sizeof(int), st));    // non-zero: the cycle goes on
      ks_init(state, m, sc + 2, st);
      init_v1(st);
      double* hest = hs + 96;
      double* hhist = hs + 256;
      int launched = 0;
      while (launched < m) {
        const int upto = std::min(m, launched + kAheadChunk);
        for (int j = launched; j < upto; ++j) inner_step(j, 0, true, st);
        launched = upto;
        TS_CUDA(cudaMemcpyAsync(hest, ks_est(state, m), 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
        TS_CUDA(cudaStreamSynchronize(st));
        k = (int)hest[4];
        if (k < launched || (int)hest[3] != 0 || hest[0] <= o.tol * normC) break;   // the cycle has ended
      }
      TS_CUDA(cudaMemcpyAsync(hhist, ks_hist(state, m), m * sizeof(double), cudaMemcpyDeviceToHost, st));
      TS_CUDA(cudaStreamSynchronize(st));
      flags = hest[3];
      for (int j = 0; j < k; ++j) push_hist(hhist[j]);
      info.iters += k;
      info.applies_fp64 += k;
      last_est = k > 0 ? hhist[k - 1] : last_est;
    } else {
      ks_init(state, m, sc + 2, st);
      init_v1(st);
      for (int j = 0; j < m; ++j) {
        inner_step(j, 0, false, st);
        if (mixed) ++info.applies_low; else ++info.applies_fp64;
        TS_CUDA(cudaMemcpyAsync(hs + 8, ks_est(state, m), 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        TS_CUDA(cudaStreamSynchronize(st));
        const double est = hs[8];
        flags = hs[11];
        k = j + 1;
        ++info.iters;
        last_est = est;
        push_hist(est);
        const bool broke = ((int)flags & 1) != 0;
        const bool bad = ((int)flags & 6) != 0;
        if (bad || broke || est <= o.tol * normC || (mixed && est <= inner_tol * res)) break;
        if (!small_steps) scale_dev<T, T>(W, basis_ptr(V, Nb, j + 1), Nb, ks_est(state, m) + 1, st);  // V_{j+1}
      }
    }
    ++info.cycles;
    // An expired tensor-core wait makes this cycle's products meaningless, whatever they produced:
    // checked before the flags those products may have set.
    if ((mixed && prec != TS_MIXED_FP32) || ozaki) {
      int e = 0;
      TS_CUDA(cudaMemcpy(&e, tc_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (e != 0) throw Error{TS_ERR_TIMEOUT, "tensor-core kernel wait expired (code " + std::to_string(e) + ")"};
    }
    if ((int)flags & 2) {
      status = TS_SINGULAR;
      break;
    }
    if ((int)flags & 4) {
      status = TS_ERR_NONFINITE;
      break;
    }
    ks_solve(state, m, k, method, st);
    if (spectral) {
      // X += V_k (*) y: combine the spectral basis, undo the slice scaling, back to real space
      double2* D = Rh;
      double* Dr = static_cast<double*>(ctx->ws.get("krylov_Dr", sizeof(double) * (size_t)N));
      fill_zero(D, sizeof(double2) * (size_t)op->K * Ts, st);
      multi_axpy<double, double>(reinterpret_cast<double*>(D), reinterpret_cast<const double*>(V), Nb, Nb,
                                 ks_y(state, m), k, 1.0, nullptr, st);
      spec_weight(D, D, Ts, op->p, true, nullptr, st);
      irfft_tube<double, double2>(D, Dr, Ts, op->p, IRFFT_STORE, nullptr, nullptr, st);
      multi_axpy<double, double>(X, Dr, N, N, sc + 12, 1, 1.0, nullptr, st);   // sc[12] = 1
    } else {
      multi_axpy<T, double>(X, V, N, N, ks_y(state, m), k, 1.0, nullptr, st);   // X = X0 + V_k (*) y
    }
    // True residual.  With progressive digits it is first formed with the fewest digits its next
    // use needs; a residual that would end the solve is formed again with every digit.
    const double res_prev = res;
    int S_step = progressive ? progressive_digits(std::max(last_est, o.tol * normC) / normC, inner_tol, op->n,
                                                  op->s, ctx->oz_digits)
                             : 0;
    for (;;) {
      ctx->oz_step_digits = S_step;
      apply_f64(ctx, op, X, R, IRFFT_RESIDUAL, C, P2, st);
      ctx->oz_step_digits = 0;
      ++info.applies_fp64;
      finalize_norm(P2, sc + 2, st);
      TS_CUDA(cudaMemcpyAsync(hs, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
      TS_CUDA(cudaStreamSynchronize(st));
      res = hs[2];
      if (S_step == 0 || S_step >= ctx->oz_digits || !(res <= o.tol * normC)) break;
      S_step = 0;
    }
    // a residual that did not at least halve: stop trusting reduced digits for this solve
    if (S_step != 0 && !(res <= 0.5 * res_prev)) progressive = false;
    push_true(res);
    if (!std::isfinite(res)) {
      status = TS_ERR_NONFINITE;
      break;
    }
    if (res <= o.tol * normC) {
      status = TS_OK;
      break;
    }
    if (((int)flags & 1) && !mixed) {
      status = TS_BREAKDOWN;
      break;
    }
  }
  if (mixed) info.outer = info.cycles;
  return finish(status);
}

ts_status solve_entry(ts_ctx* ctx, const ts_op* cop, const double* C, double* X, const ts_solve_opts* opts,
                      ts_solve_info* info_out, ts_stream stream, int method) {
  ts_op* op = const_cast<ts_op*>(cop);  // lower-precision operator copies are cached on first use
  TS_REQUIRE(op && C && X && opts, "solve: null pointer");
  const ts_solve_opts& o = *opts;
  TS_REQUIRE(o.restart >= 1 && o.restart <= 256, "solve: restart must be in 1..256");
  TS_REQUIRE(o.max_restarts >= 1, "solve: max_restarts must be >= 1");
  TS_REQUIRE(o.tol > 0.0 && std::isfinite(o.tol), "solve: tol must be positive");
  TS_REQUIRE(o.precision >= TS_FP64 && o.precision <= TS_MIXED_TF32X3, "solve: unknown precision");
  TS_REQUIRE(!(o.history && o.history_cap < 0) && !(o.true_history && o.true_history_cap < 0),
             "solve: negative history capacity");
  if (method == 1 && o.precision != TS_FP64)
    throw Error{TS_ERR_UNSUPPORTED, "tFOM runs in FP64 only"};
  if (op->sp && o.precision != TS_FP64)
    throw Error{TS_ERR_UNSUPPORTED, "sparse operators run in FP64 only"};
  TS_REQUIRE(o.fp64_engine == TS_ENGINE_DFMA || o.fp64_engine == TS_ENGINE_OZAKI, "solve: unknown fp64_engine");
  TS_REQUIRE(o.ozaki_digits == 0 || (o.ozaki_digits >= 3 && o.ozaki_digits <= 8), "solve: ozaki_digits must be 3..8");
  if (op->sp && o.fp64_engine != TS_ENGINE_DFMA)
    throw Error{TS_ERR_UNSUPPORTED, "the emulated FP64 engine takes dense operators only"};
  TS_REQUIRE(o.spectral_basis == 0 || o.spectral_basis == 1, "solve: spectral_basis must be 0 or 1");
  if (o.spectral_basis && (o.precision != TS_FP64 || op->sp))
    throw Error{TS_ERR_UNSUPPORTED, "the spectral Krylov basis is for FP64 solves with dense operators"};
  EngineScope scope(ctx, o.fp64_engine, o.ozaki_digits == 0 ? 6 : o.ozaki_digits);
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ts_solve_info info{};
  TS_CUDA(cudaEventRecord(ctx->ev0, st));
  const size_t N = (size_t)op->n * op->s * op->p;
  StagedIn c(ctx, "solve_inC", C, N, st);
  StagedOut x(ctx, "solve_ioX", X, N, true, st);
  ts_status s;
  if (o.precision == TS_FP64)
    s = krylov_solve<double>(ctx, op, c.dev, x.dev, o, info, st, method, o.precision);
  else
    s = krylov_solve<float>(ctx, op, c.dev, x.dev, o, info, st, method, o.precision);
  x.finish();
  TS_CUDA(cudaEventRecord(ctx->ev1, st));
  TS_CUDA(cudaEventSynchronize(ctx->ev1));
  float ms = 0.f;
  TS_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  info.ms_total = ms;
  if (info_out) *info_out = info;
  return s;
}

}  // namespace

}  // namespace ts

using namespace ts;

extern "C" {

void ts_solve_opts_default(ts_solve_opts* o) {
  if (!o) return;
  *o = ts_solve_opts{};
  o->restart = 20;
  o->max_restarts = 200;
  o->tol = 1e-10;
  o->precision = TS_FP64;
  o->inner_tol = 0.0;
  o->max_outer = 0;
}

ts_status ts_tgmres_solve(ts_ctx* ctx, const ts_op* op, const double* C, double* X, const ts_solve_opts* opts,
                          ts_solve_info* info, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  try {
    return solve_entry(ctx, op, C, X, opts, info, stream, 0);
  } catch (const ts::Error& e) {
    ctx->err = e.msg;
    return e.status;
  } catch (...) {
    ctx->err = "unknown error";
    return TS_ERR_CUDA;
  }
}

ts_status ts_tfom_solve(ts_ctx* ctx, const ts_op* op, const double* C, double* X, const ts_solve_opts* opts,
                        ts_solve_info* info, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  try {
    return solve_entry(ctx, op, C, X, opts, info, stream, 1);
  } catch (const ts::Error& e) {
    ctx->err = e.msg;
    return e.status;
  } catch (...) {
    ctx->err = "unknown error";
    return TS_ERR_CUDA;
  }
}

}  // extern "C"
