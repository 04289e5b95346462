// Low-precision operator application for the inner solve of mixed-precision refinement:
// W = M(V) with V, W in FP32 storage.  TS_MIXED_FP32 uses FP32 CUDA-core slice GEMMs.
#include "internal.cuh"
#include "apply.cuh"
#include "tc.cuh"

namespace ts {

void ensure_f32_operator(ts_op* op, cudaStream_t st) {
  if (op->Ah32) return;
  const size_t na = (size_t)op->K * op->n * op->n, nb = (size_t)op->K * op->s * op->s;
  op_alloc_on(op->Ah32, sizeof(float2) * na, st);
  op_alloc_on(op->Bh32, sizeof(float2) * nb, st);
  convert<double, float>(reinterpret_cast<const double*>(op->Ah), reinterpret_cast<float*>(op->Ah32),
                         (long long)(2 * na), st);
  convert<double, float>(reinterpret_cast<const double*>(op->Bh), reinterpret_cast<float*>(op->Bh32),
                         (long long)(2 * nb), st);
}

void apply_low(ts_ctx* ctx, ts_op* op, int precision, const float* X, float* Y, cudaStream_t st) {
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  const long long T = (long long)n * s;
  float2* Yh = static_cast<float2*>(ctx->ws.get("low_Yh", sizeof(float2) * (size_t)K * T));
  KernelTimer& tm = ctx->timer;
  if (precision == TS_MIXED_BF16 || precision == TS_MIXED_TF32 || precision == TS_MIXED_TF32X3) {
    tc_apply(ctx, op, precision, X, Yh, st);
    tm.begin(st, 1, 8.0 * K * T + 4.0 * T * p);
    irfft_tube<float, float2>(Yh, Y, T, p, IRFFT_STORE, nullptr, nullptr, st);
    tm.end(st);
    return;
  }
  ensure_f32_operator(op, st);
  float2* Xh = static_cast<float2*>(ctx->ws.get("low_Xh", sizeof(float2) * (size_t)K * T));
  tm.begin(st, 1, 4.0 * T * p + 8.0 * K * T);
  rfft_tube<float, float2>(X, Xh, T, p, st);
  tm.end(st);
  CGemmArgs g{};
  g.A1 = op->Ah32; g.sA1 = (long long)n * n; g.lda1 = n;
  g.B1 = Xh;       g.sB1 = T;                g.ldb1 = n; g.L1 = n;
  g.A2 = Xh;       g.sA2 = T;                g.lda2 = n;
  g.B2 = op->Bh32; g.sB2 = (long long)s * s; g.ldb2 = s; g.L2 = s;
  g.Y = Yh; g.sY = T; g.ldy = n;
  g.M = n; g.N = s; g.K = K; g.nyq = nyquist_index(p); g.sgn2 = -1.0;
  tm.begin(st, 2, gemm_flops(n, s, n, s, K, g.nyq));
  cgemm_slices_f32(g, st);
  tm.end(st);
  tm.begin(st, 1, 8.0 * K * T + 4.0 * T * p);
  irfft_tube<float, float2>(Yh, Y, T, p, IRFFT_STORE, nullptr, nullptr, st);
  tm.end(st);
}

}  // namespace ts
