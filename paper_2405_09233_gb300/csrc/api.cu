// Context, workspace, operator setup and the operator-level entry points of libtstar:
// ts_tstar (Definition 2.1 via Algorithm 1) and ts_sylv_apply (Eq. (2)).
#include <cstring>
#include <cstdio>
#include <algorithm>
#include <mutex>
#include <iterator>
#include <unordered_map>
#include "internal.cuh"
#include "apply.cuh"
#include "tc.cuh"
#include "tba.cuh"
#include "oz.cuh"

namespace ts {

void* Workspace::get(const std::string& name, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  Buf& b = bufs[name];
  if (b.bytes < bytes) {
    if (b.ptr) TS_CUDA(cudaFree(b.ptr));
    b.ptr = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.ptr, bytes + kGuardBytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      throw Error{TS_ERR_NOMEM, "workspace '" + name + "': cudaMalloc(" + std::to_string(bytes) +
                                    ") failed: " + cudaGetErrorString(e)};
    }
    TS_CUDA(cudaMemset(static_cast<char*>(b.ptr) + bytes, kGuardByte, kGuardBytes));
    b.bytes = bytes;
  }
  return b.ptr;
}

std::string Workspace::check() const {
  std::vector<unsigned char> h(kGuardBytes);
  for (const auto& kv : bufs) {
    if (!kv.second.ptr) continue;
    TS_CUDA(cudaMemcpy(h.data(), static_cast<const char*>(kv.second.ptr) + kv.second.bytes, kGuardBytes,
                       cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < kGuardBytes; ++i)
      if (h[i] != kGuardByte) return kv.first + " (guard byte " + std::to_string(i) + ")";
  }
  return "";
}

void Workspace::release_all() {
  for (auto& kv : bufs)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  bufs.clear();
}

namespace {
struct OpPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  // Released buffers wait in `pending` until kOpFreeDeferBytes have gathered, an allocation could
  // reuse one of them, an allocation fails, or a context is destroyed: then one device
  // synchronisation covers them all and they move to `cache`, idle blocks by size that later
  // allocations of the same size take without any CUDA call.  Until that synchronisation nothing can
  // reuse memory a kernel may still read.  Blocks beyond kOpCacheKeepBytes go back to the pool.
  std::unordered_map<void*, size_t> sizes;   // every block handed out (live, pending or cached)
  std::vector<void*> pending;
  size_t pending_bytes = 0;
  std::unordered_map<size_t, int> pending_count;              // pending blocks by size
  std::unordered_map<size_t, std::vector<void*>> cache;       // idle blocks by size
  size_t cache_bytes = 0;
};
constexpr size_t kOpFreeDeferBytes = 2ull << 30;
constexpr size_t kOpCacheKeepBytes = 8ull << 30;
std::mutex g_op_pool_mu;
OpPool g_op_pool[64];

int current_device_checked() {
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  TS_REQUIRE(dev >= 0 && dev < 64, "op_malloc: device index out of range");
  return dev;
}

// the pool of device `dev`; the caller holds g_op_pool_mu
OpPool& op_pool_locked(int dev) {
  OpPool& q = g_op_pool[dev];
  if (!q.pool) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    TS_CUDA(cudaMemPoolCreate(&q.pool, &props));
    unsigned long long keep = kOpPoolKeepBytes;
    TS_CUDA(cudaMemPoolSetAttribute(q.pool, cudaMemPoolAttrReleaseThreshold, &keep));
    TS_CUDA(cudaStreamCreateWithFlags(&q.stream, cudaStreamNonBlocking));
  }
  return q;
}

// Return cached blocks to the pool until at most `keep` bytes stay cached (the device is idle:
// called right after a synchronisation, or for blocks no kernel has touched since one).
void trim_cache_locked(OpPool& q, size_t keep) {
  for (auto it = q.cache.begin(); it != q.cache.end() && q.cache_bytes > keep;) {
    std::vector<void*>& v = it->second;
    while (!v.empty() && q.cache_bytes > keep) {
      cudaFreeAsync(v.back(), q.stream);
      q.sizes.erase(v.back());
      q.cache_bytes -= it->first;
      v.pop_back();
    }
    it = v.empty() ? q.cache.erase(it) : std::next(it);
  }
}

// Make every pending buffer idle with one device synchronisation and move it to the cache
// (caller holds the lock).
void flush_pending_locked(OpPool& q) {
  if (q.pending.empty()) return;
  cudaDeviceSynchronize();
  for (void* p : q.pending) {
    const size_t b = q.sizes[p];
    q.cache[b].push_back(p);
    q.cache_bytes += b;
  }
  q.pending.clear();
  q.pending_count.clear();
  q.pending_bytes = 0;
  trim_cache_locked(q, kOpCacheKeepBytes);
}

// An idle cached block of exactly `bytes`, or nullptr (caller holds the lock).
void* take_cached_locked(OpPool& q, size_t bytes) {
  auto it = q.cache.find(bytes);
  if (it == q.cache.end() || it->second.empty()) return nullptr;
  void* p = it->second.back();
  it->second.pop_back();
  q.cache_bytes -= bytes;
  return p;
}

// Allocate from the cache, or from the pool on `st` (on the pool's own stream, synchronised, when
// st_given is false).  A released block of the same size still pending is made idle first (one
// device synchronisation) and reused; a failed pool allocation frees what is pending and cached
// and tries once more.
void* op_alloc_bytes(size_t bytes, bool st_given, cudaStream_t st) {
  const int dev = current_device_checked();
  std::lock_guard<std::mutex> lock(g_op_pool_mu);
  OpPool& q = op_pool_locked(dev);
  bytes = bytes ? (bytes + 255) / 256 * 256 : 256;
  void* p = take_cached_locked(q, bytes);
  if (!p) {
    auto pc = q.pending_count.find(bytes);
    if (pc != q.pending_count.end() && pc->second > 0) {
      flush_pending_locked(q);
      p = take_cached_locked(q, bytes);
    }
  }
  if (p) return p;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, q.pool, st_given ? st : q.stream);
  if (e != cudaSuccess && (!q.pending.empty() || q.cache_bytes > 0)) {
    (void)cudaGetLastError();
    flush_pending_locked(q);
    trim_cache_locked(q, 0);
    cudaStreamSynchronize(q.stream);
    e = cudaMallocFromPoolAsync(&p, bytes, q.pool, st_given ? st : q.stream);
  }
  if (e == cudaSuccess && !st_given) e = cudaStreamSynchronize(q.stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error{TS_ERR_NOMEM, "operator buffer of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e)};
  }
  q.sizes[p] = bytes;
  return p;
}
}  // namespace

void* op_malloc(size_t bytes) { return op_alloc_bytes(bytes, false, nullptr); }

void* op_malloc_on(size_t bytes, cudaStream_t st) { return op_alloc_bytes(bytes, true, st); }

void op_free(void* p) {
  if (!p) return;
  try {   // called from destructors and ts_op_destroy: never throws
    const int dev = current_device_checked();
    std::lock_guard<std::mutex> lock(g_op_pool_mu);
    OpPool& q = op_pool_locked(dev);
    auto it = q.sizes.find(p);
    if (it == q.sizes.end()) return;   // not a block of this pool
    q.pending.push_back(p);
    q.pending_bytes += it->second;
    ++q.pending_count[it->second];
    if (q.pending_bytes >= kOpFreeDeferBytes) flush_pending_locked(q);
  } catch (const Error&) {
  }
}

void op_free_flush() {
  try {
    const int dev = current_device_checked();
    std::lock_guard<std::mutex> lock(g_op_pool_mu);
    if (g_op_pool[dev].pool) flush_pending_locked(g_op_pool[dev]);
  } catch (const Error&) {
  }
}

std::atomic<long long> g_launches{0};
thread_local int g_count_suppress = 0;

void KernelTimer::begin(cudaStream_t st, int kind, double work, double work2) {
  if (!enabled) return;
  if (pool.empty()) {
    cudaEvent_t a, b;
    TS_CUDA(cudaEventCreate(&a));
    TS_CUDA(cudaEventCreate(&b));
    pool.push_back({a, b});
  }
  auto ev = pool.back();
  pool.pop_back();
  TS_CUDA(cudaEventRecord(ev.first, st));
  done.push_back(TimedRegion{ev.first, ev.second, kind, work, work2});
}

void KernelTimer::end(cudaStream_t st) {
  if (!enabled || done.empty()) return;
  TS_CUDA(cudaEventRecord(done.back().b, st));
  if (done.size() >= 256) collect();
}

void KernelTimer::collect() {
  for (auto& r : done) {
    TS_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    TS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    if (r.kind == 0) {
      ++gemm_launches;
      gemm_ms += ms;
      gemm_flops += r.work;
    } else if (r.kind == 2) {
      ++lowp_launches;
      lowp_ms += ms;
      lowp_flops += r.work;
    } else if (r.kind == 3) {
      ++oz_launches;
      oz_ms += ms;
      oz_flops += r.work;
    } else if (r.kind == 4) {
      ++tba_launches;
      tba_ms += ms;
      tba_flops += r.work;
    } else if (r.kind == 5) {
      ++spmm_launches;
      spmm_ms += ms;
      spmm_flops += r.work;
      spmm_bytes += r.work2;
    } else {
      ++fft_launches;
      fft_ms += ms;
      fft_bytes += r.work;
    }
    pool.push_back({r.a, r.b});
  }
  done.clear();
}

void KernelTimer::reset() {
  collect();
  gemm_launches = fft_launches = lowp_launches = oz_launches = tba_launches = spmm_launches = 0;
  gemm_ms = gemm_flops = fft_ms = fft_bytes = lowp_ms = lowp_flops = oz_ms = oz_flops = tba_ms = tba_flops = 0;
  spmm_ms = spmm_flops = spmm_bytes = 0;
  host_setup_ms = graph_build_ms = host_cycles_ms = 0;
  oz_pair_flops = 0;
}

void KernelTimer::destroy() {
  for (auto& r : done) pool.push_back({r.a, r.b});
  done.clear();
  for (auto& e : pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  pool.clear();
}

double gemm_flops(int M, int N, int L1, int L2, int K, int nyq) {
  const int nreal = 1 + (nyq >= 0 ? 1 : 0);
  const double per = (double)M * N * ((double)L1 + L2);
  return per * (8.0 * (K - nreal) + 2.0 * nreal);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return false;
  int dev = -1;
  TS_CUDA(cudaGetDevice(&dev));
  if (attr.device != dev) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "pointer %p is memory of device %d, but the call runs on device %d", p,
                  attr.device, dev);
    throw Error{TS_ERR_ARG, buf};
  }
  return true;
}

void set_max_dynamic_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;   // (kernel, device) -> bytes already allowed
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int& have = done[{func, dev}];
  if (have >= bytes) return;
  TS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  have = bytes;
}

StagedIn::StagedIn(ts_ctx* ctx, const std::string& name, const double* p, size_t count, cudaStream_t st) {
  if (is_device_ptr(p)) {
    dev = p;
  } else {
    double* d = static_cast<double*>(ctx->ws.get(name, count * sizeof(double)));
    TS_CUDA(cudaMemcpyAsync(d, p, count * sizeof(double), cudaMemcpyHostToDevice, st));
    dev = d;
    staged = true;
  }
}

StagedOut::StagedOut(ts_ctx* ctx, const std::string& name, double* p, size_t count, bool copy_in,
                     cudaStream_t st)
    : host(p), count(count), stream(st) {
  if (is_device_ptr(p)) {
    dev = p;
  } else {
    dev = static_cast<double*>(ctx->ws.get(name, count * sizeof(double)));
    if (copy_in) TS_CUDA(cudaMemcpyAsync(dev, p, count * sizeof(double), cudaMemcpyHostToDevice, st));
    staged = true;
  }
}

void StagedOut::finish() {
  if (staged) {
    TS_CUDA(cudaMemcpyAsync(host, dev, count * sizeof(double), cudaMemcpyDeviceToHost, stream));
    TS_CUDA(cudaStreamSynchronize(stream));
  }
}

// Forward DFT of the operator tensors once (§8 setup: A_k, B_k for k <= p/2).
static void op_prepare(ts_op* op, const double* A, const double* B, cudaStream_t st) {
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  ts_ctx* ctx = op->ctx;
  op_alloc_on(op->Ah, sizeof(double2) * (size_t)K * n * n, st);
  op_alloc_on(op->Bh, sizeof(double2) * (size_t)K * s * s, st);
  // Host inputs go through the context's staging buffers: a copy into them waits (on the device)
  // for the DFTs of the previous creation that read them, and the call returns once its own copies
  // are done, so the caller may reuse its arrays while the DFTs run on.
  const bool host_in = !is_device_ptr(A) || !is_device_ptr(B);
  if (host_in) TS_CUDA(cudaStreamWaitEvent(st, ctx->ev_stage_free, 0));
  StagedIn a(ctx, "stage_A", A, (size_t)n * n * p, st);
  StagedIn b(ctx, "stage_B", B, (size_t)s * s * p, st);
  if (host_in) TS_CUDA(cudaEventRecord(ctx->ev_stage_copied, st));
  rfft_tube<double, double2>(a.dev, op->Ah, (long long)n * n, p, st);
  rfft_tube<double, double2>(b.dev, op->Bh, (long long)s * s, p, st);
  if (host_in) {
    TS_CUDA(cudaEventRecord(ctx->ev_stage_free, st));
    TS_CUDA(cudaEventSynchronize(ctx->ev_stage_copied));
  }
}

void apply_f64(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, int mode, const double* C,
               double* partials, cudaStream_t st, const int* gate) {
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  const long long T = (long long)n * s;
  TS_REQUIRE(!gate || (!op->sp && ctx->f64_engine != TS_ENGINE_OZAKI), "apply_f64: gate on an ungated path");
  if (op->sp) {
    // Sparse A: SpMM path; the residual epilogue becomes a subtraction and a fixed-order norm.
    apply_sparse_f64(ctx, op, X, Y, st);
    if (mode == IRFFT_RESIDUAL) {
      sub3<double>(C, Y, Y, T * p, st);
      dot_partials<double>(Y, Y, T * p, partials, st);
    }
    return;
  }
  if (ctx->f64_engine == TS_ENGINE_OZAKI) {
    const int S = ctx->oz_step_digits > 0 && ctx->oz_step_digits < ctx->oz_digits ? ctx->oz_step_digits : ctx->oz_digits;
    apply_f64_oz(ctx, op, X, Y, mode, C, partials, S, ctx->oz_digits, st);
    return;
  }
  double2* Xh = static_cast<double2*>(ctx->ws.get("apply_Xh", sizeof(double2) * (size_t)K * T));
  double2* Yh = static_cast<double2*>(ctx->ws.get("apply_Yh", sizeof(double2) * (size_t)K * T));
  KernelTimer& tm = ctx->timer;
  tm.begin(st, 1, 8.0 * T * p + 16.0 * K * T);
  rfft_tube<double, double2>(X, Xh, T, p, st, gate);
  tm.end(st);
  ZGemmArgs g{};
  g.A1 = op->Ah; g.sA1 = (long long)n * n; g.lda1 = n;
  g.B1 = Xh;     g.sB1 = T;                g.ldb1 = n; g.L1 = n;
  g.A2 = Xh;     g.sA2 = T;                g.lda2 = n;
  g.B2 = op->Bh; g.sB2 = (long long)s * s; g.ldb2 = s; g.L2 = s;
  g.Y = Yh; g.sY = T; g.ldy = n;
  g.M = n; g.N = s; g.K = K; g.nyq = nyquist_index(p); g.sgn2 = -1.0;
  g.gate = gate;
  tm.begin(st, 0, gemm_flops(n, s, n, s, K, g.nyq));
  zgemm_slices_f64(g, st);
  tm.end(st);
  tm.begin(st, 1, 16.0 * K * T + 8.0 * T * p * (mode == IRFFT_RESIDUAL ? 2 : 1));
  irfft_tube<double, double2>(Yh, Y, T, p, mode, C, partials, st, gate);
  tm.end(st);
}

void apply_f64_spectral(ts_ctx* ctx, const ts_op* op, const double2* Xh, double2* Yh, cudaStream_t st) {
  TS_REQUIRE(!op->sp, "spectral Krylov basis: dense operators only");
  if (ctx->f64_engine == TS_ENGINE_OZAKI) {
    const int S = ctx->oz_step_digits > 0 && ctx->oz_step_digits < ctx->oz_digits ? ctx->oz_step_digits : ctx->oz_digits;
    oz_apply_spectral(ctx, op, Xh, Yh, S, ctx->oz_digits, st);
    return;
  }
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  const long long T = (long long)n * s;
  ZGemmArgs g{};
  g.A1 = op->Ah; g.sA1 = (long long)n * n; g.lda1 = n;
  g.B1 = Xh;     g.sB1 = T;                g.ldb1 = n; g.L1 = n;
  g.A2 = Xh;     g.sA2 = T;                g.lda2 = n;
  g.B2 = op->Bh; g.sB2 = (long long)s * s; g.ldb2 = s; g.L2 = s;
  g.Y = Yh; g.sY = T; g.ldy = n;
  g.M = n; g.N = s; g.K = K; g.nyq = nyquist_index(p); g.sgn2 = -1.0;
  KernelTimer& tm = ctx->timer;
  tm.begin(st, 0, gemm_flops(n, s, n, s, K, g.nyq));
  zgemm_slices_f64(g, st);
  tm.end(st);
}

}  // namespace ts

using namespace ts;

#define TS_API_BEGIN try {
#define TS_API_END(ctxp)                              \
  }                                                   \
  catch (const ts::Error& e) {                        \
    if (ctxp) (ctxp)->err = e.msg;                    \
    return e.status;                                  \
  }                                                   \
  catch (const std::bad_alloc&) {                     \
    if (ctxp) (ctxp)->err = "host allocation failed"; \
    return TS_ERR_NOMEM;                              \
  }                                                   \
  catch (...) {                                       \
    if (ctxp) (ctxp)->err = "unknown error";          \
    return TS_ERR_CUDA;                               \
  }

extern "C" {

const char* ts_status_string(ts_status s) {
  switch (s) {
    case TS_OK: return "TS_OK";
    case TS_BREAKDOWN: return "TS_BREAKDOWN";
    case TS_NOT_CONVERGED: return "TS_NOT_CONVERGED";
    case TS_SINGULAR: return "TS_SINGULAR";
    case TS_ERR_ARG: return "TS_ERR_ARG";
    case TS_ERR_CUDA: return "TS_ERR_CUDA";
    case TS_ERR_NOMEM: return "TS_ERR_NOMEM";
    case TS_ERR_NONFINITE: return "TS_ERR_NONFINITE";
    case TS_ERR_TIMEOUT: return "TS_ERR_TIMEOUT";
    case TS_ERR_UNSUPPORTED: return "TS_ERR_UNSUPPORTED";
    case TS_ERR_CORRUPTION: return "TS_ERR_CORRUPTION";
  }
  return "TS_UNKNOWN";
}

ts_status ts_create(ts_ctx** out, int device) {
  if (!out) return TS_ERR_ARG;
  *out = nullptr;
  ts_ctx* ctx = nullptr;
  try {
    ctx = new ts_ctx();
    ctx->device = device;
    TS_CUDA(cudaSetDevice(device));
    TS_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    TS_CUDA(cudaMallocHost(&ctx->host_scalars, 1024 * sizeof(double)));
    TS_CUDA(cudaEventCreate(&ctx->ev0));
    TS_CUDA(cudaEventCreate(&ctx->ev1));
    TS_CUDA(cudaEventCreateWithFlags(&ctx->ev_stage_copied, cudaEventDisableTiming));
    TS_CUDA(cudaEventCreateWithFlags(&ctx->ev_stage_free, cudaEventDisableTiming));
    *out = ctx;
    return TS_OK;
  } catch (const ts::Error& e) {
    if (ctx) {
      if (ctx->host_scalars) cudaFreeHost(ctx->host_scalars);
      delete ctx;
    }
    return e.status;
  } catch (...) {
    delete ctx;
    return TS_ERR_NOMEM;
  }
}

void ts_destroy(ts_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  op_free_flush();   // operator buffers released meanwhile go back to the pool
  ctx->ws.release_all();
  ctx->timer.destroy();
  if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
  for (cudaStream_t q : ctx->side) cudaStreamDestroy(q);
  if (ctx->host_scalars) cudaFreeHost(ctx->host_scalars);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->ev_stage_copied) cudaEventDestroy(ctx->ev_stage_copied);
  if (ctx->ev_stage_free) cudaEventDestroy(ctx->ev_stage_free);
  delete ctx;
}

const char* ts_last_error(const ts_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ts_status ts_tstar(ts_ctx* ctx, const double* A, int n1, int n2, const double* B, int m, int p, double* C,
                   ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_REQUIRE(A && B && C, "ts_tstar: null pointer");
  TS_REQUIRE(n1 >= 1 && n2 >= 1 && m >= 1 && p >= 1, "ts_tstar: sizes must be >= 1");
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int K = num_slices(p);
  StagedIn a(ctx, "tstar_inA", A, (size_t)n1 * n2 * p, st);
  StagedIn b(ctx, "tstar_inB", B, (size_t)n2 * m * p, st);
  StagedOut c(ctx, "tstar_outC", C, (size_t)n1 * m * p, false, st);
  double2* Ah = static_cast<double2*>(ctx->ws.get("tstar_Ah", sizeof(double2) * (size_t)K * n1 * n2));
  double2* Bh = static_cast<double2*>(ctx->ws.get("tstar_Bh", sizeof(double2) * (size_t)K * n2 * m));
  double2* Ch = static_cast<double2*>(ctx->ws.get("tstar_Ch", sizeof(double2) * (size_t)K * n1 * m));
  rfft_tube<double, double2>(a.dev, Ah, (long long)n1 * n2, p, st);
  rfft_tube<double, double2>(b.dev, Bh, (long long)n2 * m, p, st);
  ZGemmArgs g{};
  g.A1 = Ah; g.sA1 = (long long)n1 * n2; g.lda1 = n1;
  g.B1 = Bh; g.sB1 = (long long)n2 * m;  g.ldb1 = n2; g.L1 = n2;
  g.L2 = 0;
  g.Y = Ch; g.sY = (long long)n1 * m; g.ldy = n1;
  g.M = n1; g.N = m; g.K = K; g.nyq = nyquist_index(p); g.sgn2 = 0.0;
  zgemm_slices_f64(g, st);
  irfft_tube<double, double2>(Ch, c.dev, (long long)n1 * m, p, IRFFT_STORE, nullptr, nullptr, st);
  c.finish();
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_op_create_dense(ts_ctx* ctx, const double* A, int n, const double* B, int s, int p, unsigned flags,
                             ts_op** out, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  ts_op* op = nullptr;
  TS_API_BEGIN
  TS_REQUIRE(out, "ts_op_create_dense: null output");
  *out = nullptr;
  TS_REQUIRE(A && B, "ts_op_create_dense: null pointer");
  TS_REQUIRE(n >= 1 && s >= 1 && p >= 1, "ts_op_create_dense: sizes must be >= 1");
  TS_REQUIRE(flags == 0, "ts_op_create_dense: flags must be 0");
  TS_CUDA(cudaSetDevice(ctx->device));
  op = new ts_op();
  op->ctx = ctx;
  op->n = n;
  op->s = s;
  op->p = p;
  op->K = num_slices(p);
  op_prepare(op, A, B, reinterpret_cast<cudaStream_t>(stream));
  *out = op;
  return TS_OK;
  }
  catch (const ts::Error& e) {
    ctx->err = e.msg;
    ts_op_destroy(op);
    return e.status;
  }
  catch (...) {
    ctx->err = "unknown error";
    ts_op_destroy(op);
    return TS_ERR_NOMEM;
  }
}

void ts_op_destroy(ts_op* op) {
  if (!op) return;
  if (op->ctx) cudaSetDevice(op->ctx->device);
  op_free(op->Ah);
  op_free(op->Bh);
  op_free(op->Ah32);
  op_free(op->Bh32);
  if (op->oz) {
    op->oz->release();
    delete op->oz;
  }
  if (op->tc) {
    op->tc->release();
    delete op->tc;
  }
  if (op->sp) {
    op->sp->release();
    delete op->sp;
  }
  op_free(op->Bh_row);
  op_free(op->schurT);
  op_free(op->schurQ);
  delete op;
}

ts_status ts_op_shape(const ts_op* op, int* n, int* s, int* p) {
  if (!op) return TS_ERR_ARG;
  if (n) *n = op->n;
  if (s) *s = op->s;
  if (p) *p = op->p;
  return TS_OK;
}

ts_status ts_sylv_apply(ts_ctx* ctx, const ts_op* op, const double* X, double* Y, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_REQUIRE(op && X && Y, "ts_sylv_apply: null pointer");
  TS_REQUIRE(X != Y, "ts_sylv_apply: Y must not alias X");
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t N = (size_t)op->n * op->s * op->p;
  StagedIn x(ctx, "apply_inX", X, N, st);
  StagedOut y(ctx, "apply_outY", Y, N, false, st);
  apply_f64(ctx, op, x.dev, y.dev, IRFFT_STORE, nullptr, nullptr, st);
  y.finish();
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_sylv_apply_ozaki(ts_ctx* ctx, const ts_op* op, int digits, const double* X, double* Y,
                              ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_REQUIRE(op && X && Y, "ts_sylv_apply_ozaki: null pointer");
  TS_REQUIRE(X != Y, "ts_sylv_apply_ozaki: Y must not alias X");
  TS_REQUIRE(digits == 0 || (digits >= 3 && digits <= 8), "ts_sylv_apply_ozaki: digits must be 3..8 (or 0)");
  if (op->sp) throw Error{TS_ERR_UNSUPPORTED, "ts_sylv_apply_ozaki: dense operators only"};
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t N = (size_t)op->n * op->s * op->p;
  StagedIn x(ctx, "apply_inX", X, N, st);
  StagedOut y(ctx, "apply_outY", Y, N, false, st);
  // An operator already prepared with more digits is used through its leading `digits` digits.
  const int S = digits == 0 ? 6 : digits;
  const int S_op = op->oz && op->oz->S > S ? op->oz->S : S;
  EngineScope scope(ctx, TS_ENGINE_OZAKI, S_op);
  struct StepDigits {
    ts_ctx* c;
    ~StepDigits() { c->oz_step_digits = 0; }
  } step{ctx};
  ctx->oz_step_digits = S;
  apply_f64(ctx, op, x.dev, y.dev, IRFFT_STORE, nullptr, nullptr, st);
  y.finish();
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_op_create_csr(ts_ctx* ctx, int n, int p, const int* rowptr, const int* col, const double* val,
                           const double* B, int s, unsigned flags, ts_op** out, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  ts_op* op = nullptr;
  try {
    TS_REQUIRE(out, "ts_op_create_csr: null output");
    *out = nullptr;
    TS_REQUIRE(rowptr && col && val && B, "ts_op_create_csr: null pointer");
    TS_REQUIRE(n >= 1 && s >= 1 && p >= 1, "ts_op_create_csr: sizes must be >= 1");
    TS_REQUIRE(flags == 0, "ts_op_create_csr: flags must be 0");
    TS_CUDA(cudaSetDevice(ctx->device));
    TS_REQUIRE(!is_device_ptr(rowptr) && !is_device_ptr(col) && !is_device_ptr(val),
               "ts_op_create_csr: the CSR arrays must be host memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    op = new ts_op();
    op->ctx = ctx;
    op->n = n;
    op->s = s;
    op->p = p;
    op->K = num_slices(p);
    op_alloc(op->Bh, sizeof(double2) * (size_t)op->K * s * s);
    TS_CUDA(cudaStreamWaitEvent(st, ctx->ev_stage_free, 0));   // staging buffer free (see op_prepare)
    StagedIn b(ctx, "stage_B", B, (size_t)s * s * p, st);
    rfft_tube<double, double2>(b.dev, op->Bh, (long long)s * s, p, st);
    TS_CUDA(cudaEventRecord(ctx->ev_stage_free, st));
    op_prepare_csr(op, rowptr, col, val, st);
    *out = op;
    return TS_OK;
  } catch (const ts::Error& e) {
    ctx->err = e.msg;
    ts_op_destroy(op);
    return e.status;
  } catch (...) {
    ctx->err = "unknown error";
    ts_op_destroy(op);
    return TS_ERR_NOMEM;
  }
}

ts_status ts_tba_solve(ts_ctx* ctx, const ts_op* op, const double* C, double* X, const ts_solve_opts* opts,
                       ts_solve_info* info, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  return tba_entry(ctx, op, C, X, opts, info, stream);
  TS_API_END(ctx)
}

ts_status ts_t_bartels_stewart(ts_ctx* ctx, const double* A, int n, const double* B, int s, int p, const double* C,
                               double* X, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_REQUIRE(A && B && C && X, "ts_t_bartels_stewart: null pointer");
  TS_REQUIRE(n >= 1 && s >= 1 && p >= 1, "ts_t_bartels_stewart: sizes must be >= 1");
  TS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  StagedIn a(ctx, "tbs_inA", A, (size_t)n * n * p, st);
  StagedIn b(ctx, "tbs_inB", B, (size_t)s * s * p, st);
  StagedIn c(ctx, "tbs_inC", C, (size_t)n * s * p, st);
  StagedOut x(ctx, "tbs_outX", X, (size_t)n * s * p, false, st);
  t_bartels_stewart_dev(ctx, a.dev, n, b.dev, s, p, c.dev, x.dev, st);
  x.finish();
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_sylv_apply_lowp(ts_ctx* ctx, const ts_op* op, int precision, const float* X, float* Y,
                             ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_REQUIRE(op && X && Y, "ts_sylv_apply_lowp: null pointer");
  TS_REQUIRE(X != Y, "ts_sylv_apply_lowp: Y must not alias X");
  TS_REQUIRE(precision == TS_MIXED_FP32 || precision == TS_MIXED_TF32 || precision == TS_MIXED_BF16 ||
                 precision == TS_MIXED_TF32X3,
             "ts_sylv_apply_lowp: precision must be a mixed precision");
  TS_CUDA(cudaSetDevice(ctx->device));
  TS_REQUIRE(is_device_ptr(X) && is_device_ptr(Y), "ts_sylv_apply_lowp: X and Y must be device memory");
  if (op->sp) throw Error{TS_ERR_UNSUPPORTED, "ts_sylv_apply_lowp: sparse operators run in FP64 only"};
  apply_low(ctx, const_cast<ts_op*>(op), precision, X, Y, reinterpret_cast<cudaStream_t>(stream));
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_batched_solve(ts_ctx* ctx, int count, const ts_instance* insts, const ts_solve_opts* opts,
                           ts_solve_info* infos, int* statuses, ts_stream stream) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  return batched_entry(ctx, count, insts, opts, infos, statuses, stream);
  TS_API_END(ctx)
}

ts_status ts_workspace_check(ts_ctx* ctx) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_CUDA(cudaSetDevice(ctx->device));
  TS_CUDA(cudaDeviceSynchronize());
  const std::string bad = ctx->ws.check();
  if (!bad.empty()) {
    ctx->err = "workspace buffer written past its end: " + bad;
    return TS_ERR_CORRUPTION;
  }
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_tune_entries(ts_ctx* ctx, char* buf, size_t cap, size_t* needed) {
  if (!ctx || !needed) return TS_ERR_ARG;
  TS_API_BEGIN
  std::string text;
  for (const auto& kv : ctx->tune) text += kv.first + " " + std::to_string(kv.second) + "\n";
  *needed = text.size() + 1;
  if (buf && cap > 0) {
    const size_t m = std::min(cap - 1, text.size());
    std::memcpy(buf, text.data(), m);
    buf[m] = '\0';
  }
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_stats_enable(ts_ctx* ctx, int enable) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  if (!enable) ctx->timer.collect();
  ctx->timer.enabled = enable != 0;
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_stats_get(ts_ctx* ctx, ts_stats* out) {
  if (!ctx || !out) return TS_ERR_ARG;
  TS_API_BEGIN
  ctx->timer.collect();
  const KernelTimer& t = ctx->timer;
  out->launches = g_launches.load();
  out->gemm_launches = t.gemm_launches;
  out->gemm_ms = t.gemm_ms;
  out->gemm_flops = t.gemm_flops;
  out->fft_launches = t.fft_launches;
  out->fft_ms = t.fft_ms;
  out->fft_bytes = t.fft_bytes;
  out->lowp_launches = t.lowp_launches;
  out->lowp_ms = t.lowp_ms;
  out->lowp_flops = t.lowp_flops;
  out->oz_launches = t.oz_launches;
  out->oz_ms = t.oz_ms;
  out->oz_flops = t.oz_flops;
  out->tba_launches = t.tba_launches;
  out->tba_ms = t.tba_ms;
  out->tba_flops = t.tba_flops;
  out->oz_pair_flops = t.oz_pair_flops;
  out->spmm_launches = t.spmm_launches;
  out->spmm_ms = t.spmm_ms;
  out->spmm_flops = t.spmm_flops;
  out->spmm_bytes = t.spmm_bytes;
  out->host_setup_ms = t.host_setup_ms;
  out->graph_build_ms = t.graph_build_ms;
  out->host_cycles_ms = t.host_cycles_ms;
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_probe_fp64_peak(ts_ctx* ctx, double* tflops, ts_stream stream) {
  if (!ctx || !tflops) return TS_ERR_ARG;
  TS_API_BEGIN
  TS_CUDA(cudaSetDevice(ctx->device));
  *tflops = fp64_fma_peak_tflops(ctx, reinterpret_cast<cudaStream_t>(stream));
  return TS_OK;
  TS_API_END(ctx)
}

ts_status ts_stats_reset(ts_ctx* ctx) {
  if (!ctx) return TS_ERR_ARG;
  TS_API_BEGIN
  ctx->timer.reset();
  g_launches.store(0);
  return TS_OK;
  TS_API_END(ctx)
}

}  // extern "C"
