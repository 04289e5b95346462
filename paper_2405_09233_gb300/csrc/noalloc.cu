// ts_tstar_noalloc: the T-product C = A*B with no memory allocation at call time.
//
// Some callers cannot allocate device memory when they need a T-product: latency-critical serving
// loops that must not hit an allocation (cudaMalloc and cudaFree can synchronise the whole device),
// and hosts whose device memory is already claimed by another allocator (a framework's caching
// pool), so that a fresh cudaMalloc can fail.  For them this entry point keeps its scratch -- the
// Fourier slices of A, B and C -- in a fixed-size array in the library's own device memory, loaded
// with the library and held by every GPU that loads it until the process exits.  It calls no
// cudaMalloc, cudaFree or allocating routine.
//
// Host code cannot pass the array's name to a kernel: in host code that name is a host-side
// stand-in, not a device address.  The device address is looked up once per device with
// cudaGetSymbolAddress (on the first call made while that device is current, so that first call
// belongs before any stream capture) and cached.
#include <mutex>
#include "internal.cuh"

namespace ts {
namespace {

constexpr long long kNoallocComplex = 2ll * 1024 * 1024;   // 2 Mi complex doubles = 32 MiB

__device__ __align__(256) double2 g_noalloc_scratch[kNoallocComplex];

constexpr int kMaxDevices = 64;
double2* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up on first use).
double2* scratch_on_current_device(int dev) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    TS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = static_cast<double2*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace
}  // namespace ts

using namespace ts;

extern "C" ts_status ts_tstar_noalloc(const double* A, int n1, int n2, const double* B, int m, int p, double* C,
                                      ts_stream stream) {
  try {
    if (!A || !B || !C || n1 < 1 || n2 < 1 || m < 1 || p < 1) return TS_ERR_ARG;
    const long long K = num_slices(p);
    const long long need = K * ((long long)n1 * n2 + (long long)n2 * m + (long long)n1 * m);
    if (need > kNoallocComplex) return TS_ERR_ARG;   // beyond TS_NOALLOC_MAX_COMPLEX
    if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C)) return TS_ERR_ARG;
    int dev = 0;
    TS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return TS_ERR_UNSUPPORTED;
    double2* scratch = scratch_on_current_device(dev);
    // The three spectra are fully overwritten below, so nothing has to be cleared first.
    double2* Ah = scratch;
    double2* Bh = Ah + K * n1 * n2;
    double2* Ch = Bh + K * n2 * m;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rfft_tube<double, double2>(A, Ah, (long long)n1 * n2, p, st);
    rfft_tube<double, double2>(B, Bh, (long long)n2 * m, p, st);
    ZGemmArgs g{};
    g.A1 = Ah; g.sA1 = (long long)n1 * n2; g.lda1 = n1;
    g.B1 = Bh; g.sB1 = (long long)n2 * m;  g.ldb1 = n2; g.L1 = n2;
    g.L2 = 0;
    g.Y = Ch; g.sY = (long long)n1 * m; g.ldy = n1;
    g.M = n1; g.N = m; g.K = (int)K; g.nyq = nyquist_index(p); g.sgn2 = 0.0;
    zgemm_slices_f64(g, st);
    irfft_tube<double, double2>(Ch, C, (long long)n1 * m, p, IRFFT_STORE, nullptr, nullptr, st);
    return TS_OK;
  } catch (const ts::Error& e) {
    return e.status;
  } catch (...) {
    return TS_ERR_CUDA;
  }
}
