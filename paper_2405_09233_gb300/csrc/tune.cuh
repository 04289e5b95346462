// Autotuner of launch shapes (tile widths of the tcgen05 slice products): the first call for a key
// times every candidate on the stream (one untimed launch, then two timed with events) and caches
// the fastest in the context; later calls with the key reuse it.  Tuning synchronises the stream,
// so callers tune before any capture; a call made while the stream is being captured gets the
// first candidate and tunes nothing.
#pragma once
#include <functional>
#include <string>
#include <vector>
#include "internal.cuh"

namespace ts {

inline int tune_pick(ts_ctx* ctx, const std::string& key, const std::vector<int>& candidates,
                     const std::function<void(int)>& run, cudaStream_t st) {
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return it->second;
  if (candidates.size() == 1) return ctx->tune[key] = candidates[0];
  // inside a capture nothing can be timed: take the first candidate and leave the key untuned
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TS_CUDA(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return candidates[0];
  // events of its own: the context's are timing the enclosing API call
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  TS_CUDA(cudaEventCreate(&ev.a));
  TS_CUDA(cudaEventCreate(&ev.b));
  int best = candidates[0];
  float best_ms = 1e30f;
  for (int c : candidates) {
    run(c);
    TS_CUDA(cudaEventRecord(ev.a, st));
    run(c);
    run(c);
    TS_CUDA(cudaEventRecord(ev.b, st));
    TS_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    TS_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  return ctx->tune[key] = best;
}

}  // namespace ts
