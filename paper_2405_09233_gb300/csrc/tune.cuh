// Autotuner of launch shapes (tile widths of the tcgen05 slice products): the first call for a key
// times every candidate on the stream (one untimed launch, then two timed with events) and caches
// the fastest in the context; later calls with the key reuse it.  Tuning synchronises the stream,
// so callers tune before any capture; a call made while the stream is being captured gets the
// first candidate and tunes nothing.
//
// When the environment variable TSTAR_TUNE_CACHE names a file, choices persist across processes:
// the file holds one "<device tag> <key> <value>" line per choice (the tag is the device's name,
// compute capability and SM count, spaces replaced), the first tuning call of a context reads the
// lines of its own device, and every new choice is appended.  Unreadable or malformed lines are
// ignored; a file that cannot be opened for appending only loses persistence.
#pragma once
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <string>
#include <vector>
#include "internal.cuh"

namespace ts {

inline std::string tune_device_tag(const ts_ctx* ctx) {
  cudaDeviceProp pr;
  TS_CUDA(cudaGetDeviceProperties(&pr, ctx->device));
  std::string tag = std::string(pr.name) + "/sm" + std::to_string(pr.major * 10 + pr.minor) + "/" +
                    std::to_string(pr.multiProcessorCount);
  for (char& c : tag)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  return tag;
}

inline void tune_load(ts_ctx* ctx) {
  ctx->tune_loaded = true;
  const char* path = std::getenv("TSTAR_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  const std::string tag = tune_device_tag(ctx);
  std::string line;
  int c;
  auto take = [&]() {
    const size_t a = line.find(' '), b = line.rfind(' ');
    if (a != std::string::npos && b > a && line.compare(0, a, tag) == 0 && a == tag.size()) {
      char* end = nullptr;
      const long v = std::strtol(line.c_str() + b + 1, &end, 10);
      if (end && *end == '\0' && v > 0 && v <= 4096) ctx->tune[line.substr(a + 1, b - a - 1)] = (int)v;
    }
    line.clear();
  };
  while ((c = std::fgetc(f)) != EOF) {
    if (c == '\n') take();
    else if (c != '\r') line.push_back((char)c);
  }
  if (!line.empty()) take();
  std::fclose(f);
}

inline void tune_store(const ts_ctx* ctx, const std::string& key, int value) {
  const char* path = std::getenv("TSTAR_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  const std::string line = tune_device_tag(ctx) + " " + key + " " + std::to_string(value) + "\n";
  std::fwrite(line.data(), 1, line.size(), f);
  std::fclose(f);
}

inline int tune_pick(ts_ctx* ctx, const std::string& key, const std::vector<int>& candidates,
                     const std::function<void(int)>& run, cudaStream_t st) {
  if (!ctx->tune_loaded) tune_load(ctx);
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) {
    for (int c : candidates)
      if (c == it->second) return c;
  }
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
  ctx->tune[key] = best;
  tune_store(ctx, key, best);
  return best;
}

}  // namespace ts
