// A restart cycle of a Krylov solver as one CUDA graph whose inner steps run only while needed.
//
//   [prologue] -> IF(h_0) { step 0 ; IF(h_1) { step 1 ; ... IF(h_{m-1}) { step m-1 } ... } } -> [epilogue]
//
// Step j + 1's conditional node sits at the end of step j's body, and every node has a handle of its
// own (a handle drives exactly one node), created on the graph that contains the node with the
// default value 1.  Step j is captured with the handle of step j + 1 (0 for the last step); a kernel
// of step j sets that handle to 0 (cudaGraphSetConditional) to end the cycle after step j, which
// skips the node and every step nested below it.  The epilogue follows the outermost node.
// Conditional bodies may hold kernels, memsets, memcopies and further conditionals, but no event
// records, so nothing inside a step may time itself with events.
#pragma once
#include <vector>
#include "internal.cuh"

namespace ts {

struct NestedCycleCounts {
  long long prologue = 0, epilogue = 0;
  std::vector<long long> steps;   // kernels of each step, as the lambdas report them
};

// pro(st), epi(st): record the prologue / epilogue on `st` and return their kernel counts;
// step(j, next, st): records inner step j and returns its kernel count.  The graph is owned by the
// caller.  Any error ends the capture in progress and is rethrown.
template <typename Pro, typename Step, typename Epi>
cudaGraph_t build_nested_cycle(int m, cudaStream_t st, const Pro& pro, const Step& step, const Epi& epi,
                               NestedCycleCounts& cnt) {
  cudaGraph_t g = nullptr;
  TS_CUDA(cudaGraphCreate(&g, 0));
  cnt = NestedCycleCounts{};
  try {
    cudaGraph_t cur = g, captured = nullptr;
    cudaGraphNode_t outer = nullptr;
    cudaGraphConditionalHandle handle;
    TS_CUDA(cudaGraphConditionalHandleCreate(&handle, cur, 1, cudaGraphCondAssignDefault));
    TS_CUDA(cudaStreamBeginCaptureToGraph(st, cur, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cnt.prologue = pro(st);
    for (int j = 0; j < m; ++j) {
      cudaStreamCaptureStatus cst;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      TS_CUDA(cudaStreamGetCaptureInfo(st, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
      std::vector<cudaGraphNode_t> prev(deps, deps + ndeps);
      TS_CUDA(cudaStreamEndCapture(st, &captured));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = handle;
      np.conditional.type = cudaGraphCondTypeIf;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      TS_CUDA(cudaGraphAddNode(&node, cur, prev.data(), nullptr, prev.size(), &np));
      if (j == 0) outer = node;
      cur = np.conditional.phGraph_out[0];
      cudaGraphConditionalHandle next = 0;
      if (j + 1 < m) TS_CUDA(cudaGraphConditionalHandleCreate(&next, cur, 1, cudaGraphCondAssignDefault));
      TS_CUDA(cudaStreamBeginCaptureToGraph(st, cur, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      cnt.steps.push_back(step(j, next, st));
      handle = next;
    }
    TS_CUDA(cudaStreamEndCapture(st, &captured));
    TS_CUDA(cudaStreamBeginCaptureToGraph(st, g, &outer, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    cnt.epilogue = epi(st);
    TS_CUDA(cudaStreamEndCapture(st, &captured));
  } catch (...) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t dropped = nullptr;   // g or a body graph owned by its conditional node
      cudaStreamEndCapture(st, &dropped);
    }
    (void)cudaGetLastError();
    cudaGraphDestroy(g);
    throw;
  }
  return g;
}

}  // namespace ts
