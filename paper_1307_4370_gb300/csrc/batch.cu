// Batched SDMM: many independent problems of uneven sizes advanced together.
//
// Each problem keeps its own context (tables, scratch) and SDMM state.  One
// batch iteration is captured once as a single CUDA graph with one branch per
// problem: the branches fork from one event and join into one, so a launch of
// the graph runs one SDMM iteration (Algorithm 1 steps 5-9) of every problem,
// and the GPU overlaps the small kernels of different problems.  The graph
// bakes in each state's buffers and options; a step re-captures it when a
// state's graph key (step_graph_key) differs from the one it was built with.  (A
// persistent kernel with software grid barriers between the phases was the
// other candidate; on this GPU its barriers cost more than the graph's kernel
// boundaries, so the batch is a graph.)
#include <new>
#include <vector>

#include "common.cuh"

struct purify_batch {
  int device = -1;
  std::vector<purify_ctx*> ctxs;
  std::vector<purify_sdmm_state*> sts;
  std::vector<purify::GraphKey> keys;  // per problem: what its branch was captured with
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;  // kernels in one batch iteration
};

namespace {

using namespace purify;

void release(purify_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

int capture(purify_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const unsigned long long l0 = g_launches.load(std::memory_order_relaxed);
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) return PURIFY_E_CUDA;
  int rc = check_cuda(cudaEventRecord(b->fork, b->origin));
  for (size_t i = 0; rc == PURIFY_OK && i < b->ctxs.size(); ++i) {
    rc = check_cuda(cudaStreamWaitEvent(b->branch[i], b->fork, 0));
    if (rc == PURIFY_OK) rc = enqueue_sdmm_step(b->ctxs[i], b->sts[i], b->branch[i]);
    if (rc == PURIFY_OK) rc = check_cuda(cudaEventRecord(b->done[i], b->branch[i]));
    if (rc == PURIFY_OK) rc = check_cuda(cudaStreamWaitEvent(b->origin, b->done[i], 0));
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->origin, &graph);
  if (rc != PURIFY_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != PURIFY_OK ? rc : PURIFY_E_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    b->exec = nullptr;
    cudaGetLastError();
    return PURIFY_E_CUDA;
  }
  b->launches = (int)(g_launches.load(std::memory_order_relaxed) - l0);
  g_launches.fetch_sub((unsigned long long)b->launches, std::memory_order_relaxed);  // capture is not a launch
  for (size_t i = 0; i < b->sts.size(); ++i) b->keys[i] = step_graph_key(b->sts[i]);
  return PURIFY_OK;
}

}  // namespace

extern "C" {

static int purify_batch_create_impl(purify_batch** out, purify_ctx* const* ctxs, purify_sdmm_state* const* states,
                        int32_t count) {
  if (!out) return PURIFY_E_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || !states || count < 1) return PURIFY_E_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || !states[i] || states[i]->ctx != ctxs[i]) return PURIFY_E_INVALID_ARG;
    if (ctxs[i]->device != ctxs[0]->device) return PURIFY_E_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || states[j] == states[i]) return PURIFY_E_INVALID_ARG;  // scratch is per context
  }
  purify_batch* b = new (std::nothrow) purify_batch();
  if (!b) return PURIFY_E_ALLOC;
  b->device = ctxs[0]->device;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  b->ctxs.assign(ctxs, ctxs + count);
  b->sts.assign(states, states + count);
  b->keys.assign(count, purify::GraphKey{});
  b->branch.assign(count, nullptr);
  b->done.assign(count, nullptr);
  int rc = check_cuda(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
  if (rc == PURIFY_OK) rc = check_cuda(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  for (int i = 0; rc == PURIFY_OK && i < count; ++i) {
    rc = check_cuda(cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking));
    if (rc == PURIFY_OK) rc = check_cuda(cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming));
  }
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  if (rc != PURIFY_OK) {
    release(b);
    return rc == PURIFY_E_CUDA ? PURIFY_E_ALLOC : rc;
  }
  *out = b;
  return PURIFY_OK;
}

int purify_batch_create(purify_batch** out, purify_ctx* const* ctxs, purify_sdmm_state* const* states,
                        int32_t count) {
  // host containers may throw; no exception crosses the C ABI
  try {
    return purify_batch_create_impl(out, ctxs, states, count);
  } catch (const std::bad_alloc&) {
    return PURIFY_E_ALLOC;
  }
}

int purify_batch_step(purify_batch* b, int32_t iters, purify_stream_t stream) {
  if (!b || iters < 0) return PURIFY_E_INVALID_ARG;
  if (iters == 0) return PURIFY_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  int rc = PURIFY_OK;
  bool stale = !b->exec;
  for (size_t i = 0; i < b->sts.size(); ++i)
    if (b->keys[i] != step_graph_key(b->sts[i])) stale = true;  // cg_iters, data format, prior,
                                                                 // blocks, beam or an import changed
  if (stale) rc = capture(b);
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; rc == PURIFY_OK && k < iters; ++k) {
    rc = check_cuda(cudaGraphLaunch(b->exec, s));
    if (rc == PURIFY_OK) g_launches.fetch_add((unsigned long long)b->launches, std::memory_order_relaxed);
  }
  if (rc == PURIFY_OK)
    for (purify_sdmm_state* st : b->sts) st->iters += iters;
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  return rc;
}

int purify_batch_size(const purify_batch* b, int32_t* count, int32_t* kernels_per_iteration) {
  if (!b) return PURIFY_E_INVALID_ARG;
  if (count) *count = (int32_t)b->ctxs.size();
  if (kernels_per_iteration) *kernels_per_iteration = b->launches;
  return PURIFY_OK;
}

void purify_batch_destroy(purify_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  const int dev = b->device;
  release(b);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

}  // extern "C"
