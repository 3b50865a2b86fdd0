// Batched solves of many independent Poisson problems of uneven shapes and boundary conditions.
//
// The problems are spread over a small pool of internal streams (greedy balancing by point count,
// largest first) that fork from and join back into the caller's stream through events, so the whole
// batch is asynchronous on the caller's stream and can be captured into one CUDA graph whose
// branches run concurrently.  Each problem runs the same pass kernels as a single solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "plan.cuh"

struct cans_batch_s {
  int count = 0;
  std::vector<cans_plan_t> plans;
  std::vector<size_t> ws_off;  // byte offset of each problem's workspace
  size_t ws_bytes = 0;
  std::vector<int> stream_of;  // problem -> internal stream
  std::vector<int> order;      // launch order (largest first)
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
};

// Per-problem device status after a solve: the checks of the plan's status word (cans::solve_check:
// incompatible singular right-hand side, non-finite norms, a stalled refinement sweep, and with
// opts.verify the final residual against tol), written for this problem alone.
__global__ void batch_status_kernel(const double* acc, cans::SolveCheck c, int* status) {
  if (threadIdx.x == 0) *status = cans::solve_check(acc, c);
}

static int batch_solve_impl(cans_batch_t B, const double* const* f, double* const* p, void* workspace,
                            void* cuda_stream, int* status) {
  if (!B || !f || !p) return CANS_ERR_ARG;
  if (B->ws_bytes > 0 && (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))) return CANS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int ns = (int)B->streams.size();
  if (cudaEventRecord(B->fork, st) != cudaSuccess) return CANS_ERR_CUDA;
  for (int s = 0; s < ns; ++s)
    if (cudaStreamWaitEvent(B->streams[s], B->fork, 0) != cudaSuccess) return CANS_ERR_CUDA;
  for (int q : B->order) {
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    void* w = (B->ws_bytes > 0) ? ws + B->ws_off[q] : nullptr;
    cudaStream_t sq = B->streams[B->stream_of[q]];
    const int rc = cans_poisson_solve(B->plans[q], f[q], p[q], w, sq, nullptr);
    if (rc != CANS_OK) return rc;
    if (status) {
      const cans_plan_s* P = B->plans[q];
      batch_status_kernel<<<1, 32, 0, sq>>>(P->acc_d, cans::solve_check_args(P, P->singular, P->opts.verify != 0),
                                            status + q);
      if (cudaGetLastError() != cudaSuccess) return CANS_ERR_CUDA;
    }
  }
  for (int s = 0; s < ns; ++s) {
    if (cudaEventRecord(B->joins[s], B->streams[s]) != cudaSuccess) return CANS_ERR_CUDA;
    if (cudaStreamWaitEvent(st, B->joins[s], 0) != cudaSuccess) return CANS_ERR_CUDA;
  }
  return CANS_OK;
}

// A batch's host bookkeeping (workspace offsets, launch order, stream assignment) with its stream and
// event slots left empty.
static int cans_batch_create_shape(int count, const cans_plan_t* plans, int nstreams, cans_batch_t* out) {
  if (count < 1 || !plans || !out || nstreams < 1 || nstreams > 64) return CANS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return CANS_ERR_ARG;
  cans_batch_s* B = new (std::nothrow) cans_batch_s();
  if (!B) return CANS_ERR_ARG;
  B->count = count;
  B->plans.assign(plans, plans + count);
  B->ws_off.resize(count);
  for (int i = 0; i < count; ++i) {
    size_t b = 0;
    cans_poisson_workspace_size(plans[i], &b);
    B->ws_off[i] = B->ws_bytes;
    B->ws_bytes += (b + 255) & ~size_t(255);
  }
  // greedy balance: largest problem first onto the least loaded stream
  B->order.resize(count);
  for (int i = 0; i < count; ++i) B->order[i] = i;
  auto pts = [&](int i) { return (double)plans[i]->n[0] * plans[i]->n[1] * plans[i]->n[2]; };
  std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) { return pts(a) > pts(b); });
  const int ns = std::min(nstreams, count);
  std::vector<double> load(ns, 0.0);
  B->stream_of.resize(count);
  for (int qi = 0; qi < count; ++qi) {
    const int q = B->order[qi];
    int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    // a plan's device accumulators are per plan: problems sharing a plan share a stream
    for (int pj = 0; pj < qi; ++pj)
      if (plans[B->order[pj]] == plans[q]) s = B->stream_of[B->order[pj]];
    B->stream_of[q] = s;
    load[s] += pts(q);
  }
  B->streams.assign(ns, nullptr);
  B->joins.assign(ns, nullptr);
  *out = B;
  return CANS_OK;
}

extern "C" {

int cans_batch_create(int count, const cans_plan_t* plans, int nstreams, cans_batch_t* out) {
  if (count < 1 || !plans || !out || nstreams < 1 || nstreams > 64) return CANS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return CANS_ERR_ARG;
  cans_batch_t B = nullptr;
  const int rc = cans_batch_create_shape(count, plans, nstreams, &B);
  if (rc != CANS_OK) return rc;
  const int ns = (int)B->streams.size();
  bool ok = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int s = 0; s < ns && ok; ++s) {
    ok = cudaStreamCreateWithFlags(&B->streams[s], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->joins[s], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cans_batch_destroy(B);
    return CANS_ERR_CUDA;
  }
  *out = B;
  return CANS_OK;
}

int cans_batch_workspace_size(cans_batch_t B, size_t* bytes) {
  if (!B || !bytes) return CANS_ERR_ARG;
  *bytes = B->ws_bytes;
  return CANS_OK;
}

int cans_batch_solve(cans_batch_t B, const double* const* f, double* const* p, void* workspace, void* cuda_stream) {
  return batch_solve_impl(B, f, p, workspace, cuda_stream, nullptr);
}

int cans_batch_destroy(cans_batch_t B) {
  if (!B) return CANS_ERR_ARG;
  for (cudaStream_t s : B->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->joins)
    if (e) cudaEventDestroy(e);
  if (B->fork) cudaEventDestroy(B->fork);
  delete B;
  return CANS_OK;
}

int cans_poisson_batched_workspace_size(int count, const cans_plan_t* plans, size_t* bytes) {
  if (count < 1 || !plans || !bytes) return CANS_ERR_ARG;
  size_t tot = 0;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) return CANS_ERR_ARG;
    size_t b = 0;
    cans_poisson_workspace_size(plans[i], &b);
    tot += (b + 255) & ~size_t(255);
  }
  *bytes = tot;
  return CANS_OK;
}

int cans_poisson_solve_batched(int count, const cans_plan_t* plans, const double* const* f, double* const* p,
                               void* workspace, void* cuda_stream, int* device_status) {
  if (count < 1 || !plans || !f || !p) return CANS_ERR_ARG;
  // The internal streams and events come from a per-device pool created by the first call on the
  // device, so later calls only record events and launch work (and can be captured into a graph).
  constexpr int kPoolStreams = 8, kMaxDev = 64;
  struct Pool {
    cudaStream_t streams[kPoolStreams];
    cudaEvent_t fork, joins[kPoolStreams];
    bool ready;
  };
  static Pool pools[kMaxDev] = {};
  static std::mutex pool_lock;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return CANS_ERR_CUDA;
  {
    std::lock_guard<std::mutex> g(pool_lock);
    Pool& q = pools[dev];
    if (!q.ready) {
      bool ok = cudaEventCreateWithFlags(&q.fork, cudaEventDisableTiming) == cudaSuccess;
      for (int i = 0; i < kPoolStreams && ok; ++i)
        ok = cudaStreamCreateWithFlags(&q.streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&q.joins[i], cudaEventDisableTiming) == cudaSuccess;
      if (!ok) return CANS_ERR_CUDA;  // (a partial pool is kept; its handles are valid)
      q.ready = true;
    }
  }
  cans_batch_t B = nullptr;
  int rc = cans_batch_create_shape(count, plans, kPoolStreams, &B);  // host bookkeeping only
  if (rc != CANS_OK) return rc;
  const int ns = (int)B->streams.size();
  for (int i = 0; i < ns; ++i) {
    B->streams[i] = pools[dev].streams[i];
    B->joins[i] = pools[dev].joins[i];
  }
  B->fork = pools[dev].fork;
  rc = batch_solve_impl(B, f, p, workspace, cuda_stream, device_status);
  if (rc != CANS_OK)  // a failed launch leaves the internal streams unjoined: drain them first
    for (cudaStream_t s : B->streams) cudaStreamSynchronize(s);
  delete B;  // the pool keeps its streams and events
  if (device_status && rc != CANS_OK) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<int> h(count, rc);
    if (cudaMemcpyAsync(device_status, h.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return CANS_ERR_CUDA;
    cudaStreamSynchronize(st);  // h is released on return
  }
  return rc;
}

}  // extern "C"
